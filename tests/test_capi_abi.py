"""CPU-side checks of the C-ABI library: it loads, exports every entry point the header
declares, and rejects bad arguments on the host without touching a GPU."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "coro.h")).read()
    return sorted(set(re.findall(r"^\s*(?:coro_status|const char\*|int)\s+(coro_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def dll():
    from paper_1806_06467_gb300 import build, coro
    build.build()
    return coro.Library(coro.LIB_PATH)


def test_every_declared_symbol_is_exported(dll):
    syms = header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(dll.dll, s), s


def test_binding_covers_header(dll):
    from paper_1806_06467_gb300 import coro
    assert set(header_symbols()) == set(coro.declared_symbols())


def test_version_and_error_string(dll):
    assert dll.coro_version() == 1
    assert isinstance(dll.coro_last_error(), bytes)


def test_host_side_argument_checks(dll):
    from paper_1806_06467_gb300 import coro
    # NULL out pointer is rejected before any CUDA call
    assert dll.coro_ctx_create(0, None, None) == coro.EINVAL
    assert b"NULL" in dll.coro_last_error()
    # a NULL context is rejected by every compute entry point
    w = coro.Wavefront(1, coro.C64, 1, 64, None, None)
    assert dll.coro_wavefront_init(None, ct.byref(w), 1.0) == coro.EINVAL
    assert dll.coro_propagate_fresnel(None, ct.byref(w), 1.0, 0) == coro.EINVAL
    assert dll.coro_plan_destroy(None) == coro.OK


def test_plan_entry_points_reject_null_plans(dll):
    """Every plan query and setter checks its handle on the host and fails with CORO_EINVAL
    and a message, without touching a device."""
    from paper_1806_06467_gb300 import coro
    i, d = ct.c_int(), ct.c_double()
    calls = [
        lambda: dll.coro_fresnel_plan_set_layout(None, 1),
        lambda: dll.coro_fresnel_plan_layout(None, ct.byref(i)),
        lambda: dll.coro_fresnel_plan_copy_tuning(None, None),
        lambda: dll.coro_fresnel_plan_pass_flops(None, 0, ct.byref(d)),
        lambda: dll.coro_fresnel_plan_pass_info(None, 0, ct.byref(i), ct.byref(d)),
        lambda: dll.coro_fresnel_plan_pass_kernel(None, 0, ct.byref(i), ct.byref(i)),
        lambda: dll.coro_fresnel_plan_set_pass_kernel(None, 0, 0),
        lambda: dll.coro_lyot_plan_execute(None, None, None, None, None, None),
        lambda: dll.coro_lyot_plan_peak(None, None, None),
        lambda: dll.coro_lyot_plan_gradient(None, None, None, None, None, 0, 0),
        lambda: dll.coro_wfc_plan_resident(None, ct.byref(i), ct.byref(i)),
        lambda: dll.coro_fresnel_plan_pass_radix(None, 0, None, 0, ct.byref(i)),
        lambda: dll.coro_lyot_plan_gemm_tile(None, ct.byref(i), ct.byref(i)),
        lambda: dll.coro_lyot_plan_set_gemm_tile(None, 64),
    ]
    for k, call in enumerate(calls):
        assert call() == coro.EINVAL, k
        assert dll.coro_last_error(), k


def test_no_device_reports_ecuda(dll):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1806_06467_gb300 import coro
    h = ct.c_void_p()
    assert dll.coro_ctx_create(0, None, ct.byref(h)) == coro.ECUDA


def header_members(struct: str) -> list[str]:
    """Member names, in order, of `typedef struct { ... } struct;` in include/coro.h."""
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "coro.h")).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + r"\s*;", text)
    assert m, struct
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = decl.split(",")
        names.append(re.findall(r"\w+", parts[0])[-1])
        names += [re.findall(r"\w+", q)[-1] for q in parts[1:]]
    return names


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and field offsets."""
    import subprocess

    from paper_1806_06467_gb300 import coro
    mirrors = {"coro_wavefront": coro.Wavefront, "coro_element": coro.Element, "coro_fresnel_desc": coro.FresnelDesc,
               "coro_fresnel_system_desc": coro.FresnelSystemDesc, "coro_lyot_item": coro.LyotItem,
               "coro_lyot_desc": coro.LyotDesc, "coro_wfc_desc": coro.WfcDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "coro.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            c, f, v = line.split()
            got[(c, f)] = int(v)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ct.sizeof(py), cname
        # a missing trailing member can hide in the padding: the names must match in order
        assert header_members(cname) == [f for f, _ in py._fields_], cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
