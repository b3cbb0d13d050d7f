// passes_f32.cu -- complex64 row/column pass launchers (N = 32 ... 8192).
#include "passes_launch.cuh"
#include "mixed.cuh"
#include "mixed_pair.cuh"

namespace coro {

template <>
cudaError_t launch_row_pass<float2>(int n, const RowArgs<float2>& a, const PassLaunch& l0) {
    using namespace detail;
    PassLaunch l = l0;
    if (l.variant < 0) l.variant = row_variant_default(n);
    switch (n) {
        case 32: return row_launch<float2, 32>(a, l);
        case 64: return row_launch<float2, 64>(a, l);
        case 128: return row_launch<float2, 128>(a, l);
        case 256: return row_launch<float2, 256>(a, l);
        case 512: return row_launch<float2, 512>(a, l);
        case 1024:
            if (l.variant == 5) return row_launch_mixed<float2>(n, a, l, 8);
            if (l.variant == 4) return row_launch_pair<1024, 8, 4, true>(a, l);
            if (l.variant == 3) return row_launch_pair<1024, 8, 4>(a, l);
            if (l.variant == 2) return row_launch_units<float2, 1024, 8, 4>(a, l);
            return l.variant == 1 ? row_launch<float2, 1024>(a, l) : row_launch_persistent<float2, 1024>(a, l);
        case 2048:
            if (l.variant == 5) return row_launch_mixed<float2>(n, a, l, 8);
            if (l.variant == 4) return row_launch_pair<2048, 4, 2, true>(a, l);
            if (l.variant == 3) return row_launch_pair<2048, 4, 2>(a, l);
            if (l.variant == 2) return row_launch_units<float2, 2048, 8, 4>(a, l);
            return l.variant == 1 ? row_launch<float2, 2048>(a, l) : row_launch_persistent<float2, 2048>(a, l);
        case 4096:
            if (l.variant == 5) return row_launch_mixed<float2>(n, a, l, 8);
            if (l.variant == 4) return row_launch_pair<4096, 2, 1, true>(a, l);
            if (l.variant == 3) return row_launch_pair<4096, 2, 1>(a, l);
            if (l.variant == 2) return row_launch_units<float2, 4096, 4, 2>(a, l);
            return l.variant == 1 ? row_launch<float2, 4096>(a, l) : row_launch_persistent<float2, 4096>(a, l);
        case 8192: return l.variant == 1 ? row_launch<float2, 8192>(a, l) : row_launch_persistent<float2, 8192>(a, l);
        default:
            if (l.variant == 6 && mixed_pair_length(n)) return row_launch_mixed_pair(n, a, l);
            return row_launch_mixed<float2>(n, a, l);
    }
}

// lines = columns per block; 0 = default. Wider blocks give longer contiguous segments per
// row (L * 8 bytes), narrower ones more resident blocks per SM. -1 = persistent TMA kernel,
// -2 = unit-pipelined kernel (two columns per unit), -3 = unit-pipelined kernel on packed
// FP32x2 column pairs, -4 = wide kernel (four columns, packed pairs, staged by TMA), -6 = the
// packed-pair kernel writing its result transposed to a separate plane (row variant 4 reads it),
// -7 = quad kernel (four columns as two packed pairs, whole-sector strips, swizzled exchanges),
// -8 = the shared-memory Stockham engine of mixed.cuh with radix 8 (N = 8^k x 2 or 4): the
// alternative factorisation of the power-of-two lengths; mixed-radix lengths: columns per block
// of the shared-memory engine, or -5 = the packed-pair engine of mixed_pair.cuh (its lengths).
template <>
cudaError_t launch_col_pass<float2>(int n, int lines, const ColArgs<float2>& a, const PassLaunch& l) {
    using namespace detail;
    if (lines == 0) lines = col_lines_default(n, false);
    switch (n) {
        case 32: return col_launch<float2, 32, 16>(a, l);
        case 64: return col_launch<float2, 64, 16>(a, l);
        case 128: return col_launch<float2, 128, 16>(a, l);
        case 256: return col_launch<float2, 256, 16>(a, l);
        case 512: return col_launch<float2, 512, 16>(a, l);
        case 1024:
            if (lines == -8) return col_launch_mixed<float2>(n, 0, a, l, 8);
            if (lines == -7) return col_launch_quad<1024>(a, l);
            if (lines == -4) return col_launch_wide<1024>(a, l);
            if (lines == -6) return col_launch_pair<1024, 8, 4, true>(a, l);
            if (lines == -3) return col_launch_pair<1024, 8, 4>(a, l);
            if (lines == -2) return col_launch_units<float2, 1024, 2, 8, 4>(a, l);
            if (lines == -1) return col_launch_persistent<float2, 1024, 4>(a, l);
            return lines == 8 ? col_launch<float2, 1024, 8>(a, l) : col_launch<float2, 1024, 16>(a, l);
        case 2048:
            if (lines == -8) return col_launch_mixed<float2>(n, 0, a, l, 8);
            if (lines == -7) return col_launch_quad<2048>(a, l);
            if (lines == -4) return col_launch_wide<2048>(a, l);
            if (lines == -6) return col_launch_pair<2048, 4, 2, true>(a, l);
            if (lines == -3) return col_launch_pair<2048, 4, 2>(a, l);
            if (lines == -2) return col_launch_units<float2, 2048, 2, 4, 2>(a, l);
            if (lines == -1) return col_launch_persistent<float2, 2048, 2>(a, l);
            return lines == 4 ? col_launch<float2, 2048, 4>(a, l) : col_launch<float2, 2048, 8>(a, l);
        case 4096:
            if (lines == -8) return col_launch_mixed<float2>(n, 0, a, l, 8);
            if (lines == -7) return col_launch_quad<4096>(a, l);
            if (lines == -4) return col_launch_wide<4096>(a, l);
            if (lines == -6) return col_launch_pair<4096, 2, 1, true>(a, l);
            if (lines == -3) return col_launch_pair<4096, 2, 1>(a, l);
            if (lines == -2) return col_launch_units<float2, 4096, 2, 2, 1>(a, l);
            if (lines == -1) return col_launch_persistent<float2, 4096, 2>(a, l);
            return lines == 2 ? col_launch<float2, 4096, 2>(a, l) : col_launch<float2, 4096, 4>(a, l);
        case 8192: return lines == 1 ? col_launch<float2, 8192, 1>(a, l) : col_launch<float2, 8192, 2>(a, l);
        default:
            if (lines == -5 && mixed_pair_length(n)) return col_launch_mixed_pair(n, a, l);
            return col_launch_mixed<float2>(n, lines, a, l);
    }
}

int col_lines_default(int n, bool dbl) {
    if (n & (n - 1)) return !dbl && mixed_pair_length(n) ? -5 : 0;   // mixed radix: packed pairs, or
                                                                      // the launcher picks the width
    if (dbl) {
        switch (n) {
            case 4096: return 1;
            case 2048: return 2;
            case 1024: return 4;
            case 512: case 256: return 8;
            default: return 16;
        }
    }
    switch (n) {
        case 8192: return 2;
        case 4096: case 2048: case 1024: return -3;   // packed column pairs
        default: return 16;
    }
}

int row_variant_default(int n) { return mixed_pair_length(n) ? 6 : (n >= 1024 && n <= 4096) ? 3 : 0; }

int col_candidates(int n, int* out) {
    switch (n) {
        case 8192: out[0] = 2; out[1] = 1; return 2;
        case 4096: out[5] = -4; out[6] = -7; out[7] = -8; out[0] = 4; out[1] = 2; out[2] = -1; out[3] = -2; out[4] = -3; return 8;
        case 2048: out[5] = -4; out[6] = -7; out[7] = -8; out[0] = 8; out[1] = 4; out[2] = -1; out[3] = -2; out[4] = -3; return 8;
        case 1024: out[5] = -4; out[6] = -7; out[7] = -8; out[0] = 16; out[1] = 8; out[2] = -1; out[3] = -2; out[4] = -3; return 8;
        default: {                                          // mixed radix: widest fit, and half of it
            out[0] = 0;
            if (!mixed_supported<float2>(n)) return 1;
            out[0] = mixed_col_lines<float2>(n);
            int k = 1;
            if (out[0] >= 2) out[k++] = out[0] / 2;
            if (mixed_pair_length(n)) out[k++] = -5;    // packed pairs, compile-time radix plan
            return k;
        }
    }
}

// row variants: 0 persistent, 1 one block per line group, 2 unit-pipelined, 3 packed row
// pairs, 5 the shared-memory engine with radix 8 (4, packed row pairs read from a transposed
// plane, is only paired with column lines -6 and is not a tuning candidate); mixed-radix
// lengths: 0 the shared-memory engine, 6 the packed-pair engine (its lengths)
int row_variant_count(int n) { return (n >= 1024 && n <= 4096) ? 4 : n == 8192 ? 2 : 1; }

int row_candidates(int n, int* out) {
    const int k = row_variant_count(n);
    for (int v = 0; v < k; ++v) out[v] = v;
    if (n >= 1024 && n <= 4096 && !(n & (n - 1))) {
        out[k] = 5;
        return k + 1;
    }
    if (mixed_pair_length(n)) {
        out[k] = 6;
        return k + 1;
    }
    return k;
}

// Radix sequence of the line transforms of a pass (complex64 kernels; the FP64 passes share
// the radix-16 engine): the register-resident engines take radix 16 while it divides and the
// remainder in the last stage; the shared-memory engine (mixed-radix lengths, or row variant 5 /
// column lines -8 at powers of two) follows mixed_plan.
int pass_radices(int n, bool row, int variant, int lines, int* out, int max_out) {
    MixedPlan mp;
    const bool radix8 = !(n & (n - 1)) && (row ? variant == 5 : lines == -8);   // a power-of-two choice only
    if ((n & (n - 1)) || radix8) {
        if (!mixed_plan(n, &mp, radix8 ? 8 : 16)) return 0;
    } else {
        mp.stages = 0;
        int m = n;
        while (m > 1 && mp.stages < kMixedMaxStages) {
            const int r = m >= 16 ? 16 : m;
            mp.radix[mp.stages++] = r;
            m /= r;
        }
    }
    for (int i = 0; i < mp.stages && i < max_out; ++i) out[i] = mp.radix[i];
    return mp.stages;
}

bool mixed_length_ok(int n, bool dbl) { return dbl ? mixed_supported<double2>(n) : mixed_supported<float2>(n); }

void describe_pass(int n, bool dbl, bool row, int variant, int lines, int* persistent, int* out_lines) {
    int p = 0, w = 0;
    if ((n & (n - 1)) && !dbl) {                            // the defaults of launch_*_pass<float2>
        if (row && variant < 0) variant = row_variant_default(n);
        if (!row && lines == 0) lines = col_lines_default(n, false);
    }
    if ((n & (n - 1)) && !dbl && mixed_pair_length(n) && (row ? variant == 6 : lines == -5)) {
        if (persistent) *persistent = 9;                    // mixed-radix packed pairs
        if (out_lines) *out_lines = row ? 1 : 2;
        return;
    }
    if (n & (n - 1)) {                                      // mixed-radix passes
        if (persistent) *persistent = 6;
        if (out_lines) *out_lines = row ? 1 : dbl ? mixed_col_lines<double2>(n) : lines > 0 ? lines : mixed_col_lines<float2>(n);
        return;
    }
    if (variant < 0) variant = row_variant_default(n);
    if ((row && variant == 5 && !dbl) || (!row && lines == -8 && !dbl)) {   // radix-8 shared-memory engine
        if (persistent) *persistent = 6;
        if (out_lines) *out_lines = row ? 1 : mixed_col_lines<float2>(n);
        return;
    }
    if (row) {                                              // mirrors launch_row_pass
        p = (!dbl && n >= 1024) ? (variant == 1 ? 0 : (variant == 2 || variant == 3) && n <= 4096 ? variant : 1) : 0;
        if (!dbl && variant == 4 && n >= 1024 && n <= 4096) p = 7;
    } else if (dbl) {
        w = col_lines_default(n, true);                     // the double launcher ignores `lines`
    } else {                                                // mirrors launch_col_pass<float2>
        if (lines == 0) lines = col_lines_default(n, false);
        switch (n) {
            case 1024: p = lines < 0 ? -lines : 0; w = p == 1 || p == 4 || p == 7 ? 4 : p ? 2 : (lines == 8 ? 8 : 16); break;
            case 2048: p = lines < 0 ? -lines : 0; w = p == 4 || p == 7 ? 4 : p ? 2 : (lines == 4 ? 4 : 8); break;
            case 4096: p = lines < 0 ? -lines : 0; w = p == 4 || p == 7 ? 4 : p ? 2 : (lines == 2 ? 2 : 4); break;
            case 8192: w = lines == 1 ? 1 : 2; break;
            default: w = 16; break;
        }
        if (p == 6) p = 7;                                  // lines -6: transposed packed pairs
        else if (p == 7) p = 8;                             // lines -7: quad strips
    }
    if (persistent) *persistent = p;
    if (out_lines) *out_lines = w;
}

}  // namespace coro
