// tcx_gemm.cu -- extended-precision complex GEMM from exact BF16 tensor-core slices (see
// tcx_gemm.cuh for the number format and why the level-0 accumulation is exact), its operand
// producers and launcher.
//
// One CTA owns a 128 x 64 (or 128 x 32) complex output tile. Warp 0 streams 32-byte K steps (16 BF16) of the
// eight X planes (128 rows) and the twelve W planes (64 rows) through a 4-stage shared-memory
// ring, one 4-D TMA per operand (32-byte swizzle). Warp 1 issues, per K step, the ten slice
// products of levels 0..3, each as two N = 128 MMAs (real X slice against [Re W; Im W], imaginary
// X slice against [-Im W; Re W]), grouped so that MMAs sharing an X plane take it from the
// A-operand collector, into two TMEM accumulators of 128 columns (level 0; levels 1-3),
// double-buffered across groups of four K steps (64 K elements: the operands' scaling groups).
// Warps 2-17 drain each finished group into two-float registers and run the epilogue.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include "tc_ptx.cuh"
#include "tcx_gemm.cuh"

namespace coro {

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();   // tc_gemm.cu

namespace {

constexpr int BM = 128;                  // rows of X per tile (UMMA M)
constexpr int KSTEP = 16;                // BF16 K elements per stage (32 bytes, one MMA)
constexpr int GROUP = 64;                // K elements per scaling group = per TMEM drain
constexpr int STEPS_PER_GROUP = GROUP / KSTEP;
constexpr int XPLANE_BYTES = BM * 32;    // 4 KB
constexpr int X_BYTES = TCX_X_PLANES * XPLANE_BYTES;   // 32 KB
constexpr int EPI_WARPS = 16;            // four per TMEM lane quarter
constexpr int THREADS = 64 + 32 * EPI_WARPS;

// Tile shapes: BN complex outputs per tile row (UMMA N = 2 BN). 64: fewer A reads per output;
// 32: twice the tiles, for launches with too few tiles to fill the SMs.
template <int BN> struct TcxCfg {
    static constexpr int WPLANE_BYTES = BN * 32;
    static constexpr int W_BYTES = TCX_W_PLANES * WPLANE_BYTES;
    static constexpr int STAGE_BYTES = X_BYTES + W_BYTES;
    static constexpr int STAGES = BN == 64 ? 4 : 5;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/ + 1024 /*maxima*/;
    static constexpr int EPI_COLS = BN / 4;                       // complex columns per epilogue warp
    static constexpr uint32_t ACC_COLS = 2 * BN;                  // one accumulator: Re | Im
    static constexpr uint32_t TMEM_COLS = 4 * ACC_COLS;           // 2 buffers x 2 levels
    static_assert(SMEM_BYTES <= 232448, "shared memory per block");
    static_assert(EPI_COLS % 8 == 0, "drained eight columns at a time");
};

// Shared-memory matrix descriptor, K-major, 32-byte swizzle (what a TMA load with
// CU_TENSOR_MAP_SWIZZLE_32B writes): 32-byte rows, 8-row (256-byte) atoms.
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused, K-major swizzled)
    d |= (uint64_t)(256u >> 4) << 32;                  // stride byte offset: 8 rows x 32 B
    d |= (uint64_t)1 << 46;                            // descriptor version for sm_100 family
    d |= (uint64_t)6 << 61;                            // layout: 32-byte swizzle
    return d;
}

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }   // k in [-126, 127]

// Exponent e of the smallest power of two >= |x| for x > 0 (normal).
__device__ __forceinline__ int ceil_log2(float ax) {
    const uint32_t b = __float_as_uint(ax);
    const int ex = (int)((b >> 23) & 0xff) - 127;
    return (b & 0x7fffff) ? ex + 1 : ex;
}

// Largest |value| of the warp's 32 lanes (all lanes must call), as float bits: non-negative
// floats order like their bit patterns.
__device__ __forceinline__ uint32_t warp_max_bits(float amax) {
    return __reduce_max_sync(0xffffffffu, __float_as_uint(amax));
}

// Group exponent from the group's largest magnitude m (float bits): 2^e >= every |value|.
// Clamped to [-90, 120] so that every slice scale 2^(e - 32) stays a normal float.
__device__ __forceinline__ int group_exp_of(uint32_t m) {
    if (m == 0) return -90;
    int e = ceil_log2(__uint_as_float(m));
    return e < -90 ? -90 : (e > 120 ? 120 : e);
}

// Exponent of a 64-element group held by two consecutive warps of a block (warps 2w, 2w + 1);
// every thread of the block calls (two block barriers). sh: one word per warp.
__device__ __forceinline__ int group64_exp_block(float amax, uint32_t* sh) {
    const uint32_t wm = warp_max_bits(amax);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[w] = wm;
    __syncthreads();
    const uint32_t m = max(sh[w & ~1], sh[w | 1]);
    __syncthreads();
    return group_exp_of(m);
}

// Four slices of the two-float value (h, l) in the group with exponent e.
__device__ __forceinline__ void make_slices(float h, float l, int e, float (&s)[4]) {
    const float t = h * pow2f(8 - e), tl = l * pow2f(8 - e);
    const float a0 = rintf(t);
    float r = (t - a0) + tl;                           // t - a0 is exact
    s[0] = a0 * pow2f(e - 8);
    r *= 256.f;
    const float a1 = rintf(r);
    r -= a1;
    s[1] = a1 * pow2f(e - 16);
    r *= 256.f;
    const float a2 = rintf(r);
    r -= a2;
    s[2] = a2 * pow2f(e - 24);
    s[3] = rintf(r * 256.f) * pow2f(e - 32);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}

// (h, l) * (sh, sl) -> normalised two-float product
__device__ __forceinline__ void mul22(float h, float l, float sh, float sl, float& ph, float& pl) {
    const float p = h * sh;
    float e = fmaf(h, sh, -p);
    e += h * sl + l * sh;
    ph = p + e;
    pl = e - (ph - p);
}

// Store the sliced value (re, im) of one element: planes 2i (real), 2i + 1 (imaginary).
__device__ __forceinline__ void store_sliced(__nv_bfloat16* base, size_t plane, size_t off, const float (&sr)[4],
                                             const float (&si)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        base[(2 * i) * plane + off] = __float2bfloat16_rn(sr[i]);
        base[(2 * i + 1) * plane + off] = __float2bfloat16_rn(si[i]);
    }
}

// Sum of the slices of one element as a two-float pair.
__device__ __forceinline__ void load_sliced(const __nv_bfloat16* base, size_t plane, size_t off, int c, float& h,
                                            float& l) {
    const float s0 = __bfloat162float(base[c * plane + off]), s1 = __bfloat162float(base[(2 + c) * plane + off]);
    const float s2 = __bfloat162float(base[(4 + c) * plane + off]), s3 = __bfloat162float(base[(6 + c) * plane + off]);
    two_sum(s0 + s1, s2, h, l);                        // s0 + s1 is exact
    l += s3;
}

// One tile of the persistent walk: its item, origin and K groups (all warps derive the same).
struct TcxTile {
    int b, m0, n0, g0, ngroups;
    bool live;                                       // false: outside its item's M x N
};

template <int BN, int EPI>
__device__ __forceinline__ TcxTile tcx_tile(const TcArgs& a, int t, int tiles_n, int tiles_m) {
    TcxTile tl;
    tl.b = t / (tiles_n * tiles_m);
    const int r = t % (tiles_n * tiles_m);
    tl.m0 = (r / tiles_n) * BM;
    tl.n0 = (r % tiles_n) * BN;
    const TcItem& it = a.items[tl.b];
    tl.live = tl.m0 < it.M && tl.n0 < it.N;
    tl.g0 = 0;
    tl.ngroups = (it.K + GROUP - 1) / GROUP;
    if (tl.live) tile_k_range<BM, BN>(it, tl.m0, tl.n0, GROUP, EPI == TC_EPI_SPLITT || EPI == TC_EPI_BABINET, tl.g0, tl.ngroups);
    else tl.ngroups = 0;
    return tl;
}

// Persistent: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... of the tiles_n x
// tiles_m x batch grid (column tiles fastest, so neighbouring CTAs share X rows). The TMA, MMA
// and epilogue warps follow the same walk with running stage / group counters, so the MMAs of
// the next tile start as soon as the epilogue has drained the last group of the current one,
// while the epilogue is still finishing that tile's outputs.
template <int BN, int EPI>
__global__ void __launch_bounds__(THREADS, 1)
tcx_cgemm_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw, const TcArgs a,
                 int tiles_n, int tiles_m, int batch) {
    using Cfg = TcxCfg<BN>;
    constexpr int STAGES = Cfg::STAGES, STAGE_BYTES = Cfg::STAGE_BYTES, WPLANE_BYTES = Cfg::WPLANE_BYTES;
    constexpr int EPI_COLS = Cfg::EPI_COLS;
    constexpr uint32_t ACC = Cfg::ACC_COLS, TMEM_COLS = Cfg::TMEM_COLS;
    const int total = tiles_n * tiles_m * batch;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;                // accumulator buffer holds a finished group
    uint64_t* tempty = tfull + 2;                    // accumulator buffer has been drained
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);
    uint32_t* xmax = reinterpret_cast<uint32_t*>(smem + STAGES * STAGE_BYTES + 256);   // [16][EPI_COLS]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        for (int s = 0; s < 2; ++s) { tc::mbar_init(&tfull[s], 1); tc::mbar_init(&tempty[s], EPI_WARPS); }
        tc::fence_mbar_init();
        tc::prefetch_tmap(&mx);
        tc::prefetch_tmap(&mw);
    }
    if (warp == 1) {
        tc::tmem_alloc(tslot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            long long kk = 0;                                    // running stage counter
            bool ok = true;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const TcxTile tl = tcx_tile<BN, EPI>(a, t, tiles_n, tiles_m);
                const TcItem& it = a.items[tl.b];
                const int nsteps = STEPS_PER_GROUP * tl.ngroups;
                for (int k = 0; k < nsteps; ++k, ++kk) {
                    const int s = (int)(kk % STAGES);
                    const uint32_t ph = (uint32_t)(kk / STAGES) & 1;
                    if (!(ok = tc::mbar_wait(&empty[s], ph ^ 1, a.err, 11))) break;
                    unsigned char* st = smem + s * STAGE_BYTES;
                    const int kx = tl.g0 * GROUP + k * KSTEP;
                    tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    tc::tma_load_4d(st, &mx, &full[s], kx, tl.m0, 0, it.x_idx);
                    tc::tma_load_4d(st + X_BYTES, &mw, &full[s], kx, tl.n0, 0, it.w_idx);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t ID = tc::idesc<true>(BM, 2 * BN, false);
            bool ok = true;
            long long kk = 0, gg = 0;                            // running stage / group counters
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
            const TcxTile tl = tcx_tile<BN, EPI>(a, t, tiles_n, tiles_m);
            const int nsteps = STEPS_PER_GROUP * tl.ngroups;
            for (int k = 0; k < nsteps && ok; ++k, ++kk) {
                const int s = (int)(kk % STAGES);
                const uint32_t ph = (uint32_t)(kk / STAGES) & 1;
                const long long g = gg + k / STEPS_PER_GROUP;
                const int buf = (int)(g & 1), half = k % STEPS_PER_GROUP;
                if (half == 0) {
                    if (!(ok = tc::mbar_wait(&tempty[buf], (uint32_t)((g >> 1) & 1) ^ 1, a.err, 14))) break;
                    tc::tc_fence_after();
                }
                if (!(ok = tc::mbar_wait(&full[s], ph, a.err, 12))) break;
                tc::tc_fence_after();
                const uint32_t d0 = tbase + buf * 2 * ACC, d1 = d0 + ACC;
                // descriptors of plane 0 of each operand; a plane offset adds (bytes >> 4) to the
                // start-address field (addresses stay below 256 KB, so no carry leaves it)
                const uint64_t dx = sdesc_sw32(tc::smem_u32(smem + s * STAGE_BYTES));
                const uint64_t dw = sdesc_sw32(tc::smem_u32(smem + s * STAGE_BYTES + X_BYTES));
                // the ten products (X slice i, W slice j) of levels i + j <= 3, grouped by the X slice
                // component they read: consecutive MMAs with the same A keep it in the collector,
                // so each of the eight X planes leaves shared memory once per step
#pragma unroll
                for (int i = 0; i < 4; ++i) {
#pragma unroll
                    for (int c = 0; c < 2; ++c) {                   // 0: real X slice, 1: imaginary
                        const uint64_t a_desc = dx + (uint64_t)((2 * i + c) * XPLANE_BYTES >> 4);
#pragma unroll
                        for (int j = 0; j <= 3 - i; ++j) {
                            // [Re W; Im W] for the real slice, [-Im W; Re W] for the imaginary one
                            const uint64_t b_desc = dw + (uint64_t)((3 * j + 1 - c) * WPLANE_BYTES >> 4);
                            const uint32_t d = (i + j == 0) ? d0 : d1;
                            const uint32_t acc = (half == 0 && i == 0 && c == 0 && j <= 1) ? 0u : 1u;
                            if (i == 3) tc::umma_bf16_coll<tc::COLL_NONE>(d, a_desc, b_desc, ID, acc);
                            else if (j == 0) tc::umma_bf16_coll<tc::COLL_FILL>(d, a_desc, b_desc, ID, acc);
                            else if (j == 3 - i) tc::umma_bf16_coll<tc::COLL_LASTUSE>(d, a_desc, b_desc, ID, acc);
                            else tc::umma_bf16_coll<tc::COLL_USE>(d, a_desc, b_desc, ID, acc);
                        }
                    }
                }
                tc::umma_commit(&empty[s]);             // frees the stage once these MMAs retire
                if (half == STEPS_PER_GROUP - 1 || k == nsteps - 1) tc::umma_commit(&tfull[buf]);
            }
            gg += tl.ngroups;
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..17)
        const int q = warp & 3;                          // TMEM lane quarter this warp may read
        const int cg = (warp - 2) >> 2;                  // which quarter of the tile's complex columns
        const int row = q * 32 + lane;
        const uint32_t lane_base = tbase + ((uint32_t)(q * 32) << 16) + cg * EPI_COLS;
        bool ok = true;
        long long gg = 0;                                // running group counter
        // every epilogue warp walks every tile even after a wait has failed (ok = false: no
        // further waits or stores), so that the partner warps always meet at their barriers
        for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const TcxTile tl = tcx_tile<BN, EPI>(a, t, tiles_n, tiles_m);
        if (!tl.live) continue;
        const int b = tl.b, m0 = tl.m0, n0 = tl.n0;
        const TcItem it = a.items[b];
        const int m = m0 + row;
        float hr[EPI_COLS], lr[EPI_COLS], hi_[EPI_COLS], li[EPI_COLS];
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) { hr[j] = 0.f; lr[j] = 0.f; hi_[j] = 0.f; li[j] = 0.f; }
        for (int gl = 0; gl < tl.ngroups; ++gl) {
            const long long g = gg + gl;
            const int buf = (int)(g & 1);
            if (!ok || !(ok = tc::mbar_wait(&tfull[buf], (uint32_t)(g >> 1) & 1, a.err, 13))) break;
            __syncwarp();
            tc::tc_fence_after();
            // eight columns at a time, level 0 and levels 1-3 of the same outputs; BATCH such
            // pairs of loads are in flight before each wait (32 registers)
            constexpr int PARTS = EPI_COLS / 8;                     // per component
            constexpr int BATCH = 2;
#pragma unroll
            for (int p0i = 0; p0i < 2 * PARTS; p0i += BATCH) {
                uint32_t q0[BATCH][8], q1[BATCH][8];
#pragma unroll
                for (int bb = 0; bb < BATCH; ++bb) {
                    const int part = p0i + bb;
                    const uint32_t col = buf * 2 * ACC + (part / PARTS) * BN + (part % PARTS) * 8;
                    tc::tmem_ld8(lane_base + col, q0[bb]);
                    tc::tmem_ld8(lane_base + col + ACC, q1[bb]);
                }
                tc::tmem_ld_wait();
                if (p0i + BATCH >= 2 * PARTS) {                     // the buffer is drained
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tempty[buf]);
                }
#pragma unroll
                for (int bb = 0; bb < BATCH; ++bb) {
                    const int part = p0i + bb;
                    const int c = (part % PARTS) * 8, imag = part / PARTS;   // real parts first
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float& h = imag ? hi_[c + j] : hr[c + j];
                        float& l = imag ? li[c + j] : lr[c + j];
                        float s, e;
                        two_sum(h, __uint_as_float(q0[bb][j]), s, e);
                        h = s;
                        l += e + __uint_as_float(q1[bb][j]);
                    }
                }
            }
        }
        gg += tl.ngroups;
        // scale: Y * scale64 in two-float
        const float sh = (float)it.scale64, sl = (float)(it.scale64 - (double)sh);
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) {
            mul22(hr[j], lr[j], sh, sl, hr[j], lr[j]);
            mul22(hi_[j], li[j], sh, sl, hi_[j], li[j]);
        }
        const int kx = m - it.M / 2;
        const size_t plane = (size_t)a.dst_rows * a.dst_ld;
        if constexpr (EPI == TC_EPI_SPLITT || EPI == TC_EPI_BABINET) {
            __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(a.dst);
            // pass 1: the output values (Babinet subtraction, mask) in place, and this warp's
            // largest magnitude per column; the 64 rows m0 + 64 h ... + 63 of a scaling group
            // (the next GEMM's K elements) belong to warps q = 2h and 2h + 1 of the same column group
            const int ew = warp - 2;
#pragma unroll
            for (int j = 0; j < EPI_COLS; ++j) {
                const int n = n0 + cg * EPI_COLS + j;
                const int ky = n - it.N / 2;
                const int r2 = kx * kx + ky * ky;
                const bool valid = ok && m < it.M && n < it.N;
                const bool keep = valid && r2 >= it.mask_lo && r2 <= it.mask_hi;
                float vr = 0.f, vrl = 0.f, vi = 0.f, vil = 0.f;
                if (keep) {
                    vr = hr[j]; vrl = lr[j]; vi = hi_[j]; vil = li[j];
                    if constexpr (EPI == TC_EPI_BABINET) {
                        // E_A - Y: E_A from the complex64 pupil (exact FP32) or from the slices in dst
                        const size_t off = b * a.dst_bstride + (size_t)n * a.dst_ld + m;
                        float ar, arl, ai, ail;
                        if (a.src64) {
                            const float2 e = __ldg(a.src64 + b * a.src64_bstride + (size_t)n * a.src64_ld + m);
                            ar = e.x; arl = 0.f; ai = e.y; ail = 0.f;
                        } else {
                            load_sliced(dst, plane, off, 0, ar, arl);
                            load_sliced(dst, plane, off, 1, ai, ail);
                        }
                        float s, e;
                        two_sum(ar, -vr, s, e);
                        vr = s; vrl = e + (arl - vrl);
                        two_sum(ai, -vi, s, e);
                        vi = s; vil = e + (ail - vil);
                    }
                }
                hr[j] = vr; lr[j] = vrl; hi_[j] = vi; li[j] = vil;
                const uint32_t wm = warp_max_bits(fmaxf(fabsf(vr), fabsf(vi)));
                if (lane == 0) xmax[ew * EPI_COLS + j] = wm;
            }
            // the two warps of each scaling group meet at their own named barrier (ids 1-8)
            const int pair_bar = 1 + cg * 2 + (q >> 1);
            asm volatile("bar.sync %0, 64;" ::"r"(pair_bar) : "memory");
            // epilogue warp w = 4 cg + i has TMEM lane quarter q = (i + 2) & 3 (warp = w + 2)
            const int partner = 4 * cg + (((q ^ 1) + 2) & 3);
#pragma unroll
            for (int j = 0; j < EPI_COLS; ++j) {
                const int n = n0 + cg * EPI_COLS + j;
                const bool valid = ok && m < it.M && n < it.N;
                const uint32_t gm = max(xmax[ew * EPI_COLS + j], xmax[partner * EPI_COLS + j]);
                const int ge = group_exp_of(gm);
                if (valid) {
                    float sr[4], si[4];
                    make_slices(hr[j], lr[j], ge, sr);
                    make_slices(hi_[j], li[j], ge, si);
                    const size_t off = b * a.dst_bstride + (size_t)n * a.dst_ld + m;
                    store_sliced(dst, plane, off, sr, si);
                    if (a.c64) a.c64[b * a.c64_bstride + (size_t)n * a.c64_ld + m] = make_float2(hr[j] + lr[j], hi_[j] + li[j]);
                }
            }
            // both warps have read the pair's maxima before either writes the next tile's
            asm volatile("bar.sync %0, 64;" ::"r"(pair_bar) : "memory");
        } else if constexpr (EPI == TC_EPI_C64T) {
            if (ok && m < it.M) {
#pragma unroll
                for (int j = 0; j < EPI_COLS; ++j) {
                    const int n = n0 + cg * EPI_COLS + j;
                    if (n < it.N) {
                        float2* d = reinterpret_cast<float2*>(a.dst) + b * a.dst_bstride + (size_t)n * a.dst_ld + m;
                        *d = make_float2(hr[j] + lr[j], hi_[j] + li[j]);
                    }
                }
            }
        } else {
            // intensity |Y|^2 / peak in two-float; dark-hole sum and running peak in FP64
            const float ph = (float)it.inv_peak64, pl = (float)(it.inv_peak64 - (double)ph);
            float dsh = 0.f, dsl = 0.f;
            double pk = 0.0;
            if (ok && m < it.M) {
#pragma unroll
                for (int j = 0; j < EPI_COLS; ++j) {
                    const int n = n0 + cg * EPI_COLS + j;
                    if (n < it.N) {
                        // |v|^2 = hr^2 + hi^2 + 2 (hr lr + hi li) (+ lr^2 + li^2, negligible)
                        const float q0 = hr[j] * hr[j], q1 = hi_[j] * hi_[j];
                        float e0 = fmaf(hr[j], hr[j], -q0), e1 = fmaf(hi_[j], hi_[j], -q1);
                        float ih, il;
                        two_sum(q0, q1, ih, il);
                        il += e0 + e1 + 2.f * (hr[j] * lr[j] + hi_[j] * li[j]);
                        float nh, nl;
                        mul22(ih, il, ph, pl, nh, nl);
                        const float inten = nh + nl;
                        if (a.dst) reinterpret_cast<float*>(a.dst)[b * a.dst_bstride + (size_t)n * a.dst_ld + m] = inten;
                        const int ky = n - it.N / 2;
                        const int r2 = kx * kx + ky * ky;
                        const bool keep = r2 >= it.mask_lo && r2 <= it.mask_hi;
                        if (a.c64) {
                            // field, or the gradient seed dS/dconj(E) = mask . E / peak
                            const double ip = it.inv_peak64;
                            const float2 v = !a.c64_seed ? make_float2(hr[j] + lr[j], hi_[j] + li[j])
                                             : keep ? make_float2((float)((double)hr[j] * ip + (double)lr[j] * ip),
                                                                  (float)((double)hi_[j] * ip + (double)li[j] * ip))
                                                    : make_float2(0.f, 0.f);
                            a.c64[b * a.c64_bstride + (size_t)n * a.c64_ld + m] = v;
                        }
                        if (keep) {
                            float s, e;
                            two_sum(dsh, nh, s, e);
                            dsh = s;
                            dsl += e + nl;
                        }
                        const double dv = (double)nh + (double)nl;
                        pk = dv > pk ? dv : pk;
                    }
                }
            }
            double dh = (double)dsh + (double)dsl;
            for (int o = 16; o > 0; o >>= 1) {
                dh += __shfl_down_sync(0xffffffffu, dh, o);
                const double other = __shfl_down_sync(0xffffffffu, pk, o);
                pk = other > pk ? other : pk;
            }
            if (lane == 0 && dh != 0.0 && a.dh_acc) atomicAdd(a.dh_acc + b, dh);
            // non-negative doubles order like their bit patterns as unsigned integers
            if (lane == 0 && a.peak64)
                atomicMax(reinterpret_cast<unsigned long long*>(a.peak64) + b, (unsigned long long)__double_as_longlong(pk));
        }
        }                                                // tiles
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tbase, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- operand producers

// complex64 rows -> sliced X planes; one thread per element, two warps per 64-element group
// (blocks of 128 threads).
__global__ void tcx_split_kernel(const float2* __restrict__ src, long long sb, int sld, __nv_bfloat16* dst, int rows,
                                 int cols, int ld, const int* __restrict__ keep_r2) {
    __shared__ uint32_t sh[4];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, b = blockIdx.z;
    float2 v = make_float2(0.f, 0.f);
    if (k < cols) v = src[b * sb + (size_t)r * sld + k];
    if (keep_r2) {
        const int kx = k - cols / 2, ky = r - rows / 2;
        if (kx * kx + ky * ky > keep_r2[b]) v = make_float2(0.f, 0.f);
    }
    const int ge = group64_exp_block(fmaxf(fabsf(v.x), fabsf(v.y)), sh);
    if (k >= ld) return;
    float sr[4], si[4];
    make_slices(v.x, 0.f, ge, sr);
    make_slices(v.y, 0.f, ge, si);
    const size_t plane = (size_t)rows * ld;
    store_sliced(dst, plane, (size_t)b * TCX_X_PLANES * plane + (size_t)r * ld + k, sr, si);
}

// W[r][k] = exp(sign 2 pi i (r - rows/2)(k - cols/2) c): FP64 phase reduced to its fractional
// cycle, then sliced from the FP64 value (no FP32 rounding of the basis).
__global__ void tcx_basis_kernel(double c, int sign, __nv_bfloat16* dst, int rows, int cols, int ld, int plane_rows,
                                 int item) {
    __shared__ uint32_t sh[4];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    double re = 0.0, im = 0.0;
    if (k < cols) {
        const long long rr = (long long)r - rows / 2, kk = (long long)k - cols / 2;
        double cyc = (double)(rr * kk) * c;
        cyc -= rint(cyc);
        double s, co;
        sincospi(2.0 * cyc, &s, &co);
        re = co;
        im = sign < 0 ? -s : s;
    }
    const int ge = group64_exp_block(fmaxf((float)fabs(re), (float)fabs(im)), sh);
    if (k >= ld) return;
    const float rh = (float)re, rl = (float)(re - (double)rh), ih = (float)im, il = (float)(im - (double)ih);
    float sr[4], si[4];
    make_slices(rh, rl, ge, sr);
    make_slices(ih, il, ge, si);
    const size_t plane = (size_t)plane_rows * ld;
    const size_t off = (size_t)item * TCX_W_PLANES * plane + (size_t)r * ld + k;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        dst[(3 * i) * plane + off] = __float2bfloat16_rn(-si[i]);
        dst[(3 * i + 1) * plane + off] = __float2bfloat16_rn(sr[i]);
        dst[(3 * i + 2) * plane + off] = __float2bfloat16_rn(si[i]);
    }
}

__global__ void tcx_merge_kernel(const __nv_bfloat16* src, int rows, int cols, int ld, float2* dst, long long db,
                                 int dld) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, b = blockIdx.z;
    if (k >= cols) return;
    const size_t plane = (size_t)rows * ld;
    const size_t off = (size_t)b * TCX_X_PLANES * plane + (size_t)r * ld + k;
    float h, l, h2, l2;
    load_sliced(src, plane, off, 0, h, l);
    load_sliced(src, plane, off, 1, h2, l2);
    dst[b * db + (size_t)r * dld + k] = make_float2(h + l, h2 + l2);
}

template <int BN, int EPI>
cudaError_t launch_t(const CUtensorMap& mx, const CUtensorMap& mw, int max_m, int max_n, int batch, const TcArgs& args,
                     cudaStream_t stream) {
    constexpr int SMEM = TcxCfg<BN>::SMEM_BYTES;
    static int attr_done = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_done != dev) {
        cudaError_t e = cudaFuncSetAttribute(tcx_cgemm_kernel<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr_done = dev;
    }
    static int sms[64] = {};
    if (dev >= 0 && dev < 64 && sms[dev] == 0) {
        cudaError_t e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const int tiles_n = (max_n + BN - 1) / BN, tiles_m = (max_m + BM - 1) / BM;
    const long long total = (long long)tiles_n * tiles_m * batch;
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int per_sm = (dev >= 0 && dev < 64) ? sms[dev] : 148;
    const int grid = total < per_sm ? (int)total : per_sm;
    if (grid == 0) return cudaSuccess;
    tcx_cgemm_kernel<BN, EPI><<<grid, THREADS, SMEM, stream>>>(mx, mw, args, tiles_n, tiles_m, batch);
    return cudaGetLastError();
}

template <int BN>
cudaError_t launch_bn(int epi, const CUtensorMap& mx, const CUtensorMap& mw, int max_m, int max_n, int batch,
                      const TcArgs& args, cudaStream_t stream) {
    switch (epi) {
        case TC_EPI_C64T: return launch_t<BN, TC_EPI_C64T>(mx, mw, max_m, max_n, batch, args, stream);
        case TC_EPI_SPLITT: return launch_t<BN, TC_EPI_SPLITT>(mx, mw, max_m, max_n, batch, args, stream);
        case TC_EPI_BABINET: return launch_t<BN, TC_EPI_BABINET>(mx, mw, max_m, max_n, batch, args, stream);
        case TC_EPI_INTENSITY: return launch_t<BN, TC_EPI_INTENSITY>(mx, mw, max_m, max_n, batch, args, stream);
    }
    return cudaErrorInvalidValue;
}

cudaError_t make_map(const TcOperand& op, int planes, int box_rows, CUtensorMap* map) {
    auto fn = tensor_map_encoder();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)op.base & 15) || op.ld % 16 || op.ld < op.cols) return cudaErrorInvalidValue;
    const cuuint64_t es = 2;
    cuuint64_t dims[4] = {(cuuint64_t)op.ld, (cuuint64_t)op.rows, (cuuint64_t)planes, (cuuint64_t)op.batch};
    cuuint64_t strides[3] = {(cuuint64_t)op.ld * es, (cuuint64_t)op.rows * op.ld * es,
                             (cuuint64_t)planes * op.rows * op.ld * es};
    cuuint32_t box[4] = {(cuuint32_t)KSTEP, (cuuint32_t)box_rows, (cuuint32_t)planes, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, op.base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t tcx_make_x_map(const TcOperand& op, CUtensorMap* map) { return make_map(op, TCX_X_PLANES, BM, map); }
cudaError_t tcx_make_w_map(const TcOperand& op, CUtensorMap* map, int tile_n) {
    if (tile_n != 64 && tile_n != 32) return cudaErrorInvalidValue;
    return make_map(op, TCX_W_PLANES, tile_n, map);
}

cudaError_t tcx_launch(int epi, const CUtensorMap& mx, const CUtensorMap& mw, int max_m, int max_n, int batch,
                       const TcArgs& args, cudaStream_t stream, int tile_n) {
    if (tile_n == 64) return launch_bn<64>(epi, mx, mw, max_m, max_n, batch, args, stream);
    if (tile_n == 32) return launch_bn<32>(epi, mx, mw, max_m, max_n, batch, args, stream);
    return cudaErrorInvalidValue;
}

template <int BN>
void count_bn(int epi, const TcItem* items, int batch, int max_m, int max_n, double* useful, double* issued) {
    const bool masked = epi == TC_EPI_SPLITT || epi == TC_EPI_BABINET;
    // 10 slice products, each a complex multiply-add of 4 real products = 80 flops per output per K element
    for (int b = 0; b < batch; ++b) {
        const TcItem& it = items[b];
        for (int m0 = 0; m0 < max_m && m0 < it.M; m0 += BM)
            for (int n0 = 0; n0 < max_n && n0 < it.N; n0 += BN) {
                int g0 = 0, ng = (it.K + GROUP - 1) / GROUP;
                tile_k_range<BM, BN>(it, m0, n0, GROUP, masked, g0, ng);
                if (ng <= 0) continue;
                const int rows = (m0 + BM < it.M ? BM : it.M - m0), cols = (n0 + BN < it.N ? BN : it.N - n0);
                int klo = 0, khi = it.K - 1;
                if (it.kr2 >= 0) {
                    const long long dm = dist_to_range(it.M / 2, m0, m0 + rows - 1);
                    const int w = isqrt_floor((long long)it.kr2 - (long long)it.kdy * dm * dm);
                    klo = it.K / 2 - w < 0 ? 0 : it.K / 2 - w;
                    khi = it.K / 2 + w > it.K - 1 ? it.K - 1 : it.K / 2 + w;
                }
                *useful += 80.0 * rows * cols * (double)(khi - klo + 1);
                *issued += 80.0 * BM * BN * (double)ng * GROUP;
            }
    }
}

void tcx_count_flops(int epi, const TcItem* items, int batch, int max_m, int max_n, double* useful, double* issued,
                     int tile_n) {
    if (tile_n == 32) count_bn<32>(epi, items, batch, max_m, max_n, useful, issued);
    else count_bn<64>(epi, items, batch, max_m, max_n, useful, issued);
}

cudaError_t tcx_split(const float2* src, long long src_bstride, int src_ld, const TcOperand& dst, cudaStream_t stream,
                      const int* keep_r2) {
    dim3 grid((dst.ld + 127) / 128, dst.rows, dst.batch);
    tcx_split_kernel<<<grid, 128, 0, stream>>>(src, src_bstride, src_ld, (__nv_bfloat16*)dst.base, dst.rows, dst.cols,
                                              dst.ld, keep_r2);
    return cudaGetLastError();
}

cudaError_t tcx_basis_one(double c, int sign, const TcOperand& dst, int item, int rows_valid, int cols_valid,
                          cudaStream_t stream) {
    if (rows_valid > dst.rows || cols_valid > dst.ld || item < 0 || item >= dst.batch) return cudaErrorInvalidValue;
    dim3 grid((dst.ld + 127) / 128, rows_valid, 1);
    tcx_basis_kernel<<<grid, 128, 0, stream>>>(c, sign, (__nv_bfloat16*)dst.base, rows_valid, cols_valid, dst.ld,
                                               dst.rows, item);
    return cudaGetLastError();
}

cudaError_t tcx_merge(const TcOperand& src, float2* dst, long long dst_bstride, int dst_ld, cudaStream_t stream) {
    dim3 grid((src.cols + 127) / 128, src.rows, src.batch);
    tcx_merge_kernel<<<grid, 128, 0, stream>>>((const __nv_bfloat16*)src.base, src.rows, src.cols, src.ld, dst,
                                               dst_bstride, dst_ld);
    return cudaGetLastError();
}

}  // namespace coro
