// mixed_pair.cuh -- mixed-radix line transforms on packed line pairs, the radix plan fixed at
// compile time (N = 2800 of Sec. 3.1, N = 4100 = 4 x 1025 of App. B, and 1400).
//
// The Stockham stages of mixed.cuh (stage s of radix R, NS = the product of the earlier radices:
// butterfly j reads x[j + r N/R], multiplies by W_{NS R}^{r (j mod NS)}, takes an R-point DFT and
// writes position (j / NS) NS R + j mod NS + r NS), on two lines at once in packed FP32x2
// arithmetic (fft_pair.cuh: lane 0 holds line A, lane 1 line B, every add / mul / fma issues once
// for both). With N a template parameter every stage's radix, span and butterfly count are
// compile-time constants, so there is no run-time division and the butterfly loops unroll; and
// each thread keeps its K = ceil((N/R) / T) butterflies of a stage in registers between a read
// phase and a write phase, so one buffer of N pair slots serves every stage in place (two block
// barriers per stage) and two or three blocks share an SM. Radices: 16, 8, 4, 2 (the engine's
// butterflies), odd primes up to 13 (the pair-sum DFT of mixed.cuh) and one larger prime up to
// 61 whose R - 1 splits into them, as a Rader stage last (pair_stage_rader).
#pragma once
#include "fft_pair.cuh"
#include "mixed.cuh"
#include "rader.cuh"

namespace coro {
namespace mpair {

using pk::CP;
using pk::u64;

constexpr int kMaxOddRadix = 13;

// Threads per line pair, a divisor of n where there is one, so that every thread holds exactly
// n / T samples of the pair between the transforms. With a radix-8 or radix-16 stage (n a
// multiple of 8: 16 samples per butterfly held in registers) the smallest divisor from 256 to
// 320, else the largest from 192 to 255 (280 at 1400 and 2800); without one, where the largest
// register-held group is smaller, the smallest from 384 to 448 (410 at 4100); else 256.
__host__ __device__ constexpr int pair_threads(int n) {
    if (n % 8 != 0)
        for (int t = 384; t <= 448; ++t)
            if (n % t == 0) return t;
    for (int t = 256; t <= 320; ++t)
        if (n % t == 0) return t;
    for (int t = 255; t >= 192; --t)
        if (n % t == 0) return t;
    return 256;
}

struct PairPlan {
    int stages = 0;                                // -1: not a length this engine takes
    int radix[kMixedMaxStages] = {};
};

// The radix sequence of mixed_plan (16s, then one of 8 / 4 / 2, then odd primes ascending):
// odd primes up to kMaxOddRadix, and at most one larger prime (up to kMixedMaxRadix, with a
// Rader split), which the ascending order makes the last stage.
__host__ __device__ constexpr PairPlan pair_plan(int n) {
    PairPlan p{};
    if (n < 16 || (n & 1)) {
        p.stages = -1;
        return p;
    }
    int m = n;
    while (m % 16 == 0 && p.stages < kMixedMaxStages) {
        p.radix[p.stages++] = 16;
        m /= 16;
    }
    if (m % 8 == 0) {
        p.radix[p.stages++] = 8;
        m /= 8;
    } else if (m % 4 == 0) {
        p.radix[p.stages++] = 4;
        m /= 4;
    } else if (m % 2 == 0) {
        p.radix[p.stages++] = 2;
        m /= 2;
    }
    for (int q = 3; q <= kMaxOddRadix && m > 1; q += 2)
        while (m % q == 0 && p.stages < kMixedMaxStages) {
            p.radix[p.stages++] = q;
            m /= q;
        }
    // what is left has no factor up to 13: a prime when it is at most 61 (< 17^2), taken as a
    // Rader stage where R - 1 splits into the engine's butterflies (rader.cuh)
    if (m > 1 && m <= kMixedMaxRadix && rader_l1(m) > 0 && p.stages < kMixedMaxStages) {
        p.radix[p.stages++] = m;
        m = 1;
    }
    if (m != 1) p.stages = -1;
    return p;
}

// Resident blocks per SM the kernels are compiled for (their register budget): three with
// blocks of up to 320 threads (1400, 2800), two with the 410-thread blocks of 4100.
__host__ __device__ constexpr int pair_min_blocks(int n) { return pair_threads(n) <= 320 ? 3 : 2; }

// Shared bytes of one line pair (N pair slots at mpad positions).
__host__ __device__ constexpr size_t pair_smem(int n) { return (size_t)(mpad(n) + 1) * sizeof(CP); }

// Rows per TMA box of the column pass: the largest divisor of n up to 256 (200 at 1400 and
// 2800, 205 at 4100). Boxes sit in the staging copy at a pitch of whole 8-row (128-byte) units,
// so that each starts on a 128-byte boundary; 0 (plain loads and stores) where the padded
// boxes would not fit in the line buffer.
__host__ __device__ constexpr int pair_tma_pitch(int rows) { return (rows + 7) / 8 * 8; }
__host__ __device__ constexpr int pair_tma_rows(int n) {
    for (int r = 256; r >= 8; --r)
        if (n % r == 0)
            return (size_t)(n / r) * pair_tma_pitch(r) * sizeof(CP) <= pair_smem(n) ? r : 0;
    return 0;
}
// Shared memory of the passes: the line pair (which also holds the dense staging copy of the
// rows or of the column strip on the way in, and of the strip on the way out), then the
// mbarrier of the bulk / TMA copies.
__host__ __device__ constexpr size_t pair_bar_off(int n) { return (pair_smem(n) + 15) / 16 * 16; }
__host__ __device__ constexpr size_t pair_col_smem(int n) {
    return pair_tma_rows(n) ? pair_bar_off(n) + 16 : pair_smem(n);
}

// Odd R-point DFT of a packed pair, natural order in and out, from the pair sums
// s_b = u_b + u_{R-b} and differences d_b = u_b - u_{R-b} (as odd_dft in mixed.cuh):
// re_a = u_0 + sum_b s_b cos(2 pi ab/R), im_a = sum_b d_b sin(2 pi ab/R); forward
// out[a] = re_a - i im_a, out[R-a] = re_a + i im_a, signs swapped for the inverse.
// cs[m], sn[m], ns[m] = cos, sin, -sin of 2 pi m / R on both lanes, m = 0 ... (R-1)/2.
template <int R, bool INV>
__device__ __forceinline__ void odd_dftp(CP (&u)[R], const u64* cs, const u64* sn, const u64* ns) {
    constexpr int H = (R - 1) / 2;
    CP sm[H + 1], df[H + 1];
    CP o0 = u[0];
#pragma unroll
    for (int b = 1; b <= H; ++b) {
        sm[b] = pk::cadd(u[b], u[R - b]);
        df[b] = pk::csub(u[b], u[R - b]);
        o0 = pk::cadd(o0, sm[b]);
    }
#pragma unroll
    for (int a = 1; a <= H; ++a) {
        CP re = u[0];
        CP im{0ull, 0ull};
#pragma unroll
        for (int b = 1; b <= H; ++b) {
            const int m = (a * b) % R;
            const u64 c = m <= H ? cs[m] : cs[R - m];
            const u64 s = m <= H ? sn[m] : ns[R - m];
            re.re = pk::fma2(sm[b].re, c, re.re);
            re.im = pk::fma2(sm[b].im, c, re.im);
            im.re = pk::fma2(df[b].re, s, im.re);
            im.im = pk::fma2(df[b].im, s, im.im);
        }
        // -i im = (im.im, -im.re)
        const CP p{pk::add2(re.re, im.im), pk::sub2(re.im, im.re)};
        const CP q{pk::sub2(re.re, im.im), pk::add2(re.im, im.re)};
        u[a] = INV ? q : p;
        u[R - a] = INV ? p : q;
    }
    u[0] = o0;
}

// One in-place Stockham stage over the line pair in buf (every thread of the block calls it
// after a barrier that made buf complete; it ends with one). lin: the linear table W_N^m, and
// from entry OFF the stage's twiddle block, W_{NS R}^{r k} at (r - 1) NS + k.
template <int N, int T, int R, int NS, int OFF, bool INV>
__device__ __forceinline__ void pair_stage(CP* buf, int tid, const float2* __restrict__ lin) {
    constexpr int NB = N / R;                       // butterflies
    constexpr int K = (NB + T - 1) / T;             // per thread
    constexpr bool FULL = NB % T == 0;
    CP u[K][R];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int j = tid + i * T;
        if (FULL || j < NB) {
#pragma unroll
            for (int r = 0; r < R; ++r) u[i][r] = buf[mpad(j + r * NB)];
        }
    }
    __syncthreads();
    constexpr int H = R % 2 ? (R - 1) / 2 + 1 : 1;
    u64 cs[H], sn[H], ns[H];
    if constexpr (R % 2 == 1) {
#pragma unroll
        for (int m = 0; m < H; ++m) {
            const float2 w = __ldg(lin + m * (N / R));     // cos - i sin of 2 pi m / R
            cs[m] = pk::pack(w.x, w.x);
            sn[m] = pk::pack(-w.y, -w.y);
            ns[m] = pk::pack(w.y, w.y);
        }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int j = tid + i * T;
        if (FULL || j < NB) {
            const int k = j % NS;
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    u64 wr, wi;
                    pk::load_tw(lin + OFF + (r - 1) * NS + k, wr, wi);
                    u[i][r] = pk::cmul_b<INV>(u[i][r], wr, wi);
                }
            }
            if constexpr (R % 2 == 1) odd_dftp<R, INV>(u[i], cs, sn, ns);
            else pk::dftp<R, INV>(u[i]);
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[mpad(base + r * NS)] = u[i][r];
        }
    }
    __syncthreads();
}

// Rader's stage for a prime last radix R (41 at N = 4100; rader.cuh): the butterfly's R outputs
// from a cyclic convolution of length L = R - 1 = L1 L2 done as two length-L DFTs, in place in
// the butterfly's own slots. Index i of the convolution lives at slot g^i (position
// j + g^i N/R). The second DFT is a forward one: its output at index i is the convolution at
// -i, which is X[g^i] - x[0], so every value returns to the slot it came from and no step holds
// registers across a barrier. (1) One task per butterfly and q2 < L2: the Stockham twiddles, an
// L1-point DFT over i = L2 q1 + q2, the twiddles w_L^(q2 k1). (2) One task per butterfly and
// k1 < L1: an L2-point DFT (giving A = DFT_L(a); x[0] + A[0] is X[0]), the product with the
// table B (the DFT of the convolution kernel, divided by L), another L2-point DFT and the
// twiddles of the second transform. (3) One task per butterfly and i2 < L2: an L1-point DFT,
// plus x[0].
template <int N, int T, int R, int NS, int OFF, bool INV>
__device__ __forceinline__ void pair_stage_rader(CP* buf, int tid, const float2* __restrict__ lin) {
    static_assert(NS * R == N, "a prime radix above 13 runs as the last stage");
    constexpr int NB = N / R;
    constexpr int L = R - 1;
    constexpr int L1 = rader_l1(R);
    constexpr int L2 = L / L1;
    constexpr int G = rader_root(R);
    constexpr int ROFF = OFF + (R - 1) * NS;       // the Rader tables follow the stage's block
    static_assert(L1 > 0 && L1 * L2 == L && (L2 % 2 == 1), "Rader split");
    const float2* wl = lin + ROFF;                  // w_L^m
    const float2* bt = lin + ROFF + (INV ? 2 : 1) * L;
    // static shared arrays sized in whole 128-byte units, so that the dynamic line buffer after
    // them stays 128-byte aligned for the column pass's TMA boxes
    __shared__ __align__(128) CP xs[(NB + 7) / 8 * 8];      // x[0] of every butterfly
    constexpr int H = (L2 - 1) / 2 + 1;
    u64 cs[H], sn[H], ns[H];                        // L2-point DFT constants: w_L^(m L1) = w_L2^m
#pragma unroll
    for (int m = 0; m < H; ++m) {
        const float2 w = __ldg(wl + m * L1);
        cs[m] = pk::pack(w.x, w.x);
        sn[m] = pk::pack(-w.y, -w.y);
        ns[m] = pk::pack(w.y, w.y);
    }
    __shared__ __align__(128) int gtab[(L + 31) / 32 * 32];  // g^i mod R: the slot of index i
    for (int m = tid; m < L; m += T) gtab[m] = rader_pow(G, m, R);
    __syncthreads();
    // (1)
#pragma unroll 1
    for (int task = tid; task < NB * L2; task += T) {
        const int q2 = task / NB, j = task % NB;
        CP u[L1];
        int pos[L1];                                // the slots of indices L2 q1 + q2, in and out
#pragma unroll
        for (int q1 = 0; q1 < L1; ++q1) {
            const int r = gtab[L2 * q1 + q2];
            pos[q1] = mpad(j + r * NB);
            u64 wr, wi;
            pk::load_tw(lin + OFF + (r - 1) * NS + j, wr, wi);
            u[q1] = pk::cmul_b<INV>(buf[pos[q1]], wr, wi);
        }
        pk::dftp<L1, false>(u);
#pragma unroll
        for (int k1 = 1; k1 < L1; ++k1) {
            u64 wr, wi;
            pk::load_tw(wl + q2 * k1, wr, wi);
            u[k1] = pk::cmul_b<false>(u[k1], wr, wi);
        }
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) buf[pos[k1]] = u[k1];
    }
    __syncthreads();
    // (2)
#pragma unroll 1
    for (int task = tid; task < NB * L1; task += T) {
        const int k1 = task / NB, j = task % NB;
        CP v[L2];
        int pos[L2];                                // the slots of indices L2 k1 + q2
#pragma unroll
        for (int q2 = 0; q2 < L2; ++q2) {
            pos[q2] = mpad(j + gtab[L2 * k1 + q2] * NB);
            v[q2] = buf[pos[q2]];
        }
        if constexpr (L2 > 1) odd_dftp<L2, false>(v, cs, sn, ns);        // A[k1 + L1 k2] in v[k2]
        if (k1 == 0) {
            const CP x0 = buf[mpad(j)];
            xs[j] = x0;
            buf[mpad(j)] = pk::cadd(x0, v[0]);                          // X[0] = x[0] + A[0]
        }
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) {
            u64 wr, wi;
            pk::load_tw(bt + k1 + L1 * k2, wr, wi);
            v[k2] = pk::cmul_b<false>(v[k2], wr, wi);
        }
        if constexpr (L2 > 1) odd_dftp<L2, false>(v, cs, sn, ns);
#pragma unroll
        for (int i2 = 1; i2 < L2; ++i2) {
            u64 wr, wi;
            pk::load_tw(wl + i2 * k1, wr, wi);
            v[i2] = pk::cmul_b<false>(v[i2], wr, wi);
        }
#pragma unroll
        for (int i2 = 0; i2 < L2; ++i2) buf[pos[i2]] = v[i2];
    }
    __syncthreads();
    // (3)
#pragma unroll 1
    for (int task = tid; task < NB * L2; task += T) {
        const int i2 = task / NB, j = task % NB;
        CP u[L1];
        int pos[L1];                                // the slots of indices L2 k1 + i2
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            pos[k1] = mpad(j + gtab[L2 * k1 + i2] * NB);
            u[k1] = buf[pos[k1]];
        }
        pk::dftp<L1, false>(u);
        const CP x0 = xs[j];
#pragma unroll
        for (int i1 = 0; i1 < L1; ++i1) buf[pos[i1]] = pk::cadd(x0, u[i1]);
    }
    __syncthreads();
}

// N-point DFT of the line pair in buf, natural order in and out. lin: the linear table W_N^m
// followed by the per-stage twiddle blocks of every stage with NS > 1 (OFF: the next block).
template <int N, int T, bool INV, int S = 0, int NS = 1, int OFF = N>
__device__ __forceinline__ void pair_fft(CP* buf, int tid, const float2* __restrict__ lin) {
    constexpr PairPlan P = pair_plan(N);
    static_assert(P.stages > 0, "a length of the packed-pair mixed engine");
    if constexpr (S < P.stages) {
        constexpr int R = P.radix[S];
        if constexpr (R % 2 == 1 && R > kMaxOddRadix) {
            pair_stage_rader<N, T, R, NS, OFF, INV>(buf, tid, lin);
        } else {
            pair_stage<N, T, R, NS, OFF, INV>(buf, tid, lin);
        }
        pair_fft<N, T, INV, S + 1, NS * R, (NS > 1 ? OFF + (R - 1) * NS : OFF)>(buf, tid, lin);
    }
}

}  // namespace mpair

// grid (N / 2, batch): one block per row pair (rows 2 blockIdx.x and 2 blockIdx.x + 1, packed
// as lanes 0 / 1); a.tw is the linear table of N, then the per-stage blocks and Rader tables.
// Elements are evaluated per row and sample (apply_elems_n, as in the one-line engines) between
// the inverse and the forward transform.
template <int N, int T>
__global__ void __launch_bounds__(T, mpair::pair_min_blocks(N))
row_pass_mixed_pair_kernel(const __grid_constant__ RowArgs<float2> a) {
    using mpair::CP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CP* buf = reinterpret_cast<CP*>(smem_raw);
    constexpr int S = (N + T - 1) / T;
    const int ya = 2 * blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    const size_t ra = ((size_t)b * N + ya) * N, rb = ra + N;
    // the two rows arrive by two bulk copies into the line buffer (dense, row A then row B),
    // then move through registers into the padded pair layout
    const bool bulk = !(a.flags & RF_INIT_ONE) && ((uintptr_t)a.in & 15) == 0;
    if (bulk) {
        float2* stage = reinterpret_cast<float2*>(smem_raw);
        uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + mpair::pair_bar_off(N));
        if (tid == 0) {
            tc::mbar_init(bar, 1);
            tc::fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0) {
            tc::mbar_arrive_expect_tx(bar, (uint32_t)(2 * N * sizeof(float2)));
            tc::bulk_load(stage, a.in + ra, (uint32_t)(N * sizeof(float2)), bar);
            tc::bulk_load(stage + N, a.in + rb, (uint32_t)(N * sizeof(float2)), bar);
        }
        tc::mbar_wait(bar, 0, a.err, 16);
        float2 va[S], vb[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int x = tid + s * T;
            if (S * T == N || x < N) {
                va[s] = stage[x];
                vb[s] = stage[N + x];
            }
        }
        __syncthreads();                             // every row sample read before the rearrangement
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int x = tid + s * T;
            if (S * T == N || x < N) buf[mpad(x)] = CP{pk::pack(va[s].x, vb[s].x), pk::pack(va[s].y, vb[s].y)};
        }
    } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int x = tid + s * T;
            if (S * T == N || x < N) {
                float2 va = make_float2(1.f, 0.f), vb = va;
                if (!(a.flags & RF_INIT_ONE)) {
                    va = a.in[ra + x];
                    vb = a.in[rb + x];
                }
                buf[mpad(x)] = CP{pk::pack(va.x, vb.x), pk::pack(va.y, vb.y)};
            }
        }
    }
    __syncthreads();
    if (a.flags & RF_INV_FIRST) mpair::pair_fft<N, T, true>(buf, tid, a.tw);
    if (a.elems.count) {
        if constexpr (S * T == N) {
            // every thread holds S samples of both rows: one call per row, so that the
            // element loads (OPD maps) of all S samples are in flight at once
            const float pre[S] = {};
            float2 pa[S], pb[S];
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const CP v = buf[mpad(tid + s * T)];
                pk::unpack(v.re, pa[s].x, pb[s].x);
                pk::unpack(v.im, pa[s].y, pb[s].y);
            }
            apply_elems_n<float2, T, S>(pa, tid, ya, b, N, a.elems, pre, -1);
            apply_elems_n<float2, T, S>(pb, tid, ya + 1, b, N, a.elems, pre, -1);
#pragma unroll
            for (int s = 0; s < S; ++s) buf[mpad(tid + s * T)] = CP{pk::pack(pa[s].x, pb[s].x), pk::pack(pa[s].y, pb[s].y)};
        } else {
            const float pre1[1] = {0.f};
#pragma unroll 1
            for (int s = 0; s < S; ++s) {
                const int x = tid + s * T;
                if (x < N) {
                    const CP v = buf[mpad(x)];
                    float2 pa[1], pb[1];
                    pk::unpack(v.re, pa[0].x, pb[0].x);
                    pk::unpack(v.im, pa[0].y, pb[0].y);
                    apply_elems_n<float2, 1, 1>(pa, x, ya, b, N, a.elems, pre1, -1);
                    apply_elems_n<float2, 1, 1>(pb, x, ya + 1, b, N, a.elems, pre1, -1);
                    buf[mpad(x)] = CP{pk::pack(pa[0].x, pb[0].x), pk::pack(pa[0].y, pb[0].y)};
                }
            }
        }
        __syncthreads();
    }
    if (a.flags & RF_FWD_AFTER) mpair::pair_fft<N, T, false>(buf, tid, a.tw);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int x = tid + s * T;
        if (S * T == N || x < N) {
            const CP v = buf[mpad(x)];
            float2 va, vb;
            pk::unpack(v.re, va.x, vb.x);
            pk::unpack(v.im, va.y, vb.y);
            a.out[ra + x] = va;
            a.out[rb + x] = vb;
        }
    }
}

// grid (N / 2, batch): one block per column pair (columns 2 blockIdx.x, 2 blockIdx.x + 1: one
// 16-byte segment per row); tab_y multiplies between the transforms, tab_x (per column, which
// commutes with the column transforms) after them. With BR > 0 the strip arrives and leaves by
// TMA, in boxes of 2 columns x BR rows through a staging copy, which moves the strided
// 16-byte rows faster than plain loads and stores (the 2800 column pass: 98 -> 86 us); mi / mo
// are the tensor maps of a.in / a.out (boxes 2 x BR). The staging copy is the line buffer itself,
// read into registers before it is rearranged into the padded layout (and back on the way out),
// so that three blocks still share an SM.
template <int N, int T, int BR>
__global__ void __launch_bounds__(T, mpair::pair_min_blocks(N))
col_pass_mixed_pair_kernel(const __grid_constant__ ColArgs<float2> a, const __grid_constant__ CUtensorMap mi,
                           const __grid_constant__ CUtensorMap mo) {
    using mpair::CP;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CP* buf = reinterpret_cast<CP*>(smem_raw);
    float4* stage = reinterpret_cast<float4*>(smem_raw);                 // TMA boxes of BR rows
    constexpr int BRP = mpair::pair_tma_pitch(BR > 0 ? BR : 8);          // box pitch in rows
    auto srow = [](int y) { return BR > 0 ? (y / BR) * BRP + y % BR : y; };
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + mpair::pair_bar_off(N));
    constexpr int S = (N + T - 1) / T;
    constexpr size_t ROW4 = N / 2;                  // float4 per row
    const int col = 2 * blockIdx.x, b = blockIdx.y, tid = threadIdx.x;
    // TMA wants the staging boxes on 128-byte boundaries: a block whose shared memory were placed
    // otherwise would move its strip with plain loads and stores instead (same results)
    const bool tma = BR > 0 && (tc::smem_u32(stage) & 127u) == 0;
    if (tma) {
        if (tid == 0) {
            tc::mbar_init(bar, 1);
            tc::fence_mbar_init();
            tc::prefetch_tmap(&mi);
        }
        __syncthreads();
        if (tid == 0) {
            tc::mbar_arrive_expect_tx(bar, (uint32_t)(N * sizeof(CP)));
#pragma unroll 1
            for (int q = 0; q < N / BR; ++q) tc::tma_load_2d(stage + q * BRP, &mi, bar, col, b * N + q * BR);
        }
        tc::mbar_wait(bar, 0, a.err, 16);
    }
    const float4* src = reinterpret_cast<const float4*>(a.in + (size_t)b * N * N + col);
    {
        float4 q[S];                                 // (re_A, im_A, re_B, im_B) of rows tid + s T
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int y = tid + s * T;
            if (S * T == N || y < N) q[s] = tma ? stage[srow(y)] : src[(size_t)y * ROW4];
        }
        if (tma) __syncthreads();                    // every staged row read before the rearrangement
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int y = tid + s * T;
            if (S * T == N || y < N) buf[mpad(y)] = CP{pk::pack(q[s].x, q[s].z), pk::pack(q[s].y, q[s].w)};
        }
    }
    __syncthreads();
    if (a.flags & CF_FWD) mpair::pair_fft<N, T, false>(buf, tid, a.tw);
    if (a.flags & CF_TABLE) {
        const float2* ty = a.tab_y + (size_t)b * N;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int y = tid + s * T;
            if (S * T == N || y < N) {
                const float2 h = ty[y];
                buf[mpad(y)] = pk::cmul_b<false>(buf[mpad(y)], pk::pack(h.x, h.x), pk::pack(h.y, h.y));
            }
        }
        __syncthreads();
    }
    if (a.flags & CF_INV) mpair::pair_fft<N, T, true>(buf, tid, a.tw);
    pk::u64 hr = pk::pack(1.f, 1.f), hi = 0ull;
    if (a.flags & CF_TABLE) {
        const float2 ha = a.tab_x[(size_t)b * N + col], hb = a.tab_x[(size_t)b * N + col + 1];
        hr = pk::pack(ha.x, hb.x);
        hi = pk::pack(ha.y, hb.y);
    }
    float4* dst = reinterpret_cast<float4*>(a.out + (size_t)b * N * N + col);
    float4 q[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int y = tid + s * T;
        if (S * T == N || y < N) {
            CP v = buf[mpad(y)];
            if (a.flags & CF_TABLE)
                v = CP{pk::sub2(pk::mul2(v.re, hr), pk::mul2(v.im, hi)), pk::fma2(v.re, hi, pk::mul2(v.im, hr))};
            pk::unpack(v.re, q[s].x, q[s].z);
            pk::unpack(v.im, q[s].y, q[s].w);
            if (!tma) dst[(size_t)y * ROW4] = q[s];
        }
    }
    if (tma) {
        __syncthreads();                             // every padded slot read before the staged copy
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int y = tid + s * T;
            if (S * T == N || y < N) stage[srow(y)] = q[s];
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
#pragma unroll 1
            for (int q = 0; q < N / BR; ++q) tc::tma_store_2d(&mo, stage + q * BRP, col, b * N + q * BR);
            tc::bulk_commit();
            tc::bulk_wait_read<0>();         // staging read out; the writes finish with the grid
        }
    }
}

// Whether the packed-pair engine has an instance for complex64 lines of length n.
inline bool mixed_pair_length(int n) { return n == 1400 || n == 2800 || n == 4100; }

namespace detail {

template <int N>
cudaError_t row_launch_mixed_pair_n(const RowArgs<float2>& a, const PassLaunch& l) {
    constexpr int T = mpair::pair_threads(N);
    const size_t smem = mpair::pair_bar_off(N) + 16;          // line buffer and mbarrier
    static unsigned done = 0;
    cudaError_t e = ensure_smem(row_pass_mixed_pair_kernel<N, T>, smem, done);
    if (e != cudaSuccess) return e;
    row_pass_mixed_pair_kernel<N, T><<<dim3(N / 2, l.batch), T, smem, l.stream>>>(a);
    return cudaGetLastError();
}

// The 16-byte row segments need 16-byte aligned planes (checked on the host).
template <int N>
cudaError_t col_launch_mixed_pair_n(const ColArgs<float2>& a, const PassLaunch& l) {
    constexpr int T = mpair::pair_threads(N);
    constexpr int BR = mpair::pair_tma_rows(N);
    if (((uintptr_t)a.in & 15) || ((uintptr_t)a.out & 15)) return cudaErrorInvalidValue;
    const size_t smem = mpair::pair_col_smem(N);
    static unsigned done = 0;
    cudaError_t e = ensure_smem(col_pass_mixed_pair_kernel<N, T, BR>, smem, done);
    if (e != cudaSuccess) return e;
    CUtensorMap mi, mo;
    std::memset(&mi, 0, sizeof(mi));
    std::memset(&mo, 0, sizeof(mo));
    if constexpr (BR > 0) {
        if ((e = tc_make_field_map(a.in, N, (long long)l.batch * N, 2, &mi, BR)) != cudaSuccess) return e;
        if ((e = tc_make_field_map(a.out, N, (long long)l.batch * N, 2, &mo, BR)) != cudaSuccess) return e;
    }
    col_pass_mixed_pair_kernel<N, T, BR><<<dim3(N / 2, l.batch), T, smem, l.stream>>>(a, mi, mo);
    return cudaGetLastError();
}

inline cudaError_t row_launch_mixed_pair(int n, const RowArgs<float2>& a, const PassLaunch& l) {
    switch (n) {
        case 1400: return row_launch_mixed_pair_n<1400>(a, l);
        case 2800: return row_launch_mixed_pair_n<2800>(a, l);
        case 4100: return row_launch_mixed_pair_n<4100>(a, l);
        default: return cudaErrorInvalidValue;
    }
}

inline cudaError_t col_launch_mixed_pair(int n, const ColArgs<float2>& a, const PassLaunch& l) {
    switch (n) {
        case 1400: return col_launch_mixed_pair_n<1400>(a, l);
        case 2800: return col_launch_mixed_pair_n<2800>(a, l);
        case 4100: return col_launch_mixed_pair_n<4100>(a, l);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace detail
}  // namespace coro
