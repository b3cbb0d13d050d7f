// mixed.cuh -- row and column passes for line lengths N that are not powers of two
// (N = 2800 = 16 * 5 * 5 * 7, N = 4100 = 4 * 5 * 5 * 41, ...: Sec. 3.1 notes that N = 2800 ran
// faster than the next power of two, and App. B's system uses npix = 1025).
//
// The line transform is the Stockham autosort FFT of fft_engine.cuh with mixed radices: stage
// s of radix R with NS = the product of the earlier radices reads x[j + r N/R], multiplies by
// W_{NS R}^{r (j mod NS)}, takes an R-point DFT and writes position
// (j / NS) NS R + j mod NS + r NS. Radices are 16s, then one of 8 / 4 / 2, then the odd prime
// factors in ascending order (up to 61); 2, 4, 8 and 16 use the engine's butterflies, odd
// radices the R-point DFT sum. Lines live in shared memory (two buffers, ping-pong), so the
// pass stays one HBM round trip: a row pass (IFFT, elements, FFT) per block row, a column
// pass (FFT, transfer table, IFFT) per block of L adjacent columns. Twiddles come from the
// linear table W_N^m, m in [0, N), generated in FP64.
#pragma once
#include "passes_launch.cuh"

namespace coro {

constexpr int kMixedMaxStages = 16;
constexpr int kMixedMaxRadix = 61;
constexpr int kMixedThreads = 256;        // row blocks (one line)
constexpr int kMixedColThreads = 1024;    // column blocks (L lines, the only block on its SM)
constexpr size_t kMixedMaxSmem = 200 * 1024;

struct MixedPlan {
    int n;
    int stages;
    int radix[kMixedMaxStages];
};

// Radix sequence of n; false when n is odd, below 16, has a prime factor above
// kMixedMaxRadix or needs more stages than fit. pow2_radix (16 or 8) is the radix taken while
// it divides what is left, before one smaller power of two (8 / 4 / 2) and the odd primes:
// 4096 = 16 x 16 x 16 by default, 8 x 8 x 8 x 8 with pow2_radix 8 (the shared-memory engine's
// alternative factorisation of the power-of-two lengths, a tuner candidate).
inline bool mixed_plan(int n, MixedPlan* mp, int pow2_radix = 16) {
    if (n < 16 || (n & 1)) return false;
    mp->n = n;
    mp->stages = 0;
    int m = n;
    auto push = [&](int r) {
        if (mp->stages >= kMixedMaxStages) return false;
        mp->radix[mp->stages++] = r;
        m /= r;
        return true;
    };
    if (pow2_radix != 16 && pow2_radix != 8) return false;
    while (m % pow2_radix == 0)
        if (!push(pow2_radix)) return false;
    for (int r : {8, 4, 2})
        if (r < pow2_radix && m % r == 0) {
            if (!push(r)) return false;
            break;
        }
    for (int p = 3; m > 1 && p <= kMixedMaxRadix; p += 2)
        while (m % p == 0)
            if (!push(p)) return false;
    return m == 1;
}

// Shared-memory layout: sample i of a buffer sits at mpad(i) = i + i/16, so that the
// radix-R writes of the first stage (stride R) and the column blocks (stride L) spread over
// the banks. A buffer holds n L samples.
__host__ __device__ constexpr int mpad(int i) { return i + (i >> 4); }
template <typename C> __host__ __device__ constexpr size_t mixed_buf(int n, int L) { return (size_t)mpad(n * L) + 1; }
// Shared bytes of a pass over L interleaved lines of length n (two buffers).
template <typename C> constexpr size_t mixed_smem(int n, int L) { return 2 * mixed_buf<C>(n, L) * sizeof(C); }

template <bool INV, typename C> __device__ __forceinline__ C lin_tw(const C* __restrict__ lin, int m) {
    const C w = __ldg(lin + m);
    return INV ? cconj(w) : w;
}

// Odd R-point DFT from the pair sums s_b = u_b + u_{R-b} and differences d_b = u_b - u_{R-b}:
// with re_a = u_0 + sum_b s_b cos(2 pi ab/R) and im_a = sum_b d_b sin(2 pi ab/R), the forward
// transform is out[a] = re_a - i im_a, out[R-a] = re_a + i im_a (signs swapped for the
// inverse). cs[m], sn[m] = cos, sin(2 pi m / R) for m = 0 ... (R-1)/2.
template <int R, bool INV, typename C, typename T>
__device__ __forceinline__ void odd_dft(C (&u)[R], const T* cs, const T* sn) {
    constexpr int H = (R - 1) / 2;
    C sm[H + 1], df[H + 1];
    C o0 = u[0];
#pragma unroll
    for (int b = 1; b <= H; ++b) {
        sm[b] = cadd(u[b], u[R - b]);
        df[b] = csub(u[b], u[R - b]);
        o0 = cadd(o0, sm[b]);
    }
#pragma unroll
    for (int a = 1; a <= H; ++a) {
        C re = u[0], im = mk<C>(0, 0);
#pragma unroll
        for (int b = 1; b <= H; ++b) {
            const int m = (a * b) % R;
            const T c = m <= H ? cs[m] : cs[R - m];
            const T sg = m <= H ? sn[m] : -sn[R - m];
            re = mk<C>(re.x + sm[b].x * c, re.y + sm[b].y * c);
            im = mk<C>(im.x + df[b].x * sg, im.y + df[b].y * sg);
        }
        // -i im = (im.y, -im.x)
        const C mi = INV ? mk<C>(-im.y, im.x) : mk<C>(im.y, -im.x);
        u[a] = cadd(re, mi);
        u[R - a] = csub(re, mi);
    }
    u[0] = o0;
}

// One stage of radix R over L interleaved lines: sample `row` of line c at [row * L + c].
// 2 / 4 / 8 / 16 use the engine's butterflies; odd R the pair-sum DFT with cos / sin of
// 2 pi m / R read once per stage from the linear table.
template <typename C, int R, bool INV>
__device__ __forceinline__ void mixed_stage(const C* __restrict__ src, C* __restrict__ dst, int n, int ns, int L,
                                            const C* __restrict__ lin) {
    using T = typename real_of<C>::type;
    const int nb = n / R, step = n / (ns * R);
    const int lsh = __ffs(L) - 1;                       // L is 1, 2, 4 or 8
    constexpr int H = (R - 1) / 2 + 1;
    T cs[H], sn[H];
    if constexpr (R % 2 == 1) {
#pragma unroll
        for (int m = 0; m < H; ++m) {
            const C w = __ldg(lin + m * (n / R));           // cos - i sin
            cs[m] = w.x;
            sn[m] = -w.y;
        }
    }
    for (int i = threadIdx.x; i < nb * L; i += blockDim.x) {
        const int c = i & (L - 1), j = i >> lsh, k = j % ns;
        C u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = src[mpad((j + r * nb) * L + c)];
        if (ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) u[r] = cmul(u[r], lin_tw<INV>(lin, r * k * step));
        }
        if constexpr (R % 2 == 1) odd_dft<R, INV>(u, cs, sn);
        else dft<R, INV>(u);
        const int base = (j / ns) * ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[mpad((base + r * ns) * L + c)] = u[r];
    }
}

// The same for an odd prime radix known only at run time (R <= kMixedMaxRadix); cs / sn
// (shared) hold cos, sin(2 pi m / R) for m = 0 ... (R-1)/2. Two block-wide steps, so that
// every thread has work even when the stage has few butterflies: (1) one task per butterfly
// and pair b = 1 ... (R-1)/2 twiddles u_b and u_{R-b} and leaves s_b = u_b + u_{R-b} and
// d_b = u_b - u_{R-b} in their places in src; (2) one task per butterfly and output pair
// (a, R - a) sums them (the pair-sum DFT of odd_dft), a = 0 giving u_0 + sum_b s_b.
template <typename C, bool INV>
__device__ void mixed_stage_any(C* __restrict__ src, C* __restrict__ dst, int n, int ns, int L, int R,
                                const C* __restrict__ lin, const typename real_of<C>::type* cs,
                                const typename real_of<C>::type* sn) {
    using T = typename real_of<C>::type;
    const int nb = n / R, step = n / (ns * R), H = (R - 1) / 2;
    const int tasks = nb * L, lsh = __ffs(L) - 1;      // L is 1, 2, 4 or 8
    for (int i = threadIdx.x; i < tasks * H; i += blockDim.x) {
        const int c = i & (L - 1), jb = i >> lsh, j = jb % nb, bb = jb / nb + 1;
        const int k = j % ns;
        const int pb = mpad((j + bb * nb) * L + c), pc = mpad((j + (R - bb) * nb) * L + c);
        C ub = src[pb], uc = src[pc];
        if (ns > 1) {
            ub = cmul(ub, lin_tw<INV>(lin, bb * k * step));
            uc = cmul(uc, lin_tw<INV>(lin, (R - bb) * k * step));
        }
        src[pb] = cadd(ub, uc);
        src[pc] = csub(ub, uc);
    }
    __syncthreads();
    // step (2): group 0 is a = 0; group g >= 1 holds the outputs a = 4 (g - 1) + 1 ... + 4, each
    // loaded s_b, d_b feeding all four accumulators
    constexpr int G = 4;
    const int groups = 1 + (H + G - 1) / G;
    for (int i = threadIdx.x; i < tasks * groups; i += blockDim.x) {
        const int c = i & (L - 1), jg = i >> lsh, j = jg % nb, g = jg / nb;
        const int k = j % ns;
        const int base = (j / ns) * ns * R + k;
        const C u0 = src[mpad(j * L + c)];
        if (g == 0) {
            C o0 = u0;
            for (int bb = 1; bb <= H; ++bb) o0 = cadd(o0, src[mpad((j + bb * nb) * L + c)]);
            dst[mpad(base * L + c)] = o0;
            continue;
        }
        const int a0 = G * (g - 1) + 1;
        C re[G], im[G];
        int m[G];
#pragma unroll
        for (int q = 0; q < G; ++q) { re[q] = u0; im[q] = mk<C>(0, 0); m[q] = 0; }
        for (int bb = 1; bb <= H; ++bb) {
            const C sb = src[mpad((j + bb * nb) * L + c)], db = src[mpad((j + (R - bb) * nb) * L + c)];
#pragma unroll
            for (int q = 0; q < G; ++q) {
                m[q] += a0 + q;                                // m = a b mod R
                if (m[q] >= R) m[q] -= R;
                const bool lo = m[q] <= H;
                const T cc = cs[lo ? m[q] : R - m[q]];
                const T sg = lo ? sn[m[q]] : -sn[R - m[q]];
                re[q] = mk<C>(re[q].x + sb.x * cc, re[q].y + sb.y * cc);
                im[q] = mk<C>(im[q].x + db.x * sg, im[q].y + db.y * sg);
            }
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int a = a0 + q;
            if (a > H) break;
            const C mi = INV ? mk<C>(-im[q].y, im[q].x) : mk<C>(im[q].y, -im[q].x);
            dst[mpad((base + a * ns) * L + c)] = cadd(re[q], mi);
            dst[mpad((base + (R - a) * ns) * L + c)] = csub(re[q], mi);
        }
    }
}

// Transform the L lines in buffer a (b is the other buffer); returns the buffer holding the
// result. Called by every thread of the block, after a barrier that made a complete.
template <typename C, bool INV>
__device__ C* mixed_fft(C* a, C* b, const MixedPlan& mp, int L, const C* __restrict__ lin) {
    using T = typename real_of<C>::type;
    __shared__ T cs_any[kMixedMaxRadix / 2 + 1], sn_any[kMixedMaxRadix / 2 + 1];
    int ns = 1;
    C* src = a;
    C* dst = b;
    for (int st = 0; st < mp.stages; ++st) {
        const int R = mp.radix[st];
        const bool any = R != 2 && R != 3 && R != 4 && R != 5 && R != 7 && R != 8 && R != 16;
        if (any) {                                     // uniform: the radix list is a kernel argument
            for (int m = threadIdx.x; m <= (R - 1) / 2; m += blockDim.x) {
                const C w = __ldg(lin + m * (mp.n / R));
                cs_any[m] = w.x;
                sn_any[m] = -w.y;
            }
            __syncthreads();
        }
        switch (R) {
            case 2: mixed_stage<C, 2, INV>(src, dst, mp.n, ns, L, lin); break;
            case 3: mixed_stage<C, 3, INV>(src, dst, mp.n, ns, L, lin); break;
            case 4: mixed_stage<C, 4, INV>(src, dst, mp.n, ns, L, lin); break;
            case 5: mixed_stage<C, 5, INV>(src, dst, mp.n, ns, L, lin); break;
            case 7: mixed_stage<C, 7, INV>(src, dst, mp.n, ns, L, lin); break;
            case 8: mixed_stage<C, 8, INV>(src, dst, mp.n, ns, L, lin); break;
            case 16: mixed_stage<C, 16, INV>(src, dst, mp.n, ns, L, lin); break;
            default: mixed_stage_any<C, INV>(src, dst, mp.n, ns, L, R, lin, cs_any, sn_any); break;
        }
        __syncthreads();
        ns *= R;
        C* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// grid (n, batch): one block per row; a.tw is the linear table of n.
template <typename C>
__global__ void __launch_bounds__(kMixedThreads)
row_pass_mixed_kernel(const __grid_constant__ RowArgs<C> a, const __grid_constant__ MixedPlan mp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = mp.n, y = blockIdx.x, b = blockIdx.y;
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + mixed_buf<C>(n, 1);
    const size_t row = ((size_t)b * n + y) * n;
    for (int x = threadIdx.x; x < n; x += blockDim.x) A[mpad(x)] = (a.flags & RF_INIT_ONE) ? mk<C>(1, 0) : a.in[row + x];
    __syncthreads();
    C* cur = A;
    if (a.flags & RF_INV_FIRST) cur = mixed_fft<C, true>(A, B, mp, 1, a.tw);
    if (a.elems.count) {
        for (int x = threadIdx.x; x < n; x += blockDim.x) {
            C v1[1] = {cur[mpad(x)]};
            const float pre1[1] = {0.f};
            apply_elems_n<C, 1, 1>(v1, x, y, b, n, a.elems, pre1, -1);
            cur[mpad(x)] = v1[0];
        }
        __syncthreads();
    }
    if (a.flags & RF_FWD_AFTER) cur = mixed_fft<C, false>(cur, cur == A ? B : A, mp, 1, a.tw);
    for (int x = threadIdx.x; x < n; x += blockDim.x) a.out[row + x] = cur[mpad(x)];
}

// grid (n / L, batch): one block per L adjacent columns; a.tw is the linear table of n.
template <typename C>
__global__ void __launch_bounds__(kMixedColThreads)
col_pass_mixed_kernel(const __grid_constant__ ColArgs<C> a, const __grid_constant__ MixedPlan mp, int L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = mp.n, b = blockIdx.y, col0 = blockIdx.x * L, lsh = __ffs(L) - 1;   // L: 1, 2, 4 or 8
    C* A = reinterpret_cast<C*>(smem_raw);
    C* B = A + mixed_buf<C>(n, L);
    const size_t base = (size_t)b * n * n + col0;
    for (int i = threadIdx.x; i < n * L; i += blockDim.x) A[mpad(i)] = a.in[base + (size_t)(i >> lsh) * n + (i & (L - 1))];
    __syncthreads();
    C* cur = A;
    if (a.flags & CF_FWD) cur = mixed_fft<C, false>(A, B, mp, L, a.tw);
    if (a.flags & CF_TABLE) {
        for (int i = threadIdx.x; i < n * L; i += blockDim.x) {
            const C h = cmul(a.tab_x[(size_t)b * n + col0 + (i & (L - 1))], a.tab_y[(size_t)b * n + (i >> lsh)]);
            cur[mpad(i)] = cmul(cur[mpad(i)], h);
        }
        __syncthreads();
    }
    if (a.flags & CF_INV) cur = mixed_fft<C, true>(cur, cur == A ? B : A, mp, L, a.tw);
    for (int i = threadIdx.x; i < n * L; i += blockDim.x) a.out[base + (size_t)(i >> lsh) * n + (i & (L - 1))] = cur[mpad(i)];
}

// Columns per block: the widest of 8 / 4 / 2 / 1 that divides n and fits in shared memory.
template <typename C> inline int mixed_col_lines(int n) {
    for (int L : {8, 4, 2, 1})
        if (n % L == 0 && mixed_smem<C>(n, L) <= kMixedMaxSmem) return L;
    return 0;
}

// Whether the mixed-radix passes take line length n in this dtype.
template <typename C> inline bool mixed_supported(int n) {
    MixedPlan mp;
    return mixed_plan(n, &mp) && mixed_col_lines<C>(n) > 0;
}

namespace detail {

template <typename C>
cudaError_t row_launch_mixed(int n, const RowArgs<C>& a, const PassLaunch& l, int pow2_radix = 16) {
    MixedPlan mp;
    if (!mixed_plan(n, &mp, pow2_radix)) return cudaErrorInvalidValue;
    const size_t smem = mixed_smem<C>(n, 1);
    if (smem > kMixedMaxSmem) return cudaErrorInvalidValue;
    static unsigned done = 0;
    cudaError_t e = ensure_smem(row_pass_mixed_kernel<C>, kMixedMaxSmem, done);
    if (e != cudaSuccess) return e;
    row_pass_mixed_kernel<C><<<dim3(n, l.batch), kMixedThreads, smem, l.stream>>>(a, mp);
    return cudaGetLastError();
}

// lines: columns per block (0: the widest that fits, mixed_col_lines). Blocks whose two
// buffers fit in half the shared-memory budget run 512 threads, so that two share an SM and
// one's loads and stores overlap the other's stages; larger ones run 1024 threads alone.
template <typename C>
cudaError_t col_launch_mixed(int n, int lines, const ColArgs<C>& a, const PassLaunch& l, int pow2_radix = 16) {
    MixedPlan mp;
    if (!mixed_plan(n, &mp, pow2_radix)) return cudaErrorInvalidValue;
    const int L = lines > 0 ? lines : mixed_col_lines<C>(n);
    if (L <= 0 || L > 8 || (L & (L - 1)) || n % L || mixed_smem<C>(n, L) > kMixedMaxSmem) return cudaErrorInvalidValue;
    const size_t smem = mixed_smem<C>(n, L);
    const int threads = smem <= kMixedMaxSmem / 2 ? kMixedColThreads / 2 : kMixedColThreads;
    static unsigned done = 0;
    cudaError_t e = ensure_smem(col_pass_mixed_kernel<C>, kMixedMaxSmem, done);
    if (e != cudaSuccess) return e;
    col_pass_mixed_kernel<C><<<dim3(n / L, l.batch), threads, smem, l.stream>>>(a, mp, L);
    return cudaGetLastError();
}

}  // namespace detail
}  // namespace coro
