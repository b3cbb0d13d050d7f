// fft_engine.cuh -- register/shared-memory FFT of one line (a row or a column) for sm_103a.
//
// The paper's hot loop is the sequence of 2-D FFTs of large complex arrays (Sec. 1.2, Sec. 2.2;
// 19 FFTs per wavelength for its 10-optic system). Here one line of length N = 2^k is held by
// N/16 threads, 16 complex samples each. Thread t holds x[t + s*N/16] in slot s, before and
// after the transform. The transform is a Stockham decimation-in-time FFT: every pass reads
// slot s from position t + s*N/16, multiplies by W_{Ns R}^{r k}, does an R-point DFT in
// registers and writes position (j/Ns)*Ns*R + j%Ns + r*Ns. The last pass writes back to the
// thread's own slots, so a line needs (passes - 1) shared-memory exchanges: two for N = 4096
// (radix 16 x 16 x 16). Shared memory is padded by one sample per 16 so that both the strided
// writes and the unit-stride reads are free of bank conflicts.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace coro {

template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename C> __device__ __forceinline__ C mk(typename real_of<C>::type x, typename real_of<C>::type y) {
    C c; c.x = x; c.y = y; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
// complex64: the real and imaginary parts of one sample as one FP32x2 pair, so that a complex
// add or subtract issues as one packed instruction (Blackwell .f32x2) instead of two
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return bits_f2(d);
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk<C>(a.x, -a.y); }
template <typename C> __device__ __forceinline__ C cscale(C a, typename real_of<C>::type s) { return mk<C>(a.x * s, a.y * s); }
// a * (-i) for the forward sign, a * (+i) for the inverse sign.
template <bool INV, typename C> __device__ __forceinline__ C mul_mi(C a) {
    return INV ? mk<C>(-a.y, a.x) : mk<C>(a.y, -a.x);
}

// cos(2 pi m / 16), sin(2 pi m / 16) for m = 0..15 (values of the circular functions at
// multiples of pi/8).
__host__ __device__ constexpr double kCos16(int m) {
    return m == 0 ? 1.0 : m == 1 ? 0.92387953251128675613 : m == 2 ? 0.70710678118654752440
         : m == 3 ? 0.38268343236508977173 : m == 4 ? 0.0 : m == 5 ? -0.38268343236508977173
         : m == 6 ? -0.70710678118654752440 : m == 7 ? -0.92387953251128675613 : m == 8 ? -1.0
         : m == 9 ? -0.92387953251128675613 : m == 10 ? -0.70710678118654752440
         : m == 11 ? -0.38268343236508977173 : m == 12 ? 0.0 : m == 13 ? 0.38268343236508977173
         : m == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}
__host__ __device__ constexpr double kSin16(int m) { return kCos16((m + 12) & 15); }

// Multiply by W_16^m = exp(-+ 2 pi i m / 16) (sign by INV), m a compile-time constant.
template <int M, bool INV, typename C> __device__ __forceinline__ C tw16(C a) {
    using R = typename real_of<C>::type;
    constexpr int m = M & 15;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (m == 4) {
        return mul_mi<INV>(a);
    } else if constexpr (m == 8) {
        return mk<C>(-a.x, -a.y);
    } else if constexpr (m == 12) {
        return mul_mi<!INV>(a);
    } else {
        const R c = (R)kCos16(m);
        const R s = INV ? (R)kSin16(m) : -(R)kSin16(m);   // W = c + i s
        return mk<C>(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a0, C& a1) {
    C t = a0; a0 = cadd(t, a1); a1 = csub(t, a1);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& a0, C& a1, C& a2, C& a3) {
    if constexpr (std::is_same<C, float2>::value) {
        // the -+i rotation of d folds into scalar adds; the other six complex adds are packed
        const C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
        a0 = cadd(t0, t2);
        a2 = csub(t0, t2);
        if (INV) {                                  // t3 = +i d = (-d.y, d.x)
            a1 = mk<C>(t1.x - d.y, t1.y + d.x);
            a3 = mk<C>(t1.x + d.y, t1.y - d.x);
        } else {                                    // t3 = -i d = (d.y, -d.x)
            a1 = mk<C>(t1.x + d.y, t1.y - d.x);
            a3 = mk<C>(t1.x - d.y, t1.y + d.x);
        }
    } else {
        C t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
        a0 = cadd(t0, t2); a2 = csub(t0, t2); a1 = cadd(t1, t3); a3 = csub(t1, t3);
    }
}

// R-point DFT in place, natural order in and out: out[k] = sum_r in[r] W_R^{rk}.
// R = P*Q with P = 2 (R = 8) or 4 (R = 16): Q-point DFTs over the stride-P subsequences,
// twiddle W_R^{p k1}, then P-point DFTs across them; out index k1 + Q k2.
template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C (&v)[R]) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        dft4<INV>(v[0], v[2], v[4], v[6]);
        dft4<INV>(v[1], v[3], v[5], v[7]);
        // u[p][k1] sits at v[p + 2 k1]; twiddle u[1][k1] by W_8^{k1} = W_16^{2 k1}
        v[3] = tw16<2, INV>(v[3]);
        v[5] = tw16<4, INV>(v[5]);
        v[7] = tw16<6, INV>(v[7]);
        C o[8];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C a = v[2 * k1], b = v[2 * k1 + 1];
            o[k1] = cadd(a, b);
            o[k1 + 4] = csub(a, b);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = o[i];
    } else if constexpr (R == 16) {
        dft4<INV>(v[0], v[4], v[8], v[12]);
        dft4<INV>(v[1], v[5], v[9], v[13]);
        dft4<INV>(v[2], v[6], v[10], v[14]);
        dft4<INV>(v[3], v[7], v[11], v[15]);
        // u[p][k1] sits at v[p + 4 k1]; twiddle by W_16^{p k1}
        v[5] = tw16<1, INV>(v[5]);
        v[9] = tw16<2, INV>(v[9]);
        v[13] = tw16<3, INV>(v[13]);
        v[6] = tw16<2, INV>(v[6]);
        v[10] = tw16<4, INV>(v[10]);
        v[14] = tw16<6, INV>(v[14]);
        v[7] = tw16<3, INV>(v[7]);
        v[11] = tw16<6, INV>(v[11]);
        v[15] = tw16<9, INV>(v[15]);
        // P = 4 point DFT over p for each k1; result index k1 + 4 k2
        C o[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            C a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
            dft4<INV>(a0, a1, a2, a3);
            o[k1] = a0; o[k1 + 4] = a1; o[k1 + 8] = a2; o[k1 + 12] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
}

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Twiddle table: one block per pass with span NS > 1, laid out [r - 1][k] (r in [1, R),
// k in [0, NS)) holding W_{NS R}^{r k} = exp(-2 pi i r k / (NS R)), built in FP64 and rounded.
// Threads of a warp hold consecutive k, so each load is one or two contiguous wavefronts.
// Every pass but the last has R = 16, so the block of span NS starts at 15 (16 + 256 + ...).
__host__ __device__ constexpr int twiddle_offset(int ns) {
    int off = 0;
    for (int s = 16; s < ns; s *= 16) off += 15 * s;
    return off;
}

template <bool INV, typename C> __device__ __forceinline__ C twiddle(const C* __restrict__ tw, int m) {
    C w = __ldg(tw + m);
    if (INV) w.y = -w.y;
    return w;
}

// Barrier policies for the exchanges: the whole block, or one named barrier shared by the
// threads of an independent unit inside the block (ids 1..15; count a multiple of 32).
struct SyncBlock {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncNamed {
    int id, count;
    __device__ __forceinline__ void operator()() const {
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
    }
};

// One Stockham pass with span NS; recursion continues until NS * R == N.
// buf: this line's shared-memory region, indexed through pad16().
template <typename C, int N, bool INV, int NS, typename Sync>
__device__ __forceinline__ void line_fft_pass(C (&v)[16], C* buf, int t, const C* __restrict__ tw, const Sync& sync) {
    constexpr int TPL = N / 16;
    constexpr int REM = N / NS;
    constexpr int R = REM >= 16 ? 16 : REM;
    constexpr int B = 16 / R;
    constexpr bool LAST = (NS * R == N);
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int j = t + b * TPL;
        const int k = j & (NS - 1);
        C u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = v[b + r * B];
        if constexpr (NS > 1) {
            const C* blk = tw + twiddle_offset(NS) + k;
#pragma unroll
            for (int r = 1; r < R; ++r) u[r] = cmul(u[r], twiddle<INV>(blk, (r - 1) * NS));
        }
        dft<R, INV>(u);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * B] = u[r];
        } else {
            const int base = (j / NS) * NS * R + k;
            // positions base + r*NS: for NS a multiple of 16 (or NS = 1 with base a multiple
            // of 16) the padded addresses advance by a compile-time stride
            if constexpr (NS % 16 == 0 || (NS == 1 && R == 16)) {
                constexpr int PS = NS == 1 ? 1 : NS + NS / 16;
                C* p = buf + pad16(base);
#pragma unroll
                for (int r = 0; r < R; ++r) p[r * PS] = u[r];
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) buf[pad16(base + r * NS)] = u[r];
            }
        }
    }
    if constexpr (!LAST) {
        sync();
        if constexpr (TPL % 16 == 0) {
            const C* p = buf + pad16(t);
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = p[s * (TPL + TPL / 16)];
        } else {
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = buf[pad16(t + s * TPL)];
        }
        sync();
        line_fft_pass<C, N, INV, NS * R>(v, buf, t, tw, sync);
    }
}

// Full N-point DFT of the line held by the calling threads (all threads that share the
// barrier must call it together). Without a policy the barrier is the whole block.
template <typename C, int N, bool INV, typename Sync = SyncBlock>
__device__ __forceinline__ void line_fft(C (&v)[16], C* buf, int t, const C* __restrict__ tw, const Sync& sync = Sync{}) {
    line_fft_pass<C, N, INV, 1>(v, buf, t, tw, sync);
}

template <int N> struct LineGeom {
    static constexpr int TPL = N / 16;                 // threads per line
    static constexpr int STRIDE = N + N / 16;          // padded samples per line
};

}  // namespace coro
