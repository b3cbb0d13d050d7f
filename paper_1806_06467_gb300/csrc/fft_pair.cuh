// fft_pair.cuh -- two lines transformed in lock step with packed FP32x2 arithmetic.
//
// Blackwell executes add/sub/mul/fma on a pair of FP32 values held in one 64-bit register
// pair as one instruction (PTX .f32x2). Two lines of the same length undergo exactly the
// same FFT, so lane 0 of every packed register belongs to line A and lane 1 to line B: a
// complex sample pair is CP{re = (re_A, re_B), im = (im_A, im_B)}. Butterflies, constant
// twiddles and table twiddles then issue half the instructions of the one-line engine in
// fft_engine.cuh, with the same operations in the same order on each lane (results are
// bitwise those of the one-line engine up to FMA contraction choices).
//
// Layout and pass structure are those of fft_engine.cuh (Stockham radix-16, thread t holds
// positions t + s*N/16 in slot s, pad16 shared layout), with 16-byte shared elements.
// Twiddles come from the one-line table, each entry duplicated into both lanes on load.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_engine.cuh"

namespace coro {
namespace pk {

typedef unsigned long long u64;

struct __align__(16) CP {
    u64 re, im;
};

__device__ __forceinline__ u64 pack(float a, float b) {
    u64 d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ void unpack(u64 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ CP cadd(CP a, CP b) { return CP{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ CP csub(CP a, CP b) { return CP{sub2(a.re, b.re), sub2(a.im, b.im)}; }

// v * w with w = {(w_re, w_re), (w_im, w_im)} the same on both lanes; INV uses conj(w).
template <bool INV> __device__ __forceinline__ CP cmul_b(CP v, u64 wr, u64 wi) {
    if (INV) return CP{fma2(v.im, wi, mul2(v.re, wr)), sub2(mul2(v.im, wr), mul2(v.re, wi))};
    return CP{sub2(mul2(v.re, wr), mul2(v.im, wi)), fma2(v.re, wi, mul2(v.im, wr))};
}

// Multiply by W_16^m = exp(-+ 2 pi i m / 16), m a compile-time constant.
template <int M, bool INV> __device__ __forceinline__ CP tw16p(CP a) {
    constexpr int m = M & 15;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (m == 4) {                  // * (-i) forward, * (+i) inverse
        return INV ? CP{sub2(0ull, a.im), a.re} : CP{a.im, sub2(0ull, a.re)};
    } else if constexpr (m == 8) {
        return CP{sub2(0ull, a.re), sub2(0ull, a.im)};
    } else if constexpr (m == 12) {
        return INV ? CP{a.im, sub2(0ull, a.re)} : CP{sub2(0ull, a.im), a.re};
    } else {
        const float c = (float)kCos16(m);
        const float s = INV ? (float)kSin16(m) : -(float)kSin16(m);   // W = c + i s
        const u64 cc = pack(c, c), ss = pack(s, s), ns = pack(-s, -s);
        return CP{fma2(a.re, cc, mul2(a.im, ns)), fma2(a.re, ss, mul2(a.im, cc))};
    }
}

// 4-point DFT in place; the +-i rotation folds into the output adds.
template <bool INV> __device__ __forceinline__ void dft4p(CP& a0, CP& a1, CP& a2, CP& a3) {
    const CP t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    if (INV) {                                      // t3 = +i d = (-d.im, d.re)
        a1 = CP{sub2(t1.re, d.im), add2(t1.im, d.re)};
        a3 = CP{add2(t1.re, d.im), sub2(t1.im, d.re)};
    } else {                                        // t3 = -i d = (d.im, -d.re)
        a1 = CP{add2(t1.re, d.im), sub2(t1.im, d.re)};
        a3 = CP{sub2(t1.re, d.im), add2(t1.im, d.re)};
    }
}

// R-point DFT, natural order in and out (same factorisation as the one-line dft<R>).
template <int R, bool INV> __device__ __forceinline__ void dftp(CP (&v)[R]) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        const CP t = v[0];
        v[0] = cadd(t, v[1]);
        v[1] = csub(t, v[1]);
    } else if constexpr (R == 4) {
        dft4p<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        dft4p<INV>(v[0], v[2], v[4], v[6]);
        dft4p<INV>(v[1], v[3], v[5], v[7]);
        v[3] = tw16p<2, INV>(v[3]);
        v[5] = tw16p<4, INV>(v[5]);
        v[7] = tw16p<6, INV>(v[7]);
        CP o[8];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            o[k1] = cadd(v[2 * k1], v[2 * k1 + 1]);
            o[k1 + 4] = csub(v[2 * k1], v[2 * k1 + 1]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = o[i];
    } else if constexpr (R == 16) {
        dft4p<INV>(v[0], v[4], v[8], v[12]);
        dft4p<INV>(v[1], v[5], v[9], v[13]);
        dft4p<INV>(v[2], v[6], v[10], v[14]);
        dft4p<INV>(v[3], v[7], v[11], v[15]);
        v[5] = tw16p<1, INV>(v[5]);
        v[9] = tw16p<2, INV>(v[9]);
        v[13] = tw16p<3, INV>(v[13]);
        v[6] = tw16p<2, INV>(v[6]);
        v[10] = tw16p<4, INV>(v[10]);
        v[14] = tw16p<6, INV>(v[14]);
        v[7] = tw16p<3, INV>(v[7]);
        v[11] = tw16p<6, INV>(v[11]);
        v[15] = tw16p<9, INV>(v[15]);
        CP o[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            CP a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
            dft4p<INV>(a0, a1, a2, a3);
            o[k1] = a0; o[k1 + 4] = a1; o[k1 + 8] = a2; o[k1 + 12] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = o[i];
    }
}

// Table twiddle from the one-line complex64 table, duplicated into a lane-uniform pair
// (a table of pre-duplicated pairs would double the cache footprint, which costs more).
__device__ __forceinline__ void load_tw(const float2* p, u64& wr, u64& wi) {
    const float2 w = __ldg(p);
    wr = pack(w.x, w.x);
    wi = pack(w.y, w.y);
}

// Shared-memory slot of line position p. Default: pad16 (N + N/16 slots). SWZ: exactly N slots,
// the 16-byte slot's index within its group of 8 XORed with bits 4-6 of p. Every access pattern
// of the passes below (16 consecutive positions per thread, stride-16 positions per thread,
// t + s N/16) then puts any 8 consecutive threads of a warp on 8 different 16-byte bank
// groups, the same conflict-free property the padding gives, without the 1/16 extra space.
template <bool SWZ> __device__ __forceinline__ int xslot(int p) { return SWZ ? (p ^ ((p >> 4) & 7)) : pad16(p); }

// One Stockham pass with span NS over a line pair (see line_fft_pass in fft_engine.cuh).
// HALF: the exchange goes through a buffer of N/2 (padded) entries in two rounds. Every pass
// but the last has R = 16, and the 16 positions a thread writes lie in one block of 16 NS
// positions, inside the first half of the line exactly when t < N/32; the positions a thread
// reads back, t + s N/16, lie in the first half exactly when s < 8. So round one lets the
// threads t < N/32 write and everyone read slots 0..7, round two the others and slots 8..15.
template <int N, bool INV, int NS, bool HALF, typename Sync, bool SWZ = false>
__device__ __forceinline__ void line_fft_pass2(CP (&v)[16], CP* buf, int t, const float2* __restrict__ tw,
                                               const Sync& sync) {
    static_assert(!(SWZ && HALF), "the swizzled layout has no half-size form");
    constexpr int TPL = N / 16;
    constexpr int REM = N / NS;
    constexpr int R = REM >= 16 ? 16 : REM;
    constexpr int B = 16 / R;
    constexpr bool LAST = (NS * R == N);
    if constexpr (LAST) {
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const int j = t + b * TPL;
            const int k = j & (NS - 1);
            CP u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[b + r * B];
            if constexpr (NS > 1) {
                const float2* blk = tw + twiddle_offset(NS) + k;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    u64 wr, wi;
                    load_tw(blk + (r - 1) * NS, wr, wi);
                    u[r] = cmul_b<INV>(u[r], wr, wi);
                }
            }
            dftp<R, INV>(u);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b + r * B] = u[r];
        }
    } else {
        static_assert(R == 16 && B == 1, "every pass before the last is radix 16");
        const int k = t & (NS - 1);
        if constexpr (NS > 1) {
            const float2* blk = tw + twiddle_offset(NS) + k;
#pragma unroll
            for (int r = 1; r < 16; ++r) {
                u64 wr, wi;
                load_tw(blk + (r - 1) * NS, wr, wi);
                v[r] = cmul_b<INV>(v[r], wr, wi);
            }
        }
        dftp<16, INV>(v);
        const int base = (t / NS) * NS * 16 + k;
        // positions base + r NS (minus `shift`); for NS a multiple of 16, or NS = 1, the
        // padded addresses advance by a compile-time stride
        auto write = [&](int shift) {
            if constexpr (SWZ) {
#pragma unroll
                for (int r = 0; r < 16; ++r) buf[xslot<true>(base - shift + r * NS)] = v[r];
            } else if constexpr (NS % 16 == 0 || NS == 1) {
                constexpr int PS = NS == 1 ? 1 : NS + NS / 16;
                CP* p = buf + pad16(base - shift);
#pragma unroll
                for (int r = 0; r < 16; ++r) p[r * PS] = v[r];
            } else {
#pragma unroll
                for (int r = 0; r < 16; ++r) buf[pad16(base - shift + r * NS)] = v[r];
            }
        };
        auto read = [&](CP (&dst)[16], int s0, int s1, int shift) {
            if constexpr (SWZ && TPL % 128 == 0) {
                // t + s TPL: the multiple of TPL leaves bits 4-6 alone, so the slots advance by TPL
                const CP* p = buf + xslot<true>(t + s0 * TPL - shift);
#pragma unroll
                for (int s = s0; s < s1; ++s) dst[s] = p[(s - s0) * TPL];
            } else if constexpr (SWZ) {
#pragma unroll
                for (int s = s0; s < s1; ++s) dst[s] = buf[xslot<true>(t + s * TPL - shift)];
            } else if constexpr (TPL % 16 == 0) {
                const CP* p = buf + pad16(t + s0 * TPL - shift);
#pragma unroll
                for (int s = s0; s < s1; ++s) dst[s] = p[(s - s0) * (TPL + TPL / 16)];
            } else {
#pragma unroll
                for (int s = s0; s < s1; ++s) dst[s] = buf[pad16(t + s * TPL - shift)];
            }
        };
        if constexpr (!HALF) {
            write(0);
            sync();
            read(v, 0, 16, 0);
            sync();
        } else {
            const bool lo = t < TPL / 2;
            CP w[16];
            if (lo) write(0);
            sync();
            read(w, 0, 8, 0);
            sync();
            if (!lo) write(N / 2);
            sync();
            read(w, 8, 16, N / 2);
            sync();
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = w[s];
        }
        line_fft_pass2<N, INV, NS * 16, HALF, Sync, SWZ>(v, buf, t, tw, sync);
    }
}

// Full N-point DFT of a line pair held by the TPL threads that share `sync`. buf holds
// N + N/16 padded entries, N/2 + N/32 with HALF, or exactly N with SWZ.
template <int N, bool INV, bool HALF = false, typename Sync, bool SWZ = false>
__device__ __forceinline__ void line_fft2(CP (&v)[16], CP* buf, int t, const float2* __restrict__ tw,
                                          const Sync& sync) {
    line_fft_pass2<N, INV, 1, HALF, Sync, SWZ>(v, buf, t, tw, sync);
}

}  // namespace pk
}  // namespace coro
