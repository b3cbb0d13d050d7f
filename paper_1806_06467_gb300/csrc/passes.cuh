// passes.cuh -- the two HBM passes of a 2-D FFT with fused pointwise work.
//
// A Fresnel hop (Sec. 1.1) is E -> IDFT2[H . DFT2[E]] with H separable, H = h(kx) h(ky).
// Written as row and column 1-D transforms, consecutive hops fuse into two passes per hop:
//   row pass     load -> [IFFT rows] -> elements (Eq. 3 phasors, masks, lens) -> [FFT rows] -> store
//   column pass  load -> [FFT cols] -> * tab_x[col] tab_y[row] -> [IFFT cols] -> store
// The fftshift of the centred DFT is folded in as a (-1)^(x+y) sign flip (Sec. 2.4: the paper
// moved fftshift to the GPU; here it costs no memory pass at all).
#pragma once
#include <type_traits>
#include "fft_engine.cuh"
#include "fft_pair.cuh"
#include "tc_ptx.cuh"

namespace coro {

// ------------------------------------------------------------------------------ elements

enum DevElemKind : int {
    DK_NONE = 0,
    DK_APERTURE = 1,   // ithr: [outer r2 max, obscuration r2 max (-1 none), spider |k| max (-1 none)]
    DK_CIRCLE = 2,     // ithr: [r2 max]; flags bit0: opaque inside
    DK_TABLE = 3,      // separable table tab[b][x] * tab[b][y] (lens, QPF)
    DK_OPD_MAP = 4,    // fpar: [2 / lambda as hi, lo]; map [n][n] or [b][n][n]; optional amplitude
    DK_ZERNIKE = 5,    // ithr: [r2 max]; fpar: [2 / lambda, dx/R, their lo parts]; zpoly: combined
                       // polynomials (doubles for complex128)
    DK_SINE = 6,       // fpar: [2 amp / lambda, f_hi, f_lo, -] (cycles per pixel split), flags: axis;
                       // complex128: zpoly -> [batch][f, 2 amp / lambda] doubles
    DK_SCALAR = 7,     // fpar: [s as hi, lo]
    DK_CHECKER = 8,    // (-1)^(x+y)
    DK_CONJ = 9,       // complex conjugate (direct hops with z < 0: IDFT(y) = conj(DFT(conj y)))
    DK_STORE = 10,     // checkpoint: copy the field to dst[b * map_bstride + y * n + x], the field
                       // itself unchanged; flags bit0: the copy is taken times (-1)^(x+y)
    DK_PHASE_GRAD = 11 // float dst[...] = fpar[4b] * Im(v conj(ref)), ref = tab (complex, same
                       // layout as dst; NULL = 1); flags bit0 as DK_STORE. Field unchanged.
};

// Zernike evaluation table: OPD = sum_{m=0}^{ZM-1} A_m(rho^2) Re(z^m) + B_m(rho^2) Im(z^m),
// z = (x + i y)/R, A_m and B_m polynomials of degree < ZD in rho^2 (coefficients in metres).
constexpr int ZM = 8;
constexpr int ZD = 4;

struct DevElem {
    int kind;
    int flags;
    const int* ithr;          // [batch][4] integer thresholds
    const float* fpar;        // [batch][4] float parameters
    const void* tab;          // [batch][n] complex separable table
    const float* map;         // OPD map
    const float* amp;         // amplitude map (nullable)
    long long map_bstride;    // 0 (shared) or n*n
    const float* zpoly;       // [2][ZM][ZD]
    void* dst;                // DK_STORE destination (complex, the pass's dtype)
};

constexpr int kMaxPassElems = 8;   // up to 5 user / plane elements + conj, input QPF, checker

struct PassElems {
    int count;
    DevElem e[kMaxPassElems];
};

// exp(i pi ph) for a phase ph in half-cycles. Complex64 passes reduce ph exactly to
// r = ph - 2 rint(ph / 2) in [-1, 1] (Sterbenz: ph and the even integer are within 1) and
// take the hardware sine and cosine of pi r, whose absolute error on [-pi, pi] is below
// 2^-21.4 -- far inside the FP32 field tolerance, at a fraction of the cost of sincospif.
// Complex128 passes keep sincospif.
template <typename C> __device__ __forceinline__ void phasor_hc(float ph, float& sn, float& cs) {
    if constexpr (std::is_same<C, float2>::value) {
        const float r = ph - 2.f * rintf(0.5f * ph);
        __sincosf(3.14159265358979323846f * r, &sn, &cs);
    } else {
        sincospif(ph, &sn, &cs);
    }
}

template <typename C> constexpr bool kF64 = std::is_same<C, double2>::value;

// Zernike phase for complex128 passes: the polynomial table is FP64 (zpoly then points at
// doubles), 2 / lambda and dx / R come as float pairs (hi + lo).
template <int XS, int S>
__device__ __forceinline__ void zernike_f64(double2 (&v)[S], int x0, int ky, int b, int n, const DevElem& e) {
    const int t0 = e.ithr[4 * b];
    const double k = (double)e.fpar[4 * b] + (double)e.fpar[4 * b + 2];
    const double sc = (double)e.fpar[4 * b + 1] + (double)e.fpar[4 * b + 3];
    const double* zp = reinterpret_cast<const double*>(e.zpoly);
    const double zy = ky * sc;
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        const int kx = x0 + s * XS - n / 2;
        if (kx * kx + ky * ky > t0) continue;        // zero OPD outside the disk
        const double zx = kx * sc;
        const double rho2 = zx * zx + zy * zy;
        double pr = 1.0, pim = 0.0, opd = 0.0;
#pragma unroll 1
        for (int m = 0; m < ZM; ++m) {
            const double* A = zp + m * ZD;
            const double* Bc = zp + ZM * ZD + m * ZD;
            double a = A[ZD - 1], bb = Bc[ZD - 1];
#pragma unroll
            for (int d = ZD - 2; d >= 0; --d) { a = fma(a, rho2, A[d]); bb = fma(bb, rho2, Bc[d]); }
            opd += a * pr + bb * pim;
            const double nr = pr * zx - pim * zy;
            pim = pr * zy + pim * zx;
            pr = nr;
        }
        double sn, cs;
        sincospi(k * opd, &sn, &cs);
        v[s] = cmul(v[s], make_double2(cs, sn));
    }
}

// Multiply the S samples a thread holds (row y of item b of an n x n field, columns
// x0 + s*XS) by every element of the list. The element loop is outermost and uniform across
// the block.
// pre_idx >= 0: element pre_idx is an OPD map whose S values this thread already holds in
// pre (loaded early so that their latency hides behind the inverse FFT).
template <typename C, int XS, int S>
__device__ __forceinline__ void apply_elems_n(C (&v)[S], int x0, int y, int b, int n, const PassElems& pe,
                                              const float (&pre)[S], int pre_idx) {
    using R = typename real_of<C>::type;
    const int ky = y - n / 2;
    for (int i = 0; i < pe.count; ++i) {
        const DevElem& e = pe.e[i];
        switch (e.kind) {
            case DK_APERTURE: {
                const int* th = e.ithr + 4 * b;
                const int t0 = th[0], t1 = th[1], t2 = th[2];
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int kx = x0 + s * XS - n / 2;
                    const int r2 = kx * kx + ky * ky;
                    bool pass = r2 <= t0;
                    if (t1 >= 0 && r2 <= t1) pass = false;
                    if (t2 >= 0 && (abs(kx) <= t2 || abs(ky) <= t2)) pass = false;
                    if (!pass) v[s] = mk<C>(0, 0);
                }
                break;
            }
            case DK_CIRCLE: {
                const int t0 = e.ithr[4 * b];
                const bool opaque_inside = e.flags & 1;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const int kx = x0 + s * XS - n / 2;
                    const bool inside = kx * kx + ky * ky <= t0;
                    if (inside == opaque_inside) v[s] = mk<C>(0, 0);
                }
                break;
            }
            case DK_TABLE: {
                const C* t = reinterpret_cast<const C*>(e.tab) + (size_t)b * n;
                const C ty = t[y];
#pragma unroll
                for (int s = 0; s < S; ++s) v[s] = cmul(v[s], cmul(__ldg(t + x0 + s * XS), ty));
                break;
            }
            case DK_OPD_MAP: {
                const size_t off = (size_t)b * e.map_bstride + (size_t)y * n + x0;
                if constexpr (kF64<C>) {
                    // complex128: 2 / lambda as a float pair, the phase in FP64
                    const double k = (double)e.fpar[4 * b] + (double)e.fpar[4 * b + 1];
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const double ph = k * (double)(i == pre_idx ? pre[s] : __ldg(e.map + off + s * XS));
                        double sn, cs;
                        sincospi(ph, &sn, &cs);
                        const double am = e.amp ? (double)__ldg(e.amp + off + s * XS) : 1.0;
                        v[s] = cmul(v[s], mk<C>(am * cs, am * sn));
                    }
                } else {
                    const float k = e.fpar[4 * b];
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        // phase / pi = (2 / lambda) * OPD
                        const float ph = k * (i == pre_idx ? pre[s] : __ldg(e.map + off + s * XS));
                        float sn, cs;
                        phasor_hc<C>(ph, sn, cs);
                        R am = 1;
                        if (e.amp) am = (R)__ldg(e.amp + off + s * XS);
                        v[s] = cmul(v[s], mk<C>(am * (R)cs, am * (R)sn));
                    }
                }
                break;
            }
            case DK_ZERNIKE: {
                if constexpr (kF64<C>) {
                    zernike_f64<XS, S>(v, x0, ky, b, n, e);
                } else {
                    const int t0 = e.ithr[4 * b];
                    const float k = e.fpar[4 * b], sc = e.fpar[4 * b + 1];
                    const float zy = ky * sc;
                    // the polynomial is evaluated in a rolled loop (few registers); only the phase
                    // of each of the S samples is kept
                    float ph[S];
#pragma unroll 1
                    for (int s = 0; s < S; ++s) {
                        const int kx = x0 + s * XS - n / 2;
                        float opd = 0.f;                          // zero OPD outside the disk
                        if (kx * kx + ky * ky <= t0) {
                            const float zx = kx * sc;
                            const float rho2 = zx * zx + zy * zy;
                            float pr = 1.f, pim = 0.f;
#pragma unroll 1
                            for (int m = 0; m < ZM; ++m) {
                                const float* A = e.zpoly + m * ZD;
                                const float* Bc = e.zpoly + ZM * ZD + m * ZD;
                                float a = A[ZD - 1], bb = Bc[ZD - 1];
#pragma unroll
                                for (int d = ZD - 2; d >= 0; --d) { a = fmaf(a, rho2, A[d]); bb = fmaf(bb, rho2, Bc[d]); }
                                opd += a * pr + bb * pim;
                                const float nr = pr * zx - pim * zy;
                                pim = pr * zy + pim * zx;
                                pr = nr;
                            }
                        }
                        ph[s] = k * opd;
                    }
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        float sn, cs;
                        phasor_hc<C>(ph[s], sn, cs);
                        v[s] = cmul(v[s], mk<C>((R)cs, (R)sn));
                    }
                }
                break;
            }
            case DK_SINE: {
                const float* p = e.fpar + 4 * b;
                const bool along_y = e.flags & 1;
                if constexpr (kF64<C>) {
                    // cycles per pixel and 2 amp / lambda in FP64 (zpoly points at [batch][2] doubles)
                    const double* dp = reinterpret_cast<const double*>(e.zpoly) + 2 * b;
                    const double f = dp[0], amp = dp[1];
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const int kk = along_y ? ky : x0 + s * XS - n / 2;
                        double a = (double)kk * f;
                        a -= rint(a);
                        double sn, cs;
                        sincospi(amp * sinpi(2.0 * a), &sn, &cs);
                        v[s] = cmul(v[s], mk<C>(cs, sn));
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < S; ++s) {
                        const int kk = along_y ? ky : x0 + s * XS - n / 2;
                        // cycles = kk * f with f = f_hi + f_lo and kk * f_hi exact in FP32
                        float a = (float)kk * p[1];
                        a -= rintf(a);
                        a += (float)kk * p[2];
                        float sn, cs;
                        phasor_hc<C>(p[0] * sinpif(2.f * a), sn, cs);
                        v[s] = cmul(v[s], mk<C>((R)cs, (R)sn));
                    }
                }
                break;
            }
            case DK_SCALAR: {
                const R sc = kF64<C> ? (R)((double)e.fpar[4 * b] + (double)e.fpar[4 * b + 1]) : (R)e.fpar[4 * b];
#pragma unroll
                for (int s = 0; s < S; ++s) v[s] = cscale(v[s], sc);
                break;
            }
            case DK_CHECKER: {
#pragma unroll
                for (int s = 0; s < S; ++s)
                    if ((x0 + s * XS + y) & 1) v[s] = mk<C>(-v[s].x, -v[s].y);
                break;
            }
            case DK_CONJ: {
#pragma unroll
                for (int s = 0; s < S; ++s) v[s] = cconj(v[s]);
                break;
            }
            case DK_PHASE_GRAD: {
                const size_t off = (size_t)b * e.map_bstride + (size_t)y * n + x0;
                const C* rf = static_cast<const C*>(e.tab) + off;
                float* d = static_cast<float*>(e.dst) + off;
                const R wgt = kF64<C> ? (R)((double)e.fpar[4 * b] + (double)e.fpar[4 * b + 1]) : (R)e.fpar[4 * b];
                const bool chk = e.flags & 1;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const C r = e.tab ? __ldg(rf + s * XS) : mk<C>(1, 0);   // no reference: 1
                    R im = v[s].y * r.x - v[s].x * r.y;                 // Im(v conj(r))
                    if (chk && ((x0 + s * XS + y) & 1)) im = -im;
                    __stcs(d + s * XS, (float)(wgt * im));
                }
                break;
            }
            case DK_STORE: {
                C* d = static_cast<C*>(e.dst) + (size_t)b * e.map_bstride + (size_t)y * n + x0;
                const bool chk = e.flags & 1;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    const bool neg = chk && ((x0 + s * XS + y) & 1);
                    __stcs(d + s * XS, neg ? mk<C>(-v[s].x, -v[s].y) : v[s]);
                }
                break;
            }
            default:
                break;
        }
    }
}

// The same for a compile-time line length (the power-of-two pass kernels).
template <typename C, int N, int XS>
__device__ __forceinline__ void apply_elems(C (&v)[16], int x0, int y, int b, const PassElems& pe,
                                            const float (&pre)[16], int pre_idx) {
    apply_elems_n<C, XS, 16>(v, x0, y, b, N, pe, pre, pre_idx);
}

// Elements on a packed row pair: the samples a thread holds for rows ya (lane 0) and ya + 1
// (lane 1) of item b, columns x0 + s*XS, as packed pairs (complex64 only). Per element and
// sample, the two rows' factors are evaluated as in apply_elems and applied with packed
// arithmetic, which keeps the register footprint of one sample pair.
template <int N, int XS>
__device__ __forceinline__ void apply_elems_pair(pk::CP (&v)[16], int x0, int ya, int b, const PassElems& pe) {
    using pk::CP;
    using pk::u64;
    const int kya = ya - N / 2, kyb = kya + 1;
    auto mask = [&](int s, bool pa, bool pb) {
        const u64 m = pk::pack(pa ? 1.f : 0.f, pb ? 1.f : 0.f);
        v[s] = CP{pk::mul2(v[s].re, m), pk::mul2(v[s].im, m)};
    };
    // v[s] *= (fr_a + i fi_a, fr_b + i fi_b)
    auto mulf = [&](int s, u64 fr, u64 fi) {
        v[s] = CP{pk::sub2(pk::mul2(v[s].re, fr), pk::mul2(v[s].im, fi)), pk::fma2(v[s].re, fi, pk::mul2(v[s].im, fr))};
    };
    for (int i = 0; i < pe.count; ++i) {
        const DevElem& e = pe.e[i];
        switch (e.kind) {
            case DK_APERTURE: {
                const int* th = e.ithr + 4 * b;
                const int t0 = th[0], t1 = th[1], t2 = th[2];
                auto pass = [&](int kx, int ky) {
                    const int r2 = kx * kx + ky * ky;
                    bool p = r2 <= t0;
                    if (t1 >= 0 && r2 <= t1) p = false;
                    if (t2 >= 0 && (abs(kx) <= t2 || abs(ky) <= t2)) p = false;
                    return p;
                };
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int kx = x0 + s * XS - N / 2;
                    mask(s, pass(kx, kya), pass(kx, kyb));
                }
                break;
            }
            case DK_CIRCLE: {
                const int t0 = e.ithr[4 * b];
                const bool opaque_inside = e.flags & 1;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int kx = x0 + s * XS - N / 2;
                    mask(s, (kx * kx + kya * kya <= t0) != opaque_inside, (kx * kx + kyb * kyb <= t0) != opaque_inside);
                }
                break;
            }
            case DK_TABLE: {
                const float2* t = reinterpret_cast<const float2*>(e.tab) + (size_t)b * N;
                const float2 ta = t[ya], tb = t[ya + 1];
                const u64 tyr = pk::pack(ta.x, tb.x), tyi = pk::pack(ta.y, tb.y), ntyi = pk::pack(-ta.y, -tb.y);
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const float2 tx = __ldg(t + x0 + s * XS);
                    const u64 txr = pk::pack(tx.x, tx.x), txi = pk::pack(tx.y, tx.y);
                    mulf(s, pk::fma2(txr, tyr, pk::mul2(txi, ntyi)), pk::fma2(txr, tyi, pk::mul2(txi, tyr)));
                }
                break;
            }
            case DK_OPD_MAP: {
                const float k = e.fpar[4 * b];
                const size_t off = (size_t)b * e.map_bstride + (size_t)ya * N + x0;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    float sa, ca, sb, cb;
                    phasor_hc<float2>(k * __ldg(e.map + off + s * XS), sa, ca);
                    phasor_hc<float2>(k * __ldg(e.map + off + N + s * XS), sb, cb);
                    if (e.amp) {
                        const float aa = __ldg(e.amp + off + s * XS), ab = __ldg(e.amp + off + N + s * XS);
                        sa *= aa; ca *= aa; sb *= ab; cb *= ab;
                    }
                    mulf(s, pk::pack(ca, cb), pk::pack(sa, sb));
                }
                break;
            }
            case DK_ZERNIKE: {
                const int t0 = e.ithr[4 * b];
                const float k = e.fpar[4 * b], sc = e.fpar[4 * b + 1];
                // one row at a time, through the one-line evaluator's rolled polynomial loop
#pragma unroll 1
                for (int lane = 0; lane < 2; ++lane) {
                    const int ky = lane ? kyb : kya;
                    const float zy = ky * sc;
                    float ph[16];
#pragma unroll 1
                    for (int s = 0; s < 16; ++s) {
                        const int kx = x0 + s * XS - N / 2;
                        float opd = 0.f;
                        if (kx * kx + ky * ky <= t0) {
                            const float zx = kx * sc;
                            const float rho2 = zx * zx + zy * zy;
                            float pr = 1.f, pim = 0.f;
#pragma unroll 1
                            for (int m = 0; m < ZM; ++m) {
                                const float* A = e.zpoly + m * ZD;
                                const float* Bc = e.zpoly + ZM * ZD + m * ZD;
                                float a = A[ZD - 1], bb = Bc[ZD - 1];
#pragma unroll
                                for (int d = ZD - 2; d >= 0; --d) { a = fmaf(a, rho2, A[d]); bb = fmaf(bb, rho2, Bc[d]); }
                                opd += a * pr + bb * pim;
                                const float nr = pr * zx - pim * zy;
                                pim = pr * zy + pim * zx;
                                pr = nr;
                            }
                        }
                        ph[s] = k * opd;
                    }
#pragma unroll
                    for (int s = 0; s < 16; ++s) {
                        float sn, cs;
                        phasor_hc<float2>(ph[s], sn, cs);
                        mulf(s, lane ? pk::pack(1.f, cs) : pk::pack(cs, 1.f), lane ? pk::pack(0.f, sn) : pk::pack(sn, 0.f));
                    }
                }
                break;
            }
            case DK_SINE: {
                const float* p = e.fpar + 4 * b;
                const bool along_y = e.flags & 1;
                auto phase = [&](int kk) {
                    float a = (float)kk * p[1];
                    a -= rintf(a);
                    a += (float)kk * p[2];
                    return p[0] * sinpif(2.f * a);
                };
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const int kx = x0 + s * XS - N / 2;
                    float sa, ca, sb, cb;
                    phasor_hc<float2>(phase(along_y ? kya : kx), sa, ca);
                    if (along_y) phasor_hc<float2>(phase(kyb), sb, cb);
                    else { sb = sa; cb = ca; }
                    mulf(s, pk::pack(ca, cb), pk::pack(sa, sb));
                }
                break;
            }
            case DK_SCALAR: {
                const u64 sc = pk::pack(e.fpar[4 * b], e.fpar[4 * b]);
#pragma unroll
                for (int s = 0; s < 16; ++s) v[s] = CP{pk::mul2(v[s].re, sc), pk::mul2(v[s].im, sc)};
                break;
            }
            case DK_CHECKER: {
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const float sa = ((x0 + s * XS + ya) & 1) ? -1.f : 1.f;
                    const u64 m = pk::pack(sa, -sa);        // rows ya and ya + 1 have opposite parity
                    v[s] = CP{pk::mul2(v[s].re, m), pk::mul2(v[s].im, m)};
                }
                break;
            }
            case DK_CONJ: {
                const u64 m = pk::pack(-1.f, -1.f);
#pragma unroll
                for (int s = 0; s < 16; ++s) v[s].im = pk::mul2(v[s].im, m);
                break;
            }
            case DK_PHASE_GRAD: {
                const size_t off = (size_t)b * e.map_bstride + (size_t)ya * N + x0;
                const float2* rf = static_cast<const float2*>(e.tab) + off;
                float* d = static_cast<float*>(e.dst) + off;
                const float wgt = e.fpar[4 * b];
                const bool chk = e.flags & 1;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const float2 ra = e.tab ? __ldg(rf + s * XS) : make_float2(1.f, 0.f);
                    const float2 rb = e.tab ? __ldg(rf + N + s * XS) : make_float2(1.f, 0.f);
                    float vra, vrb, via, vib;
                    pk::unpack(v[s].re, vra, vrb);
                    pk::unpack(v[s].im, via, vib);
                    const float sa = (chk && ((x0 + s * XS + ya) & 1)) ? -wgt : wgt, sb = chk ? -sa : wgt;
                    __stcs(d + s * XS, sa * (via * ra.x - vra * ra.y));
                    __stcs(d + N + s * XS, sb * (vib * rb.x - vrb * rb.y));
                }
                break;
            }
            case DK_STORE: {
                float2* d = static_cast<float2*>(e.dst) + (size_t)b * e.map_bstride + (size_t)ya * N + x0;
                const bool chk = e.flags & 1;
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    float ra, rb, ia, ib;
                    pk::unpack(v[s].re, ra, rb);
                    pk::unpack(v[s].im, ia, ib);
                    // rows ya and ya + 1 have opposite parity
                    const float sa = (chk && ((x0 + s * XS + ya) & 1)) ? -1.f : 1.f, sb = chk ? -sa : 1.f;
                    __stcs(d + s * XS, make_float2(sa * ra, sa * ia));
                    __stcs(d + N + s * XS, make_float2(sb * rb, sb * ib));
                }
                break;
            }
            default:
                break;
        }
    }
}

// ------------------------------------------------------------------------------ row pass

enum RowFlags : int {
    RF_INV_FIRST = 1,     // inverse row FFT before the elements
    RF_FWD_AFTER = 2,     // forward row FFT after the elements
    RF_INIT_ONE = 4       // do not read: the field starts as 1 + 0i
};

template <typename C>
struct RowArgs {
    const C* in;
    C* out;
    const C* tw;          // twiddles for N
    int flags;
    int* err;             // bounded-wait failure flag (persistent kernel)
    PassElems elems;
};

// First OPD-map element of a pass (its map values get prefetched), or -1.
__device__ __forceinline__ int first_map(const PassElems& pe) {
    for (int i = 0; i < pe.count; ++i)
        if (pe.e[i].kind == DK_OPD_MAP) return i;
    return -1;
}

template <int N> struct RowCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int L0 = TPL >= 256 ? 1 : 256 / TPL;
    static constexpr int L = L0 < N ? L0 : N;                      // lines per block
    static constexpr int THREADS = TPL * L;
    static constexpr int STRIDE = LineGeom<N>::STRIDE;
};

// grid: (N / L, batch); one block = L consecutive rows of one item.
template <typename C, int N>
__global__ void __launch_bounds__(RowCfg<N>::THREADS)
row_pass_kernel(const __grid_constant__ RowArgs<C> a) {
    using Cfg = RowCfg<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int line = threadIdx.x / Cfg::TPL;
    const int t = threadIdx.x % Cfg::TPL;
    const int b = blockIdx.y;
    const int y = blockIdx.x * Cfg::L + line;
    C* buf = smem + line * Cfg::STRIDE;
    const size_t row_off = ((size_t)b * N + y) * N;

    C v[16];
    if (a.flags & RF_INIT_ONE) {
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = mk<C>(1, 0);
    } else {
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = a.in[row_off + t + s * Cfg::TPL];
    }
    if (a.flags & RF_INV_FIRST) line_fft<C, N, true>(v, buf, t, a.tw);
    if (a.elems.count) {
        float none[16];
        apply_elems<C, N, Cfg::TPL>(v, t, y, b, a.elems, none, -1);
    }
    if (a.flags & RF_FWD_AFTER) line_fft<C, N, false>(v, buf, t, a.tw);
#pragma unroll
    for (int s = 0; s < 16; ++s) a.out[row_off + t + s * Cfg::TPL] = v[s];
}

// ------------------------------------------------------------------------------ persistent row pass
//
// Same arithmetic as row_pass_kernel, but each block stays resident and streams line groups:
// the rows of group g+1 arrive by a bulk asynchronous copy into one shared buffer while group
// g is transformed, and group g's result leaves by a bulk store from the buffer it arrived in,
// so HBM traffic overlaps the FFT instead of stalling on it.

template <int N> struct PRowCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int L0 = TPL >= 256 ? 1 : 256 / TPL;
    static constexpr int L = L0 < N ? L0 : N;          // lines per group
    static constexpr int THREADS = TPL * L;
    static constexpr int GROUP = L * N;                 // samples per group (contiguous rows)
    static constexpr int XSTRIDE = LineGeom<N>::STRIDE;
    template <typename C> static constexpr size_t smem() {
        return 2 * (size_t)GROUP * sizeof(C) + (size_t)L * XSTRIDE * sizeof(C) + 64;
    }
};

template <typename C, int N>
__global__ void __launch_bounds__(PRowCfg<N>::THREADS)
row_pass_persistent_kernel(const __grid_constant__ RowArgs<C> a, int groups) {
    using Cfg = PRowCfg<N>;
    constexpr uint32_t BYTES = Cfg::GROUP * sizeof(C);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + Cfg::GROUP;
    C* xbuf = buf1 + Cfg::GROUP;
    uint64_t* full = reinterpret_cast<uint64_t*>(xbuf + Cfg::L * Cfg::XSTRIDE);
    const int line = threadIdx.x / Cfg::TPL;
    const int t = threadIdx.x % Cfg::TPL;
    const bool load = !(a.flags & RF_INIT_ONE);
    C* xl = xbuf + line * Cfg::XSTRIDE;
    const int mi = first_map(a.elems);

    if (threadIdx.x == 0) {
        tc::mbar_init(&full[0], 1);
        tc::mbar_init(&full[1], 1);
        tc::fence_mbar_init();
        if (load && blockIdx.x < groups) {
            tc::mbar_arrive_expect_tx(&full[0], BYTES);
            tc::bulk_load(buf0, a.in + (size_t)blockIdx.x * Cfg::GROUP, BYTES, &full[0]);
        }
    }
    __syncthreads();
    int it = 0;
    bool ok = true;
    for (int g = blockIdx.x; g < groups; g += gridDim.x, ++it) {
        C* ib = (it & 1) ? buf1 : buf0;
        C* nb = (it & 1) ? buf0 : buf1;
        const int row0 = g * Cfg::L;
        const int b = row0 / N, y = row0 % N + line;
        C v[16];
        if (load) {
            if (ok) ok = tc::mbar_wait(&full[it & 1], (it >> 1) & 1, a.err, 5);
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = ib[line * N + t + s * Cfg::TPL];
        } else {
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = mk<C>(1, 0);
        }
        float pre[16];
        if (mi >= 0) {
            const DevElem& e = a.elems.e[mi];
            const float* mp = e.map + (size_t)b * e.map_bstride + (size_t)y * N + t;
#pragma unroll
            for (int s = 0; s < 16; ++s) pre[s] = __ldg(mp + s * Cfg::TPL);
        }
        if (threadIdx.x == 0) {
            if (load) {
                if (g + (int)gridDim.x < groups) {
                    tc::bulk_wait_read<0>();            // group g-1's store has left nb
                    tc::mbar_arrive_expect_tx(&full[(it + 1) & 1], BYTES);
                    tc::bulk_load(nb, a.in + (size_t)(g + gridDim.x) * Cfg::GROUP, BYTES, &full[(it + 1) & 1]);
                }
            } else {
                tc::bulk_wait_read<1>();                // group g-2's store has left ib
            }
        }
        __syncthreads();
        if (a.flags & RF_INV_FIRST) line_fft<C, N, true>(v, xl, t, a.tw);
        if (a.elems.count) apply_elems<C, N, Cfg::TPL>(v, t, y, b, a.elems, pre, mi);
        if (a.flags & RF_FWD_AFTER) line_fft<C, N, false>(v, xl, t, a.tw);
#pragma unroll
        for (int s = 0; s < 16; ++s) ib[line * N + t + s * Cfg::TPL] = v[s];
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::bulk_store(a.out + (size_t)g * Cfg::GROUP, ib, BYTES);
            tc::bulk_commit();
        }
    }
    if (threadIdx.x == 0) tc::bulk_wait<0>();          // shared memory must outlive the stores
}

// ------------------------------------------------------------------------------ column pass

enum ColFlags : int {
    CF_FWD = 1,           // forward column FFT first
    CF_INV = 2,           // inverse column FFT last
    CF_TABLE = 4          // multiply by tab_x[b][col] * tab_y[b][row] between them
};

template <typename C>
struct ColArgs {
    const C* in;
    C* out;
    const C* tw;
    const C* tab_x;       // [batch][N]
    const C* tab_y;       // [batch][N]
    int flags;
    int* err;             // bounded-wait failure flag (persistent kernel)
};

template <int N, int L> struct ColCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int THREADS = TPL * L;
    // column c's region starts at c * STRIDE; STRIDE = 16/L (mod 16) spreads the L columns a
    // half-warp touches over distinct banks.
    static constexpr int STRIDE = LineGeom<N>::STRIDE + ((16 / L) & 15);
    // blocks of at most 512 threads are held to 64 registers so that two fit on an SM
    static constexpr int MINB = THREADS <= 512 ? 2 : 1;
};

// grid: (N / L, batch); one block = L adjacent columns of one item. Thread (t, c) = t*L + c,
// so a warp reads 32/L rows x L contiguous columns.
template <typename C, int N, int L>
__global__ void __launch_bounds__(ColCfg<N, L>::THREADS, ColCfg<N, L>::MINB)
col_pass_kernel(const __grid_constant__ ColArgs<C> a) {
    using Cfg = ColCfg<N, L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* smem = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % L;
    const int t = threadIdx.x / L;
    const int b = blockIdx.y;
    const int col = blockIdx.x * L + c;
    C* buf = smem + c * Cfg::STRIDE;
    const size_t base = (size_t)b * N * N + col;

    C v[16];
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = a.in[base + (size_t)(t + s * Cfg::TPL) * N];
    if (a.flags & CF_FWD) line_fft<C, N, false>(v, buf, t, a.tw);
    if (a.flags & CF_TABLE) {
        const C hx = a.tab_x[(size_t)b * N + col];
        const C* ty = a.tab_y + (size_t)b * N;
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = cmul(v[s], cmul(hx, ty[t + s * Cfg::TPL]));
    }
    if (a.flags & CF_INV) line_fft<C, N, true>(v, buf, t, a.tw);
#pragma unroll
    for (int s = 0; s < 16; ++s) a.out[base + (size_t)(t + s * Cfg::TPL) * N] = v[s];
}

// ------------------------------------------------------------------------------ persistent column pass
//
// A column group (L adjacent columns x N rows) arrives as N/256 tiled TMA boxes of
// 256 rows x L samples into one of two shared buffers while the previous group is being
// transformed, and leaves by TMA tensor stores from the buffer it arrived in. The FFT
// exchanges use a separate padded buffer. `map` views the field as a 2-D array of 8-byte
// samples: x = column (N), y = item * N + row.

template <int N, int L> struct PColCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int THREADS = TPL * L;
    static constexpr int GROUP = L * N;
    static constexpr int BOXES = N / 256;
    static constexpr int STRIDE = ColCfg<N, L>::STRIDE;
    template <typename C> static constexpr size_t smem() {
        return 2 * (size_t)GROUP * sizeof(C) + (size_t)L * STRIDE * sizeof(C) + 64;
    }
};

template <typename C, int N, int L>
__global__ void __launch_bounds__(PColCfg<N, L>::THREADS)
col_pass_persistent_kernel(const __grid_constant__ ColArgs<C> a, const __grid_constant__ CUtensorMap map, int groups) {
    using Cfg = PColCfg<N, L>;
    constexpr uint32_t BYTES = Cfg::GROUP * sizeof(C);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + Cfg::GROUP;
    C* xbuf = buf1 + Cfg::GROUP;
    uint64_t* full = reinterpret_cast<uint64_t*>(xbuf + L * Cfg::STRIDE);
    const int c = threadIdx.x % L;
    const int t = threadIdx.x / L;
    C* xl = xbuf + c * Cfg::STRIDE;
    constexpr int GPI = N / L;                       // groups per item

    auto issue_load = [&](C* dst, uint64_t* bar, int g) {
        const int x = (g % GPI) * L, y = (g / GPI) * N;
        tc::mbar_arrive_expect_tx(bar, BYTES);
#pragma unroll 1
        for (int k = 0; k < Cfg::BOXES; ++k) tc::tma_load_2d(dst + k * 256 * L, &map, bar, x, y + k * 256);
    };
    if (threadIdx.x == 0) {
        tc::mbar_init(&full[0], 1);
        tc::mbar_init(&full[1], 1);
        tc::fence_mbar_init();
        tc::prefetch_tmap(&map);
        if (blockIdx.x < groups) issue_load(buf0, &full[0], blockIdx.x);
    }
    __syncthreads();
    int it = 0;
    bool ok = true;
    for (int g = blockIdx.x; g < groups; g += gridDim.x, ++it) {
        C* ib = (it & 1) ? buf1 : buf0;
        C* nb = (it & 1) ? buf0 : buf1;
        const int b = g / GPI, col = (g % GPI) * L + c;
        if (ok) ok = tc::mbar_wait(&full[it & 1], (it >> 1) & 1, a.err, 6);
        C v[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = ib[(t + s * Cfg::TPL) * L + c];
        if (threadIdx.x == 0 && g + (int)gridDim.x < groups) {
            tc::bulk_wait_read<0>();                    // group g-1's stores have left nb
            issue_load(nb, &full[(it + 1) & 1], g + gridDim.x);
        }
        if (a.flags & CF_FWD) line_fft<C, N, false>(v, xl, t, a.tw);
        if (a.flags & CF_TABLE) {
            const C hx = a.tab_x[(size_t)b * N + col];
            const C* ty = a.tab_y + (size_t)b * N;
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = cmul(v[s], cmul(hx, ty[t + s * Cfg::TPL]));
        }
        if (a.flags & CF_INV) line_fft<C, N, true>(v, xl, t, a.tw);
        __syncthreads();                                 // every thread has read ib before it is rewritten
#pragma unroll
        for (int s = 0; s < 16; ++s) ib[(t + s * Cfg::TPL) * L + c] = v[s];
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int x = (g % GPI) * L, y = b * N;
#pragma unroll 1
            for (int k = 0; k < Cfg::BOXES; ++k) tc::tma_store_2d(&map, ib + k * 256 * L, x, y + k * 256);
            tc::bulk_commit();
        }
    }
    if (threadIdx.x == 0) tc::bulk_wait<0>();
}

// ------------------------------------------------------------------------------ unit-pipelined passes
//
// One resident block per SM is split into U independent units. A unit transforms one line
// group (L adjacent columns, or one row) with its own named barrier and its own shared region,
// which serves as the FFT exchange buffer and then holds the finished group while its
// asynchronous store drains. Line groups arrive by asynchronous copy into S staging slots
// (S <= U): the k-th group of the block lands in slot k % S and is taken by unit k % U, which
// copies it into registers and then issues the copy of group k + S into the slot it just
// emptied (S divides U). Loads, FFTs and stores of different groups therefore overlap while every thread
// of the block keeps its 16 samples in registers. Unit u's j-th group completes phase j of
// mbarrier full[u]. The copy of group k + U is issued only after group k + U - S has been
// taken, which (stepping back by S, S dividing U) needs group k taken first: so phase j + 1
// of full[u] cannot complete before unit u has passed phase j, and a parity wait is exact.

template <int N, int L, int U, int S> struct UColCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int UT = TPL * L;                 // threads per unit
    static constexpr int THREADS = UT * U;
    static constexpr int GROUP = L * N;                // samples per column group
    static constexpr int BOXES = N / 256;
    static constexpr int STRIDE = ColCfg<N, L>::STRIDE;
    static constexpr int REGION = L * STRIDE;          // exchange buffer; >= GROUP
    static_assert(S >= 1 && U % S == 0 && U <= 15, "unit layout");
    template <typename C> static constexpr size_t smem() {
        return ((size_t)S * GROUP + (size_t)U * REGION) * sizeof(C) + 8 * U;
    }
};

template <typename C, int N, int L, int U, int S>
__global__ void __launch_bounds__(UColCfg<N, L, U, S>::THREADS, 1)
col_pass_units_kernel(const __grid_constant__ ColArgs<C> a, const __grid_constant__ CUtensorMap map, int groups) {
    using Cfg = UColCfg<N, L, U, S>;
    constexpr uint32_t BYTES = Cfg::GROUP * sizeof(C);
    constexpr int GPI = N / L;                         // groups per item
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C* stage = reinterpret_cast<C*>(smem_raw);
    const int u = threadIdx.x / Cfg::UT;
    const int ut = threadIdx.x % Cfg::UT;
    const int c = ut % L;
    const int t = ut / L;
    C* region = stage + S * Cfg::GROUP + u * Cfg::REGION;
    uint64_t* full = reinterpret_cast<uint64_t*>(stage + S * Cfg::GROUP + U * Cfg::REGION);
    C* xl = region + c * Cfg::STRIDE;
    const SyncNamed sync{1 + u, Cfg::UT};
    const bool leader = ut == 0;

    // group index k of this block -> slot k % S, consumer unit k % U
    auto issue_load = [&](int k) {
        const int g = blockIdx.x + k * gridDim.x;
        const int x = (g % GPI) * L, y = (g / GPI) * N;
        C* dst = stage + (k % S) * Cfg::GROUP;
        uint64_t* bar = &full[k % U];
        tc::mbar_arrive_expect_tx(bar, BYTES);
#pragma unroll 1
        for (int q = 0; q < Cfg::BOXES; ++q) tc::tma_load_2d(dst + q * 256 * L, &map, bar, x, y + q * 256);
    };
    const int mine = groups > (int)blockIdx.x ? (groups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < U; ++i) tc::mbar_init(&full[i], 1);
        tc::fence_mbar_init();
        tc::prefetch_tmap(&map);
        for (int k = 0; k < S && k < mine; ++k) issue_load(k);
    }
    __syncthreads();
    bool ok = true;
    int j = 0;
    for (int k = u; k < mine; k += U, ++j) {
        const int g = blockIdx.x + k * gridDim.x;
        const int b = g / GPI, col = (g % GPI) * L + c;
        const C* src = stage + (k % S) * Cfg::GROUP;
        if (ok) ok = tc::mbar_wait(&full[u], j & 1, a.err, 7);
        C v[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) v[s] = src[(t + s * Cfg::TPL) * L + c];
        if (leader) tc::bulk_wait_read<0>();           // this unit's previous store has left its region
        sync();                                        // slot emptied by the whole unit; region free
        if (leader && k + S < mine) issue_load(k + S);
        if (a.flags & CF_FWD) line_fft<C, N, false>(v, xl, t, a.tw, sync);
        if (a.flags & CF_TABLE) {
            const C hx = a.tab_x[(size_t)b * N + col];
            const C* ty = a.tab_y + (size_t)b * N;
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = cmul(v[s], cmul(hx, ty[t + s * Cfg::TPL]));
        }
        if (a.flags & CF_INV) line_fft<C, N, true>(v, xl, t, a.tw, sync);
#pragma unroll
        for (int s = 0; s < 16; ++s) region[(t + s * Cfg::TPL) * L + c] = v[s];
        tc::fence_proxy_async();
        sync();
        if (leader) {
            const int x = (g % GPI) * L, y = b * N;
#pragma unroll 1
            for (int q = 0; q < Cfg::BOXES; ++q) tc::tma_store_2d(&map, region + q * 256 * L, x, y + q * 256);
            tc::bulk_commit();
        }
    }
    if (leader) tc::bulk_wait<0>();
}

// Column pass on packed line pairs: a unit of N/16 threads transforms two adjacent columns
// at once, lane 0 / lane 1 of every FP32x2 register holding column A / B (fft_pair.cuh);
// otherwise the unit pipeline of col_pass_units_kernel with L = 2. hx (per column) commutes with the column transforms and is applied after the
// inverse FFT; hy (per row) sits between the two FFTs.
template <int N, int U, int S> struct PColPairCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int UT = TPL;                     // threads per unit (one column pair)
    static constexpr int THREADS = UT * U;
    static constexpr int GROUP = 2 * N;                // float2 samples per pair
    static constexpr int BOXES = N / 256;
    static constexpr int REGION = 2 * LineGeom<N>::STRIDE;   // float2 units; 16-byte pair entries
    static_assert(S >= 1 && U % S == 0 && U <= 15, "unit layout");
    template <typename C> static constexpr size_t smem() {
        return ((size_t)S * GROUP + (size_t)U * REGION) * sizeof(C) + 8 * U;
    }
};

// TOUT: the pair leaves as two contiguous rows of the transposed plane out[b][x][y] (one bulk
// store of 2N samples) instead of two strided columns of out[b][y][x]; out must not alias in.
template <int N, int U, int S, bool TOUT>
__global__ void __launch_bounds__(PColPairCfg<N, U, S>::THREADS, 1)
col_pass_pair_kernel(const __grid_constant__ ColArgs<float2> a, const __grid_constant__ CUtensorMap map, int groups) {
    using Cfg = PColPairCfg<N, U, S>;
    using pk::CP;
    constexpr uint32_t BYTES = Cfg::GROUP * sizeof(float2);
    constexpr int GPI = N / 2;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    const int u = threadIdx.x / Cfg::UT;
    const int t = threadIdx.x % Cfg::UT;
    float2* region = stage + S * Cfg::GROUP + u * Cfg::REGION;
    CP* xl = reinterpret_cast<CP*>(region);
    uint64_t* full = reinterpret_cast<uint64_t*>(stage + S * Cfg::GROUP + U * Cfg::REGION);
    const SyncNamed sync{1 + u, Cfg::UT};
    const bool leader = t == 0;
    const float2* tw = a.tw;

    auto issue_load = [&](int k) {
        const int g = blockIdx.x + k * gridDim.x;
        const int x = (g % GPI) * 2, y = (g / GPI) * N;
        float2* dst = stage + (k % S) * Cfg::GROUP;
        uint64_t* bar = &full[k % U];
        tc::mbar_arrive_expect_tx(bar, BYTES);
#pragma unroll 1
        for (int q = 0; q < Cfg::BOXES; ++q) tc::tma_load_2d(dst + q * 512, &map, bar, x, y + q * 256);
    };
    const int mine = groups > (int)blockIdx.x ? (groups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < U; ++i) tc::mbar_init(&full[i], 1);
        tc::fence_mbar_init();
        tc::prefetch_tmap(&map);
        for (int k = 0; k < S && k < mine; ++k) issue_load(k);
    }
    __syncthreads();
    bool ok = true;
    int j = 0;
    for (int k = u; k < mine; k += U, ++j) {
        const int g = blockIdx.x + k * gridDim.x;
        const int b = g / GPI, col = (g % GPI) * 2;
        const float4* src = reinterpret_cast<const float4*>(stage + (k % S) * Cfg::GROUP);
        if (ok) ok = tc::mbar_wait(&full[u], j & 1, a.err, 9);
        CP v[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const float4 q = src[t + s * Cfg::TPL];       // row t + s*TPL: (re_A, im_A, re_B, im_B)
            v[s] = CP{pk::pack(q.x, q.z), pk::pack(q.y, q.w)};
        }
        if (leader) tc::bulk_wait_read<0>();
        sync();
        if (leader && k + S < mine) issue_load(k + S);
        if (a.flags & CF_FWD) pk::line_fft2<N, false>(v, xl, t, tw, sync);
        if (a.flags & CF_TABLE) {
            const float2* ty = a.tab_y + (size_t)b * N;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const float2 h = ty[t + s * Cfg::TPL];
                v[s] = pk::cmul_b<false>(v[s], pk::pack(h.x, h.x), pk::pack(h.y, h.y));
            }
        }
        if (a.flags & CF_INV) pk::line_fft2<N, true>(v, xl, t, tw, sync);
        if (a.flags & CF_TABLE) {
            const float2 ha = a.tab_x[(size_t)b * N + col], hb = a.tab_x[(size_t)b * N + col + 1];
            const pk::u64 hr = pk::pack(ha.x, hb.x), hi = pk::pack(ha.y, hb.y);
#pragma unroll
            for (int s = 0; s < 16; ++s)
                v[s] = CP{pk::sub2(pk::mul2(v[s].re, hr), pk::mul2(v[s].im, hi)),
                          pk::fma2(v[s].re, hi, pk::mul2(v[s].im, hr))};
        }
        if constexpr (TOUT) {
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                float2 qa, qb;
                pk::unpack(v[s].re, qa.x, qb.x);
                pk::unpack(v[s].im, qa.y, qb.y);
                region[t + s * Cfg::TPL] = qa;
                region[N + t + s * Cfg::TPL] = qb;
            }
        } else {
            float4* out = reinterpret_cast<float4*>(region);
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                float4 q;
                pk::unpack(v[s].re, q.x, q.z);
                pk::unpack(v[s].im, q.y, q.w);
                out[t + s * Cfg::TPL] = q;
            }
        }
        tc::fence_proxy_async();
        sync();
        if (leader) {
            if constexpr (TOUT) {
                tc::bulk_store(a.out + ((size_t)b * N + col) * N, region, BYTES);
            } else {
                const int x = col, y = b * N;
#pragma unroll 1
                for (int q = 0; q < Cfg::BOXES; ++q) tc::tma_store_2d(&map, region + q * 512, x, y + q * 256);
            }
            tc::bulk_commit();
        }
    }
    if (leader) tc::bulk_wait<0>();
}

// Quad column pass: four adjacent columns per strip, so that every row segment the strip reads
// or writes is one whole 32-byte sector (two-column strips stream at about half the copy
// bandwidth of four-column ones). Two units of N/16 threads, unit u transforming the packed
// column pair (2u, 2u + 1) of the strip (fft_pair.cuh), both in one block that owns the SM.
// Room: the exchanges use the swizzled layout of exactly N pair slots (64 KB per unit at
// 4096), and the strip arrives by TMA in quarters (4 columns x N/4 rows, 32 KB at 4096)
// through three staging slots: 2 x 64 + 3 x 32 = 224 KB. A unit pulls its rows of each
// quarter into registers as the quarter lands (rows t + s N/16, s = 4q .. 4q + 3), the block
// releases the slot and the next quarters (of this strip, then the next) load while the
// transforms run. Results go out as 4-column TMA boxes from the two regions, read as one
// [N][4] array once both units have left their last exchange.
template <int N> struct QColCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int THREADS = 2 * TPL;
    static constexpr int QROWS = N / 4;                // rows per quarter strip
    static constexpr int SLOTS = 3;
    static constexpr int SLOT = 4 * QROWS;             // float2 per staging slot
    static constexpr int REGION = 2 * N;               // float2: N pair slots of 16 bytes
    static constexpr int QBOXES = QROWS / 256;         // TMA boxes (4 x 256) per quarter
    static constexpr int OBOXES = N / 256;
    static_assert(QROWS % 256 == 0, "quarter strips of whole 256-row boxes");
    static constexpr size_t smem() { return ((size_t)SLOTS * SLOT + 2 * (size_t)REGION) * sizeof(float2) + 64; }
};

template <int N>
__global__ void __launch_bounds__(QColCfg<N>::THREADS, 1)
col_pass_quad_kernel(const __grid_constant__ ColArgs<float2> a, const __grid_constant__ CUtensorMap map, int strips) {
    using Cfg = QColCfg<N>;
    using pk::CP;
    constexpr int SPI = N / 4;                         // strips per item
    constexpr uint32_t QBYTES = Cfg::SLOT * sizeof(float2);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    float2* regions = stage + Cfg::SLOTS * Cfg::SLOT;  // unit 0, then unit 1; together [N][4]
    uint64_t* full = reinterpret_cast<uint64_t*>(regions + 2 * Cfg::REGION);
    const int u = threadIdx.x / Cfg::TPL;
    const int t = threadIdx.x % Cfg::TPL;
    CP* xl = reinterpret_cast<CP*>(regions + u * Cfg::REGION);
    const SyncNamed sync{1 + u, Cfg::TPL};
    const float2* tw = a.tw;
    const int mine = strips > (int)blockIdx.x ? (strips - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int loads = 4 * mine;                        // quarter loads of this block, in order

    auto issue_load = [&](int i) {                     // quarter i % 4 of this block's strip i / 4
        const int g = blockIdx.x + (i >> 2) * gridDim.x;
        const int x = (g % SPI) * 4, y = (g / SPI) * N + (i & 3) * Cfg::QROWS;
        float2* dst = stage + (i % Cfg::SLOTS) * Cfg::SLOT;
        uint64_t* bar = &full[i % Cfg::SLOTS];
        tc::mbar_arrive_expect_tx(bar, QBYTES);
#pragma unroll 1
        for (int q = 0; q < Cfg::QBOXES; ++q) tc::tma_load_2d(dst + q * 1024, &map, bar, x, y + q * 256);
    };
    if (threadIdx.x == 0) {
        for (int i = 0; i < Cfg::SLOTS; ++i) tc::mbar_init(&full[i], 1);
        tc::fence_mbar_init();
        tc::prefetch_tmap(&map);
        for (int i = 0; i < Cfg::SLOTS && i < loads; ++i) issue_load(i);
    }
    __syncthreads();
    bool ok = true;
    for (int k = 0; k < mine; ++k) {
        const int g = blockIdx.x + k * gridDim.x;
        const int b = g / SPI, x0 = (g % SPI) * 4, col = x0 + 2 * u;
        // the previous strip's stores have read the regions before anything writes them again
        if (threadIdx.x == 0) tc::bulk_wait_read<0>();
        CP v[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = 4 * k + q;
            if (ok) ok = tc::mbar_wait(&full[i % Cfg::SLOTS], (i / Cfg::SLOTS) & 1, a.err, 15);
            const float4* src = reinterpret_cast<const float4*>(stage + (i % Cfg::SLOTS) * Cfg::SLOT);
#pragma unroll
            for (int s = 4 * q; s < 4 * q + 4; ++s) {
                const int r = t + s * Cfg::TPL - q * Cfg::QROWS;      // row within the quarter
                const float4 c = src[r * 2 + u];                        // (re_A, im_A, re_B, im_B)
                v[s] = CP{pk::pack(c.x, c.z), pk::pack(c.y, c.w)};
            }
            __syncthreads();                                            // both units have read the slot
            if (threadIdx.x == 0 && i + Cfg::SLOTS < loads) issue_load(i + Cfg::SLOTS);
        }
        if (a.flags & CF_FWD) pk::line_fft2<N, false, false, SyncNamed, true>(v, xl, t, tw, sync);
        if (a.flags & CF_TABLE) {
            const float2* ty = a.tab_y + (size_t)b * N;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const float2 h = ty[t + s * Cfg::TPL];
                v[s] = pk::cmul_b<false>(v[s], pk::pack(h.x, h.x), pk::pack(h.y, h.y));
            }
        }
        if (a.flags & CF_INV) pk::line_fft2<N, true, false, SyncNamed, true>(v, xl, t, tw, sync);
        if (a.flags & CF_TABLE) {
            const float2 ha = a.tab_x[(size_t)b * N + col], hb = a.tab_x[(size_t)b * N + col + 1];
            const pk::u64 hr = pk::pack(ha.x, hb.x), hi = pk::pack(ha.y, hb.y);
#pragma unroll
            for (int s = 0; s < 16; ++s)
                v[s] = CP{pk::sub2(pk::mul2(v[s].re, hr), pk::mul2(v[s].im, hi)),
                          pk::fma2(v[s].re, hi, pk::mul2(v[s].im, hr))};
        }
        __syncthreads();                               // both units are out of their exchanges
        float4* out = reinterpret_cast<float4*>(regions);                 // [N][4] float2
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            float4 q;
            pk::unpack(v[s].re, q.x, q.z);
            pk::unpack(v[s].im, q.y, q.w);
            out[(t + s * Cfg::TPL) * 2 + u] = q;
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll 1
            for (int q = 0; q < Cfg::OBOXES; ++q) tc::tma_store_2d(&map, regions + q * 1024, x0, b * N + q * 256);
            tc::bulk_commit();
        }
    }
    if (threadIdx.x == 0) tc::bulk_wait<0>();
}

// Wide column pass: four adjacent columns per group, so that every row segment read or
// written is one full 32-byte sector (two-column strips reach about half the copy bandwidth
// of four-column ones). One resident block per SM of two pair-units (N/16 threads each,
// packed FP32x2, fft_pair.cuh); thread (t, p) = 2t + p holds column pair p of the group, so
// a warp covers 16 rows x 4 columns. The next group arrives by TMA (boxes of 4 x 256) in a
// 128-KB staging buffer while the current one is transformed in registers; the FFT
// exchanges use half-size buffers (two rounds), which is what leaves room for the staging
// buffer; results leave by TMA stores through the exchange region, half a group at a time.
template <int N> struct WColCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int THREADS = 2 * TPL;
    static constexpr int MINB = THREADS >= 512 ? 1 : 512 / THREADS;   // 512 threads/SM at <= 128 regs
    static constexpr int GROUP = 4 * N;                 // float2 samples per group
    static constexpr int BOXES = N / 256;
    // CP entries per pair (half buffer); XHALF = 4 (mod 8) puts pair 1's buffer 64 bytes
    // of bank space away from pair 0's, as lanes 2t and 2t + 1 touch the same position of each
    static constexpr int XHALF = N / 2 + N / 32 + 4;
    static constexpr size_t smem() { return (size_t)GROUP * 8 + 2 * (size_t)XHALF * 16 + 16; }
};

template <int N>
__global__ void __launch_bounds__(WColCfg<N>::THREADS, WColCfg<N>::MINB)
col_pass_wide_kernel(const __grid_constant__ ColArgs<float2> a, const __grid_constant__ CUtensorMap map, int groups) {
    using Cfg = WColCfg<N>;
    using pk::CP;
    constexpr uint32_t BYTES = Cfg::GROUP * sizeof(float2);
    constexpr int GPI = N / 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    const int p = threadIdx.x & 1;
    const int t = threadIdx.x >> 1;
    CP* xl = reinterpret_cast<CP*>(stage + Cfg::GROUP) + p * Cfg::XHALF;
    uint64_t* full = reinterpret_cast<uint64_t*>(reinterpret_cast<CP*>(stage + Cfg::GROUP) + 2 * Cfg::XHALF);
    const float2* tw = a.tw;
    const SyncBlock sync{};

    auto issue_load = [&](int k) {
        const int g = blockIdx.x + k * gridDim.x;
        const int x = (g % GPI) * 4, y = (g / GPI) * N;
        tc::mbar_arrive_expect_tx(full, BYTES);
#pragma unroll 1
        for (int q = 0; q < Cfg::BOXES; ++q) tc::tma_load_2d(stage + q * 1024, &map, full, x, y + q * 256);
    };
    const int mine = groups > (int)blockIdx.x ? (groups - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        tc::mbar_init(full, 1);
        tc::fence_mbar_init();
        tc::prefetch_tmap(&map);
        if (mine > 0) issue_load(0);
    }
    __syncthreads();
    bool ok = true;
    for (int k = 0; k < mine; ++k) {
        const int g = blockIdx.x + k * gridDim.x;
        const int b = g / GPI, col = (g % GPI) * 4 + 2 * p;
        if (ok) ok = tc::mbar_wait(full, k & 1, a.err, 10);
        const float4* src = reinterpret_cast<const float4*>(stage);
        CP v[16];
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            const float4 q = src[(t + s * Cfg::TPL) * 2 + p];   // (re_A, im_A, re_B, im_B)
            v[s] = CP{pk::pack(q.x, q.z), pk::pack(q.y, q.w)};
        }
        if (threadIdx.x == 0) tc::bulk_wait_read<0>();      // previous group's second half stored
        __syncthreads();                                    // staging emptied; exchange region free
        if (threadIdx.x == 0 && k + 1 < mine) issue_load(k + 1);
        if (a.flags & CF_FWD) pk::line_fft2<N, false, true>(v, xl, t, tw, sync);
        if (a.flags & CF_TABLE) {
            const float2* ty = a.tab_y + (size_t)b * N;
#pragma unroll
            for (int s = 0; s < 16; ++s) {
                const float2 h = ty[t + s * Cfg::TPL];
                v[s] = pk::cmul_b<false>(v[s], pk::pack(h.x, h.x), pk::pack(h.y, h.y));
            }
        }
        if (a.flags & CF_INV) pk::line_fft2<N, true, true>(v, xl, t, tw, sync);
        if (a.flags & CF_TABLE) {
            const float2 ha = a.tab_x[(size_t)b * N + col], hb = a.tab_x[(size_t)b * N + col + 1];
            const pk::u64 hr = pk::pack(ha.x, hb.x), hi = pk::pack(ha.y, hb.y);
#pragma unroll
            for (int s = 0; s < 16; ++s)
                v[s] = CP{pk::sub2(pk::mul2(v[s].re, hr), pk::mul2(v[s].im, hi)),
                          pk::fma2(v[s].re, hi, pk::mul2(v[s].im, hr))};
        }
        // results leave by TMA in two halves of N/2 rows through the exchange region (slots
        // 0..7 are rows 0..N/2-1), so that no warp waits on global stores
        float4* obuf = reinterpret_cast<float4*>(stage + Cfg::GROUP);
        const int x = (g % GPI) * 4, y = b * N;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                float4 q;
                pk::unpack(v[8 * h + s].re, q.x, q.z);
                pk::unpack(v[8 * h + s].im, q.y, q.w);
                obuf[(t + s * Cfg::TPL) * 2 + p] = q;
            }
            tc::fence_proxy_async();
            __syncthreads();
            if (threadIdx.x == 0) {
#pragma unroll 1
                for (int q = 0; q < Cfg::BOXES / 2; ++q)
                    tc::tma_store_2d(&map, obuf + q * 512, x, y + h * (N / 2) + q * 256);
                tc::bulk_commit();
                if (h == 0) tc::bulk_wait_read<0>();     // first half read out before the second is written
            }
            if (h == 0) __syncthreads();
        }
    }
    if (threadIdx.x == 0) tc::bulk_wait<0>();
}

template <int N, int U, int S> struct URowCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int UT = TPL;                     // one row per unit
    static constexpr int THREADS = UT * U;
    static constexpr int STRIDE = LineGeom<N>::STRIDE; // exchange buffer; >= N
    static_assert(S >= 1 && U % S == 0 && U <= 15, "unit layout");
    template <typename C> static constexpr size_t smem() {
        return ((size_t)S * N + (size_t)U * STRIDE) * sizeof(C) + 8 * U;
    }
};

template <typename C, int N, int U, int S>
__global__ void __launch_bounds__(URowCfg<N, U, S>::THREADS, 1)
row_pass_units_kernel(const __grid_constant__ RowArgs<C> a, int rows) {
    using Cfg = URowCfg<N, U, S>;
    constexpr uint32_t BYTES = N * sizeof(C);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C* stage = reinterpret_cast<C*>(smem_raw);
    const int u = threadIdx.x / Cfg::UT;
    const int t = threadIdx.x % Cfg::UT;
    C* region = stage + S * N + u * Cfg::STRIDE;
    uint64_t* full = reinterpret_cast<uint64_t*>(stage + S * N + U * Cfg::STRIDE);
    const SyncNamed sync{1 + u, Cfg::UT};
    const bool leader = t == 0;
    const bool load = !(a.flags & RF_INIT_ONE);

    auto issue_load = [&](int k) {
        const int g = blockIdx.x + k * gridDim.x;
        uint64_t* bar = &full[k % U];
        tc::mbar_arrive_expect_tx(bar, BYTES);
        tc::bulk_load(stage + (k % S) * N, a.in + (size_t)g * N, BYTES, bar);
    };
    const int mine = rows > (int)blockIdx.x ? (rows - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < U; ++i) tc::mbar_init(&full[i], 1);
        tc::fence_mbar_init();
        if (load)
            for (int k = 0; k < S && k < mine; ++k) issue_load(k);
    }
    __syncthreads();
    bool ok = true;
    int j = 0;
    for (int k = u; k < mine; k += U, ++j) {
        const int g = blockIdx.x + k * gridDim.x;      // global row index over the batch
        const int b = g / N, y = g % N;
        C v[16];
        if (load) {
            const C* src = stage + (k % S) * N;
            if (ok) ok = tc::mbar_wait(&full[u], j & 1, a.err, 8);
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = src[t + s * Cfg::TPL];
        } else {
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = mk<C>(1, 0);
        }
        if (leader) tc::bulk_wait_read<0>();           // this unit's previous store has left its region
        sync();
        if (load && leader && k + S < mine) issue_load(k + S);
        if (a.flags & RF_INV_FIRST) line_fft<C, N, true>(v, region, t, a.tw, sync);
        if (a.elems.count) {
            float none[16];
            apply_elems<C, N, Cfg::TPL>(v, t, y, b, a.elems, none, -1);
        }
        if (a.flags & RF_FWD_AFTER) line_fft<C, N, false>(v, region, t, a.tw, sync);
#pragma unroll
        for (int s = 0; s < 16; ++s) region[t + s * Cfg::TPL] = v[s];
        tc::fence_proxy_async();
        sync();
        if (leader) {
            tc::bulk_store(a.out + (size_t)g * N, region, BYTES);
            tc::bulk_commit();
        }
    }
    if (leader) tc::bulk_wait<0>();
}

// Row pass on packed row pairs: a unit of N/16 threads transforms rows 2m and 2m + 1 (one
// contiguous bulk copy) at once, lane 0 / lane 1 of every FP32x2 register holding row A / B
// (fft_pair.cuh). Elements are applied per row on the unpacked lanes. Otherwise the unit
// pipeline of row_pass_units_kernel: S staging slots of two rows, U units, each with its own
// named barrier and a shared region that is the exchange buffer and then holds the finished
// pair while its bulk store drains.
template <int N, int U, int S> struct PRowPairCfg {
    static constexpr int TPL = LineGeom<N>::TPL;
    static constexpr int UT = TPL;
    static constexpr int THREADS = UT * U;
    static constexpr int GROUP = 2 * N;                // float2 samples per row pair
    static constexpr int REGION = 2 * LineGeom<N>::STRIDE;   // float2 units (16-byte pair entries)
    static_assert(S >= 1 && U % S == 0 && U <= 15, "unit layout");
    static constexpr size_t smem() { return ((size_t)S * GROUP + (size_t)U * REGION) * 8 + 8 * U; }
};

// TIN: the pair arrives as two columns of the transposed plane in[b][x][y] (TMA boxes of
// 2 x 256 through `map`, as in the column pass) instead of two contiguous rows; in must not
// alias out. Without TIN `map` is unused.
template <int N, int U, int S, bool TIN>
__global__ void __launch_bounds__(PRowPairCfg<N, U, S>::THREADS, 1)
row_pass_pair_kernel(const __grid_constant__ RowArgs<float2> a, const __grid_constant__ CUtensorMap map, int pairs) {
    using Cfg = PRowPairCfg<N, U, S>;
    using pk::CP;
    constexpr uint32_t BYTES = Cfg::GROUP * sizeof(float2);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* stage = reinterpret_cast<float2*>(smem_raw);
    const int u = threadIdx.x / Cfg::UT;
    const int t = threadIdx.x % Cfg::UT;
    float2* region = stage + S * Cfg::GROUP + u * Cfg::REGION;
    CP* xl = reinterpret_cast<CP*>(region);
    uint64_t* full = reinterpret_cast<uint64_t*>(stage + S * Cfg::GROUP + U * Cfg::REGION);
    const SyncNamed sync{1 + u, Cfg::UT};
    const bool leader = t == 0;
    const bool load = !(a.flags & RF_INIT_ONE);

    auto issue_load = [&](int k) {
        const int g = blockIdx.x + k * gridDim.x;
        uint64_t* bar = &full[k % U];
        float2* dst = stage + (k % S) * Cfg::GROUP;
        tc::mbar_arrive_expect_tx(bar, BYTES);
        if constexpr (TIN) {
            const int x = (2 * g) % N, y = ((2 * g) / N) * N;     // first line of the pair, item's rows
#pragma unroll 1
            for (int q = 0; q < N / 256; ++q) tc::tma_load_2d(dst + q * 512, &map, bar, x, y + q * 256);
        } else {
            tc::bulk_load(dst, a.in + (size_t)g * Cfg::GROUP, BYTES, bar);
        }
    };
    const int mine = pairs > (int)blockIdx.x ? (pairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < U; ++i) tc::mbar_init(&full[i], 1);
        tc::fence_mbar_init();
        if constexpr (TIN) tc::prefetch_tmap(&map);
        if (load)
            for (int k = 0; k < S && k < mine; ++k) issue_load(k);
    }
    __syncthreads();
    bool ok = true;
    int j = 0;
    for (int k = u; k < mine; k += U, ++j) {
        const int g = blockIdx.x + k * gridDim.x;       // row pair index over the batch
        const int b = (2 * g) / N, ya = (2 * g) % N;
        CP v[16];
        if (load) {
            const float2* src = stage + (k % S) * Cfg::GROUP;
            if (ok) ok = tc::mbar_wait(&full[u], j & 1, a.err, 11);
            if constexpr (TIN) {
                const float4* src4 = reinterpret_cast<const float4*>(src);
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const float4 q = src4[t + s * Cfg::TPL];   // sample t + s*TPL: (re_A, im_A, re_B, im_B)
                    v[s] = CP{pk::pack(q.x, q.z), pk::pack(q.y, q.w)};
                }
            } else {
#pragma unroll
                for (int s = 0; s < 16; ++s) {
                    const float2 qa = src[t + s * Cfg::TPL], qb = src[N + t + s * Cfg::TPL];
                    v[s] = CP{pk::pack(qa.x, qb.x), pk::pack(qa.y, qb.y)};
                }
            }
        } else {
            const pk::u64 one = pk::pack(1.f, 1.f);
#pragma unroll
            for (int s = 0; s < 16; ++s) v[s] = CP{one, 0ull};
        }
        if (leader) tc::bulk_wait_read<0>();            // this unit's previous store has left its region
        sync();
        if (load && leader && k + S < mine) issue_load(k + S);
        if (a.flags & RF_INV_FIRST) pk::line_fft2<N, true>(v, xl, t, a.tw, sync);
        if (a.elems.count) apply_elems_pair<N, Cfg::TPL>(v, t, ya, b, a.elems);
        if (a.flags & RF_FWD_AFTER) pk::line_fft2<N, false>(v, xl, t, a.tw, sync);
#pragma unroll
        for (int s = 0; s < 16; ++s) {
            float2 qa, qb;
            pk::unpack(v[s].re, qa.x, qb.x);
            pk::unpack(v[s].im, qa.y, qb.y);
            region[t + s * Cfg::TPL] = qa;
            region[N + t + s * Cfg::TPL] = qb;
        }
        tc::fence_proxy_async();
        sync();
        if (leader) {
            tc::bulk_store(a.out + (size_t)g * Cfg::GROUP, region, BYTES);
            tc::bulk_commit();
        }
    }
    if (leader) tc::bulk_wait<0>();
}

// ------------------------------------------------------------------------------ launchers

struct PassLaunch {
    cudaStream_t stream;
    int batch;
    int variant = -1;     // row passes: -1 default, 0 persistent, 1 per group, 2 units, 3 pairs
};

// Implemented per precision in passes_f32.cu / passes_f64.cu.
template <typename C>
cudaError_t launch_row_pass(int n, const RowArgs<C>& a, const PassLaunch& l);
template <typename C>
cudaError_t launch_col_pass(int n, int lines, const ColArgs<C>& a, const PassLaunch& l);
// Column widths per block for n (0 picks the default); -1 selects the persistent TMA kernel.
int col_lines_default(int n, bool dbl);
// Candidate column variants (at most 8) and row variants the plan autotuner times for n
// (complex64).
int col_candidates(int n, int* out);
// Whether the mixed-radix passes take line length n (even, not a power of two, prime factors
// up to 61, two lines in 200 KB of shared memory).
bool mixed_length_ok(int n, bool dbl);
int row_variant_count(int n);
// Row variants the complex64 tuner times (row_variant_count's plus the radix-8 engine); <= 8.
int row_candidates(int n, int* out);
// Radix sequence of a pass's line transforms; returns the number of stages.
int pass_radices(int n, bool row, int variant, int lines, int* out, int max_out);
// The kernels used without tuning (CORO_AUTOTUNE=0, or sizes without candidates).
int row_variant_default(int n);
// The kernel a pass with these settings launches: persistent (1) or not, and its lines.
void describe_pass(int n, bool dbl, bool row, int variant, int lines, int* persistent, int* out_lines);

}  // namespace coro
