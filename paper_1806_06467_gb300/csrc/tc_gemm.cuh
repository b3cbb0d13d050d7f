// tc_gemm.cuh -- split-precision complex GEMM on the 5th-generation tensor cores.
//
// Computes, for every batch item b,
//     Y[m][n] = sum_k X[m][k] W[n][k]                     (complex, FP32 accumulate)
// from "planar split" operands: a complex matrix Z is stored as four real planes
// [hi_re, hi_im, lo_re, lo_im], hi = round(Z) to TF32 or BF16, lo = round(Z - hi). The product
// keeps the three leading terms hi.hi + hi.lo + lo.hi; each is four real products
// (re.re - im.im, re.im + im.re), the minus sign taken by the A-negate bit of the MMA.
//
// One CTA owns a 128 x 128 complex output tile: two 128x128 FP32 accumulators in TMEM
// (real at columns 0-127, imaginary at 128-255). Warp 0 streams 64-byte-wide K slices of all
// four planes of X and W through a 3-stage shared-memory ring with one 4-D TMA per operand;
// warp 1 issues tcgen05.mma (24 per slice); warps 2-17 drain TMEM and run the epilogue, which
// always writes the TRANSPOSED tile (Y^T), so that chained GEMMs X.W^T then (X.W^T)^T.W^T
// realise A . E . A^T without any separate transpose.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

namespace coro {

enum TcEpi : int {
    TC_EPI_C64T = 0,       // complex64 Y^T * scale
    TC_EPI_SPLITT = 1,     // planar split of (Y^T * scale * mask) -> operand of the next GEMM
    TC_EPI_BABINET = 2,    // dst planes hold E_A; overwritten in place by (E_A - Y^T scale) * mask
    TC_EPI_INTENSITY = 3   // |Y^T * scale|^2 * inv_peak -> float image, dark-hole sum, peak
};

// Per-item geometry and epilogue constants.
struct TcItem {
    int M, N, K;           // complex: rows of X (and of Y), rows of W, inner length
    int x_idx, w_idx;      // batch coordinate of X and of W inside their tensor maps
    int mask_lo, mask_hi;  // epilogue keeps samples with mask_lo <= r^2 <= mask_hi (integer px^2)
    float scale;           // multiplies Y
    float inv_peak;        // intensity normalisation
    // Known support of X: X[m][k] = 0 unless (k - K/2)^2 + kdy (m - M/2)^2 <= kr2 (kdy = 1:
    // a disk, 0: a band of columns); kr2 < 0: no known zeros. Each tile then runs only the K
    // slices that can hold non-zeros (none if its rows hold none); the result is unchanged.
    int kr2 = -1, kdy = 0;
    // The extended-precision GEMM (tcx_gemm.cu) scales and normalises in FP64-class arithmetic
    // (two-float products): its scale and 1/peak are taken from these, not from the floats.
    double scale64 = 1.0, inv_peak64 = 1.0;
};

struct TcArgs {
    const TcItem* items;
    int* err;                        // nonzero after a bounded wait expired
    void* dst;                       // split planes [b][4][dst_rows][dst_ld] or complex64/float [b][dst_rows][dst_ld]
    long long dst_bstride;           // elements per item
    int dst_rows, dst_ld;
    float2* c64;                     // optional complex64 copy [b][rows][c64_ld]
    long long c64_bstride;
    int c64_ld;
    double* dh_acc;                  // dark-hole sums [b] (intensity epilogue)
    float* peak;                     // running max of the intensity [b] (intensity epilogue), or NULL
    int c64_seed;                    // intensity epilogue: c64 receives mask . E * inv_peak instead of E
    const float2* src64;             // Babinet epilogue: E_A read from this complex64 array
    long long src64_bstride;         //   [b][rows][src64_ld] (NULL: from the split planes in dst)
    int src64_ld;
    double* peak64;                  // extended-precision intensity epilogue: running max [b] (or NULL)
};

__host__ __device__ inline int isqrt_floor(long long v) {
    long long w = (long long)sqrt((double)v);
    while (w * w > v) --w;
    while ((w + 1) * (w + 1) <= v) ++w;
    return (int)w;
}

// Distance from c to the nearest of the integers lo..hi (0 if c lies inside).
__host__ __device__ inline int dist_to_range(int c, int lo, int hi) { return c < lo ? lo - c : c > hi ? c - hi : 0; }

// K slices of KE elements [kb0, kb0 + kblocks) a BM x BN tile (rows m0.., columns n0..) has to run: those that can
// hold non-zeros of X's known support, none when a masking epilogue zeroes every output of
// the tile. Shared by the kernel and the host-side flop count.
template <int BM, int BN>
__host__ __device__ inline void tile_k_range(const TcItem& it, int m0, int n0, int KE, bool masked, int& kb0,
                                             int& kblocks) {
    const int mhi = (m0 + BM < it.M ? m0 + BM : it.M) - 1, nhi = (n0 + BN < it.N ? n0 + BN : it.N) - 1;
    if (masked && (it.mask_lo > 0 || it.mask_hi < 0x7fffffff)) {
        const long long dx0 = dist_to_range(it.M / 2, m0, mhi), dy0 = dist_to_range(it.N / 2, n0, nhi);
        const long long dx1 = (it.M / 2 - m0 > mhi - it.M / 2) ? it.M / 2 - m0 : mhi - it.M / 2;
        const long long dy1 = (it.N / 2 - n0 > nhi - it.N / 2) ? it.N / 2 - n0 : nhi - it.N / 2;
        const long long r2min = dx0 * dx0 + dy0 * dy0, r2max = dx1 * dx1 + dy1 * dy1;
        if (r2min > it.mask_hi || r2max < it.mask_lo) { kb0 = 0; kblocks = 0; return; }
    }
    if (it.kr2 < 0) return;
    const long long dm = dist_to_range(it.M / 2, m0, mhi);
    const long long rem = (long long)it.kr2 - (long long)it.kdy * dm * dm;
    if (rem < 0) { kb0 = 0; kblocks = 0; return; }
    const int w = isqrt_floor(rem);
    const int klo = it.K / 2 - w < 0 ? 0 : it.K / 2 - w;
    const int khi = it.K / 2 + w > it.K - 1 ? it.K - 1 : it.K / 2 + w;
    if (khi < klo) { kb0 = 0; kblocks = 0; return; }
    kb0 = klo / KE;
    kblocks = khi / KE - kb0 + 1;
}


// Host side (tc_gemm.cu).
struct TcOperand {                   // a planar split operand in global memory
    void* base;                      // [batch][4][rows][ld] elements (float or bf16)
    int batch, rows, cols, ld;       // cols = valid K extent (complex), ld >= cols, 16-byte rows
};

cudaError_t tc_make_operand_map(const TcOperand& op, bool bf16, CUtensorMap* map);
// Tensor work of one tc_launch over host copies of its items: *useful = 24 flops (three split
// products of a complex multiply-add) per valid output per K element inside the known support,
// *issued = the same for every 128 x 128 tile and K slice the kernel runs. Added to the outputs.
void tc_count_flops(bool bf16, int epi, const TcItem* items, int batch, int max_m, int max_n, double* useful,
                    double* issued);
// A field of 8-byte samples [rows_total][n] as a 2-D tensor map with boxes of box_cols x box_rows.
cudaError_t tc_make_field_map(const void* base, int n, long long rows_total, int box_cols, CUtensorMap* map,
                              int box_rows = 256);
cudaError_t tc_launch(bool bf16, int epi, const CUtensorMap& mx, const CUtensorMap& mw, int max_m, int max_n,
                      int max_k, int batch, const TcArgs& args, cudaStream_t stream);

// complex64 [batch][rows][cols] (leading dimension src_ld) -> planar split operand; with
// keep_r2 (device [batch]) samples whose centred (row, col) radius^2 exceeds keep_r2[b] become 0
cudaError_t tc_split(bool bf16, const float2* src, long long src_bstride, int src_ld, const TcOperand& dst,
                     cudaStream_t stream, const int* keep_r2 = nullptr);
// W[r][k] for one basis (index `item` of dst), rows_valid x cols_valid centred on their own
// halves; everything else in that item's planes is left untouched
cudaError_t tc_basis_one(bool bf16, double c, int sign, const TcOperand& dst, int item, int rows_valid,
                         int cols_valid, cudaStream_t stream);
// W[r][k] = exp(sign 2 pi i (r - rows/2)(k - cols/2) c[b]) straight into planar split form
cudaError_t tc_basis(bool bf16, const double* c, int sign, const TcOperand& dst, cudaStream_t stream);
// planar split operand -> complex64 (hi + lo), dst[b * dst_bstride + r * dst_ld + k]
cudaError_t tc_merge(bool bf16, const TcOperand& src, float2* dst, long long dst_bstride, int dst_ld,
                     cudaStream_t stream);

inline size_t tc_elem_size(bool bf16) { return bf16 ? 2 : 4; }
inline int tc_ld(int cols, bool bf16) {          // 16-byte rows, at least 64 bytes
    const int q = bf16 ? 8 : 4;
    int ld = (cols + q - 1) / q * q;
    const int mn = bf16 ? 32 : 16;
    return ld < mn ? mn : ld;
}

}  // namespace coro
