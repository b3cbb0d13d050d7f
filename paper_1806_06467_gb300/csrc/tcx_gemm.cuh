// tcx_gemm.cuh -- extended-precision complex GEMM on the tensor cores: exact BF16 slices.
//
// Y[m][n] = sum_k X[m][k] W[n][k] (complex), accurate to about 2^-32 of the operands' local
// magnitude, built from BF16 tensor-core products that the hardware sums EXACTLY.
//
// Operand format ("sliced"): every complex value v of a row is written as four BF16 slices per
// real component, v = s0 + s1 + s2 + s3 with s_i = a_i 2^(e - 8(i+1)), a_i an integer, |a_0| <=
// 256, |a_i| <= 128 for i >= 1, and 2^e a power of two no smaller than max(|Re|, |Im|) over the
// value's group of 64 consecutive K elements of its row (groups aligned at K = 0, 64, ...).
// Four slices carry 32 bits below the group's largest value.
//
// Why it is exact: with both operands in this form, every product s_i(X) s_j(W) inside one
// group is an integer multiple of 2^(eX + eW - 8(i+j+2)), at most 2^16 such units for i = j = 0.
// A complex real part sums 2 x 64 of them per group: at most 2^23 units, so the FP32 tensor-core
// accumulator holds the level-0 (i = j = 0) group sum exactly, whatever order or truncation it
// uses inside. The level-1..3 products (i + j = 1..3; the terms i + j >= 4 fall below 2^-32 and
// are dropped) go to a second accumulator; they are 2^-8 smaller, so its FP32 rounding sits near
// 2^-32 of the group's magnitude. After every group the epilogue drains both into a two-float
// (hi, lo) pair per output: hi + level-0 by an error-free two-sum, the error and the level-1..3
// sum into lo. The epilogues then scale, subtract (Babinet) and square in two-float arithmetic.
//
// Storage: X-type operands [batch][8][rows][ld] BF16, plane 2i + c (slice i, c = 0 real / 1
// imaginary); W-type operands (the MFT bases) [batch][12][rows][ld], plane 3i + {0: -imag,
// 1: real, 2: imag}, so that [real; imag] and [-imag; real] are adjacent planes: one MMA with
// N = 128 over planes (3i+1, 3i+2) gives Re and Im contributions of a real X slice at once, and
// over (3i, 3i+1) those of an imaginary X slice. ld >= cols, a multiple of 16 elements.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "tc_gemm.cuh"

namespace coro {

constexpr int TCX_X_PLANES = 8;
constexpr int TCX_W_PLANES = 12;

inline int tcx_ld(int cols) { return (cols + 15) / 16 * 16 < 32 ? 32 : (cols + 15) / 16 * 16; }

// Output tile: 128 rows x tile_n complex columns, tile_n = 64 or 32 (TCX_TILE_N* below). The W
// map's boxes have tile_n rows, so a map serves launches of its own tile width only.
constexpr int TCX_TILE_N_WIDE = 64;
constexpr int TCX_TILE_N_NARROW = 32;

// Tensor maps of sliced operands (X: 128-row boxes, W: tile_n-row boxes; 32-byte K rows).
cudaError_t tcx_make_x_map(const TcOperand& op, CUtensorMap* map);
cudaError_t tcx_make_w_map(const TcOperand& op, CUtensorMap* map, int tile_n = TCX_TILE_N_WIDE);

// Same item and argument structs as tc_launch; the epilogues read scale64 / inv_peak64 and,
// for the intensity epilogue, keep the running peak in args.peak64 (double [b]). The
// destination of TC_EPI_SPLITT and TC_EPI_BABINET is a sliced X-type operand.
cudaError_t tcx_launch(int epi, const CUtensorMap& mx, const CUtensorMap& mw, int max_m, int max_n, int batch,
                       const TcArgs& args, cudaStream_t stream, int tile_n = TCX_TILE_N_WIDE);
void tcx_count_flops(int epi, const TcItem* items, int batch, int max_m, int max_n, double* useful, double* issued,
                     int tile_n = TCX_TILE_N_WIDE);

// complex64 [batch][rows][cols] (leading dimension src_ld) -> sliced X-type operand (keep_r2 as tc_split)
cudaError_t tcx_split(const float2* src, long long src_bstride, int src_ld, const TcOperand& dst,
                      cudaStream_t stream, const int* keep_r2 = nullptr);
// sliced W-type basis item: W[r][k] = exp(sign 2 pi i (r - rows_valid/2)(k - cols_valid/2) c)
cudaError_t tcx_basis_one(double c, int sign, const TcOperand& dst, int item, int rows_valid, int cols_valid,
                          cudaStream_t stream);
// sliced X-type operand -> complex64 (sum of the slices, rounded once)
cudaError_t tcx_merge(const TcOperand& src, float2* dst, long long dst_bstride, int dst_ld, cudaStream_t stream);

}  // namespace coro
