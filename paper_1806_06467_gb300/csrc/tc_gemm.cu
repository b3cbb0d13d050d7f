// tc_gemm.cu -- tcgen05 split-precision complex GEMM, its operand producers and launcher.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cudaTypedefs.h>

#include <mutex>

#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace coro {
namespace {

constexpr int BM = 128;                  // rows of X per tile (UMMA M)
constexpr int BN = 128;                  // rows of W per tile (UMMA N), complex outputs
constexpr int STAGES = 3;
constexpr int PLANE_BYTES = 128 * 64;    // 128 rows x 64-byte K slice
constexpr int OPER_BYTES = 4 * PLANE_BYTES;
constexpr int STAGE_BYTES = 2 * OPER_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int EPI_WARPS = 16;            // four per TMEM lane quarter, 32 output columns each
constexpr int EPI_COLS = 128 * 4 / EPI_WARPS;  // output columns per epilogue warp
constexpr int THREADS = 64 + 32 * EPI_WARPS;   // warp 0 TMA, warp 1 MMA, warps 2.. epilogue
constexpr uint32_t TMEM_COLS = 512;      // two accumulator buffers of (128 re + 128 im) columns
constexpr int kChunk = 1;                // K slices summed inside one tensor-core accumulator

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Split (re, im) into hi/lo and store the four planes at element offset `off`.
template <bool BF16>
__device__ __forceinline__ void store_split(void* base, size_t plane, size_t off, float re, float im) {
    if constexpr (BF16) {
        __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(base);
        const __nv_bfloat16 hr = __float2bfloat16_rn(re), hi = __float2bfloat16_rn(im);
        p[off] = hr;
        p[plane + off] = hi;
        p[2 * plane + off] = __float2bfloat16_rn(re - __bfloat162float(hr));
        p[3 * plane + off] = __float2bfloat16_rn(im - __bfloat162float(hi));
    } else {
        float* p = reinterpret_cast<float*>(base);
        const float hr = tf32_rna(re), hi = tf32_rna(im);
        p[off] = hr;
        p[plane + off] = hi;
        p[2 * plane + off] = tf32_rna(re - hr);
        p[3 * plane + off] = tf32_rna(im - hi);
    }
}

template <bool BF16>
__device__ __forceinline__ float2 load_split(const void* base, size_t plane, size_t off) {
    if constexpr (BF16) {
        const __nv_bfloat16* p = reinterpret_cast<const __nv_bfloat16*>(base);
        return make_float2(__bfloat162float(p[off]) + __bfloat162float(p[2 * plane + off]),
                           __bfloat162float(p[plane + off]) + __bfloat162float(p[3 * plane + off]));
    } else {
        const float* p = reinterpret_cast<const float*>(base);
        return make_float2(p[off] + p[2 * plane + off], p[plane + off] + p[3 * plane + off]);
    }
}

template <bool BF16, int EPI>
__global__ void __launch_bounds__(THREADS, 1)
tc_cgemm_kernel(const __grid_constant__ CUtensorMap mx, const __grid_constant__ CUtensorMap mw, const TcArgs a) {
    const int b = blockIdx.z;
    const TcItem it = a.items[b];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    if (m0 >= it.M || n0 >= it.N) return;            // uniform: uneven items skip empty tiles

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;                // accumulator buffer b holds a finished chunk
    uint64_t* tempty = tfull + 2;                    // accumulator buffer b has been drained
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KE = BF16 ? 32 : 16;               // real elements per 64-byte K slice
    int kb0 = 0, kblocks = (it.K + KE - 1) / KE;
    tile_k_range<BM, BN>(it, m0, n0, KE, EPI == TC_EPI_SPLITT || EPI == TC_EPI_BABINET, kb0, kblocks);
    const int nchunks = (kblocks + kChunk - 1) / kChunk;

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
            for (int k = 0; k < kblocks; ++k) {
                const int s = k % STAGES;
                const uint32_t ph = (k / STAGES) & 1;
                if (!tc::mbar_wait(&empty[s], ph ^ 1, a.err, 1)) break;
                unsigned char* st = smem + s * STAGE_BYTES;
                tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                tc::tma_load_4d(st, &mx, &full[s], (kb0 + k) * KE, m0, 0, it.x_idx);
                tc::tma_load_4d(st + OPER_BYTES, &mw, &full[s], (kb0 + k) * KE, n0, 0, it.w_idx);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // Each chunk of kChunk slices starts a fresh accumulator in one of two TMEM
            // buffers; the epilogue warps add finished chunks into FP32 registers with
            // round-to-nearest, so the tensor-core accumulator never sums more than a chunk.
            constexpr uint32_t ID_POS = tc::idesc<BF16>(BM, BN, false);
            constexpr uint32_t ID_NEG = tc::idesc<BF16>(BM, BN, true);
            bool ok = true;
            for (int k = 0; k < kblocks && ok; ++k) {
                const int s = k % STAGES;
                const uint32_t ph = (k / STAGES) & 1;
                const int c = k / kChunk, buf = c & 1, kc = k % kChunk;
                if (kc == 0) {
                    if (!(ok = tc::mbar_wait(&tempty[buf], ((c >> 1) & 1) ^ 1, a.err, 4))) break;
                    tc::tc_fence_after();
                }
                if (!(ok = tc::mbar_wait(&full[s], ph, a.err, 2))) break;
                tc::tc_fence_after();
                const uint32_t d_re = tbase + buf * 256, d_im = d_re + 128;
                const uint32_t xa = tc::smem_u32(smem + s * STAGE_BYTES);
                const uint32_t wa = xa + OPER_BYTES;
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {           // two MMA K-steps of 32 bytes per slice
#pragma unroll
                    for (int t = 0; t < 3; ++t) {          // hi.hi, hi.lo, lo.hi
                        const int xs = (t == 2) ? 1 : 0, ws = (t == 1) ? 1 : 0;
                        const uint64_t ar = tc::sdesc_sw64(xa + (2 * xs + 0) * PLANE_BYTES + kk * 32);
                        const uint64_t ai = tc::sdesc_sw64(xa + (2 * xs + 1) * PLANE_BYTES + kk * 32);
                        const uint64_t br = tc::sdesc_sw64(wa + (2 * ws + 0) * PLANE_BYTES + kk * 32);
                        const uint64_t bi = tc::sdesc_sw64(wa + (2 * ws + 1) * PLANE_BYTES + kk * 32);
                        const uint32_t acc = (kc | kk | t) ? 1u : 0u;
                        tc::umma<BF16>(d_re, ar, br, ID_POS, acc);
                        tc::umma<BF16>(d_re, ai, bi, ID_NEG, 1u);
                        tc::umma<BF16>(d_im, ar, bi, ID_POS, acc);
                        tc::umma<BF16>(d_im, ai, br, ID_POS, 1u);
                    }
                }
                tc::umma_commit(&empty[s]);             // frees the stage once these MMAs retire
                if (kc == kChunk - 1 || k == kblocks - 1) tc::umma_commit(&tfull[buf]);
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue (warps 2..9)
        const int q = warp & 3;                          // TMEM lane quarter this warp may read
        const int half = (warp - 2) >> 2;                // which EPI_COLS-wide group of the 128 output columns
        const int row = q * 32 + lane;
        const int m = m0 + row;
        const uint32_t lane_base = tbase + ((uint32_t)(q * 32) << 16) + half * EPI_COLS;
        float acc_re[EPI_COLS], acc_im[EPI_COLS];
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j) { acc_re[j] = 0.f; acc_im[j] = 0.f; }
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            const int buf = c & 1;
            if (!(ok = tc::mbar_wait(&tfull[buf], (c >> 1) & 1, a.err, 3))) break;
            __syncwarp();
            tc::tc_fence_after();
#pragma unroll
            for (int part = 0; part < EPI_COLS / 16; ++part) {
                uint32_t r[16];
                tc::tmem_ld16(lane_base + buf * 256 + part * 16, r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) acc_re[part * 16 + j] += __uint_as_float(r[j]);
                tc::tmem_ld16(lane_base + buf * 256 + 128 + part * 16, r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 16; ++j) acc_im[part * 16 + j] += __uint_as_float(r[j]);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);
        }
        double dh = 0.0;
        float pk = 0.f;
        if constexpr (EPI == TC_EPI_BABINET) {
            // E_A from the complex64 pupil when given (exact FP32, one 8-byte load), else from
            // its split planes; the reads of four columns are issued before any arithmetic
            if (ok && m < it.M) {
                const int kx = m - it.M / 2;
                const size_t plane = (size_t)a.dst_rows * a.dst_ld;
                constexpr int G = 4;
#pragma unroll
                for (int j0 = 0; j0 < EPI_COLS; j0 += G) {
                    float2 e[G];
                    bool keep[G];
#pragma unroll
                    for (int jj = 0; jj < G; ++jj) {
                        const int n = n0 + half * EPI_COLS + j0 + jj;
                        const int ky = n - it.N / 2;
                        const int r2 = kx * kx + ky * ky;
                        keep[jj] = n < it.N && r2 >= it.mask_lo && r2 <= it.mask_hi;
                        e[jj] = !keep[jj] ? make_float2(0.f, 0.f)
                                : a.src64 ? __ldg(a.src64 + b * a.src64_bstride + (size_t)n * a.src64_ld + m)
                                          : load_split<BF16>(a.dst, plane, b * a.dst_bstride + (size_t)n * a.dst_ld + m);
                    }
#pragma unroll
                    for (int jj = 0; jj < G; ++jj) {
                        const int n = n0 + half * EPI_COLS + j0 + jj;
                        if (n < it.N) {
                            const float re = keep[jj] ? e[jj].x - acc_re[j0 + jj] * it.scale : 0.f;
                            const float im = keep[jj] ? e[jj].y - acc_im[j0 + jj] * it.scale : 0.f;
                            const size_t off = b * a.dst_bstride + (size_t)n * a.dst_ld + m;
                            store_split<BF16>(a.dst, plane, off, re, im);
                            if (a.c64) a.c64[b * a.c64_bstride + (size_t)n * a.c64_ld + m] = make_float2(re, im);
                        }
                    }
                }
            }
        } else if (ok && m < it.M) {
            const int kx = m - it.M / 2;
#pragma unroll
            for (int j = 0; j < EPI_COLS; ++j) {
                const int n = n0 + half * EPI_COLS + j;
                if (n < it.N) {
                    float re = acc_re[j] * it.scale, im = acc_im[j] * it.scale;
                    const int ky = n - it.N / 2;
                    const int r2 = kx * kx + ky * ky;
                    const bool keep = r2 >= it.mask_lo && r2 <= it.mask_hi;
                    if constexpr (EPI == TC_EPI_C64T) {
                        float2* d = reinterpret_cast<float2*>(a.dst) + b * a.dst_bstride + (size_t)n * a.dst_ld + m;
                        *d = make_float2(re, im);
                    } else if constexpr (EPI == TC_EPI_SPLITT) {
                        if (!keep) { re = 0.f; im = 0.f; }
                        const size_t plane = (size_t)a.dst_rows * a.dst_ld;
                        store_split<BF16>(a.dst, plane, b * a.dst_bstride + (size_t)n * a.dst_ld + m, re, im);
                    } else {
                        const float inten = (re * re + im * im) * it.inv_peak;
                        if (a.dst) reinterpret_cast<float*>(a.dst)[b * a.dst_bstride + (size_t)n * a.dst_ld + m] = inten;
                        if (a.c64) {
                            // field, or the gradient seed dS/dconj(E) = mask . E / peak
                            const float2 v = !a.c64_seed ? make_float2(re, im)
                                             : keep ? make_float2(re * it.inv_peak, im * it.inv_peak)
                                                    : make_float2(0.f, 0.f);
                            a.c64[b * a.c64_bstride + (size_t)n * a.c64_ld + m] = v;
                        }
                        if (keep) dh += (double)inten;
                        pk = fmaxf(pk, inten);
                    }
                }
            }
        }
        if constexpr (EPI == TC_EPI_INTENSITY) {
            for (int o = 16; o > 0; o >>= 1) {
                dh += __shfl_down_sync(0xffffffffu, dh, o);
                pk = fmaxf(pk, __shfl_down_sync(0xffffffffu, pk, o));
            }
            if (lane == 0 && dh != 0.0 && a.dh_acc) atomicAdd(a.dh_acc + b, dh);
            // intensities are non-negative, so their IEEE bit patterns order like integers
            if (lane == 0 && a.peak) atomicMax(reinterpret_cast<int*>(a.peak) + b, __float_as_int(pk));
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tbase, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- operand producers

template <bool BF16>
__global__ void split_kernel(const float2* __restrict__ src, long long sb, int sld, void* dst, int rows, int cols,
                             int ld, const int* __restrict__ keep_r2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, b = blockIdx.z;
    if (k >= ld) return;
    float2 v = make_float2(0.f, 0.f);
    if (k < cols) v = src[b * sb + (size_t)r * sld + k];
    if (keep_r2) {
        const int kx = k - cols / 2, ky = r - rows / 2;
        if (kx * kx + ky * ky > keep_r2[b]) v = make_float2(0.f, 0.f);
    }
    const size_t plane = (size_t)rows * ld;
    store_split<BF16>(dst, plane, (size_t)b * 4 * plane + (size_t)r * ld + k, v.x, v.y);
}

// W[r][k] = exp(sign 2 pi i (r - rows/2)(k - cols/2) c_b): FP64 phase reduced to its
// fractional cycle, then rounded to FP32 and split. plane_rows = rows of the operand planes
// (>= rows), item = first item written (grid z offsets from it).
template <bool BF16>
__global__ void basis_kernel(const double* __restrict__ c, double c_one, int sign, void* dst, int rows, int cols,
                             int ld, int plane_rows, int item) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, b = blockIdx.z + item;
    if (k >= ld) return;
    float re = 0.f, im = 0.f;
    if (k < cols) {
        const long long rr = (long long)r - rows / 2, kk = (long long)k - cols / 2;
        double cyc = (double)(rr * kk) * (c ? c[b] : c_one);
        cyc -= rint(cyc);
        double s, co;
        sincospi(2.0 * cyc, &s, &co);
        re = (float)co;
        im = (float)(sign < 0 ? -s : s);
    }
    const size_t plane = (size_t)plane_rows * ld;
    store_split<BF16>(dst, plane, (size_t)b * 4 * plane + (size_t)r * ld + k, re, im);
}

template <bool BF16>
__global__ void merge_kernel(const void* src, int rows, int cols, int ld, float2* dst, long long db, int dld) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y, b = blockIdx.z;
    if (k >= cols) return;
    const size_t plane = (size_t)rows * ld;
    dst[b * db + (size_t)r * dld + k] = load_split<BF16>(src, plane, (size_t)b * 4 * plane + (size_t)r * ld + k);
}

// ---------------------------------------------------------------- driver entry point

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

template <bool BF16, int EPI>
cudaError_t launch_t(const CUtensorMap& mx, const CUtensorMap& mw, int max_m, int max_n, int batch, const TcArgs& args,
                     cudaStream_t stream) {
    static int attr_done = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_done != dev) {
        cudaError_t e = cudaFuncSetAttribute(tc_cgemm_kernel<BF16, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_done = dev;
    }
    dim3 grid((max_n + BN - 1) / BN, (max_m + BM - 1) / BM, batch);
    tc_cgemm_kernel<BF16, EPI><<<grid, THREADS, SMEM_BYTES, stream>>>(mx, mw, args);
    return cudaGetLastError();
}

}  // namespace

// The driver's tensor-map encoder, shared with tcx_gemm.cu.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() { return encode_fn(); }

void tc_count_flops(bool bf16, int epi, const TcItem* items, int batch, int max_m, int max_n, double* useful,
                    double* issued) {
    const int KE = bf16 ? 32 : 16;
    const bool masked = epi == TC_EPI_SPLITT || epi == TC_EPI_BABINET;
    for (int b = 0; b < batch; ++b) {
        const TcItem& it = items[b];
        for (int m0 = 0; m0 < max_m && m0 < it.M; m0 += BM)
            for (int n0 = 0; n0 < max_n && n0 < it.N; n0 += BN) {
                int kb0 = 0, kblocks = (it.K + KE - 1) / KE;
                tile_k_range<BM, BN>(it, m0, n0, KE, masked, kb0, kblocks);
                if (kblocks <= 0) continue;
                const int rows = (m0 + BM < it.M ? BM : it.M - m0), cols = (n0 + BN < it.N ? BN : it.N - n0);
                int klo = 0, khi = it.K - 1;                  // elements inside the support
                if (it.kr2 >= 0) {
                    const long long dm = dist_to_range(it.M / 2, m0, m0 + rows - 1);
                    const int w = isqrt_floor((long long)it.kr2 - (long long)it.kdy * dm * dm);
                    klo = it.K / 2 - w < 0 ? 0 : it.K / 2 - w;
                    khi = it.K / 2 + w > it.K - 1 ? it.K - 1 : it.K / 2 + w;
                }
                *useful += 24.0 * rows * cols * (double)(khi - klo + 1);
                *issued += 24.0 * BM * BN * (double)kblocks * KE;
            }
    }
}

cudaError_t tc_make_operand_map(const TcOperand& op, bool bf16, CUtensorMap* map) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const size_t es = tc_elem_size(bf16);
    if (((uintptr_t)op.base & 15) || (op.ld * es) % 16) return cudaErrorInvalidValue;
    cuuint64_t dims[4] = {(cuuint64_t)op.ld, (cuuint64_t)op.rows, 4, (cuuint64_t)op.batch};
    cuuint64_t strides[3] = {(cuuint64_t)op.ld * es, (cuuint64_t)op.rows * op.ld * es, (cuuint64_t)4 * op.rows * op.ld * es};
    cuuint32_t box[4] = {(cuuint32_t)(64 / es), 128, 4, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, op.base, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_make_field_map(const void* base, int n, long long rows_total, int box_cols, CUtensorMap* map,
                              int box_rows) {
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if (((uintptr_t)base & 15) || box_cols * 8 % 16 || box_rows < 1 || box_rows > 256 || rows_total < box_rows)
        return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows_total};
    cuuint64_t strides[1] = {(cuuint64_t)n * 8};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_launch(bool bf16, int epi, const CUtensorMap& mx, const CUtensorMap& mw, int max_m, int max_n,
                      int max_k, int batch, const TcArgs& args, cudaStream_t stream) {
    (void)max_k;
    if (bf16) {
        switch (epi) {
            case TC_EPI_C64T: return launch_t<true, TC_EPI_C64T>(mx, mw, max_m, max_n, batch, args, stream);
            case TC_EPI_SPLITT: return launch_t<true, TC_EPI_SPLITT>(mx, mw, max_m, max_n, batch, args, stream);
            case TC_EPI_BABINET: return launch_t<true, TC_EPI_BABINET>(mx, mw, max_m, max_n, batch, args, stream);
            case TC_EPI_INTENSITY: return launch_t<true, TC_EPI_INTENSITY>(mx, mw, max_m, max_n, batch, args, stream);
        }
    } else {
        switch (epi) {
            case TC_EPI_C64T: return launch_t<false, TC_EPI_C64T>(mx, mw, max_m, max_n, batch, args, stream);
            case TC_EPI_SPLITT: return launch_t<false, TC_EPI_SPLITT>(mx, mw, max_m, max_n, batch, args, stream);
            case TC_EPI_BABINET: return launch_t<false, TC_EPI_BABINET>(mx, mw, max_m, max_n, batch, args, stream);
            case TC_EPI_INTENSITY: return launch_t<false, TC_EPI_INTENSITY>(mx, mw, max_m, max_n, batch, args, stream);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t tc_split(bool bf16, const float2* src, long long src_bstride, int src_ld, const TcOperand& dst,
                     cudaStream_t stream, const int* keep_r2) {
    dim3 grid((dst.ld + 127) / 128, dst.rows, dst.batch);
    if (bf16) split_kernel<true><<<grid, 128, 0, stream>>>(src, src_bstride, src_ld, dst.base, dst.rows, dst.cols, dst.ld, keep_r2);
    else split_kernel<false><<<grid, 128, 0, stream>>>(src, src_bstride, src_ld, dst.base, dst.rows, dst.cols, dst.ld, keep_r2);
    return cudaGetLastError();
}

cudaError_t tc_basis(bool bf16, const double* c, int sign, const TcOperand& dst, cudaStream_t stream) {
    dim3 grid((dst.ld + 127) / 128, dst.rows, dst.batch);
    if (bf16) basis_kernel<true><<<grid, 128, 0, stream>>>(c, 0.0, sign, dst.base, dst.rows, dst.cols, dst.ld, dst.rows, 0);
    else basis_kernel<false><<<grid, 128, 0, stream>>>(c, 0.0, sign, dst.base, dst.rows, dst.cols, dst.ld, dst.rows, 0);
    return cudaGetLastError();
}

cudaError_t tc_merge(bool bf16, const TcOperand& src, float2* dst, long long dst_bstride, int dst_ld,
                     cudaStream_t stream) {
    dim3 grid((src.cols + 127) / 128, src.rows, src.batch);
    if (bf16) merge_kernel<true><<<grid, 128, 0, stream>>>(src.base, src.rows, src.cols, src.ld, dst, dst_bstride, dst_ld);
    else merge_kernel<false><<<grid, 128, 0, stream>>>(src.base, src.rows, src.cols, src.ld, dst, dst_bstride, dst_ld);
    return cudaGetLastError();
}

cudaError_t tc_basis_one(bool bf16, double c, int sign, const TcOperand& dst, int item, int rows_valid,
                         int cols_valid, cudaStream_t stream) {
    if (rows_valid > dst.rows || cols_valid > dst.ld || item < 0 || item >= dst.batch) return cudaErrorInvalidValue;
    dim3 grid((dst.ld + 127) / 128, rows_valid, 1);
    if (bf16) basis_kernel<true><<<grid, 128, 0, stream>>>(nullptr, c, sign, dst.base, rows_valid, cols_valid, dst.ld, dst.rows, item);
    else basis_kernel<false><<<grid, 128, 0, stream>>>(nullptr, c, sign, dst.base, rows_valid, cols_valid, dst.ld, dst.rows, item);
    return cudaGetLastError();
}

}  // namespace coro
