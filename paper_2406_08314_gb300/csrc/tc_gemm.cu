// Tensor-core (tcgen05) GEMM for the dense Cholesky-vector contractions of
// the mixed-precision path, in 3xTF32 split precision:
//   C[m][n] = sum_k A[m][k] B[n][k]
//           ~ sum_k (Ahi Bhi + Ahi Blo + Alo Bhi)[m][n][k],  FP32 accumulation,
// with x = hi + lo + O(2^-22 |x|), hi and lo TF32-representable.
//
// sm_103a design: one CTA per 128 x BN output tile; A and B tiles (K-major,
// 128-byte swizzle) stream through a shared-memory ring filled by TMA
// (cp.async.bulk.tensor) and tracked by mbarriers; one thread issues
// tcgen05.mma (kind::tf32) into a TMEM accumulator; tcgen05.commit frees
// ring slots; four warps read the accumulator back with tcgen05.ld. Every
// wait is bounded (about 2 s of wall clock); on expiry the kernel records
// MSD_DEV_ERR_TIMEOUT, drains what it issued and releases its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;
// SPLIT: 3xTF32 (hi/lo operands, three products per K step) or a single
// BF16 product. One k-block is 128 bytes of K per row in both cases
// (32 FP32 or 64 BF16 elements); one MMA covers 32 bytes of K.
template <int BN, bool SPLIT>
struct TcCfg {
    static constexpr int BM = 128;
    static constexpr int BK = SPLIT ? 32 : 64;   // elements per k-block
    static constexpr int NOPS = SPLIT ? 2 : 1;   // hi/lo copies of each operand
    static constexpr int STAGES = SPLIT ? (BN >= 256 ? 2 : 3) : (BN >= 256 ? 4 : 6);
    static constexpr uint32_t A_BYTES = BM * 128;
    static constexpr uint32_t B_BYTES = BN * 128;
    static constexpr uint32_t STAGE_BYTES = NOPS * (A_BYTES + B_BYTES);
    static constexpr uint32_t TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
};

template <int BN, bool SPLIT>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
          const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
          int Mr, int Nc, int K, float* __restrict__ C, long long ldc, long long c_split_stride,
          unsigned* err)
{
    using Cfg = TcCfg<BN, SPLIT>;
    constexpr int BM = Cfg::BM, BK = Cfg::BK, STAGES = Cfg::STAGES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[STAGES];
    __shared__ __align__(8) uint64_t empty_bar[STAGES];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const uint64_t wb = wait_budget(err);
    // k-blocks [kb0, kb1) of this split
    const int nkb_all = K / BK;
    const int kb0 = (int)((long long)nkb_all * blockIdx.z / gridDim.z);
    const int kb1 = (int)((long long)nkb_all * (blockIdx.z + 1) / gridDim.z);
    const int nkb = kb1 - kb0;
    C += (size_t)blockIdx.z * c_split_stride;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&done_bar, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(&tmem_base_sh)), "r"(Cfg::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (kb / STAGES) & 1;
            if (!mbar_wait(&empty_bar[s], ph ^ 1, wb)) { fail = 1; atomicOr(err, MSD_DEV_ERR_TIMEOUT); break; }
            uint8_t* st = smem + (size_t)s * Cfg::STAGE_BYTES;
            mbar_expect_tx(&full_bar[s], Cfg::STAGE_BYTES);
            const int kx = (kb0 + kb) * BK;
            tma_load_2d(st, &ta_hi, &full_bar[s], kx, m0);
            tma_load_2d(st + Cfg::NOPS * Cfg::A_BYTES, &tb_hi, &full_bar[s], kx, n0);
            if (SPLIT) {
                tma_load_2d(st + Cfg::A_BYTES, &ta_lo, &full_bar[s], kx, m0);
                tma_load_2d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, &tb_lo, &full_bar[s], kx, n0);
            }
            issued = kb + 1;
        }
        // the loads issued last must land before the CTA may exit (the MMA
        // warp may have given up on them)
        for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb)
            mbar_drain(&full_bar[kb % STAGES], (kb / STAGES) & 1);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = SPLIT ? idesc_tf32(BM, BN) : idesc_bf16(BM, BN);
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t ph = (kb / STAGES) & 1;
            if (!mbar_wait(&full_bar[s], ph, wb)) { fail = 1; atomicOr(err, MSD_DEV_ERR_TIMEOUT); break; }
            tc_fence_after();
            const uint32_t sa = su32(smem + (size_t)s * Cfg::STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {   // 4 x 32 bytes of K per k-block
                const uint64_t ah = sw128_desc(sa + kk * 32);
                const uint64_t bh = sw128_desc(sa + Cfg::NOPS * Cfg::A_BYTES + kk * 32);
                if (SPLIT) {
                    const uint64_t al = sw128_desc(sa + Cfg::A_BYTES + kk * 32);
                    const uint64_t bl = sw128_desc(sa + 2 * Cfg::A_BYTES + Cfg::B_BYTES + kk * 32);
                    mma_tf32(tmem, ah, bh, idesc, (kb | kk) != 0);
                    mma_tf32(tmem, ah, bl, idesc, 1u);
                    mma_tf32(tmem, al, bh, idesc, 1u);
                } else {
                    mma_bf16(tmem, ah, bh, idesc, (kb | kk) != 0);
                }
            }
            mma_commit(&empty_bar[s]);
        }
        mma_commit(&done_bar);
        // every product issued here completes before TMEM may be freed
        mbar_drain(&done_bar, 0);
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0, wb) ? 1 : 0);
    tc_fence_after();
    if (ok && !fail) {
        const int row = m0 + warp * 32 + lane;
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
            if (row < Mr) {
                float* dst = C + (size_t)row * ldc + n0 + c;
                if (n0 + c + 16 <= Nc && ((uintptr_t)dst & 15) == 0) {
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (n0 + c + i < Nc) dst[i] = v[i];
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(err, MSD_DEV_ERR_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS)
                     : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D tensor [outer][inner] (FP32 or BF16) with row pitch `ld` elements;
// boxes of 128 bytes x box_outer rows with 128-byte swizzle.
}  // namespace

int tc_make_map(CUtensorMap* map, const void* base, int inner, int outer, long long ld, int box_outer, bool bf16,
                int swizzle_bytes)
{
    auto fn = encode_fn();
    if (!fn) return -1;
    if (swizzle_bytes != 128 && swizzle_bytes != 64) return -1;
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(swizzle_bytes / esz), (cuuint32_t)box_outer};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base,
                    dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

int tc_make_map3(CUtensorMap* map, const float* base, int inner, int rows, int batch, int box_rows)
{
    auto fn = encode_fn();
    if (!fn) return -1;
    cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)inner * 4, (cuuint64_t)inner * rows * 4};
    cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}

namespace {

int make_map(CUtensorMap* map, const void* base, int inner, int outer, long long ld, int box_outer, bool bf16)
{
    return tc_make_map(map, base, inner, outer, ld, box_outer, bf16);
}

template <int BN, bool SPLIT>
int launch_bn(const void* a_hi, const void* a_lo, long long lda, const void* b_hi, const void* b_lo, long long ldb,
              int Mr, int Nc, int K, float* C, long long ldc, int splits, long long c_split_stride, unsigned* err,
              cudaStream_t st)
{
    CUtensorMap ah, al, bh, bl;
    if (make_map(&ah, a_hi, K, Mr, lda, 128, !SPLIT) || make_map(&bh, b_hi, K, Nc, ldb, BN, !SPLIT)) return -1;
    if (SPLIT) {
        if (make_map(&al, a_lo, K, Mr, lda, 128, false) || make_map(&bl, b_lo, K, Nc, ldb, BN, false)) return -1;
    } else {
        al = ah;
        bl = bh;
    }
    using Cfg = TcCfg<BN, SPLIT>;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_tc_gemm<BN, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Cfg::SMEM) != cudaSuccess)
            return -1;
        attr = true;
    }
    dim3 grid((Nc + BN - 1) / BN, (Mr + 127) / 128, splits);
    k_tc_gemm<BN, SPLIT><<<grid, 128, Cfg::SMEM, st>>>(ah, al, bh, bl, Mr, Nc, K, C, ldc, c_split_stride, err);
    msd_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// TF32 rounding (round to nearest, ties away from zero) of an FP32 value.
__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void split3(double x, float& hi, float& lo)
{
    hi = to_tf32((float)x);
    lo = to_tf32((float)(x - (double)hi));
}

// Rows of a complex FP64 matrix src[b][r][.] (b < nb, r < R) gathered at
// columns cols[0..Kg) (all of [0, Kg) when cols is NULL) -> real rows
// [(b, c, r)][Kp] (c = 0 real, 1 imaginary part), TF32 hi/lo, zero padded.
// Part c of block b starts at row (2b + c) PR (PR >= R; rows r >= R zero).
__global__ void k_split_complex_rows(int nb, int R, int PR, int Kg, int Kp, const double2* __restrict__ src,
                                     long long src_ld, const int* __restrict__ cols, float* __restrict__ hi,
                                     float* __restrict__ lo, int eye0)
{
    const long long total = (long long)nb * 2 * PR * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % Kp);
        const long long row = e / Kp;
        const int r = (int)(row % PR);
        const int c = (int)((row / PR) % 2);
        const long long b = row / (2 * PR);
        double x = 0;
        if (k < Kg && r < R) {
            const double2 v = src[(b * R + r) * src_ld + (cols ? cols[k] : k)];
            x = c ? v.y : v.x;
        } else if (eye0 >= 0 && k >= eye0 && k < eye0 + 2 * PR && c == 0 && r < R && (k - eye0) % PR == r) {
            x = 1.0;
        }
        float h, l;
        split3(x, h, l);
        hi[e] = h;
        lo[e] = l;
    }
}

// Real FP64 rows src[r][.] gathered at cols[0..Kg) -> [R][Kp] hi/lo.
__global__ void k_split_real_rows(long long R, int Kg, int Kp, const double* __restrict__ src, long long src_ld,
                                  const int* __restrict__ cols, float* __restrict__ hi, float* __restrict__ lo)
{
    const long long total = R * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e % Kp);
        const long long r = e / Kp;
        const double x = k < Kg ? src[r * src_ld + (cols ? cols[k] : k)] : 0.0;
        float h, l;
        split3(x, h, l);
        hi[e] = h;
        lo[e] = l;
    }
}

__global__ void k_split_blocks(long long R, int n, int RB, int ld, int k0, const double* __restrict__ x,
                               float* __restrict__ hi, float* __restrict__ lo)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < R * n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / n;
        const int j = (int)(e - r * n);
        double v = x[e];
        const float h = to_tf32((float)v);
        v -= (double)h;
        const float m = to_tf32((float)v);
        v -= (double)m;
        const float q = to_tf32((float)v);
        v -= (double)q;
        const float s = to_tf32((float)v);
        float* ph = hi + r * ld + k0 + j;
        float* pl = lo + r * ld + k0 + j;
        ph[0] = h;
        pl[0] = m;
        ph[RB] = q;
        pl[RB] = s;
    }
}

// out[w][n] = add[n] + sum_z (C_z[2w][n], C_z[2w+1][n]) over the K splits, FP64.
__global__ void k_pack_complex(int nw, int n, const float* __restrict__ C, long long ldc, int splits,
                               long long split_stride, const double* __restrict__ add,
                               double2* __restrict__ out, long long ldo)
{
    const long long total = (long long)nw * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long w = e / n;
        const int j = (int)(e % n);
        double re = add ? add[j] : 0.0, im = 0.0;
        for (int z = 0; z < splits; ++z) {
            re += C[z * split_stride + (2 * w) * ldc + j];
            im += C[z * split_stride + (2 * w + 1) * ldc + j];
        }
        out[w * ldo + j] = make_double2(re, im);
    }
}

int grid_for(long long n)
{
    const long long cap = 16ll * msd_sm_count();
    return (int)((n + 255) / 256 < cap ? (n + 255) / 256 : cap);
}

}  // namespace

int tc_gemm_3xtf32(const TcOperand& A, const TcOperand& B, int Mr, int Nc, int K, float* C, long long ldc,
                   unsigned* err, cudaStream_t st, int splits, long long c_split_stride, int bn)
{
    if (K <= 0 || K % 32 || A.ld % 4 || B.ld % 4 || Mr <= 0 || Nc <= 0) return -1;
    if (splits < 1 || splits > K / 32) return -1;
    if (bn == 0) bn = Nc >= 256 ? 256 : 128;
    if (bn == 256)
        return launch_bn<256, true>(A.hi, A.lo, A.ld, B.hi, B.lo, B.ld, Mr, Nc, K, C, ldc, splits, c_split_stride,
                                    err, st);
    if (bn == 128)
        return launch_bn<128, true>(A.hi, A.lo, A.ld, B.hi, B.lo, B.ld, Mr, Nc, K, C, ldc, splits, c_split_stride,
                                    err, st);
    return -1;
}

int tc_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, int Mr, int Nc, int K, float* C,
                 long long ldc, unsigned* err, cudaStream_t st)
{
    if (K <= 0 || K % 64 || lda % 8 || ldb % 8 || Mr <= 0 || Nc <= 0) return -1;
    if (Nc > 128) return launch_bn<256, false>(A, nullptr, lda, B, nullptr, ldb, Mr, Nc, K, C, ldc, 1, 0, err, st);
    return launch_bn<128, false>(A, nullptr, lda, B, nullptr, ldb, Mr, Nc, K, C, ldc, 1, 0, err, st);
}

void launch_split_complex_rows(int nb, int R, int Kg, int Kp, const double2* src, long long src_ld,
                               const int* cols, float* hi, float* lo, cudaStream_t st, int part_rows, int eye0)
{
    const int PR = part_rows > R ? part_rows : R;
    if ((long long)nb * R * Kp <= 0) return;
    k_split_complex_rows<<<grid_for((long long)nb * 2 * PR * Kp), 256, 0, st>>>(nb, R, PR, Kg, Kp, src, src_ld,
                                                                                 cols, hi, lo, eye0);
    msd_note_launch();
}

void launch_split_blocks(long long R, int n, int RB, int ld, int k0, const double* x, float* hi, float* lo,
                         cudaStream_t st)
{
    if (R * n <= 0) return;
    k_split_blocks<<<grid_for(R * n), 256, 0, st>>>(R, n, RB, ld, k0, x, hi, lo);
    msd_note_launch();
}

void launch_split_real_rows(long long R, int Kg, int Kp, const double* src, long long src_ld, const int* cols,
                            float* hi, float* lo, cudaStream_t st)
{
    if (R * Kp <= 0) return;
    k_split_real_rows<<<grid_for(R * Kp), 256, 0, st>>>(R, Kg, Kp, src, src_ld, cols, hi, lo);
    msd_note_launch();
}

void launch_pack_complex(int nw, int n, const float* C, long long ldc, int splits, long long split_stride,
                         const double* add, double2* out, long long ldo, cudaStream_t st)
{
    if ((long long)nw * n <= 0) return;
    k_pack_complex<<<grid_for((long long)nw * n), 256, 0, st>>>(nw, n, C, ldc, splits, split_stride, add, out, ldo);
    msd_note_launch();
}
