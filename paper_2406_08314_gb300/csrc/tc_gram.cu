// Gram matrices of the mixed-precision local energy on the tensor cores
// (the Gram form of the generalized Wick terms, Sec. III: fill_os / get_ss
// sum over the Cholesky vectors):
//   K[x][y] = sum_g P_g[x] Q_g[y]   (complex, no conjugation),
// per walker, for (P, Q) = (Lambda^a, Lambda^a), (Lambda^b, Lambda^b) and
// (Lambda^a, Lambda^b).
//
// Two passes. (1) k_gram_transpose writes each spin's Lambda, stored
// [walker][g][x] as FP32 pairs, once as real rows T[w][2x + c][g] (part c of
// entry x), so that the contraction index g is contiguous. (2) k_tc_gram
// reads the rows of P (M-tiles of 128 rows) and Q (one tile of
// N = 2 Xq rounded up to 16 rows) in k-blocks of 32 vectors through a 3-D
// TMA map (one box per walker; rows past 2X read as zero), in a two-stage
// ring. Four warps split each landed block in place into TF32 pieces
// (x = hi + lo + O(2^-22 |x|), round to nearest) and one thread issues
// tcgen05.mma kind::tf32 (hi hi, hi lo, lo hi) into one TMEM accumulator
// per M-tile. The real product C = A B^T over g holds every part
// combination of the complex entries:
//   Re K[x][y] = C[2x][2y] - C[2x+1][2y+1],  Im K[x][y] = C[2x][2y+1] + C[2x+1][2y],
// and the same four warps combine neighbouring rows on the way out. Every
// wait is bounded; on expiry the kernel records MSD_DEV_ERR_TIMEOUT, lets
// its copies and products complete, frees TMEM and returns.
#include <cuda.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int GR_BK = 32;                  // vectors per k-block (128 bytes of FP32 per row)
constexpr int GR_STAGES = 2;
constexpr int GR_THREADS = 192;            // TMA warp, MMA warp, four split / epilogue warps

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ------------------------------------------------------------------ transpose
// T[w][2x + c][g] = part c of Lam[w][g][x] (row pitch of Lam: lam_pitch(X)).
// Block (g-tile of 32, walker): the tile's rows are read along x and written
// along g, both coalesced.
__global__ void __launch_bounds__(256)
k_gram_transpose(int n_chol, int X, const float2* __restrict__ Lam, float* __restrict__ T)
{
    extern __shared__ float2 ts[];     // [32][X + 1]
    const int w = blockIdx.y, g0 = blockIdx.x * 32, t = threadIdx.x;
    const int XS = lam_pitch(X), ng = min(32, n_chol - g0);
    const float2* src = Lam + ((size_t)w * n_chol + g0) * XS;
    for (int e = t; e < ng * X; e += blockDim.x) {
        const int gg = e / X, x = e - gg * X;
        ts[gg * (X + 1) + x] = src[(size_t)gg * XS + x];
    }
    __syncthreads();
    float* dst = T + (size_t)w * 2 * X * n_chol + g0;
    for (int e = t; e < 2 * X * 32; e += blockDim.x) {
        const int r = e >> 5, gg = e & 31;
        if (gg < ng) {
            const float2 v = ts[gg * (X + 1) + (r >> 1)];
            dst[(size_t)r * n_chol + gg] = (r & 1) ? v.y : v.x;
        }
    }
}

}  // namespace

void launch_gram_transpose(int nw, int n_chol, int X, const float2* Lam, float* T, cudaStream_t st)
{
    if (nw <= 0 || n_chol <= 0 || X <= 0) return;
    const size_t smem = sizeof(float2) * 32 * (X + 1);
    dim3 grid((n_chol + 31) / 32, nw);
    k_gram_transpose<<<grid, 256, smem, st>>>(n_chol, X, Lam, T);
    msd_note_launch();
}

namespace {

struct GrJob {
    int Xp, Xq;        // entries of P and Q
    int a_map, b_map;  // which transposed spin the P and Q rows come from (0 alpha, 1 beta)
    float2* K;         // [nw][Xp][Xq]
};
struct GrArgs {
    GrJob j[3];
    int n_chol, NBmax;
    int nb[2];         // Q-tile rows of each spin: 2X rounded up to 16
    unsigned* err;
};

__global__ void __launch_bounds__(GR_THREADS, 1)
k_tc_gram(const __grid_constant__ CUtensorMap pa, const __grid_constant__ CUtensorMap pb,
          const __grid_constant__ CUtensorMap qa, const __grid_constant__ CUtensorMap qb,
          const __grid_constant__ GrArgs a)
{
    const GrJob jb = blockIdx.x == 0 ? a.j[0] : blockIdx.x == 1 ? a.j[1] : a.j[2];
    const int Xp = jb.Xp, Xq = jb.Xq;
    if (Xp <= 0 || Xq <= 0) return;
    const CUtensorMap* mapA = jb.a_map ? &pb : &pa;
    const CUtensorMap* mapB = jb.b_map ? &qb : &qa;
    const int w = blockIdx.y;
    const int mt = 2 * Xp > 128 ? 2 : 1;                 // M-tiles of 128 rows
    const int NB = a.nb[jb.b_map];                        // Q rows in the tile (MMA N)
    constexpr uint32_t A_TILE = 128 * 128;                // 128 rows x 32 FP32
    const uint32_t B_BYTES = (uint32_t)a.NBmax * 128;
    // stage: A hi [2 tiles], A lo [2 tiles], B hi, B lo
    const uint32_t STAGE = 4 * A_TILE + 2 * B_BYTES;
    const uint32_t TX = (uint32_t)mt * A_TILE + (uint32_t)NB * 128;   // bytes the TMA delivers
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[GR_STAGES], split_bar[GR_STAGES], empty_bar[GR_STAGES], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = (a.n_chol + GR_BK - 1) / GR_BK;
    const uint64_t wb = wait_budget(a.err);
    const uint32_t tcols = mt * NB <= 256 ? 256 : 512;

    if (threadIdx.x == 0) {
        for (int s = 0; s < GR_STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&split_bar[s], 4);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(&tmem_base_sh)), "r"(tcols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    volatile int* vfail = &fail;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------------------------ TMA producer
            int issued = 0;
            for (int kb = 0; kb < nkb && !*vfail; ++kb) {
                const int s = kb % GR_STAGES;
                if (!mbar_wait(&empty_bar[s], ((kb / GR_STAGES) & 1) ^ 1, wb) || *vfail) {
                    *vfail = 1;
                    atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
                    break;
                }
                uint8_t* st = smem + (size_t)s * STAGE;
                mbar_expect_tx(&full_bar[s], TX);
                for (int t = 0; t < mt; ++t) tma_load_3d(st + t * A_TILE, mapA, &full_bar[s], kb * GR_BK, t * 128, w);
                tma_load_3d(st + 4 * A_TILE, mapB, &full_bar[s], kb * GR_BK, 0, w);
                issued = kb + 1;
            }
            // the copies issued last land before the CTA may exit
            for (int k = issued - GR_STAGES < 0 ? 0 : issued - GR_STAGES; k < issued; ++k)
                mbar_drain(&full_bar[k % GR_STAGES], (k / GR_STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            const uint32_t idesc = idesc_tf32(128, NB);
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb % GR_STAGES;
                if (!mbar_wait(&split_bar[s], (kb / GR_STAGES) & 1, wb) || *vfail) {
                    *vfail = 1;
                    atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t sa = su32(smem + (size_t)s * STAGE);
                const uint32_t sbh = sa + 4 * A_TILE, sbl = sbh + B_BYTES;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {    // 4 x 32 bytes of K per k-block
                    const uint64_t bh = sw128_desc(sbh + kk * 32), bl = sw128_desc(sbl + kk * 32);
                    for (int t = 0; t < mt; ++t) {
                        const uint32_t acc = tmem + (uint32_t)(t * NB);
                        const uint64_t ah = sw128_desc(sa + t * A_TILE + kk * 32);
                        const uint64_t al = sw128_desc(sa + (2 + t) * A_TILE + kk * 32);
                        mma_tf32(acc, ah, bh, idesc, (kb | kk) != 0);
                        mma_tf32(acc, ah, bl, idesc, 1u);
                        mma_tf32(acc, al, bh, idesc, 1u);
                    }
                }
                mma_commit(&empty_bar[s]);
            }
            // every product issued here completes before TMEM is read or freed
            mma_commit(&done_bar);
            mbar_drain(&done_bar, 0);
        }
    } else {
        // ------------------------------------- split the landed blocks in place
        const int et = threadIdx.x - 64;                  // 0 .. 127
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % GR_STAGES;
            const bool ok = mbar_wait(&full_bar[s], (kb / GR_STAGES) & 1, wb);
            // one decision per warp (the flag may change between the lanes' reads)
            if (!__all_sync(0xffffffffu, ok && !*vfail)) {
                if (lane == 0) { *vfail = 1; atomicOr(a.err, MSD_DEV_ERR_TIMEOUT); }
                break;
            }
            uint8_t* st = smem + (size_t)s * STAGE;
            const int na = mt * (int)(A_TILE / 16), nbq = NB * 8;   // 16-byte pieces of A and of B
            for (int i = et; i < na + nbq; i += 128) {
                float4* hp = i < na ? reinterpret_cast<float4*>(st) + i
                                    : reinterpret_cast<float4*>(st + 4 * A_TILE) + (i - na);
                float4* lp = i < na ? reinterpret_cast<float4*>(st + 2 * A_TILE) + i
                                    : reinterpret_cast<float4*>(st + 4 * A_TILE + B_BYTES) + (i - na);
                const float4 x = *hp;
                const float4 h = make_float4(to_tf32(x.x), to_tf32(x.y), to_tf32(x.z), to_tf32(x.w));
                *hp = h;
                *lp = make_float4(to_tf32(x.x - h.x), to_tf32(x.y - h.y), to_tf32(x.z - h.z), to_tf32(x.w - h.w));
            }
            // generic-proxy stores -> visible to the tensor cores
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&split_bar[s]);
        }
        // ------------------------------------------------ epilogue
        const bool ok = mbar_wait(&done_bar, 0, wb);
        tc_fence_after();
        if (__all_sync(0xffffffffu, ok && !*vfail)) {
            const int q = warp & 3;
            float2* Kw = jb.K + (size_t)w * Xp * Xq;
            for (int t = 0; t < mt; ++t) {
                const int m = t * 128 + q * 32 + lane;     // row of C held by this lane
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * NB);
                for (int c0 = 0; c0 < NB; c0 += 16) {
                    float v[16];
                    tmem_ld16(taddr + (uint32_t)c0, v);
                    // the odd row 2x + 1 of C is the neighbouring lane
                    float o[16];
#pragma unroll
                    for (int i = 0; i < 16; ++i) o[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
                    const int x = m >> 1;
                    if ((m & 1) == 0 && x < Xp) {
#pragma unroll
                        for (int i = 0; i < 16; i += 2) {
                            const int y = (c0 + i) >> 1;
                            if (y < Xq) Kw[(size_t)x * Xq + y] = make_float2(v[i] - o[i + 1], v[i + 1] + o[i]);
                        }
                    }
                }
            }
        } else if (lane == 0) {
            atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
        }
    }
    __syncwarp();   // single-lane roles rejoin their warps
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
}

size_t gram_smem(int NBmax)
{
    return 1024 + (size_t)GR_STAGES * (4 * 128 * 128 + 2 * (size_t)NBmax * 128);
}

}  // namespace

bool tc_gram_ok(int Xa, int Xb)
{
    const int nbmax = ((2 * (Xa > Xb ? Xa : Xb) + 15) / 16) * 16;
    return Xa > 0 && Xb > 0 && 2 * Xa <= 256 && 2 * Xb <= 256 && gram_smem(nbmax) <= 227 * 1024 &&
           2 * nbmax <= 512;
}

int tc_gram(int nw, int n_chol, int Xa, int Xb, const float* Ta, const float* Tb, float2* Kaa, float2* Kbb,
            float2* Kab, unsigned* err, cudaStream_t st)
{
    if (nw <= 0 || n_chol <= 0) return 0;
    if (!tc_gram_ok(Xa, Xb) || n_chol % 4) return -1;
    GrArgs a;
    a.nb[0] = (2 * Xa + 15) / 16 * 16;
    a.nb[1] = (2 * Xb + 15) / 16 * 16;
    a.NBmax = a.nb[0] > a.nb[1] ? a.nb[0] : a.nb[1];
    a.n_chol = n_chol;
    a.err = err;
    a.j[0] = GrJob{Xa, Xa, 0, 0, Kaa};
    a.j[1] = GrJob{Xb, Xb, 1, 1, Kbb};
    a.j[2] = GrJob{Xa, Xb, 0, 1, Kab};
    CUtensorMap pa, pb, qa, qb;
    if (tc_make_map3(&pa, Ta, n_chol, 2 * Xa, nw, 128) || tc_make_map3(&pb, Tb, n_chol, 2 * Xb, nw, 128) ||
        tc_make_map3(&qa, Ta, n_chol, 2 * Xa, nw, a.nb[0]) || tc_make_map3(&qb, Tb, n_chol, 2 * Xb, nw, a.nb[1]))
        return -1;
    const size_t smem = gram_smem(a.NBmax);
    if (cudaFuncSetAttribute(k_tc_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    k_tc_gram<<<dim3(3, nw), GR_THREADS, smem, st>>>(pa, pb, qa, qb, a);
    msd_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
