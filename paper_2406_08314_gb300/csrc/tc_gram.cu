// Gram matrices of the mixed-precision local energy on the tensor cores
// (the Gram form of the generalized Wick terms, Sec. III: fill_os / get_ss
// sum over the Cholesky vectors):
//   K[x][y] = sum_g P_g[x] Q_g[y]   (complex, no conjugation),
// per walker, for (P, Q) = (Lambda^a, Lambda^a), (Lambda^b, Lambda^b) and
// (Lambda^a, Lambda^b), Lambda_g stored [walker][g][x] as FP32 pairs.
//
// With the complex entries read as interleaved reals, row m = 2x + c of the
// operand A is part c of P[.][x] and row n = 2y + d of B part d of Q[.][y];
// the real product C = A B^T over g holds every part combination, and
//   Re K[x][y] = C[2x][2y] - C[2x+1][2y+1],  Im K[x][y] = C[2x][2y+1] + C[2x+1][2y].
//
// One CTA per (walker, job), 256 threads. Per block of 32 vectors all
// threads read Lambda from global memory (coalesced along x, the next
// block's loads in flight while this block's products run), split each
// value into TF32 pieces and store them, transposed, in the K-major
// 128-byte-swizzled layout of the MMA operands (shared memory, two stages);
// one thread issues tcgen05.mma kind::tf32 over the pieces of a three-way
// TF32 split of both operands (x = x1 + x2 + x3 + O(2^-33 |x|); the six
// products x_i y_j with i + j <= 4, about the accuracy of FP32 products)
// per 8-vector step, into two TMEM accumulators (rows 0-127 and
// 128-255 of A) of N = 2 Xq columns rounded up to 16; the eight warps then
// combine neighbouring rows into complex K entries. Every wait is bounded;
// on expiry the kernel records MSD_DEV_ERR_TIMEOUT, lets its products
// complete, frees TMEM and returns.
#include <cuda.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int GR_THREADS = 256;
constexpr int GR_BK = 32;                  // vectors per k-block (128 bytes of FP32 per row)
constexpr int GR_ROWS_A = 256;             // two M-tiles of 128 rows

// Byte offset of element (row r, column k < 32) in a K-major tile with
// 128-byte rows, 8-row atoms of 1024 bytes and the 128-byte swizzle.
__device__ __forceinline__ uint32_t sw128_off(int r, int k)
{
    const int chunk = (k >> 2) ^ (r & 7);
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + chunk * 16 + (k & 3) * 4);
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

struct GrJob {
    int Xp, Xq;
    const float2* P;
    const float2* Q;
    float2* K;
};
struct GrJobs {
    GrJob j[3];
};

// This thread's share of one k-block of an operand, as float2 (one complex
// entry: rows m, m + 1 of the real operand) loaded ahead of its use.
constexpr int GR_V2 = 14;   // float2 per thread: 32 vectors x 2 X <= 32 x 224 floats

__device__ __forceinline__ void gr_load(float2 (&r)[GR_V2], const float* src, int rows, int kb, int n_chol)
{
    const int g0 = kb * GR_BK, ng = min(GR_BK, n_chol - g0);
    const int x2 = rows / 2, pitch = lam_pitch(x2);   // rows is even: x2 complex entries per vector
    const float2* b = reinterpret_cast<const float2*>(src) + (size_t)g0 * pitch;
    const int n2 = ng * x2;
#pragma unroll
    for (int i = 0; i < GR_V2; ++i) {
        const int f = threadIdx.x + i * GR_THREADS;
        const int gg = f / x2;
        r[i] = f < n2 ? b[(size_t)gg * pitch + (f - gg * x2)] : make_float2(0.f, 0.f);
    }
}

// Split the loaded values into NP TF32 pieces (x = sum of the pieces up to
// the residual of the last) and store each, transposed, into its plane.
template <int NP>
__device__ __forceinline__ void gr_store(const float2 (&r)[GR_V2], int rows, uint8_t* plane0, uint32_t plane_bytes)
{
#pragma unroll
    for (int i = 0; i < GR_V2; ++i) {
        const int f = threadIdx.x + i * GR_THREADS;
        if (f >= GR_BK * rows / 2) break;
        const int k = (2 * f) / rows, m = 2 * f - k * rows;
        const uint32_t o0 = sw128_off(m, k), o1 = sw128_off(m + 1, k);
        float x0 = r[i].x, x1 = r[i].y;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const float h0 = p + 1 < NP ? to_tf32(x0) : x0, h1 = p + 1 < NP ? to_tf32(x1) : x1;
            *reinterpret_cast<float*>(plane0 + p * plane_bytes + o0) = h0;
            *reinterpret_cast<float*>(plane0 + p * plane_bytes + o1) = h1;
            x0 -= h0;
            x1 -= h1;
        }
    }
}

template <int NP>
__global__ void __launch_bounds__(GR_THREADS, 1)
k_tc_gram(GrJobs jobs, int n_chol, int n_stages, int NB, unsigned* err)
{
    const GrJob jb = blockIdx.y == 0 ? jobs.j[0] : blockIdx.y == 1 ? jobs.j[1] : jobs.j[2];
    const int Xp = jb.Xp, Xq = jb.Xq;
    if (Xp <= 0 || Xq <= 0) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t mma_done[2];
    __shared__ __align__(8) uint64_t drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int w = blockIdx.x;
    const bool same = jb.P == jb.Q;
    const int MA = 2 * Xp, NBr = 2 * Xq;            // real rows of A and B
    const int mt = MA > 128 ? 2 : 1;                 // M-tiles
    const uint32_t A_BYTES = GR_ROWS_A * 128, B_BYTES = (uint32_t)NB * 128;
    const uint32_t STAGE = NP * A_BYTES + (same ? 0u : NP * B_BYTES);
    const uint64_t wb = wait_budget(err);

    if (t == 0) {
        mbar_init(&mma_done[0], 1);
        mbar_init(&mma_done[1], 1);
        mbar_init(&drain_bar, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(&tmem_base_sh)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // rows of A beyond 2 Xp and of B beyond 2 Xq stay zero in every stage
    for (int e = t; e < n_stages * (int)STAGE / 16; e += GR_THREADS)
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0, 0, 0, 0);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const float* Pw = reinterpret_cast<const float*>(jb.P + (size_t)w * n_chol * lam_pitch(Xp));
    const float* Qw = reinterpret_cast<const float*>(jb.Q + (size_t)w * n_chol * lam_pitch(Xq));
    const int nkb = (n_chol + GR_BK - 1) / GR_BK;
    const uint32_t idesc = idesc_tf32(128, NB);
    float2 ra[GR_V2], rb[GR_V2];
    gr_load(ra, Pw, MA, 0, n_chol);
    if (!same) gr_load(rb, Qw, NBr, 0, n_chol);
    for (int kb = 0; kb < nkb; ++kb) {
        const int s = n_stages == 2 ? (kb & 1) : 0;
        // the products that last read this stage have completed
        const int prev = kb - n_stages;
        if (prev >= 0) {
            const bool ok = mbar_wait(&mma_done[s], (uint32_t)((prev / n_stages) & 1), wb);
            if (!__syncthreads_and(ok)) {
                if (t == 0) { fail = 1; atomicOr(err, MSD_DEV_ERR_TIMEOUT); }
                break;
            }
        }
        tc_fence_after();
        uint8_t* st = smem + (size_t)s * STAGE;
        gr_store<NP>(ra, MA, st, A_BYTES);
        if (!same) gr_store<NP>(rb, NBr, st + NP * A_BYTES, B_BYTES);
        // the next block's loads fly while the products of this one run
        if (kb + 1 < nkb) {
            gr_load(ra, Pw, MA, kb + 1, n_chol);
            if (!same) gr_load(rb, Qw, NBr, kb + 1, n_chol);
        }
        // generic-proxy stores -> visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            tc_fence_after();
            const uint32_t sa = su32(st);
            const uint32_t sb = same ? sa : sa + NP * A_BYTES;
            const uint32_t bstride = same ? A_BYTES : B_BYTES;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                for (int tt = 0; tt < mt; ++tt) {
                    const uint32_t d = tmem + (uint32_t)(tt * NB);
                    bool first = kb == 0 && kk == 0;
                    // pieces (pa, pb) with pa + pb < NP: the products above the
                    // residual of the split
#pragma unroll
                    for (int pa = 0; pa < NP; ++pa)
#pragma unroll
                        for (int pb = 0; pa + pb < NP; ++pb) {
                            const uint64_t ad = sw128_desc(sa + pa * A_BYTES + tt * 16384 + kk * 32);
                            const uint64_t bd = sw128_desc(sb + pb * bstride + kk * 32);
                            mma_tf32(d, ad, bd, idesc, first ? 0u : 1u);
                            first = false;
                        }
                }
            }
            mma_commit(&mma_done[s]);
        }
    }
    if (t == 0) {
        // every product issued here completes before TMEM is read or freed
        mma_commit(&drain_bar);
        mbar_drain(&drain_bar, 0);
    }
    __syncthreads();
    tc_fence_after();
    const volatile int* vfail = &fail;
    if (!*vfail) {
        const int q = warp & 3, tt = warp >> 2;
        const int m = tt * 128 + q * 32 + lane;       // row of C held by this lane
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(tt * NB);
        float2* Kw = jb.K + (size_t)w * Xp * Xq;
        if (tt < mt) {
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
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

size_t gram_smem(int NB, int np, int stages)
{
    const size_t stage = np * ((size_t)GR_ROWS_A * 128 + (size_t)NB * 128);
    return 1024 + stages * stage;
}

}  // namespace

bool tc_gram_ok(int Xa, int Xb)
{
    return Xa > 0 && Xb > 0 && 2 * Xa <= GR_ROWS_A && 2 * Xb <= 256;
}

int tc_gram(int nw, int n_chol, const GramJobs& jobs, int nj, unsigned* err, cudaStream_t st)
{
    if (nw <= 0 || nj <= 0) return 0;
    int xq = 0;
    for (int i = 0; i < nj; ++i) {
        if (!tc_gram_ok(jobs.j[i].Xp, jobs.j[i].Xq)) return -1;
        xq = xq > jobs.j[i].Xq ? xq : jobs.j[i].Xq;
    }
    const int NB = (2 * xq + 15) / 16 * 16;
    // three TF32 pieces per value (six products: the rounding of FP32
    // products), two stages of shared memory when they fit
    constexpr int NP = 3;
    const int stages = gram_smem(NB, NP, 2) <= 227 * 1024 ? 2 : 1;
    const size_t smem = gram_smem(NB, NP, stages);
    if (cudaFuncSetAttribute(k_tc_gram<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    GrJobs g;
    for (int i = 0; i < 3; ++i)
        g.j[i] = i < nj ? GrJob{jobs.j[i].Xp, jobs.j[i].Xq, jobs.j[i].P, jobs.j[i].Q, jobs.j[i].K}
                        : GrJob{0, 0, nullptr, nullptr, nullptr};
    k_tc_gram<NP><<<dim3(nw, nj), GR_THREADS, smem, st>>>(g, n_chol, stages, NB, err);
    msd_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
