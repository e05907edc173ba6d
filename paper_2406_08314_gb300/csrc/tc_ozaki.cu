// Reference-determinant part of the mixed-precision local energy to FP64
// accuracy on the BF16 tensor cores.
//
// Per walker and spin, with the exactly known reference split G = D0 D0^T + dG
// (dG non-zero only in the columns v_r of the orbitals outside occ0) and
// u[(j, r)] = dG[occ0_j][v_r], the reference energy (Sec. II A, the
// generalized Wick theorem for a single determinant) needs, over the
// Cholesky vectors g,
//   t1_g = tr(L_g dG)           = sum_a u[a] W[a][g],   W[(j,r)][g] = L_g[v_r][o_j]
//   x2   = sum_g tr(dT_g dT_g)  = sum_ab u[a] V[a][b] u[b],
//   V[(j,r)][(l,r')] = sum_g L_g[v_r][o_l] L_g[v_r'][o_j]  (an exchange-type
//   two-electron integral, symmetric, constant per trial),
// with dT_g = (dG L_g)[occ0][occ0]. Both are products of the walker rows u
// with a constant matrix B = [V | W]^T, evaluated here as
//   P[m][n] = sum_k A[m][k] B[n][k]     (A rows: real and imaginary part of u)
// by an exact-integer split ("Ozaki scheme", Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 59 (2012)): every row of A and of B is scaled by a power
// of two to |x| < 1 and cut into S slices of BETA bits, x = 2^e sum_i
// a_i 2^(-BETA i) with integers |a_i| <= 2^BETA, stored exactly in BF16.
// The slice products a_i b_j with i + j = c share one FP32 accumulator in
// TMEM; over a chunk of KCH contraction steps every such sum stays below
// 2^24 in magnitude, so the tensor cores add integers exactly. After each
// chunk the epilogue takes the S accumulators into 64-bit integer sums
// (exact), and at the end scales them by 2^(e_A + e_B - BETA (S + 1)). The
// products with i + j > S + 1 are dropped: the result carries about
// BETA S = 35 bits relative to the row and column scales, against 24 for an
// FP32 product.
//
// V is symmetric: a tile of V columns contracts only the diagonal block and
// the blocks after it, the latter counted twice (about 40 % less work).
//
// Structure (one CTA per 128 x 96 output tile, 10 warps):
//   warp 0    TMA producer: k-blocks of 32 BF16 (64-byte swizzle) of all S
//             slices of A and B into a three-stage shared-memory ring;
//   warp 1    TMEM owner; lane 0 issues tcgen05.mma kind::f16 (15 products
//             per 16-element K step) into the S accumulators;
//   warps 2-9 epilogue: lane quarter (warp % 4), column half ((warp - 2) / 4);
//             each drains its 48 columns of the S accumulators after every
//             chunk, then forms, per row, the partial quadratic form
//             (sum_n P[m][n] u_re[n], sum_n P[m][n] u_im[n]) over the V
//             columns and writes the W columns (t1) out.
// Every wait is bounded (about 2 s); on expiry the kernel records
// MSD_DEV_ERR_TIMEOUT, every role leaves its loop, issued copies and
// products are drained and TMEM is freed.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int OZ_S = 5;                 // slices per operand
constexpr int OZ_BETA = 7;              // bits per slice
constexpr int OZ_BM = 128, OZ_BN = 96;  // output tile
constexpr int OZ_BK = 32;               // BF16 elements per k-block (64 bytes)
constexpr int OZ_KCH_KB = 16;           // k-blocks per exact chunk (512 contraction steps)
constexpr int OZ_STAGES = 3;
constexpr int OZ_THREADS = 320;
constexpr uint32_t OZ_A_SL = OZ_BM * 64, OZ_B_SL = OZ_BN * 64;
constexpr uint32_t OZ_STAGE = OZ_S * (OZ_A_SL + OZ_B_SL);
constexpr size_t OZ_SMEM = (size_t)OZ_STAGES * OZ_STAGE + 1024;
constexpr int OZ_HALF = OZ_BN / 2;      // columns per epilogue warp

static_assert(OZ_S == 5 && OZ_BETA == 7 && OZ_KCH_KB * OZ_BK == 512,
              "the exactness bound below is worked out for 5 slices of 7 bits and chunks of 512");
// Bound: |a_1|, |b_1| <= 128 and |a_i|, |b_j| <= 64 otherwise, so one K step
// adds at most 28672 (c = 6: 2 * 128 * 64 + 3 * 64 * 64) to an accumulator;
// 512 steps stay below 1.47e7 < 2^24.

struct OzArgs {
    int nrow, Mpad, NB, NBp, NV, NVp, G, Kp;   // B rows: V [0, NV), zero [NV, NVp), W [NVp, NB)
    int N, M, Kv;
    const int* ea;          // [Mpad] row exponents of A
    const int* eb;          // [NBp] row exponents of B
    const double2* Gr;      // [nrow / 2][N][M]: u[(j, r)] = Gr[w][j][virt[r]]
    const int* virt;
    double2* part;          // [n_tiles_n * 2][Mpad]
    double* t1;             // [nrow][G]
    unsigned* err;
};

__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t* r)
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
k_tc_ozaki(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
           const __grid_constant__ OzArgs a)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full_bar[OZ_STAGES], empty_bar[OZ_STAGES];
    __shared__ __align__(8) uint64_t tfull, tempty, drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Column tile: V is symmetric, so a tile of V columns [n0, n0 + BN)
    // contracts only K >= n0, its diagonal block once and the later blocks
    // with weight 2 (the mirrored earlier blocks are skipped):
    //   u^T V u = sum_n (u_n^T V_nn u_n + 2 sum_{k > n} u_k^T V_kn u_n).
    // V's rows are padded with zeros to whole tiles (NVp), so no tile mixes
    // V and W columns. The W tiles take the full K range and run first; the
    // V tiles follow, longest first.
    const int nvt = a.NVp / OZ_BN, ntile = gridDim.y;
    const int tile = (int)blockIdx.y < ntile - nvt ? nvt + (int)blockIdx.y : (int)blockIdx.y - (ntile - nvt);
    const bool sym = tile < nvt;
    const int m0 = blockIdx.x * OZ_BM, n0 = tile * OZ_BN;
    const int nkb = a.Kp / OZ_BK;
    const int kbeg = sym ? n0 / OZ_BK : 0, nkt = nkb - kbeg;            // this tile's k-blocks
    const int first = sym ? OZ_BN / OZ_BK : OZ_KCH_KB;                   // k-blocks of chunk 0
    const int nch = nkt <= first ? 1 : 1 + (nkt - first + OZ_KCH_KB - 1) / OZ_KCH_KB;
    auto chunk_begin = [&](int ch) { return ch == 0 ? 0 : first + (ch - 1) * OZ_KCH_KB; };   // relative
    const uint64_t wb = wait_budget(a.err);

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&tfull, 1);
        mbar_init(&tempty, 8);
        mbar_init(&drain_bar, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(&tmem_base_sh)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    volatile int* vfail = &fail;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- TMA producer
            int kb = 0;
            for (; kb < nkt; ++kb) {
                const int s = kb % OZ_STAGES;
                if (!mbar_wait(&empty_bar[s], ((kb / OZ_STAGES) & 1) ^ 1, wb) || *vfail) {
                    *vfail = 1;
                    atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
                    break;
                }
                uint8_t* st = smem + (size_t)s * OZ_STAGE;
                mbar_expect_tx(&full_bar[s], OZ_STAGE);
                const int kx = (kbeg + kb) * OZ_BK;
#pragma unroll
                for (int i = 0; i < OZ_S; ++i) {
                    tma_load_2d(st + i * OZ_A_SL, &ta, &full_bar[s], kx, i * a.Mpad + m0);
                    tma_load_2d(st + OZ_S * OZ_A_SL + i * OZ_B_SL, &tb, &full_bar[s], kx, i * a.NBp + n0);
                }
            }
            // the copies issued last must land before the CTA may exit
            for (int k = kb - OZ_STAGES < 0 ? 0 : kb - OZ_STAGES; k < kb; ++k)
                mbar_drain(&full_bar[k % OZ_STAGES], (k / OZ_STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer
            constexpr uint32_t idesc = idesc_bf16(OZ_BM, OZ_BN);
            bool ok = true;
            for (int ch = 0; ch < nch && ok; ++ch) {
                // the epilogue has taken the previous chunk out of TMEM
                if (ch > 0 && !mbar_wait(&tempty, (ch - 1) & 1, wb)) { ok = false; break; }
                tc_fence_after();
                const int kb0 = chunk_begin(ch), kb1 = min(nkt, chunk_begin(ch + 1));
                for (int kb = kb0; kb < kb1; ++kb) {
                    const int s = kb % OZ_STAGES;
                    if (!mbar_wait(&full_bar[s], (kb / OZ_STAGES) & 1, wb) || *vfail) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(smem + (size_t)s * OZ_STAGE);
                    const uint32_t sb = sa + OZ_S * OZ_A_SL;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {   // 2 x 16 BF16 of K per k-block
                        uint64_t da[OZ_S], db[OZ_S];
#pragma unroll
                        for (int i = 0; i < OZ_S; ++i) {
                            da[i] = sw64_desc(sa + i * OZ_A_SL + kk * 32);
                            db[i] = sw64_desc(sb + i * OZ_B_SL + kk * 32);
                        }
                        const bool first = kb == kb0 && kk == 0;
#pragma unroll
                        for (int c = 2; c <= OZ_S + 1; ++c) {
                            bool head = true;
#pragma unroll
                            for (int i = 1; i <= OZ_S; ++i) {
                                const int j = c - i;
                                if (j < 1 || j > OZ_S) continue;
                                mma_bf16(tmem + (uint32_t)((c - 2) * OZ_BN), da[i - 1], db[j - 1], idesc,
                                         (first && head) ? 0u : 1u);
                                head = false;
                            }
                        }
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&tfull);
            }
            if (!ok) {
                *vfail = 1;
                atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
            }
            // every product issued by this thread completes before TMEM is freed
            mma_commit(&drain_bar);
            mbar_drain(&drain_bar, 0);
        }
    } else {
        // -------------------------------------------------------- epilogue
        const int q = warp & 3, hf = (warp - 2) >> 2;
        const int row = m0 + q * 32 + lane;
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(hf * OZ_HALF);
        long long acc[OZ_HALF];
#pragma unroll
        for (int i = 0; i < OZ_HALF; ++i) acc[i] = 0;
        bool ok = true;
        for (int ch = 0; ch < nch; ++ch) {
            const bool got = mbar_wait(&tfull, ch & 1, wb) && !*vfail;
            if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int g3 = 0; g3 < OZ_HALF / 16; ++g3) {
                uint32_t r[OZ_S][16];
#pragma unroll
                for (int c = 0; c < OZ_S; ++c) tmem_ld16_nowait(tbase + (uint32_t)(c * OZ_BN + g3 * 16), r[c]);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    long long v = 0;
#pragma unroll
                    for (int c = 0; c < OZ_S; ++c)
                        v += (long long)__float2int_rn(__uint_as_float(r[c][i])) *
                             (1ll << (OZ_BETA * (OZ_S - 1 - c)));
                    acc[g3 * 16 + i] += (sym && ch > 0) ? 2 * v : v;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty);
        }
        if (!ok) {
            if (lane == 0) { *vfail = 1; atomicOr(a.err, MSD_DEV_ERR_TIMEOUT); }
        } else if (row < a.nrow) {
            const int w = row >> 1;
            const int er = a.ea[row] - OZ_BETA * (OZ_S + 1);
            double dre = 0, dim = 0;
#pragma unroll
            for (int i = 0; i < OZ_HALF; ++i) {
                const int n = n0 + hf * OZ_HALF + i;
                if (n >= a.NB) break;
                const double v = ldexp((double)acc[i], er + a.eb[n]);
                if (n < a.NV) {
                    const int j = n / a.Kv, r = n - j * a.Kv;
                    const double2 u = a.Gr[((size_t)w * a.N + j) * a.M + a.virt[r]];
                    dre = fma(v, u.x, dre);
                    dim = fma(v, u.y, dim);
                } else if (n >= a.NVp) {
                    a.t1[(size_t)row * a.G + (n - a.NVp)] = v;
                }
            }
            a.part[(size_t)(tile * 2 + hf) * a.Mpad + row] = make_double2(dre, dim);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

// Largest |x| of a block's values (all threads return it).
__device__ double block_absmax(double m, double* red)
{
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const double r = red[0];
    __syncthreads();
    return r;
}

// x 2^-e cut into OZ_S integer slices of OZ_BETA bits (exact in FP64 and BF16).
__device__ __forceinline__ void slice_store(double x, int e, __nv_bfloat16* out, size_t slice_stride)
{
    double r = ldexp(x, -e);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) {
        r *= (double)(1 << OZ_BETA);
        const double ai = rint(r);
        r -= ai;
        out[i * slice_stride] = __float2bfloat16_rn((float)ai);
    }
}

__device__ __forceinline__ int slice_exponent(double mx)
{
    int e = 0;
    if (mx > 0) frexp(mx, &e);   // mx = f 2^e, f in [0.5, 1): |x| 2^-e < 1
    return e;
}

// Slices of the walker rows: row 2w + c is part c (real, imaginary) of
// u_w[(j, r)] = Gr[w][j][virt[r]]; rows >= nrow and columns >= N Kv are zero.
__global__ void __launch_bounds__(256)
k_oz_slice_rows(int nrow, int N, int M, int Kv, int Kp, const double2* __restrict__ Gr, const int* __restrict__ virt,
                __nv_bfloat16* __restrict__ As, int* __restrict__ ea, size_t slice_stride)
{
    __shared__ double red[32];
    const int row = blockIdx.x, NK = N * Kv;
    const int w = row >> 1, c = row & 1;
    const bool live = row < nrow;
    double mx = 0;
    if (live)
        for (int k = threadIdx.x; k < NK; k += blockDim.x) {
            const int j = k / Kv, r = k - j * Kv;
            const double2 v = Gr[((size_t)w * N + j) * M + virt[r]];
            mx = fmax(mx, fabs(c ? v.y : v.x));
        }
    const int e = slice_exponent(block_absmax(mx, red));
    __nv_bfloat16* out = As + (size_t)row * Kp;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        double x = 0;
        if (live && k < NK) {
            const int j = k / Kv, r = k - j * Kv;
            const double2 v = Gr[((size_t)w * N + j) * M + virt[r]];
            x = c ? v.y : v.x;
        }
        slice_store(x, e, out + k, slice_stride);
    }
    if (threadIdx.x == 0) ea[row] = e;
}

// Slices of the constant rows: row b < NK = N Kv, b = (l, r'), is
// V[(j, r)][b] = C2[r N + l][r' N + j] at column a = (j, r); rows
// [NK, NVp) are zero; row NVp + g is W[(j, r)][g] = XT[r N + j][g]; rows
// >= NB are zero.
__global__ void __launch_bounds__(256)
k_oz_slice_const(int N, int Kv, int G, int NVp, int NB, int Kp, const double* __restrict__ C2,
                 const double* __restrict__ XT, __nv_bfloat16* __restrict__ Bs, int* __restrict__ eb,
                 size_t slice_stride)
{
    __shared__ double red[32];
    const int b = blockIdx.x, NK = N * Kv;
    const bool live = b < NK || (b >= NVp && b < NB);
    auto val = [&](int k) -> double {
        const int j = k / Kv, r = k - j * Kv;
        if (b < NK) {
            const int l = b / Kv, rp = b - l * Kv;
            return C2[(size_t)(r * N + l) * NK + (size_t)rp * N + j];
        }
        return XT[(size_t)(r * N + j) * G + (b - NVp)];
    };
    double mx = 0;
    if (live)
        for (int k = threadIdx.x; k < NK; k += blockDim.x) mx = fmax(mx, fabs(val(k)));
    const int e = slice_exponent(block_absmax(mx, red));
    __nv_bfloat16* out = Bs + (size_t)b * Kp;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x)
        slice_store((live && k < NK) ? val(k) : 0.0, e, out + k, slice_stride);
    if (threadIdx.x == 0) eb[b] = e;
}

// C[m][n] = sum_k A[m][k] B[n][k], real FP64; 64 x 64 tile, k-step 16.
__global__ void __launch_bounds__(256)
k_gemm_dd(int Mr, int Nc, int K, const double* __restrict__ A, long long lda, const double* __restrict__ B,
          long long ldb, double* __restrict__ C, long long ldc)
{
    __shared__ double As[16][64 + 1], Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + q * 256, rr = e / 16, kk = e % 16;
            const int m = m0 + rr, n = n0 + rr, k = k0 + kk;
            As[kk][rr] = (m < Mr && k < K) ? A[(size_t)m * lda + k] : 0.0;
            Bs[kk][rr] = (n < Nc && k < K) ? B[(size_t)n * ldb + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double x[4], y[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { x[i] = As[kk][ty * 4 + i]; y[i] = Bs[kk][tx * 4 + i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(x[i], y[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < Mr && n < Nc) C[(size_t)m * ldc + n] = acc[i][j];
        }
}

// Per walker: the reference energy's Cholesky sums from both spins
//   scal[w][s] = sum_g x_g^s = x0sum_s + 2 u_s . KK_s + x2_s
//   scal[w][2] = sum_g V0_g^2 = C2sum + 2 sum_s u_s . JJ_s + sum_g (t1a_g + t1b_g)^2
// (FP64, fixed summation order), and the walker parts t1a_g + t1b_g of V0_g
// as FP32 pairs, v0w[w][g].
__global__ void __launch_bounds__(256)
k_ref_reduce(int nw, int G, RefSpin sa, RefSpin sb, double C2sum, double2* __restrict__ scal,
             float2* __restrict__ v0w)
{
    __shared__ double2 red[4][256];
    const int w = blockIdx.x, t = threadIdx.x;
    double2 lj[2] = {cz(0, 0), cz(0, 0)}, lk[2] = {cz(0, 0), cz(0, 0)};
    const RefSpin* S[2] = {&sa, &sb};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const RefSpin& R = *S[s];
        const int NK = R.N * R.Kv;
        for (int k = t; k < NK; k += blockDim.x) {
            const int j = k / R.Kv, r = k - j * R.Kv;
            const double2 u = R.Gr[((size_t)w * R.N + j) * R.M + R.virt[r]];
            lj[s] = cadd(lj[s], cscale(u, R.JJ[k]));
            lk[s] = cadd(lk[s], cscale(u, R.KK[k]));
        }
    }
    double2 q = cz(0, 0);
    for (int g = t; g < G; g += blockDim.x) {
        const double2 v = cz(sa.t1[(size_t)(2 * w) * G + g] + sb.t1[(size_t)(2 * w) * G + g],
                             sa.t1[(size_t)(2 * w + 1) * G + g] + sb.t1[(size_t)(2 * w + 1) * G + g]);
        q = cfma(v, v, q);
        v0w[(size_t)w * G + g] = make_float2((float)v.x, (float)v.y);
    }
    red[0][t] = cadd(lj[0], lj[1]);
    red[1][t] = lk[0];
    red[2][t] = lk[1];
    red[3][t] = q;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (t < o)
            for (int i = 0; i < 4; ++i) red[i][t] = cadd(red[i][t], red[i][t + o]);
        __syncthreads();
    }
    if (t == 0) {
        double2 x2[2];
        for (int s = 0; s < 2; ++s) {
            const RefSpin& R = *S[s];
            double2 v = cz(0, 0);
            for (int p = 0; p < R.nparts; ++p) {
                const double2 pr = R.part[(size_t)p * R.Mpad + 2 * w];       // (ur.Vur, ui.Vur)
                const double2 pi = R.part[(size_t)p * R.Mpad + 2 * w + 1];   // (ur.Vui, ui.Vui)
                v = cadd(v, cz(pr.x - pi.y, pi.x + pr.y));
            }
            x2[s] = v;
        }
        double2* sc = scal + (size_t)w * 8;
        sc[0] = cadd(cz(sa.x0sum, 0), cadd(cscale(red[1][0], 2.0), x2[0]));
        sc[1] = cadd(cz(sb.x0sum, 0), cadd(cscale(red[2][0], 2.0), x2[1]));
        sc[2] = cadd(cz(C2sum, 0), cadd(cscale(red[0][0], 2.0), red[3][0]));
    }
}

}  // namespace

size_t oz_const_bytes(int N, int Kv, int G)
{
    const long long NK = (long long)N * Kv, NB = (NK + OZ_BN - 1) / OZ_BN * OZ_BN + G;
    const long long NBp = (NB + OZ_BN - 1) / OZ_BN * OZ_BN, Kp = (NK + OZ_BK - 1) / OZ_BK * OZ_BK;
    return (size_t)OZ_S * NBp * Kp * sizeof(__nv_bfloat16) + sizeof(int) * NBp;
}

int oz_rows_padded(int nrow) { return (nrow + OZ_BM - 1) / OZ_BM * OZ_BM; }
int oz_k_padded(int NK) { return (NK + OZ_BK - 1) / OZ_BK * OZ_BK; }
int oz_parts(int NB) { return 2 * ((NB + OZ_BN - 1) / OZ_BN); }
int oz_parts_for(int NK, int G) { return oz_parts((NK + OZ_BN - 1) / OZ_BN * OZ_BN + G); }
int oz_slices() { return OZ_S; }

int oz_prepare_const(int N, int Kv, int G, const double* d_XT, OzConst& out, cudaStream_t st)
{
    const int NK = N * Kv;
    out.N = N; out.Kv = Kv; out.G = G;
    out.NK = NK;
    out.NVp = (NK + OZ_BN - 1) / OZ_BN * OZ_BN;
    out.NB = out.NVp + G;
    out.NBp = (out.NB + OZ_BN - 1) / OZ_BN * OZ_BN;
    out.Kp = oz_k_padded(NK);
    double* C2 = nullptr;
    if (cudaMallocAsync((void**)&C2, sizeof(double) * (size_t)NK * NK, st) != cudaSuccess) return -1;
    dim3 grid((NK + 63) / 64, (NK + 63) / 64);
    k_gemm_dd<<<grid, 256, 0, st>>>(NK, NK, G, d_XT, G, d_XT, G, C2, NK);
    msd_note_launch();
    const size_t ss = (size_t)out.NBp * out.Kp;
    if (cudaMallocAsync((void**)&out.Bs, sizeof(__nv_bfloat16) * OZ_S * ss, st) != cudaSuccess ||
        cudaMallocAsync((void**)&out.eb, sizeof(int) * out.NBp, st) != cudaSuccess) {
        cudaFreeAsync(C2, st);
        return -1;
    }
    k_oz_slice_const<<<out.NBp, 256, 0, st>>>(N, Kv, G, out.NVp, out.NB, out.Kp, C2, d_XT,
                                              (__nv_bfloat16*)out.Bs, out.eb, ss);
    msd_note_launch();
    cudaFreeAsync(C2, st);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void oz_free_const(OzConst& c)
{
    cudaFree(c.Bs);
    cudaFree(c.eb);
    c = OzConst{};
}

int oz_spin(const OzConst& K, int nw, int M, const double2* Gr, const int* virt, void* As, int* ea, double2* part,
            double* t1, unsigned* err, cudaStream_t st)
{
    const int nrow = 2 * nw, Mpad = oz_rows_padded(nrow);
    const size_t sa = (size_t)Mpad * K.Kp;
    k_oz_slice_rows<<<Mpad, 256, 0, st>>>(nrow, K.N, M, K.Kv, K.Kp, Gr, virt, (__nv_bfloat16*)As, ea, sa);
    msd_note_launch();
    CUtensorMap ma, mb;
    if (tc_make_map(&ma, As, K.Kp, OZ_S * Mpad, K.Kp, OZ_BM, true, 64) ||
        tc_make_map(&mb, K.Bs, K.Kp, OZ_S * K.NBp, K.Kp, OZ_BN, true, 64))
        return -1;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_tc_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OZ_SMEM) !=
            cudaSuccess)
            return -1;
        attr = true;
    }
    OzArgs a;
    a.nrow = nrow; a.Mpad = Mpad; a.NB = K.NB; a.NBp = K.NBp; a.NV = K.NK; a.NVp = K.NVp; a.G = K.G; a.Kp = K.Kp;
    a.N = K.N; a.M = M; a.Kv = K.Kv;
    a.ea = ea; a.eb = K.eb; a.Gr = Gr; a.virt = virt; a.part = part; a.t1 = t1; a.err = err;
    dim3 grid(Mpad / OZ_BM, K.NBp / OZ_BN);
    k_tc_ozaki<<<grid, OZ_THREADS, OZ_SMEM, st>>>(ma, mb, a);
    msd_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_ref_reduce(int nw, int G, const RefSpin& a, const RefSpin& b, double C2sum, double2* scal,
                       float2* v0w, cudaStream_t st)
{
    k_ref_reduce<<<nw, 256, 0, st>>>(nw, G, a, b, C2sum, scal, v0w);
    msd_note_launch();
}
