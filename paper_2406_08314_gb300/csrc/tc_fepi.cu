// Fused Cholesky-vector contraction and epilogue of the mixed-precision
// local energy (Eq. 10-12 in the Gram form of the generalized Wick terms):
//
//   dF[(w, c, j)][g NCf + col] = sum_k dG_w[occ0_j][virt_k] Lh[g NCf + col][virt_k]
//
// on the tensor cores (3xTF32, FP32 accumulation in TMEM), followed on the
// same SM, per (walker w, Cholesky vector g), by the algebra on
// F = F0 + dF (T = F[:, occ0] = T0 + dT, F_P = F[:, P]):
//   v0 = c0_g + tr dT (= tr T),   x = x0_g + 2 tr(T0 dT) + tr(dT dT),
//   Lambda[j][p] = F_P[j][p] - sum_l T[j][l] G[occ0_l][P_p],
//   Lact[(h,p)] = Lambda[pos(h)][p],  Xic[(h,p)] = sum_l T[pos(h)][l] Lambda[l][p].
// The FP32 products never reach device memory.
//
// Rows of the A operand: walker w owns 2 RB rows, (w, c, j) -> (2w + c) RB + j
// (c = 0 real, 1 imaginary part of dG, j < N, rows N..RB-1 zero), RB = 8, 16
// or 32, so that one row block lies inside one TMEM lane quarter and each
// epilogue lane holds one row (w, c, j) of F in registers. Columns of the B
// operand: vector g owns NCf = RB + np rows, the N of occ0 then RB - N zero
// rows then the np particles, so that T is RB x RB with zero padding and
// every epilogue loop runs over the compile-time RB without tests.
//
// Structure (persistent, one CTA per SM, 14 warps):
//   warp 0      TMA producer: A and B k-blocks of 16 FP32 (64-byte swizzle),
//               TF32 hi and lo parts, into a two-stage shared-memory ring;
//   warp 1      TMEM owner; lane 0 issues tcgen05.mma into one of two TMEM
//               accumulators (the next tile's products overlap this tile's
//               epilogue);
//   warps 2-13  epilogue, three sets of four warps (one per lane quarter)
//               taking every third Cholesky vector of a tile. The real and
//               imaginary row blocks of a walker (lanes of one warp, or two
//               warps when RB = 32) swap their rows through a per-walker
//               shared-memory slot, so that each lane holds the complex row
//               T[j][:]; the real-part lanes then form Lambda and Xi for the
//               first half of the particles, the imaginary-part lanes for the
//               second half. Operands common to all rows (G[occ0][P] and
//               Lambda) are read as shared-memory broadcasts, the limiting
//               resource, once per part rather than once per part and
//               particle half. With the exchange traces (XTR), each set
//               prefetches the reference block F0 of its next vector with
//               cp.async while it works on the current one and adds it to
//               dF; without them (the exactly split reference sums supply
//               sum_g x_g) the contraction adds F0 itself through two
//               identity blocks of the A operand and F0 slices of the B
//               operand, and the epilogue reads no F0. The epilogue reads no
//               global memory but G[occ0][P] once a tile. Lambda and Xi rows
//               are stored with a pitch of whole 128-byte lines.
// Every wait is bounded (about 2 s); on expiry the kernel records
// MSD_DEV_ERR_TIMEOUT, every role leaves its loop, issued copies and
// products are drained and TMEM is freed.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

using namespace tcx;

namespace {

constexpr int FE_SETS = 3;                      // epilogue sets of four warps (one per TMEM lane quarter)
constexpr int FE_EPI = 128 * FE_SETS;
constexpr int FE_THREADS = 64 + FE_EPI;         // producer warp, MMA warp, epilogue warps
constexpr int FE_STAGES = 2;
constexpr int FE_TCOLS = 256;                 // TMEM columns per accumulator buffer
constexpr uint32_t FE_A_BYTES = 128 * 64;     // 128 rows x 16 FP32
constexpr int FE_XMAX = 128;                  // output entries (holes x particles) mapped in shared memory

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

struct FeArgs {
    SpinTables tb;
    int nw, M, n_chol, K;      // K: contraction length (multiple of 8)
    int BN, GPT, BNe, slot;    // B tile rows, vectors per tile, MMA N, floats per walker slot
    int NCf, NCP, f0s;         // B rows per vector, shared-memory pitch of an F0 row, floats per F0 block
    int n_rt, n_ct, n_tiles;   // row tiles (walker blocks), column tiles (vector blocks)
    const double2* Gr;
    const float* F0P;          // [n_chol][f0s]: F0[j][col] at [g][j NCP + col], zero padded
    const double* c0;
    const double* x0;
    double2* v0;
    double2* xx;
    float2* Lact;
    float2* Xic;
    unsigned* err;
};

// Tile order: the column tile (block of Cholesky vectors) runs fastest, so
// the CTAs at work share one walker row tile and the whole Cholesky operand
// (tens of MB) is what stays in L2 between its uses; with the row tile
// fastest the larger walker operand is re-read from DRAM (0.95 GB against
// 0.14 GB of reads per launch at 640 walkers x 800 vectors).
__device__ __forceinline__ int tile_rt(const FeArgs& a, int t) { return t / a.n_ct; }
__device__ __forceinline__ int tile_ct(const FeArgs& a, int t) { return t % a.n_ct; }

template <int RB>
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, float* v)
{
    uint32_t r[RB];
    if constexpr (RB == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
              "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
              "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else if constexpr (RB == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
              "=r"(r[15])
            : "r"(taddr));
    } else {
        tmem_ld8_nowait(taddr, r);
    }
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < RB; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Pair barrier of the two row blocks (real, imaginary) of one walker: two
// warps on hardware barrier `id` when RB = 32, else lanes of one warp.
template <int RB>
__device__ __forceinline__ void pair_sync(int id)
{
    if constexpr (RB == 32) bar_sync(id, 64);
    else __syncwarp();
}

// sum_l (tr + i ti)[l] (br + i bi)[l] over l < RB. tr, ti: the row as FP32
// pairs (l, l + 1); br, bi: rows of shared memory read as broadcasts, also
// taken as pairs. Two-lane FMAs: each lane an IEEE fma (round to nearest).
template <int RB>
__device__ __forceinline__ float2 cdot_row(const unsigned long long* tr, const unsigned long long* ti,
                                           const float* br, const float* bi)
{
    const ulonglong2* r2 = reinterpret_cast<const ulonglong2*>(br);
    const ulonglong2* i2 = reinterpret_cast<const ulonglong2*>(bi);
    unsigned long long rr0 = 0, rr1 = 0, ii0 = 0, ii1 = 0, ri0 = 0, ri1 = 0, ir0 = 0, ir1 = 0;
#pragma unroll
    for (int k = 0; k < RB / 2; k += 2) {       // pairs k, k + 1 = columns 2k .. 2k + 3
        const ulonglong2 r = r2[k >> 1], i = i2[k >> 1];
        fma2(rr0, tr[k], r.x);       fma2(rr1, tr[k + 1], r.y);    // tr br
        fma2(ii0, ti[k], i.x);       fma2(ii1, ti[k + 1], i.y);    // ti bi
        fma2(ri0, tr[k], i.x);       fma2(ri1, tr[k + 1], i.y);    // tr bi
        fma2(ir0, ti[k], r.x);       fma2(ir1, ti[k + 1], r.y);    // ti br
    }
    const float2 a = unpack2(rr0), b = unpack2(rr1), c = unpack2(ii0), d = unpack2(ii1);
    const float2 e = unpack2(ri0), f = unpack2(ri1), g = unpack2(ir0), h = unpack2(ir1);
    return make_float2(((a.x + a.y) + (b.x + b.y)) - ((c.x + c.y) + (d.x + d.y)),
                       ((e.x + e.y) + (f.x + f.y)) + ((g.x + g.y) + (h.x + h.y)));
}

// XTR: form the exchange traces x_g (the T0.dT and dT.dT products); the
// accumulator then holds dF and the epilogue adds F0 from shared memory.
// Without XTR only v0 and Lambda/Xi are written (the caller takes sum_g x_g
// from the exactly split reference sums), and the contraction itself adds
// F0: the A operand carries two identity blocks on its real-part rows and
// the B operand the matching slices of F0 (h + m, then r + r2), so that the
// accumulator holds F = F0 + dF and the epilogue reads no F0 block.
template <int RB, bool XTR>
// Bounds of 512 threads cap registers at 128: with 14 warps, four share a
// sub-partition's 16K-register file.
__global__ void __launch_bounds__(512, 1)
k_tc_fepi(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
          const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
          const __grid_constant__ FeArgs a)
{
    constexpr int WPT = 64 / RB;          // walkers per tile
    constexpr int PW = 16;                // particle columns read from TMEM per row (np <= PW)
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int N = a.tb.N, np = a.tb.np, NCf = a.NCf, X = a.tb.nh * np, NCP = a.NCP;
    const uint32_t B_BYTES = (uint32_t)a.BN * 64, STAGE_BYTES = 2 * (FE_A_BYTES + B_BYTES);
    float* slots = reinterpret_cast<float*>(smem + FE_STAGES * STAGE_BYTES);      // [FE_SETS][WPT][slot]
    float* gpRe = slots + FE_SETS * WPT * a.slot;                                 // [2][WPT][np][RB]
    float* gpIm = gpRe + 2 * WPT * np * RB;                                       // [2][WPT][np][RB]
    float* f0buf = gpIm + 2 * WPT * np * RB;                                      // [FE_SETS][2][f0s]
    int* oe = reinterpret_cast<int*>(f0buf + FE_SETS * 2 * a.f0s);               // [X] pos(h) np + p
    const int GE = WPT * np * RB;                 // entries of a tile's G[occ0][P] block
    // the next tile's G[occ0][P] block as FP64, copied ahead by cp.async
    double2* gst = reinterpret_cast<double2*>(((uintptr_t)(oe + FE_XMAX) + 15) & ~(uintptr_t)15);

    __shared__ __align__(8) uint64_t full_bar[FE_STAGES], empty_bar[FE_STAGES];
    __shared__ __align__(8) uint64_t tfull[2], tempty[2], drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = (a.K + 15) / 16;
    const uint64_t wb = wait_budget(a.err);

    for (int e = threadIdx.x; e < X; e += blockDim.x) oe[e] = a.tb.hole_pos[e / np] * np + e % np;
    if (threadIdx.x == 0) {
        for (int s = 0; s < FE_STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&tfull[b], 1); mbar_init(&tempty[b], FE_EPI / 32); }
        mbar_init(&drain_bar, 1);
        fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(su32(&tmem_base_sh)), "r"(2 * FE_TCOLS) : "memory");
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
            int kbg = 0;
            for (int tile = blockIdx.x; tile < a.n_tiles && !*vfail; tile += gridDim.x) {
                const int m0 = tile_rt(a, tile) * 128, n0 = tile_ct(a, tile) * a.GPT * NCf;
                for (int kb = 0; kb < nkb; ++kb, ++kbg) {
                    const int s = kbg % FE_STAGES;
                    if (!mbar_wait(&empty_bar[s], ((kbg / FE_STAGES) & 1) ^ 1, wb) || *vfail) {
                        *vfail = 1;
                        atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
                        break;
                    }
                    uint8_t* st = smem + (size_t)s * STAGE_BYTES;
                    mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                    const int kx = kb * 16;
                    tma_load_2d(st, &ta_hi, &full_bar[s], kx, m0);
                    tma_load_2d(st + FE_A_BYTES, &ta_lo, &full_bar[s], kx, m0);
                    tma_load_2d(st + 2 * FE_A_BYTES, &tb_hi, &full_bar[s], kx, n0);
                    tma_load_2d(st + 2 * FE_A_BYTES + B_BYTES, &tb_lo, &full_bar[s], kx, n0);
                }
            }
            // the copies issued last must land before the CTA may exit
            for (int k = kbg - FE_STAGES < 0 ? 0 : kbg - FE_STAGES; k < kbg; ++k)
                mbar_drain(&full_bar[k % FE_STAGES], (k / FE_STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------------------------ MMA issuer
            const uint32_t idesc = idesc_tf32(128, a.BNe);
            int kbg = 0, it = 0;
            for (int tile = blockIdx.x; tile < a.n_tiles && !*vfail; tile += gridDim.x, ++it) {
                const int b = it & 1;
                if (!mbar_wait(&tempty[b], ((it >> 1) & 1) ^ 1, wb)) {
                    *vfail = 1;
                    atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * FE_TCOLS);
                bool ok = true;
                for (int kb = 0; kb < nkb; ++kb, ++kbg) {
                    const int s = kbg % FE_STAGES;
                    if (!mbar_wait(&full_bar[s], (kbg / FE_STAGES) & 1, wb) || *vfail) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(smem + (size_t)s * STAGE_BYTES);
                    const int nk = min(2, (a.K - kb * 16) / 8);
                    for (int kk = 0; kk < nk; ++kk) {   // 2 x 32 bytes of K per k-block
                        const uint64_t ah = sw64_desc(sa + kk * 32);
                        const uint64_t al = sw64_desc(sa + FE_A_BYTES + kk * 32);
                        const uint64_t bh = sw64_desc(sa + 2 * FE_A_BYTES + kk * 32);
                        const uint64_t bl = sw64_desc(sa + 2 * FE_A_BYTES + B_BYTES + kk * 32);
                        mma_tf32(acc, ah, bh, idesc, (kb | kk) != 0);
                        mma_tf32(acc, ah, bl, idesc, 1u);
                        mma_tf32(acc, al, bh, idesc, 1u);
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) {
                    *vfail = 1;
                    atomicOr(a.err, MSD_DEV_ERR_TIMEOUT);
                    break;
                }
                mma_commit(&tfull[b]);
            }
            // every product issued by this thread completes before TMEM is freed
            mma_commit(&drain_bar);
            mbar_drain(&drain_bar, 0);
        }
    } else {
        // ---------------------------------------------------- epilogue
        const int et = threadIdx.x - 64, ew = et >> 5;
        const int q = warp & 3, set = ew >> 2;
        const int bq = lane / RB, j = lane % RB;
        const int bt = q * (32 / RB) + bq, wi = bt >> 1, c = bt & 1;
        const int pbar = 2 + set * 2 + wi;            // pair barrier id (RB = 32 only): 2 .. 7
        constexpr int SP = RB + 2;                    // pitch = 2 mod 4: conflict-free 64-bit row access
        float* slot = slots + (size_t)(set * WPT + wi) * a.slot;
        float* S0 = slot;                             // [RB][SP] dT real part
        float* S1 = slot + RB * SP;                   // [RB][SP] dT imaginary part
        float* FP = S1 + RB * SP;                     // [2][np][RB] F_P parts
        float2* XiRow = reinterpret_cast<float2*>(FP);   // later [RB][np] Xi, complex, row-major
        float* LamRe = FP + 2 * np * RB;              // [np][RB] Lambda, transposed
        float* LamIm = LamRe + np * RB;
        // [RB][np] Lambda, complex, row-major: the output reads the entries
        // (pos(h), p) of consecutive (h, p) from consecutive words
        float2* LamRow = reinterpret_cast<float2*>(LamIm + np * RB);
        float* scal = slot + a.slot - 16;             // [2][8] trace partials of the two parts
        // this part's particles: Lambda for [l0, l1) (and np - 1 when lx),
        // Xi for [x0, x1). With the traces the imaginary part, which has
        // less trace work, takes the larger half of both. Without them an
        // odd last particle is split: its Lambda goes to the real part, its
        // Xi (which needs the whole Lambda column, complete at the barrier
        // between the two phases) to the imaginary part.
        const int ph = np >> 1;
        const bool split_last = !XTR && (np & 1);
        const int l0 = c ? ph : 0, l1 = c ? np - (split_last ? 1 : 0) : ph;
        const bool lx = split_last && c == 0;
        const int x0 = c ? ph : 0, x1 = c ? np : ph;
        // this set's sequence of vectors: (tile, gl) for gl = set, set + FE_SETS, ...
        // with g = ct(tile) GPT + gl < n_chol, tiles in this CTA's order
        auto next_vec = [&](int& tile, int& gl) {
            gl += FE_SETS;
            if (gl >= a.GPT || tile_ct(a, tile) * a.GPT + gl >= a.n_chol) {
                tile += gridDim.x;
                gl = set;
                if (tile < a.n_tiles && (gl >= a.GPT || tile_ct(a, tile) * a.GPT + gl >= a.n_chol)) tile = a.n_tiles;
            }
        };
        // F0 block of vector g (the same layout in global and shared memory)
        // into buffer k of this set, in 16-byte pieces
        const int st_t = (ew & 3) * 32 + lane;        // thread index within the set
        auto prefetch = [&](int tile, int gl, int k) {
            if (tile >= a.n_tiles) return;
            const float* src = a.F0P + (size_t)(tile_ct(a, tile) * a.GPT + gl) * a.f0s;
            float* dst = f0buf + (set * 2 + k) * a.f0s;
            for (int e = st_t * 4; e < a.f0s; e += 128 * 4) cp_async16(dst + e, src + e);
            cp_async_commit();
        };
        // G block of a tile: cp.async of its valid entries into the stage,
        // then (each thread its own entries) FP32 parts into buffer b
        auto g_issue = [&](int tile) {
            if (tile >= a.n_tiles) return;
            const int rt = tile_rt(a, tile);
            for (int e = et; e < GE; e += FE_EPI) {
                const int wj = e / (np * RB), r = e % (np * RB), p = r / RB, l = r % RB;
                const int ww = rt * WPT + wj;
                if (ww < a.nw && l < N) cp_async16(gst + e, a.Gr + ((size_t)ww * N + l) * a.M + a.tb.part_orb[p]);
            }
            cp_async_commit();
        };
        auto g_convert = [&](int tile, int b) {
            const int rt = tile_rt(a, tile);
            float* gr = gpRe + b * GE;
            float* gi = gpIm + b * GE;
            for (int e = et; e < GE; e += FE_EPI) {
                const int wj = e / (np * RB), l = e % RB;
                const bool v = rt * WPT + wj < a.nw && l < N;
                const double2 d = v ? gst[e] : make_double2(0.0, 0.0);
                gr[e] = (float)d.x;
                gi[e] = (float)d.y;
            }
        };
        g_issue(blockIdx.x);
        int pf_tile = blockIdx.x, pf_gl = set;       // the next vector to prefetch
        if (pf_tile < a.n_tiles && (pf_gl >= a.GPT || tile_ct(a, pf_tile) * a.GPT + pf_gl >= a.n_chol))
            pf_tile = a.n_tiles;
        if constexpr (XTR) {
            prefetch(pf_tile, pf_gl, 0);
            next_vec(pf_tile, pf_gl);
        }
        int it = 0, vc = 0;
        for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
            const int b = it & 1, rt = tile_rt(a, tile), ct = tile_ct(a, tile);
            const float* gbr = gpRe + b * GE;
            const float* gbi = gpIm + b * GE;
            // G[occ0_l][P_p] of the tile's walkers, transposed and zero padded
            // to RB rows, from this thread's own copies of the FP64 block;
            // double buffered by tile parity (the sets may be one tile apart)
            cp_async_wait_all();
            g_convert(tile, b);
            bool ok = mbar_wait(&tfull[b], (it >> 1) & 1, wb);
            ok = bar_and(1, FE_EPI, ok && !*vfail);
            if (!ok) {
                if (et == 0) { *vfail = 1; atomicOr(a.err, MSD_DEV_ERR_TIMEOUT); }
                break;
            }
            tc_fence_after();
            // every set is past the previous tile: the stage is free for the next one
            g_issue(tile + gridDim.x);
            const int w = rt * WPT + wi;
            const bool wv = w < a.nw;
            const float* gwr = gbr + wi * np * RB;
            const float* gwi = gbi + wi * np * RB;
            for (int gl = set; gl < a.GPT; gl += FE_SETS, ++vc) {
                const int g = ct * a.GPT + gl;
                if (g >= a.n_chol) break;
                // this vector's F0 block has landed (own copies, then the set's)
                const float* f0 = f0buf + (set * 2 + (vc & 1)) * a.f0s;   // T0[j][l] = f0[j NCP + l]
                if constexpr (XTR) {
                    cp_async_wait_all();
                    bar_sync(8 + set, 128);
                    prefetch(pf_tile, pf_gl, (vc + 1) & 1);
                    next_vec(pf_tile, pf_gl);
                }
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * FE_TCOLS + gl * NCf);
                // -- this part's rows: dT (columns occ0, zero padded to RB) and dF_P;
                // dT rows and the F_P parts (real part with F0) into the slot
                float t[RB];
                tmem_ld_row<RB>(taddr, t);
                float* Sc = c ? S1 : S0;
                float s_0 = 0.f;   // sum_l dTc[j][l] T0[l][j]
                {
                    float fp[PW];
                    tmem_ld16(taddr + (uint32_t)RB, fp);
                    float z0 = 0.f, z1 = 0.f;
#pragma unroll
                    for (int l = 0; l < RB; l += 2) {
                        *reinterpret_cast<float2*>(Sc + j * SP + l) = make_float2(t[l], t[l + 1]);
                        if constexpr (XTR) {
                            z0 = fmaf(t[l], f0[l * NCP + j], z0);
                            z1 = fmaf(t[l + 1], f0[(l + 1) * NCP + j], z1);
                        }
                    }
                    s_0 = z0 + z1;
#pragma unroll
                    for (int p = 0; p < PW; ++p)
                        if (p < np) FP[(c * np + p) * RB + j] = (c || !XTR) ? fp[p] : fp[p] + f0[j * NCP + RB + p];
                }
                pair_sync<RB>(pbar);
                // -- traces from the rows and columns of S. real: s_a = sum_l A[j][l] A[l][j],
                // s_b = sum_l A[j][l] B[l][j]; imaginary: s_b = sum_l B[j][l] B[l][j]
                float s_diag, s_a = 0.f, s_b = 0.f;
                if constexpr (!XTR) {
                    s_diag = Sc[j * SP + j];   // written by this lane above
                } else {
                    const float* row = Sc + j * SP;
                    float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll 4
                    for (int l = 0; l < RB; l += 2) {
                        const float2 rr = *reinterpret_cast<const float2*>(row + l);
                        const float r0 = rr.x, r1 = rr.y;
                        b0 = fmaf(r0, S1[l * SP + j], b0);
                        b1 = fmaf(r1, S1[(l + 1) * SP + j], b1);
                        if (c == 0) {
                            a0 = fmaf(r0, S0[l * SP + j], a0);
                            a1 = fmaf(r1, S0[(l + 1) * SP + j], a1);
                        }
                    }
                    s_diag = row[j];
                    s_a = a0 + a1;
                    s_b = b0 + b1;
                }
#pragma unroll
                for (int o = RB >> 1; o; o >>= 1) {
                    s_diag += __shfl_xor_sync(0xffffffffu, s_diag, o);
                    if constexpr (XTR) {
                        s_a += __shfl_xor_sync(0xffffffffu, s_a, o);
                        s_b += __shfl_xor_sync(0xffffffffu, s_b, o);
                        s_0 += __shfl_xor_sync(0xffffffffu, s_0, o);
                    }
                }
                if (j == 0) {
                    scal[c * 8 + 0] = s_diag;
                    scal[c * 8 + 1] = s_0;
                    scal[c * 8 + 2] = s_a;
                    scal[c * 8 + 3] = s_b;
                }
                // -- the complex row T[j][:] = (T0 + dT_re) + i dT_im as FP32 pairs: this
                // part's half from t, the other part's from S (without XTR the real
                // part already holds T0). (The warp barrier keeps these loads out of
                // the trace phase's register budget.)
                __syncwarp();
                unsigned long long trp[RB / 2], tip[RB / 2];
                {
                    const unsigned long long* So =
                        reinterpret_cast<const unsigned long long*>((c ? S0 : S1) + j * SP);
                    const unsigned long long* fr = reinterpret_cast<const unsigned long long*>(f0 + j * NCP);
#pragma unroll
                    for (int k = 0; k < RB / 2; ++k) {
                        const unsigned long long m = pack2(t[2 * k], t[2 * k + 1]), o = So[k];
                        if constexpr (XTR) trp[k] = add2(c ? o : m, fr[k]);   // T0 + dT_re
                        else trp[k] = c ? o : m;
                        tip[k] = c ? m : o;
                    }
                }
                // -- Lambda[j][p] = F_P[j][p] - sum_l T[j][l] G[occ0_l][P_p], this
                // part's particles (rows j >= N: zero rows of F and T give zero)
                for (int u = l0; u < l1 + (lx ? 1 : 0); ++u) {
                    const int p = u < l1 ? u : np - 1;
                    const float2 d = cdot_row<RB>(trp, tip, gwr + p * RB, gwi + p * RB);
                    const float lr = FP[p * RB + j] - d.x, li = FP[(np + p) * RB + j] - d.y;
                    LamRe[p * RB + j] = lr;
                    LamIm[p * RB + j] = li;
                    LamRow[j * np + p] = make_float2(lr, li);
                }
                pair_sync<RB>(pbar);   // Lambda complete; F_P and S reads done
                // -- Xi[j][p] = sum_l T[j][l] Lambda[l][p] (all rows; holes kept), over
                // the F_P parts (read by both parts before the barrier above)
                for (int p = x0; p < x1; ++p)
                    XiRow[j * np + p] = cdot_row<RB>(trp, tip, LamRe + p * RB, LamIm + p * RB);
                pair_sync<RB>(pbar);   // Xi complete
                if (wv) {
                    // whole 128-byte lines (the row pitch XS; zeros past X), so that
                    // no partly written line is filled from DRAM; evict-first, so
                    // that the output stream does not push the operands out of L2
                    const size_t wg = (size_t)w * a.n_chol + g;
                    const int XS = lam_pitch(X);
                    for (int e = c * RB + j; e < XS; e += 2 * RB) {
                        float2 lv = make_float2(0.f, 0.f), xv = lv;
                        if (e < X) {
                            const int o = oe[e];
                            lv = LamRow[o];
                            xv = XiRow[o];
                        }
                        __stcs(&a.Lact[wg * XS + e], lv);
                        __stcs(&a.Xic[wg * XS + e], xv);
                    }
                    if (c == 0 && j == 0) {
                        // real part: diag A, T0.A, A.A, A.B; imaginary part: diag B, T0.B, -, B.B
                        const float ad = scal[0], t0a = scal[1], aa = scal[2], ab = scal[3];
                        const float bd = scal[8], t0b = scal[9], bb = scal[11];
                        a.v0[wg] = make_double2(XTR ? a.c0[g] + (double)ad : (double)ad, (double)bd);
                        if constexpr (XTR)
                            a.xx[wg] = make_double2(a.x0[g] + (double)(2.f * t0a + aa - bb), (double)(2.f * (t0b + ab)));
                    }
                }
                pair_sync<RB>(pbar);   // the slot is free for the next vector
            }
            // accumulator b fully read by this warp: the MMA warp may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
        }
        cp_async_wait_all();   // no copy into shared memory outlives the CTA
    }
    __syncwarp();   // single-lane roles rejoin their warps
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * FE_TCOLS)
                     : "memory");
}


}  // namespace

// Tile shape of the fused kernel for one spin; false when the shape is not
// supported (N > 32, np > 16, nh np > 128, or no B tile width leaves the
// epilogue's shared memory within 227 KB), in which case the caller takes
// the unfused GEMM + epilogue.
bool tc_fepi_plan(const SpinTables& tb, TcFepiPlan& p)
{
    const int N = tb.N, np = tb.np;
    if (N < 1 || N > 32 || np < 1 || np > 16 || tb.nh * np > FE_XMAX) return false;
    p.RB = N <= 8 ? 8 : N <= 16 ? 16 : 32;
    p.RW = 2 * p.RB;
    p.WPT = 64 / p.RB;
    p.NCf = p.RB + np;                               // B rows per vector: occ0 padded to RB, particles
    // per-walker slot: the two [RB][RB + 2] dT parts, the F_P parts
    // [2][np][RB] (later Xi as [RB][np] complex), Lambda^T as [np][RB] real and
    // imaginary rows, Lambda as [RB][np] complex, 16 scalars
    p.slot = 2 * p.RB * (p.RB + 2) + 6 * np * p.RB + 16;
    p.NCP = (p.NCf + 1) / 4 * 4 + 2;                 // = 2 mod 4: conflict-free 64-bit row reads
    p.f0s = (p.RB * p.NCP + 3) / 4 * 4;
    // columns read per vector: RB from its start (occ0 part) and 16 from
    // its particle part, inside the buffer's 256 TMEM columns
    const int span = p.RB + 16;
    for (int BN = FE_TCOLS; BN >= 16 && BN >= span; BN -= 16) {
        int gpt = (BN - span) / p.NCf + 1;
        if (gpt >= FE_SETS) gpt -= gpt % FE_SETS;    // a multiple of the sets: balanced epilogue
        const int bn = std::max(16, std::min(BN, ((gpt - 1) * p.NCf + span + 15) / 16 * 16));
        const size_t smem = 1024 + (size_t)FE_STAGES * 2 * (FE_A_BYTES + (size_t)bn * 64) +
                            4 * (size_t)FE_SETS * p.WPT * p.slot + 4 * (size_t)4 * p.WPT * np * p.RB +
                            4 * (size_t)FE_SETS * 2 * p.f0s + 4 * FE_XMAX +
                            16 * ((size_t)p.WPT * np * p.RB + 1);   // G block stage, 16-byte aligned
        if (smem + 128 > 227 * 1024) continue;   // 128: static shared memory of the kernel
        p.BN = bn;
        p.GPT = gpt;
        p.BNe = std::min(bn, (gpt * p.NCf + 15) / 16 * 16);
        p.smem = smem;
        return true;
    }
    return false;
}

int tc_fepi_fused(const SpinTables& tb, const TcFepiPlan& p, int nw, int M, int n_chol, const float* a_hi,
                  const float* a_lo, const float* b_hi, const float* b_lo, int ld, int K, const double2* Gr,
                  const float* F0P, const double* c0, const double* x0, double2* v0, double2* xx,
                  float2* Lact, float2* Xic, unsigned* err, cudaStream_t st, bool traces)
{
    if (nw <= 0 || n_chol <= 0) return 0;
    if (K < 8 || K % 8 || K > ld || ld % 4) return -1;
    CUtensorMap ah, al, bh, bl;
    if (tc_make_map(&ah, a_hi, K, nw * p.RW, ld, 128, false, 64) ||
        tc_make_map(&al, a_lo, K, nw * p.RW, ld, 128, false, 64) ||
        tc_make_map(&bh, b_hi, K, n_chol * p.NCf, ld, p.BN, false, 64) ||
        tc_make_map(&bl, b_lo, K, n_chol * p.NCf, ld, p.BN, false, 64))
        return -1;
    FeArgs a;
    a.tb = tb;
    a.nw = nw; a.M = M; a.n_chol = n_chol; a.K = K;
    a.BN = p.BN; a.GPT = p.GPT; a.BNe = p.BNe; a.slot = p.slot; a.NCf = p.NCf; a.NCP = p.NCP; a.f0s = p.f0s;
    a.n_rt = (nw + p.WPT - 1) / p.WPT;
    a.n_ct = (n_chol + p.GPT - 1) / p.GPT;
    a.n_tiles = a.n_rt * a.n_ct;
    a.Gr = Gr; a.F0P = F0P; a.c0 = c0; a.x0 = x0;
    a.v0 = v0; a.xx = xx; a.Lact = Lact; a.Xic = Xic; a.err = err;
    const int grid = std::min(a.n_tiles, msd_sm_count());
    auto go = [&](auto kern) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess)
            return -1;
        kern<<<grid, FE_THREADS, p.smem, st>>>(ah, al, bh, bl, a);
        return 0;
    };
    int rc;
    if (traces) rc = p.RB == 32 ? go(k_tc_fepi<32, true>) : p.RB == 16 ? go(k_tc_fepi<16, true>) : go(k_tc_fepi<8, true>);
    else rc = p.RB == 32 ? go(k_tc_fepi<32, false>) : p.RB == 16 ? go(k_tc_fepi<16, false>) : go(k_tc_fepi<8, false>);
    if (rc) return rc;
    msd_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
