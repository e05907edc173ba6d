// Opposite-spin exchange term of the local energy (the alpha-beta part of the
// two-body Wick contraction, Sec. III, fill_os) over runs of determinants
// that share one string:
//   sum_I c_I r_a r_b X_ab,
//   X_ab = sum_{e, f} Ba[e] Bb[f] K^ab[x_e][y_f]
// (e over the alpha minor's entries (i, j), x_e = h_j np + p_i its Gram row;
// f likewise for beta). Within one excitation-level bucket the determinants
// are ordered so that those sharing the projected string s (alpha or beta,
// chosen per bucket when the trial is set) are consecutive. For a run of
// them the projection
//   P_s[y] = sum_e Bs[e] K[x_e][y]          (all y of the other spin)
// is formed once, with the lanes of a warp over y (contiguous rows of K in
// shared memory, no bank conflicts); each determinant of the run then needs
// only the k_o^2 entries of the other string:
//   c_I r_s r_o sum_f Bo[f] P_s[y_f].
// The lanes walk the run's (determinant, entry) pairs, so a determinant's
// entries are read by neighbouring lanes (contiguous loads) and no
// per-determinant reduction is needed (the sum is linear in the pairs). Same
// value as k_pair_cross up to the order of the sums in the working
// precision T.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

#define PR_THREADS 256
#define PR_WARPS (PR_THREADS / 32)
#define PR_RPW 8                       // runs per warp and block
#define PR_RPB (PR_WARPS * PR_RPW)     // runs per block
#define PR_QMAX ((MSD_XMAX + 31) / 32) // 32-lane chunks of the projected row

template <bool SIDE_B, typename T>
__global__ void __launch_bounds__(PR_THREADS)
k_pair_run(SpinTables ta, SpinTables tbb, PairTables pt, int bidx, int ka, int kb, int hi,
           const void* __restrict__ ra_in, const void* __restrict__ rb_in, const void* __restrict__ Ba_in,
           const void* __restrict__ Bb_in, const void* __restrict__ Kin, double2* __restrict__ part, int nslot,
           int slot0)
{
    using T2 = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    // projected side s, other side o
    const SpinTables& ts = SIDE_B ? tbb : ta;
    const SpinTables& to = SIDE_B ? ta : tbb;
    const int ks = SIDE_B ? kb : ka, ko = SIDE_B ? ka : kb;
    const int Xa = ta.nh * ta.np, Xb = tbb.nh * tbb.np;
    const int Xs = SIDE_B ? Xb : Xa, Xo = SIDE_B ? Xa : Xb;
    T2* Kp = reinterpret_cast<T2*>(smraw);                 // [Xs][Xo]: rows of the projected side
    T2* pw = Kp + (size_t)Xs * Xo;                         // [PR_WARPS][32 PR_QMAX]
    __shared__ double2 red[PR_WARPS];
    const int w = blockIdx.y, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const T2* Kw = reinterpret_cast<const T2*>(Kin) + (size_t)w * Xa * Xb;
    for (int e = t; e < Xa * Xb; e += PR_THREADS) {
        const int x = e / Xb, y = e - x * Xb;
        if (SIDE_B) Kp[(size_t)y * Xa + x] = Kw[e];
        else Kp[e] = Kw[e];
    }
    __syncthreads();
    const int* runs = pt.runs + pt.run_off[bidx];
    const int n_runs = pt.run_off[bidx + 1] - pt.run_off[bidx];
    const T2* rs_arr = reinterpret_cast<const T2*>(SIDE_B ? rb_in : ra_in);
    const T2* ro_arr = reinterpret_cast<const T2*>(SIDE_B ? ra_in : rb_in);
    const T2* Bs_all = reinterpret_cast<const T2*>(SIDE_B ? Bb_in : Ba_in);
    const T2* Bo_all = reinterpret_cast<const T2*>(SIDE_B ? Ba_in : Bb_in);
    const int ns_s = ts.bucket[ks + 1] - ts.bucket[ks], ns_o = to.bucket[ko + 1] - to.bucket[ko];
    const int kks = ks * ks, kko = ko * ko;
    // a lane's first (determinant, entry) pair of a run and its step of 32
    const int dd0 = lane / kko, f0 = lane - dd0 * kko;
    const int ddq = 32 / kko, fq = 32 - ddq * kko;
    T2* P = pw + warp * 32 * PR_QMAX;
    T acc_r = 0, acc_i = 0;
    for (int u = 0; u < PR_RPW; ++u) {
        const int r = blockIdx.x * PR_RPB + warp + PR_WARPS * u;
        if (r >= n_runs) break;
        const int d0 = runs[r], d1 = r + 1 < n_runs ? runs[r + 1] : hi;
        const int s = SIDE_B ? pt.b[d0] : pt.a[d0];
        const int sl = s - ts.bucket[ks];
        // the projected string's minor entries and Gram rows, one per lane
        T2 be = T2{0, 0};
        int xe = 0;
        if (lane < kks) {
            be = Bs_all[(size_t)ts.b_off[ks] + ((size_t)w * ns_s + sl) * b_stride(ks) + lane];
            xe = ts.kx[ts.cmx_off[ks] + (size_t)sl * kks + lane] * Xo;
        }
        T2 pq[PR_QMAX];
#pragma unroll
        for (int q = 0; q < PR_QMAX; ++q) pq[q] = T2{0, 0};
        for (int e = 0; e < kks; ++e) {
            const T br = __shfl_sync(0xffffffffu, be.x, e), bi = __shfl_sync(0xffffffffu, be.y, e);
            const T2* row = Kp + __shfl_sync(0xffffffffu, xe, e) + lane;
#pragma unroll
            for (int q = 0; q < PR_QMAX; ++q)
                if (32 * q + lane < Xo) {
                    const T2 kv = row[32 * q];
                    pq[q].x += br * kv.x - bi * kv.y;
                    pq[q].y += br * kv.y + bi * kv.x;
                }
        }
#pragma unroll
        for (int q = 0; q < PR_QMAX; ++q)
            if (32 * q + lane < Xo) P[32 * q + lane] = pq[q];
        const T2 rs = rs_arr[(size_t)w * ts.n_str + s];
        __syncwarp();
        // the run's (determinant, entry) pairs, the entries of one
        // determinant on neighbouring lanes (their loads contiguous)
        int d = d0 + dd0, f = f0;
        while (d < d1) {
            const int o = SIDE_B ? pt.a[d] : pt.b[d];
            const int so = o - to.bucket[ko];
            const T2 bo = Bo_all[(size_t)to.b_off[ko] + ((size_t)w * ns_o + so) * b_stride(ko) + f];
            const T2 pv = P[to.kx[to.cmx_off[ko] + (size_t)so * kko + f]];
            const T2 ro = ro_arr[(size_t)w * to.n_str + o];
            const T c = std::is_same<T, float>::value ? (T)pt.cf[d] : (T)pt.c[d];
            // c r_s r_o (Bo P)
            const T wr = c * (rs.x * ro.x - rs.y * ro.y), wi = c * (rs.x * ro.y + rs.y * ro.x);
            const T vr = bo.x * pv.x - bo.y * pv.y, vi = bo.x * pv.y + bo.y * pv.x;
            acc_r += wr * vr - wi * vi;
            acc_i += wr * vi + wi * vr;
            d += ddq;
            f += fq;
            if (f >= kko) { f -= kko; ++d; }
        }
        __syncwarp();   // P consumed before the next run overwrites it
    }
    double sr = acc_r, si = acc_i;
    for (int o = 16; o; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) red[warp] = cz(sr, si);
    __syncthreads();
    if (t == 0) {
        double2 v = red[0];
        for (int q = 1; q < PR_WARPS; ++q) v = cadd(v, red[q]);
        part[(size_t)w * nslot + slot0 + blockIdx.x] = v;
    }
}

int pair_run_blocks(const PairTables& pt, int bidx)
{
    const int n = pt.run_off[bidx + 1] - pt.run_off[bidx];
    return n > 0 ? (n + PR_RPB - 1) / PR_RPB : 0;
}

size_t pair_run_smem(const SpinTables& ta, const SpinTables& tb, bool fp32)
{
    const size_t e = fp32 ? sizeof(float2) : sizeof(double2);
    return e * ((size_t)(ta.nh * ta.np) * (tb.nh * tb.np) + (size_t)PR_WARPS * 32 * PR_QMAX);
}

void launch_pair_run(const SpinTables& ta, const SpinTables& tb, const PairTables& pt, int bidx, int ka, int kb,
                     int nw, const void* ra, const void* rb, const void* Ba, const void* Bb, const void* K, bool fp32,
                     double2* part, int nslot, int slot, cudaStream_t st)
{
    const int nb = pair_run_blocks(pt, bidx);
    if (nb <= 0 || nw <= 0) return;
    const bool side_b = pt.run_side[bidx] == 2;
    const int hi = pt.bucket[bidx + 1];
    const size_t smem = pair_run_smem(ta, tb, fp32);
    dim3 grid(nb, nw);
#define PR_GO(SB, TT)                                                                                          \
    do {                                                                                                       \
        cudaFuncSetAttribute(k_pair_run<SB, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
        k_pair_run<SB, TT><<<grid, PR_THREADS, smem, st>>>(ta, tb, pt, bidx, ka, kb, hi, ra, rb, Ba, Bb, K,    \
                                                           part, nslot, slot);                                 \
    } while (0)
    if (fp32) {
        if (side_b) PR_GO(true, float); else PR_GO(false, float);
    } else {
        if (side_b) PR_GO(true, double); else PR_GO(false, double);
    }
#undef PR_GO
    msd_note_launch();
}
