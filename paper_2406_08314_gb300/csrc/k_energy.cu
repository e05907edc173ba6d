// Local-energy and force-bias contractions (Sec. III: fill_os / get_ss, and
// the force bias of Eq. 7), FP64 path.
//
// With G = G0^T (rows occ0 non-zero), B_s = A_s^-1 for an excitation string s
// with holes h_1..h_k and particles p_1..p_k, and
//   Lambda_g = G L_g (I - G),  Xi = sum_g G L_g G L_g (I - G),
//   K^{st}[(h,p)][(h',p')] = sum_g Lambda^s_g[h][p] Lambda^t_g[h'][p'],
//   u^s = sum_g V0_g Lambda^s_g,  V0_g = sum_s tr(L_g G^s),
// the determinant I = (a, b) has local energy
//   E_I = E_0 + e_a + e_b + X_ab,
//   E_0 = e0 + sum_s tr(h G^s) + 1/2 sum_g V0_g^2 - 1/2 sum_s sum_g tr(L_g G^s L_g G^s)
//   e_s = sum_ij B[i][j] Y[h_j][p_i] + 1/2 (Qc - Qx),   Y = Lambda_h + u - Xi
//   Qc = sum_ijkl B_ij B_kl K[(h_j,p_i)][(h_l,p_k)],  Qx = ... K[(h_j,p_k)][(h_l,p_i)]
//   X_ab = sum_ijkl Ba_ij Bb_kl K^{ab}[(ha_j,pa_i)][(hb_l,pb_k)]
// (the generalized Wick theorem of Sec. II A applied to the rank-k update
// G_I = G + (E_P - G[:,P]) B G[H,:]), and E_L = sum_I c_I r_I E_I / sum_I c_I r_I.
#include <type_traits>

#include "common.cuh"
#include "det_terms.cuh"
#include "kernels.h"

// ------------------------------------------------------------------------
// C[m][n] = sum_k A[m][k] * B[n][k], A complex, B real, FP64.
// 64 x 64 tile, k-step 16, 256 threads with a 4 x 4 register block each.
__global__ void __launch_bounds__(256)
k_gemm_zd(int Mr, int Nc, int K, const double2* __restrict__ A, long long lda,
          const double* __restrict__ B, long long ldb, double2* __restrict__ C, long long ldc)
{
    __shared__ double2 As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cz(0, 0);
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = threadIdx.x + q * 256;
            const int rr = e / 16, kk = e % 16;
            const int m = m0 + rr, n = n0 + rr, k = k0 + kk;
            As[kk][rr] = (m < Mr && k < K) ? A[(size_t)m * lda + k] : cz(0, 0);
            Bs[kk][rr] = (n < Nc && k < K) ? B[(size_t)n * ldb + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double2 a[4]; double b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(a[i].x, b[j], acc[i][j].x);
                    acc[i][j].y = fma(a[i].y, b[j], acc[i][j].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= Mr) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n < Nc) C[(size_t)m * ldc + n] = acc[i][j];
        }
    }
}

void launch_gemm_zd(int Mr, int Nc, int K, const double2* A, long long lda, const double* B,
                    long long ldb, double2* C, long long ldc, cudaStream_t st)
{
    dim3 grid((Nc + 63) / 64, (Mr + 63) / 64);
    k_gemm_zd<<<grid, 256, 0, st>>>(Mr, Nc, K, A, lda, B, ldb, C, ldc); msd_note_launch();
}

// ------------------------------------------------------------------------
// Per (walker, Cholesky vector) epilogue of F = G L_g restricted to rows
// occ0 and columns occ0 u P (F[j][c] = (G L_g)[occ0_j][col_c]):
//   T = F[:, occ0],  v0 = tr T,  x = tr(T T) = tr(L G L G)
//   Lambda[j][p] = F[j][P_p] - sum_l T[j][l] G[occ0_l][P_p]
//   Lact[(h,p)] = Lambda[pos(h)][p],  Xic[(h,p)] = sum_l T[pos(h)][l] Lambda[l][p]
__global__ void __launch_bounds__(128)
k_fepi(SpinTables tb, int M, int n_chol, const double2* __restrict__ F, long long ldf,
       const double2* __restrict__ Gr, double2* __restrict__ v0, double2* __restrict__ xx,
       double2* __restrict__ Lact, double2* __restrict__ Xic)
{
    extern __shared__ double2 sm[];
    const int N = tb.N, np = tb.np, nh = tb.nh, NC = N + np, X = nh * np;
    double2* f = sm;                 // [N][NC]
    double2* gp = f + N * NC;        // [N][np]
    double2* lam = gp + N * np;      // [N][np]
    __shared__ double2 red[2][128];
    const int g = blockIdx.x, w = blockIdx.y, t = threadIdx.x;
    const double2* Fw = F + (size_t)w * N * ldf + (size_t)g * NC;
    for (int e = t; e < N * NC; e += blockDim.x) f[e] = Fw[(size_t)(e / NC) * ldf + e % NC];
    const double2* gr = Gr + (size_t)w * N * M;
    for (int e = t; e < N * np; e += blockDim.x) gp[e] = gr[(size_t)(e / np) * M + tb.part_orb[e % np]];
    __syncthreads();
    double2 a0 = cz(0, 0), a1 = cz(0, 0);
    for (int e = t; e < N * N; e += blockDim.x) {
        const int j = e / N, l = e % N;
        a1 = cfma(f[j * NC + l], f[l * NC + j], a1);
        if (j == l) a0 = cadd(a0, f[j * NC + j]);
    }
    for (int e = t; e < N * np; e += blockDim.x) {
        const int j = e / np, p = e % np;
        double2 v = f[j * NC + N + p];
        for (int l = 0; l < N; ++l) v = cfms(f[j * NC + l], gp[l * np + p], v);
        lam[e] = v;
    }
    red[0][t] = a0; red[1][t] = a1;
    __syncthreads();
    for (int o = 64; o; o >>= 1) {
        if (t < o) { red[0][t] = cadd(red[0][t], red[0][t + o]); red[1][t] = cadd(red[1][t], red[1][t + o]); }
        __syncthreads();
    }
    const size_t wg = (size_t)w * n_chol + g;
    if (t == 0) { v0[wg] = red[0][0]; xx[wg] = red[1][0]; }
    for (int e = t; e < X; e += blockDim.x) {
        const int h = e / np, p = e % np, j = tb.hole_pos[h];
        double2 xi = cz(0, 0);
        for (int l = 0; l < N; ++l) xi = cfma(f[j * NC + l], lam[l * np + p], xi);
        Lact[wg * X + e] = lam[j * np + p];
        Xic[wg * X + e] = xi;
    }
}

size_t fepi_smem(const SpinTables& tb) { return sizeof(double2) * (tb.N * (tb.N + tb.np) + 2 * tb.N * tb.np); }

void launch_fepi(const SpinTables& tb, int nw, int M, int n_chol, const double2* F, long long ldf,
                 const double2* Gr, double2* v0, double2* xx, double2* Lact, double2* Xic,
                 cudaStream_t st)
{
    dim3 grid(n_chol, nw);
    const size_t smem = fepi_smem(tb);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_fepi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fepi<<<grid, 128, smem, st>>>(tb, M, n_chol, F, ldf, Gr, v0, xx, Lact, Xic); msd_note_launch();
}

// ------------------------------------------------------------------------
// One-body pieces per (walker, spin): e1 = tr(h G), and
// Lambda_h[(h,p)] = (G hl (I - G))[H_h][P_p] with hl = h, or the matrix the
// caller gives (linear in it: hl = h + J adds sum_g C_g Lambda_g).
__global__ void __launch_bounds__(128)
k_onebody(SpinTables tb, int M, const double* __restrict__ h1, const double* __restrict__ hl,
          const double2* __restrict__ Gr, double2* __restrict__ e1, double2* __restrict__ Lh)
{
    extern __shared__ double2 sm[];
    const int N = tb.N, np = tb.np, nh = tb.nh, NC = N + np;
    double2* fh = sm;   // [nh][NC]
    __shared__ double2 red[128];
    const int w = blockIdx.x, t = threadIdx.x;
    const double2* gr = Gr + (size_t)w * N * M;
    double2 a = cz(0, 0);
    for (int e = t; e < N * M; e += blockDim.x) {
        const int j = e / M, r = e % M;
        a = cadd(a, cscale(gr[e], h1[(size_t)tb.occ0[j] * M + r]));
    }
    for (int e = t; e < nh * NC; e += blockDim.x) {
        const int h = e / NC, c = e % NC;
        const int col = c < N ? tb.occ0[c] : tb.part_orb[c - N];
        const double2* gj = gr + (size_t)tb.hole_pos[h] * M;
        double2 v = cz(0, 0);
        for (int r = 0; r < M; ++r) v = cadd(v, cscale(gj[r], hl[(size_t)col * M + r]));
        fh[e] = v;
    }
    red[t] = a;
    __syncthreads();
    for (int o = 64; o; o >>= 1) {
        if (t < o) red[t] = cadd(red[t], red[t + o]);
        __syncthreads();
    }
    if (t == 0) e1[w] = red[0];
    for (int e = t; e < nh * np; e += blockDim.x) {
        const int h = e / np, p = e % np;
        double2 v = fh[h * NC + N + p];
        for (int l = 0; l < N; ++l) v = cfms(fh[h * NC + l], gr[(size_t)l * M + tb.part_orb[p]], v);
        Lh[(size_t)w * nh * np + e] = v;
    }
}

void launch_onebody(const SpinTables& tb, int nw, int M, const double* h1, const double2* Gr,
                    double2* e1, double2* Lh, cudaStream_t st, const double* hl)
{
    size_t smem = sizeof(double2) * tb.nh * (tb.N + tb.np);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_onebody, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_onebody<<<nw, 128, smem, st>>>(tb, M, h1, hl ? hl : h1, Gr, e1, Lh); msd_note_launch();
}

// ------------------------------------------------------------------------
// Sums over Cholesky vectors per (walker, spin):
//   Y[x] = Lh[x] + sum_g V0_g Lact_g[x] - sum_g Xic_g[x],  V0_g = v0a_g + v0b_g
//   scal[w][0 + s] = sum_g xx_g (exchange of G),  scal[w][2] = sum_g V0_g^2
template <typename TY>
__global__ void __launch_bounds__(128)
k_gamma_reduce(int X, int n_chol, int spin, const double2* __restrict__ v0a,
               const double2* __restrict__ v0b, const double2* __restrict__ xx,
               const double2* __restrict__ Lact, const double2* __restrict__ Xic,
               const double2* __restrict__ Lh, TY* __restrict__ Y, double2* __restrict__ scal)
{
    __shared__ double2 red[2][128];
    const int w = blockIdx.x, t = threadIdx.x;
    const size_t base = (size_t)w * n_chol;
    for (int x = t; x < X; x += blockDim.x) {
        double2 y = Lh[(size_t)w * X + x];
        for (int g = 0; g < n_chol; ++g) {
            const double2 V0 = cadd(v0a[base + g], v0b[base + g]);
            y = cfma(V0, Lact[(base + g) * X + x], y);
            y = csub(y, Xic[(base + g) * X + x]);
        }
        Y[2 * ((size_t)w * X + x)] = (TY)y.x;
        Y[2 * ((size_t)w * X + x) + 1] = (TY)y.y;
    }
    double2 s0 = cz(0, 0), s1 = cz(0, 0);
    for (int g = t; g < n_chol; g += blockDim.x) {
        s0 = cadd(s0, xx[base + g]);
        const double2 V0 = cadd(v0a[base + g], v0b[base + g]);
        s1 = cfma(V0, V0, s1);
    }
    red[0][t] = s0; red[1][t] = s1;
    __syncthreads();
    for (int o = 64; o; o >>= 1) {
        if (t < o) { red[0][t] = cadd(red[0][t], red[0][t + o]); red[1][t] = cadd(red[1][t], red[1][t + o]); }
        __syncthreads();
    }
    if (t == 0) {
        scal[(size_t)w * 8 + spin] = red[0][0];
        if (spin == 0) scal[(size_t)w * 8 + 2] = red[1][0];
    }
}

void launch_gamma_reduce(int nw, int X, int n_chol, int spin, const double2* v0a, const double2* v0b,
                         const double2* xx, const double2* Lact, const double2* Xic,
                         const double2* Lh, void* Y, bool fp32, double2* scal, cudaStream_t st)
{
    if (fp32)
        k_gamma_reduce<float><<<nw, 128, 0, st>>>(X, n_chol, spin, v0a, v0b, xx, Lact, Xic, Lh,
                                                  (float*)Y, scal);
    else
        k_gamma_reduce<double><<<nw, 128, 0, st>>>(X, n_chol, spin, v0a, v0b, xx, Lact, Xic, Lh,
                                                   (double*)Y, scal);
    msd_note_launch();
}

// ------------------------------------------------------------------------
// Gram matrices K[w][x][y] = sum_g P[w][g][x] Q[w][g][y] (complex, no
// conjugation) for one spin pair; 32 x 32 output tile per block.
template <typename TK>
__global__ void __launch_bounds__(256)
k_gram(int Xp, int Xq, int n_chol, const double2* __restrict__ P, const double2* __restrict__ Q,
       TK* __restrict__ Kout)
{
    __shared__ double2 ps[16][32], qs[16][32];
    const int w = blockIdx.z;
    const int x0 = blockIdx.y * 32, y0 = blockIdx.x * 32;
    const int t = threadIdx.x;
    const int ty = t / 16, tx = t % 16;      // 16 x 16 threads, 2 x 2 outputs each
    double2 acc[2][2] = {{cz(0, 0), cz(0, 0)}, {cz(0, 0), cz(0, 0)}};
    const double2* Pw = P + (size_t)w * n_chol * Xp;
    const double2* Qw = Q + (size_t)w * n_chol * Xq;
    for (int g0 = 0; g0 < n_chol; g0 += 16) {
        for (int e = t; e < 16 * 32; e += 256) {
            const int gg = e / 32, xx = e % 32, g = g0 + gg;
            ps[gg][xx] = (g < n_chol && x0 + xx < Xp) ? Pw[(size_t)g * Xp + x0 + xx] : cz(0, 0);
            qs[gg][xx] = (g < n_chol && y0 + xx < Xq) ? Qw[(size_t)g * Xq + y0 + xx] : cz(0, 0);
        }
        __syncthreads();
#pragma unroll
        for (int gg = 0; gg < 16; ++gg) {
            const double2 p0 = ps[gg][ty * 2], p1 = ps[gg][ty * 2 + 1];
            const double2 q0 = qs[gg][tx * 2], q1 = qs[gg][tx * 2 + 1];
            acc[0][0] = cfma(p0, q0, acc[0][0]); acc[0][1] = cfma(p0, q1, acc[0][1]);
            acc[1][0] = cfma(p1, q0, acc[1][0]); acc[1][1] = cfma(p1, q1, acc[1][1]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const int x = x0 + ty * 2 + i, y = y0 + tx * 2 + j;
            if (x < Xp && y < Xq) {
                const size_t e = ((size_t)w * Xp + x) * Xq + y;
                Kout[2 * e] = (TK)acc[i][j].x;
                Kout[2 * e + 1] = (TK)acc[i][j].y;
            }
        }
}

void launch_gram(int nw, int Xp, int Xq, int n_chol, const double2* P, const double2* Q, void* K,
                 bool fp32, cudaStream_t st)
{
    if (Xp <= 0 || Xq <= 0 || nw <= 0) return;
    dim3 grid((Xq + 31) / 32, (Xp + 31) / 32, nw);
    if (fp32) k_gram<float><<<grid, 256, 0, st>>>(Xp, Xq, n_chol, P, Q, (float*)K);
    else k_gram<double><<<grid, 256, 0, st>>>(Xp, Xq, n_chol, P, Q, (double*)K);
    msd_note_launch();
}

// ------------------------------------------------------------------------
// Same-spin per-string energy (get_ss and the one-body / Coulomb linear
// parts): e_s = sum_ij B_ij Y[h_j][p_i] + 1/2 (Qc - Qx), accumulated as
// r_s w_s e_s into per-walker partial sums. Precision T for B, K and the
// arithmetic; the block sum is FP64. The block first forms the walker's
// antisymmetrized pair table of K (C(nh,2) C(np,2) entries, against X^2 for
// K) in shared memory; each string then takes C(k,2)^2 gathers of it for
// (Qc - Qx) / 2 (string_energy_value).
template <int KL, typename T>
__global__ void __launch_bounds__(SE_THREADS)
k_string_energy(SpinTables tb, const double2* __restrict__ wts,
                const void* __restrict__ Bin, const void* __restrict__ Kin, const void* __restrict__ Yin,
                double2* __restrict__ part, int nslot, int slot0)
{
    using T2 = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int X = tb.nh * tb.np, np = tb.np, nh = tb.nh;
    const int nhp = nh * (nh - 1) / 2, npp = np * (np - 1) / 2;
    T2* as = reinterpret_cast<T2*>(smraw);   // [C(nh,2)][C(np,2)] antisymmetrized pairs of K
    T2* ys = as + nhp * npp;                 // [X]
    __shared__ double2 red[SE_THREADS];
    const int w = blockIdx.y, t = threadIdx.x;
    const T2* Kw = reinterpret_cast<const T2*>(Kin) + (size_t)w * X * X;
    // A[(h,h')][(p,p')] = K[(h,p)][(h',p')] - K[(h,p')][(h',p)], h < h', p < p'
    for (int e = t; e < nhp * npp; e += blockDim.x) {
        int a = e / npp, c = e - a * npp, h = 0, p = 0;
        while (a >= nh - 1 - h) { a -= nh - 1 - h; ++h; }
        while (c >= np - 1 - p) { c -= np - 1 - p; ++p; }
        const int h2 = h + 1 + a, p2 = p + 1 + c;
        const T2 kc = Kw[(size_t)(h * np + p) * X + h2 * np + p2];
        const T2 kx = Kw[(size_t)(h * np + p2) * X + h2 * np + p];
        as[e] = T2{kc.x - kx.x, kc.y - kx.y};
    }
    const T2* Yw = reinterpret_cast<const T2*>(Yin) + (size_t)w * X;
    for (int e = t; e < X; e += blockDim.x) ys[e] = Yw[e];
    __syncthreads();
    const int ns = tb.bucket[KL + 1] - tb.bucket[KL];
    double2 contrib = cz(0, 0);
    for (int it = 0; it < SE_PER_THREAD; ++it) {
        const int sl = blockIdx.x * (SE_THREADS * SE_PER_THREAD) + it * SE_THREADS + t;
        if (sl >= ns) break;
        contrib = cadd(contrib, string_energy_term<KL, T, true>(tb, w, sl, ns, Bin, as, ys, wts));
    }
    red[t] = contrib;
    __syncthreads();
    for (int o = SE_THREADS / 2; o; o >>= 1) {
        if (t < o) red[t] = cadd(red[t], red[t + o]);
        __syncthreads();
    }
    if (t == 0) part[(size_t)w * nslot + slot0 + blockIdx.x] = red[0];
}

int string_energy_blocks(const SpinTables& tb, int k)
{
    const int ns = tb.bucket[k + 1] - tb.bucket[k];
    return ns > 0 ? (ns + SE_THREADS * SE_PER_THREAD - 1) / (SE_THREADS * SE_PER_THREAD) : 0;
}

size_t string_energy_smem(const SpinTables& tb, bool fp32)
{
    const int X = tb.nh * tb.np;
    const size_t pairs = (size_t)(tb.nh * (tb.nh - 1) / 2) * (tb.np * (tb.np - 1) / 2);
    return (fp32 ? sizeof(float2) : sizeof(double2)) * (pairs + X);
}

template <int KL>
static void launch_se_k(const SpinTables& tb, int nw, const double2* wts,
                        const void* B, const void* K, const void* Y, bool fp32, double2* part,
                        int nslot, int& slot, cudaStream_t st)
{
    const int nb = string_energy_blocks(tb, KL);
    if (!nb) return;
    dim3 grid(nb, nw);
    const size_t smem = string_energy_smem(tb, fp32);
    if (fp32) {
        cudaFuncSetAttribute(k_string_energy<KL, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_string_energy<KL, float><<<grid, SE_THREADS, smem, st>>>(tb, wts, B, K, Y, part, nslot, slot); msd_note_launch();
    } else {
        cudaFuncSetAttribute(k_string_energy<KL, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_string_energy<KL, double><<<grid, SE_THREADS, smem, st>>>(tb, wts, B, K, Y, part, nslot, slot); msd_note_launch();
    }
    slot += nb;
}

void launch_string_energy(const SpinTables& tb, int nw, const double2* wts,
                          const void* B, const void* K, const void* Y, bool fp32, double2* part,
                          int nslot, int slot0, cudaStream_t st)
{
    int slot = slot0;
    launch_se_k<1>(tb, nw, wts, B, K, Y, fp32, part, nslot, slot, st);
    launch_se_k<2>(tb, nw, wts, B, K, Y, fp32, part, nslot, slot, st);
    launch_se_k<3>(tb, nw, wts, B, K, Y, fp32, part, nslot, slot, st);
    launch_se_k<4>(tb, nw, wts, B, K, Y, fp32, part, nslot, slot, st);
    launch_se_k<5>(tb, nw, wts, B, K, Y, fp32, part, nslot, slot, st);
    launch_se_k<6>(tb, nw, wts, B, K, Y, fp32, part, nslot, slot, st);
}

int string_energy_slots(const SpinTables& tb)
{
    int n = 0;
    for (int k = 1; k <= MSD_KMAX; ++k) n += string_energy_blocks(tb, k);
    return n;
}

// ------------------------------------------------------------------------
// Opposite-spin cross term (fill_os) per determinant (a, b) with levels
// (ka, KB): c_I r_a r_b X_ab with
//   X_ab = sum_ij Ba_ij sum_kl Bb_kl K^{ab}[(ha_j,pa_i)][(hb_l,pb_k)].
// The beta level KB is a template parameter (its inverse minor is held in
// registers); the alpha level runs at run time.
template <int KB, typename T>
__global__ void __launch_bounds__(PC_THREADS)
k_pair_cross(SpinTables ta, SpinTables tbb, PairTables pt, int ka, int lo, int n,
             const void* __restrict__ ra_in, const void* __restrict__ rb_in,
             const void* __restrict__ Ba_in, const void* __restrict__ Bb_in,
             const void* __restrict__ Kin, double2* __restrict__ part, int nslot, int slot0)
{
    using T2 = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Xa = ta.nh * ta.np, Xb = tbb.nh * tbb.np;
    T2* ks = reinterpret_cast<T2*>(smraw);   // [Xa][Xb]
    __shared__ double2 red[PC_THREADS];
    const int w = blockIdx.y, t = threadIdx.x;
    const T2* Kw = reinterpret_cast<const T2*>(Kin) + (size_t)w * Xa * Xb;
    for (int e = t; e < Xa * Xb; e += blockDim.x) ks[e] = Kw[e];
    __syncthreads();
    const T2* ra = reinterpret_cast<const T2*>(ra_in);
    const T2* rb = reinterpret_cast<const T2*>(rb_in);
    T2 contrib = T2{0, 0};   // this thread's determinants, in the working precision
    // the shared Gram matrix is filled once per block and reused by
    // PC_PER_THREAD determinants per thread
    for (int it = 0; it < PC_PER_THREAD; ++it) {
        const int i0 = blockIdx.x * (PC_THREADS * PC_PER_THREAD) + it * PC_THREADS + t;
        if (i0 >= n) break;
        const T2 v = pair_cross_term<KB, T>(ta, tbb, pt, ka, lo + i0, w, Ba_in, Bb_in, ks, ra, rb);
        contrib.x += v.x;
        contrib.y += v.y;
    }
    red[t] = cz((double)contrib.x, (double)contrib.y);
    __syncthreads();
    for (int o = PC_THREADS / 2; o; o >>= 1) {
        if (t < o) red[t] = cadd(red[t], red[t + o]);
        __syncthreads();
    }
    if (t == 0) part[(size_t)w * nslot + slot0 + blockIdx.x] = red[0];
}

template <int KB>
static void launch_pc_k(const SpinTables& ta, const SpinTables& tb, const PairTables& pt, int ka,
                        int nw, const void* ra, const void* rb, const void* Ba, const void* Bb,
                        const void* K, bool fp32, double2* part, int nslot, int& slot,
                        cudaStream_t st, bool use_runs)
{
    const int idx = ka * (MSD_KMAX + 1) + KB;
    const int lo = pt.bucket[idx], n = pt.bucket[idx + 1] - lo;
    if (n <= 0) return;
    if (use_runs && pt.run_side[idx]) {
        launch_pair_run(ta, tb, pt, idx, ka, KB, nw, ra, rb, Ba, Bb, K, fp32, part, nslot, slot, st);
        slot += pair_run_blocks(pt, idx);
        return;
    }
    const int nb = (n + PC_THREADS * PC_PER_THREAD - 1) / (PC_THREADS * PC_PER_THREAD);
    dim3 grid(nb, nw);
    const size_t smem = (fp32 ? sizeof(float2) : sizeof(double2)) * (size_t)(ta.nh * ta.np) * (tb.nh * tb.np);
    if (launch_pair_cross2(ka, KB, fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st)) {
        slot += nb;
        return;
    }
    if (fp32) {
        cudaFuncSetAttribute(k_pair_cross<KB, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pair_cross<KB, float><<<grid, PC_THREADS, smem, st>>>(ta, tb, pt, ka, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot); msd_note_launch();
    } else {
        cudaFuncSetAttribute(k_pair_cross<KB, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pair_cross<KB, double><<<grid, PC_THREADS, smem, st>>>(ta, tb, pt, ka, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot); msd_note_launch();
    }
    slot += nb;
}

void launch_pair_cross(const SpinTables& ta, const SpinTables& tb, const PairTables& pt, int nw,
                       const void* ra, const void* rb, const void* Ba, const void* Bb,
                       const void* K, bool fp32, double2* part, int nslot, int slot0,
                       cudaStream_t st, bool use_runs)
{
    int slot = slot0;
    for (int ka = 1; ka <= MSD_KMAX; ++ka) {
        launch_pc_k<1>(ta, tb, pt, ka, nw, ra, rb, Ba, Bb, K, fp32, part, nslot, slot, st, use_runs);
        launch_pc_k<2>(ta, tb, pt, ka, nw, ra, rb, Ba, Bb, K, fp32, part, nslot, slot, st, use_runs);
        launch_pc_k<3>(ta, tb, pt, ka, nw, ra, rb, Ba, Bb, K, fp32, part, nslot, slot, st, use_runs);
        launch_pc_k<4>(ta, tb, pt, ka, nw, ra, rb, Ba, Bb, K, fp32, part, nslot, slot, st, use_runs);
        launch_pc_k<5>(ta, tb, pt, ka, nw, ra, rb, Ba, Bb, K, fp32, part, nslot, slot, st, use_runs);
        launch_pc_k<6>(ta, tb, pt, ka, nw, ra, rb, Ba, Bb, K, fp32, part, nslot, slot, st, use_runs);
    }
}

int pair_cross_slots(const PairTables& pt, bool use_runs)
{
    int n = 0;
    for (int ka = 1; ka <= MSD_KMAX; ++ka)
        for (int kb = 1; kb <= MSD_KMAX; ++kb) {
            const int idx = ka * (MSD_KMAX + 1) + kb;
            const int c = pt.bucket[idx + 1] - pt.bucket[idx];
            if (c <= 0) continue;
            if (use_runs && pt.run_side[idx]) n += pair_run_blocks(pt, idx);
            else n += (c + PC_THREADS * PC_PER_THREAD - 1) / (PC_THREADS * PC_PER_THREAD);
        }
    return n;
}

// ------------------------------------------------------------------------
// Final assembly per walker:
//   R = sum of slots [0, nR),  S = sum of slots [nR, nslot)
//   E_0 = e0 + e1a + e1b + 1/2 sum_g V0^2 - 1/2 (xa + xb)
//   E_L = E_0 + S / R,  O_T = O0a O0b R
__global__ void k_final(int nw, const double2* __restrict__ part, int nslot, int nR, double e0,
                        const double2* __restrict__ e1a, const double2* __restrict__ e1b,
                        const double2* __restrict__ scal, const double2* __restrict__ O0a,
                        const double2* __restrict__ O0b, double2* __restrict__ eloc,
                        double2* __restrict__ ovlp)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    double2 R = cz(0, 0), S = cz(0, 0);
    for (int i = 0; i < nR; ++i) R = cadd(R, part[(size_t)w * nslot + i]);
    for (int i = nR; i < nslot; ++i) S = cadd(S, part[(size_t)w * nslot + i]);
    const double2* sc = scal + (size_t)w * 8;
    double2 E0 = cadd(cz(e0, 0), cadd(e1a[w], e1b[w]));
    E0 = cadd(E0, cscale(sc[2], 0.5));
    E0 = csub(E0, cscale(cadd(sc[0], sc[1]), 0.5));
    eloc[w] = cadd(E0, cdiv(S, R));
    if (ovlp) ovlp[w] = cmul(cmul(O0a[w], O0b[w]), R);
}

void launch_final(int nw, const double2* part, int nslot, int nR, double e0, const double2* e1a,
                  const double2* e1b, const double2* scal, const double2* O0a, const double2* O0b,
                  double2* eloc, double2* ovlp, cudaStream_t st)
{
    k_final<<<(nw + 127) / 128, 128, 0, st>>>(nw, part, nslot, nR, e0, e1a, e1b, scal, O0a, O0b,
                                             eloc, ovlp); msd_note_launch();
}
