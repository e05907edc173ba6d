// FP32 kernels of the mixed-precision path: the per-(walker, Cholesky
// vector) epilogue of F = G L_g computed on the tensor cores, the sums over
// Cholesky vectors and the Gram matrices of Lambda_g = G L_g (I - G). Same
// algebra as the FP64 kernels in k_energy.cu.
#include "common.cuh"
#include "kernels.h"

__device__ __forceinline__ float2 fcfma(float2 b, float2 c, float2 a)
{
    return make_float2(fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(b.y, c.x, a.y)));
}

__device__ __forceinline__ float2 fcfms(float2 b, float2 c, float2 a)
{
    return make_float2(fmaf(-b.x, c.x, fmaf(b.y, c.y, a.x)), fmaf(-b.x, c.y, fmaf(-b.y, c.x, a.y)));
}

// F = F0 + dF with F[j][col] = (G L_g)[occ0_j][col] (col over occ0 then P):
//   F0[j][col] = L_g[occ0_j][col]   (the reference part D0 D0^T, exact, from L;
//                                    F0T[g][j][col], FP32)
//   dF         real rows [(w, c, j)][g * NC + col] of the tensor-core GEMM over
//              the columns outside occ0 (c = 0 real, 1 imaginary part).
// With T = F[:, occ0] = T0 + dT:
//   v0 = tr T = c0_g + tr dT
//   x  = tr(T T) = x0_g + 2 tr(T0 dT) + tr(dT dT)     (c0, x0 in FP64)
//   Lambda[j][p] = F[j][P_p] - sum_l T[j][l] G[occ0_l][P_p]
//   Lact[(h,p)] = Lambda[pos(h)][p],  Xic[(h,p)] = sum_l T[pos(h)][l] Lambda[l][p]
#define FEPI_G 4   // Cholesky vectors per block
__global__ void __launch_bounds__(128)
k_fepi_f32(SpinTables tb, int M, int n_chol, const float* __restrict__ dF, long long ldf,
           const double2* __restrict__ Gr, const float* __restrict__ F0T, const double* __restrict__ c0,
           const double* __restrict__ x0, double2* __restrict__ v0, double2* __restrict__ xx,
           float2* __restrict__ Lact, float2* __restrict__ Xic)
{
    extern __shared__ float2 smf[];
    const int N = tb.N, np = tb.np, nh = tb.nh, NC = N + np, X = nh * np;
    float2* d = smf;                 // [N][NC] dF
    float2* gp = d + N * NC;         // [N][np]
    float2* lam = gp + N * np;       // [N][np]
    float* f0 = reinterpret_cast<float*>(lam + N * np);   // [N][NC] F0 (real)
    __shared__ float2 red[2][128];
    const int w = blockIdx.y, t = threadIdx.x;
    const double2* gr = Gr + (size_t)w * N * M;
    for (int e = t; e < N * np; e += blockDim.x) {
        const double2 v = gr[(size_t)(e / np) * M + tb.part_orb[e % np]];
        gp[e] = make_float2((float)v.x, (float)v.y);
    }
    for (int gi = 0; gi < FEPI_G; ++gi) {
        const int g = blockIdx.x * FEPI_G + gi;
        if (g >= n_chol) break;
        const float* Fre = dF + (size_t)w * 2 * N * ldf + (size_t)g * NC;
        const float* Fim = Fre + (size_t)N * ldf;
        const float* f0g = F0T + (size_t)g * N * NC;
        __syncthreads();   // previous vector's shared data fully consumed
        for (int e = t; e < N * NC; e += blockDim.x) {
            const int j = e / NC, cc = e % NC;
            const size_t o = (size_t)j * ldf + cc;
            d[e] = make_float2(Fre[o], Fim[o]);
            f0[e] = f0g[e];
        }
        __syncthreads();
        float2 a0 = make_float2(0, 0), a1 = make_float2(0, 0);
        for (int e = t; e < N * N; e += blockDim.x) {
            const int j = e / N, l = e % N;
            const float2 dlj = d[l * NC + j];
            // 2 T0[j][l] dT[l][j] + dT[j][l] dT[l][j]
            a1 = fcfma(d[j * NC + l], dlj, a1);
            a1.x += 2.f * f0[j * NC + l] * dlj.x;
            a1.y += 2.f * f0[j * NC + l] * dlj.y;
            if (j == l) { a0.x += d[j * NC + j].x; a0.y += d[j * NC + j].y; }
        }
        for (int e = t; e < N * np; e += blockDim.x) {
            const int j = e / np, p = e % np;
            float2 v = d[j * NC + N + p];
            v.x += f0[j * NC + N + p];
            for (int l = 0; l < N; ++l) {
                float2 tjl = d[j * NC + l];
                tjl.x += f0[j * NC + l];
                v = fcfms(tjl, gp[l * np + p], v);
            }
            lam[e] = v;
        }
        red[0][t] = a0;
        red[1][t] = a1;
        __syncthreads();
        for (int o = 64; o; o >>= 1) {
            if (t < o) {
                red[0][t].x += red[0][t + o].x; red[0][t].y += red[0][t + o].y;
                red[1][t].x += red[1][t + o].x; red[1][t].y += red[1][t + o].y;
            }
            __syncthreads();
        }
        const size_t wg = (size_t)w * n_chol + g;
        if (t == 0) {
            v0[wg] = make_double2(c0[g] + (double)red[0][0].x, (double)red[0][0].y);
            xx[wg] = make_double2(x0[g] + (double)red[1][0].x, (double)red[1][0].y);
        }
        for (int e = t; e < X; e += blockDim.x) {
            const int h = e / np, p = e % np, j = tb.hole_pos[h];
            float2 xi = make_float2(0, 0);
            for (int l = 0; l < N; ++l) {
                float2 tjl = d[j * NC + l];
                tjl.x += f0[j * NC + l];
                xi = fcfma(tjl, lam[l * np + p], xi);
            }
            Lact[wg * X + e] = lam[j * np + p];
            Xic[wg * X + e] = xi;
        }
    }
}

size_t fepi_f32_smem(const SpinTables& tb)
{
    const int N = tb.N, NC = tb.N + tb.np;
    return sizeof(float2) * (N * NC + 2 * N * tb.np) + sizeof(float) * N * NC;
}

void launch_fepi_f32(const SpinTables& tb, int nw, int M, int n_chol, const float* dF, long long ldf,
                     const double2* Gr, const float* F0T, const double* c0, const double* x0, double2* v0,
                     double2* xx, float2* Lact, float2* Xic, cudaStream_t st)
{
    dim3 grid((n_chol + FEPI_G - 1) / FEPI_G, nw);
    const size_t smem = fepi_f32_smem(tb);
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_fepi_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fepi_f32<<<grid, 128, smem, st>>>(tb, M, n_chol, dF, ldf, Gr, F0T, c0, x0, v0, xx, Lact, Xic);
    msd_note_launch();
}

// Y[x] = Lh[x] + sum_g V0_g Lact_g[x] - sum_g Xic_g[x] (FP32 terms, V0 in
// FP64), and the FP64 scalar sums of the FP64 kernel. Warps split the
// Cholesky vectors, lanes the active entries; the warp sums are added in a
// fixed order.
__global__ void __launch_bounds__(256)
k_gamma_reduce_f32(int X, int n_chol, int spin, const double2* __restrict__ v0a,
                   const double2* __restrict__ v0b, const double2* __restrict__ xx,
                   const float2* __restrict__ Lact, const float2* __restrict__ Xic,
                   const double2* __restrict__ Lh, float2* __restrict__ Y, double2* __restrict__ scal)
{
    __shared__ float2 part[8][MSD_XMAX];
    __shared__ double2 red[2][256];
    const int w = blockIdx.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const size_t base = (size_t)w * n_chol;
    double2 s0 = cz(0, 0), s1 = cz(0, 0);
    for (int g = t; g < n_chol; g += blockDim.x) {
        s0 = cadd(s0, xx[base + g]);
        const double2 V0 = cadd(v0a[base + g], v0b[base + g]);
        s1 = cfma(V0, V0, s1);
    }
    float2 acc[(MSD_XMAX + 31) / 32];
#pragma unroll
    for (int q = 0; q < (MSD_XMAX + 31) / 32; ++q) acc[q] = make_float2(0, 0);
    for (int g = warp; g < n_chol; g += 8) {
        const double2 V0d = cadd(v0a[base + g], v0b[base + g]);
        const float2 V0 = make_float2((float)V0d.x, (float)V0d.y);
        const float2* la = Lact + (base + g) * X;
        const float2* xi = Xic + (base + g) * X;
#pragma unroll
        for (int q = 0; q < (MSD_XMAX + 31) / 32; ++q) {
            const int x = q * 32 + lane;
            if (x < X) {
                acc[q] = fcfma(V0, la[x], acc[q]);
                acc[q].x -= xi[x].x;
                acc[q].y -= xi[x].y;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < (MSD_XMAX + 31) / 32; ++q) {
        const int x = q * 32 + lane;
        if (x < X) part[warp][x] = acc[q];
    }
    red[0][t] = s0;
    red[1][t] = s1;
    __syncthreads();
    for (int x = t; x < X; x += blockDim.x) {
        const double2 l = Lh[(size_t)w * X + x];
        float2 y = make_float2((float)l.x, (float)l.y);
        for (int q = 0; q < 8; ++q) { y.x += part[q][x].x; y.y += part[q][x].y; }
        Y[(size_t)w * X + x] = y;
    }
    for (int o = 128; o; o >>= 1) {
        if (t < o) { red[0][t] = cadd(red[0][t], red[0][t + o]); red[1][t] = cadd(red[1][t], red[1][t + o]); }
        __syncthreads();
    }
    if (t == 0) {
        scal[(size_t)w * 8 + spin] = red[0][0];
        if (spin == 0) scal[(size_t)w * 8 + 2] = red[1][0];
    }
}

void launch_gamma_reduce_f32(int nw, int X, int n_chol, int spin, const double2* v0a, const double2* v0b,
                             const double2* xx, const float2* Lact, const float2* Xic, const double2* Lh,
                             float2* Y, double2* scal, cudaStream_t st)
{
    k_gamma_reduce_f32<<<nw, 256, 0, st>>>(X, n_chol, spin, v0a, v0b, xx, Lact, Xic, Lh, Y, scal);
    msd_note_launch();
}

// K[w][x][y] = sum_g P[w][g][x] Q[w][g][y], FP32, 32 x 32 tile per block.
__global__ void __launch_bounds__(256)
k_gram_f32(int Xp, int Xq, int n_chol, const float2* __restrict__ P, const float2* __restrict__ Q,
           float2* __restrict__ Kout)
{
    __shared__ float2 ps[32][32 + 1], qs[32][32 + 1];
    const int w = blockIdx.z;
    const int x0 = blockIdx.y * 32, y0 = blockIdx.x * 32;
    const int t = threadIdx.x, ty = t / 16, tx = t % 16;
    float2 acc[2][2] = {{make_float2(0, 0), make_float2(0, 0)}, {make_float2(0, 0), make_float2(0, 0)}};
    const float2* Pw = P + (size_t)w * n_chol * Xp;
    const float2* Qw = Q + (size_t)w * n_chol * Xq;
    for (int g0 = 0; g0 < n_chol; g0 += 32) {
        for (int e = t; e < 32 * 32; e += 256) {
            const int gg = e / 32, xx = e % 32, g = g0 + gg;
            ps[gg][xx] = (g < n_chol && x0 + xx < Xp) ? Pw[(size_t)g * Xp + x0 + xx] : make_float2(0, 0);
            qs[gg][xx] = (g < n_chol && y0 + xx < Xq) ? Qw[(size_t)g * Xq + y0 + xx] : make_float2(0, 0);
        }
        __syncthreads();
#pragma unroll 8
        for (int gg = 0; gg < 32; ++gg) {
            const float2 p0 = ps[gg][ty * 2], p1 = ps[gg][ty * 2 + 1];
            const float2 q0 = qs[gg][tx * 2], q1 = qs[gg][tx * 2 + 1];
            acc[0][0] = fcfma(p0, q0, acc[0][0]); acc[0][1] = fcfma(p0, q1, acc[0][1]);
            acc[1][0] = fcfma(p1, q0, acc[1][0]); acc[1][1] = fcfma(p1, q1, acc[1][1]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const int x = x0 + ty * 2 + i, y = y0 + tx * 2 + j;
            if (x < Xp && y < Xq) Kout[((size_t)w * Xp + x) * Xq + y] = acc[i][j];
        }
}

void launch_gram_f32(int nw, int Xp, int Xq, int n_chol, const float2* P, const float2* Q, float2* K,
                     cudaStream_t st)
{
    if (Xp <= 0 || Xq <= 0 || nw <= 0) return;
    dim3 grid((Xq + 31) / 32, (Xp + 31) / 32, nw);
    k_gram_f32<<<grid, 256, 0, st>>>(Xp, Xq, n_chol, P, Q, K);
    msd_note_launch();
}
