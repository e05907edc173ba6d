// FP32 kernels of the mixed-precision path: the per-(walker, Cholesky
// vector) epilogue of F = G L_g computed on the tensor cores, the sums over
// Cholesky vectors and the Gram matrices of Lambda_g = G L_g (I - G). Same
// algebra as the FP64 kernels in k_energy.cu.
#include <algorithm>

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
            Lact[wg * lam_pitch(X) + e] = lam[j * np + p];
            Xic[wg * lam_pitch(X) + e] = xi;
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
// FP64), and (traces) the FP64 scalar sums of the FP64 kernel; without
// traces scal is left to the exactly split reference sums. With v0w (the
// exactly split walker parts t1_g of V0_g = C_g + t1_g, [nw][G]) the FP32
// sum runs over t1_g only; the caller's Lh then holds the reference part
// sum_g C_g Lambda_g[x] as well (the one-body term of h + J, J = sum_g C_g
// L_g, FP64). Warps split the Cholesky vectors, lanes the active entries;
// the warp sums are added in a fixed order.
__global__ void __launch_bounds__(256)
k_gamma_reduce_f32(int X, int n_chol, int spin, bool traces, const double2* __restrict__ v0a,
                   const double2* __restrict__ v0b, const double2* __restrict__ xx,
                   const float2* __restrict__ Lact, const float2* __restrict__ Xic,
                   const double2* __restrict__ Lh, float2* __restrict__ Y, double2* __restrict__ scal,
                   const float2* __restrict__ v0w)
{
    __shared__ float2 part[8][MSD_XMAX];
    __shared__ double2 red[2][256];
    const int w = blockIdx.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const size_t base = (size_t)w * n_chol;
    double2 s0 = cz(0, 0), s1 = cz(0, 0);
    for (int g = t; traces && g < n_chol; g += blockDim.x) {
        s0 = cadd(s0, xx[base + g]);
        const double2 V0 = cadd(v0a[base + g], v0b[base + g]);
        s1 = cfma(V0, V0, s1);
    }
    float2 acc[(MSD_XMAX + 31) / 32];
#pragma unroll
    for (int q = 0; q < (MSD_XMAX + 31) / 32; ++q) acc[q] = make_float2(0, 0);
    for (int g = warp; g < n_chol; g += 8) {
        float2 V0;
        if (v0w) {
            V0 = v0w[base + g];
        } else {
            const double2 V0d = cadd(v0a[base + g], v0b[base + g]);
            V0 = make_float2((float)V0d.x, (float)V0d.y);
        }
        const float2* la = Lact + (base + g) * lam_pitch(X);
        const float2* xi = Xic + (base + g) * lam_pitch(X);
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
    if (t == 0 && traces) {
        scal[(size_t)w * 8 + spin] = red[0][0];
        if (spin == 0) scal[(size_t)w * 8 + 2] = red[1][0];
    }
}

void launch_gamma_reduce_f32(int nw, int X, int n_chol, int spin, const double2* v0a, const double2* v0b,
                             const double2* xx, const float2* Lact, const float2* Xic, const double2* Lh,
                             float2* Y, double2* scal, cudaStream_t st, bool traces, const float2* v0w)
{
    k_gamma_reduce_f32<<<nw, 256, 0, st>>>(X, n_chol, spin, traces, v0a, v0b, xx, Lact, Xic, Lh, Y, scal, v0w);
    msd_note_launch();
}

// K[x][y] = sum_g P_g[x] Q_g[y] (complex, no conjugation) per walker: one
// block per walker computes the whole Xp x Xq Gram matrix. 16 x 16 threads,
// thread (ty, tx) owns rows ty + 16 i and columns tx + 16 j (i, j < R, R =
// ceil(max(Xp, Xq) / 16)), so each P value read from shared memory (a
// broadcast to the 16 threads of a row) and each Q value (consecutive,
// conflict-free) serves R complex FMAs. Cholesky vectors stream through
// shared memory GRAM_G at a time; the sum over g runs in a fixed order.
// When P and Q are the same vectors (the same-spin Gram matrices, symmetric)
// only the sub-tiles i <= j are accumulated, one operand is staged, and the
// upper sub-tiles are mirrored on the way out.
#define GRAM_G 32
template <int R, bool SYM>
__device__ __forceinline__ void gram_body(int Xp, int Xq, int n_chol, const float2* __restrict__ Pw,
                                          const float2* __restrict__ Qw, float2* __restrict__ Kw, float2* gsm)
{
    constexpr int W = 16 * R;
    float2* ps = gsm;                                 // [GRAM_G][16 R]
    float2* qs = SYM ? gsm : gsm + GRAM_G * W;        // [GRAM_G][16 R]
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    const int Pp = lam_pitch(Xp), Qp = lam_pitch(Xq);
    float2 acc[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int g0 = 0; g0 < n_chol; g0 += GRAM_G) {
        __syncthreads();   // previous chunk consumed
        for (int e = t; e < GRAM_G * W; e += 256) {
            const int gg = e / W, xx = e - gg * W, g = g0 + gg;
            ps[e] = (g < n_chol && xx < Xp) ? Pw[(size_t)g * Pp + xx] : make_float2(0.f, 0.f);
            if (!SYM) qs[e] = (g < n_chol && xx < Xq) ? Qw[(size_t)g * Qp + xx] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 2
        for (int gg = 0; gg < GRAM_G; ++gg) {
            float2 pv[R], qv[R];
#pragma unroll
            for (int i = 0; i < R; ++i) {
                pv[i] = ps[gg * W + ty + 16 * i];
                qv[i] = qs[gg * W + tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < R; ++i)
#pragma unroll
                for (int j = SYM ? i : 0; j < R; ++j) acc[i][j] = fcfma(pv[i], qv[j], acc[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = SYM ? i : 0; j < R; ++j) {
            const int x = ty + 16 * i, y = tx + 16 * j;
            if (x < Xp && y < Xq) {
                Kw[(size_t)x * Xq + y] = acc[i][j];
                if (SYM && j > i) Kw[(size_t)y * Xq + x] = acc[i][j];
            }
        }
}

template <int R>
__global__ void __launch_bounds__(256, R <= 5 ? 3 : 1)
k_gram_f32(GramJobs jobs, int n_chol)
{
    // static indices keep the job table in the parameter space
    const GramJob jb = blockIdx.y == 0 ? jobs.j[0] : blockIdx.y == 1 ? jobs.j[1] : jobs.j[2];
    const int Xp = jb.Xp, Xq = jb.Xq;
    if (Xp <= 0 || Xq <= 0) return;
    extern __shared__ float2 gsm[];
    const int w = blockIdx.x;
    const float2* Pw = jb.P + (size_t)w * n_chol * lam_pitch(Xp);
    const float2* Qw = jb.Q + (size_t)w * n_chol * lam_pitch(Xq);
    float2* Kw = jb.K + (size_t)w * Xp * Xq;
    if (jb.P == jb.Q && Xp == Xq) gram_body<R, true>(Xp, Xq, n_chol, Pw, Qw, Kw, gsm);
    else gram_body<R, false>(Xp, Xq, n_chol, Pw, Qw, Kw, gsm);
}

template <int R>
static void launch_gram_r(int nw, int n_chol, const GramJobs& jobs, int nj, cudaStream_t st)
{
    const size_t smem = sizeof(float2) * 2 * GRAM_G * 16 * R;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_gram_f32<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_gram_f32<R><<<dim3(nw, nj), 256, smem, st>>>(jobs, n_chol);
    msd_note_launch();
}

void launch_gram_f32(int nw, int n_chol, const GramJobs& jobs, int nj, cudaStream_t st)
{
    int xm = 0;
    for (int i = 0; i < nj; ++i) xm = std::max(xm, std::max(jobs.j[i].Xp, jobs.j[i].Xq));
    if (xm <= 0 || nw <= 0 || nj <= 0) return;
    switch ((xm + 15) / 16) {   // MSD_XMAX = 112: R <= 7
        case 1: launch_gram_r<1>(nw, n_chol, jobs, nj, st); break;
        case 2: launch_gram_r<2>(nw, n_chol, jobs, nj, st); break;
        case 3: launch_gram_r<3>(nw, n_chol, jobs, nj, st); break;
        case 4: launch_gram_r<4>(nw, n_chol, jobs, nj, st); break;
        case 5: launch_gram_r<5>(nw, n_chol, jobs, nj, st); break;
        case 6: launch_gram_r<6>(nw, n_chol, jobs, nj, st); break;
        default: launch_gram_r<7>(nw, n_chol, jobs, nj, st); break;
    }
}
