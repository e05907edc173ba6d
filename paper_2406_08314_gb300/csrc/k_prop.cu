// One phaseless AFQMC propagation step (Sec. II A, Eq. 7-12), FP64:
//   c_g     = i sqrt(dt) (x_g - xbar_g) = i sqrt(dt) x_g - dt vbias_g,  xbar = -i sqrt(dt) vbias
//   V       = sum_g c_g L_g                                (a GEMM over g, k_gemm_zd)
//   phi'    = E T_n(V) E phi,  E = exp(-dt h'/2),  T_n(V) = sum_{k<=n} V^k / k!
//   I       = S exp(x.xbar - xbar.xbar/2),  S = O_T(phi') / O_T(phi)
//   w'      = w |I| max(0, cos arg S)
// and, optionally, the Q factor of phi' = Q R (modified Gram-Schmidt; the
// diagonal of R real and positive).
#include "common.cuh"
#include "kernels.h"

// sum_g L_g L_g (real, M x M) from the transposed Cholesky vectors
// Lt[(p, q)][g] = L_g[p][q]: corr[p][q] = sum_g sum_r L_g[p][r] L_g[r][q].
__global__ void k_sum_LL(int M, int G, const double* __restrict__ Lt, double* __restrict__ corr)
{
    const int p = blockIdx.y, q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M) return;
    double acc = 0.0;
    for (int r = 0; r < M; ++r) {
        const double* a = Lt + ((size_t)p * M + r) * G;
        const double* b = Lt + ((size_t)r * M + q) * G;
        for (int g = 0; g < G; ++g) acc = fma(a[g], b[g], acc);
    }
    corr[(size_t)p * M + q] = acc;
}

void launch_sum_LL(int M, int G, const double* Lt, double* corr, cudaStream_t st)
{
    dim3 grid((M + 127) / 128, M);
    k_sum_LL<<<grid, 128, 0, st>>>(M, G, Lt, corr);
    msd_note_launch();
}

// Per walker: c[w][g] and the exponent sum_g (x_g xbar_g - xbar_g^2 / 2),
// summed in a fixed order.
__global__ void __launch_bounds__(256)
k_prop_coef(int G, double dt, const double* __restrict__ x, const double2* __restrict__ vbias,
            double2* __restrict__ c, double2* __restrict__ expo)
{
    __shared__ double2 red[256];
    const int w = blockIdx.x, t = threadIdx.x;
    const double sd = sqrt(dt);
    double2 e = cz(0, 0);
    for (int g = t; g < G; g += blockDim.x) {
        const double xg = x[(size_t)w * G + g];
        const double2 v = vbias[(size_t)w * G + g];
        c[(size_t)w * G + g] = cz(-dt * v.x, sd * xg - dt * v.y);
        const double2 xb = cz(sd * v.y, -sd * v.x);            // -i sqrt(dt) v
        const double2 xb2 = cmul(xb, xb);
        e = cadd(e, cz(xg * xb.x - 0.5 * xb2.x, xg * xb.y - 0.5 * xb2.y));
    }
    red[t] = e;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (t < o) red[t] = cadd(red[t], red[t + o]);
        __syncthreads();
    }
    if (t == 0) expo[w] = red[0];
}

void launch_prop_coef(int nw, int G, double dt, const double* x, const double2* vbias, double2* c, double2* expo,
                      cudaStream_t st)
{
    k_prop_coef<<<nw, 256, 0, st>>>(G, dt, x, vbias, c, expo);
    msd_note_launch();
}

// out_w = scale A_w in_w (+ acc_w += out_w), in_w and out_w [M][N] complex,
// A_w [M][M] complex (per walker, stride a_stride) or real (shared, a_real
// non-null). One block per (row tile of 32, walker); in_w staged in shared
// memory; the block's 32 x N outputs are spread over its threads.
template <bool REAL_A>
__global__ void __launch_bounds__(256)
k_apply_rows(int M, int N, const double2* __restrict__ A, long long a_stride, const double* __restrict__ Ar,
             const double2* __restrict__ in, double2* __restrict__ out, double2* __restrict__ acc, double scale)
{
    extern __shared__ double2 sin_[];   // [M][N]
    const int w = blockIdx.y, p0 = blockIdx.x * 32;
    const double2* iw = in + (size_t)w * M * N;
    for (int e = threadIdx.x; e < M * N; e += blockDim.x) sin_[e] = iw[e];
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * N; e += blockDim.x) {
        const int pr = e / N, j = e - pr * N, p = p0 + pr;
        if (p < M) {
            double2 s = cz(0, 0);
            if (REAL_A) {
                const double* a = Ar + (size_t)p * M;
                for (int q = 0; q < M; ++q) {
                    const double2 v = sin_[q * N + j];
                    s.x = fma(a[q], v.x, s.x);
                    s.y = fma(a[q], v.y, s.y);
                }
            } else {
                const double2* a = A + (size_t)w * a_stride + (size_t)p * M;
                for (int q = 0; q < M; ++q) s = cfma(a[q], sin_[q * N + j], s);
            }
            s = cscale(s, scale);
            const size_t o = (size_t)w * M * N + (size_t)p * N + j;
            out[o] = s;
            if (acc) acc[o] = cadd(acc[o], s);
        }
    }
}

static int apply_rows_smem_ok(int M, int N)
{
    return sizeof(double2) * (size_t)M * N <= 200 * 1024;
}

int launch_apply_rows(int nw, int M, int N, const double2* A, long long a_stride, const double* Ar,
                      const double2* in, double2* out, double2* acc, double scale, cudaStream_t st)
{
    if (!apply_rows_smem_ok(M, N)) return -1;
    const size_t smem = sizeof(double2) * (size_t)M * N;
    dim3 grid((M + 31) / 32, nw);
    if (Ar) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_apply_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_apply_rows<true><<<grid, 256, smem, st>>>(M, N, A, a_stride, Ar, in, out, acc, scale);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k_apply_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_apply_rows<false><<<grid, 256, smem, st>>>(M, N, A, a_stride, Ar, in, out, acc, scale);
    }
    msd_note_launch();
    return 0;
}

// S = ovlp_new / ovlp_old, I = S exp(expo), w' = w |I| max(0, cos arg S).
__global__ void k_prop_weight(int nw, const double2* __restrict__ o_old, const double2* __restrict__ o_new,
                              const double2* __restrict__ expo, double* __restrict__ w, double2* __restrict__ ratio)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw) return;
    const double2 S = cdiv(o_new[i], o_old[i]);
    const double aS = hypot(S.x, S.y);
    const double cth = aS > 0 ? S.x / aS : 0.0;                 // cos arg S
    const double mag = aS * exp(expo[i].x);                      // |S exp(expo)|
    w[i] = w[i] * mag * (cth > 0 ? cth : 0.0);
    if (ratio) ratio[i] = S;
}

void launch_prop_weight(int nw, const double2* o_old, const double2* o_new, const double2* expo, double* w,
                        double2* ratio, cudaStream_t st)
{
    k_prop_weight<<<(nw + 127) / 128, 128, 0, st>>>(nw, o_old, o_new, expo, w, ratio);
    msd_note_launch();
}

// Q of phi = Q R per walker (modified Gram-Schmidt, columns in order; the
// diagonal of R is the column norm, real and positive). phi [M][N] in shared
// memory; warp k handles column k's projections; norms and projections are
// warp-shuffle reductions in a fixed order.
__global__ void __launch_bounds__(256)
k_qr_mgs(int M, int N, double2* __restrict__ phi, unsigned* err)
{
    extern __shared__ double2 sq[];   // [M][N]
    __shared__ double nrm_inv;
    const int w = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    double2* pw = phi + (size_t)w * M * N;
    for (int e = threadIdx.x; e < M * N; e += blockDim.x) sq[e] = pw[e];
    __syncthreads();
    for (int j = 0; j < N; ++j) {
        if (warp == 0) {
            double s = 0;
            for (int r = lane; r < M; r += 32) s += sq[r * N + j].x * sq[r * N + j].x + sq[r * N + j].y * sq[r * N + j].y;
            for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                if (!(s > 0)) atomicOr(err, MSD_DEV_ERR_SINGULAR);
                nrm_inv = s > 0 ? 1.0 / sqrt(s) : 0.0;
            }
        }
        __syncthreads();
        const double ni = nrm_inv;
        for (int r = threadIdx.x; r < M; r += blockDim.x) sq[r * N + j] = cscale(sq[r * N + j], ni);
        __syncthreads();
        for (int k = j + 1 + warp; k < N; k += nwarp) {
            double2 d = cz(0, 0);   // q_j^H phi_k
            for (int r = lane; r < M; r += 32) {
                const double2 q = sq[r * N + j], v = sq[r * N + k];
                d.x += q.x * v.x + q.y * v.y;
                d.y += q.x * v.y - q.y * v.x;
            }
            for (int o = 16; o; o >>= 1) {
                d.x += __shfl_xor_sync(0xffffffffu, d.x, o);
                d.y += __shfl_xor_sync(0xffffffffu, d.y, o);
            }
            for (int r = lane; r < M; r += 32) sq[r * N + k] = cfms(d, sq[r * N + j], sq[r * N + k]);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < M * N; e += blockDim.x) pw[e] = sq[e];
}

int launch_qr_mgs(int nw, int M, int N, double2* phi, unsigned* err, cudaStream_t st)
{
    const size_t smem = sizeof(double2) * (size_t)M * N;
    if (smem > 200 * 1024) return -1;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_qr_mgs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_qr_mgs<<<nw, 256, smem, st>>>(M, N, phi, err);
    msd_note_launch();
    return 0;
}
