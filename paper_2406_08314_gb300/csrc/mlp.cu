// Learned control variate for the local energy: a small MLP on features of
// the reference Green's function (its non-zero rows, or its active-space
// block), trained on local energies the
// library itself computes. Inference and training run in these kernels: BF16
// weights and activations, FP32 accumulation (tcgen05 kind::f16 GEMMs),
// FP32 master weights with Adam. The paper has no counterpart.
//
// Network: x (n_in) -> [W0, b0] -> GELU -> [W1, b1] -> GELU -> [W2, b2] ->
// GELU -> [w3, b3] -> y (scalar), width `width`; GELU(z) = z Phi(z) with the
// normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2. Loss (training): mean
// squared error (1/B) sum_b (y_b - t_b)^2.
#include <cuda_bf16.h>

#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/msd.h"
#include "common.cuh"
#include "kernels.h"

typedef __nv_bfloat16 bf16;

namespace {

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z)
{
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

int grid_of(long long n)
{
    const long long cap = 32ll * msd_sm_count();
    return (int)((n + 255) / 256 < cap ? (n + 255) / 256 : cap);
}

// x fp32 [B][n] -> row-major bf16 [B][n] and transposed bf16 [n][ldt]
__global__ void k_in_bf16(int B, int n, const float* __restrict__ x, bf16* __restrict__ xb, bf16* __restrict__ xt,
                          int ldt)
{
    const long long total = (long long)B * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n), j = (int)(e % n);
        const bf16 v = __float2bfloat16(x[e]);
        xb[e] = v;
        xt[(size_t)j * ldt + b] = v;
    }
}

// z = acc + bias (fp32, kept for the backward pass); h = GELU(z) in bf16,
// row-major [B][n] and transposed [n][ldt]
__global__ void k_bias_gelu(int B, int n, float* __restrict__ z, const float* __restrict__ bias,
                            bf16* __restrict__ h, bf16* __restrict__ ht, int ldt)
{
    const long long total = (long long)B * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n), j = (int)(e % n);
        const float v = z[e] + bias[j];
        z[e] = v;
        const bf16 hv = __float2bfloat16(gelu(v));
        h[e] = hv;
        ht[(size_t)j * ldt + b] = hv;
    }
}

// y_b = sum_j h[b][j] w[j] + c (one warp per sample)
__global__ void k_out(int B, int n, const bf16* __restrict__ h, const float* __restrict__ w, const float* __restrict__ c,
                      float* __restrict__ y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    float a = 0;
    for (int j = lane; j < n; j += 32) a += __bfloat162float(h[(size_t)warp * n + j]) * w[j];
    for (int o = 16; o; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) y[warp] = a + c[0];
}

// dy_b = 2 (y_b - t_b) / B, loss = (1/B) sum (y - t)^2 (one block, fixed order)
__global__ void k_loss(int B, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                       float* __restrict__ loss)
{
    __shared__ double red[1024];
    double a = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float d = y[b] - t[b];
        dy[b] = 2.f * d / (float)B;
        a += (double)d * d;
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) loss[0] = (float)(red[0] / B);
}

// output layer backward: gw[j] = sum_b dy_b h[b][j], gc = sum_b dy_b (block j),
// dz[b][j] = dy_b w[j] GELU'(z[b][j]) as bf16 (row-major and transposed),
// dzf: the same in fp32 for the bias gradient of the layer below
__global__ void k_out_back_w(int B, int n, const float* __restrict__ dy, const bf16* __restrict__ h,
                             float* __restrict__ gw, float* __restrict__ gc)
{
    __shared__ float red[256];
    const int j = blockIdx.x;
    float a = 0, c = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        a += dy[b] * __bfloat162float(h[(size_t)b * n + j]);
        c += dy[b];
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) gw[j] = red[0];
    if (j == 0) {
        __syncthreads();
        red[threadIdx.x] = c;
        __syncthreads();
        for (int o = blockDim.x / 2; o; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) gc[0] = red[0];
    }
}

__global__ void k_out_back_dz(int B, int n, const float* __restrict__ dy, const float* __restrict__ w,
                              const float* __restrict__ z, float* __restrict__ dzf, bf16* __restrict__ dz,
                              bf16* __restrict__ dzt, int ldt)
{
    const long long total = (long long)B * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n), j = (int)(e % n);
        const float v = dy[b] * w[j] * gelu_d(z[e]);
        dzf[e] = v;
        const bf16 vb = __float2bfloat16(v);
        dz[e] = vb;
        dzt[(size_t)j * ldt + b] = vb;
    }
}

// hidden backward: dz = dh * GELU'(z) with dh = (dz_above W_above) from the GEMM
__global__ void k_gelu_back(int B, int n, const float* __restrict__ dh, const float* __restrict__ z,
                            float* __restrict__ dzf, bf16* __restrict__ dz, bf16* __restrict__ dzt, int ldt)
{
    const long long total = (long long)B * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n), j = (int)(e % n);
        const float v = dh[e] * gelu_d(z[e]);
        dzf[e] = v;
        const bf16 vb = __float2bfloat16(v);
        dz[e] = vb;
        dzt[(size_t)j * ldt + b] = vb;
    }
}

// column sums: g[j] = sum_b a[b][j] (block j, fixed order)
__global__ void k_colsum(int B, int n, const float* __restrict__ a, float* __restrict__ g)
{
    __shared__ float red[256];
    const int j = blockIdx.x;
    float s = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += a[(size_t)b * n + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) g[j] = red[0];
}

// Adam (Kingma & Ba) on FP32 master parameters
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// bf16 copies of a weight matrix W [out][in]: row-major and transposed [in][out]
__global__ void k_weights_bf16(int out, int in, const float* __restrict__ w, bf16* __restrict__ wb,
                               bf16* __restrict__ wt)
{
    const long long total = (long long)out * in;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e / in), i = (int)(e % in);
        const bf16 v = __float2bfloat16(w[e]);
        wb[e] = v;
        wt[(size_t)i * out + o] = v;
    }
}

// rows x cols fp32 GEMM result -> in place add? (not needed)

}  // namespace

// Active-space features of the reference Green's function G = G0^T per
// walker: feat[w][s][p][q][c] = (Re, Im) G^s[n_core + p][n_core + q] for
// p, q < n_act, from the rows Gr[j][.] = G[occ0_j][.] (zero for rows outside
// occ0).
__global__ void k_features(int nw, int M, int N, int n_core, int n_act, const int* __restrict__ pos0,
                           const double2* __restrict__ Gr, float* __restrict__ feat, int spin)
{
    const long long per = (long long)n_act * n_act;
    const long long total = (long long)nw * per;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(e / per);
        const int p = (int)((e % per) / n_act), q = (int)(e % n_act);
        const int j = pos0[n_core + p];
        double2 g = make_double2(0, 0);
        if (j >= 0) g = Gr[((size_t)w * N + j) * M + n_core + q];
        float* o = feat + ((size_t)w * 2 * per + (size_t)spin * per + (size_t)p * n_act + q) * 2;
        o[0] = (float)g.x;
        o[1] = (float)g.y;
    }
}

// Full non-zero rows of G (rows occ0, all orbitals): feat[w][off + (j*M + q)*2 + c]
// for j < N, q < M; row pitch ld floats per walker.
__global__ void k_features_rows(int nw, int M, int N, const double2* __restrict__ Gr, float* __restrict__ feat,
                                long long ld, long long off)
{
    const long long per = (long long)N * M;
    const long long total = (long long)nw * per;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long w = e / per, jq = e % per;
        const double2 g = Gr[e];
        float* o = feat + w * ld + off + jq * 2;
        o[0] = (float)g.x;
        o[1] = (float)g.y;
    }
}

void launch_features_rows(int nw, int M, int N, const double2* Gr, float* feat, long long ld, long long off,
                          cudaStream_t st)
{
    const long long total = (long long)nw * N * M;
    if (total <= 0) return;
    k_features_rows<<<grid_of(total), 256, 0, st>>>(nw, M, N, Gr, feat, ld, off);
    msd_note_launch();
}

void launch_features(int nw, int M, int N, int n_core, int n_act, const int* pos0, const double2* Gr, float* feat,
                     int spin, cudaStream_t st)
{
    const long long total = (long long)nw * n_act * n_act;
    if (total <= 0) return;
    k_features<<<grid_of(total), 256, 0, st>>>(nw, M, N, n_core, n_act, pos0, Gr, feat, spin);
    msd_note_launch();
}

// ========================================================================
struct msd_mlp {
    int device = 0, n_in = 0, width = 0;
    std::string err;
    long long n_params = 0;
    long long off_w[4], off_b[4];
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wb[3] = {}, *wt[3] = {};
    int cap = 0, capt = 0;       // batch capacity, transposed leading dimension (multiple of 64)
    bf16 *xb = nullptr, *xt = nullptr;
    float* z[3] = {};
    bf16 *h[3] = {}, *ht[3] = {};
    float *dzf[3] = {}, *dh = nullptr, *y = nullptr, *dy = nullptr, *acc = nullptr;
    bf16 *dz[3] = {}, *dzt[3] = {};
    unsigned* d_err = nullptr;
    long long step = 0;
};

namespace {

int mfail(msd_mlp* m, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (m) m->err = buf;
    return code;
}

#define MCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return mfail(m, MSD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void mfree(msd_mlp* m)
{
    cudaFree(m->xb); cudaFree(m->xt); cudaFree(m->dh); cudaFree(m->y); cudaFree(m->dy); cudaFree(m->acc);
    for (int l = 0; l < 3; ++l) {
        cudaFree(m->z[l]); cudaFree(m->h[l]); cudaFree(m->ht[l]); cudaFree(m->dzf[l]); cudaFree(m->dz[l]);
        cudaFree(m->dzt[l]);
        m->z[l] = m->dzf[l] = nullptr;
        m->h[l] = m->ht[l] = m->dz[l] = m->dzt[l] = nullptr;
    }
    m->xb = m->xt = nullptr;
    m->dh = m->y = m->dy = m->acc = nullptr;
    m->cap = m->capt = 0;
}

int ensure_batch(msd_mlp* m, int B)
{
    if (B <= m->cap) return MSD_OK;
    mfree(m);
    const int cap = (B + 63) / 64 * 64, W = m->width;
    m->cap = cap;
    m->capt = cap;
    MCK(cudaMalloc(&m->xb, sizeof(bf16) * cap * m->n_in));
    MCK(cudaMalloc(&m->xt, sizeof(bf16) * cap * m->n_in));
    for (int l = 0; l < 3; ++l) {
        MCK(cudaMalloc(&m->z[l], sizeof(float) * cap * W));
        MCK(cudaMalloc(&m->h[l], sizeof(bf16) * cap * W));
        MCK(cudaMalloc(&m->ht[l], sizeof(bf16) * cap * W));
        MCK(cudaMalloc(&m->dzf[l], sizeof(float) * cap * W));
        MCK(cudaMalloc(&m->dz[l], sizeof(bf16) * cap * W));
        MCK(cudaMalloc(&m->dzt[l], sizeof(bf16) * cap * W));
    }
    MCK(cudaMalloc(&m->dh, sizeof(float) * cap * W));
    MCK(cudaMalloc(&m->y, sizeof(float) * cap));
    MCK(cudaMalloc(&m->dy, sizeof(float) * cap));
    MCK(cudaMalloc(&m->acc, sizeof(float) * (size_t)cap * (W > m->n_in ? W : m->n_in)));
    return MSD_OK;
}

int refresh_bf16(msd_mlp* m, cudaStream_t st)
{
    const int ins[3] = {m->n_in, m->width, m->width};
    for (int l = 0; l < 3; ++l) {
        k_weights_bf16<<<grid_of((long long)m->width * ins[l]), 256, 0, st>>>(m->width, ins[l], m->p + m->off_w[l],
                                                                              m->wb[l], m->wt[l]);
        msd_note_launch();
    }
    MCK(cudaGetLastError());
    return MSD_OK;
}

int forward(msd_mlp* m, int B, const float* x, cudaStream_t st)
{
    int rc = ensure_batch(m, B);
    if (rc) return rc;
    const int W = m->width, ld = m->capt;
    // transposed copies: columns beyond B stay zero (they are the K padding
    // of the weight-gradient products)
    MCK(cudaMemsetAsync(m->xt, 0, sizeof(bf16) * (size_t)ld * m->n_in, st));
    for (int l = 0; l < 3; ++l) MCK(cudaMemsetAsync(m->ht[l], 0, sizeof(bf16) * (size_t)ld * W, st));
    k_in_bf16<<<grid_of((long long)B * m->n_in), 256, 0, st>>>(B, m->n_in, x, m->xb, m->xt, ld);
    msd_note_launch();
    const bf16* in = m->xb;
    int K = m->n_in;
    for (int l = 0; l < 3; ++l) {
        if (tc_gemm_bf16(in, K, m->wb[l], K, B, W, K, m->z[l], W, m->d_err, st))
            return mfail(m, MSD_ERR_CUDA, "tensor-core GEMM launch failed (forward layer %d)", l);
        k_bias_gelu<<<grid_of((long long)B * W), 256, 0, st>>>(B, W, m->z[l], m->p + m->off_b[l], m->h[l], m->ht[l],
                                                                ld);
        msd_note_launch();
        in = m->h[l];
        K = W;
    }
    k_out<<<(B * 32 + 255) / 256, 256, 0, st>>>(B, W, m->h[2], m->p + m->off_w[3], m->p + m->off_b[3], m->y);
    msd_note_launch();
    MCK(cudaGetLastError());
    return MSD_OK;
}

}  // namespace

extern "C" {

int msd_mlp_create(msd_mlp** out, int n_in, int width, int device)
{
    if (!out) return MSD_ERR_ARG;
    *out = nullptr;
    if (n_in <= 0 || width <= 0 || n_in % 64 || width % 64) return MSD_ERR_SHAPE;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return MSD_ERR_CUDA; }
    msd_mlp* m = new msd_mlp();
    m->device = device;
    m->n_in = n_in;
    m->width = width;
    const int ins[4] = {n_in, width, width, width}, outs[4] = {width, width, width, 1};
    long long off = 0;
    for (int l = 0; l < 4; ++l) {
        m->off_w[l] = off; off += (long long)outs[l] * ins[l];
        m->off_b[l] = off; off += outs[l];
    }
    m->n_params = off;
    bool ok = cudaMalloc(&m->p, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc(&m->g, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc(&m->m, sizeof(float) * off) == cudaSuccess &&
              cudaMalloc(&m->v, sizeof(float) * off) == cudaSuccess &&
              msd_err_word_alloc(&m->d_err) == 0;
    for (int l = 0; ok && l < 3; ++l)
        ok = cudaMalloc(&m->wb[l], sizeof(bf16) * width * ins[l]) == cudaSuccess &&
             cudaMalloc(&m->wt[l], sizeof(bf16) * width * ins[l]) == cudaSuccess;
    if (!ok) { cudaGetLastError(); delete m; return MSD_ERR_NOMEM; }
    cudaMemset(m->p, 0, sizeof(float) * off);
    cudaMemset(m->g, 0, sizeof(float) * off);
    cudaMemset(m->m, 0, sizeof(float) * off);
    cudaMemset(m->v, 0, sizeof(float) * off);
    *out = m;
    return MSD_OK;
}

void msd_mlp_destroy(msd_mlp* m)
{
    if (!m) return;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    mfree(m);
    cudaFree(m->p); cudaFree(m->g); cudaFree(m->m); cudaFree(m->v); cudaFree(m->d_err);
    for (int l = 0; l < 3; ++l) { cudaFree(m->wb[l]); cudaFree(m->wt[l]); }
    delete m;
}

const char* msd_mlp_last_error(const msd_mlp* m) { return m ? m->err.c_str() : ""; }

long long msd_mlp_param_count(const msd_mlp* m) { return m ? m->n_params : 0; }

int msd_mlp_set_params(msd_mlp* m, const float* params)
{
    if (!m || !params) return MSD_ERR_ARG;
    MCK(cudaSetDevice(m->device));
    MCK(cudaMemcpy(m->p, params, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
    MCK(cudaMemset(m->m, 0, sizeof(float) * m->n_params));
    MCK(cudaMemset(m->v, 0, sizeof(float) * m->n_params));
    m->step = 0;
    int rc = refresh_bf16(m, nullptr);
    if (rc) return rc;
    MCK(cudaDeviceSynchronize());
    return MSD_OK;
}

int msd_mlp_get_params(msd_mlp* m, float* params)
{
    if (!m || !params) return MSD_ERR_ARG;
    MCK(cudaSetDevice(m->device));
    MCK(cudaMemcpy(params, m->p, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
    return MSD_OK;
}

int msd_mlp_forward(msd_mlp* m, int batch, const float* x, float* y, void* stream)
{
    if (!m || batch < 0 || (batch > 0 && (!x || !y))) return m ? mfail(m, MSD_ERR_ARG, "bad arguments") : MSD_ERR_ARG;
    if (batch == 0) return MSD_OK;
    cudaStream_t st = (cudaStream_t)stream;
    MCK(cudaSetDevice(m->device));
    int rc = forward(m, batch, x, st);
    if (rc) return rc;
    MCK(cudaMemcpyAsync(y, m->y, sizeof(float) * batch, cudaMemcpyDeviceToDevice, st));
    return MSD_OK;
}

int msd_mlp_grad(msd_mlp* m, int batch, const float* x, const float* target, float* grads, float* loss,
                 void* stream)
{
    if (!m || batch <= 0 || !x || !target) return m ? mfail(m, MSD_ERR_ARG, "bad arguments") : MSD_ERR_ARG;
    if (batch > 65536) return mfail(m, MSD_ERR_SHAPE, "batch above 65536");
    cudaStream_t st = (cudaStream_t)stream;
    MCK(cudaSetDevice(m->device));
    int rc = forward(m, batch, x, st);
    if (rc) return rc;
    const int B = batch, W = m->width, ld = m->capt;
    k_loss<<<1, 1024, 0, st>>>(B, m->y, target, m->dy, loss);
    msd_note_launch();
    // output layer
    k_out_back_w<<<W, 256, 0, st>>>(B, W, m->dy, m->h[2], m->g + m->off_w[3], m->g + m->off_b[3]);
    msd_note_launch();
    for (int l = 0; l < 3; ++l) MCK(cudaMemsetAsync(m->dzt[l], 0, sizeof(bf16) * (size_t)ld * W, st));
    k_out_back_dz<<<grid_of((long long)B * W), 256, 0, st>>>(B, W, m->dy, m->p + m->off_w[3], m->z[2], m->dzf[2],
                                                             m->dz[2], m->dzt[2], ld);
    msd_note_launch();
    for (int l = 2; l >= 0; --l) {
        const int in = l ? W : m->n_in;
        // dW_l[n][k] = sum_b dz_l[b][n] a_l[b][k]: K = batch (padded columns are zero)
        const bf16* at = l ? m->ht[l - 1] : m->xt;
        if (tc_gemm_bf16(m->dzt[l], ld, at, ld, W, in, ld, m->g + m->off_w[l], in, m->d_err, st))
            return mfail(m, MSD_ERR_CUDA, "tensor-core GEMM launch failed (weight gradient %d)", l);
        k_colsum<<<W, 256, 0, st>>>(B, W, m->dzf[l], m->g + m->off_b[l]);
        msd_note_launch();
        if (l == 0) break;
        // dh_{l-1}[b][k] = sum_n dz_l[b][n] W_l[n][k]
        if (tc_gemm_bf16(m->dz[l], W, m->wt[l], W, B, W, W, m->dh, W, m->d_err, st))
            return mfail(m, MSD_ERR_CUDA, "tensor-core GEMM launch failed (input gradient %d)", l);
        k_gelu_back<<<grid_of((long long)B * W), 256, 0, st>>>(B, W, m->dh, m->z[l - 1], m->dzf[l - 1], m->dz[l - 1],
                                                               m->dzt[l - 1], ld);
        msd_note_launch();
    }
    MCK(cudaGetLastError());
    if (grads) MCK(cudaMemcpyAsync(grads, m->g, sizeof(float) * m->n_params, cudaMemcpyDeviceToDevice, st));
    return MSD_OK;
}

int msd_mlp_adam_step(msd_mlp* m, float lr, float beta1, float beta2, float eps, void* stream)
{
    if (!m) return MSD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    MCK(cudaSetDevice(m->device));
    m->step += 1;
    const float c1 = 1.f - powf(beta1, (float)m->step), c2 = 1.f - powf(beta2, (float)m->step);
    k_adam<<<grid_of(m->n_params), 256, 0, st>>>(m->n_params, m->p, m->g, m->m, m->v, lr, beta1, beta2, eps, c1, c2);
    msd_note_launch();
    return refresh_bf16(m, st);
}

}  // extern "C"
