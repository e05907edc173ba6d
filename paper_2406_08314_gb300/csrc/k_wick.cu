// Reference inverse, excitation-string minors and CI weights: the overlap
// part of the generalized-Wick evaluation (Sec. III "Implementation":
// get_dets), plus the cofactor accumulation behind the mixed Green's
// function (reduce_CI) and its rank-n_p update.
#include <type_traits>

#include "common.cuh"
#include "kernels.h"

// ------------------------------------------------------------------------
// Reference determinant per (walker, spin): S = D0^dag phi = phi[occ0, :]
// (Sec. II A overlap of two determinants). LU with partial pivoting in
// FP64 gives O0 = det S and S^-1; then
//   Gr[j][r]  = (phi S^-1)[r][j] = G[occ0_j][r]   (G = G0^T, G0 = Theta D0^dag)
//               (rows r in occ0 of phi are S itself, so there Gr is exactly
//               the identity and is written, not computed)
//   Gact[h][p] = G[H_h][P_p]                       (active hole x particle block)
// One block per walker. A walker whose |det S| falls below 1e-14 times the
// product of the column norms of S is flagged singular.
__global__ void __launch_bounds__(256)
k_ref(const double2* __restrict__ phi, int M, int N, const int* __restrict__ occ0,
      const int* __restrict__ pos0, const int* __restrict__ hole_pos, int nh, const int* __restrict__ part_orb,
      int np,
      double2* __restrict__ Gr, double2* __restrict__ O0, double2* __restrict__ Gact,
      unsigned* err)
{
    extern __shared__ double2 sm[];
    double2* S = sm;              // [N][N] LU in place
    double2* Si = S + N * N;      // [N][N] inverse
    __shared__ int piv[MSD_NMAX];
    __shared__ double cn[MSD_NMAX];
    __shared__ int singular;
    const int w = blockIdx.x;
    const int t = threadIdx.x, nt = blockDim.x;
    const double2* ph = phi + (size_t)w * M * N;

    for (int e = t; e < N * N; e += nt) S[e] = ph[(size_t)occ0[e / N] * N + e % N];
    if (t == 0) singular = 0;
    __syncthreads();
    for (int j = t; j < N; j += nt) {
        double a = 0;
        for (int i = 0; i < N; ++i) a += S[i * N + j].x * S[i * N + j].x + S[i * N + j].y * S[i * N + j].y;
        cn[j] = sqrt(a);
    }
    for (int k = 0; k < N; ++k) {
        if (t < 32) {
            double best = -1; int bi = k;
            for (int i = k + t; i < N; i += 32) {
                double v = S[i * N + k].x * S[i * N + k].x + S[i * N + k].y * S[i * N + k].y;
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o; o >>= 1) {
                double ob = __shfl_down_sync(0xffffffffu, best, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (t == 0) { piv[k] = bi; if (best == 0.0) singular = 1; }
        }
        __syncthreads();
        if (singular) break;
        const int p = piv[k];
        if (p != k)
            for (int j = t; j < N; j += nt) { double2 a = S[k * N + j]; S[k * N + j] = S[p * N + j]; S[p * N + j] = a; }
        __syncthreads();
        for (int i = k + 1 + t; i < N; i += nt) S[i * N + k] = cdiv(S[i * N + k], S[k * N + k]);
        __syncthreads();
        const int m = N - k - 1;
        for (int e = t; e < m * m; e += nt) {
            int i = k + 1 + e / m, j = k + 1 + e % m;
            S[i * N + j] = cfms(S[i * N + k], S[k * N + j], S[i * N + j]);
        }
        __syncthreads();
    }
    __shared__ double2 det;
    if (t == 0) {
        double2 d = cz(1, 0);
        double nrm = 1;
        if (!singular) {
            for (int k = 0; k < N; ++k) { d = cmul(d, S[k * N + k]); if (piv[k] != k) d = cz(-d.x, -d.y); nrm *= cn[k]; }
            if (!(sqrt(d.x * d.x + d.y * d.y) > 1e-14 * nrm)) singular = 1;
        }
        if (singular) { d = cz(0, 0); atomicOr(err, MSD_DEV_ERR_SINGULAR); }
        det = d;
        O0[w] = d;
    }
    __syncthreads();
    if (singular) {
        for (int e = t; e < N * M; e += nt) Gr[(size_t)w * N * M + e] = cz(0, 0);
        for (int e = t; e < nh * np; e += nt) Gact[(size_t)w * nh * np + e] = cz(0, 0);
        return;
    }
    // S^-1 column c: solve L U x = P e_c
    for (int c = t; c < N; c += nt) {
        double2 x[MSD_NMAX];
        for (int i = 0; i < N; ++i) x[i] = cz(i == c ? 1 : 0, 0);
        for (int k = 0; k < N; ++k) { int p = piv[k]; if (p != k) { double2 a = x[k]; x[k] = x[p]; x[p] = a; } }
        for (int i = 0; i < N; ++i)
            for (int k = 0; k < i; ++k) x[i] = cfms(S[i * N + k], x[k], x[i]);
        for (int i = N - 1; i >= 0; --i) {
            for (int k = i + 1; k < N; ++k) x[i] = cfms(S[i * N + k], x[k], x[i]);
            x[i] = cdiv(x[i], S[i * N + i]);
        }
        for (int i = 0; i < N; ++i) Si[i * N + c] = x[i];
    }
    __syncthreads();
    double2* gr = Gr + (size_t)w * N * M;
    // lanes over the columns j (S^-1 row reads contiguous, the phi element a
    // broadcast), warps over the rows r
    const int JW = N <= 32 ? 32 : 64;
    for (int e = t; e < M * JW; e += nt) {
        const int r = e / JW, j = e - r * JW;
        if (j >= N) continue;
        const int q = pos0[r];
        if (q >= 0) {
            gr[(size_t)j * M + r] = cz(q == j ? 1.0 : 0.0, 0.0);
            continue;
        }
        const double2* pr = ph + (size_t)r * N;
        double2 a = cz(0, 0);
        for (int k = 0; k < N; ++k) a = cfma(pr[k], Si[k * N + j], a);
        gr[(size_t)j * M + r] = a;
    }
    for (int e = t; e < nh * np; e += nt) {
        const int h = e / np, p = e % np;
        const double2* pr = ph + (size_t)part_orb[p] * N;
        const int j = hole_pos[h];
        double2 a = cz(0, 0);
        for (int k = 0; k < N; ++k) a = cfma(pr[k], Si[k * N + j], a);
        Gact[(size_t)w * nh * np + e] = a;
    }
}

void launch_ref(const double2* phi, int nw, int M, int N, const SpinTables& T, double2* Gr,
                double2* O0, double2* Gact, unsigned* err, cudaStream_t st)
{
    size_t smem = sizeof(double2) * 2 * N * N;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k_ref, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ref<<<nw, 256, smem, st>>>(phi, M, N, T.occ0, T.pos0, T.hole_pos, T.nh, T.part_orb, T.np, Gr, O0,
                                 Gact, err); msd_note_launch();
}

// ------------------------------------------------------------------------
// Excitation strings of level K for one spin (get_dets / build_det_matrix):
// A[i][j] = G[h_i][p_j] (a K x K minor of G). LU with partial pivoting in
// FP64 gives r = sign * det A, the overlap ratio <D_s|phi>/<D_0|phi> of the
// string's spin sector. B = A^-1 is stored per string, K*K entries
// contiguous (B[i][j] at i*K + j), for the Green's-function and energy
// terms: in FP64 mode solved from the FP64 LU factors; in mixed mode from an
// FP32 elimination of the same row order (the FP64 pivots) on an FP32 copy of
// the active block. One thread per (walker, string); the walker's active
// block lives in shared memory.
//
// FP64 issue rate is the bound here (a few FP64 operations per clock per
// SM), so the LU spends FP64 operations on the elimination and the
// determinant only: the pivot search compares integer magnitude keys (the
// larger high word of |Re|, |Im|: partial pivoting by the max-norm), the row
// swaps count parity in an integer, and the pivot reciprocals are
// Newton-Raphson iterations from an FP32 seed.

// 1 / m for m > 0: y <- y + y (1 - m y) (Newton-Raphson for f(y) = 1/y - m),
// two steps from the FP32 reciprocal (~2^-22 relative) reach FP64 rounding
// (2^-44, then below 2^-53 before rounding). Outside the FP32 normal range
// the quotient is taken directly.
__device__ __forceinline__ double recip_nr(double m)
{
    if (!(m > 1e-36 && m < 1e36)) return 1.0 / m;
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"((float)m));
    double y = (double)yf;
    double e = fma(-m, y, 1.0);
    y = fma(y, e, y);
    e = fma(-m, y, 1.0);
    return fma(y, e, y);
}

// monotone in max(|Re v|, |Im v|) up to the low 32 bits of each mantissa
__device__ __forceinline__ int mag_key(double2 v)
{
    return max(__double2hiint(v.x) & 0x7fffffff, __double2hiint(v.y) & 0x7fffffff);
}

template <int K, typename T>
__global__ void __launch_bounds__(128)
k_strings(SpinTables tb, int nw, const double2* __restrict__ Gact, double2* __restrict__ r,
          float2* __restrict__ rf, void* __restrict__ Bout, int want_b)
{
    using T2 = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;
    constexpr bool F32B = std::is_same<T, float>::value;
    __shared__ double2 g[MSD_XMAX];
    __shared__ float2 gf[F32B ? MSD_XMAX : 1];
    const int w = blockIdx.y;
    const int X = tb.nh * tb.np;
    for (int e = threadIdx.x; e < X; e += blockDim.x) {
        const double2 v = Gact[(size_t)w * X + e];
        g[e] = v;
        if constexpr (F32B) gf[e] = make_float2((float)v.x, (float)v.y);
    }
    __syncthreads();
    const int ns = tb.bucket[K + 1] - tb.bucket[K];
    const int sl = blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= ns) return;
    const int s = tb.bucket[K] + sl;
    const uint4 rec = tb.str_hp[s];
    double2 a[K][K];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j < K; ++j) a[i][j] = g[rec_h(rec, i) * tb.np + rec_p(rec, j)];
    int perm[K];
#pragma unroll
    for (int i = 0; i < K; ++i) perm[i] = i;
    double2 det = cz(tb.str_sign[s], 0);
    double2 dinv[K];
    bool sing = false;
    int odd = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int p = k, best = mag_key(a[k][k]);
        double2 pv = a[k][k];
#pragma unroll
        for (int i = k + 1; i < K; ++i) {
            const int v = mag_key(a[i][k]);
            if (v > best) { best = v; p = i; pv = a[i][k]; }
        }
        if (pv.x == 0.0 && pv.y == 0.0) sing = true;
#pragma unroll
        for (int i = k + 1; i < K; ++i) {
            if (i == p) {
#pragma unroll
                for (int j = 0; j < K; ++j) { double2 tt = a[k][j]; a[k][j] = a[i][j]; a[i][j] = tt; }
                int tp = perm[k]; perm[k] = perm[i]; perm[i] = tp;
                odd ^= 1;
            }
        }
        det = cmul(det, a[k][k]);
        const double m2 = fma(a[k][k].x, a[k][k].x, a[k][k].y * a[k][k].y);
        const double im2 = sing ? 0.0 : recip_nr(m2);
        dinv[k] = cz(a[k][k].x * im2, -a[k][k].y * im2);
        if (k + 1 < K) {
#pragma unroll
            for (int i = k + 1; i < K; ++i) {
                const double2 f = cmul(a[i][k], dinv[k]);
                a[i][k] = f;
#pragma unroll
                for (int j = k + 1; j < K; ++j) a[i][j] = cfms(f, a[k][j], a[i][j]);
            }
        }
    }
    if (odd) det = cz(-det.x, -det.y);
    if (sing) det = cz(0, 0);
    r[(size_t)w * tb.n_str + s] = det;
    if (rf) rf[(size_t)w * tb.n_str + s] = make_float2((float)det.x, (float)det.y);
    if (!want_b) return;
    // B = A^-1 from P A = L U: column c solves L U x = P e_c, in precision T.
    T2 lu[K][K], di[K];
    if constexpr (F32B) {
        // FP32 elimination of the rows in the FP64 pivot order
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int ro = rec_h(rec, perm[i]) * tb.np;
#pragma unroll
            for (int j = 0; j < K; ++j) lu[i][j] = gf[ro + rec_p(rec, j)];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float m2 = fmaf(lu[k][k].x, lu[k][k].x, lu[k][k].y * lu[k][k].y);
            const float im2 = (sing || !(m2 > 0.f)) ? 0.f : 1.f / m2;
            di[k] = make_float2(lu[k][k].x * im2, -lu[k][k].y * im2);
#pragma unroll
            for (int i = k + 1; i < K; ++i) {
                const float2 f = fmul(lu[i][k], di[k]);
                lu[i][k] = f;
#pragma unroll
                for (int j = k + 1; j < K; ++j) {
                    lu[i][j].x -= f.x * lu[k][j].x - f.y * lu[k][j].y;
                    lu[i][j].y -= f.x * lu[k][j].y + f.y * lu[k][j].x;
                }
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            di[i] = T2{(T)dinv[i].x, (T)dinv[i].y};
#pragma unroll
            for (int j = 0; j < K; ++j) lu[i][j] = T2{(T)a[i][j].x, (T)a[i][j].y};
        }
    }
    T2* B = reinterpret_cast<T2*>(Bout) + (size_t)tb.b_off[K] + ((size_t)w * ns + sl) * b_stride(K);
    if (K & 1) B[K * K] = T2{0, 0};   // the pad entry
#pragma unroll
    for (int c = 0; c < K; ++c) {
        T2 x[K];
#pragma unroll
        for (int i = 0; i < K; ++i) x[i] = T2{(T)(perm[i] == c ? 1 : 0), (T)0};
#pragma unroll
        for (int i = 0; i < K; ++i)
#pragma unroll
            for (int k = 0; k < i; ++k) {
                x[i].x -= lu[i][k].x * x[k].x - lu[i][k].y * x[k].y;
                x[i].y -= lu[i][k].x * x[k].y + lu[i][k].y * x[k].x;
            }
#pragma unroll
        for (int i = K - 1; i >= 0; --i) {
#pragma unroll
            for (int k = i + 1; k < K; ++k) {
                x[i].x -= lu[i][k].x * x[k].x - lu[i][k].y * x[k].y;
                x[i].y -= lu[i][k].x * x[k].y + lu[i][k].y * x[k].x;
            }
            const T2 t = x[i];
            x[i] = T2{t.x * di[i].x - t.y * di[i].y, t.x * di[i].y + t.y * di[i].x};
        }
#pragma unroll
        for (int i = 0; i < K; ++i) B[i * K + c] = x[i];
    }
}

template <int K>
static void launch_strings_k(const SpinTables& tb, int nw, const double2* Gact, double2* r, float2* rf, void* B,
                             bool fp32, int want_b, cudaStream_t st)
{
    const int ns = tb.bucket[K + 1] - tb.bucket[K];
    if (ns <= 0) return;
    dim3 grid((ns + 127) / 128, nw);
    if (fp32) k_strings<K, float><<<grid, 128, 0, st>>>(tb, nw, Gact, r, rf, B, want_b);
    else k_strings<K, double><<<grid, 128, 0, st>>>(tb, nw, Gact, r, rf, B, want_b);
    msd_note_launch();
}

// Reference string (level 0): ratio 1.
__global__ void k_ref_string(int nw, int n_str, double2* r, float2* rf)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) {
        r[(size_t)w * n_str] = cz(1, 0);
        if (rf) rf[(size_t)w * n_str] = make_float2(1.f, 0.f);
    }
}

void launch_strings(const SpinTables& tb, int nw, const double2* Gact, double2* r, float2* rf, void* B,
                    bool fp32, bool want_b, cudaStream_t st, const TimerHook& th)
{
    if (tb.bucket[1] > tb.bucket[0]) {
        th.begin("k_ref_string", st);
        k_ref_string<<<(nw + 127) / 128, 128, 0, st>>>(nw, tb.n_str, r, rf); msd_note_launch();
        th.end(st);
    }
    th.begin("k_strings", st);
    launch_strings_k<1>(tb, nw, Gact, r, rf, B, fp32, want_b, st);
    launch_strings_k<2>(tb, nw, Gact, r, rf, B, fp32, want_b, st);
    launch_strings_k<3>(tb, nw, Gact, r, rf, B, fp32, want_b, st);
    launch_strings_k<4>(tb, nw, Gact, r, rf, B, fp32, want_b, st);
    launch_strings_k<5>(tb, nw, Gact, r, rf, B, fp32, want_b, st);
    launch_strings_k<6>(tb, nw, Gact, r, rf, B, fp32, want_b, st);
    th.end(st);
}

// ------------------------------------------------------------------------
// CI weights per string: w_s = sum over determinants I containing string s
// of c_I * r_other(I), so that sum_I c_I r_a r_b = sum_a r_a w_a. Stored is
// the product r_s w_s (what every consumer needs); for spin alpha the block
// also reduces it into per-walker partial sums. A thread takes one string
// for WB walkers: each entry of the string's determinant list (index and
// coefficient) is read once and feeds WB independent gathers; every
// walker's sum runs in list order as with one walker per thread.
template <int WB>
__global__ void __launch_bounds__(256)
k_weights(SpinTables tb, int nw, const double2* __restrict__ r_self, const double2* __restrict__ r_other,
          int n_other, double2* __restrict__ wts, double2* __restrict__ part, int nslot,
          int slot0)
{
    const int w0 = blockIdx.y * WB;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double2 rw[WB];
#pragma unroll
    for (int k = 0; k < WB; ++k) rw[k] = cz(0, 0);
    if (s < tb.n_str) {
        double2 acc[WB];
#pragma unroll
        for (int k = 0; k < WB; ++k) acc[k] = cz(0, 0);
        const double2* ro = r_other + (size_t)w0 * n_other;
        const int e1 = tb.csr_off[s + 1];
        for (int e = tb.csr_off[s]; e < e1; ++e) {
            const int o = tb.csr_other[e];
            const double c = tb.csr_c[e];
#pragma unroll
            for (int k = 0; k < WB; ++k)
                if (w0 + k < nw) acc[k] = cadd(acc[k], cscale(ro[(size_t)k * n_other + o], c));
        }
#pragma unroll
        for (int k = 0; k < WB; ++k)
            if (w0 + k < nw) {
                rw[k] = cmul(r_self[(size_t)(w0 + k) * tb.n_str + s], acc[k]);
                wts[(size_t)(w0 + k) * tb.n_str + s] = rw[k];
            }
    }
    if (part) {
        __shared__ double2 red[256];
        for (int k = 0; k < WB && w0 + k < nw; ++k) {
            red[threadIdx.x] = rw[k];
            __syncthreads();
            for (int o = blockDim.x / 2; o; o >>= 1) {
                if (threadIdx.x < o) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + o]);
                __syncthreads();
            }
            if (threadIdx.x == 0) part[(size_t)(w0 + k) * nslot + slot0 + blockIdx.x] = red[0];
            __syncthreads();   // red is reused by the next walker
        }
    }
}

int weights_blocks(const SpinTables& tb) { return (tb.n_str + 255) / 256; }

void launch_weights(const SpinTables& tb, int nw, const double2* r_self, const double2* r_other,
                    int n_other, double2* wts, double2* part, int nslot, int slot0, cudaStream_t st)
{
    constexpr int WB = 4;
    dim3 grid(weights_blocks(tb), (nw + WB - 1) / WB);
    k_weights<WB><<<grid, 256, 0, st>>>(tb, nw, r_self, r_other, n_other, wts, part, nslot, slot0);
    msd_note_launch();
}

// ------------------------------------------------------------------------
// Per-determinant ratios r_I = r_a(I) * r_b(I) in the caller's order.
__global__ void k_det_ratios(PairTables pt, int n_str_a, int n_str_b, const double2* __restrict__ ra,
                             const double2* __restrict__ rb, double2* __restrict__ out)
{
    const int w = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pt.n_det) return;
    out[(size_t)w * pt.n_det + pt.det_index[i]] =
        cmul(ra[(size_t)w * n_str_a + pt.a[i]], rb[(size_t)w * n_str_b + pt.b[i]]);
}

void launch_det_ratios(const PairTables& pt, int nw, int n_str_a, int n_str_b, const double2* ra,
                       const double2* rb, double2* out, cudaStream_t st)
{
    dim3 grid((pt.n_det + 255) / 256, nw);
    k_det_ratios<<<grid, 256, 0, st>>>(pt, n_str_a, n_str_b, ra, rb, out); msd_note_launch();
}

// Sum of partial slots [slot0, slot0 + n) per walker -> out[w] (and
// O_T = O0a * O0b * sum when ovlp is given).
__global__ void k_sum_slots(int nw, const double2* __restrict__ part, int nslot, int slot0, int n,
                            double2* __restrict__ out, const double2* __restrict__ O0a,
                            const double2* __restrict__ O0b, double2* __restrict__ ovlp)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nw) return;
    double2 a = cz(0, 0);
    for (int i = 0; i < n; ++i) a = cadd(a, part[(size_t)w * nslot + slot0 + i]);
    if (out) out[w] = a;
    if (ovlp) ovlp[w] = cmul(cmul(O0a[w], O0b[w]), a);
}

void launch_sum_slots(int nw, const double2* part, int nslot, int slot0, int n, double2* out,
                      const double2* O0a, const double2* O0b, double2* ovlp, cudaStream_t st)
{
    k_sum_slots<<<(nw + 127) / 128, 128, 0, st>>>(nw, part, nslot, slot0, n, out, O0a, O0b, ovlp); msd_note_launch();
}

// ------------------------------------------------------------------------
// Cofactor accumulation (reduce_CI): per (walker, spin)
//   Cm[p][h] = sum_s w_s r_s B_s[i][j]  at (p_i, h_j) = (p, h)
// (wts holds the products r_s w_s).
// One block per walker. The k^2 entries of one string's minor land on
// distinct (p, h), so a group of lanes takes a whole string at once and adds
// its entries into the group's own shared-memory copy of Cm with plain
// read-modify-writes: B is read in its stored order (coalesced) and nothing
// is atomic. Strings with k^2 <= 16 go two to a warp (half-warp groups),
// longer ones one to a warp. Each group takes its strings in ascending order
// and the copies are summed in a fixed order, so the result does not depend
// on scheduling. Products and the per-copy sums are in T (double in FP64
// mode, float in mixed mode); the copies are summed in double.
#define CMAT_COPIES 16
template <typename T, int GS, int EPL, int U>
__device__ __forceinline__ void cmat_level(T* __restrict__ a, int g, int ng, int l, int kk, int kst, int ns, int s0,
                                           const T* __restrict__ B, const uint8_t* __restrict__ xt,
                                           const double2* __restrict__ ww)
{
    for (int base = 0; base < ns; base += ng * U) {
        T vr[U][EPL], vi[U][EPL];
        int vx[U][EPL];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int sl = base + u * ng + g;
            double2 f = cz(0, 0);
            if (sl < ns) f = ww[s0 + sl];
            const T fr = (T)f.x, fi = (T)f.y;
#pragma unroll
            for (int q = 0; q < EPL; ++q) {
                const int e = l + q * GS;
                vx[u][q] = -1;
                vr[u][q] = 0;
                vi[u][q] = 0;
                if (sl < ns && e < kk) {
                    const size_t o = (size_t)sl * kk + e, ob = (size_t)sl * kst + e;
                    const T br = B[2 * ob], bi = B[2 * ob + 1];
                    vx[u][q] = xt[o];
                    vr[u][q] = fr * br - fi * bi;
                    vi[u][q] = fr * bi + fi * br;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int q = 0; q < EPL; ++q)
                if (vx[u][q] >= 0) {
                    a[2 * vx[u][q]] += vr[u][q];
                    a[2 * vx[u][q] + 1] += vi[u][q];
                }
            __syncwarp();   // the group's next string may share entries with this one
        }
    }
}

template <typename T>
__device__ __forceinline__ void cmat_walker(const SpinTables& tb, int w, const double2* __restrict__ wts,
                                            const void* __restrict__ Bin, double2* __restrict__ Cm, T* accp)
{
    T (*acc)[2 * MSD_XMAX] = reinterpret_cast<T (*)[2 * MSD_XMAX]>(accp);
    const int X = tb.nh * tb.np;
    for (int e = threadIdx.x; e < CMAT_COPIES * 2 * MSD_XMAX; e += blockDim.x) accp[e] = 0;
    __syncthreads();
    const T* Bb = reinterpret_cast<const T*>(Bin);
    const double2* ww = wts + (size_t)w * tb.n_str;
    for (int k = 1; k <= MSD_KMAX; ++k) {
        const int s0 = tb.bucket[k], ns = tb.bucket[k + 1] - s0, kk = k * k;
        if (ns == 0) continue;
        const T* B = Bb + 2 * ((size_t)tb.b_off[k] + (size_t)w * ns * b_stride(k));
        const uint8_t* xt = tb.cmx + tb.cmx_off[k];
        if (kk <= 16)
            cmat_level<T, 16, 1, 3>(acc[threadIdx.x >> 4], threadIdx.x >> 4, 16, threadIdx.x & 15, kk, b_stride(k), ns, s0, B, xt,
                                    ww);
        else if (kk <= 32)
            cmat_level<T, 32, 1, 3>(acc[(threadIdx.x >> 5) * 2], threadIdx.x >> 5, 8, threadIdx.x & 31, kk, b_stride(k), ns, s0, B,
                                    xt, ww);
        else
            cmat_level<T, 32, 2, 3>(acc[(threadIdx.x >> 5) * 2], threadIdx.x >> 5, 8, threadIdx.x & 31, kk, b_stride(k), ns, s0, B,
                                    xt, ww);
    }
    __syncthreads();
    for (int x = threadIdx.x; x < X; x += blockDim.x) {
        double re = 0, im = 0;
        for (int q = 0; q < CMAT_COPIES; ++q) { re += (double)acc[q][2 * x]; im += (double)acc[q][2 * x + 1]; }
        Cm[(size_t)w * X + x] = cz(re, im);
    }
}

// Both spins in one grid (blockIdx.y = spin), so the two spins' blocks fill
// the machine together.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 3)
k_cmat(SpinTables ta, SpinTables tb, const double2* __restrict__ wts_a, const double2* __restrict__ wts_b,
       const void* __restrict__ Ba, const void* __restrict__ Bb, double2* __restrict__ Cm_a,
       double2* __restrict__ Cm_b)
{
    __shared__ T acc[CMAT_COPIES][2 * MSD_XMAX];
    if (blockIdx.y == 0) {
        if (ta.nh * ta.np > 0) cmat_walker<T>(ta, blockIdx.x, wts_a, Ba, Cm_a, &acc[0][0]);
    } else {
        if (tb.nh * tb.np > 0) cmat_walker<T>(tb, blockIdx.x, wts_b, Bb, Cm_b, &acc[0][0]);
    }
}

void launch_cmat(const SpinTables& ta, const SpinTables& tb, int nw, const double2* wts_a, const double2* wts_b,
                 const void* Ba, const void* Bb, bool fp32, double2* Cm_a, double2* Cm_b, cudaStream_t st)
{
    if (ta.nh * ta.np <= 0 && tb.nh * tb.np <= 0) return;
    const dim3 grid(nw, 2);
    if (fp32) k_cmat<float><<<grid, 256, 0, st>>>(ta, tb, wts_a, wts_b, Ba, Bb, Cm_a, Cm_b);
    else k_cmat<double><<<grid, 256, 0, st>>>(ta, tb, wts_a, wts_b, Ba, Bb, Cm_a, Cm_b);
    msd_note_launch();
}

// ------------------------------------------------------------------------
// Rows of the mixed Green's function G_T (Eq. 7 numerator), per (walker,
// spin), restricted to the rows that can be non-zero (occ0 then P):
//   Y[p][c] = sum_h Cm[p][h] G[H_h][c]
//   G_T[occ0_l][c] = G[occ0_l][c] - sum_p G[occ0_l][P_p] Y[p][c] / R
//   G_T[P_p][c]    = Y[p][c] / R
// Written to GT[w][row][c] with row stride M, at column offset `off` of a
// row of length ld (both spins are concatenated per walker). With
// minus_ref the reference part D0 D0^T (ones at (occ0_l, occ0_l)) is
// subtracted, for the mixed path that adds its contraction in FP64.
#define GT_COLS 16   // output columns per block
__global__ void __launch_bounds__(256)
k_gt(SpinTables tb, int M, const double2* __restrict__ Gr, const double2* __restrict__ Cm,
     const double2* __restrict__ Rsum, double2* __restrict__ GT, long long ld, long long off, int minus_ref)
{
    __shared__ double2 cm[MSD_XMAX];
    __shared__ double2 y[MSD_XMAX * GT_COLS];   // [np][GT_COLS columns]
    const int w = blockIdx.y;
    const int c0 = blockIdx.x * GT_COLS;
    const int N = tb.N, nh = tb.nh, np = tb.np;
    const double2* gr = Gr + (size_t)w * N * M;
    for (int e = threadIdx.x; e < nh * np; e += blockDim.x) cm[e] = Cm[(size_t)w * nh * np + e];
    __syncthreads();
    const double2 R = Rsum[w];
    const double2 iR = cdiv(cz(1, 0), R);
    for (int e = threadIdx.x; e < np * GT_COLS; e += blockDim.x) {
        const int p = e / GT_COLS, c = c0 + e % GT_COLS;
        double2 a = cz(0, 0);
        if (c < M)
            for (int h = 0; h < nh; ++h) a = cfma(cm[p * nh + h], gr[(size_t)tb.hole_pos[h] * M + c], a);
        y[e] = cmul(a, iR);
    }
    __syncthreads();
    double2* out = GT + (size_t)w * ld + off;
    for (int e = threadIdx.x; e < (N + np) * GT_COLS; e += blockDim.x) {
        const int x = e / GT_COLS, c = c0 + e % GT_COLS;
        if (c >= M) continue;
        double2 v;
        if (x < N) {
            v = gr[(size_t)x * M + c];
            for (int p = 0; p < np; ++p) v = cfms(gr[(size_t)x * M + tb.part_orb[p]], y[p * GT_COLS + e % GT_COLS], v);
            if (minus_ref && c == tb.occ0[x]) v.x -= 1.0;   // G_T - D0 D0^T
        } else {
            v = y[(x - N) * GT_COLS + e % GT_COLS];
        }
        out[(size_t)x * M + c] = v;
    }
}

void launch_gt(const SpinTables& tb, int nw, int M, const double2* Gr, const double2* Cm,
               const double2* R, double2* GT, long long ld, long long off, bool minus_ref, cudaStream_t st)
{
    dim3 grid((M + GT_COLS - 1) / GT_COLS, nw);
    k_gt<<<grid, 256, 0, st>>>(tb, M, Gr, Cm, R, GT, ld, off, minus_ref ? 1 : 0); msd_note_launch();
}

// The mixed one-body density matrix as full M x M matrices per walker and
// spin: rdm[w][spin][orb(x)][c] = GT[w][off + x M + c] for the rows x of G_T
// (occ0, then the particles); the caller zeroes the other rows.
__global__ void k_rdm_scatter(SpinTables tb, int M, const double2* __restrict__ GT, long long ld, long long off,
                              int spin, double2* __restrict__ rdm)
{
    const int x = blockIdx.x, w = blockIdx.y;
    const int orb = x < tb.N ? tb.occ0[x] : tb.part_orb[x - tb.N];
    const double2* src = GT + (size_t)w * ld + off + (size_t)x * M;
    double2* dst = rdm + (((size_t)w * 2 + spin) * M + orb) * M;
    for (int c = threadIdx.x; c < M; c += blockDim.x) dst[c] = src[c];
}

void launch_rdm_scatter(const SpinTables& tb, int nw, int M, const double2* GT, long long ld, long long off, int spin,
                        double2* rdm, cudaStream_t st)
{
    if (nw <= 0) return;
    k_rdm_scatter<<<dim3(tb.N + tb.np, nw), 128, 0, st>>>(tb, M, GT, ld, off, spin, rdm);
    msd_note_launch();
}

// <D_0|phi> = det(D0^dag phi_a) det(D0^dag phi_b) per walker.
__global__ void k_ref_ovlp(int nw, const double2* __restrict__ O0a, const double2* __restrict__ O0b,
                           double2* __restrict__ out)
{
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < nw) out[w] = cmul(O0a[w], O0b[w]);
}

void launch_ref_ovlp(int nw, const double2* O0a, const double2* O0b, double2* out, cudaStream_t st)
{
    k_ref_ovlp<<<(nw + 127) / 128, 128, 0, st>>>(nw, O0a, O0b, out); msd_note_launch();
}
