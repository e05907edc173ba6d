// Per-determinant energy terms shared by the per-system kernels
// (k_energy.cu) and the persistent batched kernel (k_batch.cu).
//
// string_energy_term: same-spin term of one excitation string s (level KL,
// index sl in its bucket) of walker w (string_energy_value: e_s alone):
//   r_s w_s e_s,  e_s = sum_ij B_ij Y[h_j][p_i] + 1/2 (Qc - Qx),
//   Qc = sum_ijkl B_ij B_kl K[(h_j,p_i)][(h_l,p_k)],
//   Qx = sum_ijkl B_ij B_kl K[(h_j,p_k)][(h_l,p_i)]
// (K = the walker's same-spin Gram matrix and Y its linear coefficients),
// evaluated through the antisymmetrized pair table (below).
//
// pair_cross_term: opposite-spin term of determinant I = (a, b) with levels
// (ka, KB) of walker w (pair_cross_value: X_ab alone):
//   c_I r_a r_b X_ab,  X_ab = sum_ij Ba_ij sum_kl Bb_kl K^{ab}[(ha_j,pa_i)][(hb_l,pb_k)]
// (K^{ab} in shared memory).
#pragma once

#include <type_traits>

#include "common.cuh"

template <typename T>
using cplx_t = typename std::conditional<std::is_same<T, float>::value, float2, double2>::type;

// The K x K inverse minor of one string (row-major, at a b_stride(K) offset)
// into registers; in FP32 two entries per 16-byte load.
template <int K, typename T>
__device__ __forceinline__ void load_minor(const cplx_t<T>* __restrict__ B, cplx_t<T> (&b)[K][K])
{
    if constexpr (std::is_same<T, float>::value) {
        const float4* B4 = reinterpret_cast<const float4*>(B);
#pragma unroll
        for (int v = 0; v < (K * K + 1) / 2; ++v) {
            const float4 q = B4[v];
            b[(2 * v) / K][(2 * v) % K] = make_float2(q.x, q.y);
            if (2 * v + 1 < K * K) b[(2 * v + 1) / K][(2 * v + 1) % K] = make_float2(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i)
#pragma unroll
            for (int j = 0; j < K; ++j) b[i][j] = B[i * K + j];
    }
}

// Index of the pair (a, b), a < b < n, among the n (n - 1) / 2 pairs in
// lexicographic order.
__host__ __device__ __forceinline__ int pair_index(int a, int b, int n) { return a * n - a * (a + 1) / 2 + (b - a - 1); }

// e_s of string s = bucket[KL] + sl (unweighted); string_energy_term below
// multiplies it by r_s w_s. K is symmetric (a same-spin Gram matrix), so
//   A[h,h';p,p'] = K[(h,p)][(h',p')] - K[(h,p')][(h',p)]
// is antisymmetric in (h, h') and in (p, p'), and the four orderings of two
// index pairs collapse:
//   (Qc - Qx) / 2 = sum_{i<k} sum_{j<l} (b_ij b_kl - b_il b_kj) A[h_j,h_l;p_i,p_k]
// (the holes and particles of a string are ascending), C(k,2)^2 terms
// instead of 2 k^4 gathers. ATAB: kt is A as a table [C(nh,2)][C(np,2)]
// (pair_index order, computed in precision T); otherwise kt is K and each
// difference is formed where it is used, in the same precision, so both
// give the same value.
template <int KL, typename T, bool ATAB = false>
__device__ __forceinline__ double2 string_energy_value(const SpinTables& tb, int w, int sl, int ns,
                                                       const void* __restrict__ Bin, const cplx_t<T>* kt,
                                                       const cplx_t<T>* ys)
{
    using T2 = cplx_t<T>;
    const int X = tb.nh * tb.np, np = tb.np, nh = tb.nh, npp = np * (np - 1) / 2;
    const int s = tb.bucket[KL] + sl;
    const uint4 rec = tb.str_hp[s];
    int hh[KL], pp[KL];   // hole and particle indices, ascending
#pragma unroll
    for (int i = 0; i < KL; ++i) { hh[i] = rec_h(rec, i); pp[i] = rec_p(rec, i); }
    const T2* B = reinterpret_cast<const T2*>(Bin) + (size_t)tb.b_off[KL] + ((size_t)w * ns + sl) * b_stride(KL);
    constexpr bool REG = KL <= 4;   // the inverse minor in registers (levels 5, 6: from memory)
    T2 b[REG ? KL : 1][REG ? KL : 1];
    if constexpr (REG) load_minor<KL, T>(B, b);
    auto bij = [&](int i, int j) -> T2 {
        if constexpr (REG) return b[i][j];
        else return B[i * KL + j];
    };
    T lr = 0, li = 0;      // linear part sum_ij b_ij Y[(h_j, p_i)]
#pragma unroll
    for (int i = 0; i < KL; ++i)
#pragma unroll
        for (int j = 0; j < KL; ++j) {
            const T2 bv = bij(i, j), y = ys[hh[j] * np + pp[i]];
            lr += bv.x * y.x - bv.y * y.y;
            li += bv.x * y.y + bv.y * y.x;
        }
    T qr = 0, qi = 0;      // (Qc - Qx) / 2
#pragma unroll
    for (int i = 0; i < KL; ++i)
#pragma unroll
        for (int k = i + 1; k < KL; ++k) {
            const int pik = pair_index(pp[i], pp[k], np);
#pragma unroll
            for (int j = 0; j < KL; ++j)
#pragma unroll
                for (int l = j + 1; l < KL; ++l) {
                    T2 a;
                    if constexpr (ATAB) {
                        a = kt[(size_t)pair_index(hh[j], hh[l], nh) * npp + pik];
                    } else {
                        const T2 kc = kt[(size_t)(hh[j] * np + pp[i]) * X + hh[l] * np + pp[k]];
                        const T2 kx = kt[(size_t)(hh[j] * np + pp[k]) * X + hh[l] * np + pp[i]];
                        a = T2{kc.x - kx.x, kc.y - kx.y};
                    }
                    const T2 b1 = bij(i, j), b2 = bij(k, l), b3 = bij(i, l), b4 = bij(k, j);
                    const T mr = (b1.x * b2.x - b1.y * b2.y) - (b3.x * b4.x - b3.y * b4.y);
                    const T mi = (b1.x * b2.y + b1.y * b2.x) - (b3.x * b4.y + b3.y * b4.x);
                    qr += mr * a.x - mi * a.y;
                    qi += mr * a.y + mi * a.x;
                }
        }
    return cz((double)lr + (double)qr, (double)li + (double)qi);
}

template <int KL, typename T, bool ATAB = false>
__device__ __forceinline__ double2 string_energy_term(const SpinTables& tb, int w, int sl, int ns,
                                                      const void* __restrict__ Bin, const cplx_t<T>* kt,
                                                      const cplx_t<T>* ys, const double2* __restrict__ wts)
{
    const double2 e_s = string_energy_value<KL, T, ATAB>(tb, w, sl, ns, Bin, kt, ys);
    return cmul(wts[(size_t)w * tb.n_str + tb.bucket[KL] + sl], e_s);   // wts holds r_s w_s
}

// The determinant's weight c_I r_a r_b and its product with X_ab are formed
// in the working precision T (the ratios and coefficients come in T: the
// FP64 arrays in FP64 mode, their FP32 copies in mixed mode).
template <typename T>
__device__ __forceinline__ cplx_t<T> pair_weight_times(const PairTables& pt, int I, cplx_t<T> ra, cplx_t<T> rb,
                                                       T xr, T xi)
{
    using T2 = cplx_t<T>;
    const T c = std::is_same<T, float>::value ? (T)pt.cf[I] : (T)pt.c[I];
    const T2 r = T2{ra.x * rb.x - ra.y * rb.y, ra.x * rb.y + ra.y * rb.x};
    const T2 rr = T2{r.x * c, r.y * c};
    return T2{rr.x * xr - rr.y * xi, rr.x * xi + rr.y * xr};
}

// X_ab of alpha string a (level ka) and beta string b (level KB), unweighted.
template <int KB, typename T>
__device__ __forceinline__ cplx_t<T> pair_cross_value(const SpinTables& ta, const SpinTables& tbb, int ka, int a,
                                                      int b, int w, const void* __restrict__ Ba_in,
                                                      const void* __restrict__ Bb_in, const cplx_t<T>* ks)
{
    using T2 = cplx_t<T>;
    const int Xb = tbb.nh * tbb.np;
    const int nsa = ta.bucket[ka + 1] - ta.bucket[ka], sa = a - ta.bucket[ka];
    const int nsb = tbb.bucket[KB + 1] - tbb.bucket[KB], sb = b - tbb.bucket[KB];
    int xb[KB][KB];
    const uint4 rb_rec = tbb.str_hp[b];
#pragma unroll
    for (int k = 0; k < KB; ++k)
#pragma unroll
        for (int l = 0; l < KB; ++l) xb[k][l] = rec_h(rb_rec, l) * tbb.np + rec_p(rb_rec, k);
    const T2* Ba = reinterpret_cast<const T2*>(Ba_in) + (size_t)ta.b_off[ka] + ((size_t)w * nsa + sa) * b_stride(ka);
    const T2* Bb = reinterpret_cast<const T2*>(Bb_in) + (size_t)tbb.b_off[KB] + ((size_t)w * nsb + sb) * b_stride(KB);
    T2 bb[KB][KB];
    load_minor<KB, T>(Bb, bb);
    const uint4 ra_rec = ta.str_hp[a];
    T xr = 0, xim = 0;
#pragma unroll 1
    for (int i = 0; i < ka; ++i)
#pragma unroll 1
        for (int j = 0; j < ka; ++j) {
            const T2 ba = Ba[i * ka + j];
            const T2* krow = ks + (size_t)(rec_h(ra_rec, j) * ta.np + rec_p(ra_rec, i)) * Xb;
            T zr = 0, zi = 0;
#pragma unroll
            for (int k = 0; k < KB; ++k)
#pragma unroll
                for (int l = 0; l < KB; ++l) {
                    const T2 kv = krow[xb[k][l]];
                    zr += bb[k][l].x * kv.x - bb[k][l].y * kv.y;
                    zi += bb[k][l].x * kv.y + bb[k][l].y * kv.x;
                }
            xr += ba.x * zr - ba.y * zi;
            xim += ba.x * zi + ba.y * zr;
        }
    return T2{xr, xim};
}

template <int KB, typename T>
__device__ __forceinline__ cplx_t<T> pair_cross_term(const SpinTables& ta, const SpinTables& tbb, const PairTables& pt,
                                                     int ka, int I, int w, const void* __restrict__ Ba_in,
                                                     const void* __restrict__ Bb_in, const cplx_t<T>* ks,
                                                     const cplx_t<T>* __restrict__ ra, const cplx_t<T>* __restrict__ rb)
{
    const int a = pt.a[I], b = pt.b[I];
    const cplx_t<T> x = pair_cross_value<KB, T>(ta, tbb, ka, a, b, w, Ba_in, Bb_in, ks);
    return pair_weight_times<T>(pt, I, ra[(size_t)w * ta.n_str + a], rb[(size_t)w * tbb.n_str + b], x.x, x.y);
}

// The opposite-spin term with both levels known at compile time: indices and
// both inverse minors in registers, the ka^2 kb^2 gathers from shared memory
// fully unrolled (same value as pair_cross_term).
template <int KA, int KB, typename T>
__device__ __forceinline__ cplx_t<T> pair_cross_term2(const SpinTables& ta, const SpinTables& tbb, const PairTables& pt,
                                                      int I, int w, const void* __restrict__ Ba_in,
                                                      const void* __restrict__ Bb_in, const cplx_t<T>* ks,
                                                      const cplx_t<T>* __restrict__ ra, const cplx_t<T>* __restrict__ rb)
{
    using T2 = cplx_t<T>;
    const int Xb = tbb.nh * tbb.np;
    const int a = pt.a[I], b = pt.b[I];
    const int nsa = ta.bucket[KA + 1] - ta.bucket[KA], sa = a - ta.bucket[KA];
    const int nsb = tbb.bucket[KB + 1] - tbb.bucket[KB], sb = b - tbb.bucket[KB];
    int ha[KA], pa[KA], xb[KB][KB];
    const uint4 ra_rec = ta.str_hp[a], rb_rec = tbb.str_hp[b];
#pragma unroll
    for (int i = 0; i < KA; ++i) {
        ha[i] = rec_h(ra_rec, i) * ta.np;
        pa[i] = rec_p(ra_rec, i);
    }
    {
        int hb[KB], pb[KB];
#pragma unroll
        for (int k = 0; k < KB; ++k) {
            hb[k] = rec_h(rb_rec, k) * tbb.np;
            pb[k] = rec_p(rb_rec, k);
        }
#pragma unroll
        for (int k = 0; k < KB; ++k)
#pragma unroll
            for (int l = 0; l < KB; ++l) xb[k][l] = hb[l] + pb[k];
    }
    const T2* Ba = reinterpret_cast<const T2*>(Ba_in) + (size_t)ta.b_off[KA] + ((size_t)w * nsa + sa) * b_stride(KA);
    const T2* Bb = reinterpret_cast<const T2*>(Bb_in) + (size_t)tbb.b_off[KB] + ((size_t)w * nsb + sb) * b_stride(KB);
    T2 ba[KA][KA], bb[KB][KB];
    load_minor<KA, T>(Ba, ba);
    load_minor<KB, T>(Bb, bb);
    const cplx_t<T> rav = ra[(size_t)w * ta.n_str + a], rbv = rb[(size_t)w * tbb.n_str + b];
    T xr = 0, xim = 0;
#pragma unroll
    for (int i = 0; i < KA; ++i)
#pragma unroll
        for (int j = 0; j < KA; ++j) {
            const T2* krow = ks + (size_t)(ha[j] + pa[i]) * Xb;
            T zr = 0, zi = 0;
#pragma unroll
            for (int k = 0; k < KB; ++k)
#pragma unroll
                for (int l = 0; l < KB; ++l) {
                    const T2 kv = krow[xb[k][l]];
                    zr += bb[k][l].x * kv.x - bb[k][l].y * kv.y;
                    zi += bb[k][l].x * kv.y + bb[k][l].y * kv.x;
                }
            xr += ba[i][j].x * zr - ba[i][j].y * zi;
            xim += ba[i][j].x * zi + ba[i][j].y * zr;
        }
    return pair_weight_times<T>(pt, I, rav, rbv, xr, xim);
}
