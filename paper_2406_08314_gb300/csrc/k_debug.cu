// Per-determinant local energies E_I for sampled (walker, determinant) pairs,
// from the same per-walker quantities and per-determinant device functions
// as the energy kernels (the localisation output of the energy path): with
// the reference energy E_0 of the walker (the k_final assembly),
//   E_I = E_0 + e_a + e_b + X_ab
// (Sec. II A, the generalized Wick theorem applied to the rank-k update of
// the reference Green's function; e_s the same-spin string terms, X_ab the
// opposite-spin term; a level-0 string contributes nothing).
#include "common.cuh"
#include "det_terms.cuh"
#include "kernels.h"

namespace {

template <typename T>
__device__ double2 string_value(const SpinTables& t, int k, int s, int w, const void* B, const void* K,
                                const void* Y)
{
    using T2 = cplx_t<T>;
    const int X = t.nh * t.np;
    const T2* ks = reinterpret_cast<const T2*>(K) + (size_t)w * X * X;
    const T2* ys = reinterpret_cast<const T2*>(Y) + (size_t)w * X;
    const int ns = t.bucket[k + 1] - t.bucket[k], sl = s - t.bucket[k];
    switch (k) {
    case 1: return string_energy_value<1, T>(t, w, sl, ns, B, ks, ys);
    case 2: return string_energy_value<2, T>(t, w, sl, ns, B, ks, ys);
    case 3: return string_energy_value<3, T>(t, w, sl, ns, B, ks, ys);
    case 4: return string_energy_value<4, T>(t, w, sl, ns, B, ks, ys);
    case 5: return string_energy_value<5, T>(t, w, sl, ns, B, ks, ys);
    default: return string_energy_value<6, T>(t, w, sl, ns, B, ks, ys);
    }
}

template <typename T>
__device__ double2 cross_value(const SpinTables& ta, const SpinTables& tb, int ka, int kb, int a, int b, int w,
                               const void* Ba, const void* Bb, const void* Kab)
{
    using T2 = cplx_t<T>;
    const T2* ks = reinterpret_cast<const T2*>(Kab) + (size_t)w * (ta.nh * ta.np) * (tb.nh * tb.np);
    T2 x;
    switch (kb) {
    case 1: x = pair_cross_value<1, T>(ta, tb, ka, a, b, w, Ba, Bb, ks); break;
    case 2: x = pair_cross_value<2, T>(ta, tb, ka, a, b, w, Ba, Bb, ks); break;
    case 3: x = pair_cross_value<3, T>(ta, tb, ka, a, b, w, Ba, Bb, ks); break;
    case 4: x = pair_cross_value<4, T>(ta, tb, ka, a, b, w, Ba, Bb, ks); break;
    case 5: x = pair_cross_value<5, T>(ta, tb, ka, a, b, w, Ba, Bb, ks); break;
    default: x = pair_cross_value<6, T>(ta, tb, ka, a, b, w, Ba, Bb, ks); break;
    }
    return cz((double)x.x, (double)x.y);
}

template <typename T>
__global__ void __launch_bounds__(128)
k_det_energy(int n, const DetRec* __restrict__ recs, int w0, int nw, SpinTables ta, SpinTables tb, const void* Ba,
             const void* Bb, const void* Kaa, const void* Kbb, const void* Kab, const void* Ya, const void* Yb,
             const double2* __restrict__ scal, const double2* __restrict__ e1a, const double2* __restrict__ e1b,
             double e0, double2* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DetRec r = recs[i];
    if (r.w < w0 || r.w >= w0 + nw) return;
    const int w = r.w - w0;
    const double2* sc = scal + (size_t)w * 8;
    double2 E = cadd(cz(e0, 0), cadd(e1a[w], e1b[w]));
    E = cadd(E, cscale(sc[2], 0.5));
    E = csub(E, cscale(cadd(sc[0], sc[1]), 0.5));
    if (r.ka > 0) E = cadd(E, string_value<T>(ta, r.ka, r.a, w, Ba, Kaa, Ya));
    if (r.kb > 0) E = cadd(E, string_value<T>(tb, r.kb, r.b, w, Bb, Kbb, Yb));
    if (r.ka > 0 && r.kb > 0) E = cadd(E, cross_value<T>(ta, tb, r.ka, r.kb, r.a, r.b, w, Ba, Bb, Kab));
    out[i] = E;
}

}  // namespace

void launch_det_energy(int n, const DetRec* recs, int w0, int nw, const SpinTables& ta, const SpinTables& tb,
                       const void* Ba, const void* Bb, const void* Kaa, const void* Kbb, const void* Kab,
                       const void* Ya, const void* Yb, const double2* scal, const double2* e1a, const double2* e1b,
                       double e0, bool fp32, double2* out, cudaStream_t st)
{
    if (n <= 0) return;
    const int grid = (n + 127) / 128;
    if (fp32)
        k_det_energy<float><<<grid, 128, 0, st>>>(n, recs, w0, nw, ta, tb, Ba, Bb, Kaa, Kbb, Kab, Ya, Yb, scal, e1a,
                                                  e1b, e0, out);
    else
        k_det_energy<double><<<grid, 128, 0, st>>>(n, recs, w0, nw, ta, tb, Ba, Bb, Kaa, Kbb, Kab, Ya, Yb, scal,
                                                   e1a, e1b, e0, out);
    msd_note_launch();
}
