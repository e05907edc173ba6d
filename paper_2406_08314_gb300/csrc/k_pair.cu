// Opposite-spin cross term (fill_os) per determinant with both excitation
// levels (ka, kb) known at compile time, for ka + kb <= 8: the indices and
// both inverse minors sit in registers and the ka^2 kb^2 gathers from the
// shared Gram matrix K^{ab} are fully unrolled, so a determinant's global
// loads are all issued before its first gather. Same value, partial-sum
// slots and block shape as k_pair_cross in k_energy.cu, which serves the
// other level pairs.
#include <type_traits>

#include "common.cuh"
#include "det_terms.cuh"
#include "kernels.h"

template <int KA, int KB, typename T>
__global__ void __launch_bounds__(PC_THREADS)
k_pair_cross2(SpinTables ta, SpinTables tbb, PairTables pt, int lo, int n, const void* __restrict__ ra_in,
              const void* __restrict__ rb_in, const void* __restrict__ Ba_in, const void* __restrict__ Bb_in,
              const void* __restrict__ Kin, double2* __restrict__ part, int nslot, int slot0)
{
    using T2 = cplx_t<T>;
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
    for (int it = 0; it < PC_PER_THREAD; ++it) {
        const int i0 = blockIdx.x * (PC_THREADS * PC_PER_THREAD) + it * PC_THREADS + t;
        if (i0 >= n) break;
        const T2 v = pair_cross_term2<KA, KB, T>(ta, tbb, pt, lo + i0, w, Ba_in, Bb_in, ks, ra, rb);
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

template <int KA, int KB>
static bool go(bool fp32, dim3 grid, size_t smem, const SpinTables& ta, const SpinTables& tb, const PairTables& pt,
               int lo, int n, const void* ra, const void* rb, const void* Ba, const void* Bb, const void* K,
               double2* part, int nslot, int slot, cudaStream_t st)
{
    if (fp32) {
        cudaFuncSetAttribute(k_pair_cross2<KA, KB, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pair_cross2<KA, KB, float><<<grid, PC_THREADS, smem, st>>>(ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part,
                                                                     nslot, slot);
    } else {
        cudaFuncSetAttribute(k_pair_cross2<KA, KB, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pair_cross2<KA, KB, double><<<grid, PC_THREADS, smem, st>>>(ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part,
                                                                      nslot, slot);
    }
    msd_note_launch();
    return true;
}

bool launch_pair_cross2(int ka, int kb, bool fp32, dim3 grid, size_t smem, const SpinTables& ta, const SpinTables& tb,
                        const PairTables& pt, int lo, int n, const void* ra, const void* rb, const void* Ba,
                        const void* Bb, const void* K, double2* part, int nslot, int slot, cudaStream_t st)
{
    switch (ka * 8 + kb) {
        case 9: return go<1, 1>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 10: return go<1, 2>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 11: return go<1, 3>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 12: return go<1, 4>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 13: return go<1, 5>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 14: return go<1, 6>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 17: return go<2, 1>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 18: return go<2, 2>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 19: return go<2, 3>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 20: return go<2, 4>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 21: return go<2, 5>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 22: return go<2, 6>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 25: return go<3, 1>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 26: return go<3, 2>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 27: return go<3, 3>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 28: return go<3, 4>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 29: return go<3, 5>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 33: return go<4, 1>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 34: return go<4, 2>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 35: return go<4, 3>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 36: return go<4, 4>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 41: return go<5, 1>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 42: return go<5, 2>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 43: return go<5, 3>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 49: return go<6, 1>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        case 50: return go<6, 2>(fp32, grid, smem, ta, tb, pt, lo, n, ra, rb, Ba, Bb, K, part, nslot, slot, st);
        default: return false;
    }
}
