// Persistent batched kernel for the per-determinant energy terms of many
// independent systems (uneven orbital counts, determinant counts and
// excitation levels) in one launch. Work items are (system, walker, kind,
// spin or opposite-spin level pair, block of strings or determinants); a
// resident grid of CTAs takes items from a global counter (atomicAdd, no
// waiting), so small and large systems share the machine. Each item computes
// exactly what one block of k_string_energy / k_pair_cross computes and
// writes the same partial-sum slot, so batched and per-system results agree.
#include "common.cuh"
#include "det_terms.cuh"
#include "kernels.h"

template <typename T>
__device__ double2 batch_se(const BatchSys& S, const BatchItem& it, int t, const cplx_t<T>* ks,
                            const cplx_t<T>* ys)
{
    const SpinTables& tb = S.t[it.spin];
    const int k = it.ka;
    const int ns = tb.bucket[k + 1] - tb.bucket[k];
    double2 acc = cz(0, 0);
    for (int q = 0; q < SE_PER_THREAD; ++q) {
        const int sl = it.blk * (SE_THREADS * SE_PER_THREAD) + q * SE_THREADS + t;
        if (sl >= ns) break;
        double2 v;
        switch (k) {
        case 1: v = string_energy_term<1, T>(tb, it.w, sl, ns, S.B[it.spin], ks, ys, S.wts[it.spin]); break;
        case 2: v = string_energy_term<2, T>(tb, it.w, sl, ns, S.B[it.spin], ks, ys, S.wts[it.spin]); break;
        case 3: v = string_energy_term<3, T>(tb, it.w, sl, ns, S.B[it.spin], ks, ys, S.wts[it.spin]); break;
        case 4: v = string_energy_term<4, T>(tb, it.w, sl, ns, S.B[it.spin], ks, ys, S.wts[it.spin]); break;
        case 5: v = string_energy_term<5, T>(tb, it.w, sl, ns, S.B[it.spin], ks, ys, S.wts[it.spin]); break;
        default: v = string_energy_term<6, T>(tb, it.w, sl, ns, S.B[it.spin], ks, ys, S.wts[it.spin]); break;
        }
        acc = cadd(acc, v);
    }
    return acc;
}

template <typename T>
__device__ double2 batch_pc(const BatchSys& S, const BatchItem& it, int t, const cplx_t<T>* ks)
{
    using T2 = cplx_t<T>;
    const int idx = it.ka * (MSD_KMAX + 1) + it.kb;
    const int lo = S.pt.bucket[idx], n = S.pt.bucket[idx + 1] - lo;
    // the ratios in the working precision, as in the per-system kernels
    const T2* ra = std::is_same<T, float>::value ? reinterpret_cast<const T2*>(S.rf[0])
                                                 : reinterpret_cast<const T2*>(S.r[0]);
    const T2* rb = std::is_same<T, float>::value ? reinterpret_cast<const T2*>(S.rf[1])
                                                 : reinterpret_cast<const T2*>(S.r[1]);
    T2 acc = T2{0, 0};
    for (int q = 0; q < PC_PER_THREAD; ++q) {
        const int i0 = it.blk * (PC_THREADS * PC_PER_THREAD) + q * PC_THREADS + t;
        if (i0 >= n) break;
        const int I = lo + i0;
        T2 v;
        switch (it.kb) {
        case 1: v = pair_cross_term<1, T>(S.t[0], S.t[1], S.pt, it.ka, I, it.w, S.B[0], S.B[1], ks, ra, rb); break;
        case 2: v = pair_cross_term<2, T>(S.t[0], S.t[1], S.pt, it.ka, I, it.w, S.B[0], S.B[1], ks, ra, rb); break;
        case 3: v = pair_cross_term<3, T>(S.t[0], S.t[1], S.pt, it.ka, I, it.w, S.B[0], S.B[1], ks, ra, rb); break;
        case 4: v = pair_cross_term<4, T>(S.t[0], S.t[1], S.pt, it.ka, I, it.w, S.B[0], S.B[1], ks, ra, rb); break;
        case 5: v = pair_cross_term<5, T>(S.t[0], S.t[1], S.pt, it.ka, I, it.w, S.B[0], S.B[1], ks, ra, rb); break;
        default: v = pair_cross_term<6, T>(S.t[0], S.t[1], S.pt, it.ka, I, it.w, S.B[0], S.B[1], ks, ra, rb); break;
        }
        acc.x += v.x;
        acc.y += v.y;
    }
    return cz((double)acc.x, (double)acc.y);
}

template <typename T>
__global__ void __launch_bounds__(256, 2)
k_det_batched(const BatchSys* __restrict__ systems, const BatchItem* __restrict__ items, int n_items,
              unsigned* __restrict__ counter)
{
    static_assert(SE_THREADS == 256 && PC_THREADS == 256, "one block shape for both item kinds");
    using T2 = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    T2* ks = reinterpret_cast<T2*>(smraw);
    __shared__ BatchItem it;
    __shared__ int cur;
    __shared__ double2 red[256];
    __shared__ __align__(16) unsigned char sys_raw[sizeof(BatchSys)];
    const BatchSys& S = *reinterpret_cast<const BatchSys*>(sys_raw);
    const int t = threadIdx.x;
    int loaded = -1;
    while (true) {
        if (t == 0) {
            cur = (int)atomicAdd(counter, 1u);
            if (cur < n_items) it = items[cur];
        }
        __syncthreads();
        if (cur >= n_items) break;
        if (it.sys != loaded) {   // uniform: every thread sees the same item
            const int* src = reinterpret_cast<const int*>(systems + it.sys);
            int* dst = reinterpret_cast<int*>(sys_raw);
            for (int e = t; e < (int)(sizeof(BatchSys) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
            loaded = it.sys;
            __syncthreads();
        }
        const int X0 = S.t[0].nh * S.t[0].np, X1 = S.t[1].nh * S.t[1].np;
        T2* ys = nullptr;
        if (it.kind == 0) {
            const int X = it.spin ? X1 : X0;
            const T2* K = reinterpret_cast<const T2*>(S.K[it.spin]) + (size_t)it.w * X * X;
            const T2* Y = reinterpret_cast<const T2*>(S.Y[it.spin]) + (size_t)it.w * X;
            ys = ks + X * X;
            for (int e = t; e < X * X; e += blockDim.x) ks[e] = K[e];
            for (int e = t; e < X; e += blockDim.x) ys[e] = Y[e];
        } else {
            const T2* K = reinterpret_cast<const T2*>(S.K[2]) + (size_t)it.w * X0 * X1;
            for (int e = t; e < X0 * X1; e += blockDim.x) ks[e] = K[e];
        }
        __syncthreads();
        red[t] = it.kind == 0 ? batch_se<T>(S, it, t, ks, ys) : batch_pc<T>(S, it, t, ks);
        __syncthreads();
        for (int o = 128; o; o >>= 1) {
            if (t < o) red[t] = cadd(red[t], red[t + o]);
            __syncthreads();
        }
        if (t == 0) S.part[(size_t)it.w * S.nslot + it.slot] = red[0];
        __syncthreads();
    }
}

int launch_det_batched(const BatchSys* systems, const BatchItem* items, int n_items, unsigned* counter,
                       size_t smem, bool fp32, int grid, cudaStream_t st)
{
    if (n_items <= 0) return 0;
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned), st) != cudaSuccess) return -1;
    if (fp32) {
        cudaFuncSetAttribute(k_det_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_det_batched<float><<<grid, 256, smem, st>>>(systems, items, n_items, counter);
    } else {
        cudaFuncSetAttribute(k_det_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_det_batched<double><<<grid, 256, smem, st>>>(systems, items, n_items, counter);
    }
    msd_note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
