// Opposite-spin exchange term of the local energy (the alpha-beta part of the
// two-body Wick contraction, Sec. III) in mixed precision, formed per beta
// string instead of per determinant:
//   sum_I c_I r_a r_b X_ab,
//   X_ab = sum_ij Ba[i][j] sum_kl Bb[k][l] K^ab[(h^a_j, p^a_i)][(h^b_l, p^b_k)]
//        = sum_ij Ba[i][j] Y_b[(h^a_j, p^a_i)],
//   Y_b[x] = sum_kl Bb[k][l] K^ab[x][(h^b_l, p^b_k)].
// Y_b is formed once per beta string (k_b^2 rows of K^ab), so a determinant
// costs k_a^2 gathers instead of k_a^2 k_b^2.
//
// One block per (walker, slice of beta-string chunks). K^ab is staged
// transposed in shared memory once per block (KT[y][x], x contiguous). Per
// chunk of PY_CB excited beta strings:
//   phase A: a warp per beta string, its lanes over x (XQ values each), adds
//            Bb[e] * KT[y_e][x] over the string's k_b^2 entries -> Ys[b][x];
//   phase B: groups of PY_G lanes walk the chunk's determinants (the beta
//            spin's determinant list, ordered by beta string), one
//            determinant per group at a time; lane l takes the entries
//            e = l, l + PY_G, ... of the alpha minor (the group's loads of
//            Ba are contiguous), gathers Ys[b][x_e] and adds
//            c_I r_a r_b Ba[e] Ys[b][x_e] (FP32) to its own sum: the total
//            is linear in the (determinant, entry) terms, so no
//            per-determinant reduction is needed;
// and the block's FP32 partial sums are combined in FP64 in a fixed order
// into the chunk's partial-sum slot. Determinants whose alpha string is the
// reference string contribute nothing and are skipped. The ratios come as
// their FP32 copies (rf, written by the string-minor kernel).
#include "common.cuh"
#include "kernels.h"

#define PY_CB 32          // beta strings per chunk
#define PY_THREADS 512
#define PY_WARPS (PY_THREADS / 32)
#define PY_SPW (PY_CB / PY_WARPS)   // beta strings per warp in phase A
#define PY_EMAX (MSD_KMAX * MSD_KMAX)
#define PY_G 4            // lanes per determinant in phase B
#define PY_NG (PY_THREADS / PY_G)   // lane groups
#define PY_DPG (PY_THREADS / PY_NG) // staged determinants per group and tile

static __host__ __device__ __forceinline__ int py_xq(int Xa) { return (Xa + 31) / 32; }

// per staged determinant of phase B
struct __align__(16) PyDet {
    long long aoff;   // offset of its alpha inverse minor in Ba
    int xoff;         // offset of its alpha entries in ta.kx
    int kk;           // k_a^2 (0: nothing to add)
    int yoff;         // offset of its beta string's row in Ys
    float wr, wi;     // c_I r_a r_b
    int pad;
};

// bytes of the staging area (phase A's entries or phase B's tile)
#define PY_STAGE_BYTES (sizeof(float4) * PY_CB * PY_EMAX > sizeof(PyDet) * PY_THREADS \
                            ? sizeof(float4) * PY_CB * PY_EMAX : sizeof(PyDet) * PY_THREADS)

static size_t py_smem(int Xa, int Xb)
{
    const int XPP = 32 * py_xq(Xa) + 1;
    return PY_STAGE_BYTES + sizeof(float2) * ((size_t)Xb * XPP + (size_t)PY_CB * XPP);
}

template <int XQ>
__global__ void __launch_bounds__(PY_THREADS)
k_pair_y(SpinTables ta, SpinTables tbb, const float2* __restrict__ rfa, const float2* __restrict__ rfb,
         const float2* __restrict__ Ba, const float2* __restrict__ Bb, const float2* __restrict__ Kab,
         double2* __restrict__ part, int nslot, int slot0, int n_chunks)
{
    constexpr int XPP = 32 * XQ + 1;   // row pitch (float2) of KT and Ys
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Xa = ta.nh * ta.np, Xb = tbb.nh * tbb.np;
    // staging area: phase A's (Bb entry, KT row offset) per string and entry,
    // then phase B's determinant tile
    float4* stg = reinterpret_cast<float4*>(smraw);                  // [PY_CB][PY_EMAX]
    PyDet* dst = reinterpret_cast<PyDet*>(smraw);                    // [PY_THREADS]
    float2* KT = reinterpret_cast<float2*>(smraw + PY_STAGE_BYTES);   // [Xb][XPP]
    float2* Ys = KT + (size_t)Xb * XPP;                                  // [PY_CB][XPP]
    __shared__ int offs[PY_CB + 1];
    __shared__ float2 rbs[PY_CB];
    __shared__ double2 red[PY_WARPS];
    const int w = blockIdx.y, t = threadIdx.x, lane = t & 31, warp = t >> 5;

    // KT[y][x] = K^ab[x][y]; columns x >= Xa are zero
    const float2* Kw = Kab + (size_t)w * Xa * Xb;
    for (int e = t; e < Xa * Xb; e += PY_THREADS) {
        const int x = e / Xb, y = e - x * Xb;
        KT[y * XPP + x] = Kw[e];
    }
    for (int e = t; e < Xb * (XPP - Xa); e += PY_THREADS) {
        const int y = e / (XPP - Xa), x = Xa + (e - y * (XPP - Xa));
        KT[y * XPP + x] = make_float2(0.f, 0.f);
    }
    const int s_lo = tbb.bucket[1];
    for (int ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const int b0 = s_lo + ch * PY_CB, nb = min(PY_CB, tbb.n_str - b0);
        __syncthreads();   // KT ready / the previous chunk's staging, Ys, offs, rbs consumed
        if (t <= nb) offs[t] = tbb.csr_off[b0 + t];
        // phase A: the warp stages its strings' entries, then forms their Y rows
        int kks[PY_SPW];
#pragma unroll
        for (int u = 0; u < PY_SPW; ++u) {
            const int bl = warp + PY_WARPS * u, b = b0 + bl;
            kks[u] = 0;
            if (bl < nb) {
                int kb = 1;
                while (b >= tbb.bucket[kb + 1]) ++kb;
                const int nsb = tbb.bucket[kb + 1] - tbb.bucket[kb], sb = b - tbb.bucket[kb], kk = kb * kb;
                const float2* B = Bb + (size_t)tbb.b_off[kb] + ((size_t)w * nsb + sb) * b_stride(kb);
                const uint8_t* yx = tbb.kx + tbb.cmx_off[kb] + (size_t)sb * kk;
                for (int e = lane; e < kk; e += 32) {
                    const float2 v = B[e];
                    stg[bl * PY_EMAX + e] = make_float4(v.x, v.y, __int_as_float((int)yx[e] * XPP), 0.f);
                }
                if (lane == 0) rbs[bl] = rfb[(size_t)w * tbb.n_str + b];
                kks[u] = kk;
            }
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < PY_SPW; ++u) {
            const int bl = warp + PY_WARPS * u;
            if (bl >= nb) break;
            const float4* sg = stg + bl * PY_EMAX;
            float2 acc[XQ];
#pragma unroll
            for (int q = 0; q < XQ; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int e = 0; e < kks[u]; ++e) {
                const float4 sv = sg[e];
                const float2* kt = KT + __float_as_int(sv.z) + lane;
#pragma unroll
                for (int q = 0; q < XQ; ++q) {
                    const float2 kv = kt[32 * q];
                    acc[q].x = fmaf(sv.x, kv.x, fmaf(-sv.y, kv.y, acc[q].x));
                    acc[q].y = fmaf(sv.x, kv.y, fmaf(sv.y, kv.x, acc[q].y));
                }
            }
#pragma unroll
            for (int q = 0; q < XQ; ++q) Ys[bl * XPP + lane + 32 * q] = acc[q];
        }
        __syncthreads();   // Ys, offs, rbs complete; the staging area is free
        // phase B, in tiles of PY_THREADS determinants
        const int d0 = offs[0], d1 = offs[nb];
        const int grp = t / PY_G, l = t % PY_G;
        float vr_sum = 0.f, vi_sum = 0.f;
        for (int tile = d0; tile < d1; tile += PY_THREADS) {
            {   // stage: thread t takes determinant tile + t
                const int d = tile + t;
                PyDet q;
                q.aoff = 0; q.xoff = 0; q.kk = 0; q.yoff = 0; q.wr = 0.f; q.wi = 0.f; q.pad = 0;
                if (d < d1) {
                    const int a = tbb.csr_other[d];
                    if (a >= ta.bucket[1]) {
                        int lo = 0, hi = nb - 1;   // offs[bl] <= d < offs[bl + 1]
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (offs[mid] <= d) lo = mid; else hi = mid - 1;
                        }
                        int ka = 1;
                        while (a >= ta.bucket[ka + 1]) ++ka;
                        const float2 wab = fmul(rfa[(size_t)w * ta.n_str + a], rbs[lo]);
                        const float c = tbb.csr_cf[d];
                        const int nsa = ta.bucket[ka + 1] - ta.bucket[ka], sa = a - ta.bucket[ka];
                        q.kk = ka * ka;
                        q.aoff = ta.b_off[ka] + ((long long)w * nsa + sa) * b_stride(ka);
                        q.xoff = (int)ta.cmx_off[ka] + sa * q.kk;
                        q.yoff = lo * XPP;
                        q.wr = c * wab.x; q.wi = c * wab.y;
                    }
                }
                dst[t] = q;
            }
            __syncthreads();
            // process: group grp takes the staged determinants grp + u PY_NG
            // (u < PY_DPG) together, so their loads are in flight at once
            const int n_here = min(PY_THREADS, d1 - tile);
            PyDet q[PY_DPG];
            int kmax = 0;
#pragma unroll
            for (int u = 0; u < PY_DPG; ++u) {
                const int j = grp + u * PY_NG;
                if (j < n_here) {
                    q[u] = dst[j];
                } else {
                    q[u].aoff = 0; q[u].xoff = 0; q[u].kk = 0; q[u].yoff = 0; q[u].wr = 0.f; q[u].wi = 0.f;
                }
                kmax = max(kmax, q[u].kk);
            }
            float xr[PY_DPG], xi[PY_DPG];
#pragma unroll
            for (int u = 0; u < PY_DPG; ++u) { xr[u] = 0.f; xi[u] = 0.f; }
            for (int e = l; e < kmax; e += PY_G) {
#pragma unroll
                for (int u = 0; u < PY_DPG; ++u)
                    if (e < q[u].kk) {
                        const float2 bv = Ba[q[u].aoff + e], yv = Ys[q[u].yoff + ta.kx[q[u].xoff + e]];
                        xr[u] = fmaf(bv.x, yv.x, fmaf(-bv.y, yv.y, xr[u]));
                        xi[u] = fmaf(bv.x, yv.y, fmaf(bv.y, yv.x, xi[u]));
                    }
            }
#pragma unroll
            for (int u = 0; u < PY_DPG; ++u) {
                vr_sum = fmaf(q[u].wr, xr[u], fmaf(-q[u].wi, xi[u], vr_sum));
                vi_sum = fmaf(q[u].wr, xi[u], fmaf(q[u].wi, xr[u], vi_sum));
            }
            __syncthreads();   // the tile is consumed
        }
        double sr = vr_sum, si = vi_sum;
        for (int o = 16; o; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if (lane == 0) red[warp] = cz(sr, si);
        __syncthreads();
        if (t == 0) {
            double2 s = red[0];
            for (int q = 1; q < PY_WARPS; ++q) s = cadd(s, red[q]);
            part[(size_t)w * nslot + slot0 + ch] = s;
        }
    }
}

bool pair_y_ok(const SpinTables& ta, const SpinTables& tb)
{
    const int Xa = ta.nh * ta.np, Xb = tb.nh * tb.np;
    return Xa > 0 && Xb > 0 && py_xq(Xa) <= 4 && py_smem(Xa, Xb) <= 227 * 1024;
}

int pair_y_slots(const SpinTables& tb)
{
    const int n = tb.n_str - tb.bucket[1];
    return n > 0 ? (n + PY_CB - 1) / PY_CB : 0;
}

template <int XQ>
static void launch_py(dim3 grid, size_t smem, const SpinTables& ta, const SpinTables& tb, const float2* ra,
                      const float2* rb, const void* Ba, const void* Bb, const void* Kab, double2* part, int nslot,
                      int slot0, int n_chunks, cudaStream_t st)
{
    cudaFuncSetAttribute(k_pair_y<XQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pair_y<XQ><<<grid, PY_THREADS, smem, st>>>(ta, tb, ra, rb, (const float2*)Ba, (const float2*)Bb,
                                                 (const float2*)Kab, part, nslot, slot0, n_chunks);
    msd_note_launch();
}

void launch_pair_y(const SpinTables& ta, const SpinTables& tb, int nw, const float2* ra, const float2* rb,
                   const void* Ba, const void* Bb, const void* Kab, double2* part, int nslot, int slot0,
                   cudaStream_t st)
{
    const int n_chunks = pair_y_slots(tb);
    if (n_chunks <= 0 || nw <= 0) return;
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // enough blocks for two waves of the SMs; each block reuses its staged
    // K^ab over several chunks
    const int per_w = std::min(n_chunks, std::max(4, (2 * n_sm + nw - 1) / nw));
    dim3 grid(per_w, nw);
    const int Xa = ta.nh * ta.np, Xb = tb.nh * tb.np;
    const size_t smem = py_smem(Xa, Xb);
    switch (py_xq(Xa)) {
        case 1: launch_py<1>(grid, smem, ta, tb, ra, rb, Ba, Bb, Kab, part, nslot, slot0, n_chunks, st); break;
        case 2: launch_py<2>(grid, smem, ta, tb, ra, rb, Ba, Bb, Kab, part, nslot, slot0, n_chunks, st); break;
        case 3: launch_py<3>(grid, smem, ta, tb, ra, rb, Ba, Bb, Kab, part, nslot, slot0, n_chunks, st); break;
        default: launch_py<4>(grid, smem, ta, tb, ra, rb, Ba, Bb, Kab, part, nslot, slot0, n_chunks, st); break;
    }
}
