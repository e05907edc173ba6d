// C-ABI entry points of libmsd (declared in include/msd.h): context, trial
// preprocessing, workspace management and the orchestration of the
// kernels for overlap, per-determinant ratios, force bias and local energy.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/msd.h"
#include "common.cuh"
#include "kernels.h"

static std::atomic<long long> g_launches{0};
void msd_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int msd_err_word_alloc(unsigned** out)
{
    *out = nullptr;
    unsigned w[MSD_ERR_WORDS] = {0, 0, 0, 0};
    const unsigned long long budget = MSD_WAIT_DEFAULT_NS;
    std::memcpy(&w[2], &budget, sizeof budget);
    if (cudaMalloc((void**)out, sizeof w) != cudaSuccess) { cudaGetLastError(); *out = nullptr; return -1; }
    if (cudaMemcpy(*out, w, sizeof w, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(*out);
        *out = nullptr;
        return -1;
    }
    return 0;
}

int msd_sm_count()
{
    static std::atomic<int> cache[256];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 1;
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

namespace {

std::string g_create_error;

struct SpinHost {
    int N = 0, nh = 0, np = 0, n_str = 0;
    std::vector<int> occ0, hole_pos, part_orb, hole_orb;
    std::vector<uint8_t> str_h, str_p;
    std::vector<int8_t> str_sign;
    std::vector<int> str_k;
    std::vector<int> csr_off, csr_other;
    std::vector<double> csr_c;
    int bucket[MSD_KMAX + 2] = {0};
    long long b_per_walker = 0;
    // device copies
    int *d_occ0 = nullptr, *d_hole_pos = nullptr, *d_part_orb = nullptr;
    uint8_t* d_str_hp = nullptr;   // [n_str][16] packed records (SpinTables::str_hp)
    int8_t* d_str_sign = nullptr;
    int *d_csr_off = nullptr, *d_csr_other = nullptr;
    double* d_csr_c = nullptr;
    double* d_Lh = nullptr;   // [n_chol][N + np][M]
    uint8_t* d_cmx = nullptr;
    uint8_t* d_kx = nullptr;
    float* d_csr_cf = nullptr;
    int* d_pos0 = nullptr;    // [M] position of an orbital in occ0, or -1
};

struct PairHost {
    int n_det = 0;
    std::vector<int> a, b, det_index;
    std::vector<double> c;
    int bucket[(MSD_KMAX + 1) * (MSD_KMAX + 1) + 1] = {0};
    int *d_a = nullptr, *d_b = nullptr, *d_det_index = nullptr;
    double* d_c = nullptr;
    float* d_cf = nullptr;   // FP32 copy of c
    // runs form of the opposite-spin term (see PairTables)
    int run_side[(MSD_KMAX + 1) * (MSD_KMAX + 1)] = {0};
    int run_off[(MSD_KMAX + 1) * (MSD_KMAX + 1) + 1] = {0};
    std::vector<int> runs;
    int* d_runs = nullptr;
};

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct msd_ctx {
    int device = 0, M = 0, n[2] = {0, 0}, prec = MSD_FP64;
    std::string err;
    bool have_ham = false, have_trial = false;
    int n_chol = 0;
    double e0 = 0;
    std::vector<double> h_h1, h_L;
    double* d_h1 = nullptr;
    double* d_Lcat = nullptr;   // [n_chol][Kd]
    long long Kd = 0;
    SpinHost sp[2];
    PairHost pairs;
    std::map<std::string, Buf> arena;
    size_t ws_limit = (size_t)16 << 30;
    int chunk = 0;
    unsigned* d_err = nullptr;
    unsigned* h_err = nullptr;
    bool sync = true;
    // timing
    bool timing = false;
    std::vector<std::string> knames;
    std::vector<long long> klaunch;
    std::vector<double> kms;
    struct Pending { int k; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
    int open_k = -1;
    cudaEvent_t open_ev = nullptr;
    // host inputs: the beta walkers are copied on their own stream while the
    // alpha spin's first kernels run (created on first use)
    cudaStream_t copy_st = nullptr;
    cudaEvent_t ev_in = nullptr, ev_b = nullptr;
    // mixed evaluation: the energy's remaining per-walker contractions run on
    // a side stream while the strings, weights and force bias run on the
    // caller's stream (msd_set_stream_overlap; created on first use)
    bool overlap = true;
    cudaStream_t side_st = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_rest = nullptr, ev_w = nullptr;
    TimerHook hook;
    // TF32 hi/lo splits of the half-rotated Cholesky vectors (mixed path)
    bool mixed_ready = false;
    int Kp = 0;                 // M padded to a multiple of 32
    long long Kdp = 0;          // Kd padded to a multiple of 32
    float *LhF_hi[2] = {nullptr, nullptr}, *LhF_lo[2] = {nullptr, nullptr};
    // fused path: the same rows with each vector's occ0 block padded to RB
    // columns (zero rows), and F0 padded to [RB][RB + np]
    float *LhP_hi[2] = {nullptr, nullptr}, *LhP_lo[2] = {nullptr, nullptr};
    float* d_F0P[2] = {nullptr, nullptr};
    float *Lv_hi = nullptr, *Lv_lo = nullptr;
    int Kvp[2] = {0, 0};        // virtual orbitals (not in occ0) padded to 32
    // fused path: contraction length Kv8 (Kv padded to 8), then two column
    // blocks of RB for the F0 slices; Kfp = Kv8 + 2 RB is the operands' pitch
    int Kv8[2] = {0, 0}, Kfp[2] = {0, 0};
    int* d_virt[2] = {nullptr, nullptr};
    double *d_c0[2] = {nullptr, nullptr}, *d_x0[2] = {nullptr, nullptr}, *d_c0sum = nullptr;
    float* d_F0T[2] = {nullptr, nullptr};   // [n_chol][N][N + np] = L_g[occ0_j][col]
    int tc_bn = 0;                // tensor-core output tile width (0 = by shape)
    int Kv[2] = {0, 0};           // virtual orbitals per spin
    bool fuse = true;             // fused energy contraction + epilogue when the shape allows
    bool tc_gram = false;         // Gram matrices on the tensor cores (msd_set_tensor_gram)
    int pair_form = -1;           // mixed mode, opposite-spin term: -1 auto, 0 per determinant, 1 per beta string
    bool pair_y_auto = false;     // the auto choice for the current trial (set_trial)
    bool fused_ok[2] = {false, false};
    // exact reference-determinant sums of the mixed energy (tc_ozaki.cu)
    bool exact_ref = true;        // requested (msd_set_exact_reference)
    bool oz_ready = false;        // constants built for the current Hamiltonian and trial
    bool oz_ok = false;           // the shapes allow it (set with oz_ready)
    bool oz_shared = false;       // spin 1 uses spin 0's constants (same reference orbitals)
    OzConst oz[2];
    double *d_JJ[2] = {nullptr, nullptr}, *d_KK[2] = {nullptr, nullptr};
    double* d_hJ = nullptr;       // [2][M][M] h_s + J, J = sum_g C_g L_g (C_g = sum_s tr(L_g D0_s D0_s^T))
    double oz_x0sum[2] = {0, 0}, oz_C2sum = 0;
    TcFepiPlan fplan[2];
    long long gen = 0;            // bumped whenever a device buffer may move
    // propagation (msd_propagate): transposed Cholesky vectors, sum_g L_g L_g
    // and exp(-dt h'/2) per spin for the last dt
    double* d_Lt = nullptr;       // [M * M][n_chol]
    std::vector<double> h_corr;   // [M][M]
    double* d_E[2] = {nullptr, nullptr};
    double prop_dt = -1.0;
};

namespace {

void free_mixed(msd_ctx* ctx);
void free_exact_ref(msd_ctx* ctx);
void free_prop(msd_ctx* ctx);

int fail(msd_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, MSD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define CKLAUNCH()                                                                        \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return fail(ctx, MSD_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int upload(msd_ctx* ctx, T** dst, const std::vector<T>& src)
{
    if (*dst) { cudaFree(*dst); *dst = nullptr; }
    if (src.empty()) return MSD_OK;
    CK(cudaMalloc((void**)dst, sizeof(T) * src.size()));
    CK(cudaMemcpy(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return MSD_OK;
}

void timer_begin(void* self, const char* name, cudaStream_t st)
{
    msd_ctx* c = (msd_ctx*)self;
    int k = -1;
    for (size_t i = 0; i < c->knames.size(); ++i)
        if (c->knames[i] == name) { k = (int)i; break; }
    if (k < 0) {
        k = (int)c->knames.size();
        c->knames.push_back(name);
        c->klaunch.push_back(0);
        c->kms.push_back(0);
    }
    cudaEvent_t e;
    if (c->ev_pool.empty()) cudaEventCreate(&e);
    else { e = c->ev_pool.back(); c->ev_pool.pop_back(); }
    cudaEventRecord(e, st);
    c->open_k = k;
    c->open_ev = e;
}

void timer_end(void* self, cudaStream_t st)
{
    msd_ctx* c = (msd_ctx*)self;
    if (c->open_k < 0) return;
    cudaEvent_t e;
    if (c->ev_pool.empty()) cudaEventCreate(&e);
    else { e = c->ev_pool.back(); c->ev_pool.pop_back(); }
    cudaEventRecord(e, st);
    c->pending.push_back({c->open_k, c->open_ev, e});
    c->open_k = -1;
}

void collect_timing(msd_ctx* c)
{
    for (auto& p : c->pending) {
        cudaEventSynchronize(p.b);
        float ms = 0;
        cudaEventElapsedTime(&ms, p.a, p.b);
        c->kms[p.k] += ms;
        c->klaunch[p.k] += 1;
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->pending.clear();
}

// Named device buffer of at least `bytes` (contents undefined on growth).
int arena_get(msd_ctx* ctx, const char* name, size_t bytes, void** out)
{
    Buf& b = ctx->arena[name];
    if (b.bytes < bytes) {
        if (b.p) { cudaDeviceSynchronize(); cudaFree(b.p); b.p = nullptr; b.bytes = 0; }
        bytes = (bytes + 255) & ~(size_t)255;
        ctx->gen++;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, MSD_ERR_NOMEM, "device allocation of %zu bytes for %s failed", bytes, name);
        }
        b.bytes = bytes;
    }
    *out = b.p;
    return MSD_OK;
}

bool is_device_ptr(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

SpinTables tables(const SpinHost& s, int cap)
{
    SpinTables t;
    t.N = s.N; t.nh = s.nh; t.np = s.np; t.n_str = s.n_str;
    for (int k = 0; k < MSD_KMAX + 2; ++k) t.bucket[k] = s.bucket[k];
    t.occ0 = s.d_occ0; t.pos0 = s.d_pos0; t.hole_pos = s.d_hole_pos; t.part_orb = s.d_part_orb;
    t.str_hp = reinterpret_cast<const uint4*>(s.d_str_hp); t.str_sign = s.d_str_sign;
    t.csr_off = s.d_csr_off; t.csr_other = s.d_csr_other; t.csr_c = s.d_csr_c;
    t.cmx = s.d_cmx;
    t.kx = s.d_kx;
    t.csr_cf = s.d_csr_cf;
    long long off = 0, xo = 0;
    for (int k = 0; k <= MSD_KMAX; ++k) {
        t.b_off[k] = off;
        t.cmx_off[k] = xo;
        off += (long long)cap * b_stride(k) * (s.bucket[k + 1] - s.bucket[k]);
        xo += (long long)k * k * (s.bucket[k + 1] - s.bucket[k]);
    }
    t.b_off[MSD_KMAX + 1] = off;
    t.cmx_off[MSD_KMAX + 1] = xo;
    t.b_per_walker = s.b_per_walker;
    return t;
}

PairTables pair_tables(const PairHost& p)
{
    PairTables t;
    t.n_det = p.n_det;
    for (int i = 0; i < (MSD_KMAX + 1) * (MSD_KMAX + 1) + 1; ++i) t.bucket[i] = p.bucket[i];
    t.a = p.d_a; t.b = p.d_b; t.c = p.d_c; t.cf = p.d_cf; t.det_index = p.d_det_index;
    for (int i = 0; i < (MSD_KMAX + 1) * (MSD_KMAX + 1); ++i) t.run_side[i] = p.run_side[i];
    for (int i = 0; i <= (MSD_KMAX + 1) * (MSD_KMAX + 1); ++i) t.run_off[i] = p.run_off[i];
    t.runs = p.d_runs;
    return t;
}

// Excitation strings of one spin from the occupation lists (Sec. II B: CI
// determinants as excitations of the reference, grouped by level).
int build_spin(msd_ctx* ctx, int s, const int32_t* occ, int n_det, std::vector<int>& sid)
{
    SpinHost& S = ctx->sp[s];
    const int N = ctx->n[s], M = ctx->M;
    S = SpinHost{};
    S.N = N;
    S.occ0.assign(occ, occ + N);
    std::vector<int> pos0(M, -1);
    for (int j = 0; j < N; ++j) {
        const int o = S.occ0[j];
        if (o < 0 || o >= M) return fail(ctx, MSD_ERR_ARG, "occupation %d out of range [0,%d)", o, M);
        if (j && o <= S.occ0[j - 1]) return fail(ctx, MSD_ERR_ARG, "reference occupations not strictly ascending");
        pos0[o] = j;
    }
    std::map<std::vector<int>, int> key2tmp;
    std::vector<std::vector<int>> keys;
    std::vector<int> tmp_of_det(n_det);
    std::vector<char> is_hole(M, 0), is_part(M, 0);
    std::vector<int> holes, parts, key;
    for (int I = 0; I < n_det; ++I) {
        const int32_t* o = occ + (size_t)I * N;
        holes.clear(); parts.clear();
        std::vector<char> in(M, 0);
        for (int j = 0; j < N; ++j) {
            if (o[j] < 0 || o[j] >= M)
                return fail(ctx, MSD_ERR_ARG, "determinant %d: orbital %d out of range", I, o[j]);
            if (j && o[j] <= o[j - 1])
                return fail(ctx, MSD_ERR_ARG, "determinant %d: occupations not strictly ascending", I);
            in[o[j]] = 1;
            if (pos0[o[j]] < 0) parts.push_back(o[j]);
        }
        for (int j = 0; j < N; ++j)
            if (!in[S.occ0[j]]) holes.push_back(S.occ0[j]);
        if ((int)holes.size() > MSD_KMAX)
            return fail(ctx, MSD_ERR_SHAPE, "determinant %d: excitation level %d above %d", I,
                        (int)holes.size(), MSD_KMAX);
        for (int h : holes) is_hole[h] = 1;
        for (int p : parts) is_part[p] = 1;
        key.assign(holes.begin(), holes.end());
        key.insert(key.end(), parts.begin(), parts.end());
        auto it = key2tmp.find(key);
        if (it == key2tmp.end()) {
            it = key2tmp.emplace(key, (int)keys.size()).first;
            keys.push_back(key);
        }
        tmp_of_det[I] = it->second;
    }
    for (int o = 0; o < M; ++o) {
        if (is_hole[o]) { S.hole_orb.push_back(o); S.hole_pos.push_back(pos0[o]); }
        if (is_part[o]) S.part_orb.push_back(o);
    }
    S.nh = (int)S.hole_orb.size();
    S.np = (int)S.part_orb.size();
    if (S.nh * S.np > MSD_XMAX)
        return fail(ctx, MSD_ERR_SHAPE, "spin %d: active block %d x %d exceeds %d entries", s, S.nh,
                    S.np, MSD_XMAX);
    std::vector<int> hidx(M, -1), pidx(M, -1);
    for (int i = 0; i < S.nh; ++i) hidx[S.hole_orb[i]] = i;
    for (int i = 0; i < S.np; ++i) pidx[S.part_orb[i]] = i;
    // order strings by level, then lexicographically
    std::vector<int> order(keys.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int x, int y) {
        if (keys[x].size() != keys[y].size()) return keys[x].size() < keys[y].size();
        return keys[x] < keys[y];
    });
    std::vector<int> final_of_tmp(keys.size());
    S.n_str = (int)keys.size();
    S.str_h.assign((size_t)S.n_str * MSD_KMAX, 0);
    S.str_p.assign((size_t)S.n_str * MSD_KMAX, 0);
    S.str_sign.assign(S.n_str, 1);
    S.str_k.assign(S.n_str, 0);
    for (int f = 0; f < S.n_str; ++f) {
        const std::vector<int>& k = keys[order[f]];
        final_of_tmp[order[f]] = f;
        const int lvl = (int)k.size() / 2;
        S.str_k[f] = lvl;
        std::vector<int> inplace(S.occ0);
        for (int i = 0; i < lvl; ++i) {
            S.str_h[(size_t)f * MSD_KMAX + i] = (uint8_t)hidx[k[i]];
            S.str_p[(size_t)f * MSD_KMAX + i] = (uint8_t)pidx[k[lvl + i]];
            inplace[pos0[k[i]]] = k[lvl + i];
        }
        int inv = 0;   // parity of the permutation that sorts the in-place list
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) inv += inplace[i] > inplace[j];
        S.str_sign[f] = (inv & 1) ? -1 : 1;
    }
    for (int k = 0; k <= MSD_KMAX + 1; ++k) S.bucket[k] = 0;
    for (int f = 0; f < S.n_str; ++f) S.bucket[S.str_k[f] + 1]++;
    for (int k = 1; k <= MSD_KMAX + 1; ++k) S.bucket[k] += S.bucket[k - 1];
    if (S.bucket[1] != 1 || keys[order[0]].size() != 0)
        return fail(ctx, MSD_ERR_ARG, "spin %d: the reference string is missing", s);
    S.b_per_walker = 0;
    for (int k = 0; k <= MSD_KMAX; ++k) S.b_per_walker += (long long)b_stride(k) * (S.bucket[k + 1] - S.bucket[k]);
    sid.resize(n_det);
    for (int I = 0; I < n_det; ++I) sid[I] = final_of_tmp[tmp_of_det[I]];
    return MSD_OK;
}

int upload_spin(msd_ctx* ctx, SpinHost& S)
{
    int rc;
    if ((rc = upload(ctx, &S.d_occ0, S.occ0))) return rc;
    if ((rc = upload(ctx, &S.d_hole_pos, S.hole_pos))) return rc;
    if ((rc = upload(ctx, &S.d_part_orb, S.part_orb))) return rc;
    {
        std::vector<uint8_t> rec((size_t)S.n_str * 16, 0);
        for (int f = 0; f < S.n_str; ++f)
            for (int i = 0; i < MSD_KMAX; ++i) {
                rec[(size_t)f * 16 + i] = S.str_h[(size_t)f * MSD_KMAX + i];
                rec[(size_t)f * 16 + 8 + i] = S.str_p[(size_t)f * MSD_KMAX + i];
            }
        if ((rc = upload(ctx, &S.d_str_hp, rec))) return rc;
    }
    if ((rc = upload(ctx, &S.d_str_sign, S.str_sign))) return rc;
    if ((rc = upload(ctx, &S.d_csr_off, S.csr_off))) return rc;
    if ((rc = upload(ctx, &S.d_csr_other, S.csr_other))) return rc;
    if ((rc = upload(ctx, &S.d_csr_c, S.csr_c))) return rc;
    std::vector<int> pos0(ctx->M, -1);
    for (int j = 0; j < S.N; ++j) pos0[S.occ0[j]] = j;
    if ((rc = upload(ctx, &S.d_pos0, pos0))) return rc;
    // active entry x = p_i nh + h_j of every (i, j) of every string's minor,
    // in the order of the inverse minors B
    // and the same entry's row of the Gram matrices, h_j np + p_i
    std::vector<uint8_t> cmx, kx;
    cmx.reserve((size_t)std::max<long long>(1, S.b_per_walker));
    kx.reserve((size_t)std::max<long long>(1, S.b_per_walker));
    for (int k = 1; k <= MSD_KMAX; ++k)
        for (int sidx = S.bucket[k]; sidx < S.bucket[k + 1]; ++sidx)
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j) {
                    const int p = S.str_p[(size_t)sidx * MSD_KMAX + i], h = S.str_h[(size_t)sidx * MSD_KMAX + j];
                    cmx.push_back((uint8_t)(p * S.nh + h));
                    kx.push_back((uint8_t)(h * S.np + p));
                }
    if (cmx.empty()) { cmx.push_back(0); kx.push_back(0); }
    if ((rc = upload(ctx, &S.d_cmx, cmx))) return rc;
    if ((rc = upload(ctx, &S.d_kx, kx))) return rc;
    std::vector<float> cf(S.csr_c.begin(), S.csr_c.end());
    if (cf.empty()) cf.push_back(0.f);
    if ((rc = upload(ctx, &S.d_csr_cf, cf))) return rc;
    return MSD_OK;
}

void free_spin(SpinHost& S)
{
    cudaFree(S.d_occ0); cudaFree(S.d_hole_pos); cudaFree(S.d_part_orb); cudaFree(S.d_str_hp);
    cudaFree(S.d_str_sign); cudaFree(S.d_csr_off); cudaFree(S.d_csr_other);
    cudaFree(S.d_csr_c); cudaFree(S.d_Lh); cudaFree(S.d_pos0);
    cudaFree(S.d_cmx); cudaFree(S.d_kx); cudaFree(S.d_csr_cf);
    S.d_cmx = nullptr;
    S.d_kx = nullptr;
    S.d_csr_cf = nullptr;
    S.d_pos0 = nullptr;
    S.d_occ0 = S.d_hole_pos = S.d_part_orb = nullptr;
    S.d_str_hp = nullptr;
    S.d_str_sign = nullptr;
    S.d_csr_off = S.d_csr_other = nullptr;
    S.d_csr_c = nullptr;
    S.d_Lh = nullptr;
}

// Half-rotated Cholesky vectors (the "half_rotate" of the trial, Sec. III):
// rows occ0 then P of each L_g, per spin, and both spins concatenated.
int build_half_rotated(msd_ctx* ctx)
{
    free_mixed(ctx);
    if (!ctx->have_ham || !ctx->have_trial) return MSD_OK;
    const int M = ctx->M, G = ctx->n_chol;
    long long Kd = 0;
    for (int s = 0; s < 2; ++s) Kd += (long long)(ctx->sp[s].N + ctx->sp[s].np) * M;
    ctx->Kd = Kd;
    std::vector<double> cat((size_t)G * Kd);
    long long off = 0;
    for (int s = 0; s < 2; ++s) {
        SpinHost& S = ctx->sp[s];
        const int NC = S.N + S.np;
        std::vector<double> lh((size_t)G * NC * M);
        for (int g = 0; g < G; ++g)
            for (int c = 0; c < NC; ++c) {
                const int row = c < S.N ? S.occ0[c] : S.part_orb[c - S.N];
                const double* src = &ctx->h_L[((size_t)g * M + row) * M];
                std::copy(src, src + M, &lh[((size_t)g * NC + c) * M]);
                std::copy(src, src + M, &cat[(size_t)g * Kd + off + (size_t)c * M]);
            }
        int rc = upload(ctx, &S.d_Lh, lh);
        if (rc) return rc;
        off += (long long)NC * M;
    }
    return upload(ctx, &ctx->d_Lcat, cat);
}

void free_mixed(msd_ctx* ctx)
{
    ctx->gen++;
    for (int s = 0; s < 2; ++s) {
        cudaFree(ctx->LhF_hi[s]); cudaFree(ctx->LhF_lo[s]);
        ctx->LhF_hi[s] = ctx->LhF_lo[s] = nullptr;
        cudaFree(ctx->LhP_hi[s]); cudaFree(ctx->LhP_lo[s]); cudaFree(ctx->d_F0P[s]);
        ctx->LhP_hi[s] = ctx->LhP_lo[s] = ctx->d_F0P[s] = nullptr;
    }
    cudaFree(ctx->Lv_hi); cudaFree(ctx->Lv_lo);
    ctx->Lv_hi = ctx->Lv_lo = nullptr;
    for (int s = 0; s < 2; ++s) {
        cudaFree(ctx->d_virt[s]); cudaFree(ctx->d_c0[s]); cudaFree(ctx->d_x0[s]); cudaFree(ctx->d_F0T[s]);
        ctx->d_virt[s] = nullptr; ctx->d_c0[s] = ctx->d_x0[s] = nullptr; ctx->d_F0T[s] = nullptr;
    }
    cudaFree(ctx->d_c0sum);
    ctx->d_c0sum = nullptr;
    ctx->mixed_ready = false;
    free_exact_ref(ctx);
}

void free_exact_ref(msd_ctx* ctx)
{
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && ctx->oz_shared) {
            ctx->oz[1] = OzConst{};
            ctx->d_JJ[1] = ctx->d_KK[1] = nullptr;
            continue;
        }
        oz_free_const(ctx->oz[s]);
        cudaFree(ctx->d_JJ[s]); cudaFree(ctx->d_KK[s]);
        ctx->d_JJ[s] = ctx->d_KK[s] = nullptr;
    }
    cudaFree(ctx->d_hJ);
    ctx->d_hJ = nullptr;
    ctx->oz_shared = false;
    ctx->oz_ready = ctx->oz_ok = false;
}

// Largest N (M - N) per spin for which the exact reference sums are built
// (their constant operand takes about 10 (N (M - N) + n_chol) N (M - N) bytes).
constexpr long long OZ_MAX_NK = 16384;

bool exact_ref_shapes_ok(const msd_ctx* ctx)
{
    for (int s = 0; s < 2; ++s) {
        const long long NK = (long long)ctx->sp[s].N * (ctx->M - ctx->sp[s].N);
        if (NK <= 0 || NK > OZ_MAX_NK) return false;
    }
    return ctx->n_chol > 0;
}

// Constants of the exact reference part, once per Hamiltonian and trial.
// With C_g = c0a_g + c0b_g (c0 = tr(L_g D0 D0^T) per spin), v_r the orbitals
// outside occ0 and u[(j, r)] = dG[occ0_j][v_r]:
//   sum_g C_g t1_g      = u . JJ,  JJ[(j, r)] = (sum_g C_g L_g)[v_r][o_j]
//   sum_g tr(T0_g dT_g) = u . KK,  KK[(j, r)] = (sum_g L_g D0 D0^T L_g)[v_r][o_j]
// (both linear in dG, FP64), x0sum = sum_g x0_g, C2sum = sum_g C_g^2, and the
// sliced constant operand [V | W] of tc_ozaki.cu.
int prepare_exact_ref(msd_ctx* ctx, cudaStream_t st)
{
    if (ctx->oz_ready) return MSD_OK;
    free_exact_ref(ctx);
    ctx->oz_ready = true;
    if (!exact_ref_shapes_ok(ctx)) return MSD_OK;
    const int M = ctx->M, G = ctx->n_chol;
    const double* L = ctx->h_L.data();
    auto Lv = [&](int g, int p, int q) { return L[((size_t)g * M + p) * M + q]; };
    std::vector<double> C(G, 0.0);
    for (int s = 0; s < 2; ++s)
        for (int g = 0; g < G; ++g)
            for (int o : ctx->sp[s].occ0) C[g] += Lv(g, o, o);
    ctx->oz_C2sum = 0;
    for (int g = 0; g < G; ++g) ctx->oz_C2sum += C[g] * C[g];
    ctx->oz_shared = ctx->sp[1].occ0 == ctx->sp[0].occ0;
    for (int s = 0; s < 2; ++s) {
        const SpinHost& S = ctx->sp[s];
        const int N = S.N;
        double x0 = 0;
        for (int g = 0; g < G; ++g)
            for (int j = 0; j < N; ++j)
                for (int l = 0; l < N; ++l) x0 += Lv(g, S.occ0[j], S.occ0[l]) * Lv(g, S.occ0[j], S.occ0[l]);
        ctx->oz_x0sum[s] = x0;
        if (s == 1 && ctx->oz_shared) {
            ctx->oz[1] = ctx->oz[0];
            ctx->d_JJ[1] = ctx->d_JJ[0];
            ctx->d_KK[1] = ctx->d_KK[0];
            continue;
        }
        std::vector<char> in0(M, 0);
        for (int o : S.occ0) in0[o] = 1;
        std::vector<int> v;
        for (int o = 0; o < M; ++o) if (!in0[o]) v.push_back(o);
        const int Kv = (int)v.size(), NK = N * Kv;
        std::vector<double> XT((size_t)NK * G), JJ(NK, 0.0), KK(NK, 0.0);
        for (int r = 0; r < Kv; ++r)
            for (int l = 0; l < N; ++l)
                for (int g = 0; g < G; ++g) XT[((size_t)r * N + l) * G + g] = Lv(g, v[r], S.occ0[l]);
        std::vector<double> row(N);
        for (int g = 0; g < G; ++g)
            for (int r = 0; r < Kv; ++r) {
                for (int l = 0; l < N; ++l) row[l] = Lv(g, v[r], S.occ0[l]);
                for (int j = 0; j < N; ++j) {
                    double k = 0;
                    for (int l = 0; l < N; ++l) k += row[l] * Lv(g, S.occ0[l], S.occ0[j]);
                    JJ[(size_t)j * Kv + r] += C[g] * row[j];
                    KK[(size_t)j * Kv + r] += k;
                }
            }
        int rc;
        if ((rc = upload(ctx, &ctx->d_JJ[s], JJ)) || (rc = upload(ctx, &ctx->d_KK[s], KK))) return rc;
        double* d_XT = nullptr;
        if ((rc = upload(ctx, &d_XT, XT))) return rc;
        const int pr = oz_prepare_const(N, Kv, G, d_XT, ctx->oz[s], st);
        CK(cudaStreamSynchronize(st));
        cudaFree(d_XT);
        if (pr) return fail(ctx, MSD_ERR_NOMEM, "exact reference constants (%lld bytes) could not be built",
                            (long long)oz_const_bytes(N, Kv, G));
    }
    {
        // J = sum_g C_g L_g: the reference part of sum_g V0_g Lambda_g is the
        // one-body term of J, (G J (I - G))[H][P]; kept as h_s + J
        std::vector<double> hJ(ctx->h_h1.begin(), ctx->h_h1.begin() + (size_t)2 * M * M);
        for (int g = 0; g < G; ++g) {
            const double* Lg = L + (size_t)g * M * M;
            for (size_t e = 0; e < (size_t)M * M; ++e) {
                hJ[e] += C[g] * Lg[e];
                hJ[(size_t)M * M + e] += C[g] * Lg[e];
            }
        }
        int rc;
        if ((rc = upload(ctx, &ctx->d_hJ, hJ))) return rc;
    }
    ctx->oz_ok = true;
    return MSD_OK;
}

// The exact reference sums run for this call.
bool exact_ref_on(const msd_ctx* ctx) { return ctx->prec == MSD_MIXED && ctx->exact_ref && exact_ref_shapes_ok(ctx); }

// Mixed-path operands, once per Hamiltonian and trial. The reference part
// of the Green's function is known exactly: Theta[occ0, :] = I, so
// G = D0 D0^T + dG with dG non-zero only in the columns of the orbitals
// outside occ0 ("virtual" columns). The tensor cores contract only dG with
// L (TF32 hi/lo splits gathered at the virtual columns); the reference
// parts enter in FP64:
//   c0_g = tr(L_g D0 D0^T) = sum_j L_g[occ0_j][occ0_j],
//   x0_g = tr(L_g D0 D0^T L_g D0 D0^T) = sum_jl L_g[occ0_j][occ0_l]^2.
int prepare_mixed(msd_ctx* ctx, cudaStream_t st)
{
    if (ctx->mixed_ready) return MSD_OK;
    const int M = ctx->M, G = ctx->n_chol;
    ctx->Kp = (M + 31) / 32 * 32;
    ctx->Kdp = (ctx->Kd + 31) / 32 * 32;
    std::vector<double> c0sum(G, 0.0);
    for (int s = 0; s < 2; ++s) {
        const SpinHost& S = ctx->sp[s];
        std::vector<char> in0(M, 0);
        for (int o : S.occ0) in0[o] = 1;
        std::vector<int> virt;
        for (int o = 0; o < M; ++o) if (!in0[o]) virt.push_back(o);
        const int Kv = (int)virt.size();
        ctx->Kv[s] = Kv;
        ctx->Kvp[s] = std::max(32, (Kv + 31) / 32 * 32);
        ctx->fused_ok[s] = tc_fepi_plan(tables(S, 1), ctx->fplan[s]);
        ctx->Kv8[s] = std::max(8, (Kv + 7) / 8 * 8);
        ctx->Kfp[s] = ctx->fused_ok[s] ? ctx->Kv8[s] + 2 * ctx->fplan[s].RB : ctx->Kvp[s];
        if (Kv == 0) virt.push_back(0);   // keeps the gather pointer valid; Kg = 0 pads with zeros
        int rc = upload(ctx, &ctx->d_virt[s], virt);
        if (rc) return rc;
        std::vector<double> c0(G), x0(G);
        for (int g = 0; g < G; ++g) {
            const double* Lg = &ctx->h_L[(size_t)g * M * M];
            double a = 0, b = 0;
            for (int j = 0; j < S.N; ++j) {
                a += Lg[(size_t)S.occ0[j] * M + S.occ0[j]];
                for (int l = 0; l < S.N; ++l) {
                    const double v = Lg[(size_t)S.occ0[j] * M + S.occ0[l]];
                    b += v * v;
                }
            }
            c0[g] = a; x0[g] = b; c0sum[g] += a;
        }
        if ((rc = upload(ctx, &ctx->d_c0[s], c0))) return rc;
        if ((rc = upload(ctx, &ctx->d_x0[s], x0))) return rc;
        const int NC = S.N + S.np;
        std::vector<float> f0t((size_t)G * S.N * NC);
        for (int g = 0; g < G; ++g)
            for (int j = 0; j < S.N; ++j)
                for (int cc = 0; cc < NC; ++cc) {
                    const int col = cc < S.N ? S.occ0[cc] : S.part_orb[cc - S.N];
                    f0t[((size_t)g * S.N + j) * NC + cc] = (float)ctx->h_L[((size_t)g * M + S.occ0[j]) * M + col];
                }
        if ((rc = upload(ctx, &ctx->d_F0T[s], f0t))) return rc;
        const long long R = (long long)G * (S.N + S.np);
        CK(cudaMalloc(&ctx->LhF_hi[s], sizeof(float) * R * ctx->Kvp[s]));
        CK(cudaMalloc(&ctx->LhF_lo[s], sizeof(float) * R * ctx->Kvp[s]));
        launch_split_real_rows(R, Kv, ctx->Kvp[s], S.d_Lh, M, ctx->d_virt[s], ctx->LhF_hi[s], ctx->LhF_lo[s], st);
        if (ctx->fused_ok[s]) {
            // vector g's columns: occ0 (N), zero (RB - N), particles (np)
            const int RB = ctx->fplan[s].RB, NCf = RB + S.np, NCP = ctx->fplan[s].NCP, f0s = ctx->fplan[s].f0s;
            std::vector<double> lp((size_t)G * NCf * M, 0.0);
            std::vector<float> f0p((size_t)G * f0s, 0.f);   // [g][j NCP + col], the kernel's shared layout
            std::vector<double> f0r((size_t)G * NCf * S.N, 0.0);   // [(g, col)][j] = F0_g[j][col] in FP64
            for (int g = 0; g < G; ++g)
                for (int cc = 0; cc < NCf; ++cc) {
                    const int col = cc < S.N ? S.occ0[cc] : cc >= RB ? S.part_orb[cc - RB] : -1;
                    if (col < 0) continue;
                    const double* src = &ctx->h_L[((size_t)g * M + col) * M];
                    std::copy(src, src + M, &lp[((size_t)g * NCf + cc) * M]);
                    for (int j = 0; j < S.N; ++j) {
                        const double v = ctx->h_L[((size_t)g * M + S.occ0[j]) * M + col];
                        f0p[(size_t)g * f0s + (size_t)j * NCP + cc] = (float)v;
                        f0r[((size_t)g * NCf + cc) * S.N + j] = v;
                    }
                }
            double *d_lp = nullptr, *d_f0r = nullptr;
            if ((rc = upload(ctx, &d_lp, lp))) return rc;
            if ((rc = upload(ctx, &d_f0r, f0r))) { cudaFree(d_lp); return rc; }
            if ((rc = upload(ctx, &ctx->d_F0P[s], f0p))) { cudaFree(d_lp); cudaFree(d_f0r); return rc; }
            const long long RP = (long long)G * NCf;
            CK(cudaMalloc(&ctx->LhP_hi[s], sizeof(float) * RP * ctx->Kfp[s]));
            CK(cudaMalloc(&ctx->LhP_lo[s], sizeof(float) * RP * ctx->Kfp[s]));
            launch_split_real_rows(RP, Kv, ctx->Kfp[s], d_lp, M, ctx->d_virt[s], ctx->LhP_hi[s], ctx->LhP_lo[s], st);
            // the F0 slices behind the contraction columns (used when the
            // contraction adds F0 itself)
            launch_split_blocks(RP, S.N, RB, ctx->Kfp[s], ctx->Kv8[s], d_f0r, ctx->LhP_hi[s], ctx->LhP_lo[s], st);
            CK(cudaStreamSynchronize(st));
            cudaFree(d_lp);
            cudaFree(d_f0r);
        }
    }
    int rc = upload(ctx, &ctx->d_c0sum, c0sum);
    if (rc) return rc;
    CK(cudaMalloc(&ctx->Lv_hi, sizeof(float) * G * ctx->Kdp));
    CK(cudaMalloc(&ctx->Lv_lo, sizeof(float) * G * ctx->Kdp));
    launch_split_real_rows(G, (int)ctx->Kd, (int)ctx->Kdp, ctx->d_Lcat, ctx->Kd, nullptr, ctx->Lv_hi, ctx->Lv_lo,
                           st);
    CKLAUNCH();
    CK(cudaStreamSynchronize(st));
    ctx->mixed_ready = true;
    return MSD_OK;
}

int check_ready(msd_ctx* ctx)
{
    if (!ctx) return MSD_ERR_ARG;
    if (!ctx->have_ham || !ctx->have_trial)
        return fail(ctx, MSD_ERR_STATE, "set the Hamiltonian and the trial first");
    return MSD_OK;
}

// Walkers per chunk for a given per-walker footprint.
int chunk_for(msd_ctx* ctx, size_t per_walker, int n_w)
{
    size_t c = per_walker ? ctx->ws_limit / per_walker : (size_t)n_w;
    if (c < 1) c = 1;
    if (c > (size_t)n_w) c = n_w;
    ctx->chunk = (int)c;
    return (int)c;
}

// Inputs: device pointers pass through; host pointers are copied into
// context-owned staging buffers.
struct Staged {
    const double2* pa;
    const double2* pb;
    bool host_any;
    cudaEvent_t b_ready = nullptr;   // the beta copy has landed (wait before its first use)
};

// With defer_b, host beta walkers are copied on the context's copy stream
// (after the work already on st, which may still use the staging buffer);
// out.b_ready then marks the copy's completion.
int stage_inputs(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                 cudaStream_t st, Staged& out, bool defer_b = false)
{
    const size_t ba = sizeof(double2) * (size_t)n_w * ctx->M * ctx->n[0];
    const size_t bb = sizeof(double2) * (size_t)n_w * ctx->M * ctx->n[1];
    out.host_any = false;
    out.b_ready = nullptr;
    if (defer_b && !is_device_ptr(phi_b) && !ctx->copy_st) {
        if (cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_b, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, MSD_ERR_CUDA, "copy stream could not be created");
    }
    if (is_device_ptr(phi_a)) out.pa = (const double2*)phi_a;
    else {
        void* p; int rc = arena_get(ctx, "stage_phi_a", ba, &p); if (rc) return rc;
        CK(cudaMemcpyAsync(p, phi_a, ba, cudaMemcpyHostToDevice, st));
        out.pa = (const double2*)p; out.host_any = true;
    }
    if (is_device_ptr(phi_b)) out.pb = (const double2*)phi_b;
    else {
        void* p; int rc = arena_get(ctx, "stage_phi_b", bb, &p); if (rc) return rc;
        if (defer_b) {
            CK(cudaEventRecord(ctx->ev_in, st));
            CK(cudaStreamWaitEvent(ctx->copy_st, ctx->ev_in, 0));
            CK(cudaMemcpyAsync(p, phi_b, bb, cudaMemcpyHostToDevice, ctx->copy_st));
            CK(cudaEventRecord(ctx->ev_b, ctx->copy_st));
            out.b_ready = ctx->ev_b;
        } else {
            CK(cudaMemcpyAsync(p, phi_b, bb, cudaMemcpyHostToDevice, st));
        }
        out.pb = (const double2*)p; out.host_any = true;
    }
    return MSD_OK;
}

// Output either written directly (device) or via staging then copied back.
struct Out {
    double* user = nullptr;
    double2* dev = nullptr;
    size_t bytes = 0;
    bool host = false;
};

int stage_output(msd_ctx* ctx, const char* name, double* user, size_t n_complex, Out& o)
{
    o.user = user;
    o.bytes = sizeof(double2) * n_complex;
    if (!user) { o.dev = nullptr; return MSD_OK; }
    if (is_device_ptr(user)) { o.dev = (double2*)user; o.host = false; return MSD_OK; }
    void* p; int rc = arena_get(ctx, name, o.bytes, &p); if (rc) return rc;
    o.dev = (double2*)p; o.host = true;
    return MSD_OK;
}

int finish(msd_ctx* ctx, cudaStream_t st, std::initializer_list<Out*> outs, bool host_in)
{
    bool host = host_in;
    for (Out* o : outs)
        if (o->user && o->host) {
            CK(cudaMemcpyAsync(o->user, o->dev, o->bytes, cudaMemcpyDeviceToHost, st));
            host = true;
        }
    CKLAUNCH();
    if (ctx->sync || host) {
        CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const unsigned e = *ctx->h_err;
        if (e & MSD_DEV_ERR_SINGULAR)
            return fail(ctx, MSD_ERR_REF_SINGULAR, "D_0^dag phi is singular for some walker");
        if (e & MSD_DEV_ERR_TIMEOUT) return fail(ctx, MSD_ERR_TIMEOUT, "a device-side wait expired");
        if (e & MSD_DEV_ERR_BOUNDS) return fail(ctx, MSD_ERR_SHAPE, "a device-side bounds check failed");
    }
    return MSD_OK;
}

// Per-chunk workspace for the overlap part.
struct Chunk {
    double2 *Gr[2], *O0[2], *Gact[2], *r[2], *wts[2], *part;
    float2* rf[2];   // FP32 copies of r (mixed mode, with B)
    void* B[2];
    int nslot, nR;
};

size_t overlap_bytes_per_walker(msd_ctx* ctx, bool want_b, int nslot)
{
    size_t b = 0;
    for (int s = 0; s < 2; ++s) {
        const SpinHost& S = ctx->sp[s];
        b += (size_t)S.N * ctx->M + 1 + (size_t)S.nh * S.np + 2 * (size_t)S.n_str;
        if (want_b) b += S.b_per_walker + (S.n_str + 1) / 2;
    }
    b += nslot;
    return b * sizeof(double2);
}

int chunk_alloc(msd_ctx* ctx, int cap, bool want_b, int nslot, Chunk& c)
{
    int rc;
    static const char* nGr[2] = {"Gr_a", "Gr_b"}, *nO0[2] = {"O0_a", "O0_b"};
    static const char* nGa[2] = {"Gact_a", "Gact_b"}, *nr[2] = {"r_a", "r_b"};
    static const char* nw[2] = {"wts_a", "wts_b"}, *nB[2] = {"B_a", "B_b"}, *nrf[2] = {"rf_a", "rf_b"};
    for (int s = 0; s < 2; ++s) {
        const SpinHost& S = ctx->sp[s];
        void* p;
        if ((rc = arena_get(ctx, nGr[s], sizeof(double2) * cap * S.N * ctx->M, &p))) return rc; c.Gr[s] = (double2*)p;
        if ((rc = arena_get(ctx, nO0[s], sizeof(double2) * cap, &p))) return rc; c.O0[s] = (double2*)p;
        if ((rc = arena_get(ctx, nGa[s], sizeof(double2) * cap * std::max(1, S.nh * S.np), &p))) return rc; c.Gact[s] = (double2*)p;
        if ((rc = arena_get(ctx, nr[s], sizeof(double2) * cap * S.n_str, &p))) return rc; c.r[s] = (double2*)p;
        if ((rc = arena_get(ctx, nw[s], sizeof(double2) * cap * S.n_str, &p))) return rc; c.wts[s] = (double2*)p;
        c.B[s] = nullptr;
        c.rf[s] = nullptr;
        if (want_b) {
            if ((rc = arena_get(ctx, nB[s], sizeof(double2) * std::max<long long>(1, cap * S.b_per_walker), &p))) return rc;
            c.B[s] = p;
            if ((rc = arena_get(ctx, nrf[s], sizeof(float2) * cap * S.n_str, &p))) return rc;
            c.rf[s] = (float2*)p;
        }
    }
    void* p;
    if ((rc = arena_get(ctx, "part", sizeof(double2) * cap * std::max(1, nslot), &p))) return rc;
    c.part = (double2*)p;
    c.nslot = nslot;
    c.nR = weights_blocks(tables(ctx->sp[0], cap));
    return MSD_OK;
}

// Reference inverse of walkers [w0, w0 + nw), both spins.
int run_refs(msd_ctx* ctx, const Staged& in, int w0, int nw, int cap, Chunk& c, cudaStream_t st)
{
    const int M = ctx->M;
    const TimerHook& th = ctx->hook;
    SpinTables T[2] = {tables(ctx->sp[0], cap), tables(ctx->sp[1], cap)};
    const double2* phi[2] = {in.pa + (size_t)w0 * M * ctx->n[0], in.pb + (size_t)w0 * M * ctx->n[1]};
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && in.b_ready) CK(cudaStreamWaitEvent(st, in.b_ready, 0));
        th.begin("k_ref", st);
        launch_ref(phi[s], nw, M, ctx->n[s], T[s], c.Gr[s], c.O0[s], c.Gact[s], ctx->d_err, st);
        th.end(st);
        CKLAUNCH();
    }
    return MSD_OK;
}

// String minors, ratios and weights of a chunk whose reference inverse is done.
int run_strings_weights(msd_ctx* ctx, int nw, int cap, Chunk& c, bool want_b, bool fp32_b, cudaStream_t st)
{
    const TimerHook& th = ctx->hook;
    SpinTables T[2] = {tables(ctx->sp[0], cap), tables(ctx->sp[1], cap)};
    for (int s = 0; s < 2; ++s) {
        launch_strings(T[s], nw, c.Gact[s], c.r[s], fp32_b ? c.rf[s] : nullptr, c.B[s], fp32_b, want_b, st, th);
        CKLAUNCH();
    }
    th.begin("k_weights", st);
    launch_weights(T[0], nw, c.r[0], c.r[1], T[1].n_str, c.wts[0], c.part, c.nslot, 0, st);
    launch_weights(T[1], nw, c.r[1], c.r[0], T[0].n_str, c.wts[1], nullptr, c.nslot, 0, st);
    th.end(st);
    CKLAUNCH();
    return MSD_OK;
}

// Reference inverse, string minors and weights for walkers [w0, w0 + nw).
int run_overlap_part(msd_ctx* ctx, const Staged& in, int w0, int nw, int cap, Chunk& c,
                     bool want_b, bool fp32_b, cudaStream_t st)
{
    int rc = run_refs(ctx, in, w0, nw, cap, c, st);
    return rc ? rc : run_strings_weights(ctx, nw, cap, c, want_b, fp32_b, st);
}

int begin_call(msd_ctx* ctx, int n_w, const double* pa, const double* pb, cudaStream_t st)
{
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (n_w < 0 || (n_w > 0 && (!pa || !pb))) return fail(ctx, MSD_ERR_ARG, "bad walker arguments");
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), st));
    return MSD_OK;
}


// ------------------------------------------------------------------ parts
// Force-bias part for one chunk: cofactor matrix, G_T rows, contraction
// with the half-rotated Cholesky vectors.
struct FbWork {
    void *GT = nullptr, *Rs = nullptr, *Cm[2] = {nullptr, nullptr};
    void *Ah = nullptr, *Al = nullptr, *C32 = nullptr;
    int ks = 1;
};

size_t fb_bytes_per_walker(msd_ctx* ctx, bool fp32)
{
    size_t b = sizeof(double2) * (ctx->Kd + 1);
    for (int s = 0; s < 2; ++s) {
        const SpinTables t = tables(ctx->sp[s], 1);
        b += sizeof(double2) * (size_t)t.nh * t.np;
    }
    if (fp32) b += sizeof(float) * 2 * 2 * ctx->Kdp + sizeof(float) * 16 * 2 * ctx->n_chol;
    return b;
}

int fb_alloc(msd_ctx* ctx, int cap, bool fp32, FbWork& f)
{
    int rc;
    if ((rc = arena_get(ctx, "GT", sizeof(double2) * cap * ctx->Kd, &f.GT))) return rc;
    if ((rc = arena_get(ctx, "Rsum", sizeof(double2) * cap, &f.Rs))) return rc;
    for (int s = 0; s < 2; ++s) {
        const SpinTables t = tables(ctx->sp[s], 1);
        static const char* nm[2] = {"Cm_a", "Cm_b"};
        if ((rc = arena_get(ctx, nm[s], sizeof(double2) * cap * std::max(1, t.nh * t.np), &f.Cm[s]))) return rc;
    }
    if (fp32) {
        f.ks = std::max(1, std::min(16, (int)(ctx->Kdp / 32 / 64)));
        if ((rc = arena_get(ctx, "Av_hi", sizeof(float) * 2 * cap * ctx->Kdp, &f.Ah))) return rc;
        if ((rc = arena_get(ctx, "Av_lo", sizeof(float) * 2 * cap * ctx->Kdp, &f.Al))) return rc;
        if ((rc = arena_get(ctx, "Cv32", sizeof(float) * f.ks * 2 * cap * ctx->n_chol, &f.C32))) return rc;
    }
    return MSD_OK;
}

int fb_chunk(msd_ctx* ctx, Chunk& c, FbWork& f, int w0, int nw, int cap, bool fp32, double2* vb_out,
             double2* ov_out, cudaStream_t st)
{
    const TimerHook& th = ctx->hook;
    int rc;
    th.begin("k_sum_slots", st);
    launch_sum_slots(nw, c.part, c.nslot, 0, c.nR, (double2*)f.Rs, c.O0[0], c.O0[1],
                     ov_out ? ov_out + w0 : nullptr, st);
    th.end(st);
    long long off = 0;
    th.begin("k_cmat", st);
    launch_cmat(tables(ctx->sp[0], cap), tables(ctx->sp[1], cap), nw, c.wts[0], c.wts[1], c.B[0], c.B[1], fp32,
                (double2*)f.Cm[0], (double2*)f.Cm[1], st);
    th.end(st);
    for (int s = 0; s < 2; ++s) {
        const SpinTables T = tables(ctx->sp[s], cap);
        th.begin("k_gt", st);
        launch_gt(T, nw, ctx->M, c.Gr[s], (double2*)f.Cm[s], (double2*)f.Rs, (double2*)f.GT, ctx->Kd, off, fp32,
                  st);
        th.end(st);
        off += (long long)(T.N + T.np) * ctx->M;
    }
    CKLAUNCH();
    double2* out = vb_out + (size_t)w0 * ctx->n_chol;
    if (fp32) {
        // vbias = c0_a + c0_b + (GT - D0 D0^T) . Lcat^T, the contraction on the
        // tensor cores (3xTF32, rows (w, re/im), K split over CTAs, the splits
        // summed in FP64)
        th.begin("k_split_vbias", st);
        launch_split_complex_rows(nw, 1, (int)ctx->Kd, (int)ctx->Kdp, (const double2*)f.GT, ctx->Kd, nullptr,
                                  (float*)f.Ah, (float*)f.Al, st);
        th.end(st);
        th.begin("tc_gemm_vbias", st);
        const long long sstride = (long long)2 * nw * ctx->n_chol;
        rc = tc_gemm_3xtf32({(float*)f.Ah, (float*)f.Al, ctx->Kdp}, {ctx->Lv_hi, ctx->Lv_lo, ctx->Kdp}, 2 * nw,
                            ctx->n_chol, (int)ctx->Kdp, (float*)f.C32, ctx->n_chol, ctx->d_err, st, f.ks, sstride);
        th.end(st);
        if (rc) return fail(ctx, MSD_ERR_CUDA, "tensor-core GEMM launch failed (force bias)");
        th.begin("k_pack_vbias", st);
        launch_pack_complex(nw, ctx->n_chol, (float*)f.C32, ctx->n_chol, f.ks, sstride, ctx->d_c0sum, out,
                            ctx->n_chol, st);
        th.end(st);
    } else {
        th.begin("k_gemm_vbias", st);
        launch_gemm_zd(nw, ctx->n_chol, (int)ctx->Kd, (const double2*)f.GT, ctx->Kd, ctx->d_Lcat, ctx->Kd, out,
                       ctx->n_chol, st);
        th.end(st);
    }
    CKLAUNCH();
    return MSD_OK;
}

// Energy part for one chunk.
struct EnWork {
    void *F[2] = {nullptr, nullptr}, *F32 = nullptr, *Ah = nullptr, *Al = nullptr;
    void *v0[2], *xx[2], *La[2], *Xi[2], *Lh1[2], *e1[2], *Y[2], *Kaa, *Kbb, *Kab, *scal;
    void *ozA = nullptr, *ozE = nullptr, *ozP[2] = {nullptr, nullptr}, *ozT[2] = {nullptr, nullptr};
    void* v0w = nullptr;   // [nw][G] FP32 walker parts of V0_g (exact reference sums)
    void* GT[2] = {nullptr, nullptr};   // [nw][2X][G] Lambda rows for the tensor-core Gram
};

// The Gram matrices run on the tensor cores (msd_set_tensor_gram, shapes allowing).
bool tensor_gram(const msd_ctx* ctx)
{
    const int Xa = ctx->sp[0].nh * ctx->sp[0].np, Xb = ctx->sp[1].nh * ctx->sp[1].np;
    return ctx->prec == MSD_MIXED && ctx->tc_gram && ctx->n_chol % 4 == 0 && tc_gram_ok(Xa, Xb);
}

// The fused tensor-core contraction + epilogue serves spin s.
bool fused(const msd_ctx* ctx, int s) { return ctx->fuse && ctx->fused_ok[s]; }

// Rows of the split A operand per walker: 2N, or the fused kernel's padded RW.
int a_rows(const msd_ctx* ctx, int s) { return fused(ctx, s) ? ctx->fplan[s].RW : 2 * ctx->sp[s].N; }
int a_ld(const msd_ctx* ctx, int s) { return fused(ctx, s) ? ctx->Kfp[s] : ctx->Kvp[s]; }

// The form of the opposite-spin term this call takes: 0 per determinant,
// 1 per beta string (mixed precision only), 2 runs sharing a string.
int pair_form_now(const msd_ctx* ctx)
{
    const int want = ctx->pair_form < 0 ? 2 : ctx->pair_form;
    if (want == 1 && !(ctx->prec == MSD_MIXED && pair_y_ok(tables(ctx->sp[0], 1), tables(ctx->sp[1], 1))))
        return 0;
    return want;
}

bool use_pair_y(const msd_ctx* ctx) { return pair_form_now(ctx) == 1; }
bool use_runs(const msd_ctx* ctx) { return pair_form_now(ctx) == 2; }

int energy_slots(msd_ctx* ctx)
{
    const SpinTables ta = tables(ctx->sp[0], 1), tb = tables(ctx->sp[1], 1);
    return string_energy_slots(ta) + string_energy_slots(tb) +
           (use_pair_y(ctx) ? pair_y_slots(tb) : pair_cross_slots(pair_tables(ctx->pairs), use_runs(ctx)));
}

size_t en_bytes_per_walker(msd_ctx* ctx, bool fp32)
{
    const int G = ctx->n_chol;
    SpinTables T1[2] = {tables(ctx->sp[0], 1), tables(ctx->sp[1], 1)};
    const int X[2] = {T1[0].nh * T1[0].np, T1[1].nh * T1[1].np};
    size_t e = 8 + 2;
    // per vector: v0, xx and the two Lambda / Xi rows (FP64 rows of X entries,
    // or FP32 rows of the pitch lam_pitch(X), counted in double2 units)
    for (int s = 0; s < 2; ++s)
        e += (size_t)G * (2 + std::max(2 * X[s], lam_pitch(std::max(1, X[s])))) + 3 * X[s] + 1;
    e += (size_t)X[0] * X[0] + (size_t)X[1] * X[1] + (size_t)X[0] * X[1];
    size_t b = e * sizeof(double2);
    if (fp32 && exact_ref_on(ctx)) {
        int kp = 0;
        for (int s = 0; s < 2; ++s) kp = std::max(kp, oz_k_padded(T1[s].N * (ctx->M - T1[s].N)));
        b += (size_t)2 * oz_slices() * kp * 2 + 2 * sizeof(int);
        b += sizeof(float2) * (size_t)G;   // v0w
        for (int s = 0; s < 2; ++s)
            b += (size_t)2 * oz_parts_for(T1[s].N * (ctx->M - T1[s].N), G) * sizeof(double2) + 2 * sizeof(double) * G;
    }
    if (fp32 && tensor_gram(ctx)) b += sizeof(float) * 2 * (size_t)(X[0] + X[1]) * G;   // GT
    if (fp32) {
        size_t f = 0, a = 0;
        for (int s = 0; s < 2; ++s) {
            if (!fused(ctx, s))
                f = std::max(f, sizeof(float) * 2 * T1[s].N * (size_t)G * (T1[s].N + T1[s].np));
            a = std::max(a, sizeof(float) * 2 * a_rows(ctx, s) * (size_t)a_ld(ctx, s));
        }
        b += f + a;
    } else {
        for (int s = 0; s < 2; ++s) b += sizeof(double2) * T1[s].N * (size_t)G * (T1[s].N + T1[s].np);
    }
    return b;
}

int en_alloc(msd_ctx* ctx, int cap, bool fp32, EnWork& E)
{
    const int G = ctx->n_chol;
    SpinTables T1[2] = {tables(ctx->sp[0], 1), tables(ctx->sp[1], 1)};
    const int X[2] = {T1[0].nh * T1[0].np, T1[1].nh * T1[1].np};
    const int NC[2] = {T1[0].N + T1[0].np, T1[1].N + T1[1].np};
    int rc;
    static const char* nm[2][8] = {{"F_a", "v0_a", "xx_a", "Lact_a", "Xic_a", "Lh1_a", "e1_a", "Y_a"},
                                   {"F_b", "v0_b", "xx_b", "Lact_b", "Xic_b", "Lh1_b", "e1_b", "Y_b"}};
    if (fp32) {
        size_t f = 0, a = 0;
        for (int s = 0; s < 2; ++s) {
            if (!fused(ctx, s)) f = std::max(f, sizeof(float) * 2 * T1[s].N * (size_t)G * NC[s]);
            a = std::max(a, sizeof(float) * a_rows(ctx, s) * (size_t)a_ld(ctx, s));
        }
        if (f && (rc = arena_get(ctx, "F32", f * cap, &E.F32))) return rc;
        if ((rc = arena_get(ctx, "AF_hi", a * cap, &E.Ah))) return rc;
        if ((rc = arena_get(ctx, "AF_lo", a * cap, &E.Al))) return rc;
    }
    for (int s = 0; s < 2; ++s) {
        const size_t xs = std::max(1, X[s]);
        if (!fp32 && (rc = arena_get(ctx, nm[s][0], sizeof(double2) * cap * T1[s].N * (size_t)G * NC[s], &E.F[s])))
            return rc;
        if ((rc = arena_get(ctx, nm[s][1], sizeof(double2) * cap * (size_t)G, &E.v0[s]))) return rc;
        if ((rc = arena_get(ctx, nm[s][2], sizeof(double2) * cap * (size_t)G, &E.xx[s]))) return rc;
        // FP64 rows of X entries, or FP32 rows of the pitch lam_pitch(X)
        const size_t ls = fp32 ? sizeof(float2) * lam_pitch((int)xs) : sizeof(double2) * xs;
        if ((rc = arena_get(ctx, nm[s][3], ls * cap * (size_t)G, &E.La[s]))) return rc;
        if ((rc = arena_get(ctx, nm[s][4], ls * cap * (size_t)G, &E.Xi[s]))) return rc;
        if ((rc = arena_get(ctx, nm[s][5], sizeof(double2) * cap * xs, &E.Lh1[s]))) return rc;
        if ((rc = arena_get(ctx, nm[s][6], sizeof(double2) * cap, &E.e1[s]))) return rc;
        if ((rc = arena_get(ctx, nm[s][7], sizeof(double2) * cap * xs, &E.Y[s]))) return rc;
    }
    if ((rc = arena_get(ctx, "K_aa", sizeof(double2) * cap * std::max(1, X[0] * X[0]), &E.Kaa))) return rc;
    if ((rc = arena_get(ctx, "K_bb", sizeof(double2) * cap * std::max(1, X[1] * X[1]), &E.Kbb))) return rc;
    if ((rc = arena_get(ctx, "K_ab", sizeof(double2) * cap * std::max(1, X[0] * X[1]), &E.Kab))) return rc;
    if ((rc = arena_get(ctx, "scal", sizeof(double2) * cap * 8, &E.scal))) return rc;
    if (fp32 && exact_ref_on(ctx)) {
        const int Mpad = oz_rows_padded(2 * cap);
        int kp = 0;
        for (int s = 0; s < 2; ++s) kp = std::max(kp, oz_k_padded(T1[s].N * (ctx->M - T1[s].N)));
        if ((rc = arena_get(ctx, "oz_A", (size_t)oz_slices() * Mpad * kp * 2, &E.ozA))) return rc;
        if ((rc = arena_get(ctx, "oz_ea", sizeof(int) * Mpad, &E.ozE))) return rc;
        static const char* np_[2] = {"oz_part_a", "oz_part_b"};
        static const char* nt_[2] = {"oz_t1_a", "oz_t1_b"};
        for (int s = 0; s < 2; ++s) {
            const int nparts = oz_parts_for(T1[s].N * (ctx->M - T1[s].N), G);
            if ((rc = arena_get(ctx, np_[s], sizeof(double2) * nparts * Mpad, &E.ozP[s]))) return rc;
            if ((rc = arena_get(ctx, nt_[s], sizeof(double) * 2 * cap * (size_t)G, &E.ozT[s]))) return rc;
        }
        if ((rc = arena_get(ctx, "v0w", sizeof(float2) * cap * (size_t)G, &E.v0w))) return rc;
    }
    if (fp32 && tensor_gram(ctx)) {
        static const char* ng_[2] = {"GT_a", "GT_b"};
        for (int s = 0; s < 2; ++s)
            if ((rc = arena_get(ctx, ng_[s], sizeof(float) * cap * 2 * (size_t)std::max(1, X[s]) * G, &E.GT[s])))
                return rc;
    }
    return MSD_OK;
}

// Energy part, first stage: the Cholesky contractions F_g = G L_g and their
// epilogue (v0, Lambda, Xi) per spin.
int en_fepi(msd_ctx* ctx, Chunk& c, EnWork& E, int nw, int cap, bool fp32, cudaStream_t st)
{
    const int M = ctx->M, G = ctx->n_chol;
    const TimerHook& th = ctx->hook;
    SpinTables T[2] = {tables(ctx->sp[0], cap), tables(ctx->sp[1], cap)};
    const int NC[2] = {T[0].N + T[0].np, T[1].N + T[1].np};
    // with the exact reference sums the FP32 exchange traces are not needed
    const bool exact = fp32 && exact_ref_on(ctx);
    if (exact && !ctx->oz_ok) return fail(ctx, MSD_ERR_STATE, "exact reference constants missing");
    const bool traces = !exact;
    for (int s = 0; s < 2; ++s) {
        const int N = T[s].N;
        if (fp32 && fused(ctx, s)) {
            th.begin("k_split_F", st);
            // without the traces the contraction also adds F0 (identity blocks)
            launch_split_complex_rows(nw, N, M - N, ctx->Kfp[s], c.Gr[s], M, ctx->d_virt[s], (float*)E.Ah,
                                      (float*)E.Al, st, ctx->fplan[s].RB, traces ? -1 : ctx->Kv8[s]);
            th.end(st);
            th.begin("tc_fepi", st);
            const int K = traces ? ctx->Kv8[s] : ctx->Kfp[s];
            const int g = tc_fepi_fused(T[s], ctx->fplan[s], nw, M, G, (float*)E.Ah, (float*)E.Al, ctx->LhP_hi[s],
                                        ctx->LhP_lo[s], ctx->Kfp[s], K, c.Gr[s], ctx->d_F0P[s], ctx->d_c0[s],
                                        ctx->d_x0[s], (double2*)E.v0[s], (double2*)E.xx[s], (float2*)E.La[s],
                                        (float2*)E.Xi[s], ctx->d_err, st, traces);
            th.end(st);
            if (g) return fail(ctx, MSD_ERR_CUDA, "fused tensor-core contraction launch failed (energy)");
        } else if (fp32) {
            th.begin("k_split_F", st);
            launch_split_complex_rows(nw, N, M - N, ctx->Kvp[s], c.Gr[s], M, ctx->d_virt[s], (float*)E.Ah,
                                      (float*)E.Al, st);
            th.end(st);
            th.begin("tc_gemm_F", st);
            const int g = tc_gemm_3xtf32({(float*)E.Ah, (float*)E.Al, ctx->Kvp[s]},
                                         {ctx->LhF_hi[s], ctx->LhF_lo[s], ctx->Kvp[s]}, 2 * nw * N, G * NC[s],
                                         ctx->Kvp[s], (float*)E.F32, (long long)G * NC[s], ctx->d_err, st, 1, 0,
                                         ctx->tc_bn);
            th.end(st);
            if (g) return fail(ctx, MSD_ERR_CUDA, "tensor-core GEMM launch failed (energy)");
            th.begin("k_fepi_f32", st);
            launch_fepi_f32(T[s], nw, M, G, (float*)E.F32, (long long)G * NC[s], c.Gr[s], ctx->d_F0T[s],
                            ctx->d_c0[s], ctx->d_x0[s], (double2*)E.v0[s], (double2*)E.xx[s], (float2*)E.La[s],
                            (float2*)E.Xi[s], st);
            th.end(st);
        } else {
            th.begin("k_gemm_F", st);
            launch_gemm_zd(nw * N, G * NC[s], M, c.Gr[s], M, ctx->sp[s].d_Lh, M, (double2*)E.F[s],
                           (long long)G * NC[s], st);
            th.end(st);
            th.begin("k_fepi", st);
            launch_fepi(T[s], nw, M, G, (double2*)E.F[s], (long long)G * NC[s], c.Gr[s], (double2*)E.v0[s],
                        (double2*)E.xx[s], (double2*)E.La[s], (double2*)E.Xi[s], st);
            th.end(st);
        }
        CKLAUNCH();
    }
    return MSD_OK;
}

// Energy part, second stage (reads only the reference inverse and the first
// stage's outputs): one-body terms, the exactly split reference sums, the
// per-walker sums of Lambda and Xi, the Gram matrices.
int en_rest(msd_ctx* ctx, Chunk& c, EnWork& E, int nw, int cap, bool fp32, cudaStream_t st)
{
    const int M = ctx->M, G = ctx->n_chol;
    const TimerHook& th = ctx->hook;
    SpinTables T[2] = {tables(ctx->sp[0], cap), tables(ctx->sp[1], cap)};
    const int X[2] = {T[0].nh * T[0].np, T[1].nh * T[1].np};
    const bool exact = fp32 && exact_ref_on(ctx);
    const bool traces = !exact;
    for (int s = 0; s < 2; ++s) {
        th.begin("k_onebody", st);
        launch_onebody(T[s], nw, M, ctx->d_h1 + (size_t)s * M * M, c.Gr[s], (double2*)E.e1[s],
                       (double2*)E.Lh1[s], st, exact && ctx->d_hJ ? ctx->d_hJ + (size_t)s * M * M : nullptr);
        th.end(st);
        CKLAUNCH();
    }
    RefSpin rs[2];
    if (exact) {
        // the reference-determinant sums exactly split on the tensor cores:
        // they replace the FP32 traces in scal[0..2], and their walker parts
        // t1_g of V0_g leave only the small part of sum_g V0_g Lambda_g to
        // the FP32 sum (the reference part C_g is in Lh1, the one-body term
        // of h + J)
        for (int s = 0; s < 2; ++s) {
            const OzConst& K = ctx->oz[s];
            th.begin("tc_ozaki", st);
            if (oz_spin(K, nw, M, c.Gr[s], ctx->d_virt[s], E.ozA, (int*)E.ozE, (double2*)E.ozP[s],
                        (double*)E.ozT[s], ctx->d_err, st))
                return fail(ctx, MSD_ERR_CUDA, "exact reference tensor-core launch failed");
            th.end(st);
            rs[s] = RefSpin{K.N, M, K.Kv, oz_parts(K.NB), oz_rows_padded(2 * nw), c.Gr[s], ctx->d_virt[s],
                            ctx->d_JJ[s], ctx->d_KK[s], (const double*)E.ozT[s], (const double2*)E.ozP[s],
                            ctx->oz_x0sum[s]};
        }
        th.begin("k_ref_reduce", st);
        launch_ref_reduce(nw, G, rs[0], rs[1], ctx->oz_C2sum, (double2*)E.scal, (float2*)E.v0w, st);
        th.end(st);
        CKLAUNCH();
    }
    th.begin("k_gamma_reduce", st);
    for (int s = 0; s < 2; ++s) {
        if (fp32)
            launch_gamma_reduce_f32(nw, X[s], G, s, (double2*)E.v0[0], (double2*)E.v0[1], (double2*)E.xx[s],
                                    (float2*)E.La[s], (float2*)E.Xi[s], (double2*)E.Lh1[s], (float2*)E.Y[s],
                                    (double2*)E.scal, st, traces, exact ? (const float2*)E.v0w : nullptr);
        else
            launch_gamma_reduce(nw, X[s], G, s, (double2*)E.v0[0], (double2*)E.v0[1], (double2*)E.xx[s],
                                (double2*)E.La[s], (double2*)E.Xi[s], (double2*)E.Lh1[s], E.Y[s], false,
                                (double2*)E.scal, st);
    }
    th.end(st);
    th.begin(fp32 && tensor_gram(ctx) ? "tc_gram" : "k_gram", st);
    if (fp32) {
        GramJobs jobs = {{{X[0], X[0], (float2*)E.La[0], (float2*)E.La[0], (float2*)E.Kaa},
                          {X[1], X[1], (float2*)E.La[1], (float2*)E.La[1], (float2*)E.Kbb},
                          {X[0], X[1], (float2*)E.La[0], (float2*)E.La[1], (float2*)E.Kab}}};
        if (tensor_gram(ctx)) {
            for (int s = 0; s < 2; ++s)
                launch_gram_transpose(nw, G, X[s], (float2*)E.La[s], (float*)E.GT[s], st);
            if (tc_gram(nw, G, X[0], X[1], (float*)E.GT[0], (float*)E.GT[1], (float2*)E.Kaa, (float2*)E.Kbb,
                        (float2*)E.Kab, ctx->d_err, st))
                return fail(ctx, MSD_ERR_CUDA, "tensor-core Gram launch failed");
        } else {
            launch_gram_f32(nw, G, jobs, 3, st);
        }
    } else {
        launch_gram(nw, X[0], X[0], G, (double2*)E.La[0], (double2*)E.La[0], E.Kaa, false, st);
        launch_gram(nw, X[1], X[1], G, (double2*)E.La[1], (double2*)E.La[1], E.Kbb, false, st);
        launch_gram(nw, X[0], X[1], G, (double2*)E.La[0], (double2*)E.La[1], E.Kab, false, st);
    }
    th.end(st);
    CKLAUNCH();
    return MSD_OK;
}

// Energy part, last stage (after the string weights): the per-determinant
// terms and the final reduction.
int en_terms(msd_ctx* ctx, Chunk& c, EnWork& E, int w0, int nw, int cap, bool fp32, double2* e_out,
             double2* ov_out, cudaStream_t st)
{
    const TimerHook& th = ctx->hook;
    SpinTables T[2] = {tables(ctx->sp[0], cap), tables(ctx->sp[1], cap)};
    int slot = c.nR;
    void* Kss[2] = {E.Kaa, E.Kbb};
    th.begin("k_string_energy", st);
    for (int s = 0; s < 2; ++s) {
        launch_string_energy(T[s], nw, c.wts[s], c.B[s], Kss[s], E.Y[s], fp32, c.part, c.nslot, slot, st);
        slot += string_energy_slots(T[s]);
    }
    th.end(st);
    CKLAUNCH();
    if (use_pair_y(ctx)) {
        th.begin("k_pair_y", st);
        launch_pair_y(T[0], T[1], nw, c.rf[0], c.rf[1], c.B[0], c.B[1], E.Kab, c.part, c.nslot, slot, st);
    } else {
        const bool runs = use_runs(ctx);
        th.begin(runs ? "k_pair_run" : "k_pair_cross", st);
        // the ratios in the working precision: FP32 copies in mixed mode
        const void* ra = fp32 ? (const void*)c.rf[0] : (const void*)c.r[0];
        const void* rb = fp32 ? (const void*)c.rf[1] : (const void*)c.r[1];
        launch_pair_cross(T[0], T[1], pair_tables(ctx->pairs), nw, ra, rb, c.B[0], c.B[1], E.Kab, fp32, c.part,
                          c.nslot, slot, st, runs);
    }
    th.end(st);
    CKLAUNCH();
    th.begin("k_final", st);
    launch_final(nw, c.part, c.nslot, c.nR, ctx->e0, (double2*)E.e1[0], (double2*)E.e1[1], (double2*)E.scal,
                 c.O0[0], c.O0[1], e_out + w0, ov_out ? ov_out + w0 : nullptr, st);
    th.end(st);
    CKLAUNCH();
    return MSD_OK;
}

int en_chunk(msd_ctx* ctx, Chunk& c, EnWork& E, int w0, int nw, int cap, bool fp32, double2* e_out,
             double2* ov_out, cudaStream_t st, bool defer_det = false)
{
    int rc;
    if ((rc = en_fepi(ctx, c, E, nw, cap, fp32, st))) return rc;
    if ((rc = en_rest(ctx, c, E, nw, cap, fp32, st))) return rc;
    if (defer_det) return MSD_OK;   // the batched kernel and the final sum follow
    return en_terms(ctx, c, E, w0, nw, cap, fp32, e_out, ov_out, st);
}

// Overlap (always), force bias (vbias != NULL) and local energy (e_loc !=
// NULL) of n_w walkers, sharing the reference inverse, string minors and
// CI weights between the last two.
struct Deferred {
    Chunk c;
    EnWork E;
    int cap = 0;
};

int evaluate_impl(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* ovlp, double* vbias,
                  double* e_loc, void* stream, Deferred* defer)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    if (n_w == 0) return MSD_OK;
    const bool fp32 = ctx->prec == MSD_MIXED;
    if (fp32 && (rc = prepare_mixed(ctx, st))) return rc;
    if (fp32 && e_loc && exact_ref_on(ctx) && (rc = prepare_exact_ref(ctx, st))) return rc;
    Staged in;
    if ((rc = stage_inputs(ctx, n_w, phi_a, phi_b, st, in, true))) return rc;
    // the caller's beta buffer is read by the copy stream: it has been read
    // completely before this call returns, on every path
    struct CopyDone {
        cudaEvent_t e;
        ~CopyDone() { if (e) cudaEventSynchronize(e); }
    } copy_done{in.b_ready};
    Out o_v, o_e, o_ov;
    if ((rc = stage_output(ctx, "out_vbias", vbias, (size_t)n_w * ctx->n_chol, o_v))) return rc;
    if ((rc = stage_output(ctx, "out_eloc", e_loc, n_w, o_e))) return rc;
    if ((rc = stage_output(ctx, "out_ovlp", ovlp, n_w, o_ov))) return rc;
    const bool want_v = vbias != nullptr, want_e = e_loc != nullptr;
    const int nR = weights_blocks(tables(ctx->sp[0], 1));
    const int nslot = nR + (want_e ? energy_slots(ctx) : 0);
    size_t per = overlap_bytes_per_walker(ctx, true, nslot);
    if (want_v) per += fb_bytes_per_walker(ctx, fp32);
    if (want_e) per += en_bytes_per_walker(ctx, fp32);
    const int cap = chunk_for(ctx, per, n_w);
    Chunk c;
    if ((rc = chunk_alloc(ctx, cap, true, nslot, c))) return rc;
    FbWork f;
    EnWork E;
    if (want_v && (rc = fb_alloc(ctx, cap, fp32, f))) return rc;
    if (want_e && (rc = en_alloc(ctx, cap, fp32, E))) return rc;
    if (defer && (cap < n_w || !want_e || in.host_any || o_e.host || o_v.host || o_ov.host))
        return fail(ctx, MSD_ERR_SHAPE, "batched evaluation needs device buffers, the energy output and all "
                                        "walkers in one chunk (%d walkers, %d fit)", n_w, cap);
    // mixed energy: the second energy stage on a side stream, concurrent
    // with the strings and weights (FP64-bound) on this stream; then the force
    // bias on the side stream, concurrent with the per-determinant terms
    const bool side = fp32 && want_e && !defer && ctx->overlap;
    if (side && !ctx->side_st) {
        // the highest stream priority: the second stage's blocks are placed
        // first and it finishes early instead of trailing into the weights
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (cudaStreamCreateWithPriority(&ctx->side_st, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_rest, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_w, cudaEventDisableTiming) != cudaSuccess)
            return fail(ctx, MSD_ERR_CUDA, "side stream could not be created");
    }
    // every return after a fork first makes this stream wait for the side stream
    struct Join {
        cudaStream_t st = nullptr, side = nullptr;
        cudaEvent_t ev = nullptr;
        void now() {
            if (side) { cudaEventRecord(ev, side); cudaStreamWaitEvent(st, ev, 0); side = nullptr; }
        }
        ~Join() { now(); }
    } join;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        if (side) {
            if ((rc = run_refs(ctx, in, w0, nw, cap, c, st))) return rc;
            if ((rc = en_fepi(ctx, c, E, nw, cap, fp32, st))) return rc;
            CK(cudaEventRecord(ctx->ev_fork, st));
            CK(cudaStreamWaitEvent(ctx->side_st, ctx->ev_fork, 0));
            join.st = st;
            join.side = ctx->side_st;
            join.ev = ctx->ev_join;
            if ((rc = en_rest(ctx, c, E, nw, cap, fp32, ctx->side_st))) return rc;
            CK(cudaEventRecord(ctx->ev_rest, ctx->side_st));
            if ((rc = run_strings_weights(ctx, nw, cap, c, true, fp32, st))) return rc;
            // the force bias (cofactors, G_T, contraction) follows the weights
            // on the second stream, beside the per-determinant terms here
            if (want_v) {
                CK(cudaEventRecord(ctx->ev_w, st));
                CK(cudaStreamWaitEvent(ctx->side_st, ctx->ev_w, 0));
                if ((rc = fb_chunk(ctx, c, f, w0, nw, cap, fp32, o_v.dev, nullptr, ctx->side_st))) return rc;
            }
            CK(cudaStreamWaitEvent(st, ctx->ev_rest, 0));
            if ((rc = en_terms(ctx, c, E, w0, nw, cap, fp32, o_e.dev, o_ov.dev, st))) return rc;
            join.now();   // before the next chunk's reference inverse and before the outputs
            CKLAUNCH();
            continue;
        }
        if ((rc = run_overlap_part(ctx, in, w0, nw, cap, c, true, fp32, st))) return rc;
        if (want_v && (rc = fb_chunk(ctx, c, f, w0, nw, cap, fp32, o_v.dev, want_e ? nullptr : o_ov.dev, st)))
            return rc;
        if (want_e && (rc = en_chunk(ctx, c, E, w0, nw, cap, fp32, o_e.dev, o_ov.dev, st, defer != nullptr)))
            return rc;
    }
    if (defer) {
        defer->c = c;
        defer->E = E;
        defer->cap = cap;
        CKLAUNCH();
        return MSD_OK;
    }
    return finish(ctx, st, {&o_v, &o_e, &o_ov}, in.host_any);
}

int evaluate(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* ovlp, double* vbias,
             double* e_loc, void* stream)
{
    return evaluate_impl(ctx, n_w, phi_a, phi_b, ovlp, vbias, e_loc, stream, nullptr);
}

// Mixed one-body density matrix G_T per walker and spin: the force-bias
// path up to G_T (cofactor accumulation, rank-k update), written out as full
// matrices.
int rdm1(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* rdm, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    if (n_w == 0) return MSD_OK;
    if (!rdm) return fail(ctx, MSD_ERR_ARG, "no output");
    const bool fp32 = ctx->prec == MSD_MIXED;
    const int M = ctx->M;
    Staged in;
    if ((rc = stage_inputs(ctx, n_w, phi_a, phi_b, st, in))) return rc;
    Out o_r;
    if ((rc = stage_output(ctx, "out_rdm", rdm, (size_t)n_w * 2 * M * M, o_r))) return rc;
    CK(cudaMemsetAsync(o_r.dev, 0, o_r.bytes, st));
    const int nR = weights_blocks(tables(ctx->sp[0], 1));
    const int cap = chunk_for(ctx, overlap_bytes_per_walker(ctx, true, nR) + fb_bytes_per_walker(ctx, false), n_w);
    Chunk c;
    FbWork f;
    if ((rc = chunk_alloc(ctx, cap, true, nR, c))) return rc;
    if ((rc = fb_alloc(ctx, cap, false, f))) return rc;
    const TimerHook& th = ctx->hook;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        if ((rc = run_overlap_part(ctx, in, w0, nw, cap, c, true, fp32, st))) return rc;
        th.begin("k_sum_slots", st);
        launch_sum_slots(nw, c.part, c.nslot, 0, c.nR, (double2*)f.Rs, c.O0[0], c.O0[1], nullptr, st);
        th.end(st);
        th.begin("k_cmat", st);
        launch_cmat(tables(ctx->sp[0], cap), tables(ctx->sp[1], cap), nw, c.wts[0], c.wts[1], c.B[0], c.B[1], fp32,
                    (double2*)f.Cm[0], (double2*)f.Cm[1], st);
        th.end(st);
        long long off = 0;
        for (int s = 0; s < 2; ++s) {
            const SpinTables T = tables(ctx->sp[s], cap);
            th.begin("k_gt", st);
            launch_gt(T, nw, M, c.Gr[s], (double2*)f.Cm[s], (double2*)f.Rs, (double2*)f.GT, ctx->Kd, off, false, st);
            th.end(st);
            th.begin("k_rdm_scatter", st);
            launch_rdm_scatter(T, nw, M, (const double2*)f.GT, ctx->Kd, off, s, o_r.dev + (size_t)w0 * 2 * M * M, st);
            th.end(st);
            off += (long long)(T.N + T.np) * M;
        }
        CKLAUNCH();
    }
    return finish(ctx, st, {&o_r}, in.host_any);
}

// E_I for sampled (walker, determinant) pairs: the energy path up to the
// per-walker Gram matrices, then one thread per pair.
int det_energies(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, int n_pairs,
                 const int32_t* w_idx, const int32_t* det_idx, double* e_det, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    if (n_pairs < 0 || (n_pairs > 0 && (!w_idx || !det_idx || !e_det)))
        return fail(ctx, MSD_ERR_ARG, "bad pair arguments");
    if (n_pairs == 0) return MSD_OK;
    if (is_device_ptr(w_idx) || is_device_ptr(det_idx))
        return fail(ctx, MSD_ERR_ARG, "w_idx and det_idx must be host arrays");
    const PairHost& P = ctx->pairs;
    std::vector<int> pos(P.n_det);
    for (int i = 0; i < P.n_det; ++i) pos[P.det_index[i]] = i;
    std::vector<DetRec> recs(n_pairs);
    for (int i = 0; i < n_pairs; ++i) {
        if (w_idx[i] < 0 || w_idx[i] >= n_w || det_idx[i] < 0 || det_idx[i] >= P.n_det)
            return fail(ctx, MSD_ERR_ARG, "pair %d: walker %d or determinant %d out of range", i, w_idx[i],
                        det_idx[i]);
        const int at = pos[det_idx[i]], a = P.a[at], b = P.b[at];
        recs[i] = DetRec{w_idx[i], a, b, ctx->sp[0].str_k[a], ctx->sp[1].str_k[b]};
    }
    const bool fp32 = ctx->prec == MSD_MIXED;
    if (fp32 && (rc = prepare_mixed(ctx, st))) return rc;
    if (fp32 && exact_ref_on(ctx) && (rc = prepare_exact_ref(ctx, st))) return rc;
    Staged in;
    if ((rc = stage_inputs(ctx, n_w, phi_a, phi_b, st, in))) return rc;
    Out o_e;
    if ((rc = stage_output(ctx, "out_edet", e_det, n_pairs, o_e))) return rc;
    void* d_rec;
    if ((rc = arena_get(ctx, "det_rec", sizeof(DetRec) * n_pairs, &d_rec))) return rc;
    CK(cudaMemcpyAsync(d_rec, recs.data(), sizeof(DetRec) * n_pairs, cudaMemcpyHostToDevice, st));
    const int nR = weights_blocks(tables(ctx->sp[0], 1));
    const size_t per = overlap_bytes_per_walker(ctx, true, nR) + en_bytes_per_walker(ctx, fp32);
    const int cap = chunk_for(ctx, per, n_w);
    Chunk c;
    EnWork E;
    if ((rc = chunk_alloc(ctx, cap, true, nR, c))) return rc;
    if ((rc = en_alloc(ctx, cap, fp32, E))) return rc;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        if ((rc = run_overlap_part(ctx, in, w0, nw, cap, c, true, fp32, st))) return rc;
        if ((rc = en_chunk(ctx, c, E, w0, nw, cap, fp32, nullptr, nullptr, st, true))) return rc;
        launch_det_energy(n_pairs, (const DetRec*)d_rec, w0, nw, tables(ctx->sp[0], cap), tables(ctx->sp[1], cap),
                          c.B[0], c.B[1], E.Kaa, E.Kbb, E.Kab, E.Y[0], E.Y[1], (const double2*)E.scal,
                          (const double2*)E.e1[0], (const double2*)E.e1[1], ctx->e0, fp32, o_e.dev, st);
        CKLAUNCH();
    }
    rc = finish(ctx, st, {&o_e}, in.host_any);
    CK(cudaStreamSynchronize(st));   // recs is a host vector
    return rc;
}

// ------------------------------------------------------------ propagation
void free_prop(msd_ctx* ctx)
{
    cudaFree(ctx->d_Lt);
    ctx->d_Lt = nullptr;
    for (int s = 0; s < 2; ++s) { cudaFree(ctx->d_E[s]); ctx->d_E[s] = nullptr; }
    ctx->h_corr.clear();
    ctx->prop_dt = -1.0;
}

// exp(A) of a real M x M matrix: scaling to norm <= 1/4, Taylor series to
// order 18 (remainder below 1e-17 relative), then squaring.
std::vector<double> expm_host(const std::vector<double>& A, int M)
{
    double nrm = 0;
    for (int i = 0; i < M; ++i) {
        double r = 0;
        for (int j = 0; j < M; ++j) r += std::fabs(A[(size_t)i * M + j]);
        nrm = std::max(nrm, r);
    }
    int sq = 0;
    while (nrm > 0.25) { nrm *= 0.5; ++sq; }
    const double scale = std::ldexp(1.0, -sq);
    std::vector<double> B(A.size()), X((size_t)M * M, 0.0), T((size_t)M * M, 0.0), tmp((size_t)M * M);
    for (size_t e = 0; e < A.size(); ++e) B[e] = A[e] * scale;
    for (int i = 0; i < M; ++i) X[(size_t)i * M + i] = T[(size_t)i * M + i] = 1.0;
    auto mul = [M](const std::vector<double>& a, const std::vector<double>& b, std::vector<double>& c) {
        std::fill(c.begin(), c.end(), 0.0);
        for (int i = 0; i < M; ++i)
            for (int k = 0; k < M; ++k) {
                const double aik = a[(size_t)i * M + k];
                for (int j = 0; j < M; ++j) c[(size_t)i * M + j] += aik * b[(size_t)k * M + j];
            }
    };
    for (int k = 1; k <= 18; ++k) {
        mul(T, B, tmp);
        for (size_t e = 0; e < tmp.size(); ++e) T[e] = tmp[e] / k;
        for (size_t e = 0; e < X.size(); ++e) X[e] += T[e];
    }
    for (int i = 0; i < sq; ++i) {
        mul(X, X, tmp);
        X.swap(tmp);
    }
    return X;
}

// Transposed Cholesky vectors and sum_g L_g L_g once per Hamiltonian;
// E_s = exp(-dt h'_s / 2), h'_s = h_s - 1/2 sum_g L_g L_g, once per dt.
int prepare_prop(msd_ctx* ctx, double dt, cudaStream_t st)
{
    const int M = ctx->M, G = ctx->n_chol;
    if (!ctx->d_Lt) {
        std::vector<double> lt((size_t)M * M * G);
        for (int g = 0; g < G; ++g)
            for (size_t pq = 0; pq < (size_t)M * M; ++pq) lt[pq * G + g] = ctx->h_L[(size_t)g * M * M + pq];
        int rc = upload(ctx, &ctx->d_Lt, lt);
        if (rc) return rc;
        double* d_corr = nullptr;
        CK(cudaMalloc(&d_corr, sizeof(double) * M * M));
        launch_sum_LL(M, G, ctx->d_Lt, d_corr, st);
        ctx->h_corr.resize((size_t)M * M);
        cudaError_t e = cudaMemcpyAsync(ctx->h_corr.data(), d_corr, sizeof(double) * M * M, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaFree(d_corr);
        if (e != cudaSuccess) return fail(ctx, MSD_ERR_CUDA, "sum of L_g L_g failed: %s", cudaGetErrorString(e));
        ctx->prop_dt = -1.0;
    }
    if (ctx->prop_dt != dt) {
        for (int s = 0; s < 2; ++s) {
            std::vector<double> a((size_t)M * M);
            for (size_t e = 0; e < a.size(); ++e)
                a[e] = -0.5 * dt * (ctx->h_h1[(size_t)s * M * M + e] - 0.5 * ctx->h_corr[e]);
            int rc = upload(ctx, &ctx->d_E[s], expm_host(a, M));
            if (rc) return rc;
        }
        ctx->prop_dt = dt;
    }
    return MSD_OK;
}

int propagate(msd_ctx* ctx, int n_w, double* phi_a, double* phi_b, double* weights, const double* x, double dt,
              int order, int orthonormalize, double* ratio, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    if (n_w == 0) return MSD_OK;
    if (!(dt > 0) || order < 1 || order > 16)
        return fail(ctx, MSD_ERR_ARG, "need dt > 0 and 1 <= taylor_order <= 16 (got %g, %d)", dt, order);
    if (!weights || !x) return fail(ctx, MSD_ERR_ARG, "weights and x are required");
    if (!is_device_ptr(phi_a) || !is_device_ptr(phi_b) || !is_device_ptr(weights) || !is_device_ptr(x) ||
        (ratio && !is_device_ptr(ratio)))
        return fail(ctx, MSD_ERR_ARG, "msd_propagate takes device pointers only");
    const int M = ctx->M, G = ctx->n_chol, Nm = std::max(ctx->n[0], ctx->n[1]);
    if (sizeof(double2) * (size_t)M * Nm > 200 * 1024)
        return fail(ctx, MSD_ERR_SHAPE, "M x N = %d x %d walker blocks exceed the kernels' shared memory", M, Nm);
    if ((rc = prepare_prop(ctx, dt, st))) return rc;
    void *o0, *o1, *ex, *vb, *cf;
    if ((rc = arena_get(ctx, "pr_o0", sizeof(double2) * n_w, &o0))) return rc;
    if ((rc = arena_get(ctx, "pr_o1", sizeof(double2) * n_w, &o1))) return rc;
    if ((rc = arena_get(ctx, "pr_expo", sizeof(double2) * n_w, &ex))) return rc;
    if ((rc = arena_get(ctx, "pr_vb", sizeof(double2) * (size_t)n_w * G, &vb))) return rc;
    if ((rc = arena_get(ctx, "pr_c", sizeof(double2) * (size_t)n_w * G, &cf))) return rc;
    // Eq. 7: overlap and mixed <L_g> of the current walkers
    if ((rc = evaluate_impl(ctx, n_w, phi_a, phi_b, (double*)o0, (double*)vb, nullptr, stream, nullptr))) return rc;
    const TimerHook& th = ctx->hook;
    th.begin("k_prop_coef", st);
    launch_prop_coef(n_w, G, dt, x, (const double2*)vb, (double2*)cf, (double2*)ex, st);
    th.end(st);
    // B(x - xbar) on walker chunks: V, half steps, Taylor series
    const size_t per = sizeof(double2) * ((size_t)M * M + 3 * (size_t)M * Nm);
    const int cap = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_w, ctx->ws_limit / 2 / per));
    void *V, *t0, *t1, *ac;
    if ((rc = arena_get(ctx, "pr_V", sizeof(double2) * (size_t)cap * M * M, &V))) return rc;
    if ((rc = arena_get(ctx, "pr_t0", sizeof(double2) * (size_t)cap * M * Nm, &t0))) return rc;
    if ((rc = arena_get(ctx, "pr_t1", sizeof(double2) * (size_t)cap * M * Nm, &t1))) return rc;
    if ((rc = arena_get(ctx, "pr_acc", sizeof(double2) * (size_t)cap * M * Nm, &ac))) return rc;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        th.begin("k_gemm_V", st);
        launch_gemm_zd(nw, M * M, G, (const double2*)cf + (size_t)w0 * G, G, ctx->d_Lt, G, (double2*)V,
                       (long long)M * M, st);
        th.end(st);
        for (int s = 0; s < 2; ++s) {
            const int N = ctx->n[s];
            double2* phi = (double2*)(s ? phi_b : phi_a) + (size_t)w0 * M * N;
            double2 *cur = (double2*)t0, *nxt = (double2*)t1, *acc = (double2*)ac;
            th.begin("k_apply_rows", st);
            int g = launch_apply_rows(nw, M, N, nullptr, 0, ctx->d_E[s], phi, cur, nullptr, 1.0, st);
            CK(cudaMemcpyAsync(acc, cur, sizeof(double2) * (size_t)nw * M * N, cudaMemcpyDeviceToDevice, st));
            for (int k = 1; k <= order && !g; ++k) {
                g = launch_apply_rows(nw, M, N, (const double2*)V, (long long)M * M, nullptr, cur, nxt, acc,
                                      1.0 / k, st);
                std::swap(cur, nxt);
            }
            if (!g) g = launch_apply_rows(nw, M, N, nullptr, 0, ctx->d_E[s], acc, phi, nullptr, 1.0, st);
            th.end(st);
            if (g) return fail(ctx, MSD_ERR_SHAPE, "walker block too large for the propagation kernels");
            CKLAUNCH();
        }
    }
    // Eq. 8: overlap of the propagated walkers; Eq. 10-11: weights
    if ((rc = msd_overlap(ctx, n_w, phi_a, phi_b, (double*)o1, nullptr, stream))) return rc;
    th.begin("k_prop_weight", st);
    launch_prop_weight(n_w, (const double2*)o0, (const double2*)o1, (const double2*)ex, weights, (double2*)ratio,
                       st);
    th.end(st);
    if (orthonormalize) {
        th.begin("k_qr_mgs", st);
        for (int s = 0; s < 2; ++s)
            if (launch_qr_mgs(n_w, M, ctx->n[s], (double2*)(s ? phi_b : phi_a), ctx->d_err, st))
                return fail(ctx, MSD_ERR_SHAPE, "walker block too large for the QR kernel");
        th.end(st);
    }
    return finish(ctx, st, {}, false);
}

}  // namespace

// ========================================================================
extern "C" {

int msd_create(msd_ctx** out, int M, int n_alpha, int n_beta, int precision, int device)
{
    msd_ctx* ctx = nullptr;
    if (!out) return fail(nullptr, MSD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (M <= 0 || n_alpha <= 0 || n_beta <= 0 || n_alpha > M || n_beta > M)
        return fail(nullptr, MSD_ERR_ARG, "invalid sizes M=%d n_alpha=%d n_beta=%d", M, n_alpha, n_beta);
    if (n_alpha > MSD_NMAX || n_beta > MSD_NMAX)
        return fail(nullptr, MSD_ERR_SHAPE, "at most %d electrons per spin", MSD_NMAX);
    if (precision != MSD_FP64 && precision != MSD_MIXED)
        return fail(nullptr, MSD_ERR_ARG, "unknown precision %d", precision);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, MSD_ERR_CUDA, "CUDA device %d not available", device);
    }
    if (cudaSetDevice(device) != cudaSuccess) return fail(nullptr, MSD_ERR_CUDA, "cudaSetDevice failed");
    ctx = new msd_ctx();
    ctx->device = device; ctx->M = M; ctx->n[0] = n_alpha; ctx->n[1] = n_beta; ctx->prec = precision;
    if (msd_err_word_alloc(&ctx->d_err) != 0 ||
        cudaMallocHost(&ctx->h_err, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->d_err);
        delete ctx;
        return fail(nullptr, MSD_ERR_NOMEM, "allocation failed");
    }
    ctx->hook.self = ctx;
    *out = ctx;
    return MSD_OK;
}

void msd_destroy(msd_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->arena) cudaFree(kv.second.p);
    for (int s = 0; s < 2; ++s) free_spin(ctx->sp[s]);
    cudaFree(ctx->pairs.d_a); cudaFree(ctx->pairs.d_b); cudaFree(ctx->pairs.d_c); cudaFree(ctx->pairs.d_runs);
    cudaFree(ctx->pairs.d_det_index); cudaFree(ctx->pairs.d_cf);
    free_mixed(ctx);
    free_prop(ctx);
    cudaFree(ctx->d_h1); cudaFree(ctx->d_Lcat); cudaFree(ctx->d_err);
    cudaFreeHost(ctx->h_err);
    for (auto& p : ctx->pending) { ctx->ev_pool.push_back(p.a); ctx->ev_pool.push_back(p.b); }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
    if (ctx->side_st) cudaStreamDestroy(ctx->side_st);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_rest) cudaEventDestroy(ctx->ev_rest);
    if (ctx->ev_w) cudaEventDestroy(ctx->ev_w);
    if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
    if (ctx->ev_b) cudaEventDestroy(ctx->ev_b);
    delete ctx;
}

const char* msd_last_error(const msd_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int msd_set_hamiltonian(msd_ctx* ctx, const double* h1, double e0, int n_chol, const double* L)
{
    if (!ctx) return MSD_ERR_ARG;
    if (!h1 || !L || n_chol <= 0) return fail(ctx, MSD_ERR_ARG, "h1, L and n_chol > 0 are required");
    CK(cudaSetDevice(ctx->device));
    const int M = ctx->M;
    ctx->h_h1.assign(h1, h1 + (size_t)2 * M * M);
    ctx->h_L.assign(L, L + (size_t)n_chol * M * M);
    ctx->n_chol = n_chol;
    ctx->e0 = e0;
    int rc = upload(ctx, &ctx->d_h1, ctx->h_h1);
    if (rc) return rc;
    free_prop(ctx);
    ctx->have_ham = true;
    return build_half_rotated(ctx);
}

int msd_set_trial(msd_ctx* ctx, int n_det, const double* coeff, const int32_t* occ_a,
                  const int32_t* occ_b)
{
    if (!ctx) return MSD_ERR_ARG;
    if (n_det <= 0 || !coeff || !occ_a || !occ_b) return fail(ctx, MSD_ERR_ARG, "empty trial");
    CK(cudaSetDevice(ctx->device));
    ctx->have_trial = false;
    std::vector<int> sid[2];
    const int32_t* occ[2] = {occ_a, occ_b};
    for (int s = 0; s < 2; ++s) {
        free_spin(ctx->sp[s]);
        int rc = build_spin(ctx, s, occ[s], n_det, sid[s]);
        if (rc) return rc;
    }
    // determinants ordered by (level_a, level_b, a, b)
    PairHost& P = ctx->pairs;
    cudaFree(P.d_a); cudaFree(P.d_b); cudaFree(P.d_c); cudaFree(P.d_det_index); cudaFree(P.d_cf);
    cudaFree(P.d_runs);
    P = PairHost{};
    P.n_det = n_det;
    std::vector<int> order(n_det);
    for (int i = 0; i < n_det; ++i) order[i] = i;
    auto lv = [&](int s, int I) { return ctx->sp[s].str_k[sid[s][I]]; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int bx = lv(0, x) * (MSD_KMAX + 1) + lv(1, x), by = lv(0, y) * (MSD_KMAX + 1) + lv(1, y);
        if (bx != by) return bx < by;
        if (sid[0][x] != sid[0][y]) return sid[0][x] < sid[0][y];
        return sid[1][x] < sid[1][y];
    });
    for (int i = 0; i < n_det; ++i) {
        const int I = order[i];
        P.a.push_back(sid[0][I]); P.b.push_back(sid[1][I]);
        P.c.push_back(coeff[I]); P.det_index.push_back(I);
        P.bucket[lv(0, I) * (MSD_KMAX + 1) + lv(1, I) + 1]++;
    }
    for (int i = 1; i < (MSD_KMAX + 1) * (MSD_KMAX + 1) + 1; ++i) P.bucket[i] += P.bucket[i - 1];
    // runs form of the opposite-spin term: per bucket, project the string
    // that the bucket's determinants share most (alpha: the order above
    // already groups them; beta: the bucket is re-sorted by (b, a)), unless
    // its determinants are too few per string to pay for the projection.
    // Costs in warp instructions per walker (shared-memory gathers at random
    // addresses ~3.5, a projection entry over a 32-lane chunk ~1.5, a
    // (determinant, entry) pair ~8/32).
    {
        const int Xs[2] = {ctx->sp[0].nh * ctx->sp[0].np, ctx->sp[1].nh * ctx->sp[1].np};
        // the runs kernel's shared memory in FP64 must fit (else no runs)
        SpinTables t0 = tables(ctx->sp[0], 1), t1 = tables(ctx->sp[1], 1);
        const bool runs_fit = pair_run_smem(t0, t1, false) <= 227 * 1024;
        P.runs.clear();
        for (int idx = 0; idx < (MSD_KMAX + 1) * (MSD_KMAX + 1); ++idx) {
            const int ka = idx / (MSD_KMAX + 1), kb = idx % (MSD_KMAX + 1);
            const int lo = P.bucket[idx], hi = P.bucket[idx + 1];
            P.run_off[idx] = (int)P.runs.size();
            P.run_side[idx] = 0;
            if (ka == 0 || kb == 0 || hi <= lo || !runs_fit) continue;
            const double n = hi - lo, qa = (Xs[0] + 31) / 32, qb = (Xs[1] + 31) / 32;
            int na = 1;
            for (int i = lo + 1; i < hi; ++i) na += P.a[i] != P.a[i - 1];
            std::vector<int> bs(P.b.begin() + lo, P.b.begin() + hi);
            std::sort(bs.begin(), bs.end());
            const int nb = (int)(std::unique(bs.begin(), bs.end()) - bs.begin());
            const double kka = ka * ka, kkb = kb * kb;
            const double direct = n * (3.5 * kka * kkb + 2.0 * (kka + kkb)) / 32.0;
            const double proj_a = na * (1.5 * kka * qb + kka + 4.0) + n * kkb * 8.0 / 32.0;
            const double proj_b = nb * (1.5 * kkb * qa + kkb + 4.0) + n * kka * 8.0 / 32.0;
            // measured: with ~10-17 determinants per string (the iron-sulfur
            // trial) the projection only breaks even, with ~80 (the 1e6
            // copper-oxo trial) the runs take 0.46 of the double sum's time
            int side = 0;
            const double per_a = n / na, per_b = n / nb;
            if (proj_a < direct && proj_a <= proj_b && per_a >= 24.0) side = 1;
            else if (proj_b < direct && per_b >= 24.0) side = 2;
            P.run_side[idx] = side;
            if (side == 2) {
                std::vector<int> perm(hi - lo);
                for (int i = 0; i < hi - lo; ++i) perm[i] = lo + i;
                std::stable_sort(perm.begin(), perm.end(), [&](int x, int y) {
                    if (P.b[x] != P.b[y]) return P.b[x] < P.b[y];
                    return P.a[x] < P.a[y];
                });
                std::vector<int> a2(hi - lo), b2(hi - lo), d2(hi - lo);
                std::vector<double> c2(hi - lo);
                for (int i = 0; i < hi - lo; ++i) {
                    a2[i] = P.a[perm[i]]; b2[i] = P.b[perm[i]];
                    c2[i] = P.c[perm[i]]; d2[i] = P.det_index[perm[i]];
                }
                std::copy(a2.begin(), a2.end(), P.a.begin() + lo);
                std::copy(b2.begin(), b2.end(), P.b.begin() + lo);
                std::copy(c2.begin(), c2.end(), P.c.begin() + lo);
                std::copy(d2.begin(), d2.end(), P.det_index.begin() + lo);
            }
            if (side) {
                const std::vector<int>& key = side == 1 ? P.a : P.b;
                for (int i = lo; i < hi; ++i)
                    if (i == lo || key[i] != key[i - 1]) P.runs.push_back(i);
            }
        }
        P.run_off[(MSD_KMAX + 1) * (MSD_KMAX + 1)] = (int)P.runs.size();
    }
    // CSR per spin: determinants containing each string
    for (int s = 0; s < 2; ++s) {
        SpinHost& S = ctx->sp[s];
        S.csr_off.assign(S.n_str + 1, 0);
        for (int I = 0; I < n_det; ++I) S.csr_off[sid[s][I] + 1]++;
        for (int i = 0; i < S.n_str; ++i) S.csr_off[i + 1] += S.csr_off[i];
        std::vector<int> fill(S.csr_off.begin(), S.csr_off.end() - 1);
        S.csr_other.assign(n_det, 0);
        S.csr_c.assign(n_det, 0);
        for (int i = 0; i < n_det; ++i) {   // in pair order: deterministic sums
            const int I = order[i];
            const int e = fill[sid[s][I]]++;
            S.csr_other[e] = sid[1 - s][I];
            S.csr_c[e] = coeff[I];
        }
        int rc = upload_spin(ctx, S);
        if (rc) return rc;
    }
    // cost model for the two forms of the opposite-spin term (per walker;
    // unit costs measured on GB300 with the iron-sulfur-shaped 1.2e5- and
    // the copper-oxo-shaped 1e6-determinant trials): per beta string
    // ~1.0 per (entry x 32-lane x slot) of Y_b plus ~3.7 per alpha entry of
    // each determinant, per determinant ~1.1 per k_a^2 k_b^2 gather
    {
        const SpinHost& Sa = ctx->sp[0];
        const SpinHost& Sb = ctx->sp[1];
        const double xpp = 32.0 * ((Sa.nh * Sa.np + 31) / 32) + 1.0;
        double cost_y = 0.0, cost_d = 0.0;
        for (int k = 1; k <= MSD_KMAX; ++k) cost_y += xpp * k * k * (Sb.bucket[k + 1] - Sb.bucket[k]);
        for (int I = 0; I < n_det; ++I) {
            const double ka = lv(0, I), kb = lv(1, I);
            if (ka > 0 && kb > 0) {
                cost_y += 3.7 * ka * ka;
                cost_d += 1.1 * ka * ka * kb * kb;
            }
        }
        ctx->pair_y_auto = cost_y < cost_d;
        ctx->chunk = 0;
    }
    int rc;
    if ((rc = upload(ctx, &P.d_a, P.a))) return rc;
    if ((rc = upload(ctx, &P.d_b, P.b))) return rc;
    if ((rc = upload(ctx, &P.d_c, P.c))) return rc;
    {
        std::vector<float> cf(P.c.begin(), P.c.end());
        if ((rc = upload(ctx, &P.d_cf, cf))) return rc;
    }
    if ((rc = upload(ctx, &P.d_det_index, P.det_index))) return rc;
    {
        std::vector<int> runs = P.runs;
        if (runs.empty()) runs.push_back(0);
        if ((rc = upload(ctx, &P.d_runs, runs))) return rc;
    }
    // shared-memory needs of the energy kernels
    for (int s = 0; s < 2; ++s) {
        const SpinTables t = tables(ctx->sp[s], 1);
        if (fepi_smem(t) > 200 * 1024 || string_energy_smem(t, false) > 220 * 1024)
            return fail(ctx, MSD_ERR_SHAPE, "spin %d: N=%d, active block %dx%d too large", s, t.N, t.nh, t.np);
    }
    ctx->have_trial = true;
    return build_half_rotated(ctx);
}

int msd_set_precision(msd_ctx* ctx, int precision)
{
    if (!ctx) return MSD_ERR_ARG;
    if (precision != MSD_FP64 && precision != MSD_MIXED)
        return fail(ctx, MSD_ERR_ARG, "unknown precision %d", precision);
    if (ctx->prec != precision) ctx->gen++;
    ctx->prec = precision;
    return MSD_OK;
}

int msd_overlap(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* ovlp,
                double* ratio_sum, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    if (n_w == 0) return MSD_OK;
    if (!ovlp && !ratio_sum) return fail(ctx, MSD_ERR_ARG, "no output requested");
    Staged in;
    if ((rc = stage_inputs(ctx, n_w, phi_a, phi_b, st, in))) return rc;
    Out o_ov, o_rs;
    if ((rc = stage_output(ctx, "out_ovlp", ovlp, n_w, o_ov))) return rc;
    if ((rc = stage_output(ctx, "out_rsum", ratio_sum, n_w, o_rs))) return rc;
    const int nR = weights_blocks(tables(ctx->sp[0], 1));
    const int cap = chunk_for(ctx, overlap_bytes_per_walker(ctx, false, nR), n_w);
    Chunk c;
    if ((rc = chunk_alloc(ctx, cap, false, nR, c))) return rc;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        if ((rc = run_overlap_part(ctx, in, w0, nw, cap, c, false, false, st))) return rc;
        ctx->hook.begin("k_sum_slots", st);
        launch_sum_slots(nw, c.part, c.nslot, 0, c.nR, o_rs.dev ? o_rs.dev + w0 : nullptr, c.O0[0],
                         c.O0[1], o_ov.dev ? o_ov.dev + w0 : nullptr, st);
        ctx->hook.end(st);
        CKLAUNCH();
    }
    return finish(ctx, st, {&o_ov, &o_rs}, in.host_any);
}

int msd_det_ratios(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* ratios,
                   double* ref_ovlp, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    if (n_w == 0) return MSD_OK;
    if (!ratios) return fail(ctx, MSD_ERR_ARG, "ratios is NULL");
    Staged in;
    if ((rc = stage_inputs(ctx, n_w, phi_a, phi_b, st, in))) return rc;
    Out o_r, o_o;
    if ((rc = stage_output(ctx, "out_ratios", ratios, (size_t)n_w * ctx->pairs.n_det, o_r))) return rc;
    if ((rc = stage_output(ctx, "out_refovlp", ref_ovlp, n_w, o_o))) return rc;
    const int nR = weights_blocks(tables(ctx->sp[0], 1));
    const int cap = chunk_for(ctx, overlap_bytes_per_walker(ctx, false, nR), n_w);
    Chunk c;
    if ((rc = chunk_alloc(ctx, cap, false, nR, c))) return rc;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        if ((rc = run_overlap_part(ctx, in, w0, nw, cap, c, false, false, st))) return rc;
        ctx->hook.begin("k_det_ratios", st);
        launch_det_ratios(pair_tables(ctx->pairs), nw, ctx->sp[0].n_str, ctx->sp[1].n_str, c.r[0],
                          c.r[1], o_r.dev + (size_t)w0 * ctx->pairs.n_det, st);
        if (o_o.dev) launch_ref_ovlp(nw, c.O0[0], c.O0[1], o_o.dev + w0, st);
        ctx->hook.end(st);
        CKLAUNCH();
    }
    return finish(ctx, st, {&o_r, &o_o}, in.host_any);
}

int msd_force_bias(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* vbias,
                   double* ovlp, void* stream)
{
    if (ctx && n_w > 0 && !vbias) return fail(ctx, MSD_ERR_ARG, "vbias is NULL");
    return evaluate(ctx, n_w, phi_a, phi_b, ovlp, vbias, nullptr, stream);
}

int msd_local_energy(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* e_loc,
                     double* ovlp, void* stream)
{
    if (ctx && n_w > 0 && !e_loc) return fail(ctx, MSD_ERR_ARG, "e_loc is NULL");
    return evaluate(ctx, n_w, phi_a, phi_b, ovlp, nullptr, e_loc, stream);
}

int msd_rdm1(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* rdm, void* stream)
{
    return rdm1(ctx, n_w, phi_a, phi_b, rdm, stream);
}

int msd_det_energies(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, int n_pairs,
                     const int32_t* w_idx, const int32_t* det_idx, double* e_det, void* stream)
{
    return det_energies(ctx, n_w, phi_a, phi_b, n_pairs, w_idx, det_idx, e_det, stream);
}

int msd_evaluate(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* ovlp,
                 double* vbias, double* e_loc, void* stream)
{
    if (ctx && n_w > 0 && !ovlp && !vbias && !e_loc) return fail(ctx, MSD_ERR_ARG, "no output requested");
    return evaluate(ctx, n_w, phi_a, phi_b, ovlp, vbias, e_loc, stream);
}

int msd_propagate(msd_ctx* ctx, int n_w, double* phi_a, double* phi_b, double* weights, const double* x,
                  double dt, int taylor_order, int orthonormalize, double* ratio, void* stream)
{
    return propagate(ctx, n_w, phi_a, phi_b, weights, x, dt, taylor_order, orthonormalize, ratio, stream);
}

int msd_features(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, int n_core, int n_act,
                 float* feat, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    if (n_core < 0 || n_act <= 0 || n_core + n_act > ctx->M)
        return fail(ctx, MSD_ERR_ARG, "active window [%d, %d) outside the %d orbitals", n_core, n_core + n_act, ctx->M);
    if (n_w == 0) return MSD_OK;
    if (!feat || !is_device_ptr(feat)) return fail(ctx, MSD_ERR_ARG, "feat must be a device pointer");
    Staged in;
    if ((rc = stage_inputs(ctx, n_w, phi_a, phi_b, st, in))) return rc;
    const int nR = weights_blocks(tables(ctx->sp[0], 1));
    const int cap = chunk_for(ctx, overlap_bytes_per_walker(ctx, false, nR), n_w);
    Chunk c;
    if ((rc = chunk_alloc(ctx, cap, false, nR, c))) return rc;
    const int M = ctx->M;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        const double2* phi[2] = {in.pa + (size_t)w0 * M * ctx->n[0], in.pb + (size_t)w0 * M * ctx->n[1]};
        for (int s = 0; s < 2; ++s) {
            const SpinTables T = tables(ctx->sp[s], cap);
            launch_ref(phi[s], nw, M, ctx->n[s], T, c.Gr[s], c.O0[s], c.Gact[s], ctx->d_err, st);
            launch_features(nw, M, ctx->n[s], n_core, n_act, ctx->sp[s].d_pos0, c.Gr[s],
                            feat + (size_t)w0 * 2 * 2 * n_act * n_act, s, st);
        }
        CKLAUNCH();
    }
    Out none;
    return finish(ctx, st, {&none}, in.host_any);
}

int msd_features_rows(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, int ld, float* feat,
                      void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = begin_call(ctx, n_w, phi_a, phi_b, st);
    if (rc) return rc;
    const long long need = 2LL * (ctx->n[0] + ctx->n[1]) * ctx->M;
    if (ld < need) return fail(ctx, MSD_ERR_ARG, "ld = %d below the %lld features per walker", ld, need);
    if (n_w == 0) return MSD_OK;
    if (!feat || !is_device_ptr(feat)) return fail(ctx, MSD_ERR_ARG, "feat must be a device pointer");
    Staged in;
    if ((rc = stage_inputs(ctx, n_w, phi_a, phi_b, st, in))) return rc;
    const int nR = weights_blocks(tables(ctx->sp[0], 1));
    const int cap = chunk_for(ctx, overlap_bytes_per_walker(ctx, false, nR), n_w);
    Chunk c;
    if ((rc = chunk_alloc(ctx, cap, false, nR, c))) return rc;
    const int M = ctx->M;
    if (ld > need) CK(cudaMemsetAsync(feat, 0, sizeof(float) * (size_t)n_w * ld, st));
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        const double2* phi[2] = {in.pa + (size_t)w0 * M * ctx->n[0], in.pb + (size_t)w0 * M * ctx->n[1]};
        long long off = 0;
        for (int s = 0; s < 2; ++s) {
            const SpinTables T = tables(ctx->sp[s], cap);
            launch_ref(phi[s], nw, M, ctx->n[s], T, c.Gr[s], c.O0[s], c.Gact[s], ctx->d_err, st);
            launch_features_rows(nw, M, ctx->n[s], c.Gr[s], feat + (size_t)w0 * ld, ld, off, st);
            off += 2LL * ctx->n[s] * M;
        }
        CKLAUNCH();
    }
    Out none;
    return finish(ctx, st, {&none}, in.host_any);
}

int msd_info(const msd_ctx* ctx, int key, long long* value)
{
    if (!ctx || !value) return MSD_ERR_ARG;
    switch (key) {
    case MSD_INFO_N_DET: *value = ctx->pairs.n_det; break;
    case MSD_INFO_N_CHOL: *value = ctx->n_chol; break;
    case MSD_INFO_N_STRINGS_A: *value = ctx->sp[0].n_str; break;
    case MSD_INFO_N_STRINGS_B: *value = ctx->sp[1].n_str; break;
    case MSD_INFO_N_HOLES_A: *value = ctx->sp[0].nh; break;
    case MSD_INFO_N_PARTS_A: *value = ctx->sp[0].np; break;
    case MSD_INFO_N_HOLES_B: *value = ctx->sp[1].nh; break;
    case MSD_INFO_N_PARTS_B: *value = ctx->sp[1].np; break;
    case MSD_INFO_WORKSPACE_BYTES: {
        long long b = 0;
        for (auto& kv : ctx->arena) b += (long long)kv.second.bytes;
        *value = b;
        break;
    }
    case MSD_INFO_WALKER_CHUNK: *value = ctx->chunk; break;
    case MSD_INFO_EXACT_REFERENCE: *value = exact_ref_on(ctx) ? 1 : 0; break;
    default: return MSD_ERR_ARG;
    }
    return MSD_OK;
}

int msd_set_timing(msd_ctx* ctx, int enable)
{
    if (!ctx) return MSD_ERR_ARG;
    ctx->timing = enable != 0;
    ctx->hook.begin_fn = ctx->timing ? timer_begin : nullptr;
    ctx->hook.end_fn = ctx->timing ? timer_end : nullptr;
    return MSD_OK;
}

int msd_reset_stats(msd_ctx* ctx)
{
    if (!ctx) return MSD_ERR_ARG;
    collect_timing(ctx);
    std::fill(ctx->klaunch.begin(), ctx->klaunch.end(), 0);
    std::fill(ctx->kms.begin(), ctx->kms.end(), 0.0);
    return MSD_OK;
}

int msd_kernel_count(const msd_ctx* ctx) { return ctx ? (int)ctx->knames.size() : 0; }

int msd_kernel_stat(msd_ctx* ctx, int index, const char** name, long long* launches, double* total_ms)
{
    if (!ctx || index < 0 || index >= (int)ctx->knames.size()) return MSD_ERR_ARG;
    collect_timing(ctx);
    if (name) *name = ctx->knames[index].c_str();
    if (launches) *launches = ctx->klaunch[index];
    if (total_ms) *total_ms = ctx->kms[index];
    return MSD_OK;
}

int msd_set_workspace_limit(msd_ctx* ctx, size_t bytes)
{
    if (!ctx) return MSD_ERR_ARG;
    ctx->ws_limit = bytes ? bytes : ((size_t)16 << 30);
    return MSD_OK;
}

long long msd_launch_count(void) { return g_launches.load(); }

int msd_set_sync(msd_ctx* ctx, int sync)
{
    if (!ctx) return MSD_ERR_ARG;
    ctx->sync = sync != 0;
    return MSD_OK;
}

int msd_set_pair_form(msd_ctx* ctx, int form)
{
    if (!ctx) return MSD_ERR_ARG;
    if (form < -1 || form > 2) return fail(ctx, MSD_ERR_ARG, "pair form must be -1 (auto), 0, 1 or 2");
    if (ctx->pair_form != form) {
        ctx->pair_form = form;
        ctx->chunk = 0;   // the partial-sum slots per walker may change
        ++ctx->gen;
    }
    return MSD_OK;
}

int msd_set_wait_budget(msd_ctx* ctx, unsigned long long ns)
{
    if (!ctx) return MSD_ERR_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpy(ctx->d_err + 2, &ns, sizeof ns, cudaMemcpyHostToDevice));
    return MSD_OK;
}

int msd_set_tensor_gram(msd_ctx* ctx, int on)
{
    if (!ctx) return MSD_ERR_ARG;
    ctx->tc_gram = on != 0;
    return MSD_OK;
}

int msd_set_stream_overlap(msd_ctx* ctx, int on)
{
    if (!ctx) return MSD_ERR_ARG;
    ctx->overlap = on != 0;
    return MSD_OK;
}

int msd_set_exact_reference(msd_ctx* ctx, int on)
{
    if (!ctx) return MSD_ERR_ARG;
    if (ctx->exact_ref != (on != 0)) {
        ctx->exact_ref = on != 0;
        ctx->chunk = 0;   // workspace sizes per walker change
        ++ctx->gen;
    }
    return MSD_OK;
}

int msd_set_fused(msd_ctx* ctx, int fused)
{
    if (!ctx) return MSD_ERR_ARG;
    if (ctx->fuse != (fused != 0)) {
        ctx->fuse = fused != 0;
        ctx->chunk = 0;   // workspace sizes per walker change
        ++ctx->gen;
    }
    return MSD_OK;
}

}  // extern "C"

// ========================================================================
// Overlap without device allocation.
//
// msd_overlap obtains its workspace from the context, which grows it with
// cudaMalloc on first use. Some callers cannot let a library allocate during
// a call: a framework that owns every device allocation through its own
// caching allocator or a memory budget fixed at start-up, or a latency-
// critical loop that must not take the device-wide synchronisation that
// cudaMalloc / cudaFree can imply. For them msd_overlap_noalloc computes the
// same overlap with its scratch in the file-scope device array below, whose
// size is fixed at build time. The array lives on every GPU that loads the
// library until the process exits; every call shares it.
#include <mutex>

static __device__ __align__(256) unsigned char g_static_scratch[MSD_STATIC_SCRATCH_BYTES];

namespace {

std::mutex g_static_mu;
void* g_static_ptr[256] = {nullptr};

// Device address of the static scratch on the current device (resolved once
// per device; host code cannot use the symbol itself as a device pointer).
int static_scratch(msd_ctx* ctx, void** out)
{
    std::lock_guard<std::mutex> lock(g_static_mu);
    const int dev = ctx->device;
    if (dev < 0 || dev >= 256) return fail(ctx, MSD_ERR_ARG, "device index %d out of range", dev);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p)
            return fail(ctx, MSD_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                        cudaGetErrorString(e));
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return MSD_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int msd_overlap_noalloc(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                                   double* ovlp, double* ratio_sum, void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    int rc = check_ready(ctx);
    if (rc) return rc;
    if (n_w < 0 || (n_w > 0 && (!phi_a || !phi_b))) return fail(ctx, MSD_ERR_ARG, "bad walker arguments");
    if (n_w > 0 && !ovlp && !ratio_sum) return fail(ctx, MSD_ERR_ARG, "no output requested");
    CK(cudaSetDevice(ctx->device));
    void* scratch = nullptr;
    if ((rc = static_scratch(ctx, &scratch))) return rc;   // first call on a device: set-up
    if (n_w == 0) return MSD_OK;
    const void* ptrs[4] = {phi_a, phi_b, ovlp, ratio_sum};
    for (const void* p : ptrs)
        if (p && !is_device_ptr(p))
            return fail(ctx, MSD_ERR_ARG, "msd_overlap_noalloc takes device pointers only (no staging buffers)");
    const int M = ctx->M;
    SpinTables T1[2] = {tables(ctx->sp[0], 1), tables(ctx->sp[1], 1)};
    const int nR = weights_blocks(T1[0]);
    // scratch per walker: Gr, O0, Gact, r of both spins, alpha weights, partial sums
    size_t per = 0;
    for (int s = 0; s < 2; ++s)
        per += sizeof(double2) * ((size_t)T1[s].N * M + 1 + std::max(1, T1[s].nh * T1[s].np) + T1[s].n_str);
    per += sizeof(double2) * ((size_t)T1[0].n_str + nR);
    const size_t slack = 16 * 256;   // alignment of the carved arrays
    if (per + slack > (size_t)MSD_STATIC_SCRATCH_BYTES)
        return fail(ctx, MSD_ERR_SHAPE,
                    "one walker needs %zu bytes of scratch; the static scratch holds %zu bytes", per + slack,
                    (size_t)MSD_STATIC_SCRATCH_BYTES);
    const int cap = (int)std::min<size_t>((size_t)n_w, ((size_t)MSD_STATIC_SCRATCH_BYTES - slack) / per);
    // carve the static scratch for `cap` walkers; every entry a kernel reads
    // is written earlier in the same call, so nothing needs clearing
    unsigned char* base = (unsigned char*)scratch;
    size_t off = 0;
    auto take = [&](size_t bytes) { void* p = base + off; off += align256(bytes); return p; };
    double2 *Gr[2], *O0[2], *Gact[2], *r[2];
    for (int s = 0; s < 2; ++s) {
        Gr[s] = (double2*)take(sizeof(double2) * cap * T1[s].N * (size_t)M);
        O0[s] = (double2*)take(sizeof(double2) * cap);
        Gact[s] = (double2*)take(sizeof(double2) * cap * (size_t)std::max(1, T1[s].nh * T1[s].np));
        r[s] = (double2*)take(sizeof(double2) * cap * (size_t)T1[s].n_str);
    }
    double2* wts = (double2*)take(sizeof(double2) * cap * (size_t)T1[0].n_str);
    double2* part = (double2*)take(sizeof(double2) * cap * (size_t)nR);
    if (off > (size_t)MSD_STATIC_SCRATCH_BYTES)
        return fail(ctx, MSD_ERR_SHAPE, "static scratch layout overflow (%zu bytes)", off);
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), st));
    TimerHook none;   // no event timing here: events are not created on this path
    const double2* pa = (const double2*)phi_a;
    const double2* pb = (const double2*)phi_b;
    for (int w0 = 0; w0 < n_w; w0 += cap) {
        const int nw = std::min(cap, n_w - w0);
        SpinTables T[2] = {tables(ctx->sp[0], cap), tables(ctx->sp[1], cap)};
        launch_ref(pa + (size_t)w0 * M * ctx->n[0], nw, M, ctx->n[0], T[0], Gr[0], O0[0], Gact[0], ctx->d_err, st);
        launch_ref(pb + (size_t)w0 * M * ctx->n[1], nw, M, ctx->n[1], T[1], Gr[1], O0[1], Gact[1], ctx->d_err, st);
        launch_strings(T[0], nw, Gact[0], r[0], nullptr, nullptr, false, false, st, none);
        launch_strings(T[1], nw, Gact[1], r[1], nullptr, nullptr, false, false, st, none);
        launch_weights(T[0], nw, r[0], r[1], T[1].n_str, wts, part, nR, 0, st);
        launch_sum_slots(nw, part, nR, 0, nR, ratio_sum ? (double2*)ratio_sum + w0 : nullptr, O0[0], O0[1],
                         ovlp ? (double2*)ovlp + w0 : nullptr, st);
        CKLAUNCH();
    }
    if (ctx->sync) {
        CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (*ctx->h_err & MSD_DEV_ERR_SINGULAR)
            return fail(ctx, MSD_ERR_REF_SINGULAR, "D_0^dag phi is singular for some walker");
    }
    return MSD_OK;
}

// ========================================================================
// Batched independent systems (uneven orbital, electron and determinant
// counts) evaluated together: every system's overlap, force-bias and dense
// energy steps, then the per-determinant energy terms of all systems in one
// persistent launch (k_det_batched), then the final sums. The first call with
// a given set of buffers runs eagerly and records the whole sequence as a
// CUDA graph; later calls with the same buffers replay it with one graph
// launch.
#include <cinttypes>
#include <fstream>
#include <sstream>

struct msd_batch {
    std::vector<msd_ctx*> ctx;
    int device = 0;
    int n_sm = 1;                 // set from the device at creation
    std::string err;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<long long> sig;
    BatchSys* d_sys = nullptr;
    size_t sys_cap = 0;
    BatchItem* d_items = nullptr;
    size_t items_cap = 0;
    int n_items = 0;
    unsigned* d_counter = nullptr;
    size_t smem = 0;
    bool fp32 = false;
    int ctas_per_sm = 2, order = 0, bn = 0;
    bool sync = true;
    // systems run concurrently on these streams (graph branches when recorded)
    static const int NSTREAM = 8;
    cudaStream_t aux[NSTREAM] = {};
    cudaEvent_t fork = nullptr, join[NSTREAM] = {};
    long long graph_kernels = 0;
    // CUDA-event time of the persistent kernel in the next eager run
    bool time_pk = false, pk_pending = false;
    cudaEvent_t pk_ev[2] = {nullptr, nullptr};
};

namespace {

int bfail(msd_batch* b, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
    return code;
}

#define BCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bfail(b, MSD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Work items of one system in the slot layout of the per-system kernels
// (same-spin strings of alpha then beta by level, then determinant buckets).
void system_items(msd_ctx* ctx, int sys, int n_w, std::vector<BatchItem>& out, std::vector<double>& cost)
{
    SpinTables T[2] = {tables(ctx->sp[0], 1), tables(ctx->sp[1], 1)};
    const PairTables pt = pair_tables(ctx->pairs);
    const int nR = weights_blocks(T[0]);
    for (int w = 0; w < n_w; ++w) {
        int slot = nR;
        for (int s = 0; s < 2; ++s)
            for (int k = 1; k <= MSD_KMAX; ++k) {
                const int ns = T[s].bucket[k + 1] - T[s].bucket[k];
                const int nb = string_energy_blocks(T[s], k);
                for (int blk = 0; blk < nb; ++blk) {
                    out.push_back({sys, w, 0, s, k, 0, blk, slot++});
                    const int cnt = std::min(SE_THREADS * SE_PER_THREAD, ns - blk * SE_THREADS * SE_PER_THREAD);
                    cost.push_back((double)cnt * (2.0 * k * k * k * k + 2.0 * k * k));
                }
            }
        for (int ka = 1; ka <= MSD_KMAX; ++ka)
            for (int kb = 1; kb <= MSD_KMAX; ++kb) {
                const int idx = ka * (MSD_KMAX + 1) + kb;
                const int n = pt.bucket[idx + 1] - pt.bucket[idx];
                if (n <= 0) continue;
                const int nb = (n + PC_THREADS * PC_PER_THREAD - 1) / (PC_THREADS * PC_PER_THREAD);
                for (int blk = 0; blk < nb; ++blk) {
                    out.push_back({sys, w, 1, 0, ka, kb, blk, slot++});
                    const int cnt = std::min(PC_THREADS * PC_PER_THREAD, n - blk * PC_THREADS * PC_PER_THREAD);
                    cost.push_back((double)cnt * (ka * ka * kb * kb + ka * ka));
                }
            }
    }
}

// Enqueue the whole batched evaluation on `st`. With upload, the system
// descriptors and work items are (re)built and copied to the device first
// (not done while recording a graph: the copies there are already current).
int batch_run(msd_batch* b, const int* n_w, const double* const* pa, const double* const* pb,
              double* const* ovlp, double* const* vbias, double* const* e_loc, cudaStream_t st, bool upload)
{
    const int n = (int)b->ctx.size();
    std::vector<Deferred> d(n);
    // fork: system i runs on aux[i % NSTREAM] after everything queued on st
    BCK(cudaEventRecord(b->fork, st));
    for (int k = 0; k < msd_batch::NSTREAM; ++k) BCK(cudaStreamWaitEvent(b->aux[k], b->fork, 0));
    for (int i = 0; i < n; ++i) {
        msd_ctx* ctx = b->ctx[i];
        const bool saved = ctx->sync;
        ctx->sync = false;
        ctx->tc_bn = b->bn;
        const int rc = evaluate_impl(ctx, n_w[i], pa[i], pb[i], ovlp ? ovlp[i] : nullptr,
                                     vbias ? vbias[i] : nullptr, e_loc[i], b->aux[i % msd_batch::NSTREAM], &d[i]);
        ctx->sync = saved;
        if (rc) return bfail(b, rc, "system %d: %s", i, ctx->err.c_str());
    }
    // join
    for (int k = 0; k < msd_batch::NSTREAM; ++k) {
        BCK(cudaEventRecord(b->join[k], b->aux[k]));
        BCK(cudaStreamWaitEvent(st, b->join[k], 0));
    }
    if (upload) {
        std::vector<BatchSys> sys(n);
        std::vector<BatchItem> items;
        std::vector<double> cost;
        size_t smem = 0;
        for (int i = 0; i < n; ++i) {
            msd_ctx* ctx = b->ctx[i];
            const int cap = d[i].cap;
            BatchSys& S = sys[i];
            memset(&S, 0, sizeof S);
            S.t[0] = tables(ctx->sp[0], cap);
            S.t[1] = tables(ctx->sp[1], cap);
            S.pt = pair_tables(ctx->pairs);
            for (int s = 0; s < 2; ++s) {
                S.r[s] = d[i].c.r[s];
                S.rf[s] = d[i].c.rf[s];
                S.wts[s] = d[i].c.wts[s];
                S.B[s] = d[i].c.B[s];
                S.Y[s] = d[i].E.Y[s];
            }
            S.K[0] = d[i].E.Kaa; S.K[1] = d[i].E.Kbb; S.K[2] = d[i].E.Kab;
            S.part = d[i].c.part;
            S.nslot = d[i].c.nslot;
            const size_t X0 = (size_t)S.t[0].nh * S.t[0].np, X1 = (size_t)S.t[1].nh * S.t[1].np;
            smem = std::max(smem, std::max(std::max(X0 * X0 + X0, X1 * X1 + X1), X0 * X1));
            system_items(ctx, i, n_w[i], items, cost);
        }
        if (b->order == 1) {          // largest work first
            std::vector<size_t> idx(items.size());
            for (size_t k = 0; k < idx.size(); ++k) idx[k] = k;
            std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
            std::vector<BatchItem> o(items.size());
            for (size_t k = 0; k < idx.size(); ++k) o[k] = items[idx[k]];
            items.swap(o);
        } else if (b->order == 2) {   // walkers interleaved across systems
            std::stable_sort(items.begin(), items.end(),
                             [](const BatchItem& x, const BatchItem& y) { return x.w < y.w; });
        }
        b->smem = smem * (b->fp32 ? sizeof(float2) : sizeof(double2));
        if (b->sys_cap < (size_t)n) {
            cudaFree(b->d_sys);
            BCK(cudaMalloc(&b->d_sys, sizeof(BatchSys) * n));
            b->sys_cap = n;
        }
        if (b->items_cap < items.size()) {
            cudaFree(b->d_items);
            BCK(cudaMalloc(&b->d_items, sizeof(BatchItem) * items.size()));
            b->items_cap = items.size();
        }
        BCK(cudaMemcpy(b->d_sys, sys.data(), sizeof(BatchSys) * n, cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
        b->n_items = (int)items.size();
    }
    const bool timed = upload && b->time_pk && b->pk_ev[0];
    if (timed) BCK(cudaEventRecord(b->pk_ev[0], st));
    if (launch_det_batched(b->d_sys, b->d_items, b->n_items, b->d_counter, b->smem, b->fp32,
                           b->ctas_per_sm * b->n_sm, st))
        return bfail(b, MSD_ERR_CUDA, "persistent batched launch failed");
    if (timed) {
        BCK(cudaEventRecord(b->pk_ev[1], st));
        b->pk_pending = true;
    }
    for (int i = 0; i < n; ++i) {
        msd_ctx* ctx = b->ctx[i];
        launch_final(n_w[i], d[i].c.part, d[i].c.nslot, d[i].c.nR, ctx->e0, (double2*)d[i].E.e1[0],
                     (double2*)d[i].E.e1[1], (double2*)d[i].E.scal, d[i].c.O0[0], d[i].c.O0[1],
                     (double2*)e_loc[i], ovlp && ovlp[i] ? (double2*)ovlp[i] : nullptr, st);
    }
    BCK(cudaGetLastError());
    return MSD_OK;
}

int batch_check(msd_batch* b, cudaStream_t st)
{
    BCK(cudaStreamSynchronize(st));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        msd_ctx* ctx = b->ctx[i];
        unsigned e = 0;
        BCK(cudaMemcpy(&e, ctx->d_err, sizeof e, cudaMemcpyDeviceToHost));
        if (e & MSD_DEV_ERR_SINGULAR) return bfail(b, MSD_ERR_REF_SINGULAR, "system %zu: singular reference", i);
        if (e & MSD_DEV_ERR_TIMEOUT) return bfail(b, MSD_ERR_TIMEOUT, "system %zu: a device wait expired", i);
    }
    return MSD_OK;
}

std::vector<long long> batch_signature(msd_batch* b, const int* n_w, const double* const* pa,
                                       const double* const* pb, double* const* ovlp, double* const* vbias,
                                       double* const* e_loc)
{
    std::vector<long long> s;
    s.push_back(b->bn); s.push_back(b->ctas_per_sm); s.push_back(b->order);
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        s.push_back(n_w[i]);
        s.push_back((long long)(uintptr_t)pa[i]);
        s.push_back((long long)(uintptr_t)pb[i]);
        s.push_back((long long)(uintptr_t)(ovlp ? ovlp[i] : nullptr));
        s.push_back((long long)(uintptr_t)(vbias ? vbias[i] : nullptr));
        s.push_back((long long)(uintptr_t)e_loc[i]);
        s.push_back(b->ctx[i]->gen);
    }
    return s;
}

void drop_graph(msd_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->sig.clear();
}

std::string batch_key(msd_batch* b, const int* n_w)
{
    uint64_t h = 1469598103934665603ull;   // FNV-1a over the shapes
    auto mix = [&](long long v) {
        for (int k = 0; k < 8; ++k) { h ^= (uint64_t)((v >> (8 * k)) & 0xff); h *= 1099511628211ull; }
    };
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        msd_ctx* c = b->ctx[i];
        mix(c->M); mix(c->n[0]); mix(c->n[1]); mix(c->pairs.n_det); mix(c->n_chol); mix(n_w[i]); mix(c->prec);
        mix(c->sp[0].n_str); mix(c->sp[1].n_str);
    }
    char buf[32];
    snprintf(buf, sizeof buf, "%016" PRIx64, h);
    return buf;
}

}  // namespace

extern "C" {

int msd_batch_create(msd_batch** out, msd_ctx* const* ctxs, int n_sys)
{
    if (!out || !ctxs || n_sys <= 0) return MSD_ERR_ARG;
    *out = nullptr;
    msd_batch* b = new msd_batch();
    for (int i = 0; i < n_sys; ++i) {
        if (!ctxs[i] || !ctxs[i]->have_ham || !ctxs[i]->have_trial) {
            delete b;
            return fail(nullptr, MSD_ERR_STATE, "batch: system %d is not set up", i);
        }
        if (i && (ctxs[i]->device != ctxs[0]->device || ctxs[i]->prec != ctxs[0]->prec)) {
            delete b;
            return fail(nullptr, MSD_ERR_ARG, "batch: all systems need one device and one precision");
        }
        b->ctx.push_back(ctxs[i]);
    }
    // the persistent per-determinant kernel implements the per-determinant
    // opposite-spin form; the systems' own evaluations use the same form, so
    // batched and per-system results agree
    for (int i = 0; i < n_sys; ++i) msd_set_pair_form(ctxs[i], 0);
    b->device = ctxs[0]->device;
    b->fp32 = ctxs[0]->prec == MSD_MIXED;
    cudaSetDevice(b->device);
    cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device);
    bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&b->d_counter, sizeof(unsigned)) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < msd_batch::NSTREAM; ++k)
        ok = cudaStreamCreateWithFlags(&b->aux[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        delete b;
        return fail(nullptr, MSD_ERR_CUDA, "batch: stream or counter allocation failed");
    }
    *out = b;
    return MSD_OK;
}

void msd_batch_destroy(msd_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    drop_graph(b);
    cudaFree(b->d_sys); cudaFree(b->d_items); cudaFree(b->d_counter);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int k = 0; k < msd_batch::NSTREAM; ++k) {
        if (b->aux[k]) cudaStreamDestroy(b->aux[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->pk_ev[0]) { cudaEventDestroy(b->pk_ev[0]); cudaEventDestroy(b->pk_ev[1]); }
    delete b;
}

const char* msd_batch_last_error(const msd_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int msd_batch_evaluate(msd_batch* b, const int* n_w, const double* const* phi_a, const double* const* phi_b,
                       double* const* ovlp, double* const* vbias, double* const* e_loc, void* stream)
{
    if (!b || !n_w || !phi_a || !phi_b || !e_loc) return b ? bfail(b, MSD_ERR_ARG, "null argument") : MSD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    const std::vector<long long> sig = batch_signature(b, n_w, phi_a, phi_b, ovlp, vbias, e_loc);
    if (b->exec && sig == b->sig) {
        BCK(cudaGraphLaunch(b->exec, st));
        return b->sync ? batch_check(b, st) : MSD_OK;
    }
    drop_graph(b);
    std::vector<bool> timing(b->ctx.size());
    int rc = batch_run(b, n_w, phi_a, phi_b, ovlp, vbias, e_loc, st, true);
    if (rc) return rc;
    if (b->sync && (rc = batch_check(b, st))) return rc;
    // record the same sequence (no allocation can happen now: every buffer
    // has its size) for replay by the next calls with these buffers
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        timing[i] = b->ctx[i]->timing;
        msd_set_timing(b->ctx[i], 0);
    }
    BCK(cudaStreamSynchronize(st));
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
    rc = batch_run(b, n_w, phi_a, phi_b, ovlp, vbias, e_loc, b->cap, false);
    const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
    for (size_t i = 0; i < b->ctx.size(); ++i) msd_set_timing(b->ctx[i], timing[i] ? 1 : 0);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (ce != cudaSuccess) return bfail(b, MSD_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    size_t n_nodes = 0;
    cudaGraphGetNodes(g, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    if (n_nodes) cudaGraphGetNodes(g, nodes.data(), &n_nodes);
    b->graph_kernels = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) b->graph_kernels++;
    }
    const cudaError_t ie = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { b->exec = nullptr; return bfail(b, MSD_ERR_CUDA, "graph instantiate failed"); }
    b->sig = sig;
    return MSD_OK;
}

int msd_batch_autotune(msd_batch* b, const int* n_w, const double* const* phi_a, const double* const* phi_b,
                       double* const* ovlp, double* const* vbias, double* const* e_loc, void* stream,
                       const char* cache_path)
{
    if (!b || !n_w || !phi_a || !phi_b || !e_loc) return b ? bfail(b, MSD_ERR_ARG, "null argument") : MSD_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    BCK(cudaSetDevice(b->device));
    const std::string key = batch_key(b, n_w);
    if (cache_path && *cache_path) {
        std::ifstream f(cache_path);
        std::string line;
        while (std::getline(f, line)) {
            std::istringstream is(line);
            std::string k;
            int bn, cps, ord;
            if (is >> k >> bn >> cps >> ord && k == key) {
                b->bn = bn; b->ctas_per_sm = cps; b->order = ord;
                drop_graph(b);
                return MSD_OK;
            }
        }
    }
    const int bns[2] = {128, 256}, cpss[3] = {1, 2, 4}, ords[3] = {0, 1, 2};
    float best = 1e30f;
    int bb = 0, bc = 2, bo = 0;
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    const bool saved_sync = b->sync;
    b->sync = false;
    int rc = MSD_OK;
    for (int bn : bns)
        for (int cps : cpss)
            for (int ord : ords) {
                b->bn = bn; b->ctas_per_sm = cps; b->order = ord;
                if ((rc = batch_run(b, n_w, phi_a, phi_b, ovlp, vbias, e_loc, st, true))) goto done;
                cudaEventRecord(e0, st);
                for (int rep = 0; rep < 2; ++rep)
                    if ((rc = batch_run(b, n_w, phi_a, phi_b, ovlp, vbias, e_loc, st, false))) goto done;
                cudaEventRecord(e1, st);
                if ((rc = batch_check(b, st))) goto done;
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; bb = bn; bc = cps; bo = ord; }
            }
done:
    b->sync = saved_sync;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->bn = bb; b->ctas_per_sm = bc; b->order = bo;
    drop_graph(b);
    if (cache_path && *cache_path) {
        std::ofstream f(cache_path, std::ios::app);
        f << key << " " << bb << " " << bc << " " << bo << " " << best / 2 << "\n";
    }
    return MSD_OK;
}

int msd_batch_config(const msd_batch* b, int* tile_n, int* ctas_per_sm, int* order)
{
    if (!b) return MSD_ERR_ARG;
    if (tile_n) *tile_n = b->bn;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    if (order) *order = b->order;
    return MSD_OK;
}

int msd_batch_set_config(msd_batch* b, int tile_n, int ctas_per_sm, int order)
{
    if (!b || (tile_n != 0 && tile_n != 128 && tile_n != 256) || ctas_per_sm < 1 || ctas_per_sm > 8 ||
        order < 0 || order > 2)
        return b ? bfail(b, MSD_ERR_ARG, "bad batch configuration") : MSD_ERR_ARG;
    b->bn = tile_n; b->ctas_per_sm = ctas_per_sm; b->order = order;
    drop_graph(b);
    return MSD_OK;
}

int msd_batch_time_persistent(msd_batch* b, int enable, double* last_ms)
{
    if (!b) return MSD_ERR_ARG;
    BCK(cudaSetDevice(b->device));
    if (enable && !b->pk_ev[0]) {
        BCK(cudaEventCreate(&b->pk_ev[0]));
        BCK(cudaEventCreate(&b->pk_ev[1]));
    }
    b->time_pk = enable != 0;
    if (last_ms) {
        *last_ms = -1.0;
        if (b->pk_pending) {
            BCK(cudaEventSynchronize(b->pk_ev[1]));
            float ms = 0;
            BCK(cudaEventElapsedTime(&ms, b->pk_ev[0], b->pk_ev[1]));
            *last_ms = ms;
        }
    }
    return MSD_OK;
}

int msd_batch_graph_ready(const msd_batch* b) { return b && b->exec ? 1 : 0; }

long long msd_batch_graph_kernels(const msd_batch* b) { return b && b->exec ? b->graph_kernels : 0; }

}  // extern "C"
