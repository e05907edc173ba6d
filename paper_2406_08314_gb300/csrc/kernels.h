// Host-side launchers of the libmsd kernels (internal to csrc/).
#pragma once

#include "common.cuh"

// Optional per-kernel event timing, supplied by the context.
struct TimerHook {
    void* self = nullptr;
    void (*begin_fn)(void*, const char*, cudaStream_t) = nullptr;
    void (*end_fn)(void*, cudaStream_t) = nullptr;
    void begin(const char* name, cudaStream_t st) const { if (begin_fn) begin_fn(self, name, st); }
    void end(cudaStream_t st) const { if (end_fn) end_fn(self, st); }
};

// k_wick.cu
void launch_ref(const double2* phi, int nw, int M, int N, const SpinTables& T, double2* Gr,
                double2* O0, double2* Gact, unsigned* err, cudaStream_t st);
void launch_strings(const SpinTables& tb, int nw, const double2* Gact, double2* r, float2* rf, void* B,
                    bool fp32, bool want_b, cudaStream_t st, const TimerHook& th);
int weights_blocks(const SpinTables& tb);
void launch_weights(const SpinTables& tb, int nw, const double2* r_self, const double2* r_other,
                    int n_other, double2* wts, double2* part, int nslot, int slot0, cudaStream_t st);
void launch_det_ratios(const PairTables& pt, int nw, int n_str_a, int n_str_b, const double2* ra,
                       const double2* rb, double2* out, cudaStream_t st);
void launch_sum_slots(int nw, const double2* part, int nslot, int slot0, int n, double2* out,
                      const double2* O0a, const double2* O0b, double2* ovlp, cudaStream_t st);
void launch_ref_ovlp(int nw, const double2* O0a, const double2* O0b, double2* out, cudaStream_t st);
void launch_cmat(const SpinTables& ta, const SpinTables& tb, int nw, const double2* wts_a, const double2* wts_b,
                 const void* Ba, const void* Bb, bool fp32, double2* Cm_a, double2* Cm_b, cudaStream_t st);
void launch_gt(const SpinTables& tb, int nw, int M, const double2* Gr, const double2* Cm,
               const double2* R, double2* GT, long long ld, long long off, bool minus_ref, cudaStream_t st);
void launch_rdm_scatter(const SpinTables& tb, int nw, int M, const double2* GT, long long ld, long long off, int spin,
                        double2* rdm, cudaStream_t st);

// k_energy.cu
void launch_gemm_zd(int Mr, int Nc, int K, const double2* A, long long lda, const double* B,
                    long long ldb, double2* C, long long ldc, cudaStream_t st);
size_t fepi_smem(const SpinTables& tb);
void launch_fepi(const SpinTables& tb, int nw, int M, int n_chol, const double2* F, long long ldf,
                 const double2* Gr, double2* v0, double2* xx, double2* Lact, double2* Xic,
                 cudaStream_t st);
// hl (optional): the matrix of the Lambda_h part instead of h1.
void launch_onebody(const SpinTables& tb, int nw, int M, const double* h1, const double2* Gr,
                    double2* e1, double2* Lh, cudaStream_t st, const double* hl = nullptr);
void launch_gamma_reduce(int nw, int X, int n_chol, int spin, const double2* v0a, const double2* v0b,
                         const double2* xx, const double2* Lact, const double2* Xic,
                         const double2* Lh, void* Y, bool fp32, double2* scal, cudaStream_t st);
void launch_gram(int nw, int Xp, int Xq, int n_chol, const double2* P, const double2* Q, void* K,
                 bool fp32, cudaStream_t st);
int string_energy_blocks(const SpinTables& tb, int k);
size_t string_energy_smem(const SpinTables& tb, bool fp32);
int string_energy_slots(const SpinTables& tb);
void launch_string_energy(const SpinTables& tb, int nw, const double2* wts,
                          const void* B, const void* K, const void* Y, bool fp32, double2* part,
                          int nslot, int slot0, cudaStream_t st);
int pair_cross_slots(const PairTables& pt, bool use_runs = false);
// k_pair_y.cu: the opposite-spin term per beta string (mixed precision)
bool pair_y_ok(const SpinTables& ta, const SpinTables& tb);
int pair_y_slots(const SpinTables& tb);
void launch_pair_y(const SpinTables& ta, const SpinTables& tb, int nw, const float2* rfa, const float2* rfb,
                   const void* Ba, const void* Bb, const void* Kab, double2* part, int nslot, int slot0,
                   cudaStream_t st);
// ra, rb: the string ratios in the working precision (double2 in FP64 mode,
// their FP32 copies in mixed mode)
// use_runs: buckets with run_side != 0 take the runs form (k_pair_run.cu).
void launch_pair_cross(const SpinTables& ta, const SpinTables& tb, const PairTables& pt, int nw,
                       const void* ra, const void* rb, const void* Ba, const void* Bb,
                       const void* K, bool fp32, double2* part, int nslot, int slot0,
                       cudaStream_t st, bool use_runs = false);
// k_pair_run.cu
int pair_run_blocks(const PairTables& pt, int bidx);
size_t pair_run_smem(const SpinTables& ta, const SpinTables& tb, bool fp32);
void launch_pair_run(const SpinTables& ta, const SpinTables& tb, const PairTables& pt, int bidx, int ka, int kb,
                     int nw, const void* ra, const void* rb, const void* Ba, const void* Bb, const void* K, bool fp32,
                     double2* part, int nslot, int slot, cudaStream_t st);
void launch_final(int nw, const double2* part, int nslot, int nR, double e0, const double2* e1a,
                  const double2* e1b, const double2* scal, const double2* O0a, const double2* O0b,
                  double2* eloc, double2* ovlp, cudaStream_t st);

// tc_gemm.cu: 3xTF32 tensor-core GEMM C[m][n] = sum_k A[m][k] B[n][k] with
// A, B given as hi/lo TF32 parts, K-major with row pitch ld (elements).
struct TcOperand {
    const float* hi;
    const float* lo;
    long long ld;
};
// K is split over `splits` CTAs along grid.z; split z writes C + z * c_split_stride.
// bn: output tile width (128 or 256; 0 picks by Nc).
int tc_gemm_3xtf32(const TcOperand& A, const TcOperand& B, int Mr, int Nc, int K, float* C, long long ldc,
                   unsigned* err, cudaStream_t st, int splits = 1, long long c_split_stride = 0, int bn = 0);
// BF16 tensor-core GEMM C[m][n] = sum_k A[m][k] B[n][k] (FP32 accumulation;
// A, B row-major BF16 with K contiguous, K a multiple of 64).
int tc_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, int Mr, int Nc, int K, float* C,
                 long long ldc, unsigned* err, cudaStream_t st);
// part_rows: rows per (block, part) in the output (0: R; larger pads each
// part with zero rows). eye0 >= 0: columns [eye0, eye0 + 2 part_rows) hold
// two identity blocks on the real-part rows r < R (1 at column eye0 + r and
// eye0 + part_rows + r), zero on the imaginary-part rows.
void launch_split_complex_rows(int nb, int R, int Kg, int Kp, const double2* src, long long src_ld,
                               const int* cols, float* hi, float* lo, cudaStream_t st, int part_rows = 0,
                               int eye0 = -1);
void launch_split_real_rows(long long R, int Kg, int Kp, const double* src, long long src_ld, const int* cols,
                            float* hi, float* lo, cudaStream_t st);
// Slices of x[r][j] (r < R, j < n, FP64) into two column blocks of rows of
// pitch ld: hi/lo[r][k0 + j] = (h, m) and hi/lo[r][k0 + RB + j] = (q, s),
// h = tf32(x), m = tf32(x - h), q = tf32(x - h - m), s = tf32(x - h - m - q),
// so that h + m + q + s equals x to about 44 bits.
void launch_split_blocks(long long R, int n, int RB, int ld, int k0, const double* x, float* hi, float* lo,
                         cudaStream_t st);
void launch_pack_complex(int nw, int n, const float* C, long long ldc, int splits, long long split_stride,
                         const double* add, double2* out, long long ldo, cudaStream_t st);

// tc_fepi.cu: the Cholesky contraction of the energy fused with its
// per-(walker, vector) epilogue (same outputs as tc_gemm_3xtf32 followed by
// launch_fepi_f32). A: split rows of dG[occ0][virt], part c of walker w at
// rows (2w + c) RB; B: split half-rotated Cholesky rows, vector g's at
// g NCf + [occ0 (N), zero (RB - N), particles (np)]; both pitch ld,
// contraction K. F0P: [n_chol][f0s], F0[j][col] = L_g[occ0_j][col] at
// g f0s + j NCP + col in the same column order, zero padded.
struct TcFepiPlan {
    int RB = 0, RW = 0, WPT = 0, NCf = 0, BN = 0, GPT = 0, BNe = 0, slot = 0, NCP = 0, f0s = 0;
    size_t smem = 0;
};
bool tc_fepi_plan(const SpinTables& tb, TcFepiPlan& p);
int tc_fepi_fused(const SpinTables& tb, const TcFepiPlan& p, int nw, int M, int n_chol, const float* a_hi,
                  const float* a_lo, const float* b_hi, const float* b_lo, int ld, int K, const double2* Gr,
                  const float* F0P, const double* c0, const double* x0, double2* v0, double2* xx,
                  float2* Lact, float2* Xic, unsigned* err, cudaStream_t st, bool traces);

// tc_ozaki.cu: the reference-determinant Cholesky sums of the mixed local
// energy in FP64 accuracy (exact-integer BF16 slices on the tensor cores).
// Constant operand of one spin: B = [V | 0 | W]^T sliced, V's N Kv rows padded
// with zero rows to a whole number of column tiles (NVp), NB = NVp + G rows.
struct OzConst {
    int N = 0, Kv = 0, G = 0, NK = 0, NVp = 0, NB = 0, NBp = 0, Kp = 0;   // V rows padded to NVp
    void* Bs = nullptr;   // [OZ_S][NBp][Kp] BF16
    int* eb = nullptr;    // [NBp] row exponents
};
// One spin's inputs to the per-walker reduction.
struct RefSpin {
    int N, M, Kv, nparts, Mpad;
    const double2* Gr;
    const int* virt;
    const double* JJ;     // [N Kv] J[v_r][o_j], J = sum_g (c0a_g + c0b_g) L_g
    const double* KK;     // [N Kv] (sum_g L_g P0 L_g)[v_r][o_j]
    const double* t1;     // [2 nw][G]
    const double2* part;  // [nparts][Mpad]
    double x0sum;         // sum_g x0_g of this spin
};
size_t oz_const_bytes(int N, int Kv, int G);
int oz_rows_padded(int nrow);
int oz_k_padded(int NK);
int oz_parts(int NB);                // partial-sum rows of a constant operand with NB rows
int oz_parts_for(int NK, int G);     // the same from N (M - N) and n_chol
int oz_slices();
// d_XT: [N Kv][G] FP64, XT[r N + l][g] = L_g[v_r][o_l]. Allocates out's arrays.
int oz_prepare_const(int N, int Kv, int G, const double* d_XT, OzConst& out, cudaStream_t st);
void oz_free_const(OzConst& c);
// As: [OZ_S][pad(2 nw)][Kp] BF16 scratch, ea: [pad(2 nw)]; writes part
// [oz_parts(NB)][pad(2 nw)] and t1 [2 nw][G].
int oz_spin(const OzConst& K, int nw, int M, const double2* Gr, const int* virt, void* As, int* ea, double2* part,
            double* t1, unsigned* err, cudaStream_t st);
// Also writes the walker parts t1a_g + t1b_g of V0_g as FP32 pairs v0w[w][g].
void launch_ref_reduce(int nw, int G, const RefSpin& a, const RefSpin& b, double C2sum, double2* scal,
                       float2* v0w, cudaStream_t st);

// k_debug.cu: E_I of sampled (walker, determinant) pairs.
struct DetRec {
    int w, a, b, ka, kb;   // walker, alpha and beta string, their levels
};
void launch_det_energy(int n, const DetRec* recs, int w0, int nw, const SpinTables& ta, const SpinTables& tb,
                       const void* Ba, const void* Bb, const void* Kaa, const void* Kbb, const void* Kab,
                       const void* Ya, const void* Yb, const double2* scal, const double2* e1a, const double2* e1b,
                       double e0, bool fp32, double2* out, cudaStream_t st);

// k_mixed.cu
size_t fepi_f32_smem(const SpinTables& tb);
void launch_fepi_f32(const SpinTables& tb, int nw, int M, int n_chol, const float* dF, long long ldf,
                     const double2* Gr, const float* F0T, const double* c0, const double* x0, double2* v0,
                     double2* xx, float2* Lact, float2* Xic, cudaStream_t st);
void launch_gamma_reduce_f32(int nw, int X, int n_chol, int spin, const double2* v0a, const double2* v0b,
                             const double2* xx, const float2* Lact, const float2* Xic, const double2* Lh,
                             float2* Y, double2* scal, cudaStream_t st, bool traces,
                             const float2* v0w = nullptr);
// K[w][x][y] = sum_g P[w][g][x] Q[w][g][y] (FP32) for up to three
// (P, Q, K) products of shapes Xp x Xq in one launch.
struct GramJob {
    int Xp, Xq;          // entries; P and Q rows have the pitch lam_pitch(X)
    const float2* P;
    const float2* Q;
    float2* K;
};
struct GramJobs {
    GramJob j[3];
};
void launch_gram_f32(int nw, int n_chol, const GramJobs& jobs, int nj, cudaStream_t st);
// tc_gram.cu: the same Gram matrices on the tensor cores (3xTF32, FP32
// accumulation in TMEM) for 2 X <= 256 per spin; returns 0 or -1.
// Rows first: T[w][2x + c][g] = part c of Lam[w][g][x] (FP32, Lam rows of the
// pitch lam_pitch(X)); then K_aa, K_bb, K_ab from Ta, Tb ([nw][X][X'] pairs).
// tc_gram needs n_chol a multiple of 4 and tc_gram_ok; returns 0 or -1.
bool tc_gram_ok(int Xa, int Xb);
void launch_gram_transpose(int nw, int n_chol, int X, const float2* Lam, float* T, cudaStream_t st);
int tc_gram(int nw, int n_chol, int Xa, int Xb, const float* Ta, const float* Tb, float2* Kaa, float2* Kbb,
            float2* Kab, unsigned* err, cudaStream_t st);

// k_batch.cu: per-determinant energy terms of many systems in one
// persistent launch.
struct BatchSys {
    SpinTables t[2];
    PairTables pt;
    const double2* r[2];
    const float2* rf[2];  // FP32 copies of r (mixed mode)
    const double2* wts[2];
    const void* B[2];
    const void* K[3];   // same-spin alpha, same-spin beta, opposite-spin Gram matrices
    const void* Y[2];
    double2* part;
    int nslot;
    int pad_;
};
struct BatchItem {
    int sys, w;
    int kind;           // 0: same-spin string block, 1: opposite-spin determinant block
    int spin;           // kind 0
    int ka, kb;         // level (kind 0: ka); level pair (kind 1)
    int blk, slot;      // block within the bucket, partial-sum slot
};
int launch_det_batched(const BatchSys* systems, const BatchItem* items, int n_items, unsigned* counter,
                       size_t smem, bool fp32, int grid, cudaStream_t st);

// mlp.cu
void launch_features(int nw, int M, int N, int n_core, int n_act, const int* pos0, const double2* Gr, float* feat,
                     int spin, cudaStream_t st);
void launch_features_rows(int nw, int M, int N, const double2* Gr, float* feat, long long ld, long long off,
                          cudaStream_t st);

// k_prop.cu: one phaseless propagation step (FP64).
void launch_sum_LL(int M, int G, const double* Lt, double* corr, cudaStream_t st);
void launch_prop_coef(int nw, int G, double dt, const double* x, const double2* vbias, double2* c, double2* expo,
                      cudaStream_t st);
int launch_apply_rows(int nw, int M, int N, const double2* A, long long a_stride, const double* Ar,
                      const double2* in, double2* out, double2* acc, double scale, cudaStream_t st);
void launch_prop_weight(int nw, const double2* o_old, const double2* o_new, const double2* expo, double* w,
                        double2* ratio, cudaStream_t st);
int launch_qr_mgs(int nw, int M, int N, double2* phi, unsigned* err, cudaStream_t st);

// k_pair.cu: the opposite-spin term with both levels compiled in (ka + kb <=
// 8); false for other level pairs.
bool launch_pair_cross2(int ka, int kb, bool fp32, dim3 grid, size_t smem, const SpinTables& ta, const SpinTables& tb,
                        const PairTables& pt, int lo, int n, const void* ra, const void* rb, const void* Ba,
                        const void* Bb, const void* K, double2* part, int nslot, int slot, cudaStream_t st);
