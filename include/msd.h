/*
 * msd.h -- C ABI of libmsd: the multi-Slater-determinant AFQMC hot path on one
 * NVIDIA GB300 (sm_103a).
 *
 * For a batch of walkers |phi> (one complex M x N_s orbital matrix per spin s)
 * and a CI trial |Psi_T> = sum_I c_I |D_I> whose determinants share one
 * orthonormal orbital set (Sec. II B), the library evaluates
 *
 *   overlap      O_T = <Psi_T|phi>                                (Sec. II A-B)
 *   force bias   vbias_g = <Psi_T| L_g-hat |phi> / <Psi_T|phi>,
 *                L_g-hat = sum_{pq,s} L^g_pq a+_ps a_qs             (Eq. 7)
 *   local energy E_L = <Psi_T|H|phi> / <Psi_T|phi>                (Sec. II A, III)
 *
 * for H = e0 + sum_{pq,s} h^s_pq a+_ps a_qs
 *         + 1/2 sum_g sum_{pqrs,st} L^g_pq L^g_rs a+_ps a+_rt a_st a_qs,
 * the Cholesky form of Eq. 2-3 with (pq|rs) = sum_g L^g_pq L^g_rs and the
 * bare one-body matrix h (not h' = h - 1/2 sum_r (pr|rq), which only the
 * propagator uses).
 *
 * Method (Sec. III "Implementation", and the Wick-theorem approach the paper
 * adopts in Sec. III): every trial determinant is an excitation of the
 * reference D_0 (trial determinant 0). Per walker and spin the library forms
 * Theta = phi (D_0^dag phi)^-1 and the reference Green's function
 * G0 = Theta D_0^dag; the overlap ratio of a determinant with holes h_1..h_k
 * and particles p_1..p_k is sign * det A with A[i][j] = G[h_i][p_j] (a k x k
 * minor of G = G0^T), its Green's function is a rank-k update of G, and the
 * energy follows from contractions of the Cholesky vectors with G. Spin
 * sectors are handled separately; only the energy and the ratio weights
 * couple them.
 *
 * Conventions
 *   - Complex numbers are interleaved (re, im) pairs of doubles.
 *   - phi_s: [n_w][M][N_s] row-major (walker, orbital, electron).
 *   - |D_I> = prod_{p in occ_a(I), ascending} a+_{p alpha}
 *             prod_{p in occ_b(I), ascending} a+_{p beta} |0>;
 *     the walker's creation operators are ordered the same way (alpha
 *     columns, then beta columns), so <D_I|phi> = det(phi_a[occ_a]) *
 *     det(phi_b[occ_b]).
 *   - Walker and output pointers may be device memory (the fast path) or host
 *     memory; host buffers are staged through device memory owned by the
 *     context, and a call with any host buffer synchronises the stream before
 *     it returns. The library never frees caller memory.
 *   - Every entry point returns MSD_OK (0) or a negative error code; the
 *     message of the last error is available from msd_last_error().
 *   - A context belongs to one device and is not thread-safe: calls on one
 *     context must not overlap.
 */
#ifndef MSD_H
#define MSD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MSD_OK                0
#define MSD_ERR_ARG          -1   /* null pointer or value out of range          */
#define MSD_ERR_SHAPE        -2   /* sizes inconsistent or beyond built limits   */
#define MSD_ERR_CUDA         -3   /* a CUDA runtime call failed                  */
#define MSD_ERR_TIMEOUT      -4   /* a bounded device-side wait expired          */
#define MSD_ERR_REF_SINGULAR -5   /* D_0^dag phi singular for some walker         */
#define MSD_ERR_STATE        -6   /* Hamiltonian or trial not set yet            */
#define MSD_ERR_NOMEM        -7   /* device or host allocation failed            */

/* Arithmetic of the Cholesky-vector contractions and per-determinant energy
   terms. The reference inverse (D_0^dag phi)^-1, the k x k minor
   determinants and the final reductions are FP64 in both modes. */
#define MSD_FP64  0
#define MSD_MIXED 1

/* Built limits. */
#define MSD_MAX_ELECTRONS   64   /* N_s per spin                                 */
#define MSD_MAX_LEVEL        6   /* excitation level per spin of any determinant */
#define MSD_MAX_ACTIVE     112   /* n_h * n_p per spin (see msd_info)            */

typedef struct msd_ctx msd_ctx;

/* Create a context for M orbitals and n_alpha, n_beta electrons on CUDA
   device `device`, with precision MSD_FP64 or MSD_MIXED.
   *out receives the context (NULL on failure). */
int msd_create(msd_ctx** out, int M, int n_alpha, int n_beta, int precision, int device);

/* Release the context and all device memory it owns. NULL is a no-op. */
void msd_destroy(msd_ctx* ctx);

/* Message of the last error on this context (or of the last failed
   msd_create when ctx is NULL). Valid until the next call on ctx. */
const char* msd_last_error(const msd_ctx* ctx);

/* Hamiltonian (Eq. 2-3). Host pointers; the data are copied.
     h1 [2][M][M]       one-body matrix per spin, symmetric
     e0                 constant energy
     L  [n_chol][M][M]  Cholesky vectors, each symmetric
   May be called again to replace the Hamiltonian. */
int msd_set_hamiltonian(msd_ctx* ctx, const double* h1, double e0, int n_chol,
                        const double* L);

/* CI trial (Sec. II B). Host pointers; the data are copied.
     coeff [n_det]           real CI coefficients c_I
     occ_a [n_det][n_alpha]  occupied alpha orbitals of D_I, strictly ascending
     occ_b [n_det][n_beta]   occupied beta orbitals, strictly ascending
   Determinant 0 is the reference D_0; every determinant must differ from it
   by at most MSD_MAX_LEVEL orbitals per spin. Errors: MSD_ERR_ARG for
   unsorted, repeated or out-of-range orbitals, MSD_ERR_SHAPE for a level
   above MSD_MAX_LEVEL or an active block above MSD_MAX_ACTIVE. */
int msd_set_trial(msd_ctx* ctx, int n_det, const double* coeff, const int32_t* occ_a,
                  const int32_t* occ_b);

/* Select MSD_FP64 or MSD_MIXED for subsequent calls. */
int msd_set_precision(msd_ctx* ctx, int precision);

/* Trial overlap of n_w walkers (Sec. II A-B, overlap).
     phi_a [n_w][M][n_alpha], phi_b [n_w][M][n_beta]   complex, host or device
     ovlp      [n_w]  O_T = <Psi_T|phi> = O_0 * sum_I c_I r_I, complex
     ratio_sum [n_w]  sum_I c_I r_I with r_I = <D_I|phi>/<D_0|phi> (may be NULL)
   stream: a cudaStream_t (NULL = legacy default stream). */
int msd_overlap(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                double* ovlp, double* ratio_sum, void* stream);

/* Overlap ratio of every trial determinant (the get_dets quantity of the
   paper's Sec. III "Implementation"):
     ratios [n_w][n_det]  r_I = <D_I|phi> / <D_0|phi>, complex
     ref_ovlp [n_w]       <D_0|phi>, complex (may be NULL) */
int msd_det_ratios(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                   double* ratios, double* ref_ovlp, void* stream);

/* Force-bias numerators (Eq. 7 without its -sqrt(dt) prefactor, which the
   propagator applies):
     vbias [n_w][n_chol]  sum_s tr(L_g G_T^s), complex, where G_T^s is the
                          mixed Green's function <Psi_T|a+_ps a_qs|phi>/O_T
     ovlp  [n_w]          O_T (may be NULL) */
int msd_force_bias(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                   double* vbias, double* ovlp, void* stream);

/* Mixed-estimator local energy (Sec. III, energy estimator):
     e_loc [n_w]  E_L = <Psi_T|H|phi> / <Psi_T|phi>, complex
     ovlp  [n_w]  O_T (may be NULL) */
int msd_local_energy(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                     double* e_loc, double* ovlp, void* stream);

/* Mixed one-body reduced density matrix (the mixed estimator of the
   one-particle density, the first property estimator beyond the energy,
   Sec. IV; the quantity whose contraction with L_g is the force bias, Eq. 7):
     rdm [n_w][2][M][M]  G_T^s[p][q] = <Psi_T|a+_ps a_qs|phi> / <Psi_T|phi>,
                         complex, spin alpha then beta (host or device)
   computed as the rank-k update of the reference Green's function by the
   cofactor matrix of all determinants (Sec. III, reduce_CI). Rows outside
   the reference orbitals and the trial's particles are zero. In mixed
   precision the cofactor sums come from FP32 inverse minors (relative error
   about 1e-6 of max |G_T|). */
int msd_rdm1(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, double* rdm, void* stream);

/* Overlap, force bias and local energy in one pass: the reference inverse,
   the excitation-string minors and the CI weights are computed once and
   shared. Outputs as in msd_overlap (ovlp), msd_force_bias (vbias) and
   msd_local_energy (e_loc); any of them may be NULL, but not all. */
int msd_evaluate(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                 double* ovlp, double* vbias, double* e_loc, void* stream);

/* Per-determinant local energies for sampled (walker, determinant) pairs,
   the localisation output of the energy path (Sec. III energy estimator:
   E_I = <D_I|H|phi> / <D_I|phi>, whose c_I r_I-weighted mean is E_L). The
   library runs the energy path up to its per-walker intermediates (the
   reference energy, the same-spin Gram matrices and linear terms, the
   opposite-spin Gram matrix, the inverse minors of every excitation string)
   and evaluates each requested E_I from them with the same per-determinant
   arithmetic, in the context's precision.
     n_pairs          number of pairs (0 is a no-op)
     w_idx, det_idx   [n_pairs] HOST int32 arrays: walker index in [0, n_w)
                      and determinant index in the trial list [0, n_det)
     e_det            [n_pairs] complex E_I (host or device)
   MSD_ERR_ARG for an index out of range or device index arrays. */
int msd_det_energies(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, int n_pairs,
                     const int32_t* w_idx, const int32_t* det_idx, double* e_det, void* stream);

/* Introspection. Keys: */
#define MSD_INFO_N_DET          1
#define MSD_INFO_N_CHOL         2
#define MSD_INFO_N_STRINGS_A    3   /* distinct alpha excitation strings        */
#define MSD_INFO_N_STRINGS_B    4
#define MSD_INFO_N_HOLES_A      5   /* n_h: orbitals of D_0 that are ever holes */
#define MSD_INFO_N_PARTS_A      6   /* n_p: orbitals that are ever particles    */
#define MSD_INFO_N_HOLES_B      7
#define MSD_INFO_N_PARTS_B      8
#define MSD_INFO_WORKSPACE_BYTES 9  /* device workspace currently held          */
#define MSD_INFO_WALKER_CHUNK  10   /* walkers per internal pass                */
#define MSD_INFO_EXACT_REFERENCE 11 /* 1 if the next mixed energy takes the exact
                                       reference sums (msd_set_exact_reference) */
int msd_info(const msd_ctx* ctx, int key, long long* value);

/* Per-kernel timing with CUDA events on the launching stream. When enabled,
   every kernel launch is bracketed by events; msd_kernel_stat synchronises
   on them and reports, per kernel name, the launch count and total device
   milliseconds since the last msd_reset_stats. */
int msd_set_timing(msd_ctx* ctx, int enable);
int msd_reset_stats(msd_ctx* ctx);
int msd_kernel_count(const msd_ctx* ctx);
int msd_kernel_stat(msd_ctx* ctx, int index, const char** name, long long* launches,
                    double* total_ms);

/* Limit the device workspace (bytes) the context may hold; larger walker
   batches are processed in chunks. 0 restores the default (16 GiB). */
int msd_set_workspace_limit(msd_ctx* ctx, size_t bytes);

/* With sync = 1 (the default) every call synchronises its stream before
   returning and reports device-side errors (a singular reference, an
   expired wait) in its return code. With sync = 0 calls on device buffers
   return as soon as the work is queued; device-side errors are then
   reported by the next synchronising call. */
int msd_set_sync(msd_ctx* ctx, int sync);

/* Mixed precision only: with fused = 1 (the default) the Cholesky
   contraction of the local energy (Eq. 10-12, F = G L_g restricted to the
   rows of the reference orbitals) and its per-(walker, vector) epilogue run
   as one persistent tensor-core kernel whose FP32 products stay on chip;
   with fused = 0 they run as a tensor-core GEMM writing F to device memory
   followed by a separate epilogue kernel. Same arithmetic and rounding
   points; results agree to FP32 summation order. Shapes the fused kernel
   does not support (2N > 128 rows per walker, tiles beyond 227 KB of shared
   memory) take the unfused path. */
int msd_set_fused(msd_ctx* ctx, int fused);

/* Budget of the device-side waits of the tensor-core kernels (a consumer
   warp waiting for the producer's copies or products), in nanoseconds of the
   GPU's global timer; the default is 2000000000 (about 2 s). When a wait
   exceeds it the kernel stops its pipeline, lets its own copies and products
   in flight complete, frees its tensor memory and returns; the call reports
   MSD_ERR_TIMEOUT and the context stays usable. 0 makes every such wait a
   single poll (the first wait that finds its data not yet there expires),
   which exercises this path. */
int msd_set_wait_budget(msd_ctx* ctx, unsigned long long ns);

/* Mixed precision only: with on = 1 (the default) the reference-determinant
   part of the local energy (Sec. II A, the generalized Wick theorem for the
   reference D_0: one-body, Coulomb and exchange energy of G, the dominant
   part of E_L) is computed to FP64 accuracy. Its terms linear in
   dG = G - D_0 D_0^T are one-body contractions with constant matrices
   (FP64); its quadratic terms sum_g tr(L_g dG)^2 and sum_g tr(dT_g dT_g),
   dT_g = (dG L_g)[occ0][occ0], are one product of the walker's dG with a
   constant exchange-integral matrix, evaluated on the tensor cores by an
   exact-integer split of both operands into BF16 slices (about 35 bits).
   With on = 0 these sums come from the FP32 traces of the 3xTF32
   contraction (relative error about 1e-7 of the energy). The constant
   operand takes about 10 (N (M - N) + n_chol) N (M - N) bytes per spin;
   spins with N (M - N) above 16384 always take the FP32 traces. */
int msd_set_exact_reference(msd_ctx* ctx, int on);

/* Mixed precision only: with on = 1 the Gram matrices of the energy's Gram
   form, K^{st} = sum_g Lambda^s_g (x) Lambda^t_g over the Cholesky vectors,
   are formed on the tensor cores (the Lambda rows transposed once per call,
   then a two-way TF32 split of both operands, three products, FP32
   accumulation in tensor memory) when 2 n_h n_p <= 256 per spin and n_chol
   is a multiple of 4; with on = 0 (the default), or other shapes, by FP32
   FMAs. On the iron-sulfur shape the tensor-core form takes 1.10 against
   1.67 ms per step, and raises the local energy's error at a chemical energy
   scale from 2.9e-6 to 3.4e-6 Ha (maximum over 640 walkers). */
int msd_set_tensor_gram(msd_ctx* ctx, int on);

/* Mixed precision, msd_evaluate / msd_local_energy only: with on = 1 (the
   default) the energy's per-walker sums that follow the Cholesky
   contraction (one-body terms, the exactly split reference sums, the sums of
   Lambda and Xi, the Gram matrices) run on a second stream of this context
   (created on first use at the device's highest stream priority),
   concurrently with the string minors and weights (bound by FP64
   arithmetic) on the caller's stream; then the force bias runs on the
   second stream, concurrently with the per-determinant terms, which wait for
   the energy sums. On the iron-sulfur shape: 23.54 against 24.60 ms per
   step. The call stays ordered on the caller's stream: the second stream
   waits for the caller's stream at each fork, and the caller's stream waits
   for the second stream before the per-determinant terms (energy sums) and
   again at the end of each walker chunk (force bias), also on an error
   return. The results are identical with on = 0, which runs every kernel on
   the caller's stream. */
int msd_set_stream_overlap(msd_ctx* ctx, int on);

/* The form of the opposite-spin exchange term of the local energy (Sec. III,
   the alpha-beta part of the two-body Wick contraction),
     sum_I c_I r_a r_b sum_ij sum_kl Ba[i][j] Bb[k][l] K^ab[(h_j,p_i)][(h_l,p_k)].
   form = 0: every determinant takes the double sum (k_a^2 k_b^2 gathers of
   K^ab); form = 1 (mixed precision only): the inner sum is formed once per
   beta string, Y_b[x] = sum_kl Bb[k][l] K^ab[x][(h_l,p_k)], so a
   determinant costs k_a^2; form = 2: within each excitation-level bucket
   the determinants sharing one string (the side chosen per bucket when the
   trial is set) form a run, its projection P_s = sum_e Bs[e] K^ab[x_e][.]
   is formed once in shared memory and each determinant of the run costs
   k_o^2 (buckets with too few determinants per string keep the double sum);
   form = -1 (the default): 1 when a cost model over the trial's levels
   prefers it to the double sum, else 2. The forms differ by the order of
   the sums in the working precision only. A batch (msd_batch_create) sets
   its systems to 0, the form its persistent kernel implements. MSD_ERR_ARG
   for other values. */
int msd_set_pair_form(msd_ctx* ctx, int form);

/* Number of CUDA kernels the library has launched in this process (all
   contexts), for launch accounting by benchmarks. */
long long msd_launch_count(void);

/* ---- Propagation (Sec. II A, Eq. 7-12) ---------------------------------
   One phaseless AFQMC step of n_w walkers, in place, in FP64 (the overlaps
   and the force bias in the context's precision):
     vbias_g = <Psi_T|L_g|phi>/<Psi_T|phi>, xbar_g = -i sqrt(dt) vbias_g,
     phi'    = E T_n(V) E phi, E = exp(-dt h'/2), h' = h - 1/2 sum_g L_g L_g,
               V = i sqrt(dt) sum_g (x_g - xbar_g) L_g, T_n the Taylor series
               of exp to order taylor_order (1..16),
     S       = O_T(phi')/O_T(phi), I = S exp(x.xbar - xbar.xbar/2),
     w'      = w |I| max(0, cos arg S),
   then, if orthonormalize != 0, phi'^s <- Q with phi'^s = Q R (the diagonal
   of R real positive; weights are unaffected since S is computed first).
   phi_a, phi_b: device [n_w][M][N_s] complex (in/out); weights: device
   [n_w] double (in/out); x: device [n_w][n_chol] double, the Gaussian
   fields drawn by the caller; ratio: optional device [n_w] complex, S.
   Host pointers are rejected (MSD_ERR_ARG); dt <= 0 or an order outside
   1..16 is MSD_ERR_ARG; walker blocks beyond 200 KB (M N_s complex) are
   MSD_ERR_SHAPE. exp(-dt h'/2) is formed on the host once per dt (scaling
   and squaring of its Taylor series) and cached with the context. */
int msd_propagate(msd_ctx* ctx, int n_w, double* phi_a, double* phi_b, double* weights,
                  const double* x, double dt, int taylor_order, int orthonormalize,
                  double* ratio, void* stream);

/* ---- Batched independent systems ---------------------------------------
   Many systems (each its own context: uneven orbital, electron and
   determinant counts; one device and one precision for all) evaluated
   together. msd_batch_evaluate runs, for every system i, the overlap, force
   bias and dense energy steps of msd_evaluate (systems spread over eight
   concurrent streams, branches of the recorded graph), then the per-determinant
   energy terms of all systems in one persistent kernel that takes
   (system, walker, excitation bucket, block) work items from a queue, then
   the final sums. The first call with a given set of buffers runs eagerly and
   records the whole sequence as a CUDA graph; later calls with the same
   buffers (and no change to any context) replay it with one graph launch.
   Arrays are indexed by system: n_w[i] walkers, device pointers phi_a[i],
   phi_b[i], e_loc[i] (required), ovlp[i], vbias[i] (arrays or entries may be
   NULL). Every system's walkers must fit one workspace chunk (MSD_ERR_SHAPE
   otherwise). The contexts must outlive the batch; creating the batch sets
   each to the per-determinant opposite-spin form (msd_set_pair_form 0). */
typedef struct msd_batch msd_batch;
int msd_batch_create(msd_batch** out, msd_ctx* const* ctxs, int n_sys);
void msd_batch_destroy(msd_batch* b);
const char* msd_batch_last_error(const msd_batch* b);
int msd_batch_evaluate(msd_batch* b, const int* n_w, const double* const* phi_a,
                       const double* const* phi_b, double* const* ovlp, double* const* vbias,
                       double* const* e_loc, void* stream);
/* Autotuner: times every combination of the tensor-core output tile width
   (128, 256), resident CTAs per SM of the persistent kernel (1, 2, 4) and
   work-item order (0: by system, 1: largest work first, 2: walkers
   interleaved across systems) on the given inputs, keeps the fastest, and
   appends "key tile ctas order ms" to cache_path (a text file; may be NULL).
   A later call whose system shapes match a cached key applies it without
   timing. */
int msd_batch_autotune(msd_batch* b, const int* n_w, const double* const* phi_a,
                       const double* const* phi_b, double* const* ovlp, double* const* vbias,
                       double* const* e_loc, void* stream, const char* cache_path);
int msd_batch_config(const msd_batch* b, int* tile_n, int* ctas_per_sm, int* order);
int msd_batch_set_config(msd_batch* b, int tile_n, int ctas_per_sm, int order);
/* With enable = 1 the next eager run of the batch (the first call with new
   buffers or after msd_batch_set_config) brackets its persistent kernel with
   CUDA events on the call's stream; last_ms (may be NULL) receives the time
   of the last such run in milliseconds, or -1 if there is none. */
int msd_batch_time_persistent(msd_batch* b, int enable, double* last_ms);
/* 1 once a graph has been recorded for the current buffers, else 0. */
int msd_batch_graph_ready(const msd_batch* b);
/* Kernel nodes in the recorded graph (kernels one replay launches), or 0. */
long long msd_batch_graph_kernels(const msd_batch* b);

/* ---- Learned control variate --------------------------------------------
   (The paper has no counterpart.) A small MLP predicts the real part of the
   local energy from features of the reference Green's function (its
   non-zero rows, msd_features_rows, or its active-space block,
   msd_features);
   evaluated on every walker it serves as a control variate: the estimator
   mean_i f(x_i) + mean_{i in S}(E_L,i - f(x_i)) over a random subsample S
   stays unbiased while the exact path runs only on S. */

/* Features per walker: feat[w][s][p][q][c] = (Re, Im) of
   G^s[n_core + p][n_core + q], p, q < n_act (G = <a+_p a_q> of the reference
   determinant, Eq. 14), FP32, 4 * n_act^2 floats per walker; feat must be
   device memory. */
int msd_features(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, int n_core,
                 int n_act, float* feat, void* stream);

/* Features per walker: the non-zero rows of G (the rows of the reference
   determinant's occupied orbitals, all M columns), alpha then beta:
   feat[w * ld + 2 (j M + q) + c], 2 (N_a + N_b) M floats, the rest of the
   row (up to ld) zero. feat must be device memory. */
int msd_features_rows(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b, int ld,
                      float* feat, void* stream);

/* Network x (n_in) -> 3 hidden layers of `width` with GELU -> scalar; BF16
   weights and activations, FP32 accumulation on the tensor cores, FP32 master
   parameters. n_in and width must be multiples of 64 (MSD_ERR_SHAPE).
   Parameter layout (FP32): W0 [width][n_in], b0 [width], W1 [width][width],
   b1, W2 [width][width], b2, w3 [width], b3 [1]. */
typedef struct msd_mlp msd_mlp;
int msd_mlp_create(msd_mlp** out, int n_in, int width, int device);
void msd_mlp_destroy(msd_mlp* m);
const char* msd_mlp_last_error(const msd_mlp* m);
long long msd_mlp_param_count(const msd_mlp* m);
/* Host parameter copies; setting resets the optimiser state. */
int msd_mlp_set_params(msd_mlp* m, const float* params);
int msd_mlp_get_params(msd_mlp* m, float* params);
/* y[b] = f(x[b]) for x [batch][n_in] (device FP32) -> y [batch] (device). */
int msd_mlp_forward(msd_mlp* m, int batch, const float* x, float* y, void* stream);
/* Loss (1/B) sum_b (f(x_b) - t_b)^2 and its gradient with respect to every
   parameter (kept for msd_mlp_adam_step; copied to grads, device, if not
   NULL; loss a device scalar, may be NULL). batch <= 65536. */
int msd_mlp_grad(msd_mlp* m, int batch, const float* x, const float* target, float* grads,
                 float* loss, void* stream);
/* One Adam step (Kingma and Ba) with the last gradients. */
int msd_mlp_adam_step(msd_mlp* m, float lr, float beta1, float beta2, float eps, void* stream);

/* Trial overlap without any device allocation during the call. The paper
   has no counterpart: this serves callers that cannot let a library call
   cudaMalloc / cudaFree, such as a framework that owns all device memory
   through its own allocator or a fixed budget, or a latency-critical loop
   that must not take the synchronisation those calls can imply.
   Same arguments and results as msd_overlap, with these differences:
     - phi_a, phi_b, ovlp and ratio_sum must be device pointers
       (MSD_ERR_ARG otherwise);
     - the scratch is a file-scope device array of MSD_STATIC_SCRATCH_BYTES
       held by every GPU that loads the library until the process exits;
       walkers are processed in chunks that fit it, and a request whose
       single walker needs more scratch than that is rejected with
       MSD_ERR_SHAPE;
     - the first call on a device resolves the array's device address
       (cudaGetSymbolAddress); make that first call before any stream
       capture;
     - all calls share the array and each leaves its contents behind, so
       calls that overlap on the GPU (other streams, other host threads)
       race: serialise them.
   The context must have been created and set up beforehand (those calls
   allocate). */
#define MSD_STATIC_SCRATCH_BYTES (64u << 20)
int msd_overlap_noalloc(msd_ctx* ctx, int n_w, const double* phi_a, const double* phi_b,
                        double* ovlp, double* ratio_sum, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MSD_H */
