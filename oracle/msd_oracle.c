/*
 * CPU oracle for the multi-Slater-determinant AFQMC hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path calls this code: only
 * the tests, the smoke check and the CPU-baseline leg of the benchmark load
 * it. It shares no code, header or table with the CUDA library.
 *
 * It follows the naive approach the paper names as the slow alternative
 * (Sec. II B: one single-determinant evaluation per trial determinant, linear
 * in the number of determinants) in plain complex double precision:
 *
 *   overlap     O_I = <D_I|phi> = det(D_I^dag phi_a) det(D_I^dag phi_b)
 *               (Eq. 13, overlap of two Slater determinants), computed as
 *               a full N x N determinant by LU with partial pivoting;
 *   Green's fn  G_I[p][q] = <D_I|a+_p a_q|phi> / <D_I|phi>
 *               = [phi (D_I^dag phi)^-1 D_I^dag]_{qp}   (Eq. 14);
 *   energy      E_I = <D_I|H|phi> / <D_I|phi> from G_I by the generalized
 *               Wick theorem (Sec. II A), for
 *               H = e0 + sum_{pq,s} h_pq a+_ps a_qs
 *                   + 1/2 sum_g sum_{pqrs,st} L^g_pq L^g_rs a+_ps a+_rt a_st a_qs
 *               (Eq. 2 with (pq|rs) = sum_g L^g_pq L^g_rs, Sec. II A), i.e.
 *               E_I = e0 + sum_s tr(h G_I^s)
 *                     + 1/2 sum_g [ (sum_s tr(L_g G_I^s))^2
 *                                   - sum_s tr(L_g G_I^s L_g G_I^s) ],
 *               with tr(X G) = sum_pq X_pq G_pq;
 *   trial sums  O_T = sum_I c_I O_I,  E_L = sum_I c_I O_I E_I / O_T,
 *               G_T = sum_I c_I O_I G_I / O_T (Eq. 15, Psi_T = sum c_I D_I),
 *               force-bias numerator vbias_g = sum_s tr(L_g G_T^s) (Eq. 7
 *               without its -sqrt(dt) prefactor).
 *
 * Since D_I^dag has non-zero columns only at the occupied orbitals occ_I,
 * G_I has non-zero rows only at occ_I; the sums below run over those rows.
 *
 * Layouts: complex arrays are interleaved (re, im) doubles. phi_s is
 * [M][N_s] row-major per walker; h1 is [2][M][M]; L is [n_chol][M][M]
 * (each L_g symmetric); occupation lists are sorted ascending.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

struct problem {
    int M, n[2], n_chol;
    const double* h1;   /* [2][M][M] */
    double e0;
    const double* L;    /* [n_chol][M][M] */
};

/* LU factorisation with partial pivoting of the n x n matrix a (in place).
   Returns det(a); on an exactly zero pivot returns 0 and leaves inv unset. */
static cplx lu_det_inverse(int n, cplx* a, cplx* inv, int* piv, cplx* col)
{
    cplx det = 1.0;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = cabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = cabs(a[i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return 0.0;
        if (p != k) {
            for (int j = 0; j < n; ++j) {
                cplx t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t;
            }
            det = -det;
        }
        det *= a[k * n + k];
        for (int i = k + 1; i < n; ++i) {
            cplx f = a[i * n + k] / a[k * n + k];
            a[i * n + k] = f;
            for (int j = k + 1; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
        }
    }
    if (!inv) return det;
    /* solve a x = e_c for every column c */
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) col[i] = (i == c) ? 1.0 : 0.0;
        for (int k = 0; k < n; ++k) {            /* apply the row swaps */
            cplx t = col[k]; col[k] = col[piv[k]]; col[piv[k]] = t;
        }
        for (int i = 0; i < n; ++i)              /* unit lower triangle */
            for (int k = 0; k < i; ++k) col[i] -= a[i * n + k] * col[k];
        for (int i = n - 1; i >= 0; --i) {       /* upper triangle */
            for (int k = i + 1; k < n; ++k) col[i] -= a[i * n + k] * col[k];
            col[i] /= a[i * n + i];
        }
        for (int i = 0; i < n; ++i) inv[i * n + c] = col[i];
    }
    return det;
}

struct scratch {
    cplx *S, *Sinv, *col, *GI, *GL;
    int* piv;
};

static int scratch_alloc(struct scratch* w, int M, int nmax)
{
    w->S = malloc(sizeof(cplx) * nmax * nmax);
    w->Sinv = malloc(sizeof(cplx) * nmax * nmax);
    w->col = malloc(sizeof(cplx) * nmax);
    w->GI = malloc(sizeof(cplx) * 2 * nmax * M);
    w->GL = malloc(sizeof(cplx) * nmax * nmax);
    w->piv = malloc(sizeof(int) * nmax);
    return (w->S && w->Sinv && w->col && w->GI && w->GL && w->piv) ? 0 : -1;
}

static void scratch_free(struct scratch* w)
{
    free(w->S); free(w->Sinv); free(w->col); free(w->GI); free(w->GL); free(w->piv);
}

/* One determinant pair (occ[0], occ[1]) against one walker (phi[0], phi[1]).
   Writes O_I, E_I and the non-zero rows of G_I^s into w->GI:
   GI[s][j][q] = G_I^s[occ_s[j]][q]. Returns 0, or 1 if O_I = 0 exactly
   (E_I and G_I are then undefined and left unset). */
static int det_terms(const struct problem* P, const int* const occ[2],
                     const cplx* const phi[2], struct scratch* w,
                     cplx* ovlp, cplx* energy)
{
    const int M = P->M;
    cplx O = 1.0;
    for (int s = 0; s < 2; ++s) {
        const int n = P->n[s];
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) w->S[i * n + j] = phi[s][occ[s][i] * n + j];
        cplx d = lu_det_inverse(n, w->S, w->Sinv, w->piv, w->col);
        if (d == 0.0) { *ovlp = 0.0; return 1; }
        O *= d;
        /* G_I^s[occ_j][q] = (phi S^-1)[q][j] */
        cplx* G = w->GI + (size_t)s * P->n[0] * M;
        for (int q = 0; q < M; ++q)
            for (int j = 0; j < n; ++j) {
                cplx acc = 0.0;
                for (int k = 0; k < n; ++k) acc += phi[s][q * n + k] * w->Sinv[k * n + j];
                G[j * M + q] = acc;
            }
    }
    *ovlp = O;
    if (!energy) return 0;
    cplx E = P->e0;
    for (int s = 0; s < 2; ++s) {
        const int n = P->n[s];
        const double* h = P->h1 + (size_t)s * M * M;
        const cplx* G = w->GI + (size_t)s * P->n[0] * M;
        for (int j = 0; j < n; ++j)
            for (int q = 0; q < M; ++q) E += h[occ[s][j] * M + q] * G[j * M + q];
    }
    cplx two = 0.0;
    for (int g = 0; g < P->n_chol; ++g) {
        const double* Lg = P->L + (size_t)g * M * M;
        cplx J = 0.0, X = 0.0;
        for (int s = 0; s < 2; ++s) {
            const int n = P->n[s];
            const cplx* G = w->GI + (size_t)s * P->n[0] * M;
            for (int j = 0; j < n; ++j)
                for (int q = 0; q < M; ++q) J += Lg[occ[s][j] * M + q] * G[j * M + q];
            /* tr(L G L G) = sum_{i,j in occ} (G L)[i][j] (G L)[j][i] */
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    cplx acc = 0.0;
                    for (int q = 0; q < M; ++q) acc += G[i * M + q] * Lg[q * M + occ[s][j]];
                    w->GL[i * n + j] = acc;
                }
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) X += w->GL[i * n + j] * w->GL[j * n + i];
        }
        two += J * J - X;
    }
    *energy = E + 0.5 * two;
    return 0;
}

static int nmax_of(const struct problem* P) { return P->n[0] > P->n[1] ? P->n[0] : P->n[1]; }

/* Single determinant pair against one walker: O_I, E_I and the full
   G_I^s (both spins, [2][M][M], may be NULL). Returns 0, 1 if O_I = 0,
   -1 on allocation failure. */
int oracle_det(int M, int n_alpha, int n_beta, const int* occ_a, const int* occ_b,
               const double* h1, double e0, int n_chol, const double* L,
               const double* phi_a, const double* phi_b,
               double* ovlp, double* energy, double* G_out)
{
    struct problem P = {M, {n_alpha, n_beta}, n_chol, h1, e0, L};
    struct scratch w;
    if (scratch_alloc(&w, M, nmax_of(&P))) { scratch_free(&w); return -1; }
    const int* occ[2] = {occ_a, occ_b};
    const cplx* phi[2] = {(const cplx*)phi_a, (const cplx*)phi_b};
    cplx O = 0.0, E = 0.0;
    int rc = det_terms(&P, occ, phi, &w, &O, energy ? &E : NULL);
    memcpy(ovlp, &O, sizeof O);
    if (energy) memcpy(energy, &E, sizeof E);
    if (G_out && rc == 0) {
        cplx* G = (cplx*)G_out;
        memset(G, 0, sizeof(cplx) * 2 * M * M);
        for (int s = 0; s < 2; ++s) {
            const cplx* GI = w.GI + (size_t)s * P.n[0] * M;
            for (int j = 0; j < P.n[s]; ++j)
                for (int q = 0; q < M; ++q) G[(size_t)s * M * M + occ[s][j] * M + q] = GI[j * M + q];
        }
    }
    scratch_free(&w);
    return rc;
}

/* The whole trial against n_w walkers. Outputs (each may be NULL):
     ovlp   [n_w]            O_T
     e_loc  [n_w]            E_L
     vbias  [n_w][n_chol]    sum_s tr(L_g G_T^s)
     G_T    [n_w][2][M][M]   mixed Green's function
     det_ovlp [n_w][n_det]   O_I
     det_e    [n_w][n_det]   E_I
   n_threads <= 0 uses the OpenMP default. Returns 0, -1 on allocation
   failure, or 1 + (walker index) of a walker with some O_I = 0 exactly. */
int oracle_msd(int M, int n_alpha, int n_beta, int n_det, const double* coeff,
               const int* occ_a, const int* occ_b, const double* h1, double e0,
               int n_chol, const double* L, int n_w, const double* phi_a,
               const double* phi_b, double* ovlp, double* e_loc, double* vbias,
               double* G_T, double* det_ovlp, double* det_e, int n_threads)
{
    struct problem P = {M, {n_alpha, n_beta}, n_chol, h1, e0, L};
    const int need_e = (e_loc != NULL) || (det_e != NULL);
    const int need_g = (vbias != NULL) || (G_T != NULL);
    const size_t gsz = (size_t)2 * M * M;
#ifdef _OPENMP
    int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    int nt = 1;
    (void)n_threads;
#endif
    cplx* accO = calloc((size_t)nt, sizeof(cplx));
    cplx* accE = calloc((size_t)nt, sizeof(cplx));
    cplx* accG = need_g ? calloc((size_t)nt * gsz, sizeof(cplx)) : NULL;
    cplx* GT = need_g ? malloc(gsz * sizeof(cplx)) : NULL;
    int* bad = calloc((size_t)nt, sizeof(int));
    if (!accO || !accE || !bad || (need_g && (!accG || !GT))) {
        free(accO); free(accE); free(accG); free(GT); free(bad);
        return -1;
    }
    int status = 0;
    for (int wk = 0; wk < n_w && status == 0; ++wk) {
        const cplx* phi[2] = {(const cplx*)phi_a + (size_t)wk * M * n_alpha,
                              (const cplx*)phi_b + (size_t)wk * M * n_beta};
        memset(accO, 0, sizeof(cplx) * nt);
        memset(accE, 0, sizeof(cplx) * nt);
        if (need_g) memset(accG, 0, sizeof(cplx) * nt * gsz);
        memset(bad, 0, sizeof(int) * nt);
#pragma omp parallel num_threads(nt)
        {
#ifdef _OPENMP
            const int t = omp_get_thread_num();
#else
            const int t = 0;
#endif
            struct scratch w;
            int ok = scratch_alloc(&w, M, nmax_of(&P)) == 0;
            if (!ok) bad[t] = -1;
#pragma omp for schedule(static)
            for (int d = 0; d < n_det; ++d) {
                if (!ok) continue;
                const int* occ[2] = {occ_a + (size_t)d * n_alpha, occ_b + (size_t)d * n_beta};
                cplx O = 0.0, E = 0.0;
                if (det_terms(&P, occ, phi, &w, &O, need_e ? &E : NULL)) { bad[t] = 1; continue; }
                const cplx cO = coeff[d] * O;
                accO[t] += cO;
                accE[t] += cO * E;
                if (det_ovlp) ((cplx*)det_ovlp)[(size_t)wk * n_det + d] = O;
                if (det_e) ((cplx*)det_e)[(size_t)wk * n_det + d] = E;
                if (need_g) {
                    cplx* acc = accG + (size_t)t * gsz;
                    for (int s = 0; s < 2; ++s) {
                        const cplx* GI = w.GI + (size_t)s * P.n[0] * M;
                        for (int j = 0; j < P.n[s]; ++j)
                            for (int q = 0; q < M; ++q)
                                acc[(size_t)s * M * M + occ[s][j] * M + q] += cO * GI[j * M + q];
                    }
                }
            }
            scratch_free(&w);
        }
        for (int t = 0; t < nt; ++t) {
            if (bad[t] < 0) status = -1;
            else if (bad[t] > 0 && status == 0) status = 1 + wk;
        }
        cplx OT = 0.0, num = 0.0;
        for (int t = 0; t < nt; ++t) { OT += accO[t]; num += accE[t]; }
        if (ovlp) ((cplx*)ovlp)[wk] = OT;
        if (e_loc) ((cplx*)e_loc)[wk] = num / OT;
        if (need_g) {
            for (size_t i = 0; i < gsz; ++i) {
                cplx a = 0.0;
                for (int t = 0; t < nt; ++t) a += accG[(size_t)t * gsz + i];
                GT[i] = a / OT;
            }
            if (G_T) memcpy((cplx*)G_T + (size_t)wk * gsz, GT, gsz * sizeof(cplx));
            if (vbias) {
                for (int g = 0; g < n_chol; ++g) {
                    const double* Lg = L + (size_t)g * M * M;
                    cplx v = 0.0;
                    for (int s = 0; s < 2; ++s)
                        for (int pq = 0; pq < M * M; ++pq) v += Lg[pq] * GT[(size_t)s * M * M + pq];
                    ((cplx*)vbias)[(size_t)wk * n_chol + g] = v;
                }
            }
        }
    }
    free(accO); free(accE); free(accG); free(GT); free(bad);
    return status;
}
