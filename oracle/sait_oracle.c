/*
 * SAIT oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of what the GPU path
 * computes, written from the paper (Z. Lu, "A sparse approximate inverse for
 * triangular matrices based on Jacobi iteration", arXiv 2106.12836) and from
 * the textbook algorithms it relies on.  It shares no code, header, table or
 * helper with the CUDA library; only tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.
 *
 * Compile with -O2 -ffp-contract=off: every fused multiply-add below is an
 * explicit fma() call, every other product is rounded on its own.
 *
 * Status codes returned by every entry point:
 *   0 ok, 1 invalid argument, 2 not triangular, 3 zero or non-finite pivot,
 *   4 out of memory, 5 not converged, 6 breakdown.
 *
 * Drop rules (argument drop_kind of ora_sait):
 *   0 none     keep every structural entry of T~M + I
 *   1 abs      Algorithm 2 (SAIT_Thr): drop |v| < tau
 *   2 rowrel   drop |v| < tau * max_j |v_ij| of the current row (diagonal included)
 *   3 pattern  Algorithm 3 (SAIT_Pat): p undropped iterations fix the pattern S,
 *              the remaining iterations drop every entry outside S
 *   4 hybrid   the hybrid strategy the paper's source leaves commented out after
 *              Algorithm 3: p undropped iterations, then drop |v| < tau
 * The diagonal is never dropped (Section 3: the unit diagonal keeps M full rank).
 *
 * Parity pins: see tests/test_oracle_pins.py.  Every function here is pinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_OK 0
#define ORA_INVALID 1
#define ORA_NOT_TRIANGULAR 2
#define ORA_ZERO_PIVOT 3
#define ORA_OOM 4
#define ORA_NOT_CONVERGED 5
#define ORA_BREAKDOWN 6

typedef struct {
    int64_t n, nnz, cap;
    int32_t *rp;
    int32_t *ci;
    double *va;
} ora_mat;

void ora_free(ora_mat *m)
{
    if (!m) return;
    free(m->rp);
    free(m->ci);
    free(m->va);
    m->rp = NULL; m->ci = NULL; m->va = NULL;
    m->n = m->nnz = m->cap = 0;
}

static int mat_init(ora_mat *m, int64_t n, int64_t cap)
{
    m->n = n; m->nnz = 0; m->cap = cap > 16 ? cap : 16;
    m->rp = (int32_t *)malloc((size_t)(n + 1) * sizeof(int32_t));
    m->ci = (int32_t *)malloc((size_t)m->cap * sizeof(int32_t));
    m->va = (double *)malloc((size_t)m->cap * sizeof(double));
    if (!m->rp || !m->ci || !m->va) { ora_free(m); return ORA_OOM; }
    m->rp[0] = 0;
    return ORA_OK;
}

static int mat_push(ora_mat *m, int32_t c, double v)
{
    if (m->nnz == m->cap) {
        int64_t cap = m->cap * 2;
        int32_t *ci = (int32_t *)realloc(m->ci, (size_t)cap * sizeof(int32_t));
        if (!ci) return ORA_OOM;
        m->ci = ci;
        double *va = (double *)realloc(m->va, (size_t)cap * sizeof(double));
        if (!va) return ORA_OOM;
        m->va = va;
        m->cap = cap;
    }
    m->ci[m->nnz] = c;
    m->va[m->nnz] = v;
    m->nnz++;
    return ORA_OK;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* Sparse matrix-vector product y = A x, summed in stored order.            */
/* ------------------------------------------------------------------------ */
void ora_spmv(int64_t n, const int32_t *rp, const int32_t *ci, const double *va,
              const double *x, double *y)
{
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) s += va[e] * x[ci[e]];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Forward (lower) / backward (upper) substitution T x = b.  The exact      */
/* triangular solve the paper's SAIT apply replaces (Section 3.1).          */
/* ------------------------------------------------------------------------ */
int ora_trisolve(int64_t n, const int32_t *rp, const int32_t *ci, const double *va,
                 int lower, const double *b, double *x)
{
    for (int64_t t = 0; t < n; t++) {
        int64_t i = lower ? t : n - 1 - t;
        double s = b[i], d = 0.0;
        int have_d = 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            int64_t j = ci[e];
            if (j == i) { d = va[e]; have_d = 1; }
            else if ((lower && j < i) || (!lower && j > i)) s -= va[e] * x[j];
            else return ORA_NOT_TRIANGULAR;
        }
        if (!have_d || d == 0.0 || !isfinite(d)) return ORA_ZERO_PIVOT;
        x[i] = s / d;
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* ILU(0), IKJ variant (Saad, Iterative Methods for Sparse Linear Systems,   */
/* 2nd ed., Algorithm 10.4).  Overwrites a (values of A in A's pattern)      */
/* with L (strict lower part, unit diagonal implied) and U (upper part with  */
/* the diagonal).  The paper takes level-0 ILU factors as the triangular    */
/* inputs of SAIT (Section 4).  Columns must be sorted ascending.            */
/* ------------------------------------------------------------------------ */
int ora_ilu0(int64_t n, const int32_t *rp, const int32_t *ci, double *a)
{
    int64_t *pos = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *dpos = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!pos || !dpos) { free(pos); free(dpos); return ORA_OOM; }
    int st = ORA_OK;
    for (int64_t i = 0; i < n; i++) {
        pos[i] = -1;
        dpos[i] = -1;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            if (e > rp[i] && ci[e] <= ci[e - 1]) { st = ORA_INVALID; goto done; }
            if (ci[e] == i) dpos[i] = e;
        }
        if (dpos[i] < 0) { st = ORA_ZERO_PIVOT; goto done; }
    }
    for (int64_t i = 0; i < n; i++) {
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) pos[ci[e]] = e;
        for (int32_t e = rp[i]; e < rp[i + 1] && ci[e] < i; e++) {
            int64_t k = ci[e];
            double ukk = a[dpos[k]];
            if (ukk == 0.0 || !isfinite(ukk)) { st = ORA_ZERO_PIVOT; goto done; }
            a[e] = a[e] / ukk;                       /* a_ik := a_ik / a_kk */
            for (int32_t f = dpos[k] + 1; f < rp[k + 1]; f++) {
                int64_t p = pos[ci[f]];              /* (i,j) in NZ(A), j > k */
                if (p >= 0) a[p] = fma(-a[e], a[f], a[p]);   /* a_ij -= a_ik a_kj */
            }
        }
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) pos[ci[e]] = -1;
        if (a[dpos[i]] == 0.0 || !isfinite(a[dpos[i]])) { st = ORA_ZERO_PIVOT; goto done; }
    }
done:
    free(pos);
    free(dpos);
    return st;
}

/* ------------------------------------------------------------------------ */
/* ILUT(tau, lfil) (Saad, Iterative Methods for Sparse Linear Systems, 2nd   */
/* ed., Algorithm 10.6), the threshold ILU whose factors the paper's         */
/* experiments also feed to SAIT (level-1 and threshold factors, Section 4). */
/* Row i:                                                                   */
/*   w := a_i*,  tau_i := tau * ||a_i*||_2  (sum of squares in column order) */
/*   for k < i with w_k != 0, in increasing k (fill included):              */
/*       w_k := w_k / u_kk;  drop w_k if |w_k| < tau_i  (first rule)        */
/*       if w_k != 0:  w_j := fma(-w_k, u_kj, w_j)  for u_kj != 0, j > k    */
/*   second rule: drop |w_j| < tau_i, then keep the lfil largest |w_j| of   */
/*   the L part (j < i) and of the U part (j > i); the diagonal is always   */
/*   kept.  Ties in |w_j| keep the smaller column.                          */
/* Output: combined CSR, strict lower part of L (unit diagonal implied) and  */
/* U with its diagonal, columns ascending.  A zero or non-finite pivot      */
/* u_ii returns ORA_ZERO_PIVOT.                                             */
/* ------------------------------------------------------------------------ */
static int keep_largest(const int32_t *cols, const double *w, int cnt, int lfil, int32_t *out)
{
    /* out gets the kept columns (rank < lfil), ascending; returns how many */
    int m = 0;
    for (int a = 0; a < cnt; a++) {
        double va = fabs(w[cols[a]]);
        int rank = 0;
        for (int b = 0; b < cnt; b++) {
            double vb = fabs(w[cols[b]]);
            if (vb > va || (vb == va && cols[b] < cols[a])) rank++;
        }
        if (rank < lfil) out[m++] = cols[a];
    }
    qsort(out, (size_t)m, sizeof(int32_t), cmp_i32);
    return m;
}

int ora_ilut(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, double tau, int lfil,
             ora_mat *out)
{
    if (n < 0 || lfil < 0 || !(tau >= 0.0)) return ORA_INVALID;
    ora_mat LU = {0};
    double *w = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *inw = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *list = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *cand = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *kept = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t *udiag = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int st = ORA_OK;
    if (!w || !inw || !list || !cand || !kept || !udiag || mat_init(&LU, n, rp[n] * 2 + 16)) { st = ORA_OOM; goto done; }
    for (int64_t i = 0; i < n; i++) inw[i] = 0;
    for (int64_t i = 0; i < n; i++) {
        int nw = 0;
        double ss = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            if (ci[e] < 0 || ci[e] >= n || (e > rp[i] && ci[e] <= ci[e - 1])) { st = ORA_INVALID; goto done; }
            ss += va[e] * va[e];
            w[ci[e]] = va[e];
            inw[ci[e]] = 1;
            list[nw++] = ci[e];
        }
        if (!inw[i]) { inw[i] = 1; w[i] = 0.0; list[nw++] = (int32_t)i; }
        const double tau_i = tau * sqrt(ss);
        int64_t k = -1;
        for (;;) {
            int64_t next = n;
            for (int t = 0; t < nw; t++)
                if (list[t] > k && list[t] < i && list[t] < next) next = list[t];
            if (next == n) break;
            k = next;
            if (w[k] == 0.0) continue;
            w[k] = w[k] / LU.va[udiag[k]];
            if (fabs(w[k]) < tau_i) { w[k] = 0.0; continue; }
            for (int64_t f = udiag[k] + 1; f < LU.rp[k + 1]; f++) {
                int32_t j = LU.ci[f];
                if (!inw[j]) { inw[j] = 1; w[j] = 0.0; list[nw++] = j; }
                w[j] = fma(-w[k], LU.va[f], w[j]);
            }
        }
        const double piv = w[i];
        if (piv == 0.0 || !isfinite(piv)) { st = ORA_ZERO_PIVOT; goto done; }
        /* L part */
        int nc = 0;
        for (int t = 0; t < nw; t++)
            if (list[t] < i && w[list[t]] != 0.0 && fabs(w[list[t]]) >= tau_i) cand[nc++] = list[t];
        int nk = keep_largest(cand, w, nc, lfil, kept);
        for (int t = 0; t < nk; t++)
            if (mat_push(&LU, kept[t], w[kept[t]])) { st = ORA_OOM; goto done; }
        udiag[i] = LU.nnz;
        if (mat_push(&LU, (int32_t)i, piv)) { st = ORA_OOM; goto done; }
        /* U part */
        nc = 0;
        for (int t = 0; t < nw; t++)
            if (list[t] > i && w[list[t]] != 0.0 && fabs(w[list[t]]) >= tau_i) cand[nc++] = list[t];
        nk = keep_largest(cand, w, nc, lfil, kept);
        for (int t = 0; t < nk; t++)
            if (mat_push(&LU, kept[t], w[kept[t]])) { st = ORA_OOM; goto done; }
        LU.rp[i + 1] = (int32_t)LU.nnz;
        for (int t = 0; t < nw; t++) { inw[list[t]] = 0; w[list[t]] = 0.0; }
    }
    *out = LU;
    LU.rp = NULL; LU.ci = NULL; LU.va = NULL;
done:
    ora_free(&LU);
    free(w); free(inw); free(list); free(cand); free(kept); free(udiag);
    return st;
}

/* ------------------------------------------------------------------------ */
/* ILU(p), level-of-fill incomplete LU (Saad, Iterative Methods for Sparse    */
/* Linear Systems, 2nd ed., Section 10.3.3, Algorithm 10.5).  The paper      */
/* feeds level-0 and level-1 ILU factors to SAIT (Section 4, Tables          */
/* runtime_SAIT and runtime_Jacobi).                                         */
/* Every structural entry of A has level 0.  Row i:                          */
/*   w := a_i*, lev_ij := 0 on A's pattern (infinite elsewhere)              */
/*   for k < i in increasing order with lev_ik <= p (fill included):         */
/*       w_k := w_k / u_kk                                                   */
/*       w_j := fma(-w_k, u_kj, w_j)  for u_kj stored, j > k                 */
/*       lev_ij := min(lev_ij, lev_ik + lev_kj + 1)                          */
/*   keep the entries with lev_ij <= p (the diagonal included).              */
/* A level only decreases while the row is processed, and every update of   */
/* lev_ik comes from a column before k, so lev_ik is final when k is         */
/* reached.  Output as ora_ilut: strict lower part of L (unit diagonal       */
/* implied) and U with its diagonal, columns ascending, plus the level of    */
/* every stored entry in lev_out (may be NULL).  The diagonal must be in     */
/* A's pattern; a zero or non-finite pivot returns ORA_ZERO_PIVOT.  p = 0 is  */
/* ILU(0) (same fma chains), and p >= n is the complete LU without pivoting. */
/* ------------------------------------------------------------------------ */
int ora_iluk(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, int p, ora_mat *out,
             int32_t **lev_out)
{
    if (n < 0 || p < 0) return ORA_INVALID;
    const int32_t INF = 0x7fffffff;
    ora_mat LU = {0};
    int64_t lcap = rp[n] * 2 + 16, lnnz = 0;
    int32_t *levs = (int32_t *)malloc((size_t)lcap * sizeof(int32_t));   /* level of each stored entry */
    double *w = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *lev = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t *list = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t *udiag = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int st = ORA_OK;
    if (!levs || !w || !lev || !list || !udiag || mat_init(&LU, n, lcap)) { st = ORA_OOM; goto done; }
    for (int64_t i = 0; i < n; i++) lev[i] = INF;
    for (int64_t i = 0; i < n; i++) {
        int nw = 0, have_d = 0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            if (ci[e] < 0 || ci[e] >= n || (e > rp[i] && ci[e] <= ci[e - 1])) { st = ORA_INVALID; goto done; }
            w[ci[e]] = va[e];
            lev[ci[e]] = 0;
            list[nw++] = ci[e];
            if (ci[e] == i) have_d = 1;
        }
        if (!have_d) { st = ORA_ZERO_PIVOT; goto done; }
        int64_t k = -1;
        for (;;) {
            int64_t next = n;   /* the smallest column above k and below i in the row */
            for (int t = 0; t < nw; t++)
                if (list[t] > k && list[t] < i && list[t] < next) next = list[t];
            if (next == n) break;
            k = next;
            if (lev[k] > p) continue;
            w[k] = w[k] / LU.va[udiag[k]];
            for (int64_t f = udiag[k] + 1; f < LU.rp[k + 1]; f++) {
                int32_t j = LU.ci[f];
                if (lev[j] == INF) { w[j] = 0.0; list[nw++] = j; }
                w[j] = fma(-w[k], LU.va[f], w[j]);
                int32_t lj = lev[k] + levs[f] + 1;
                if (lj < lev[j]) lev[j] = lj;
            }
        }
        if (w[i] == 0.0 || !isfinite(w[i])) { st = ORA_ZERO_PIVOT; goto done; }
        qsort(list, (size_t)nw, sizeof(int32_t), cmp_i32);
        for (int t = 0; t < nw; t++) {
            int32_t j = list[t];
            if (lev[j] > p) continue;
            if (j == i) udiag[i] = LU.nnz;
            if (mat_push(&LU, j, w[j])) { st = ORA_OOM; goto done; }
            if (lnnz == lcap) {
                int32_t *nl = (int32_t *)realloc(levs, (size_t)(lcap * 2) * sizeof(int32_t));
                if (!nl) { st = ORA_OOM; goto done; }
                levs = nl;
                lcap *= 2;
            }
            levs[lnnz++] = lev[j];
        }
        LU.rp[i + 1] = (int32_t)LU.nnz;
        for (int t = 0; t < nw; t++) { lev[list[t]] = INF; w[list[t]] = 0.0; }
    }
    *out = LU;
    LU.rp = NULL; LU.ci = NULL; LU.va = NULL;
    if (lev_out) { *lev_out = levs; levs = NULL; }
done:
    ora_free(&LU);
    free(levs); free(w); free(lev); free(list); free(udiag);
    return st;
}

void ora_free_i32(int32_t *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* SAIT (Algorithms 1-3).                                                   */
/*                                                                          */
/* With D = diag(T) and T~ = I - D^-1 T (strictly triangular, Section 2),    */
/* the Horner / Qin Jiushao recursion (equation Recursive) is               */
/*     M_0 D = I,   M_k D = T~ (M_{k-1} D) + I,                              */
/* and after the loop M = (M D) D^-1.  m_terms is the number of series      */
/* terms of M = sum_{i < m_terms} T~^i D^-1 (equation M_poly), i.e. the loop */
/* runs m_terms - 1 times; the paper's SAIT_Thr(tau, m) is m_terms = m + 1 */
/* and SAIT_Pat(p, m) is m_terms = p + m + 1.                               */
/*                                                                          */
/* Each product row is formed in a dense accumulator: for k over row i of   */
/* T~ in ascending column order, for j over row k of the iterate,           */
/*     acc_j = fma(T~_ik, (MD)_kj, acc_j),                                   */
/* then the diagonal entry 1 is added, then the drop rule is applied to the */
/* whole row (the thresholds act on the unit-diagonal iterate MD, as in     */
/* step 3 of Algorithms 1-2, before the final scaling by D^-1).             */
/* ------------------------------------------------------------------------ */
int ora_sait(int64_t n, const int32_t *rp, const int32_t *ci, const double *va,
             int m_terms, int drop_kind, double tau, int p, ora_mat *out)
{
    memset(out, 0, sizeof(*out));
    if (n < 0 || m_terms < 1 || drop_kind < 0 || drop_kind > 4 || p < 0 ||
        ((drop_kind == 1 || drop_kind == 2 || drop_kind == 4) && !(tau >= 0.0)))
        return ORA_INVALID;
    int st = ORA_OK;
    int side = 0;   /* -1 lower, +1 upper, 0 diagonal only so far */
    double *dinv = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *acc = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int64_t *stamp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *sstamp = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int32_t *list = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    ora_mat tt = {0}, M = {0}, S = {0};
    if (!dinv || !acc || !stamp || !sstamp || !list) { st = ORA_OOM; goto done; }

    /* Step 1: D^-1 and T~ = I - D^-1 T, whose off-diagonal entries are
     * -(d_i^-1 T_ij) and whose diagonal is exactly zero. */
    if ((st = mat_init(&tt, n, rp[n] > 0 ? rp[n] : 1)) != ORA_OK) goto done;
    for (int64_t i = 0; i < n; i++) {
        int have_d = 0;
        double d = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++) {
            if (e > rp[i] && ci[e] <= ci[e - 1]) { st = ORA_INVALID; goto done; }
            if (ci[e] == i) { have_d = 1; d = va[e]; continue; }
            int s = ci[e] < i ? -1 : 1;
            if (side == 0) side = s;
            else if (side != s) { st = ORA_NOT_TRIANGULAR; goto done; }
        }
        if (!have_d || d == 0.0 || !isfinite(d)) { st = ORA_ZERO_PIVOT; goto done; }
        dinv[i] = 1.0 / d;
    }
    for (int64_t i = 0; i < n; i++) {
        for (int32_t e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] != i && (st = mat_push(&tt, ci[e], -(dinv[i] * va[e]))) != ORA_OK) goto done;
        tt.rp[i + 1] = (int32_t)tt.nnz;
    }

    /* M D = I. */
    if ((st = mat_init(&M, n, n)) != ORA_OK) goto done;
    for (int64_t i = 0; i < n; i++) {
        if ((st = mat_push(&M, (int32_t)i, 1.0)) != ORA_OK) goto done;
        M.rp[i + 1] = (int32_t)(i + 1);
    }
    if (drop_kind == 3 && p == 0) {          /* S = pattern of M_1 = pattern(T^0) */
        if ((st = mat_init(&S, n, n)) != ORA_OK) goto done;
        for (int64_t i = 0; i < n; i++) { mat_push(&S, (int32_t)i, 1.0); S.rp[i + 1] = (int32_t)(i + 1); }
    }

    for (int64_t i = 0; i < n; i++) { stamp[i] = -1; sstamp[i] = -1; }
    int64_t epoch = 0;
    for (int it = 1; it < m_terms; it++) {
        ora_mat Mn = {0};
        if ((st = mat_init(&Mn, n, M.nnz + n)) != ORA_OK) goto done;
        for (int64_t i = 0; i < n; i++) {
            epoch++;
            int64_t cnt = 0;
            /* T~ (M D), row i, ascending k */
            for (int32_t e = tt.rp[i]; e < tt.rp[i + 1]; e++) {
                int64_t k = tt.ci[e];
                double t = tt.va[e];
                for (int32_t f = M.rp[k]; f < M.rp[k + 1]; f++) {
                    int32_t j = M.ci[f];
                    if (stamp[j] != epoch) { stamp[j] = epoch; acc[j] = 0.0; list[cnt++] = j; }
                    acc[j] = fma(t, M.va[f], acc[j]);
                }
            }
            /* + I */
            if (stamp[i] != epoch) { stamp[i] = epoch; acc[i] = 0.0; list[cnt++] = (int32_t)i; }
            acc[i] = acc[i] + 1.0;
            qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);

            /* dropping rule on the whole new row */
            int kind = drop_kind;
            if (kind == 3 && it <= p) kind = 0;          /* pattern-building iterations */
            if (kind == 4) kind = it <= p ? 0 : 1;       /* hybrid: undropped, then threshold */
            double thr = tau;
            if (kind == 2) {
                double mx = 0.0;
                for (int64_t q = 0; q < cnt; q++) { double a = fabs(acc[list[q]]); if (a > mx) mx = a; }
                thr = tau * mx;
            }
            if (kind == 3)
                for (int32_t f = S.rp[i]; f < S.rp[i + 1]; f++) sstamp[S.ci[f]] = epoch;
            for (int64_t q = 0; q < cnt; q++) {
                int32_t j = list[q];
                double v = acc[j];
                int keep = 1;
                if (j != i) {
                    if (kind == 1 || kind == 2) keep = !(fabs(v) < thr);
                    else if (kind == 3) keep = (sstamp[j] == epoch);
                }
                if (keep && (st = mat_push(&Mn, j, v)) != ORA_OK) { ora_free(&Mn); goto done; }
            }
            Mn.rp[i + 1] = (int32_t)Mn.nnz;
        }
        ora_free(&M);
        M = Mn;
        if (drop_kind == 3 && it == p) {       /* keep the sparsity pattern S of M */
            if ((st = mat_init(&S, n, M.nnz)) != ORA_OK) goto done;
            for (int64_t i = 0; i < n; i++) {
                for (int32_t f = M.rp[i]; f < M.rp[i + 1]; f++) mat_push(&S, M.ci[f], 1.0);
                S.rp[i + 1] = (int32_t)S.nnz;
            }
        }
    }

    /* M = (M D) D^-1: column j scaled by d_j^-1 */
    for (int64_t e = 0; e < M.nnz; e++) M.va[e] = M.va[e] * dinv[M.ci[e]];
    *out = M;
    M.rp = NULL; M.ci = NULL; M.va = NULL;
done:
    ora_free(&M);
    ora_free(&tt);
    ora_free(&S);
    free(dinv); free(acc); free(stamp); free(sstamp); free(list);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Preconditioners for the Krylov solvers.                                   */
/*   kind 0: none (z = r)                                                    */
/*   kind 1: SAIT pair, z = M_U (M_L r)        (Section 3.1)                 */
/*   kind 2: exact ILU, z = U^-1 (L^-1 r)      (substitution; Section 3.1)   */
/*   kind 3: Jacobi sweeps, `sweeps` iterations of equation Jacobi_iter on   */
/*           L y = r and then on U z = y, each from a zero start             */
/*           (Section 4, comparison with Jacobi iteration)                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind;
    int64_t n;
    const int32_t *l_rp, *l_ci;
    const double *l_va;
    const int32_t *u_rp, *u_ci;
    const double *u_va;
    int sweeps;
} ora_prec;

/* k sweeps of x^j = T~ x^{j-1} + D^-1 b from x^0 = 0 (Section 2, equation
 * Jacobi_iter), T~ = I - D^-1 T, so (T~ x)_i = -sum_{j != i} (t_ij / t_ii) x_j.
 * Works for any square T with a nonzero diagonal. */
int ora_jacobi(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, int sweeps,
               const double *b, double *x)
{
    if (n < 0 || sweeps < 0) return ORA_INVALID;
    double *d = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *xo = (double *)malloc((size_t)n * sizeof(double) + 8);
    if (!d || !xo) { free(d); free(xo); return ORA_OOM; }
    int st = ORA_OK;
    for (int64_t i = 0; i < n; i++) {
        d[i] = 0.0;
        for (int32_t e = rp[i]; e < rp[i + 1]; e++)
            if (ci[e] == i) d[i] = va[e];
        if (d[i] == 0.0 || !isfinite(d[i])) st = ORA_ZERO_PIVOT;
        x[i] = 0.0;
    }
    for (int k = 0; k < sweeps && st == ORA_OK; k++) {
        memcpy(xo, x, (size_t)n * sizeof(double));
        for (int64_t i = 0; i < n; i++) {
            double s = 0.0;
            for (int32_t e = rp[i]; e < rp[i + 1]; e++)
                if (ci[e] != i) s += (-va[e] / d[i]) * xo[ci[e]];
            x[i] = s + b[i] / d[i];
        }
    }
    free(d); free(xo);
    return st;
}

static int prec_apply(const ora_prec *P, const double *r, double *z, double *tmp)
{
    int64_t n = P->n;
    if (P->kind == 0) { memcpy(z, r, (size_t)n * sizeof(double)); return ORA_OK; }
    if (P->kind == 1) {
        ora_spmv(n, P->l_rp, P->l_ci, P->l_va, r, tmp);
        ora_spmv(n, P->u_rp, P->u_ci, P->u_va, tmp, z);
        return ORA_OK;
    }
    if (P->kind == 2) {
        int st = ora_trisolve(n, P->l_rp, P->l_ci, P->l_va, 1, r, tmp);
        if (st) return st;
        return ora_trisolve(n, P->u_rp, P->u_ci, P->u_va, 0, tmp, z);
    }
    if (P->kind == 3) {
        int st = ora_jacobi(n, P->l_rp, P->l_ci, P->l_va, P->sweeps, r, tmp);
        if (st) return st;
        return ora_jacobi(n, P->u_rp, P->u_ci, P->u_va, P->sweeps, tmp, z);
    }
    return ORA_INVALID;
}

static double dot(int64_t n, const double *x, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += x[i] * y[i];
    return s;
}

static double nrm2(int64_t n, const double *x) { return sqrt(dot(n, x, x)); }

/* true residual r = b - A x, returns ||r|| */
static double residual(int64_t n, const int32_t *rp, const int32_t *ci, const double *va,
                       const double *b, const double *x, double *r)
{
    ora_spmv(n, rp, ci, va, x, r);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - r[i];
    return nrm2(n, r);
}

/* ------------------------------------------------------------------------ */
/* Restarted GMRES(m) with right preconditioning: Arnoldi by modified        */
/* Gram-Schmidt, Givens rotations for the least-squares problem, x updated   */
/* as x + P (V y) at the end of each cycle (Saad, Algorithms 6.9 and 9.5).   */
/* Stops when ||b - A x|| / ||b|| <= tol (true residual, checked at the end  */
/* of each cycle; the Givens estimate decides when a cycle ends).  *iters    */
/* counts Arnoldi steps (matrix-vector products with A).                     */
/* ------------------------------------------------------------------------ */
int ora_gmres(int64_t n, const int32_t *rp, const int32_t *ci, const double *va,
              const ora_prec *P, const double *b, double *x, int restart, double tol,
              int maxit, int *iters, double *relres)
{
    if (restart < 1 || maxit < 0 || n < 0) return ORA_INVALID;
    int m = restart;
    double *V = (double *)malloc((size_t)(m + 1) * (size_t)n * sizeof(double) + 8);
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc((size_t)m * sizeof(double));
    double *sn = (double *)malloc((size_t)m * sizeof(double));
    double *g = (double *)malloc((size_t)(m + 1) * sizeof(double));
    double *y = (double *)malloc((size_t)m * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *z = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *tmp = (double *)malloc((size_t)n * sizeof(double) + 8);
    int st = ORA_NOT_CONVERGED;
    *iters = 0;
    *relres = 0.0;
    if (!V || !H || !cs || !sn || !g || !y || !w || !z || !tmp) { st = ORA_OOM; goto done; }
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) { for (int64_t i = 0; i < n; i++) x[i] = 0.0; st = ORA_OK; goto done; }
#define Hij(i, j) H[(size_t)(j) * (size_t)(m + 1) + (size_t)(i)]
    for (;;) {
        double beta = residual(n, rp, ci, va, b, x, w);
        *relres = beta / bnorm;
        if (*relres <= tol) { st = ORA_OK; break; }
        if (*iters >= maxit) break;
        for (int64_t i = 0; i < n; i++) V[i] = w[i] / beta;
        g[0] = beta;
        int jj = 0;
        for (int j = 0; j < m; j++) {
            double *vj = V + (size_t)j * n, *vn = V + (size_t)(j + 1) * n;
            int ps = prec_apply(P, vj, z, tmp);
            if (ps) { st = ps; goto done; }
            ora_spmv(n, rp, ci, va, z, w);
            (*iters)++;
            for (int i = 0; i <= j; i++) {                       /* MGS */
                double *vi = V + (size_t)i * n;
                double h = dot(n, w, vi);
                Hij(i, j) = h;
                for (int64_t q = 0; q < n; q++) w[q] -= h * vi[q];
            }
            double hn = nrm2(n, w);
            Hij(j + 1, j) = hn;
            for (int i = 0; i < j; i++) {                        /* old rotations */
                double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
                Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
                Hij(i, j) = t;
            }
            double a = Hij(j, j), bb = Hij(j + 1, j);             /* new rotation */
            if (bb == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { double t = hypot(a, bb); cs[j] = a / t; sn[j] = bb / t; }
            Hij(j, j) = cs[j] * a + sn[j] * bb;
            Hij(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            jj = j + 1;
            if (hn != 0.0)
                for (int64_t q = 0; q < n; q++) vn[q] = w[q] / hn;
            if (fabs(g[j + 1]) <= tol * bnorm || hn == 0.0 || *iters >= maxit) break;
        }
        for (int i = jj - 1; i >= 0; i--) {                      /* H y = g */
            double s = g[i];
            for (int k = i + 1; k < jj; k++) s -= Hij(i, k) * y[k];
            if (Hij(i, i) == 0.0) { st = ORA_BREAKDOWN; goto done; }
            y[i] = s / Hij(i, i);
        }
        for (int64_t q = 0; q < n; q++) {
            double s = 0.0;
            for (int i = 0; i < jj; i++) s += y[i] * V[(size_t)i * n + q];
            w[q] = s;
        }
        int ps = prec_apply(P, w, z, tmp);
        if (ps) { st = ps; goto done; }
        for (int64_t q = 0; q < n; q++) x[q] += z[q];
    }
#undef Hij
done:
    free(V); free(H); free(cs); free(sn); free(g); free(y); free(w); free(z); free(tmp);
    return st;
}

/* ------------------------------------------------------------------------ */
/* BiCGSTAB with right preconditioning (van der Vorst 1992; Saad,           */
/* Algorithm 7.7 applied to A P u = b, x = P u).  *iters counts full        */
/* iterations (two products with A each).  Convergence is tested on the     */
/* recursive residuals s and r and confirmed on the true residual.          */
/* ------------------------------------------------------------------------ */
int ora_bicgstab(int64_t n, const int32_t *rp, const int32_t *ci, const double *va,
                 const ora_prec *P, const double *b, double *x, double tol, int maxit,
                 int *iters, double *relres)
{
    double *r = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *rh = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *p = (double *)calloc((size_t)n + 1, sizeof(double));
    double *v = (double *)calloc((size_t)n + 1, sizeof(double));
    double *ph = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *s = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *sh = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *t = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *tmp = (double *)malloc((size_t)n * sizeof(double) + 8);
    int st = ORA_NOT_CONVERGED;
    *iters = 0;
    *relres = 0.0;
    if (!r || !rh || !p || !v || !ph || !s || !sh || !t || !tmp) { st = ORA_OOM; goto done; }
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) { for (int64_t i = 0; i < n; i++) x[i] = 0.0; st = ORA_OK; goto done; }
    double rn = residual(n, rp, ci, va, b, x, r);
    *relres = rn / bnorm;
    if (*relres <= tol) { st = ORA_OK; goto done; }
    memcpy(rh, r, (size_t)n * sizeof(double));
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    while (*iters < maxit) {
        double rho = dot(n, rh, r);
        if (rho == 0.0 || omega == 0.0) { st = ORA_BREAKDOWN; break; }
        double beta = (rho / rho_old) * (alpha / omega);
        for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        int ps = prec_apply(P, p, ph, tmp);
        if (ps) { st = ps; break; }
        ora_spmv(n, rp, ci, va, ph, v);
        double rv = dot(n, rh, v);
        if (rv == 0.0) { st = ORA_BREAKDOWN; break; }
        alpha = rho / rv;
        for (int64_t i = 0; i < n; i++) s[i] = r[i] - alpha * v[i];
        (*iters)++;
        if (nrm2(n, s) / bnorm <= tol) {
            for (int64_t i = 0; i < n; i++) x[i] += alpha * ph[i];
            rn = residual(n, rp, ci, va, b, x, r);
            *relres = rn / bnorm;
            if (*relres <= tol) { st = ORA_OK; break; }
            memcpy(rh, r, (size_t)n * sizeof(double));     /* restart the recurrence */
            rho_old = alpha = omega = 1.0;
            memset(p, 0, (size_t)n * sizeof(double));
            memset(v, 0, (size_t)n * sizeof(double));
            continue;
        }
        ps = prec_apply(P, s, sh, tmp);
        if (ps) { st = ps; break; }
        ora_spmv(n, rp, ci, va, sh, t);
        double tt = dot(n, t, t);
        omega = tt == 0.0 ? 0.0 : dot(n, t, s) / tt;
        for (int64_t i = 0; i < n; i++) {
            x[i] += alpha * ph[i] + omega * sh[i];
            r[i] = s[i] - omega * t[i];
        }
        rho_old = rho;
        if (nrm2(n, r) / bnorm <= tol) {
            rn = residual(n, rp, ci, va, b, x, r);
            *relres = rn / bnorm;
            if (*relres <= tol) { st = ORA_OK; break; }
            memcpy(rh, r, (size_t)n * sizeof(double));
            rho_old = alpha = omega = 1.0;
            memset(p, 0, (size_t)n * sizeof(double));
            memset(v, 0, (size_t)n * sizeof(double));
        }
    }
    if (st == ORA_NOT_CONVERGED) *relres = residual(n, rp, ci, va, b, x, r) / bnorm;
done:
    free(r); free(rh); free(p); free(v); free(ph); free(s); free(sh); free(t); free(tmp);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Preconditioned conjugate gradients (Saad, Algorithm 9.1), the paper's    */
/* linear solver (Section 4).  The preconditioner is applied as given, even */
/* when it is not symmetric (the SAIT pair M_U M_L is not).  Convergence is  */
/* tested on the recursive residual ||r|| / ||b|| and the returned relres is */
/* the true residual.                                                       */
/* ------------------------------------------------------------------------ */
int ora_pcg(int64_t n, const int32_t *rp, const int32_t *ci, const double *va,
            const ora_prec *P, const double *b, double *x, double tol, int maxit,
            int *iters, double *relres)
{
    double *r = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *z = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *p = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *q = (double *)malloc((size_t)n * sizeof(double) + 8);
    double *tmp = (double *)malloc((size_t)n * sizeof(double) + 8);
    int st = ORA_NOT_CONVERGED;
    *iters = 0;
    *relres = 0.0;
    if (!r || !z || !p || !q || !tmp) { st = ORA_OOM; goto done; }
    double bnorm = nrm2(n, b);
    if (bnorm == 0.0) { for (int64_t i = 0; i < n; i++) x[i] = 0.0; st = ORA_OK; goto done; }
    double rn = residual(n, rp, ci, va, b, x, r);
    if (rn / bnorm <= tol) { *relres = rn / bnorm; st = ORA_OK; goto done; }
    int ps = prec_apply(P, r, z, tmp);
    if (ps) { st = ps; goto done; }
    memcpy(p, z, (size_t)n * sizeof(double));
    double rho = dot(n, r, z);
    while (*iters < maxit) {
        ora_spmv(n, rp, ci, va, p, q);
        double pq = dot(n, p, q);
        if (pq == 0.0) { st = ORA_BREAKDOWN; break; }
        double alpha = rho / pq;
        for (int64_t i = 0; i < n; i++) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        (*iters)++;
        if (nrm2(n, r) / bnorm <= tol) { st = ORA_OK; break; }
        ps = prec_apply(P, r, z, tmp);
        if (ps) { st = ps; break; }
        double rho_new = dot(n, r, z);
        if (rho == 0.0) { st = ORA_BREAKDOWN; break; }
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        rho = rho_new;
    }
    *relres = residual(n, rp, ci, va, b, x, r) / bnorm;
done:
    free(r); free(z); free(p); free(q); free(tmp);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Dense helpers for LOBPCG (row-major blocks, column-major small matrices    */
/* are avoided: every small matrix here is row-major m x m).                 */
/* ------------------------------------------------------------------------ */

/* G (p x q) = Y^T Z, Y n x p, Z n x q, row-major blocks */
static void gram(int64_t n, const double *Y, int p, const double *Z, int q, double *G)
{
    for (int a = 0; a < p; a++)
        for (int b = 0; b < q; b++) {
            double s = 0.0;
            for (int64_t i = 0; i < n; i++) s += Y[i * p + a] * Z[i * q + b];
            G[a * q + b] = s;
        }
}

/* Y (n x p) = Z (n x q) C (q x p) */
static void block_mul(int64_t n, const double *Z, int q, const double *C, int p, double *Y)
{
    for (int64_t i = 0; i < n; i++)
        for (int b = 0; b < p; b++) {
            double s = 0.0;
            for (int a = 0; a < q; a++) s += Z[i * q + a] * C[a * p + b];
            Y[i * p + b] = s;
        }
}

/* lower Cholesky factor of SPD G (m x m) in place; 1 if not positive definite */
static int chol(int m, double *G)
{
    double mx = 0.0;
    for (int i = 0; i < m; i++) if (G[i * m + i] > mx) mx = G[i * m + i];
    for (int j = 0; j < m; j++) {
        double d = G[j * m + j];
        for (int k = 0; k < j; k++) d -= G[j * m + k] * G[j * m + k];
        if (!(d > 1e-14 * mx)) return 1;
        d = sqrt(d);
        G[j * m + j] = d;
        for (int i = j + 1; i < m; i++) {
            double s = G[i * m + j];
            for (int k = 0; k < j; k++) s -= G[i * m + k] * G[j * m + k];
            G[i * m + j] = s / d;
        }
        for (int i = 0; i < j; i++) G[i * m + j] = 0.0;
    }
    return 0;
}

/* R (m x m) = L^{-1}, L lower triangular */
static void tri_inv_lower(int m, const double *L, double *R)
{
    for (int j = 0; j < m; j++)
        for (int i = 0; i < m; i++) {
            if (i < j) { R[i * m + j] = 0.0; continue; }
            double s = (i == j) ? 1.0 : 0.0;
            for (int k = j; k < i; k++) s -= L[i * m + k] * R[k * m + j];
            R[i * m + j] = s / L[i * m + i];
        }
}

/* Cyclic Jacobi eigenvalue algorithm for symmetric C (Golub and Van Loan,
 * Algorithm 8.5.3): C is overwritten; eigenvalues ascending in w, the
 * corresponding eigenvectors are the columns of V (row-major m x m). */
static void jacobi_eig(int m, double *C, double *w, double *V)
{
    for (int i = 0; i < m; i++)
        for (int j = 0; j < m; j++) V[i * m + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int i = 0; i < m * m; i++) fro += C[i] * C[i];
    fro = sqrt(fro);
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0;
        for (int i = 0; i < m; i++)
            for (int j = 0; j < m; j++) if (i != j) off += C[i * m + j] * C[i * m + j];
        if (sqrt(off) <= 1e-15 * fro || fro == 0.0) break;
        for (int p = 0; p < m - 1; p++)
            for (int q = p + 1; q < m; q++) {
                double apq = C[p * m + q];
                if (apq == 0.0) continue;
                /* symmetric 2x2 Schur decomposition (Golub and Van Loan, Algorithm 8.5.2) */
                double tau = (C[q * m + q] - C[p * m + p]) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < m; k++) {       /* C <- C J */
                    double a = C[k * m + p], b = C[k * m + q];
                    C[k * m + p] = c * a - s * b;
                    C[k * m + q] = s * a + c * b;
                }
                for (int k = 0; k < m; k++) {       /* C <- J^T C */
                    double a = C[p * m + k], b = C[q * m + k];
                    C[p * m + k] = c * a - s * b;
                    C[q * m + k] = s * a + c * b;
                }
                for (int k = 0; k < m; k++) {       /* V <- V J */
                    double a = V[k * m + p], b = V[k * m + q];
                    V[k * m + p] = c * a - s * b;
                    V[k * m + q] = s * a + c * b;
                }
            }
    }
    for (int i = 0; i < m; i++) w[i] = C[i * m + i];
    for (int i = 0; i < m; i++) {                   /* selection sort, ascending */
        int best = i;
        for (int j = i + 1; j < m; j++) if (w[j] < w[best]) best = j;
        if (best != i) {
            double t = w[i]; w[i] = w[best]; w[best] = t;
            for (int k = 0; k < m; k++) { t = V[k * m + i]; V[k * m + i] = V[k * m + best]; V[k * m + best] = t; }
        }
    }
}

/* Y (n x p) <- Y D L^{-T} where D = diag(Y^T Y)^{-1/2} and D Y^T Y D = L L^T
 * (Cholesky QR of the column-equilibrated block); AY likewise when given.
 * Returns 1 when the Gram matrix is not numerically positive definite. */
static int cholqr(int64_t n, double *Y, double *AY, int p, double *work)
{
    double *G = work, *R = work + p * p, *RT = work + 2 * p * p;
    double dsc[64];
    gram(n, Y, p, Y, p, G);
    for (int a = 0; a < p; a++) {
        if (!(G[a * p + a] > 0.0)) return 1;
        dsc[a] = 1.0 / sqrt(G[a * p + a]);
    }
    for (int a = 0; a < p; a++) for (int b = 0; b < p; b++) G[a * p + b] *= dsc[a] * dsc[b];
    if (chol(p, G)) return 1;
    tri_inv_lower(p, G, R);
    for (int a = 0; a < p; a++) for (int b = 0; b < p; b++) RT[a * p + b] = dsc[a] * R[b * p + a];
    double *tmp = (double *)malloc((size_t)n * p * sizeof(double) + 8);
    if (!tmp) return 1;
    block_mul(n, Y, p, RT, p, tmp);
    memcpy(Y, tmp, (size_t)n * p * sizeof(double));
    if (AY) { block_mul(n, AY, p, RT, p, tmp); memcpy(AY, tmp, (size_t)n * p * sizeof(double)); }
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* LOBPCG for the k smallest eigenpairs of SPD A (Knyazev 2001, the method   */
/* the paper's eigenvalue experiments use, Section 4.4) with a              */
/* preconditioner T applied to the residual block, soft locking of          */
/* converged columns, Cholesky-QR orthonormalisation of the W and P blocks, */
/* and the Rayleigh-Ritz step on S = [X, W, P] in FP64.  Convergence of     */
/* column j: ||A x_j - lambda_j x_j|| <= tol * lambda_j ||x_j||.            */
/* X: n x k row-major, initial guess in, eigenvectors out.                   */
/* ------------------------------------------------------------------------ */
int ora_lobpcg(int64_t n, const int32_t *rp, const int32_t *ci, const double *va, const ora_prec *P,
               int k, double *X, double *lambda, double tol, int maxit, int *iters, double *resmax)
{
    if (k < 1 || 3 * k > n || maxit < 0) return ORA_INVALID;
    const int m3 = 3 * k;
    size_t nk = (size_t)n * k;
    double *AX = malloc(nk * 8 + 8), *R = malloc(nk * 8 + 8), *W = malloc(nk * 8 + 8), *AW = malloc(nk * 8 + 8);
    double *Pb = malloc(nk * 8 + 8), *AP = malloc(nk * 8 + 8), *S = malloc(nk * 3 * 8 + 8), *AS = malloc(nk * 3 * 8 + 8);
    double *v = malloc((size_t)n * 8 + 8), *z = malloc((size_t)n * 8 + 8), *tmp = malloc((size_t)n * 8 + 8);
    double *GA = malloc(m3 * m3 * 8), *GB = malloc(m3 * m3 * 8), *LI = malloc(m3 * m3 * 8), *C = malloc(m3 * m3 * 8);
    double *Y = malloc(m3 * m3 * 8), *Cf = malloc(m3 * m3 * 8), *th = malloc(m3 * 8), *work = malloc(3 * m3 * m3 * 8);
    double *res = malloc(k * 8);
    int *act = malloc(k * sizeof(int));
    int st = ORA_NOT_CONVERGED, havep = 0;
    *iters = 0;
    *resmax = 0.0;
    if (!AX || !R || !W || !AW || !Pb || !AP || !S || !AS || !v || !z || !tmp || !GA || !GB || !LI || !C ||
        !Y || !Cf || !th || !work || !res || !act) { st = ORA_OOM; goto done; }
    /* initial Rayleigh-Ritz on span(X) */
    if (cholqr(n, X, NULL, k, work)) { st = ORA_BREAKDOWN; goto done; }
    for (int j = 0; j < k; j++) {
        for (int64_t i = 0; i < n; i++) v[i] = X[i * k + j];
        ora_spmv(n, rp, ci, va, v, z);
        for (int64_t i = 0; i < n; i++) AX[i * k + j] = z[i];
    }
    gram(n, X, k, AX, k, GA);
    for (int a = 0; a < k; a++) for (int b = 0; b < a; b++) {
        double s = 0.5 * (GA[a * k + b] + GA[b * k + a]); GA[a * k + b] = GA[b * k + a] = s;
    }
    jacobi_eig(k, GA, th, Y);
    block_mul(n, X, k, Y, k, S); memcpy(X, S, nk * 8);
    block_mul(n, AX, k, Y, k, S); memcpy(AX, S, nk * 8);
    for (int j = 0; j < k; j++) lambda[j] = th[j];

    for (int it = 0; it <= maxit; it++) {
        /* residuals and soft locking */
        int na = 0;
        *resmax = 0.0;
        for (int j = 0; j < k; j++) {
            double rn = 0.0, xn = 0.0;
            for (int64_t i = 0; i < n; i++) {
                double r = AX[i * k + j] - lambda[j] * X[i * k + j];
                R[i * k + j] = r;
                rn += r * r;
                xn += X[i * k + j] * X[i * k + j];
            }
            res[j] = sqrt(rn) / (fabs(lambda[j]) * sqrt(xn));
            if (res[j] > *resmax) *resmax = res[j];
            if (res[j] > tol) act[na++] = j;
        }
        if (na == 0) { st = ORA_OK; break; }
        if (it == maxit) break;
        *iters = it + 1;
        /* W = T R(:, active), orthogonal to X, orthonormal */
        for (int a = 0; a < na; a++) {
            for (int64_t i = 0; i < n; i++) v[i] = R[i * k + act[a]];
            int ps = prec_apply(P, v, z, tmp);
            if (ps) { st = ps; goto done; }
            for (int64_t i = 0; i < n; i++) W[i * na + a] = z[i];
        }
        gram(n, X, k, W, na, C);                              /* C = X^T W (k x na) */
        block_mul(n, X, k, C, na, S);
        for (size_t q = 0; q < (size_t)n * na; q++) W[q] -= S[q];
        if (cholqr(n, W, NULL, na, work)) { st = ORA_BREAKDOWN; goto done; }
        for (int a = 0; a < na; a++) {
            for (int64_t i = 0; i < n; i++) v[i] = W[i * na + a];
            ora_spmv(n, rp, ci, va, v, z);
            for (int64_t i = 0; i < n; i++) AW[i * na + a] = z[i];
        }
        /* P(:, active), orthonormal, with A P transformed alike */
        int np = 0;
        if (havep) {
            for (int64_t i = 0; i < n; i++)
                for (int a = 0; a < na; a++) {
                    S[i * na + a] = Pb[i * k + act[a]];
                    AS[i * na + a] = AP[i * k + act[a]];
                }
            memcpy(Pb, S, (size_t)n * na * 8);
            memcpy(AP, AS, (size_t)n * na * 8);
            np = cholqr(n, Pb, AP, na, work) ? 0 : na;
        }
        for (int attempt = 0; attempt < 2; attempt++) {
            int m = k + na + np;
            /* S = [X W P], AS = [AX AW AP] */
            for (int64_t i = 0; i < n; i++) {
                for (int a = 0; a < k; a++) { S[i * m + a] = X[i * k + a]; AS[i * m + a] = AX[i * k + a]; }
                for (int a = 0; a < na; a++) { S[i * m + k + a] = W[i * na + a]; AS[i * m + k + a] = AW[i * na + a]; }
                for (int a = 0; a < np; a++) {
                    S[i * m + k + na + a] = Pb[i * na + a];
                    AS[i * m + k + na + a] = AP[i * na + a];
                }
            }
            gram(n, S, m, AS, m, GA);
            gram(n, S, m, S, m, GB);
            for (int a = 0; a < m; a++) for (int b = 0; b < a; b++) {
                double s = 0.5 * (GA[a * m + b] + GA[b * m + a]); GA[a * m + b] = GA[b * m + a] = s;
                s = 0.5 * (GB[a * m + b] + GB[b * m + a]); GB[a * m + b] = GB[b * m + a] = s;
            }
            if (chol(m, GB)) {
                if (np > 0) { np = 0; continue; }              /* drop P and retry */
                st = ORA_BREAKDOWN;
                goto done;
            }
            tri_inv_lower(m, GB, LI);
            /* C = L^{-1} GA L^{-T} */
            for (int a = 0; a < m; a++) for (int b = 0; b < m; b++) {
                double s = 0.0;
                for (int q = 0; q <= a; q++) s += LI[a * m + q] * GA[q * m + b];
                Cf[a * m + b] = s;
            }
            for (int a = 0; a < m; a++) for (int b = 0; b < m; b++) {
                double s = 0.0;
                for (int q = 0; q <= b; q++) s += Cf[a * m + q] * LI[b * m + q];
                C[a * m + b] = s;
            }
            for (int a = 0; a < m; a++) for (int b = 0; b < a; b++) {
                double s = 0.5 * (C[a * m + b] + C[b * m + a]); C[a * m + b] = C[b * m + a] = s;
            }
            jacobi_eig(m, C, th, Y);
            /* coefficients c = L^{-T} Y(:, 0:k) */
            for (int a = 0; a < m; a++) for (int b = 0; b < k; b++) {
                double s = 0.0;
                for (int q = a; q < m; q++) s += LI[q * m + a] * Y[q * m + b];
                Cf[a * k + b] = s;
            }
            /* X = S c, AX = AS c, P = [W P] c(k:, :), AP = [AW AP] c(k:, :) */
            block_mul(n, S, m, Cf, k, X);
            block_mul(n, AS, m, Cf, k, AX);
            int mw = na + np;
            for (int64_t i = 0; i < n; i++)
                for (int b = 0; b < k; b++) {
                    double sp = 0.0, sa = 0.0;
                    for (int a = 0; a < mw; a++) {
                        sp += S[i * m + k + a] * Cf[(k + a) * k + b];
                        sa += AS[i * m + k + a] * Cf[(k + a) * k + b];
                    }
                    Pb[i * k + b] = sp;
                    AP[i * k + b] = sa;
                }
            havep = 1;
            for (int j = 0; j < k; j++) lambda[j] = th[j];
            break;
        }
    }
done:
    free(AX); free(R); free(W); free(AW); free(Pb); free(AP); free(S); free(AS); free(v); free(z); free(tmp);
    free(GA); free(GB); free(LI); free(C); free(Y); free(Cf); free(th); free(work); free(res); free(act);
    return st;
}

/* dense symmetric eigenvalues (Jacobi), exposed for pinning the helper */
int ora_sym_eig(int m, double *C, double *w, double *V)
{
    jacobi_eig(m, C, w, V);
    return ORA_OK;
}
