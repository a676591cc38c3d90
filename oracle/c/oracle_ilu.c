/*
 * Oracle (test infrastructure only): plain, slow, single-threaded C loops for
 * the incomplete factorisations and triangular substitutions that the GeMSLR
 * oracle needs.  Only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark may load this file; the CUDA library never does.
 *
 * Every matrix here is one diagonal block B^{(j)} in local 0-based CSR with
 * ascending column indices.  Factors are returned as
 *   L : strictly lower part, unit diagonal implied, ascending columns;
 *   U : upper part including the diagonal, ascending columns (so the
 *       diagonal is the first entry of each row).
 *
 * Readings of the paper that this file follows:
 *   - B_l^{-1} is replaced by (L_l U_l)^{-1} from an incomplete LU (Sec. 2.3,
 *     Alg. 1 "Compute ILU factorization").
 *   - ILU(0): the IKJ variant restricted to the pattern of B (Saad 2003, Alg. 10.4).
 *   - ILUT(tau, lfil): Saad's dual-threshold ILUT (the ILUT reference of Sec. 2.1),
 *     with every candidate entry measured in the units of the row being
 *     reduced so that the rule does not depend on the scaling of A: an L entry
 *     l_ik = w_k / u_kk is measured by |l_ik * u_kk| (the size of the entry it
 *     eliminates), a U entry by |u_ij|.  During the elimination l_ik is dropped
 *     when its measure is below tau*||a_i||_2; afterwards off-diagonal entries
 *     below tau*||a_i||_2 are dropped and only the lfil largest (by the same
 *     measure) of the L part and of the U part are kept (ties: smaller column
 *     first); the diagonal is always kept.  lfil < 0 means "keep all".
 *   - Small pivots (not discussed by the paper): if |u_ii| < 1e-12*||a_i||_2
 *     then u_ii = sign(u_ii)*1e-12*||a_i||_2 (+ for 0), and the event is
 *     counted; an all-zero row gets u_ii = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double row_norm2(const int64_t *rp, const double *val, int64_t i) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += val[p] * val[p];
    return sqrt(s);
}

static double clamp_pivot(double u, double nrm, int64_t *nclamp) {
    double thr = 1e-12 * nrm;
    if (nrm == 0.0) {
        if (u == 0.0) { (*nclamp)++; return 1.0; }
        return u;
    }
    if (fabs(u) < thr) {
        (*nclamp)++;
        return (u < 0.0) ? -thr : thr;
    }
    return u;
}

/* Growable row storage used by both factorisations. */
typedef struct { int64_t *rp; int32_t *ci; double *v; int64_t cap, nnz; } rows_t;

static int rows_init(rows_t *r, int64_t n, int64_t cap) {
    r->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    r->ci = (int32_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    r->v = (double *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(double));
    r->cap = cap > 0 ? cap : 1;
    r->nnz = 0;
    return (r->rp && r->ci && r->v) ? 0 : -1;
}

static int rows_push(rows_t *r, int32_t c, double v) {
    if (r->nnz == r->cap) {
        int64_t nc = r->cap * 2;
        int32_t *ci = (int32_t *)realloc(r->ci, (size_t)nc * sizeof(int32_t));
        double *vv = (double *)realloc(r->v, (size_t)nc * sizeof(double));
        if (!ci || !vv) return -1;
        r->ci = ci; r->v = vv; r->cap = nc;
    }
    r->ci[r->nnz] = c;
    r->v[r->nnz] = v;
    r->nnz++;
    return 0;
}

/* Result handle returned to Python (freed with oracle_free_factors). */
typedef struct {
    int64_t n;
    int64_t *lrp; int32_t *lci; double *lv;
    int64_t *urp; int32_t *uci; double *uv;
    int64_t nclamp;
} oracle_factors;

void oracle_free_factors(oracle_factors *f) {
    if (!f) return;
    free(f->lrp); free(f->lci); free(f->lv);
    free(f->urp); free(f->uci); free(f->uv);
    free(f);
}

static oracle_factors *finish(int64_t n, rows_t *L, rows_t *U, int64_t nclamp) {
    oracle_factors *f = (oracle_factors *)calloc(1, sizeof(oracle_factors));
    f->n = n;
    f->lrp = L->rp; f->lci = L->ci; f->lv = L->v;
    f->urp = U->rp; f->uci = U->ci; f->uv = U->v;
    f->nclamp = nclamp;
    return f;
}

/* ILU(0), IKJ variant on the pattern of B. */
oracle_factors *oracle_ilu0(int64_t n, const int64_t *rp, const int32_t *ci, const double *val) {
    rows_t L, U;
    int64_t nnz = rp[n];
    if (rows_init(&L, n, nnz) || rows_init(&U, n, nnz)) return NULL;
    /* w: dense row, pos: column -> marker (row index + 1 when in pattern of row i) */
    double *w = (double *)calloc((size_t)n + 1, sizeof(double));
    int64_t *mark = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    double *udiag = (double *)calloc((size_t)n + 1, sizeof(double));
    int64_t nclamp = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { w[ci[p]] = val[p]; mark[ci[p]] = i + 1; }
        /* eliminate in ascending k < i over the pattern of row i */
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t k = ci[p];
            if (k >= i) break;
            w[k] = w[k] / udiag[k];
            double wk = w[k];
            for (int64_t q = U.rp[k]; q < U.rp[k + 1]; ++q) {
                int32_t j = U.ci[q];
                if (j <= k) continue;           /* skip the diagonal */
                if (mark[j] == i + 1) w[j] -= wk * U.v[q];
            }
        }
        double nrm = row_norm2(rp, val, i);
        int has_diag = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) if (ci[p] == i) has_diag = 1;
        double d = has_diag ? w[i] : 0.0;
        d = clamp_pivot(d, nrm, &nclamp);
        udiag[i] = d;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t c = ci[p];
            if (c < i) rows_push(&L, c, w[c]);
        }
        rows_push(&U, (int32_t)i, d);
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t c = ci[p];
            if (c > i) rows_push(&U, c, w[c]);
        }
        L.rp[i + 1] = L.nnz;
        U.rp[i + 1] = U.nnz;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { w[ci[p]] = 0.0; }
    }
    free(w); free(mark); free(udiag);
    return finish(n, &L, &U, nclamp);
}

/* selection helper: order by |value| descending, then column ascending */
typedef struct { int32_t c; double v; } ent_t;
static int cmp_mag(const void *a, const void *b) {
    const ent_t *x = (const ent_t *)a, *y = (const ent_t *)b;
    double ax = fabs(x->v), ay = fabs(y->v);
    if (ax > ay) return -1;
    if (ax < ay) return 1;
    return (x->c < y->c) ? -1 : (x->c > y->c);
}
static int cmp_col(const void *a, const void *b) {
    const ent_t *x = (const ent_t *)a, *y = (const ent_t *)b;
    return (x->c < y->c) ? -1 : (x->c > y->c);
}

/* ILUT(tau, lfil), Saad's dual threshold rule. */
oracle_factors *oracle_ilut(int64_t n, const int64_t *rp, const int32_t *ci, const double *val,
                            double tau, int64_t lfil) {
    rows_t L, U;
    int64_t nnz = rp[n];
    if (rows_init(&L, n, 2 * nnz) || rows_init(&U, n, 2 * nnz)) return NULL;
    double *w = (double *)calloc((size_t)n + 1, sizeof(double));
    char *in = (char *)calloc((size_t)n + 1, 1);         /* column j in the pattern of w */
    int32_t *lst = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    ent_t *buf = (ent_t *)malloc(((size_t)n + 1) * sizeof(ent_t));
    double *udiag = (double *)calloc((size_t)n + 1, sizeof(double));
    char *done = (char *)calloc((size_t)n + 1, 1);       /* k already eliminated in this row */
    int64_t nclamp = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t len = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            w[ci[p]] = val[p];
            if (!in[ci[p]]) { in[ci[p]] = 1; lst[len++] = ci[p]; }
        }
        double nrm = row_norm2(rp, val, i);
        double thr = tau * nrm;
        /* eliminate columns k < i in ascending order, including fill that appears */
        for (;;) {
            int32_t k = -1;
            for (int64_t t = 0; t < len; ++t) {
                int32_t c = lst[t];
                if (c < i && !done[c] && (k < 0 || c < k)) k = c;
            }
            if (k < 0) break;
            done[k] = 1;
            if (fabs(w[k]) < thr) { w[k] = 0.0; continue; }   /* |l_ik * u_kk| = |w_k| */
            w[k] = w[k] / udiag[k];
            double wk = w[k];
            for (int64_t q = U.rp[k]; q < U.rp[k + 1]; ++q) {
                int32_t j = U.ci[q];
                if (j <= k) continue;
                if (!in[j]) { in[j] = 1; w[j] = 0.0; lst[len++] = j; }
                w[j] -= wk * U.v[q];
            }
        }
        /* L part */
        int64_t nl = 0;
        for (int64_t t = 0; t < len; ++t) {
            int32_t c = lst[t];
            /* measure of l_ic: |l_ic * u_cc| */
            if (c < i && w[c] != 0.0 && fabs(w[c] * udiag[c]) >= thr) {
                buf[nl].c = c; buf[nl].v = w[c] * udiag[c]; nl++;
            }
        }
        if (lfil >= 0 && nl > lfil) { qsort(buf, (size_t)nl, sizeof(ent_t), cmp_mag); nl = lfil; }
        qsort(buf, (size_t)nl, sizeof(ent_t), cmp_col);
        for (int64_t t = 0; t < nl; ++t) rows_push(&L, buf[t].c, w[buf[t].c]);
        /* U part: diagonal first, then the kept off-diagonals in column order */
        double d = in[i] ? w[i] : 0.0;
        d = clamp_pivot(d, nrm, &nclamp);
        udiag[i] = d;
        rows_push(&U, (int32_t)i, d);
        int64_t nu = 0;
        for (int64_t t = 0; t < len; ++t) {
            int32_t c = lst[t];
            if (c > i && w[c] != 0.0 && fabs(w[c]) >= thr) { buf[nu].c = c; buf[nu].v = w[c]; nu++; }
        }
        if (lfil >= 0 && nu > lfil) { qsort(buf, (size_t)nu, sizeof(ent_t), cmp_mag); nu = lfil; }
        qsort(buf, (size_t)nu, sizeof(ent_t), cmp_col);
        for (int64_t t = 0; t < nu; ++t) rows_push(&U, buf[t].c, buf[t].v);
        L.rp[i + 1] = L.nnz;
        U.rp[i + 1] = U.nnz;
        for (int64_t t = 0; t < len; ++t) { int32_t c = lst[t]; w[c] = 0.0; in[c] = 0; done[c] = 0; }
    }
    free(w); free(in); free(lst); free(buf); free(udiag); free(done);
    return finish(n, &L, &U, nclamp);
}

/* x = L^{-1} b with unit diagonal (L strictly lower). In place allowed. */
void oracle_lsolve(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                   const double *b, double *x) {
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s -= v[p] * x[ci[p]];
        x[i] = s;
    }
}

/* x = U^{-1} b, U upper with its diagonal as the first entry of each row. In place allowed. */
void oracle_usolve(int64_t n, const int64_t *rp, const int32_t *ci, const double *v,
                   const double *b, double *x) {
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = b[i];
        double d = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (ci[p] == i) d = v[p];
            else s -= v[p] * x[ci[p]];
        }
        x[i] = s / d;
    }
}
