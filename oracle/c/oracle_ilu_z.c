/*
 * Oracle (test infrastructure only): the complex counterparts of
 * oracle_ilu.c, for the complex version of the method (Sec. 5.2.3: the
 * on-diagonal blocks are factored with a complex diagonal shift, so the
 * factors and every vector of the application are complex).  Only tests/,
 * the smoke check and the CPU-baseline leg of the benchmark may load this
 * file; the CUDA library never does.
 *
 * Same conventions as oracle_ilu.c (local 0-based CSR blocks, ascending
 * columns; L strictly lower with unit diagonal implied; U with its diagonal
 * first), with these readings for complex entries:
 *   - every magnitude in the dual-threshold rule is the complex modulus
 *     |z| (Saad's ILUT for complex matrices), measured as in the real file:
 *     l_ik by |l_ik * u_kk|, u_ij by |u_ij|, against tau*||a_i||_2 where
 *     ||a_i||_2 is the 2-norm of the row's moduli;
 *   - a small pivot keeps its phase: if |u_ii| < 1e-12*||a_i||_2 then
 *     u_ii = (u_ii/|u_ii|)*1e-12*||a_i||_2 (+1e-12*||a_i||_2 for 0), counted;
 *     an all-zero row gets u_ii = 1.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex zd;

static double row_norm2_z(const int64_t *rp, const zd *val, int64_t i) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += creal(val[p] * conj(val[p]));
    return sqrt(s);
}

static zd clamp_pivot_z(zd u, double nrm, int64_t *nclamp) {
    double thr = 1e-12 * nrm;
    if (nrm == 0.0) {
        if (u == 0.0) { (*nclamp)++; return 1.0; }
        return u;
    }
    if (cabs(u) < thr) {
        (*nclamp)++;
        return (u == 0.0) ? thr : u * (thr / cabs(u));
    }
    return u;
}

typedef struct { int64_t *rp; int32_t *ci; zd *v; int64_t cap, nnz; } zrows_t;

static int zrows_init(zrows_t *r, int64_t n, int64_t cap) {
    r->rp = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    r->ci = (int32_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int32_t));
    r->v = (zd *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(zd));
    r->cap = cap > 0 ? cap : 1;
    r->nnz = 0;
    return (r->rp && r->ci && r->v) ? 0 : -1;
}

static int zrows_push(zrows_t *r, int32_t c, zd v) {
    if (r->nnz == r->cap) {
        int64_t nc = r->cap * 2;
        int32_t *ci = (int32_t *)realloc(r->ci, (size_t)nc * sizeof(int32_t));
        zd *vv = (zd *)realloc(r->v, (size_t)nc * sizeof(zd));
        if (!ci || !vv) return -1;
        r->ci = ci; r->v = vv; r->cap = nc;
    }
    r->ci[r->nnz] = c;
    r->v[r->nnz] = v;
    r->nnz++;
    return 0;
}

typedef struct {
    int64_t n;
    int64_t *lrp; int32_t *lci; zd *lv;
    int64_t *urp; int32_t *uci; zd *uv;
    int64_t nclamp;
} oracle_factors_z;

void oracle_free_factors_z(oracle_factors_z *f) {
    if (!f) return;
    free(f->lrp); free(f->lci); free(f->lv);
    free(f->urp); free(f->uci); free(f->uv);
    free(f);
}

static oracle_factors_z *finish_z(int64_t n, zrows_t *L, zrows_t *U, int64_t nclamp) {
    oracle_factors_z *f = (oracle_factors_z *)calloc(1, sizeof(oracle_factors_z));
    f->n = n;
    f->lrp = L->rp; f->lci = L->ci; f->lv = L->v;
    f->urp = U->rp; f->uci = U->ci; f->uv = U->v;
    f->nclamp = nclamp;
    return f;
}

/* ILU(0), IKJ variant on the pattern of B (complex). */
oracle_factors_z *oracle_ilu0_z(int64_t n, const int64_t *rp, const int32_t *ci, const zd *val) {
    zrows_t L, U;
    int64_t nnz = rp[n];
    if (zrows_init(&L, n, nnz) || zrows_init(&U, n, nnz)) return NULL;
    zd *w = (zd *)calloc((size_t)n + 1, sizeof(zd));
    int64_t *mark = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    zd *udiag = (zd *)calloc((size_t)n + 1, sizeof(zd));
    int64_t nclamp = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { w[ci[p]] = val[p]; mark[ci[p]] = i + 1; }
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t k = ci[p];
            if (k >= i) break;
            w[k] = w[k] / udiag[k];
            zd wk = w[k];
            for (int64_t q = U.rp[k]; q < U.rp[k + 1]; ++q) {
                int32_t j = U.ci[q];
                if (j <= k) continue;
                if (mark[j] == i + 1) w[j] -= wk * U.v[q];
            }
        }
        double nrm = row_norm2_z(rp, val, i);
        int has_diag = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) if (ci[p] == i) has_diag = 1;
        zd d = has_diag ? w[i] : 0.0;
        d = clamp_pivot_z(d, nrm, &nclamp);
        udiag[i] = d;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t c = ci[p];
            if (c < i) zrows_push(&L, c, w[c]);
        }
        zrows_push(&U, (int32_t)i, d);
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t c = ci[p];
            if (c > i) zrows_push(&U, c, w[c]);
        }
        L.rp[i + 1] = L.nnz;
        U.rp[i + 1] = U.nnz;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) { w[ci[p]] = 0.0; }
    }
    free(w); free(mark); free(udiag);
    return finish_z(n, &L, &U, nclamp);
}

typedef struct { int32_t c; double mag; zd v; } zent_t;
static int cmp_mag_z(const void *a, const void *b) {
    const zent_t *x = (const zent_t *)a, *y = (const zent_t *)b;
    if (x->mag > y->mag) return -1;
    if (x->mag < y->mag) return 1;
    return (x->c < y->c) ? -1 : (x->c > y->c);
}
static int cmp_col_z(const void *a, const void *b) {
    const zent_t *x = (const zent_t *)a, *y = (const zent_t *)b;
    return (x->c < y->c) ? -1 : (x->c > y->c);
}

/* ILUT(tau, lfil) for complex entries, Saad's dual threshold rule. */
oracle_factors_z *oracle_ilut_z(int64_t n, const int64_t *rp, const int32_t *ci, const zd *val,
                                double tau, int64_t lfil) {
    zrows_t L, U;
    int64_t nnz = rp[n];
    if (zrows_init(&L, n, 2 * nnz) || zrows_init(&U, n, 2 * nnz)) return NULL;
    zd *w = (zd *)calloc((size_t)n + 1, sizeof(zd));
    char *in = (char *)calloc((size_t)n + 1, 1);
    int32_t *lst = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    zent_t *buf = (zent_t *)malloc(((size_t)n + 1) * sizeof(zent_t));
    zd *udiag = (zd *)calloc((size_t)n + 1, sizeof(zd));
    char *done = (char *)calloc((size_t)n + 1, 1);
    int64_t nclamp = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t len = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            w[ci[p]] = val[p];
            if (!in[ci[p]]) { in[ci[p]] = 1; lst[len++] = ci[p]; }
        }
        double nrm = row_norm2_z(rp, val, i);
        double thr = tau * nrm;
        for (;;) {
            int32_t k = -1;
            for (int64_t t = 0; t < len; ++t) {
                int32_t c = lst[t];
                if (c < i && !done[c] && (k < 0 || c < k)) k = c;
            }
            if (k < 0) break;
            done[k] = 1;
            if (cabs(w[k]) < thr) { w[k] = 0.0; continue; }   /* |l_ik * u_kk| = |w_k| */
            w[k] = w[k] / udiag[k];
            zd wk = w[k];
            for (int64_t q = U.rp[k]; q < U.rp[k + 1]; ++q) {
                int32_t j = U.ci[q];
                if (j <= k) continue;
                if (!in[j]) { in[j] = 1; w[j] = 0.0; lst[len++] = j; }
                w[j] -= wk * U.v[q];
            }
        }
        int64_t nl = 0;
        for (int64_t t = 0; t < len; ++t) {
            int32_t c = lst[t];
            if (c < i && w[c] != 0.0 && cabs(w[c] * udiag[c]) >= thr) {
                buf[nl].c = c; buf[nl].mag = cabs(w[c] * udiag[c]); buf[nl].v = w[c]; nl++;
            }
        }
        if (lfil >= 0 && nl > lfil) { qsort(buf, (size_t)nl, sizeof(zent_t), cmp_mag_z); nl = lfil; }
        qsort(buf, (size_t)nl, sizeof(zent_t), cmp_col_z);
        for (int64_t t = 0; t < nl; ++t) zrows_push(&L, buf[t].c, buf[t].v);
        zd d = in[i] ? w[i] : 0.0;
        d = clamp_pivot_z(d, nrm, &nclamp);
        udiag[i] = d;
        zrows_push(&U, (int32_t)i, d);
        int64_t nu = 0;
        for (int64_t t = 0; t < len; ++t) {
            int32_t c = lst[t];
            if (c > i && w[c] != 0.0 && cabs(w[c]) >= thr) {
                buf[nu].c = c; buf[nu].mag = cabs(w[c]); buf[nu].v = w[c]; nu++;
            }
        }
        if (lfil >= 0 && nu > lfil) { qsort(buf, (size_t)nu, sizeof(zent_t), cmp_mag_z); nu = lfil; }
        qsort(buf, (size_t)nu, sizeof(zent_t), cmp_col_z);
        for (int64_t t = 0; t < nu; ++t) zrows_push(&U, buf[t].c, buf[t].v);
        L.rp[i + 1] = L.nnz;
        U.rp[i + 1] = U.nnz;
        for (int64_t t = 0; t < len; ++t) { int32_t c = lst[t]; w[c] = 0.0; in[c] = 0; done[c] = 0; }
    }
    free(w); free(in); free(lst); free(buf); free(udiag); free(done);
    return finish_z(n, &L, &U, nclamp);
}

/* x = L^{-1} b with unit diagonal (complex). In place allowed. */
void oracle_lsolve_z(int64_t n, const int64_t *rp, const int32_t *ci, const zd *v, const zd *b, zd *x) {
    for (int64_t i = 0; i < n; ++i) {
        zd s = b[i];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s -= v[p] * x[ci[p]];
        x[i] = s;
    }
}

/* x = U^{-1} b, diagonal first in each row (complex). In place allowed. */
void oracle_usolve_z(int64_t n, const int64_t *rp, const int32_t *ci, const zd *v, const zd *b, zd *x) {
    for (int64_t i = n - 1; i >= 0; --i) {
        zd s = b[i];
        zd d = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (ci[p] == i) d = v[p];
            else s -= v[p] * x[ci[p]];
        }
        x[i] = s / d;
    }
}
