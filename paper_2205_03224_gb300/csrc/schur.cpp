// Dense Schur machinery for the low-rank correction (Sec. 2.3): the Ritz
// matrix H_m of the Arnoldi relation is brought to complex Schur form
// H_m = Q T Q^H (the paper's "complex Schur decomposition of H_m"), the
// wanted Ritz values are moved to the leading positions, and because the
// data are real and conjugate pairs are never split, the leading invariant
// subspace is real: an orthonormal real basis of it is extracted and
// T_k = Q_k^T H_m Q_k is formed.  W H W^T does not depend on the basis of
// that subspace, so this is the same correction as the real-Schur one.
//
// Methods (textbook, own code): Householder reduction to Hessenberg form;
// implicit single-shift complex QR with Wilkinson shifts and deflation
// (Golub & Van Loan, 4th ed., Sec. 7.4-7.5); swapping of adjacent diagonal
// entries of a triangular matrix by one plane rotation built from the
// eigenvector of the 2x2 block (Sec. 7.6.2); pivoted Gram-Schmidt for the
// real basis.
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>

#include "internal.h"

namespace gemslr {

namespace {

using cplx = std::complex<double>;
constexpr double kEps = 2.220446049250313e-16;

// G = [c s; -conj(s) c] with G [x; y] = [r; 0], c real.
void rotation(cplx x, cplx y, double &c, cplx &s) {
    if (y == cplx(0.0)) { c = 1.0; s = 0.0; return; }
    if (x == cplx(0.0)) { c = 0.0; s = 1.0; return; }
    const double ax = std::abs(x), ay = std::abs(y);
    const double rho = std::hypot(ax, ay);
    c = ax / rho;
    s = (x / ax) * std::conj(y) / rho;
}

struct CMat {
    int m;
    std::vector<cplx> a;
    explicit CMat(int m_) : m(m_), a((size_t)m_ * m_, 0.0) {}
    cplx &operator()(int i, int j) { return a[i + (size_t)j * m]; }
};

// rows p, p+1 of T (columns j0..m-1) <- G * rows
void rot_rows(CMat &T, int p, int j0, double c, cplx s) {
    for (int j = j0; j < T.m; ++j) {
        const cplx t1 = T(p, j), t2 = T(p + 1, j);
        T(p, j) = c * t1 + s * t2;
        T(p + 1, j) = -std::conj(s) * t1 + c * t2;
    }
}
// columns p, p+1 of M (rows 0..i1) <- cols * G^H
void rot_cols(CMat &M, int p, int i1, double c, cplx s) {
    for (int i = 0; i <= i1; ++i) {
        const cplx t1 = M(i, p), t2 = M(i, p + 1);
        M(i, p) = t1 * c + t2 * std::conj(s);
        M(i, p + 1) = -t1 * s + t2 * c;
    }
}

// Real Householder Hessenberg reduction: A <- Q^T A Q, returns Q (column-major).
void hessenberg(std::vector<double> &A, int m, std::vector<double> &Q) {
    Q.assign((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Q[i + (size_t)i * m] = 1.0;
    std::vector<double> v(m);
    for (int k = 0; k + 2 < m; ++k) {
        double nx = 0.0;
        for (int i = k + 1; i < m; ++i) nx += A[i + (size_t)k * m] * A[i + (size_t)k * m];
        nx = std::sqrt(nx);
        if (nx == 0.0) continue;
        const double x0 = A[(k + 1) + (size_t)k * m];
        const double alpha = x0 >= 0.0 ? -nx : nx;
        std::fill(v.begin(), v.end(), 0.0);
        for (int i = k + 1; i < m; ++i) v[i] = A[i + (size_t)k * m];
        v[k + 1] -= alpha;
        double nv = 0.0;
        for (int i = k + 1; i < m; ++i) nv += v[i] * v[i];
        nv = std::sqrt(nv);
        if (nv == 0.0) continue;
        for (int i = k + 1; i < m; ++i) v[i] /= nv;
        for (int j = 0; j < m; ++j) {            // A <- (I - 2vv^T) A
            double d = 0.0;
            for (int i = k + 1; i < m; ++i) d += v[i] * A[i + (size_t)j * m];
            for (int i = k + 1; i < m; ++i) A[i + (size_t)j * m] -= 2.0 * d * v[i];
        }
        for (int i = 0; i < m; ++i) {            // A <- A (I - 2vv^T), Q <- Q (I - 2vv^T)
            double d = 0.0, e = 0.0;
            for (int j = k + 1; j < m; ++j) { d += A[i + (size_t)j * m] * v[j]; e += Q[i + (size_t)j * m] * v[j]; }
            for (int j = k + 1; j < m; ++j) { A[i + (size_t)j * m] -= 2.0 * d * v[j]; Q[i + (size_t)j * m] -= 2.0 * e * v[j]; }
        }
        for (int i = k + 2; i < m; ++i) A[i + (size_t)k * m] = 0.0;
    }
}

// Complex Schur form of an upper Hessenberg T (in place), accumulating Z.
void complex_schur(CMat &T, CMat &Z) {
    const int m = T.m;
    double anorm = 0.0;
    for (auto &z : T.a) anorm += std::norm(z);
    anorm = std::sqrt(anorm);
    int hi = m - 1, iter = 0, total = 0;
    while (hi > 0) {
        int l = hi;
        for (; l > 0; --l) {
            double tst = std::abs(T(l - 1, l - 1)) + std::abs(T(l, l));
            if (tst == 0.0) tst = anorm;
            if (std::abs(T(l, l - 1)) <= kEps * tst) { T(l, l - 1) = 0.0; break; }
        }
        if (l == hi) { --hi; iter = 0; continue; }
        ++iter;
        if (++total > 200 * m) fail(GEMSLR_ERR_NOT_CONVERGED, "complex QR iteration did not converge");
        cplx mu;
        if (iter % 12 == 11) {
            mu = T(hi, hi) + 0.75 * std::abs(T(hi, hi - 1));   // exceptional shift
        } else {
            const cplx a = T(hi - 1, hi - 1), b = T(hi - 1, hi), c = T(hi, hi - 1), d = T(hi, hi);
            const cplx half = 0.5 * (a + d);
            const cplx disc = std::sqrt(0.25 * (a - d) * (a - d) + b * c);
            const cplx m1 = half + disc, m2 = half - disc;
            mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        }
        for (int k = l; k < hi; ++k) {
            cplx x, y;
            if (k == l) { x = T(l, l) - mu; y = T(l + 1, l); }
            else { x = T(k, k - 1); y = T(k + 1, k - 1); }
            double c;
            cplx s;
            rotation(x, y, c, s);
            rot_rows(T, k, k == l ? l : k - 1, c, s);
            rot_cols(T, k, std::min(k + 2, hi), c, s);
            rot_cols(Z, k, m - 1, c, s);
            if (k > l) T(k + 1, k - 1) = 0.0;
        }
    }
    for (int j = 0; j < m; ++j)
        for (int i = j + 1; i < m; ++i) T(i, j) = 0.0;
}

// Exchange diagonal entries p and p+1 of the triangular T (Z accumulates).
void swap_adjacent(CMat &T, CMat &Z, int p) {
    const cplx t11 = T(p, p), t22 = T(p + 1, p + 1);
    double c;
    cplx s;
    rotation(T(p, p + 1), t22 - t11, c, s);
    rot_rows(T, p, p, c, s);
    rot_cols(T, p, p + 1, c, s);
    rot_cols(Z, p, Z.m - 1, c, s);
    T(p, p) = t22;
    T(p + 1, p + 1) = t11;
    T(p + 1, p) = 0.0;
}

double score(cplx t) {
    const double den = std::abs(1.0 - t);
    return den == 0.0 ? INFINITY : std::abs(t) / den;
}

// Complex Householder reduction to upper Hessenberg form: T <- P T P with
// P = I - 2 v v^H / (v^H v) per column (P Hermitian and unitary), Z <- Z P.
void complex_hessenberg(CMat &T, CMat &Z) {
    const int m = T.m;
    std::vector<cplx> v(m);
    for (int k = 0; k + 2 < m; ++k) {
        double nx = 0.0;
        for (int i = k + 1; i < m; ++i) nx += std::norm(T(i, k));
        nx = std::sqrt(nx);
        if (nx == 0.0) continue;
        const cplx x0 = T(k + 1, k);
        const cplx phase = std::abs(x0) == 0.0 ? cplx(1.0) : x0 / std::abs(x0);
        const cplx alpha = -phase * nx;
        std::fill(v.begin(), v.end(), cplx(0.0));
        for (int i = k + 1; i < m; ++i) v[i] = T(i, k);
        v[k + 1] -= alpha;
        double nv = 0.0;
        for (int i = k + 1; i < m; ++i) nv += std::norm(v[i]);
        if (nv == 0.0) continue;
        const double f = 2.0 / nv;
        for (int j = 0; j < m; ++j) {          // rows: T <- P T
            cplx d = 0.0;
            for (int i = k + 1; i < m; ++i) d += std::conj(v[i]) * T(i, j);
            d *= f;
            for (int i = k + 1; i < m; ++i) T(i, j) -= v[i] * d;
        }
        for (int i = 0; i < m; ++i) {          // columns: T <- T P, Z <- Z P
            cplx d = 0.0, e = 0.0;
            for (int j = k + 1; j < m; ++j) { d += T(i, j) * v[j]; e += Z(i, j) * v[j]; }
            d *= f;
            e *= f;
            for (int j = k + 1; j < m; ++j) {
                T(i, j) -= d * std::conj(v[j]);
                Z(i, j) -= e * std::conj(v[j]);
            }
        }
        for (int i = k + 2; i < m; ++i) T(i, k) = 0.0;
    }
}

}  // namespace

int schur_wanted(const std::vector<double> &Hm, int m, int k, std::vector<double> &Q,
                 std::vector<double> &Tk, std::vector<double> &theta_re,
                 std::vector<double> &theta_im) {
    k = std::min(k, m);
    std::vector<double> Hh = Hm, Q0;
    hessenberg(Hh, m, Q0);
    CMat T(m), Z(m);
    for (size_t i = 0; i < Hh.size(); ++i) { T.a[i] = Hh[i]; Z.a[i] = Q0[i]; }
    complex_schur(T, Z);
    // ranking: |theta/(1-theta)| desc, |theta| desc, position asc
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::vector<cplx> th(m);
    for (int i = 0; i < m; ++i) th[i] = T(i, i);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        const double sa = score(th[a]), sb = score(th[b]);
        if (sa != sb) return sa > sb;
        const double ma = std::abs(th[a]), mb = std::abs(th[b]);
        if (ma != mb) return ma > mb;
        return a < b;
    });
    std::vector<int> want(ord.begin(), ord.begin() + k);
    if (k > 0 && k < m) {
        const cplx last = th[want.back()];
        if (std::abs(last.imag()) > 1e-10 * std::abs(last)) {
            // keep the pair whole: add the closest remaining value to conj(last)
            bool have = false;
            for (int i = 0; i + 1 < k; ++i)
                if (std::abs(th[want[i]] - std::conj(last)) <= 1e-8 * std::abs(last)) have = true;
            if (!have) {
                int best = -1;
                for (int i = k; i < m; ++i)
                    if (best < 0 || std::abs(th[ord[i]] - std::conj(last)) < std::abs(th[best] - std::conj(last)))
                        best = ord[i];
                want.push_back(best);
            }
        }
    }
    const int keff = (int)want.size();
    // move the wanted values to the front, in rank order
    std::vector<int> at(m), who(m);   // at[orig] = current position, who[pos] = orig
    std::iota(at.begin(), at.end(), 0);
    std::iota(who.begin(), who.end(), 0);
    for (int t = 0; t < keff; ++t) {
        for (int p = at[want[t]] - 1; p >= t; --p) {
            swap_adjacent(T, Z, p);
            std::swap(who[p], who[p + 1]);
            at[who[p]] = p;
            at[who[p + 1]] = p + 1;
        }
    }
    theta_re.resize(keff);
    theta_im.resize(keff);
    for (int t = 0; t < keff; ++t) { theta_re[t] = T(t, t).real(); theta_im[t] = T(t, t).imag(); }
    // real orthonormal basis of span(Z[:, :keff]) by pivoted Gram-Schmidt on [Re | Im]
    std::vector<std::vector<double>> cols;
    for (int t = 0; t < keff; ++t) {
        std::vector<double> re(m), im(m);
        for (int i = 0; i < m; ++i) { re[i] = Z(i, t).real(); im[i] = Z(i, t).imag(); }
        cols.push_back(re);
        cols.push_back(im);
    }
    Q.assign((size_t)m * keff, 0.0);
    std::vector<char> used(cols.size(), 0);
    for (int t = 0; t < keff; ++t) {
        int best = -1;
        double bn = -1.0;
        for (size_t c = 0; c < cols.size(); ++c) {
            if (used[c]) continue;
            double nn = 0.0;
            for (double x : cols[c]) nn += x * x;
            if (nn > bn) { bn = nn; best = (int)c; }
        }
        used[best] = 1;
        std::vector<double> q = cols[best];
        for (int pass = 0; pass < 2; ++pass)
            for (int r = 0; r < t; ++r) {
                double d = 0.0;
                for (int i = 0; i < m; ++i) d += Q[i + (size_t)r * m] * q[i];
                for (int i = 0; i < m; ++i) q[i] -= d * Q[i + (size_t)r * m];
            }
        double nq = 0.0;
        for (double x : q) nq += x * x;
        nq = std::sqrt(nq);
        if (nq == 0.0) fail(GEMSLR_ERR_NOT_CONVERGED, "degenerate invariant subspace");
        for (int i = 0; i < m; ++i) Q[i + (size_t)t * m] = q[i] / nq;
        for (size_t c = 0; c < cols.size(); ++c) {
            if (used[c]) continue;
            for (int pass = 0; pass < 2; ++pass) {
                double d = 0.0;
                for (int i = 0; i < m; ++i) d += Q[i + (size_t)t * m] * cols[c][i];
                for (int i = 0; i < m; ++i) cols[c][i] -= d * Q[i + (size_t)t * m];
            }
        }
    }
    // Tk = Q^T Hm Q
    std::vector<double> HQ((size_t)m * keff, 0.0);
    for (int t = 0; t < keff; ++t)
        for (int j = 0; j < m; ++j) {
            const double q = Q[j + (size_t)t * m];
            if (q == 0.0) continue;
            for (int i = 0; i < m; ++i) HQ[i + (size_t)t * m] += Hm[i + (size_t)j * m] * q;
        }
    Tk.assign((size_t)keff * keff, 0.0);
    for (int b = 0; b < keff; ++b)
        for (int a = 0; a < keff; ++a) {
            double d = 0.0;
            for (int i = 0; i < m; ++i) d += Q[i + (size_t)a * m] * HQ[i + (size_t)b * m];
            Tk[a + (size_t)b * keff] = d;
        }
    return keff;
}

// Complex counterpart (complex-shifted hierarchy): complex Schur form of a
// general m x m Hm (Householder Hessenberg, then the complex QR above), the
// same ranking of the Ritz values, exactly k kept (no conjugate pairs to keep
// whole), moved to the front by adjacent swaps; Q = Z[:, :k] is already an
// orthonormal basis of the wanted invariant subspace and Tk = T[:k, :k].
int schur_wanted_z(const std::vector<cplx> &Hm, int m, int k, std::vector<cplx> &Q, std::vector<cplx> &Tk,
                   std::vector<cplx> &theta) {
    k = std::min(k, m);
    CMat T(m), Z(m);
    T.a = Hm;
    for (int i = 0; i < m; ++i) Z(i, i) = 1.0;
    complex_hessenberg(T, Z);
    complex_schur(T, Z);
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::vector<cplx> th(m);
    for (int i = 0; i < m; ++i) th[i] = T(i, i);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        const double sa = score(th[a]), sb = score(th[b]);
        if (sa != sb) return sa > sb;
        const double ma = std::abs(th[a]), mb = std::abs(th[b]);
        if (ma != mb) return ma > mb;
        return a < b;
    });
    std::vector<int> at(m), who(m);
    std::iota(at.begin(), at.end(), 0);
    std::iota(who.begin(), who.end(), 0);
    for (int t = 0; t < k; ++t) {
        for (int p = at[ord[t]] - 1; p >= t; --p) {
            swap_adjacent(T, Z, p);
            std::swap(who[p], who[p + 1]);
            at[who[p]] = p;
            at[who[p + 1]] = p + 1;
        }
    }
    Q.assign((size_t)m * k, 0.0);
    for (int t = 0; t < k; ++t)
        for (int i = 0; i < m; ++i) Q[i + (size_t)t * m] = Z(i, t);
    Tk.assign((size_t)k * k, 0.0);
    theta.resize(k);
    for (int b = 0; b < k; ++b) {
        theta[b] = T(b, b);
        for (int a = 0; a <= b; ++a) Tk[a + (size_t)b * k] = T(a, b);
    }
    return k;
}

std::vector<cplx> correction_matrix_z(const std::vector<cplx> &Tk, int k) {
    // (I - Tk)^{-1} - I by Gaussian elimination with partial pivoting (moduli)
    std::vector<cplx> M((size_t)k * k), X((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) M[i + (size_t)j * k] = (i == j ? cplx(1.0) : cplx(0.0)) - Tk[i + (size_t)j * k];
    for (int i = 0; i < k; ++i) X[i + (size_t)i * k] = 1.0;
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int i = c + 1; i < k; ++i)
            if (std::abs(M[i + (size_t)c * k]) > std::abs(M[piv + (size_t)c * k])) piv = i;
        if (M[piv + (size_t)c * k] == cplx(0.0)) fail(GEMSLR_ERR_NOT_CONVERGED, "I - T_k is singular");
        if (piv != c)
            for (int j = 0; j < k; ++j) {
                std::swap(M[c + (size_t)j * k], M[piv + (size_t)j * k]);
                std::swap(X[c + (size_t)j * k], X[piv + (size_t)j * k]);
            }
        for (int i = c + 1; i < k; ++i) {
            const cplx f = M[i + (size_t)c * k] / M[c + (size_t)c * k];
            if (f == cplx(0.0)) continue;
            for (int j = c; j < k; ++j) M[i + (size_t)j * k] -= f * M[c + (size_t)j * k];
            for (int j = 0; j < k; ++j) X[i + (size_t)j * k] -= f * X[c + (size_t)j * k];
        }
    }
    for (int j = 0; j < k; ++j)
        for (int i = k - 1; i >= 0; --i) {
            cplx s = X[i + (size_t)j * k];
            for (int t = i + 1; t < k; ++t) s -= M[i + (size_t)t * k] * X[t + (size_t)j * k];
            X[i + (size_t)j * k] = s / M[i + (size_t)i * k];
        }
    for (int i = 0; i < k; ++i) X[i + (size_t)i * k] -= 1.0;
    return X;
}

std::vector<double> correction_matrix(const std::vector<double> &Tk, int k) {
    // solve (I - Tk) X = I by Gaussian elimination with partial pivoting, then X - I
    std::vector<double> M((size_t)k * k), X((size_t)k * k, 0.0);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) M[i + (size_t)j * k] = (i == j ? 1.0 : 0.0) - Tk[i + (size_t)j * k];
    for (int i = 0; i < k; ++i) X[i + (size_t)i * k] = 1.0;
    for (int c = 0; c < k; ++c) {
        int piv = c;
        for (int i = c + 1; i < k; ++i)
            if (std::fabs(M[i + (size_t)c * k]) > std::fabs(M[piv + (size_t)c * k])) piv = i;
        if (M[piv + (size_t)c * k] == 0.0) fail(GEMSLR_ERR_NOT_CONVERGED, "I - T_k is singular");
        if (piv != c)
            for (int j = 0; j < k; ++j) {
                std::swap(M[c + (size_t)j * k], M[piv + (size_t)j * k]);
                std::swap(X[c + (size_t)j * k], X[piv + (size_t)j * k]);
            }
        for (int i = c + 1; i < k; ++i) {
            const double f = M[i + (size_t)c * k] / M[c + (size_t)c * k];
            if (f == 0.0) continue;
            for (int j = c; j < k; ++j) M[i + (size_t)j * k] -= f * M[c + (size_t)j * k];
            for (int j = 0; j < k; ++j) X[i + (size_t)j * k] -= f * X[c + (size_t)j * k];
        }
    }
    for (int j = 0; j < k; ++j)
        for (int i = k - 1; i >= 0; --i) {
            double s = X[i + (size_t)j * k];
            for (int t = i + 1; t < k; ++t) s -= M[i + (size_t)t * k] * X[t + (size_t)j * k];
            X[i + (size_t)j * k] = s / M[i + (size_t)i * k];
        }
    for (int i = 0; i < k; ++i) X[i + (size_t)i * k] -= 1.0;
    return X;
}

}  // namespace gemslr
