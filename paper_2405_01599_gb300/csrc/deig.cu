// Dense eigen-decomposition of a small general real matrix: the projected
// matrix of the restarted Arnoldi eigensolver (m <= 512).  Householder
// reduction to upper Hessenberg form, shifted QR steps in complex arithmetic
// (Wilkinson shift, deflation of converged subdiagonals) for the complex
// Schur form, reordering by adjacent swaps, and eigenvectors by back
// substitution in the triangular factor.  Host code: the matrix is tiny next
// to the Krylov basis it describes.
#include "common.cuh"
#include "deig.cuh"

#include <algorithm>
#include <cmath>

namespace {

using xb::cplx;
constexpr double kEps = 2.220446049250313e-16;

// In place: A (n x n, row-major) -> Hessenberg H = Q^T A Q; Q row-major.
void hessenberg(int n, std::vector<double> &A, std::vector<double> &Q) {
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; i++) Q[(size_t)i * n + i] = 1.0;
    std::vector<double> v(n);
    for (int k = 0; k + 2 < n; k++) {
        double alpha = 0.0;
        for (int i = k + 1; i < n; i++) alpha += A[(size_t)i * n + k] * A[(size_t)i * n + k];
        alpha = std::sqrt(alpha);
        if (alpha == 0.0) continue;
        const double beta = A[(size_t)(k + 1) * n + k] >= 0.0 ? -alpha : alpha;
        double vn = 0.0;
        for (int i = k + 1; i < n; i++) {
            v[i] = A[(size_t)i * n + k] - (i == k + 1 ? beta : 0.0);
            vn += v[i] * v[i];
        }
        if (vn == 0.0) continue;
        // reflector P = I - 2 v v^T / (v^T v) on indices k+1..n-1
        for (int c = 0; c < n; c++) {  // A = P A
            double s = 0.0;
            for (int i = k + 1; i < n; i++) s += v[i] * A[(size_t)i * n + c];
            s *= 2.0 / vn;
            for (int i = k + 1; i < n; i++) A[(size_t)i * n + c] -= s * v[i];
        }
        for (int r = 0; r < n; r++) {  // A = A P, Q = Q P
            double s = 0.0, t = 0.0;
            for (int i = k + 1; i < n; i++) {
                s += A[(size_t)r * n + i] * v[i];
                t += Q[(size_t)r * n + i] * v[i];
            }
            s *= 2.0 / vn;
            t *= 2.0 / vn;
            for (int i = k + 1; i < n; i++) {
                A[(size_t)r * n + i] -= s * v[i];
                Q[(size_t)r * n + i] -= t * v[i];
            }
        }
        for (int i = k + 2; i < n; i++) A[(size_t)i * n + k] = 0.0;
    }
}

// Rotation U = [[conj(a), conj(b)], [-b, a]] / r with U (a, b)^T = (r, 0)^T.
struct Rot {
    cplx a, b;  // already divided by r
};

Rot make_rot(cplx a, cplx b) {
    const double r = std::hypot(std::abs(a), std::abs(b));
    if (r == 0.0) return {cplx(1.0, 0.0), cplx(0.0, 0.0)};
    return {a / r, b / r};
}

// rows i, i+1 of T (columns c0..m-1) <- U rows
void rot_rows(int m, std::vector<cplx> &T, int i, int c0, Rot g) {
    for (int c = c0; c < m; c++) {
        const cplx x = T[(size_t)i * m + c], y = T[(size_t)(i + 1) * m + c];
        T[(size_t)i * m + c] = std::conj(g.a) * x + std::conj(g.b) * y;
        T[(size_t)(i + 1) * m + c] = -g.b * x + g.a * y;
    }
}

// columns i, i+1 of X (rows 0..r1) <- X U^H
void rot_cols(int m, std::vector<cplx> &X, int i, int r1, Rot g) {
    for (int r = 0; r <= r1; r++) {
        const cplx x = X[(size_t)r * m + i], y = X[(size_t)r * m + i + 1];
        X[(size_t)r * m + i] = g.a * x + g.b * y;
        X[(size_t)r * m + i + 1] = -std::conj(g.b) * x + std::conj(g.a) * y;
    }
}

// Shifted QR steps on the Hessenberg T until it is upper triangular; every
// step is a unitary similarity applied to the whole matrix (rows of the
// active window across all later columns, columns across all earlier rows)
// and accumulated into Z.
bool complex_qr(int m, std::vector<cplx> &T, std::vector<cplx> &Z) {
    double fro = 0.0;
    for (const cplx &x : T) fro += std::norm(x);
    fro = std::sqrt(fro);
    if (fro == 0.0) return true;
    std::vector<Rot> rots(m);
    int hi = m - 1, its = 0, total = 0;
    while (hi > 0) {
        int lo = hi;
        while (lo > 0) {
            double s = std::abs(T[(size_t)(lo - 1) * m + lo - 1]) + std::abs(T[(size_t)lo * m + lo]);
            if (s == 0.0) s = fro;
            if (std::abs(T[(size_t)lo * m + lo - 1]) <= kEps * s) {
                T[(size_t)lo * m + lo - 1] = 0.0;
                break;
            }
            lo--;
        }
        if (lo == hi) {
            hi--;
            its = 0;
            continue;
        }
        if (++total > 40 * m) return false;
        ++its;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer
        // its last diagonal entry; an ad hoc shift every 10 stalled steps
        const cplx a = T[(size_t)(hi - 1) * m + hi - 1], b = T[(size_t)(hi - 1) * m + hi];
        const cplx c = T[(size_t)hi * m + hi - 1], d = T[(size_t)hi * m + hi];
        cplx mu;
        if (its % 10 == 0) {
            mu = d + cplx(0.75 * std::abs(c), 0.0);
        } else {
            const cplx h = 0.5 * (a - d);
            const cplx disc = std::sqrt(h * h + b * c);
            const cplx m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
            mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        }
        // explicit step on the window: T_w - mu = Q R, T_w <- R Q + mu
        for (int i = lo; i <= hi; i++) T[(size_t)i * m + i] -= mu;
        for (int i = lo; i < hi; i++) {
            rots[i] = make_rot(T[(size_t)i * m + i], T[(size_t)(i + 1) * m + i]);
            rot_rows(m, T, i, i, rots[i]);
            T[(size_t)(i + 1) * m + i] = 0.0;
        }
        for (int i = lo; i < hi; i++) {
            rot_cols(m, T, i, i + 1, rots[i]);
            rot_cols(m, Z, i, m - 1, rots[i]);
        }
        for (int i = lo; i <= hi; i++) T[(size_t)i * m + i] += mu;
    }
    // below the diagonal only rounding remains
    for (int r = 1; r < m; r++)
        for (int c = 0; c < r; c++) T[(size_t)r * m + c] = 0.0;
    return true;
}

double sort_key(cplx w, int which) { return which == XB_EIG_LM ? std::abs(w) : w.real(); }

}  // namespace

namespace xb {

int schur(int m, const double *A, std::vector<cplx> &T, std::vector<cplx> &Z) {
    std::vector<double> H(A, A + (size_t)m * m), Q;
    hessenberg(m, H, Q);
    T.assign((size_t)m * m, cplx(0.0, 0.0));
    Z.assign((size_t)m * m, cplx(0.0, 0.0));
    for (size_t i = 0; i < H.size(); i++) {
        T[i] = H[i];
        Z[i] = Q[i];
    }
    if (!complex_qr(m, T, Z)) return set_error(XB_ENOCONV, "dense eigensolver: QR iteration stalled");
    return XB_OK;
}

void eig_order(int m, const std::vector<cplx> &T, int which, std::vector<int> &ord,
               std::vector<signed char> &kind, std::vector<cplx> &w) {
    double fro = 0.0;
    for (const cplx &x : T) fro += std::norm(x);
    // imaginary parts below this are rounding of a real eigenvalue
    const double tol_im = 1e-10 * std::max(std::sqrt(fro), 1e-300);
    std::vector<int> idx(m);
    for (int i = 0; i < m; i++) idx[i] = i;
    auto ev = [&](int i) { return T[(size_t)i * m + i]; };
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        const double kx = sort_key(ev(x), which), ky = sort_key(ev(y), which);
        if (kx != ky) return kx > ky;
        return ev(x).imag() > ev(y).imag();
    });
    ord.clear();
    kind.clear();
    w.clear();
    std::vector<char> used(m, 0);
    for (int t = 0; t < m; t++) {
        const int e = idx[t];
        if (used[e]) continue;
        used[e] = 1;
        const cplx we = ev(e);
        int p = -1;
        if (std::fabs(we.imag()) > tol_im) {
            double best = 0.0;
            for (int q = 0; q < m; q++) {
                if (used[q] || ev(q).imag() * we.imag() >= 0.0) continue;
                const double dq = std::abs(ev(q) - std::conj(we));
                if (p < 0 || dq < best) {
                    p = q;
                    best = dq;
                }
            }
        }
        if (p < 0) {
            ord.push_back(e);
            kind.push_back(0);
            w.push_back(cplx(we.real(), 0.0));
            continue;
        }
        used[p] = 1;
        const cplx wp = ev(p);
        const double re = 0.5 * (we.real() + wp.real());
        const double im = 0.5 * (std::fabs(we.imag()) + std::fabs(wp.imag()));
        const int first = we.imag() > 0.0 ? e : p, second = first == e ? p : e;
        ord.push_back(first);
        kind.push_back(1);
        w.push_back(cplx(re, im));
        ord.push_back(second);
        kind.push_back(-1);
        w.push_back(cplx(re, -im));
    }
}

void schur_reorder(int m, std::vector<cplx> &T, std::vector<cplx> &Z, const std::vector<int> &ord,
                   int k) {
    std::vector<int> at(m);  // at[pos] = original diagonal index now at pos
    for (int i = 0; i < m; i++) at[i] = i;
    for (int t = 0; t < k; t++) {
        int c = t;
        while (at[c] != ord[t]) c++;
        for (int q = c - 1; q >= t; q--) {
            // swap diagonal entries q, q+1: G's first column is the unit
            // eigenvector of the 2 x 2 block for its second eigenvalue
            const cplx t11 = T[(size_t)q * m + q], t22 = T[(size_t)(q + 1) * m + q + 1];
            const cplx t12 = T[(size_t)q * m + q + 1];
            const double r = std::hypot(std::abs(t12), std::abs(t22 - t11));
            if (r > 0.0) {
                const cplx u1 = t12 / r, u2 = (t22 - t11) / r;
                // T <- G^H T G, Z <- Z G with G = [[u1, -conj(u2)], [u2, conj(u1)]]
                for (int cc = q; cc < m; cc++) {
                    const cplx x = T[(size_t)q * m + cc], y = T[(size_t)(q + 1) * m + cc];
                    T[(size_t)q * m + cc] = std::conj(u1) * x + std::conj(u2) * y;
                    T[(size_t)(q + 1) * m + cc] = -u2 * x + u1 * y;
                }
                for (int rr = 0; rr <= q + 1; rr++) {
                    const cplx x = T[(size_t)rr * m + q], y = T[(size_t)rr * m + q + 1];
                    T[(size_t)rr * m + q] = u1 * x + u2 * y;
                    T[(size_t)rr * m + q + 1] = -std::conj(u2) * x + std::conj(u1) * y;
                }
                for (int rr = 0; rr < m; rr++) {
                    const cplx x = Z[(size_t)rr * m + q], y = Z[(size_t)rr * m + q + 1];
                    Z[(size_t)rr * m + q] = u1 * x + u2 * y;
                    Z[(size_t)rr * m + q + 1] = -std::conj(u2) * x + std::conj(u1) * y;
                }
            }
            T[(size_t)(q + 1) * m + q] = 0.0;
            T[(size_t)q * m + q] = t22;
            T[(size_t)(q + 1) * m + q + 1] = t11;
            std::swap(at[q], at[q + 1]);
        }
    }
}

void schur_eigvec(int m, const std::vector<cplx> &T, const std::vector<cplx> &Z, int i,
                  bool real_ev, std::vector<cplx> &y) {
    double fro = 0.0;
    for (const cplx &x : T) fro += std::norm(x);
    const double smin = std::max(kEps * std::sqrt(fro), 1e-290);
    std::vector<cplx> s(i + 1);
    const cplx lam = T[(size_t)i * m + i];
    s[i] = 1.0;
    for (int r = i - 1; r >= 0; r--) {
        cplx acc = 0.0;
        for (int c = r + 1; c <= i; c++) acc += T[(size_t)r * m + c] * s[c];
        cplx den = T[(size_t)r * m + r] - lam;
        if (std::abs(den) < smin) den = smin;
        s[r] = -acc / den;
        // keep the partial solution bounded (rescaling does not change the direction)
        const double big = std::abs(s[r]);
        if (big > 1e100)
            for (int c = r; c <= i; c++) s[c] /= big;
    }
    y.assign(m, cplx(0.0, 0.0));
    for (int r = 0; r < m; r++) {
        cplx acc = 0.0;
        for (int c = 0; c <= i; c++) acc += Z[(size_t)r * m + c] * s[c];
        y[r] = acc;
    }
    int big = 0;
    for (int r = 1; r < m; r++)
        if (std::abs(y[r]) > std::abs(y[big])) big = r;
    const cplx ph = std::abs(y[big]) > 0.0 ? std::conj(y[big]) / std::abs(y[big]) : cplx(1.0, 0.0);
    double nrm = 0.0;
    for (int r = 0; r < m; r++) {
        y[r] *= ph;
        if (real_ev) y[r] = cplx(y[r].real(), 0.0);
        nrm += std::norm(y[r]);
    }
    nrm = std::sqrt(nrm);
    if (nrm > 0.0)
        for (int r = 0; r < m; r++) y[r] /= nrm;
}

int keep_count(const std::vector<signed char> &kind, int k0, int m) {
    if (k0 >= 1 && k0 <= m && kind[k0 - 1] == 1) return k0 + 1 <= m - 1 ? k0 + 1 : k0 - 1;
    return k0;
}

int real_basis(int m, const std::vector<cplx> &Z, int k, std::vector<double> &Q) {
    const int nc = 2 * k;
    std::vector<double> C((size_t)nc * m);  // candidate columns, column-major
    for (int c = 0; c < k; c++)
        for (int r = 0; r < m; r++) {
            C[(size_t)c * m + r] = Z[(size_t)r * m + c].real();
            C[(size_t)(k + c) * m + r] = Z[(size_t)r * m + c].imag();
        }
    Q.assign((size_t)m * k, 0.0);
    std::vector<char> taken(nc, 0);
    int got = 0;
    while (got < k) {
        int piv = -1;
        double best = 0.0;
        for (int c = 0; c < nc; c++) {
            if (taken[c]) continue;
            double s = 0.0;
            for (int r = 0; r < m; r++) s += C[(size_t)c * m + r] * C[(size_t)c * m + r];
            if (s > best) {
                best = s;
                piv = c;
            }
        }
        if (piv < 0 || best < 1e-16) break;  // the Z columns are unit: nothing independent left
        taken[piv] = 1;
        double *q = &Q[(size_t)got * m];
        for (int r = 0; r < m; r++) q[r] = C[(size_t)piv * m + r];
        for (int pass = 0; pass < 2; pass++)  // against the basis so far, twice
            for (int j = 0; j < got; j++) {
                const double *qj = &Q[(size_t)j * m];
                double d = 0.0;
                for (int r = 0; r < m; r++) d += qj[r] * q[r];
                for (int r = 0; r < m; r++) q[r] -= d * qj[r];
            }
        double nq = 0.0;
        for (int r = 0; r < m; r++) nq += q[r] * q[r];
        nq = std::sqrt(nq);
        if (!(nq > 1e-8)) break;
        for (int r = 0; r < m; r++) q[r] /= nq;
        got++;
        for (int c = 0; c < nc; c++) {  // deflate the remaining candidates
            if (taken[c]) continue;
            double d = 0.0;
            for (int r = 0; r < m; r++) d += q[r] * C[(size_t)c * m + r];
            for (int r = 0; r < m; r++) C[(size_t)c * m + r] -= d * q[r];
        }
    }
    return got;
}

}  // namespace xb

extern "C" {

int xb_dense_restart_basis(int32_t n, const double *A, int32_t which, int32_t k, double *Q,
                           int32_t *kout) {
    if (n < 2 || n > 512 || !A || !Q || !kout || k < 1 || k >= n ||
        (which != XB_EIG_LR && which != XB_EIG_LM))
        return xb::set_error(XB_EINVAL, "dense_restart_basis: bad argument");
    std::vector<xb::cplx> T, Z, w;
    XB_TRY(xb::schur(n, A, T, Z));
    std::vector<int> ord;
    std::vector<signed char> kind;
    xb::eig_order(n, T, which, ord, kind, w);
    const int kk = xb::keep_count(kind, k, n);
    xb::schur_reorder(n, T, Z, ord, kk);
    std::vector<double> q;
    *kout = xb::real_basis(n, Z, kk, q);
    std::copy(q.begin(), q.begin() + (size_t)n * *kout, Q);
    return XB_OK;
}

int xb_dense_eig(int32_t n, const double *A, int32_t which, double *wr, double *wi, double *vr,
                 double *vi) {
    if (n < 1 || n > 512 || !A || !wr || !wi || (!vr) != (!vi) ||
        (which != XB_EIG_LR && which != XB_EIG_LM))
        return xb::set_error(XB_EINVAL, "dense_eig: bad argument");
    std::vector<xb::cplx> T, Z, w, y;
    XB_TRY(xb::schur(n, A, T, Z));
    std::vector<int> ord;
    std::vector<signed char> kind;
    xb::eig_order(n, T, which, ord, kind, w);
    if (vr) xb::schur_reorder(n, T, Z, ord, n);
    for (int t = 0; t < n; t++) {
        wr[t] = w[t].real();
        wi[t] = w[t].imag();
        if (!vr) continue;
        xb::schur_eigvec(n, T, Z, t, kind[t] == 0, y);
        for (int r = 0; r < n; r++) {
            vr[(size_t)t * n + r] = y[r].real();
            vi[(size_t)t * n + r] = y[r].imag();
        }
    }
    return XB_OK;
}

}  // extern "C"
