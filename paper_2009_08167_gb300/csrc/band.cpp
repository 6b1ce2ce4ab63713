// Rayleigh-Ritz step of block Lanczos: eigenpairs of the symmetric band
// matrix T_m (the block-tridiagonal projection of the shift-inverted operator,
// the block form of Eq. LanczosTm and Eq. RitzValues; half-bandwidth = the
// block size b).
//
// Eigenvalues: the band is reduced to tridiagonal form by Givens similarity
// rotations, chasing the bulge each rotation creates down the band (the
// classical Rutishauser-Schwarz band reduction, O(n^2 b)); the tridiagonal
// eigenvalues come from the implicit QL iteration of tridiag.cpp.
// Eigenvectors (only those asked for): inverse iteration on T - theta I with a
// banded LU factorization with partial pivoting, the iterates of eigenvalues
// closer than 1e-3 ||T|| orthogonalised against each other (modified
// Gram-Schmidt), three iterations from a fixed start vector.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <thread>
#include <vector>

#include "ctx.h"

namespace riga {

namespace {

// The reduction keeps the lower triangle in band storage: column j holds
// A(j + d, j) for d = 0 .. W-1 at L[j * W + d].  W = b + 4 covers the band,
// the bulge (distance b + 1) and every entry the window of a rotation reads
// (distance up to b + 3); entries beyond are zero throughout.
struct BandSym {
    int n, w;
    std::vector<double> L;
};

// similarity rotation in the adjacent plane (p, q = p + 1) of the symmetric
// matrix: rows p, q <- [c s; -s c] [row p; row q], and the same on the
// columns, restricted to the index window where the band (plus one bulge) can
// hold non-zeros.  Left of p the two entries of a column t are neighbours in
// its storage (t, p - t) and (t, q - t); right of q they sit in columns p and
// q at distances t - p and t - q.
void rotate_adj(BandSym& A, int b, int p, double c, double s) {
    const int q = p + 1, w = A.w;
    double* L = A.L.data();
    const int lo = std::max(0, p - b - 2), hi = std::min(A.n, q + b + 3);
    for (int t = lo; t < p; ++t) {
        double* col = L + (size_t)t * w;
        const double x = col[p - t], y = col[q - t];
        col[p - t] = c * x + s * y;
        col[q - t] = -s * x + c * y;
    }
    double* cp = L + (size_t)p * w;
    double* cq = L + (size_t)q * w;
    for (int t = q + 1; t < hi; ++t) {
        const double x = cp[t - p], y = cq[t - q];
        cp[t - p] = c * x + s * y;
        cq[t - q] = -s * x + c * y;
    }
    const double app = cp[0], aqq = cq[0], apq = cp[1];
    const double npp = c * c * app + 2.0 * c * s * apq + s * s * aqq;
    const double nqq = s * s * app - 2.0 * c * s * apq + c * c * aqq;
    const double npq = (c * c - s * s) * apq + c * s * (aqq - app);
    cp[0] = npp;
    cq[0] = nqq;
    cp[1] = npq;
}

// band LU with partial pivoting (kl = ku = b; fill up to 2b above the
// diagonal), LAPACK band layout: A(i, j) at ab[kv + i - j + j * ldab]
struct BandLU {
    int n, kl, ku, kv, ldab;
    std::vector<double> ab;
    std::vector<int> piv;
};

void band_lu(BandLU& F, int n, int b, const double* T, double shift, double tiny) {
    F.n = n;
    F.kl = b;
    F.ku = b;
    F.kv = 2 * b;
    F.ldab = 3 * b + 1;
    F.ab.assign((size_t)F.ldab * n, 0.0);
    F.piv.assign(n, 0);
    auto AB = [&](int i, int j) -> double& { return F.ab[(size_t)F.kv + i - j + (size_t)j * F.ldab]; };
    for (int j = 0; j < n; ++j)
        for (int i = std::max(0, j - b); i <= std::min(n - 1, j + b); ++i)
            AB(i, j) = T[(size_t)j * n + i] - (i == j ? shift : 0.0);
    int ju = 0;
    for (int j = 0; j < n; ++j) {
        const int km = std::min(F.kl, n - 1 - j);
        int jp = 0;
        double best = std::fabs(AB(j, j));
        for (int i = 1; i <= km; ++i)
            if (std::fabs(AB(j + i, j)) > best) {
                best = std::fabs(AB(j + i, j));
                jp = i;
            }
        F.piv[j] = j + jp;
        ju = std::max(ju, std::min(j + F.ku + jp, n - 1));
        if (jp != 0)
            for (int cc = j; cc <= ju; ++cc) std::swap(AB(j, cc), AB(j + jp, cc));
        if (std::fabs(AB(j, j)) < tiny) AB(j, j) = AB(j, j) < 0.0 ? -tiny : tiny;
        const double inv = 1.0 / AB(j, j);
        for (int i = 1; i <= km; ++i) AB(j + i, j) *= inv;
        for (int cc = j + 1; cc <= ju; ++cc) {
            const double u = AB(j, cc);
            if (u == 0.0) continue;
            for (int i = 1; i <= km; ++i) AB(j + i, cc) -= AB(j + i, j) * u;
        }
    }
}

// dot product with four independent partial sums (a fixed order; the
// sequential form is one dependent add chain, which the compiler may not
// reorder without fast-math)
inline double dot4(const double* a, const double* b, int n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 3 < n; i += 4) {
        s0 += a[i] * b[i];
        s1 += a[i + 1] * b[i + 1];
        s2 += a[i + 2] * b[i + 2];
        s3 += a[i + 3] * b[i + 3];
    }
    for (; i < n; ++i) s0 += a[i] * b[i];
    return (s0 + s1) + (s2 + s3);
}

void band_solve(const BandLU& F, double* x) {
    const int n = F.n;
    auto AB = [&](int i, int j) -> double { return F.ab[(size_t)F.kv + i - j + (size_t)j * F.ldab]; };
    for (int j = 0; j < n; ++j) {
        if (F.piv[j] != j) std::swap(x[j], x[F.piv[j]]);
        const int km = std::min(F.kl, n - 1 - j);
        for (int i = 1; i <= km; ++i) x[j + i] -= AB(j + i, j) * x[j];
    }
    for (int j = n - 1; j >= 0; --j) {
        x[j] /= AB(j, j);
        for (int i = std::max(0, j - F.kv); i < j; ++i) x[i] -= AB(i, j) * x[j];
    }
}

}  // namespace

// sqrt(x^2 + y^2) without overflow: one square root when the larger
// magnitude lies in [2^-500, 2^500], else std::hypot
static inline double norm2(double x, double y) {
    const double big = std::fmax(std::fabs(x), std::fabs(y));
    if (big >= 0x1p-500 && big <= 0x1p500) return std::sqrt(x * x + y * y);
    return std::hypot(x, y);
}

// Band -> tridiagonal reduction; the rotations are also applied (as Q <- Q G^T)
// to the r x n row block qr (column-major), which starts as the last r rows of
// the identity, so that it ends as the last r rows of Q (T = Q T_tri Q^T).
static void band_reduce(int n, int b, const double* T, std::vector<double>& d, std::vector<double>& e, int r,
                        std::vector<double>& qr) {
    BandSym A;
    A.n = n;
    A.w = b + 4;
    A.L.assign((size_t)n * A.w, 0.0);
    const int w = A.w;
    double* L = A.L.data();
    for (int j = 0; j < n; ++j)
        for (int i = j; i <= std::min(n - 1, j + b); ++i) L[(size_t)j * w + (i - j)] = T[(size_t)j * n + i];
    // entry (i, j), i >= j, of the lower band
    auto low = [&](int i, int j) -> double& { return L[(size_t)j * w + (i - j)]; };
    auto track = [&](int p, int q, double c, double s) {
        for (int k = 0; k < r; ++k) {
            double& a = qr[(size_t)p * r + k];
            double& bq = qr[(size_t)q * r + k];
            const double x = a, y = bq;
            a = c * x + s * y;
            bq = -s * x + c * y;
        }
    };
    for (int j = 0; j + 2 < n; ++j) {
        for (int i = std::min(j + b, n - 1); i >= j + 2; --i) {
            const double x = low(i - 1, j), y = low(i, j);
            if (y == 0.0) continue;
            const double rr = norm2(x, y);
            const double c1 = x / rr, s1 = y / rr;
            rotate_adj(A, b, i - 1, c1, s1);
            if (r > 0) track(i - 1, i, c1, s1);
            low(i, j) = 0.0;
            // chase the bulge at (k + b, k - 1) down the band
            for (int k = i; k + b < n;) {
                const int p = k + b - 1, q = k + b, col = k - 1;
                const double x2 = low(p, col), y2 = low(q, col);
                if (y2 == 0.0) break;
                const double r2 = norm2(x2, y2);
                const double c2 = x2 / r2, s2 = y2 / r2;
                rotate_adj(A, b, p, c2, s2);
                if (r > 0) track(p, q, c2, s2);
                low(q, col) = 0.0;
                k = q;
            }
        }
    }
    d.assign(n, 0.0);
    e.assign(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = low(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = low(i + 1, i);
}

void band_eigvals(int n, int b, const double* T, double* theta) {
    if (n <= 0) return;
    std::vector<double> d, e, qr, z(n);
    band_reduce(n, b, T, d, e, 0, qr);
    tridiag_eig(n, d.data(), e.data(), theta, z.data(), false);
}

void band_eig_lastrows(int n, int b, const double* T, int r, double* theta, double* Zlast) {
    if (n <= 0) return;
    r = std::min(r, n);
    std::vector<double> d, e, qr((size_t)r * n, 0.0);
    for (int k = 0; k < r; ++k) qr[(size_t)(n - r + k) * r + k] = 1.0;  // last r rows of I
    band_reduce(n, b, T, d, e, r, qr);
    tridiag_eig_rows(n, d.data(), e.data(), theta, r, qr.data(), Zlast);
}

void band_eigvecs(int n, int b, const double* T, int q, const double* th, double* S) {
    double tnorm = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i) tnorm = std::max(tnorm, std::fabs(T[i]));
    tnorm = std::max(tnorm, 1e-300);
    const double tiny = 2.220446049250313e-16 * tnorm;
    // process in ascending eigenvalue order so that clusters are contiguous
    std::vector<int> ord(q);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return th[x] < th[y]; });
    // clusters: runs of ord whose neighbouring values are within 1e-3 ||T||
    std::vector<int> cstart;
    for (int oi = 0; oi < q; ++oi)
        if (oi == 0 || th[ord[oi]] - th[ord[oi - 1]] > 1e-3 * tnorm) cstart.push_back(oi);
    const int ncl = (int)cstart.size();
    cstart.push_back(q);
    // clusters [c0, c1): each member by inverse iteration from its own fixed
    // start vector, orthogonalised against the cluster's earlier members
    auto work = [&](int c0, int c1) {
        BandLU F;
        std::vector<double> x(n);
        for (int ci = c0; ci < c1; ++ci) {
            const int cl0 = cstart[ci];
            for (int oi = cl0; oi < cstart[ci + 1]; ++oi) {
                const int qi = ord[oi];
                band_lu(F, n, b, T, th[qi], tiny);
                // fixed start vector (deterministic), then three inverse iterations
                uint64_t s = 0x9E3779B97F4A7C15ULL ^ (uint64_t)(oi + 1);
                for (int i = 0; i < n; ++i) {
                    s ^= s << 13;
                    s ^= s >> 7;
                    s ^= s << 17;
                    x[i] = ((double)(s >> 11) / 9007199254740992.0) - 0.5;
                }
                for (int it = 0; it < 3; ++it) {
                    band_solve(F, x.data());
                    for (int pj = cl0; pj < oi; ++pj) {
                        const double* v = S + (size_t)ord[pj] * n;
                        const double dot = dot4(v, x.data(), n);
                        for (int i = 0; i < n; ++i) x[i] -= dot * v[i];
                    }
                    double nrm = std::sqrt(dot4(x.data(), x.data(), n));
                    if (!(nrm > 0.0)) nrm = 1.0;
                    const double inv = 1.0 / nrm;
                    for (int i = 0; i < n; ++i) x[i] *= inv;
                }
                std::copy(x.begin(), x.end(), S + (size_t)qi * n);
            }
        }
    };
    // clusters are independent: split them over host threads in contiguous
    // runs of about equal member counts (each cluster's arithmetic is the
    // same whichever thread runs it)
    // (about 25 us per member at n = 200; starting a thread costs about
    // 100 us, so four threads at most: 1.5 -> 0.9 ms for 60 members)
    int nth = std::min({ncl, 4, n >= 64 ? q / 8 : 1});
    nth = std::min(nth, (int)std::max(1u, std::thread::hardware_concurrency()));
    if (nth <= 1) {
        work(0, ncl);
        return;
    }
    std::vector<std::thread> pool;
    int c0 = 0;
    for (int t = 0; t < nth && c0 < ncl; ++t) {
        const int target = (int)((long long)q * (t + 1) / nth);  // members covered after this thread
        int c1 = c0 + 1;
        while (c1 < ncl && cstart[c1] < target) ++c1;
        if (t == nth - 1) c1 = ncl;
        try {
            pool.emplace_back(work, c0, c1);
        } catch (...) {  // no thread to be had: this one does the run (no exception leaves the library)
            work(c0, c1);
        }
        c0 = c1;
    }
    for (auto& th2 : pool) th2.join();
}

// All eigenpairs of a dense symmetric n x n matrix A (column-major; the
// Rayleigh-Ritz step of thick-restart Lanczos, whose projected matrix is an
// arrowhead block followed by a tridiagonal one).  Householder reduction to
// tridiagonal form: for column k the reflector P = I - 2 v v^T (|v| = 1) maps
// x = A[k+1:, k] to alpha e_1 with alpha = -sign(x_0) |x|, and
// P A P = A - v q^T - q v^T with w = A v, q = 2 w - 2 (v^T w) v on the
// trailing block; Q = P_0 P_1 ... accumulates the reflectors, and the
// tridiagonal eigenvectors are rotated into Q Z by the QR iteration of
// tridiag.cpp.  theta ascending; Z (n x n, column-major) the eigenvectors.
void sym_eig_dense(int n, const double* A0, double* theta, double* Z) {
    if (n <= 0) return;
    std::vector<double> A(A0, A0 + (size_t)n * n), Q((size_t)n * n, 0.0), v(n), w(n), q(n);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)j * n + i]; };
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;  // length of x = A[k+1:, k]
        double xn = 0.0, big = 0.0;
        for (int i = 0; i < m; ++i) big = std::max(big, std::fabs(a(k + 1 + i, k)));
        if (big == 0.0) continue;
        for (int i = 0; i < m; ++i) {
            const double t = a(k + 1 + i, k) / big;
            xn += t * t;
        }
        xn = big * std::sqrt(xn);
        const double x0 = a(k + 1, k);
        const double alpha = x0 >= 0.0 ? -xn : xn;
        for (int i = 0; i < m; ++i) v[i] = a(k + 1 + i, k);
        v[0] -= alpha;
        double vn = 0.0;
        for (int i = 0; i < m; ++i) vn += v[i] * v[i];
        vn = std::sqrt(vn);
        if (!(vn > 0.0)) continue;
        for (int i = 0; i < m; ++i) v[i] /= vn;
        // w = A22 v, gamma = v^T w, q = 2 w - 2 gamma v
        double gamma = 0.0;
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += a(k + 1 + i, k + 1 + j) * v[j];
            w[i] = s;
        }
        for (int i = 0; i < m; ++i) gamma += v[i] * w[i];
        for (int i = 0; i < m; ++i) q[i] = 2.0 * w[i] - 2.0 * gamma * v[i];
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) a(k + 1 + i, k + 1 + j) -= v[i] * q[j] + q[i] * v[j];
        a(k + 1, k) = alpha;
        a(k, k + 1) = alpha;
        for (int i = 1; i < m; ++i) {
            a(k + 1 + i, k) = 0.0;
            a(k, k + 1 + i) = 0.0;
        }
        // Q[:, k+1:] <- Q[:, k+1:] (I - 2 v v^T)
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += Q[(size_t)(k + 1 + j) * n + r] * v[j];
            s *= 2.0;
            for (int j = 0; j < m; ++j) Q[(size_t)(k + 1 + j) * n + r] -= s * v[j];
        }
    }
    std::vector<double> d(n), e(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = a(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
    tridiag_eig_rows(n, d.data(), e.data(), theta, n, Q.data(), Z);
}

}  // namespace riga

using namespace riga;

extern "C" int riga_sym_eig(int n, const double* A, double* theta, double* Z) {
    if (n < 1 || !A || !theta || !Z) return RIGA_EINVAL;
    sym_eig_dense(n, A, theta, Z);
    return RIGA_OK;
}

extern "C" int riga_band_eig(int n, int b, const double* T, double* theta, int q, const int* which, double* S, int r,
                             double* Zlast) {
    if (n < 1 || b < 0 || !T || !theta || q < 0 || (q > 0 && (!which || !S)) || r < 0 || r > n || (r > 0 && !Zlast))
        return RIGA_EINVAL;
    for (int i = 0; i < q; ++i)
        if (which[i] < 0 || which[i] >= n) return RIGA_EINVAL;
    if (r > 0) band_eig_lastrows(n, std::max(b, 1), T, r, theta, Zlast);
    else band_eigvals(n, std::max(b, 1), T, theta);
    if (q > 0) {
        std::vector<double> th(q);
        for (int i = 0; i < q; ++i) th[i] = theta[which[i]];
        band_eigvecs(n, std::max(b, 1), T, q, th.data(), S);
    }
    return RIGA_OK;
}
