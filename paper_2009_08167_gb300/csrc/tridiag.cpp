// Eigenpairs of the symmetric tridiagonal Lanczos matrix T_m (Eq. LanczosTm),
// the Rayleigh-Ritz step of Eq. RitzValues.  Implicit QL iteration with
// Wilkinson-type shifts and Givens rotations (the classical method for
// symmetric tridiagonal matrices); m is a few hundred at most.
//
// alpha[0..m-1] diagonal, beta[0..m-2] off-diagonal T[i][i+1].
// theta[0..m-1] ascending.  With vectors, Z (m x m, column-major) holds the
// eigenvectors; without, Z[0..m-1] receives only the LAST ROW of the
// eigenvector matrix (what the Lanczos residual estimates need), obtained by
// applying the same rotations to e_m^T alone.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "ctx.h"

namespace riga {

namespace {
// sqrt(x^2 + y^2) for the rotations: the plain formula (the library hypot
// costs several times more and the iteration makes O(m^2) rotations), scaled
// only when the squares could leave the double range
inline double rot_norm(double x, double y) {
    const double ax = std::fabs(x), ay = std::fabs(y);
    const double mx = ax > ay ? ax : ay;
    if (mx > 1e150 || (mx < 1e-150 && mx > 0.0)) {
        const double a = ax / mx, b = ay / mx;
        return mx * std::sqrt(a * a + b * b);
    }
    return std::sqrt(x * x + y * y);
}
}  // namespace

// General form: the rotations of the iteration are applied to the columns of
// a zr x m row block z0 (column-major: entry (row, j) at z0[j * zr + row]);
// Zout receives that block times the eigenvector matrix, columns in
// ascending eigenvalue order.  z0 = I gives the eigenvectors, z0 = e_m^T
// their last row.
void tridiag_eig_rows(int m, const double* alpha, const double* beta, double* theta, int zr, const double* z0,
                      double* Zout) {
    std::vector<double> d(alpha, alpha + m), e(m, 0.0);
    for (int i = 0; i + 1 < m; ++i) e[i] = beta[i];
    std::vector<double> z(z0, z0 + (size_t)zr * m);
    auto zat = [&](int row, int colj) -> double& { return z[(size_t)colj * zr + row]; };
    const double eps = 2.220446049250313e-16;
    for (int l = 0; l < m; ++l) {
        int iter = 0;
        for (;;) {
            int mm = l;
            for (; mm < m - 1; ++mm) {
                double dd = std::fabs(d[mm]) + std::fabs(d[mm + 1]);
                if (std::fabs(e[mm]) <= eps * dd) break;
            }
            if (mm == l) break;
            if (++iter > 200) break;
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = rot_norm(g, 1.0);
            g = d[mm] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            int i;
            bool early = false;
            for (i = mm - 1; i >= l; --i) {
                double f = s * e[i], b = c * e[i];
                r = rot_norm(f, g);
                e[i + 1] = r;
                if (r == 0.0) {
                    d[i + 1] -= p;
                    e[mm] = 0.0;
                    early = true;
                    break;
                }
                const double ir = 1.0 / r;
                s = f * ir;
                c = g * ir;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                for (int k = 0; k < zr; ++k) {
                    double& a0 = zat(k, i);
                    double& a1 = zat(k, i + 1);
                    double t1 = a1;
                    a1 = s * a0 + c * t1;
                    a0 = c * a0 - s * t1;
                }
            }
            if (early) continue;
            d[l] -= p;
            e[l] = g;
            e[mm] = 0.0;
        }
    }
    std::vector<int> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d[a] < d[b]; });
    for (int i = 0; i < m; ++i) theta[i] = d[order[i]];
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < zr; ++k) Zout[(size_t)i * zr + k] = z[(size_t)order[i] * zr + k];
}

void tridiag_eig(int m, const double* alpha, const double* beta, double* theta, double* Z, bool vectors) {
    const int zr = vectors ? m : 1;
    std::vector<double> z0((size_t)zr * m, 0.0);
    if (vectors)
        for (int i = 0; i < m; ++i) z0[(size_t)i * m + i] = 1.0;
    else if (m > 0)
        z0[m - 1] = 1.0;
    tridiag_eig_rows(m, alpha, beta, theta, zr, z0.data(), Z);
}

}  // namespace riga
