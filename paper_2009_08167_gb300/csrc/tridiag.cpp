// Eigenpairs of the symmetric tridiagonal Lanczos matrix T_m (Eq. LanczosTm),
// the Rayleigh-Ritz step of Eq. RitzValues; m is a few hundred at most.
//
// Method: the implicitly shifted symmetric QR iteration as Golub and Van Loan
// describe it (Matrix Computations, 4th ed., Sec. 8.3: Wilkinson shift from
// the trailing 2 x 2 block, then one Givens rotation per row that chases the
// bulge it creates down the band), with deflation from the bottom: the
// iteration always works on the lowest unreduced diagonal block [lo, hi],
// and an off-diagonal entry counts as zero once it is below
// eps (|t_ii| + |t_i+1,i+1|).
//
// One step on [lo, hi] with shift mu.  A rotation R_j in the plane (j, j+1),
// rows  r_j' = c r_j + s r_j+1,  r_j+1' = -s r_j + c r_j+1  (and the same
// for the columns), replaces T by R_j T R_j^T.  For j = lo it is chosen by
// (t_lo,lo - mu, t_lo+1,lo); for j > lo it annihilates the bulge b at
// (j+1, j-1) against t_j,j-1.  On the 2 x 2 block (a, e; e, g) of rows j, j+1
// it gives
//     a' = c^2 a + 2cs e + s^2 g,   g' = s^2 a - 2cs e + c^2 g,
//     e' = cs (g - a) + (c^2 - s^2) e,
// and it moves the bulge to (j+2, j): b' = s t_j+2,j+1, t_j+2,j+1' = c t_j+2,j+1.
// T = Q Lambda Q^T accumulates as Z <- Z R_j^T: columns j, j+1 of Z become
// (c z_j + s z_j+1, -s z_j + c z_j+1).
//
// alpha[0..m-1] diagonal, beta[0..m-2] off-diagonal T[i][i+1].
// theta[0..m-1] ascending.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "ctx.h"

namespace riga {

namespace {

// c, s with c x + s y = r >= 0 and -s x + c y = 0 (a plane rotation that
// takes (x, y) to (r, 0)).  When the larger magnitude lies in
// [2^-500, 2^500] the squares cannot overflow and the larger one stays
// normal: one square root and one division; otherwise both are scaled by
// the larger magnitude first.  (The rotations of the bulge chase form a
// dependent chain, so their latency is the iteration's cost.)
inline void plane_rotation(double x, double y, double& c, double& s, double& r) {
    const double ax = std::fabs(x), ay = std::fabs(y);
    if (ay == 0.0) {
        c = x >= 0.0 ? 1.0 : -1.0;
        s = 0.0;
        r = ax;
        return;
    }
    if (ax == 0.0) {
        c = 0.0;
        s = y > 0.0 ? 1.0 : -1.0;
        r = ay;
        return;
    }
    const double big = ax > ay ? ax : ay;
    if (big >= 0x1p-500 && big <= 0x1p500) {
        r = std::sqrt(x * x + y * y);
        const double inv = 1.0 / r;
        c = x * inv;
        s = y * inv;
        return;
    }
    const double xs = x / big, ys = y / big;
    const double h = std::sqrt(xs * xs + ys * ys);
    r = big * h;
    c = xs / h;
    s = ys / h;
}

// Wilkinson shift of the trailing block (a, b; b, g): the eigenvalue of the
// block closer to g.  |den| >= |b|, so b (b / den) cannot overflow; the
// root is formed by the same scaled norm as the rotations.
inline double wilkinson_shift(double a, double b, double g) {
    const double delta = 0.5 * (a - g);
    if (b == 0.0) return g;
    double c, s, root;
    plane_rotation(delta, b, c, s, root);
    const double den = delta >= 0.0 ? delta + root : delta - root;
    return g - b * (b / den);
}

struct TridiagQR {
    std::vector<double> diag, off;  // off[i] couples rows i and i+1
    int zr;                         // rows of the accumulated block
    std::vector<double> z;          // zr x m, column-major

    void rotate_columns(int j, double c, double s) {
        double* zj = &z[(size_t)j * zr];
        double* zk = zj + zr;
        for (int row = 0; row < zr; ++row) {
            const double u = zj[row], v = zk[row];
            zj[row] = c * u + s * v;
            zk[row] = -s * u + c * v;
        }
    }

    // one implicit shifted QR step on rows lo..hi (hi > lo, unreduced)
    void qr_step(int lo, int hi) {
        const double mu = wilkinson_shift(diag[hi - 1], off[hi - 1], diag[hi]);
        double x = diag[lo] - mu, y = off[lo];
        double bulge = 0.0;
        for (int j = lo; j < hi; ++j) {
            double c, s, r;
            if (j == lo) {
                plane_rotation(x, y, c, s, r);
            } else {
                plane_rotation(off[j - 1], bulge, c, s, r);
                off[j - 1] = r;
            }
            const double a = diag[j], e = off[j], g = diag[j + 1];
            const double cc = c * c, ss = s * s, cs = c * s;
            diag[j] = cc * a + 2.0 * cs * e + ss * g;
            diag[j + 1] = ss * a - 2.0 * cs * e + cc * g;
            off[j] = cs * (g - a) + (cc - ss) * e;
            if (j + 1 < hi) {
                bulge = s * off[j + 1];
                off[j + 1] *= c;
            }
            rotate_columns(j, c, s);
        }
    }

    void run() {
        const int m = (int)diag.size();
        const double eps = 2.220446049250313e-16;
        const long long budget = 60LL * std::max(m, 1);  // QR steps in all (about 2 per eigenvalue)
        long long steps = 0;
        int hi = m - 1;
        while (hi > 0) {
            // deflate negligible couplings at the bottom
            if (std::fabs(off[hi - 1]) <= eps * (std::fabs(diag[hi - 1]) + std::fabs(diag[hi]))) {
                off[hi - 1] = 0.0;
                --hi;
                continue;
            }
            // top of the unreduced block that ends at hi
            int lo = hi - 1;
            while (lo > 0) {
                if (std::fabs(off[lo - 1]) <= eps * (std::fabs(diag[lo - 1]) + std::fabs(diag[lo]))) {
                    off[lo - 1] = 0.0;
                    break;
                }
                --lo;
            }
            if (++steps > budget) break;  // leave the remaining block as it stands
            qr_step(lo, hi);
        }
    }
};

}  // namespace

// General form: the rotations of the iteration are applied to the columns of
// a zr x m row block z0 (column-major: entry (row, j) at z0[j * zr + row]);
// Zout receives that block times the eigenvector matrix, columns in
// ascending eigenvalue order.  z0 = I gives the eigenvectors, z0 = e_m^T
// their last row.
void tridiag_eig_rows(int m, const double* alpha, const double* beta, double* theta, int zr, const double* z0,
                      double* Zout) {
    if (m <= 0) return;
    TridiagQR q;
    q.diag.assign(alpha, alpha + m);
    q.off.assign(m, 0.0);
    for (int i = 0; i + 1 < m; ++i) q.off[i] = beta[i];
    q.zr = zr;
    q.z.assign(z0, z0 + (size_t)zr * m);
    q.run();
    std::vector<int> order(m);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return q.diag[a] < q.diag[b]; });
    for (int i = 0; i < m; ++i) {
        theta[i] = q.diag[order[i]];
        const double* src = &q.z[(size_t)order[i] * zr];
        std::copy(src, src + zr, Zout + (size_t)i * zr);
    }
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
