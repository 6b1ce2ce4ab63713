// Device B-spline helpers shared by the assembly and the accuracy kernels:
// Gauss-Legendre rules (Newton iteration on the Legendre polynomial) and the
// Cox-de Boor recursion of Eq. N over one knot span (Sec. 3.1).
#pragma once

namespace riga {

constexpr int PMAX = 6;

__device__ inline void gauss_legendre_dev(int nq, double* t, double* w) {
    // Newton iteration on P_nq (three-term recurrence), initial guesses
    // cos(pi (i + 3/4) / (nq + 1/2)).
    for (int i = 0; i < nq; ++i) {
        double x = cos(M_PI * (i + 0.75) / (nq + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 1; j < nq; ++j) {
                double p2 = ((2 * j + 1) * x * p1 - j * p0) / (j + 1);
                p0 = p1;
                p1 = p2;
            }
            double pn = (nq == 1) ? x : p1;
            double pm = (nq == 1) ? 1.0 : p0;
            dp = nq * (x * pn - pm) / (x * x - 1.0);
            double dx = pn / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int j = 1; j < nq; ++j) {
            double p2 = ((2 * j + 1) * x * p1 - j * p0) / (j + 1);
            p0 = p1;
            p1 = p2;
        }
        dp = nq * (x * p1 - p0) / (x * x - 1.0);
        // ascending order: the guesses are descending in i
        t[nq - 1 - i] = x;
        w[nq - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

// Values and derivatives of B_{sp-p+t,p}(x), t = 0..p, by the recursion of
// Eq. N over degrees 0..p (0/0 := 0).
__device__ inline void basis_span(const int* kv, double inv_ne, int p, int sp, double x, double* N, double* dN) {
    double v[PMAX + 1][PMAX + 1];
    v[0][0] = 1.0;
    for (int d = 1; d <= p; ++d) {
        for (int t = 0; t <= d; ++t) {
            int i = sp - d + t;
            double r = 0.0;
            if (t >= 1) {
                double xi = kv[i] * inv_ne, xid = kv[i + d] * inv_ne;
                double den = xid - xi;
                if (den > 0.0) r += (x - xi) / den * v[d - 1][t - 1];
            }
            if (t <= d - 1) {
                double xi1 = kv[i + 1] * inv_ne, xid1 = kv[i + d + 1] * inv_ne;
                double den = xid1 - xi1;
                if (den > 0.0) r += (xid1 - x) / den * v[d - 1][t];
            }
            v[d][t] = r;
        }
    }
    for (int t = 0; t <= p; ++t) {
        N[t] = v[p][t];
        int i = sp - p + t;
        double dv = 0.0;
        if (t >= 1) {
            double den = (kv[i + p] - kv[i]) * inv_ne;
            if (den > 0.0) dv += p / den * v[p - 1][t - 1];
        }
        if (t <= p - 1) {
            double den = (kv[i + p + 1] - kv[i + 1]) * inv_ne;
            if (den > 0.0) dv -= p / den * v[p - 1][t];
        }
        dN[t] = dv;
    }
}

}  // namespace riga
