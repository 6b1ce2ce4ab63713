// Eigenvalue adjoint (not in the paper): for K = sum_e cK_e K_e,
// M = sum_e cM_e M_e and M-normalised eigenvectors u_i of simple eigenvalues,
//   dL/da_e =  sum_i w_i cK_e u_ie^T K_e u_ie,
//   dL/db_e = -sum_i w_i lambda_i cM_e u_ie^T M_e u_ie,
// with a_e = log cK_e, b_e = log cM_e and K_e, M_e the unit-coefficient
// element matrices: tensor products of the 1D element matrices of
// Eq. 1Dmatrix (Eq. 2Dmatrix element by element).  One thread per element.
#include "ctx.h"

namespace riga {

constexpr int QDMAX = 64;  // (p+1)^dim limit

struct AdjDir {
    const int* ef;
    const double* Ke;
    const double* Me;
    int ne, ndof;
};

__global__ void adjoint_kernel(int dim, int p, long long n_elem, AdjDir X, AdjDir Y, AdjDir Z, int nx, int ny,
                               const int* __restrict__ ipos, int nev, const double* __restrict__ U, long long ldu,
                               const double* __restrict__ lam, const double* __restrict__ w,
                               const double* __restrict__ cK, const double* __restrict__ cM,
                               double* __restrict__ ga, double* __restrict__ gb) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    const int q = p + 1, qq = q * q;
    int ex = (int)(e % X.ne);
    long long rem = e / X.ne;
    int ey = dim > 1 ? (int)(rem % Y.ne) : 0;
    int ez = dim > 2 ? (int)(rem / Y.ne) : 0;
    const int nloc = dim == 1 ? q : (dim == 2 ? q * q : q * q * q);
    int posl[QDMAX];
    for (int I = 0; I < nloc; ++I) {
        int a = I % q, b = (I / q) % q, cidx = I / (q * q);
        int gx = X.ef[ex] + a - 1;
        int gy = dim > 1 ? Y.ef[ey] + b - 1 : 0;
        int gz = dim > 2 ? Z.ef[ez] + cidx - 1 : 0;
        bool ok = gx >= 0 && gx < X.ndof && (dim < 2 || (gy >= 0 && gy < Y.ndof)) && (dim < 3 || (gz >= 0 && gz < Z.ndof));
        posl[I] = ok ? ipos[gx + nx * (gy + ny * gz)] : -1;
    }
    const double* kx = X.Ke + (size_t)ex * qq;
    const double* mx = X.Me + (size_t)ex * qq;
    const double* ky = dim > 1 ? Y.Ke + (size_t)ey * qq : nullptr;
    const double* my = dim > 1 ? Y.Me + (size_t)ey * qq : nullptr;
    const double* kz = dim > 2 ? Z.Ke + (size_t)ez * qq : nullptr;
    const double* mz = dim > 2 ? Z.Me + (size_t)ez * qq : nullptr;
    double sa = 0.0, sb = 0.0;
    for (int i = 0; i < nev; ++i) {
        double ue[QDMAX];
        for (int I = 0; I < nloc; ++I) ue[I] = posl[I] >= 0 ? U[(long long)i * ldu + posl[I]] : 0.0;
        double qk = 0.0, qm = 0.0;
        for (int I = 0; I < nloc; ++I) {
            if (ue[I] == 0.0) continue;
            int a = I % q, b = (I / q) % q, cc = I / (q * q);
            for (int J = 0; J < nloc; ++J) {
                int a2 = J % q, b2 = (J / q) % q, c2 = J / (q * q);
                double Kx = kx[a * q + a2], Mx = mx[a * q + a2];
                double kl, ml;
                if (dim == 1) {
                    kl = Kx;
                    ml = Mx;
                } else if (dim == 2) {
                    double Ky = ky[b * q + b2], My = my[b * q + b2];
                    kl = My * Kx + Ky * Mx;
                    ml = My * Mx;
                } else {
                    double Ky = ky[b * q + b2], My = my[b * q + b2];
                    double Kz = kz[cc * q + c2], Mz = mz[cc * q + c2];
                    kl = Mz * My * Kx + Mz * Ky * Mx + Kz * My * Mx;
                    ml = Mz * My * Mx;
                }
                double uu = ue[I] * ue[J];
                qk += uu * kl;
                qm += uu * ml;
            }
        }
        sa += w[i] * qk;
        sb += w[i] * lam[i] * qm;
    }
    if (ga) ga[e] = (cK ? cK[e] : 1.0) * sa;
    if (gb) gb[e] = -(cM ? cM[e] : 1.0) * sb;
}

int eig_grad_device(riga_ctx* c, int k, const double* w_dev, double* ga_dev, double* gb_dev) {
    Symbolic& S = c->S;
    int q = S.p + 1, nloc = 1;
    for (int a = 0; a < S.dim; ++a) nloc *= q;
    if (nloc > QDMAX) return set_error(c, RIGA_EINVAL, "(p+1)^dim too large for the adjoint kernel");
    AdjDir d[3];
    for (int a = 0; a < 3; ++a) {
        d[a] = AdjDir{nullptr, nullptr, nullptr, 1, 1};
        if (a < S.dim) d[a] = AdjDir{c->elem_first[a].ptr, c->Ke1[a].ptr, c->Me1[a].ptr, S.dir[a].ne, S.dir[a].ndof};
    }
    DevBuf<double> lam;
    std::vector<double> l(c->evals.begin(), c->evals.begin() + k);
    RIGA_CUDA_TRY(c, lam.upload(l, c->stream));
    { count_launch(c); adjoint_kernel<<<(unsigned)((S.n_elem + 127) / 128), 128, 0, c->stream>>>(
        S.dim, S.p, S.n_elem, d[0], d[1], d[2], S.n1[0], S.n1[1], c->ipos.ptr, k, c->evec_perm.ptr, S.N, lam.ptr,
        w_dev, c->coefK.empty() ? nullptr : c->dcoefK.ptr, c->coefM.empty() ? nullptr : c->dcoefM.ptr, ga_dev, gb_dev); }
    RIGA_CUDA_TRY(c, cudaGetLastError());
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RIGA_OK;
}

}  // namespace riga
