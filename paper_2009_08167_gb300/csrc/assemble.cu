// Device assembly of K and M (Sec. 3.1: Eq. U, Eq. N, Eq. 1Dmatrix, Eq. 2Dmatrix).
//
// 1. elem1d_kernel: per direction and element, the p+1 non-zero B-splines and
//    their derivatives at p+1 Gauss-Legendre points (Cox-de Boor recursion of
//    Eq. N restricted to the element's span), then the (p+1)^2 element
//    stiffness and mass matrices.
// 2. band1d_kernel: global banded 1D matrices K^x, M^x, each entry summed over
//    the shared elements in ascending order (deterministic, no atomics).
// 3. csr_kron_kernel / csr_coef_kernel: CSR values in elimination order, one
//    warp per row.  Constant coefficients use the Kronecker formulas of
//    Eq. 2Dmatrix on the banded 1D matrices; per-element coefficients sum
//    c_e times the tensor-product element matrices over the shared elements.
#include "ctx.h"

namespace riga {

constexpr int PMAX = 6;

__device__ void gauss_legendre_dev(int nq, double* t, double* w) {
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
__device__ void basis_span(const int* kv, double inv_ne, int p, int sp, double x, double* N, double* dN) {
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

__global__ void elem1d_kernel(int ne, int p, const int* __restrict__ kv, const int* __restrict__ elem_first,
                              double* __restrict__ Ke, double* __restrict__ Me) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int nq = p + 1, q = p + 1;
    double t[PMAX + 1], w[PMAX + 1];
    gauss_legendre_dev(nq, t, w);
    const double inv_ne = 1.0 / ne, h = 1.0 / ne;
    const int sp = elem_first[e] + p;
    double k[(PMAX + 1) * (PMAX + 1)], m[(PMAX + 1) * (PMAX + 1)];
    for (int a = 0; a < q * q; ++a) k[a] = m[a] = 0.0;
    for (int g = 0; g < nq; ++g) {
        double x = (e + (t[g] + 1.0) / 2.0) * h;
        double wq = w[g] * h / 2.0;
        double N[PMAX + 1], dN[PMAX + 1];
        basis_span(kv, inv_ne, p, sp, x, N, dN);
        for (int a = 0; a < q; ++a)
            for (int b = 0; b < q; ++b) {
                k[a * q + b] += dN[a] * wq * dN[b];
                m[a * q + b] += N[a] * wq * N[b];
            }
    }
    for (int a = 0; a < q * q; ++a) {
        Ke[(size_t)e * q * q + a] = k[a];
        Me[(size_t)e * q * q + a] = m[a];
    }
}

// banded 1D matrix: B[i*(2p+1) + (j-i+p)] for DOFs i, j (after Dirichlet removal)
__global__ void band1d_kernel(int ndof, int p, const int* __restrict__ kv, const int* __restrict__ elem_first,
                              const double* __restrict__ Ke, const double* __restrict__ Me,
                              double* __restrict__ Kb, double* __restrict__ Mb) {
    const int w = 2 * p + 1, q = p + 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ndof * w) return;
    int i = idx / w, d = idx % w, j = i + d - p;
    double ks = 0.0, ms = 0.0;
    if (j >= 0 && j < ndof) {
        int f = i + 1, g = j + 1;
        int lo = max(kv[f], kv[g]), hi = min(kv[f + p + 1], kv[g + p + 1]);
        for (int e = lo; e < hi; ++e) {
            int a = f - elem_first[e], b = g - elem_first[e];
            ks += Ke[(size_t)e * q * q + a * q + b];
            ms += Me[(size_t)e * q * q + a * q + b];
        }
    }
    Kb[idx] = ks;
    Mb[idx] = ms;
}

struct DirDev {
    const int* kv;
    const int* ef;
    const double* Ke;
    const double* Me;
    const double* Kb;
    const double* Mb;
    int n;  // DOFs
    int ne;
};

__global__ void csr_kron_kernel(int dim, int p, long long N, long long row0, long long goff,
                                const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const int* __restrict__ perm, DirDev X, DirDev Y, DirDev Z, double* __restrict__ Kv,
                                double* __restrict__ Mv) {
    const int lane = threadIdx.x & 31;
    long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= N) return;
    row += row0;
    const int w = 2 * p + 1;
    int g = (int)(perm[row] - goff);
    int ix = g % X.n, rem = g / X.n;
    int iy = dim > 1 ? rem % Y.n : 0;
    int iz = dim > 2 ? rem / Y.n : 0;
    for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
        int h = (int)(perm[col[e]] - goff);
        int jx = h % X.n, r2 = h / X.n;
        int jy = dim > 1 ? r2 % Y.n : 0;
        int jz = dim > 2 ? r2 / Y.n : 0;
        double kx = X.Kb[ix * w + jx - ix + p], mx = X.Mb[ix * w + jx - ix + p];
        double kval, mval;
        if (dim == 1) {
            kval = kx;
            mval = mx;
        } else if (dim == 2) {
            double ky = Y.Kb[iy * w + jy - iy + p], my = Y.Mb[iy * w + jy - iy + p];
            kval = my * kx + ky * mx;
            mval = my * mx;
        } else {
            double ky = Y.Kb[iy * w + jy - iy + p], my = Y.Mb[iy * w + jy - iy + p];
            double kz = Z.Kb[iz * w + jz - iz + p], mz = Z.Mb[iz * w + jz - iz + p];
            kval = mz * my * kx + mz * ky * mx + kz * my * mx;
            mval = mz * my * mx;
        }
        Kv[e] = kval;
        Mv[e] = mval;
    }
}

__device__ __forceinline__ void elem_range(const DirDev& D, int p, int i, int j, int& lo, int& hi) {
    int f = i + 1, g = j + 1;
    lo = max(D.kv[f], D.kv[g]);
    hi = min(D.kv[f + p + 1], D.kv[g + p + 1]);
}

__global__ void csr_coef_kernel(int dim, int p, long long N, long long row0, long long goff,
                                const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const int* __restrict__ perm, DirDev X, DirDev Y, DirDev Z,
                                const double* __restrict__ cK, const double* __restrict__ cM, double* __restrict__ Kv,
                                double* __restrict__ Mv) {
    const int lane = threadIdx.x & 31;
    long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= N) return;
    row += row0;
    const int q = p + 1, qq = q * q;
    int g = (int)(perm[row] - goff);
    int ix = g % X.n, rem = g / X.n;
    int iy = dim > 1 ? rem % Y.n : 0;
    int iz = dim > 2 ? rem / Y.n : 0;
    for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
        int h = (int)(perm[col[e]] - goff);
        int jx = h % X.n, r2 = h / X.n;
        int jy = dim > 1 ? r2 % Y.n : 0;
        int jz = dim > 2 ? r2 / Y.n : 0;
        int xlo, xhi, ylo = 0, yhi = 1, zlo = 0, zhi = 1;
        elem_range(X, p, ix, jx, xlo, xhi);
        if (dim > 1) elem_range(Y, p, iy, jy, ylo, yhi);
        if (dim > 2) elem_range(Z, p, iz, jz, zlo, zhi);
        double ks = 0.0, ms = 0.0;
        for (int ez = zlo; ez < zhi; ++ez) {
            double kz = 1.0, mz = 1.0;
            if (dim > 2) {
                int a = iz + 1 - Z.ef[ez], b = jz + 1 - Z.ef[ez];
                kz = Z.Ke[(size_t)ez * qq + a * q + b];
                mz = Z.Me[(size_t)ez * qq + a * q + b];
            }
            for (int ey = ylo; ey < yhi; ++ey) {
                double ky = 1.0, my = 1.0;
                if (dim > 1) {
                    int a = iy + 1 - Y.ef[ey], b = jy + 1 - Y.ef[ey];
                    ky = Y.Ke[(size_t)ey * qq + a * q + b];
                    my = Y.Me[(size_t)ey * qq + a * q + b];
                }
                for (int ex = xlo; ex < xhi; ++ex) {
                    int a = ix + 1 - X.ef[ex], b = jx + 1 - X.ef[ex];
                    double kx = X.Ke[(size_t)ex * qq + a * q + b];
                    double mx = X.Me[(size_t)ex * qq + a * q + b];
                    long long el = ex + (long long)X.ne * (ey + (long long)Y.ne * ez);
                    double kl, ml;
                    if (dim == 1) {
                        kl = kx;
                        ml = mx;
                    } else if (dim == 2) {
                        kl = my * kx + ky * mx;
                        ml = my * mx;
                    } else {
                        kl = mz * my * kx + mz * ky * mx + kz * my * mx;
                        ml = mz * my * mx;
                    }
                    ks += (cK ? cK[el] : 1.0) * kl;
                    ms += (cM ? cM[el] : 1.0) * ml;
                }
            }
        }
        Kv[e] = ks;
        Mv[e] = ms;
    }
}

// Assembles one problem (its 1D data in P) into rows [row0, row0 + P.N) of the
// context's CSR; goff is the problem's first global DOF.  cK / cM: device
// coefficient arrays of the problem (NULL = constant).
int assemble_problem(riga_ctx* c, const Symbolic& P, long long row0, long long goff, const double* cK,
                     const double* cM) {
    cudaStream_t st = c->stream;
    DirDev dd[3];
    for (int a = 0; a < 3; ++a) {
        dd[a] = DirDev{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1, 1};
        if (a >= P.dim) continue;
        const Dir1D& D = P.dir[a];
        const int q = P.p + 1, w = 2 * P.p + 1;
        RIGA_CUDA_TRY(c, c->kv[a].upload(D.kv, st));
        RIGA_CUDA_TRY(c, c->elem_first[a].upload(D.elem_first, st));
        RIGA_CUDA_TRY(c, c->Ke1[a].alloc((size_t)D.ne * q * q));
        RIGA_CUDA_TRY(c, c->Me1[a].alloc((size_t)D.ne * q * q));
        RIGA_CUDA_TRY(c, c->Kb1[a].alloc((size_t)D.ndof * w));
        RIGA_CUDA_TRY(c, c->Mb1[a].alloc((size_t)D.ndof * w));
        { count_launch(c); elem1d_kernel<<<(D.ne + 127) / 128, 128, 0, st>>>(D.ne, P.p, c->kv[a].ptr, c->elem_first[a].ptr,
                                                          c->Ke1[a].ptr, c->Me1[a].ptr); }
        { count_launch(c); band1d_kernel<<<(D.ndof * w + 127) / 128, 128, 0, st>>>(D.ndof, P.p, c->kv[a].ptr, c->elem_first[a].ptr,
                                                                c->Ke1[a].ptr, c->Me1[a].ptr, c->Kb1[a].ptr,
                                                                c->Mb1[a].ptr); }
        dd[a] = DirDev{c->kv[a].ptr, c->elem_first[a].ptr, c->Ke1[a].ptr, c->Me1[a].ptr,
                       c->Kb1[a].ptr, c->Mb1[a].ptr, D.ndof, D.ne};
    }
    long long threads = P.N * 32;
    int blocks = (int)((threads + 255) / 256);
    if (!cK && !cM) {
        { count_launch(c); csr_kron_kernel<<<blocks, 256, 0, st>>>(P.dim, P.p, P.N, row0, goff, c->rowptr.ptr, c->col.ptr, c->perm.ptr,
                                                dd[0], dd[1], dd[2], c->Kval.ptr, c->Mval.ptr); }
    } else {
        { count_launch(c); csr_coef_kernel<<<blocks, 256, 0, st>>>(P.dim, P.p, P.N, row0, goff, c->rowptr.ptr, c->col.ptr, c->perm.ptr,
                                                dd[0], dd[1], dd[2], cK, cM, c->Kval.ptr, c->Mval.ptr); }
    }
    RIGA_CUDA_TRY(c, cudaGetLastError());
    return RIGA_OK;
}

int assemble_device(riga_ctx* c) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_ASSEMBLE, (double)S.nnz * 16.0);
    RIGA_CUDA_TRY(c, c->Kval.alloc(S.nnz));
    RIGA_CUDA_TRY(c, c->Mval.alloc(S.nnz));
    const double* cK = nullptr;
    const double* cM = nullptr;
    if (!c->coefK.empty()) {
        RIGA_CUDA_TRY(c, c->dcoefK.upload(c->coefK, st));
        cK = c->dcoefK.ptr;
    }
    if (!c->coefM.empty()) {
        RIGA_CUDA_TRY(c, c->dcoefM.upload(c->coefM, st));
        cM = c->dcoefM.ptr;
    }
    if (S.dim > 0) return assemble_problem(c, S, 0, 0, cK, cM);
    // batch: one problem at a time into its rows of the merged CSR
    for (size_t b = 0; b < c->probs.size(); ++b) {
        const long long e0 = S.prob_elem[b];
        int rc = assemble_problem(c, c->probs[b], S.prob_pos[b], S.prob_pos[b], cK ? cK + e0 : nullptr,
                                  cM ? cM + e0 : nullptr);
        if (rc) return rc;
    }
    return RIGA_OK;
}

}  // namespace riga
