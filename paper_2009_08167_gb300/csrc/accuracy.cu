// Eigenvalue and eigenfunction errors of computed eigenpairs against the
// exact Laplace eigenpairs of the unit interval, square or cube (Sec. 2,
// Eq. exact: lambda = pi^2 (i^2 + j^2 [+ k^2]),
// u = 2^{d/2} sin(i pi x) sin(j pi y) [sin(k pi z)]; Eq. eigerrors):
//   EVerr    = (lambda_h - lambda) / lambda,
//   EFerr_L2 = ||s u_h - u||^2,
//   EFerr_E  = a(s u_h - u, s u_h - u) / lambda,
// u_h the M-normalised computed eigenvector (L2 norm 1), s = sign (u_h, u).
// Sec. 8 studies them against the mode number (Figs. 12-14); Eq. Pythagorean
// says EFerr_E = EVerr + EFerr_L2 for a Rayleigh-quotient eigenvalue.
//
// Integrals: nq Gauss-Legendre points per element and direction.
//   acc_table_kernel  per direction, element and point: the point, its
//                     weight and the p + 1 non-zero B-splines and derivatives
//                     (Cox-de Boor, Eq. N);
//   acc_sum_kernel    one pass over the tensor grid of points per eigenpair
//                     (blockIdx.y): u_h and grad u_h from the element's
//                     (p + 1)^d coefficients, the exact mode, and per-block
//                     partial sums of w u_h u (pass 0, for the sign) or of
//                     w (s u_h - u)^2 and w |s grad u_h - grad u|^2 (pass 1;
//                     the differences are formed point by point, so tiny
//                     errors keep their relative accuracy); the host adds the
//                     partial sums in a fixed order.
#include <cstring>

#include "basis.cuh"
#include "ctx.h"

namespace riga {

namespace {

constexpr int ACC_NQ_MAX = 16;
constexpr int ACC_BLOCKS = 304;  // partial sums per eigenpair (2 x the SM count)

// table entry of (element e, point g): x, w, first DOF (after Dirichlet
// removal, may be -1), then N[0..p], dN[0..p]
__global__ void acc_table_kernel(int ne, int p, int nq, int ndof, const int* __restrict__ kv,
                                 const int* __restrict__ elem_first, double* __restrict__ tab) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ne * nq) return;
    const int e = idx / nq, g = idx % nq;
    double t[ACC_NQ_MAX], w[ACC_NQ_MAX];
    gauss_legendre_dev(nq, t, w);
    const double h = 1.0 / ne;
    const double x = (e + (t[g] + 1.0) * 0.5) * h;
    double N[PMAX + 1], dN[PMAX + 1];
    basis_span(kv, 1.0 / ne, p, elem_first[e] + p, x, N, dN);
    const int stride = 3 + 2 * (p + 1);
    double* o = tab + (size_t)idx * stride;
    o[0] = x;
    o[1] = w[g] * h * 0.5;
    o[2] = (double)(elem_first[e] - 1);
    for (int a = 0; a <= p; ++a) {
        o[3 + a] = N[a];
        o[3 + p + 1 + a] = dN[a];
    }
    (void)ndof;
}

struct AccDir {
    const double* tab;  // per (element, point) entries, stride 3 + 2 (p + 1)
    int npts;           // ne * nq
    int ndof;
    int n1;             // DOFs of the direction (index stride)
};

template <int DIM>
__global__ void __launch_bounds__(256) acc_sum_kernel(int p, AccDir d0, AccDir d1, AccDir d2, long long npts,
                                                      const int* __restrict__ ipos, const double* __restrict__ U,
                                                      long long N, const int* __restrict__ modes,
                                                      const double* __restrict__ sgn, int pass,
                                                      double* __restrict__ partial) {
    __shared__ double red[2][8];
    const int q = blockIdx.y;
    const int stride = 3 + 2 * (p + 1);
    const double* u = U + (long long)q * N;
    int mode[3] = {1, 1, 1};
    for (int a = 0; a < DIM; ++a) mode[a] = modes[q * DIM + a];
    const double s = pass == 1 ? sgn[q] : 1.0;
    const double amp = DIM == 1 ? 1.4142135623730951 : (DIM == 2 ? 2.0 : 2.8284271247461903);
    double acc0 = 0.0, acc1 = 0.0;
    const AccDir dirs[3] = {d0, d1, d2};
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < npts; t += (long long)gridDim.x * blockDim.x) {
        // point indices per direction, x fastest
        int pi[3] = {0, 0, 0};
        long long r = t;
        for (int a = 0; a < DIM; ++a) {
            pi[a] = (int)(r % dirs[a].npts);
            r /= dirs[a].npts;
        }
        const double* e[3];
        double wt = 1.0, ex = 1.0;
        double sv[3], cv[3];
        for (int a = 0; a < DIM; ++a) {
            e[a] = dirs[a].tab + (size_t)pi[a] * stride;
            wt *= e[a][1];
            sincospi((double)mode[a] * e[a][0], &sv[a], &cv[a]);
            cv[a] *= mode[a] * 3.141592653589793;
        }
        // exact mode and gradient
        double ue = amp, ge[3] = {amp, amp, amp};
        for (int a = 0; a < DIM; ++a) {
            ue *= sv[a];
            for (int b = 0; b < DIM; ++b) ge[b] *= (a == b) ? cv[a] : sv[a];
        }
        // computed field and gradient over the (p + 1)^DIM local functions
        double uh = 0.0, gh[3] = {0.0, 0.0, 0.0};
        const int f0x = (int)e[0][2];
        const int f0y = DIM > 1 ? (int)e[1][2] : 0;
        const int f0z = DIM > 2 ? (int)e[2][2] : 0;
        for (int kz = 0; kz <= (DIM > 2 ? p : 0); ++kz) {
            const int iz = f0z + kz;
            if (DIM > 2 && (iz < 0 || iz >= dirs[2].ndof)) continue;
            const double Nz = DIM > 2 ? e[2][3 + kz] : 1.0, dNz = DIM > 2 ? e[2][3 + p + 1 + kz] : 0.0;
            for (int ky = 0; ky <= (DIM > 1 ? p : 0); ++ky) {
                const int iy = f0y + ky;
                if (DIM > 1 && (iy < 0 || iy >= dirs[1].ndof)) continue;
                const double Ny = DIM > 1 ? e[1][3 + ky] : 1.0, dNy = DIM > 1 ? e[1][3 + p + 1 + ky] : 0.0;
                for (int kx = 0; kx <= p; ++kx) {
                    const int ix = f0x + kx;
                    if (ix < 0 || ix >= dirs[0].ndof) continue;
                    const double Nx = e[0][3 + kx], dNx = e[0][3 + p + 1 + kx];
                    long long g = ix;
                    if (DIM > 1) g += (long long)iy * dirs[0].n1;
                    if (DIM > 2) g += (long long)iz * dirs[0].n1 * dirs[1].n1;
                    const double cf = u[ipos[g]];
                    uh += cf * Nx * Ny * Nz;
                    gh[0] += cf * dNx * Ny * Nz;
                    if (DIM > 1) gh[1] += cf * Nx * dNy * Nz;
                    if (DIM > 2) gh[2] += cf * Nx * Ny * dNz;
                }
            }
        }
        if (pass == 0) {
            acc0 += wt * uh * ue;
        } else {
            const double du = s * uh - ue;
            acc0 += wt * du * du;
            double gg = 0.0;
            for (int a = 0; a < DIM; ++a) {
                const double dg = s * gh[a] - ge[a];
                gg += dg * dg;
            }
            acc1 += wt * gg;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc0 += __shfl_xor_sync(0xffffffffu, acc0, o);
        acc1 += __shfl_xor_sync(0xffffffffu, acc1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = acc0;
        red[1][threadIdx.x >> 5] = acc1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < 8; ++w) {
            a0 += red[0][w];
            a1 += red[1][w];
        }
        partial[((size_t)q * gridDim.x + blockIdx.x) * 2] = a0;
        partial[((size_t)q * gridDim.x + blockIdx.x) * 2 + 1] = a1;
    }
}

}  // namespace

int eig_errors_device(riga_ctx* c, int nev, const int* modes_host, int nq, double* everr, double* efl2, double* efe) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    const int dim = S.dim, p = S.p;
    if (dim < 1 || dim > 3) return set_error(c, RIGA_ESTATE, "single-problem context needed");
    if (nq <= 0) nq = p + 6;
    if (nq > ACC_NQ_MAX) return set_error(c, RIGA_EINVAL, "nq must be at most 16");
    for (int q = 0; q < nev * dim; ++q)
        if (modes_host[q] < 1) return set_error(c, RIGA_EINVAL, "mode indices start at 1");
    const int stride = 3 + 2 * (p + 1);
    DevBuf<double> tab[3];
    AccDir dirs[3];
    long long npts = 1;
    for (int a = 0; a < 3; ++a) {
        dirs[a] = AccDir{nullptr, 1, 1, 1};
        if (a >= dim) continue;
        const int ne = S.dir[a].ne;
        RIGA_CUDA_TRY(c, tab[a].alloc((size_t)ne * nq * stride));
        count_launch(c);
        acc_table_kernel<<<(ne * nq + 127) / 128, 128, 0, st>>>(ne, p, nq, S.dir[a].ndof, c->kv[a].ptr,
                                                               c->elem_first[a].ptr, tab[a].ptr);
        dirs[a] = AccDir{tab[a].ptr, ne * nq, S.dir[a].ndof, S.n1[a]};
        npts *= (long long)ne * nq;
    }
    DevBuf<int> dmodes;
    DevBuf<double> dsgn, part;
    std::vector<int> mv(modes_host, modes_host + (size_t)nev * dim);
    RIGA_CUDA_TRY(c, dmodes.upload(mv, st));
    RIGA_CUDA_TRY(c, dsgn.alloc(nev));
    RIGA_CUDA_TRY(c, part.alloc((size_t)nev * ACC_BLOCKS * 2));
    std::vector<double> hp((size_t)nev * ACC_BLOCKS * 2), sg(nev, 1.0);
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) RIGA_CUDA_TRY(c, cudaMemcpyAsync(dsgn.ptr, sg.data(), nev * sizeof(double), cudaMemcpyHostToDevice, st));
        dim3 grid(ACC_BLOCKS, nev);
        count_launch(c);
        if (dim == 1)
            acc_sum_kernel<1><<<grid, 256, 0, st>>>(p, dirs[0], dirs[1], dirs[2], npts, c->ipos.ptr, c->evec_perm.ptr, S.N,
                                                    dmodes.ptr, dsgn.ptr, pass, part.ptr);
        else if (dim == 2)
            acc_sum_kernel<2><<<grid, 256, 0, st>>>(p, dirs[0], dirs[1], dirs[2], npts, c->ipos.ptr, c->evec_perm.ptr, S.N,
                                                    dmodes.ptr, dsgn.ptr, pass, part.ptr);
        else
            acc_sum_kernel<3><<<grid, 256, 0, st>>>(p, dirs[0], dirs[1], dirs[2], npts, c->ipos.ptr, c->evec_perm.ptr, S.N,
                                                    dmodes.ptr, dsgn.ptr, pass, part.ptr);
        RIGA_CUDA_TRY(c, cudaGetLastError());
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(hp.data(), part.ptr, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
        for (int q = 0; q < nev; ++q) {
            double a0 = 0.0, a1 = 0.0;
            for (int b = 0; b < ACC_BLOCKS; ++b) {
                a0 += hp[((size_t)q * ACC_BLOCKS + b) * 2];
                a1 += hp[((size_t)q * ACC_BLOCKS + b) * 2 + 1];
            }
            double lam_e = 0.0;
            for (int a = 0; a < dim; ++a) lam_e += (double)mv[q * dim + a] * mv[q * dim + a];
            lam_e *= 9.869604401089358;  // pi^2
            if (pass == 0) {
                sg[q] = a0 >= 0.0 ? 1.0 : -1.0;
            } else {
                everr[q] = (c->evals[q] - lam_e) / lam_e;
                efl2[q] = a0;
                efe[q] = a1 / lam_e;
            }
        }
    }
    return RIGA_OK;
}

}  // namespace riga
