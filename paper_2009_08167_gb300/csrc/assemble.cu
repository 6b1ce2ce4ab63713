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
#include "basis.cuh"

namespace riga {

__device__ void elem1d_one(int e, int ne, int p, const int* __restrict__ kv, const int* __restrict__ elem_first,
                           double* __restrict__ Ke, double* __restrict__ Me) {
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

__global__ void elem1d_kernel(int ne, int p, const int* __restrict__ kv, const int* __restrict__ elem_first,
                              double* __restrict__ Ke, double* __restrict__ Me) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < ne) elem1d_one(e, ne, p, kv, elem_first, Ke, Me);
}

// banded 1D matrix: B[i*(2p+1) + (j-i+p)] for DOFs i, j (after Dirichlet removal)
__device__ void band1d_one(int idx, int ndof, int p, const int* __restrict__ kv, const int* __restrict__ elem_first,
                           const double* __restrict__ Ke, const double* __restrict__ Me, double* __restrict__ Kb,
                           double* __restrict__ Mb) {
    const int w = 2 * p + 1, q = p + 1;
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

__global__ void band1d_kernel(int ndof, int p, const int* __restrict__ kv, const int* __restrict__ elem_first,
                              const double* __restrict__ Ke, const double* __restrict__ Me,
                              double* __restrict__ Kb, double* __restrict__ Mb) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < ndof * (2 * p + 1)) band1d_one(idx, ndof, p, kv, elem_first, Ke, Me, Kb, Mb);
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

// one row of the CSR (one warp), constant coefficients
__device__ __forceinline__ void csr_kron_row(int dim, int p, long long row, long long goff, int lane,
                                             const long long* __restrict__ rowptr, const int* __restrict__ col,
                                             const int* __restrict__ perm, const DirDev& X, const DirDev& Y,
                                             const DirDev& Z, double* __restrict__ Kv, double* __restrict__ Mv) {
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

__global__ void csr_kron_kernel(int dim, int p, long long N, long long row0, long long goff,
                                const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const int* __restrict__ perm, DirDev X, DirDev Y, DirDev Z, double* __restrict__ Kv,
                                double* __restrict__ Mv) {
    long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row < N) csr_kron_row(dim, p, row + row0, goff, threadIdx.x & 31, rowptr, col, perm, X, Y, Z, Kv, Mv);
}

__device__ __forceinline__ void elem_range(const DirDev& D, int p, int i, int j, int& lo, int& hi) {
    int f = i + 1, g = j + 1;
    lo = max(D.kv[f], D.kv[g]);
    hi = min(D.kv[f + p + 1], D.kv[g + p + 1]);
}

// one row of the CSR (one warp), per-element coefficients
__device__ __forceinline__ void csr_coef_row(int dim, int p, long long row, long long goff, int lane,
                                             const long long* __restrict__ rowptr, const int* __restrict__ col,
                                             const int* __restrict__ perm, const DirDev& X, const DirDev& Y,
                                             const DirDev& Z, const double* __restrict__ cK,
                                             const double* __restrict__ cM, double* __restrict__ Kv,
                                             double* __restrict__ Mv) {
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

__global__ void csr_coef_kernel(int dim, int p, long long N, long long row0, long long goff,
                                const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const int* __restrict__ perm, DirDev X, DirDev Y, DirDev Z,
                                const double* __restrict__ cK, const double* __restrict__ cM, double* __restrict__ Kv,
                                double* __restrict__ Mv) {
    long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row < N)
        csr_coef_row(dim, p, row + row0, goff, threadIdx.x & 31, rowptr, col, perm, X, Y, Z, cK, cM, Kv, Mv);
}

// ------------------------------------------------------------------ batches
// All problems of a batch in three launches: the 1D element matrices of every
// (problem, direction) segment, the banded 1D matrices, and the CSR rows,
// each row finding its problem (and that problem's segments) from its
// position.
__device__ __forceinline__ int find_segment(const long long* __restrict__ prefix, int nseg, long long t) {
    int lo = 0, hi = nseg;  // prefix[lo] <= t < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void elem1d_batch_kernel(int nseg, const long long* __restrict__ eprefix, const SegDev* __restrict__ segs,
                                    const int* __restrict__ kv, const int* __restrict__ ef, double* __restrict__ Ke,
                                    double* __restrict__ Me) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= eprefix[nseg]) return;
    const int sgi = find_segment(eprefix, nseg, t);
    const SegDev sg = segs[sgi];
    elem1d_one((int)(t - eprefix[sgi]), sg.ne, sg.p, kv + sg.kv_off, ef + sg.ef_off, Ke + sg.ke_off, Me + sg.ke_off);
}

__global__ void band1d_batch_kernel(int nseg, const long long* __restrict__ bprefix, const SegDev* __restrict__ segs,
                                    const int* __restrict__ kv, const int* __restrict__ ef,
                                    const double* __restrict__ Ke, const double* __restrict__ Me,
                                    double* __restrict__ Kb, double* __restrict__ Mb) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= bprefix[nseg]) return;
    const int sgi = find_segment(bprefix, nseg, t);
    const SegDev sg = segs[sgi];
    band1d_one((int)(t - bprefix[sgi]), sg.ndof, sg.p, kv + sg.kv_off, ef + sg.ef_off, Ke + sg.ke_off,
               Me + sg.ke_off, Kb + sg.kb_off, Mb + sg.kb_off);
}

__global__ void csr_batch_kernel(long long N, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                 const int* __restrict__ perm, const int* __restrict__ prob_of_pos,
                                 const ProbDev* __restrict__ probs, const SegDev* __restrict__ segs,
                                 const int* __restrict__ kv, const int* __restrict__ ef, const double* __restrict__ Ke,
                                 const double* __restrict__ Me, const double* __restrict__ Kb,
                                 const double* __restrict__ Mb, const double* __restrict__ cK,
                                 const double* __restrict__ cM, double* __restrict__ Kv, double* __restrict__ Mv) {
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= N) return;
    const ProbDev pr = probs[prob_of_pos[row]];
    DirDev d[3];
    for (int a = 0; a < 3; ++a) {
        d[a] = DirDev{nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 1, 1};
        if (a >= pr.dim) continue;
        const SegDev sg = segs[pr.seg0 + a];
        d[a] = DirDev{kv + sg.kv_off, ef + sg.ef_off, Ke + sg.ke_off, Me + sg.ke_off, Kb + sg.kb_off, Mb + sg.kb_off,
                      sg.ndof, sg.ne};
    }
    const int lane = threadIdx.x & 31;
    if (cK || cM)
        csr_coef_row(pr.dim, pr.p, row, pr.goff, lane, rowptr, col, perm, d[0], d[1], d[2], cK ? cK + pr.e0 : nullptr,
                     cM ? cM + pr.e0 : nullptr, Kv, Mv);
    else
        csr_kron_row(pr.dim, pr.p, row, pr.goff, lane, rowptr, col, perm, d[0], d[1], d[2], Kv, Mv);
}

// The batch's 1D data (knot vectors, element-to-function maps) and the
// descriptors of its segments and problems, uploaded once per batch pattern.
int prepare_batch_assembly(riga_ctx* c) {
    cudaStream_t st = c->stream;
    std::vector<int> kv, ef;
    std::vector<SegDev> segs;
    std::vector<ProbDev> probs;
    std::vector<long long> ep{0}, bp{0};
    long long ke = 0, kb = 0;
    for (size_t b = 0; b < c->probs.size(); ++b) {
        const Symbolic& P = c->probs[b];
        ProbDev pd{P.dim, P.p, (int)segs.size(), 0, c->S.prob_pos[b], c->S.prob_pos[b], c->S.prob_elem[b]};
        probs.push_back(pd);
        const int q = P.p + 1, w = 2 * P.p + 1;
        for (int a = 0; a < P.dim; ++a) {
            const Dir1D& D = P.dir[a];
            SegDev sg{D.ne, P.p, D.ndof, 0, (long long)kv.size(), (long long)ef.size(), ke, kb};
            kv.insert(kv.end(), D.kv.begin(), D.kv.end());
            ef.insert(ef.end(), D.elem_first.begin(), D.elem_first.end());
            ke += (long long)D.ne * q * q;
            kb += (long long)D.ndof * w;
            ep.push_back(ep.back() + D.ne);
            bp.push_back(bp.back() + (long long)D.ndof * w);
            segs.push_back(sg);
        }
    }
    c->b_nseg = (int)segs.size();
    c->b_nelem1d = ep.back();
    c->b_nband = bp.back();
    RIGA_CUDA_TRY(c, c->b_kv.upload(kv, st));
    RIGA_CUDA_TRY(c, c->b_ef.upload(ef, st));
    RIGA_CUDA_TRY(c, c->b_segs.upload(segs, st));
    RIGA_CUDA_TRY(c, c->b_probs.upload(probs, st));
    RIGA_CUDA_TRY(c, c->b_eprefix.upload(ep, st));
    RIGA_CUDA_TRY(c, c->b_bprefix.upload(bp, st));
    RIGA_CUDA_TRY(c, c->b_Ke.alloc(ke));
    RIGA_CUDA_TRY(c, c->b_Me.alloc(ke));
    RIGA_CUDA_TRY(c, c->b_Kb.alloc(kb));
    RIGA_CUDA_TRY(c, c->b_Mb.alloc(kb));
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
    return RIGA_OK;
}

// Assembles a single problem (its 1D data in P).  cK / cM: device
// coefficient arrays (NULL = constant).
int assemble_problem(riga_ctx* c, const Symbolic& P, const double* cK, const double* cM) {
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
        { count_launch(c); csr_kron_kernel<<<blocks, 256, 0, st>>>(P.dim, P.p, P.N, 0, 0, c->rowptr.ptr, c->col.ptr, c->perm.ptr,
                                                dd[0], dd[1], dd[2], c->Kval.ptr, c->Mval.ptr); }
    } else {
        { count_launch(c); csr_coef_kernel<<<blocks, 256, 0, st>>>(P.dim, P.p, P.N, 0, 0, c->rowptr.ptr, c->col.ptr, c->perm.ptr,
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
    if (S.dim > 0) return assemble_problem(c, S, cK, cM);
    // batch: every problem in three launches
    if (c->b_nseg < 1) return set_error(c, RIGA_ESTATE, "batch assembly data missing");
    { count_launch(c); elem1d_batch_kernel<<<(unsigned)((c->b_nelem1d + 127) / 128), 128, 0, st>>>(
        c->b_nseg, c->b_eprefix.ptr, c->b_segs.ptr, c->b_kv.ptr, c->b_ef.ptr, c->b_Ke.ptr, c->b_Me.ptr); }
    { count_launch(c); band1d_batch_kernel<<<(unsigned)((c->b_nband + 127) / 128), 128, 0, st>>>(
        c->b_nseg, c->b_bprefix.ptr, c->b_segs.ptr, c->b_kv.ptr, c->b_ef.ptr, c->b_Ke.ptr, c->b_Me.ptr, c->b_Kb.ptr,
        c->b_Mb.ptr); }
    { count_launch(c); csr_batch_kernel<<<(unsigned)((S.N * 32 + 255) / 256), 256, 0, st>>>(
        S.N, c->rowptr.ptr, c->col.ptr, c->perm.ptr, c->prob_of_pos.ptr, c->b_probs.ptr, c->b_segs.ptr, c->b_kv.ptr,
        c->b_ef.ptr, c->b_Ke.ptr, c->b_Me.ptr, c->b_Kb.ptr, c->b_Mb.ptr, cK, cM, c->Kval.ptr, c->Mval.ptr); }
    RIGA_CUDA_TRY(c, cudaGetLastError());
    return RIGA_OK;
}

}  // namespace riga
