// C ABI entry points (include/riga.h).  Argument checking, host/device
// pointer handling, and the order of the device phases; every numeric step
// runs in the kernels of assemble.cu, factor.cu, solve.cu, lanczos.cu and
// adjoint.cu (the tridiagonal Rayleigh-Ritz step of tridiag.cpp runs on the
// host, inside this library).
#include <cstring>
#include <new>

#include "ctx.h"

namespace riga {

int set_error(riga_ctx* c, int code, const std::string& msg) {
    if (c) c->last_error = msg;
    return code;
}

void sign_fix(riga_ctx* c, double* U, int ncols);

namespace {

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy n values between a user pointer (host or device) and a device buffer
template <typename T>
int to_device(riga_ctx* c, const T* user, T* dev, size_t n) {
    if (n == 0) return RIGA_OK;
    cudaMemcpyKind kind = is_device_ptr(user) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(dev, user, n * sizeof(T), kind, c->stream));
    if (kind == cudaMemcpyHostToDevice) RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RIGA_OK;
}

template <typename T>
int to_user(riga_ctx* c, const T* dev, T* user, size_t n) {
    if (n == 0) return RIGA_OK;
    cudaMemcpyKind kind = is_device_ptr(user) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(user, dev, n * sizeof(T), kind, c->stream));
    if (kind == cudaMemcpyDeviceToHost) RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RIGA_OK;
}

}  // namespace

int upload_symbolic(riga_ctx* c) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    RIGA_CUDA_TRY(c, c->rowptr.upload(S.rowptr, st));
    RIGA_CUDA_TRY(c, c->col.upload(S.col, st));
    RIGA_CUDA_TRY(c, c->perm.upload(S.perm, st));
    RIGA_CUDA_TRY(c, c->ipos.upload(S.ipos, st));
    RIGA_CUDA_TRY(c, c->node_ptr.upload(S.node_ptr, st));
    RIGA_CUDA_TRY(c, c->kk.upload(S.k, st));
    RIGA_CUDA_TRY(c, c->nn.upload(S.n, st));
    RIGA_CUDA_TRY(c, c->parent.upload(S.parent, st));
    RIGA_CUDA_TRY(c, c->front_off.upload(S.front_off, st));
    RIGA_CUDA_TRY(c, c->front_ptr.upload(S.front_ptr, st));
    RIGA_CUDA_TRY(c, c->front_pos.upload(S.front_pos, st));
    RIGA_CUDA_TRY(c, c->child_ptr.upload(S.child_ptr, st));
    RIGA_CUDA_TRY(c, c->child_list.upload(S.child_list.empty() ? std::vector<int>{0} : S.child_list, st));
    RIGA_CUDA_TRY(c, c->rel.upload(S.rel.empty() ? std::vector<int>{0} : S.rel, st));
    RIGA_CUDA_TRY(c, c->rel_ptr.upload(S.rel_ptr, st));
    RIGA_CUDA_TRY(c, c->upd_off.upload(S.upd_off, st));
    RIGA_CUDA_TRY(c, c->scatter.upload(S.scatter, st));
    RIGA_CUDA_TRY(c, c->perm_to_glob.upload(S.perm_to_glob, st));
    RIGA_CUDA_TRY(c, c->glob_rowptr.upload(S.glob_rowptr, st));
    RIGA_CUDA_TRY(c, c->sitems.upload(S.sitems, st));
    RIGA_CUDA_TRY(c, c->crec.upload(S.crec.empty() ? std::vector<ChildRec>{ChildRec{0, 0, 0, 0, 0, 0}} : S.crec, st));
    RIGA_CUDA_TRY(c, c->parts_f.upload(S.parts_f, st));
    RIGA_CUDA_TRY(c, c->parts_b.upload(S.parts_b, st));
    RIGA_CUDA_TRY(c, c->qitems.upload(S.qitems.empty() ? std::vector<PanelItem>{PanelItem{0, 0}} : S.qitems, st));
    // front of each persistent-solve work item (for traces)
    std::vector<int> order;
    for (const SolveItem& it : S.sitems) order.push_back(it.front);
    RIGA_CUDA_TRY(c, c->solve_order.upload(order, st));
    c->solve_flags.release();
    RIGA_CUDA_TRY(c, c->pitems.upload(S.pitems.empty() ? std::vector<PanelItem>{PanelItem{0, 0}} : S.pitems, st));
    RIGA_CUDA_TRY(c, c->titems.upload(S.titems.empty() ? std::vector<TileItem>{TileItem{0, 0, 0}} : S.titems, st));
    RIGA_CUDA_TRY(c, c->tcitems.upload(S.tc_tiles.empty() ? std::vector<TcTile>{TcTile{0, 0, 0, 0, 0, 0}} : S.tc_tiles, st));
    RIGA_CUDA_TRY(c, c->tcpacks.upload(S.tc_packs.empty() ? std::vector<TcPack>{TcPack{0, 0, 0, 0}} : S.tc_packs, st));
    RIGA_CUDA_TRY(c, c->tcnarrow.upload(S.tc_narrow.empty() ? std::vector<TileItemL>{TileItemL{0, 0, 0, 0}} : S.tc_narrow, st));
    RIGA_CUDA_TRY(c, c->ozpacks.upload(S.oz_packs.empty() ? std::vector<TcPack>{TcPack{0, 0, 0, 0}} : S.oz_packs, st));
    RIGA_CUDA_TRY(c, c->oztiles.upload(S.oz_tiles.empty() ? std::vector<TcTile>{TcTile{0, 0, 0, 0, 0, 0}} : S.oz_tiles, st));
    RIGA_CUDA_TRY(c, c->eitems.upload(S.eitems.empty() ? std::vector<ExtItem>{ExtItem{0, 0, 0}} : S.eitems, st));
    if (S.dim == 0) RIGA_CUDA_TRY(c, c->prob_of_pos.upload(S.prob_of_pos, st));
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
    ++c->sched_gen;
    return RIGA_OK;
}

namespace {

__global__ void scatter_glob_kernel(long long nnz, const long long* __restrict__ p2g, const double* __restrict__ src,
                                    double* __restrict__ dst) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz) dst[p2g[e]] = src[e];
}

__global__ void glob_col_kernel(long long N, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const int* __restrict__ perm, const long long* __restrict__ p2g,
                                int* __restrict__ gcol) {
    long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= N) return;
    for (long long e = rowptr[row]; e < rowptr[row + 1]; ++e) gcol[p2g[e]] = perm[col[e]];
}

__global__ void resid_partial_kernel(long long N, const double* __restrict__ Ku, const double* __restrict__ Mu,
                                     double lam, double* __restrict__ partial) {
    __shared__ double sa[8], sb[8];
    double xa = 0.0, xb = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        double r = Ku[i] - lam * Mu[i];
        xa += r * r;
        xb += Mu[i] * Mu[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xa += __shfl_xor_sync(0xffffffffu, xa, o);
        xb += __shfl_xor_sync(0xffffffffu, xb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = xa;
        sb[threadIdx.x >> 5] = xb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 8; ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        partial[2 * blockIdx.x] = ta;
        partial[2 * blockIdx.x + 1] = tb;
    }
}

std::vector<int> mesh_key(const riga_mesh* m) {
    std::vector<int> key{m->dim, m->p, m->leaf_extent > 0 ? m->leaf_extent : 8};
    for (int a = 0; a < m->dim; ++a) {
        key.push_back(m->ne[a]);
        for (int i = 0; i + 1 < m->ne[a]; ++i) key.push_back(m->mult[a] ? m->mult[a][i] : 1);
    }
    return key;
}

}  // namespace
}  // namespace riga

using namespace riga;

extern "C" {

int riga_create(riga_ctx** out, int device, void* cuda_stream) {
    if (!out) return RIGA_EINVAL;
    *out = nullptr;
    if (device == -1) {
        riga_ctx* h = new (std::nothrow) riga_ctx();
        if (!h) return RIGA_ENOMEM;
        h->device = -1;
        *out = h;
        return RIGA_OK;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return RIGA_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return RIGA_ECUDA;
    riga_ctx* c = new (std::nothrow) riga_ctx();
    if (!c) return RIGA_ENOMEM;
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    return RIGA_OK;
}

void riga_destroy(riga_ctx* c) {
    if (!c) return;
    if (c->device < 0) {
        delete c;
        return;
    }
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->bpin) cudaFreeHost(c->bpin);
    for (auto& g : c->fgraph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

const char* riga_strerror(int s) {
    switch (s) {
        case RIGA_OK: return "RIGA_OK";
        case RIGA_EINVAL: return "RIGA_EINVAL";
        case RIGA_ESTATE: return "RIGA_ESTATE";
        case RIGA_EPIVOT: return "RIGA_EPIVOT";
        case RIGA_ENOCONV: return "RIGA_ENOCONV";
        case RIGA_EREFINE: return "RIGA_EREFINE";
        case RIGA_ETIMEOUT: return "RIGA_ETIMEOUT";
        case RIGA_ECUDA: return "RIGA_ECUDA";
        case RIGA_ENOMEM: return "RIGA_ENOMEM";
        default: return "RIGA_UNKNOWN";
    }
}

const char* riga_last_error(riga_ctx* c) { return c ? c->last_error.c_str() : ""; }

static int check_mesh(riga_ctx* c, const riga_mesh* m) {
    if (m->dim < 1 || m->dim > 3) return set_error(c, RIGA_EINVAL, "dim must be 1, 2 or 3");
    if (m->dirichlet != 1) return set_error(c, RIGA_EINVAL, "only homogeneous Dirichlet (dirichlet = 1) is supported");
    if (m->p < 1 || m->p > 6) return set_error(c, RIGA_EINVAL, "p must be in 1..6");
    if (m->leaf_extent < 0) return set_error(c, RIGA_EINVAL, "leaf_extent must be >= 0");
    for (int a = 0; a < m->dim; ++a)
        if (m->ne[a] < 1 || m->ne[a] > (1 << 20)) return set_error(c, RIGA_EINVAL, "ne out of range");
    return RIGA_OK;
}

int riga_analyze(riga_ctx* c, const riga_mesh* m) {
    if (!c || !m) return RIGA_EINVAL;
    c->last_error.clear();
    int rc = check_mesh(c, m);
    if (rc) return rc;
    c->assembled = false;
    c->factored = false;
    c->nev = 0;
    c->mesh_key.clear();
    std::string err = build_symbolic(c->S, m->dim, m->ne, m->p, m->mult, m->leaf_extent);
    if (!err.empty()) return set_error(c, RIGA_EINVAL, err);
    c->analyzed_only = true;
    return RIGA_OK;
}

namespace riga {
// c[e] = exp(c[e]): the coefficient map of the log-coefficient form
// K = sum_e exp(a_e) K_e, M = sum_e exp(b_e) M_e
__global__ void exp_inplace_kernel(long long n, double* __restrict__ v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = exp(v[i]);
}
}  // namespace riga

static int assemble_impl(riga_ctx* c, const riga_mesh* m, const double* coefK, const double* coefM, bool logs);

int riga_assemble(riga_ctx* c, const riga_mesh* m, const double* coefK, const double* coefM) {
    return assemble_impl(c, m, coefK, coefM, false);
}

int riga_assemble_log(riga_ctx* c, const riga_mesh* m, const double* logK, const double* logM) {
    return assemble_impl(c, m, logK, logM, true);
}

static int assemble_impl(riga_ctx* c, const riga_mesh* m, const double* coefK, const double* coefM, bool logs) {
    if (!c || !m) return RIGA_EINVAL;
    c->last_error.clear();
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    cudaSetDevice(c->device);
    {
        int rc0 = check_mesh(c, m);
        if (rc0) return rc0;
    }
    c->analyzed_only = false;
    c->assembled = false;
    c->factored = false;
    c->nev = 0;
    std::vector<int> key = mesh_key(m);
    if (key != c->mesh_key) {
        std::string err = build_symbolic(c->S, m->dim, m->ne, m->p, m->mult, m->leaf_extent);
        long long nchk = 0;
        if (err.empty()) err = check_bulk_copies(c->S, &nchk);  // every bulk copy aligned and in range
        if (!err.empty()) {
            c->mesh_key.clear();
            return set_error(c, RIGA_EINVAL, err);
        }
        int rc = upload_symbolic(c);
        if (rc) {
            c->mesh_key.clear();
            return rc;
        }
        c->mesh_key = key;
    }
    const long long ne_tot = c->S.n_elem;
    c->coefK.clear();
    c->coefM.clear();
    if (coefK) {
        c->coefK.resize(ne_tot);
        DevBuf<double> tmp;
        RIGA_CUDA_TRY(c, tmp.alloc(ne_tot));
        int rc = to_device(c, coefK, tmp.ptr, ne_tot);
        if (rc) return rc;
        if (logs && ne_tot > 0) {
            count_launch(c);
            exp_inplace_kernel<<<(unsigned)std::min<long long>((ne_tot + 255) / 256, 1024), 256, 0, c->stream>>>(ne_tot, tmp.ptr);
        }
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->coefK.data(), tmp.ptr, ne_tot * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    if (coefM) {
        c->coefM.resize(ne_tot);
        DevBuf<double> tmp;
        RIGA_CUDA_TRY(c, tmp.alloc(ne_tot));
        int rc = to_device(c, coefM, tmp.ptr, ne_tot);
        if (rc) return rc;
        if (logs && ne_tot > 0) {
            count_launch(c);
            exp_inplace_kernel<<<(unsigned)std::min<long long>((ne_tot + 255) / 256, 1024), 256, 0, c->stream>>>(ne_tot, tmp.ptr);
        }
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->coefM.data(), tmp.ptr, ne_tot * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (double v : c->coefK)
        if (!(v > 0.0) || !std::isfinite(v)) return set_error(c, RIGA_EINVAL, "coefK must be positive and finite");
    for (double v : c->coefM)
        if (!(v > 0.0) || !std::isfinite(v)) return set_error(c, RIGA_EINVAL, "coefM must be positive and finite");
    int rc = assemble_device(c);
    if (rc) return rc;
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->assembled = true;
    return RIGA_OK;
}

int riga_factor(riga_ctx* c, double sigma, int precision, long long* n_neg) {
    if (!c) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->assembled) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    if (precision != RIGA_FP64 && precision != RIGA_FP32 && precision != RIGA_TF32 && precision != RIGA_BF16)
        return set_error(c, RIGA_EINVAL, "unknown precision");
    if (!std::isfinite(sigma)) return set_error(c, RIGA_EINVAL, "sigma must be finite");
    c->sigma = sigma;
    c->sigma_prob.clear();
    c->precision = precision;
    c->factored = false;
    int rc = enqueue_factor(c);
    if (rc) return rc;
    rc = finish_factor(c);
    if (n_neg) *n_neg = c->inertia;
    return rc;
}

// Re-upload the factorization's level schedule (after build_schedule)
static int upload_schedule(riga_ctx* c) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    RIGA_CUDA_TRY(c, c->pitems.upload(S.pitems.empty() ? std::vector<PanelItem>{PanelItem{0, 0}} : S.pitems, st));
    RIGA_CUDA_TRY(c, c->titems.upload(S.titems.empty() ? std::vector<TileItem>{TileItem{0, 0, 0}} : S.titems, st));
    RIGA_CUDA_TRY(c, c->tcitems.upload(S.tc_tiles.empty() ? std::vector<TcTile>{TcTile{0, 0, 0, 0, 0, 0}} : S.tc_tiles, st));
    RIGA_CUDA_TRY(c, c->tcpacks.upload(S.tc_packs.empty() ? std::vector<TcPack>{TcPack{0, 0, 0, 0}} : S.tc_packs, st));
    RIGA_CUDA_TRY(c, c->tcnarrow.upload(S.tc_narrow.empty() ? std::vector<TileItemL>{TileItemL{0, 0, 0, 0}} : S.tc_narrow, st));
    RIGA_CUDA_TRY(c, c->ozpacks.upload(S.oz_packs.empty() ? std::vector<TcPack>{TcPack{0, 0, 0, 0}} : S.oz_packs, st));
    RIGA_CUDA_TRY(c, c->oztiles.upload(S.oz_tiles.empty() ? std::vector<TcTile>{TcTile{0, 0, 0, 0, 0, 0}} : S.oz_tiles, st));
    RIGA_CUDA_TRY(c, c->eitems.upload(S.eitems.empty() ? std::vector<ExtItem>{ExtItem{0, 0, 0}} : S.eitems, st));
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
    ++c->sched_gen;
    return RIGA_OK;
}

int riga_autotune(riga_ctx* c, int* small_trail_out, double* ms_out) {
    if (!c) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->assembled) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    static const int cand[6] = {0, 128, 256, 512, 1024, 4096};
    cudaEvent_t e0, e1;
    RIGA_CUDA_TRY(c, cudaEventCreate(&e0));
    RIGA_CUDA_TRY(c, cudaEventCreate(&e1));
    int best = c->S.small_trail;
    double best_ms = 1e300;
    int rc = RIGA_OK;
    for (int i = 0; i < 6 && rc == RIGA_OK; ++i) {
        c->S.small_trail = cand[i];
        build_schedule(c->S);
        rc = upload_schedule(c);
        std::vector<double> t3;
        for (int rep = 0; rep < 4 && rc == RIGA_OK; ++rep) {  // the first run also sizes the pools
            c->sigma = 0.0;
            c->sigma_prob.clear();
            c->precision = RIGA_FP64;
            c->inertia_only = false;
            c->factored = false;
            cudaEventRecord(e0, c->stream);
            rc = enqueue_factor(c);
            if (rc == RIGA_OK) {
                cudaEventRecord(e1, c->stream);
                rc = finish_factor(c);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                if (rep > 0) t3.push_back(t);
            }
        }
        std::sort(t3.begin(), t3.end());
        const double ms = t3.size() == 3 ? t3[1] : 1e300;  // median of three
        if (ms_out) ms_out[i] = ms;
        if (rc == RIGA_OK && ms < best_ms) {
            best_ms = ms;
            best = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->S.small_trail = best;
    build_schedule(c->S);
    const int rc2 = upload_schedule(c);
    if (small_trail_out) *small_trail_out = best;
    return rc ? rc : rc2;
}

int riga_solve(riga_ctx* c, const double* b, double* x, int nrhs, double tol, int* iters_out) {
    if (!c || !b || !x || nrhs < 1) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->factored) return set_error(c, RIGA_ESTATE, "riga_factor first");
    const long long N = c->S.N;
    const bool refine = (c->precision != RIGA_FP64) || tol > 0.0;
    // all columns in one buffer: one tree traversal carries up to four of them
    DevBuf<double> g, y;
    RIGA_CUDA_TRY(c, g.alloc((size_t)N * nrhs));
    RIGA_CUDA_TRY(c, y.alloc((size_t)N * nrhs));
    for (int i = 2; i < 4; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    int rc = to_device(c, b, g.ptr, (size_t)N * nrhs);
    if (rc) return rc;
    enqueue_permute(c, g.ptr, y.ptr, 1, nrhs);
    int status = RIGA_OK;
    if (!refine) {
        rc = enqueue_solve(c, y.ptr, nrhs);
        if (rc) return rc;
        if (iters_out) *iters_out = 1;
    } else {
        const double t = tol > 0.0 ? tol : 1e-13;
        for (int col = 0; col < nrhs; ++col) {
            int sweeps = 1;
            rc = solve_refined(c, y.ptr + (long long)col * N, c->vwork[2].ptr, c->vwork[3].ptr, t, 30, 1, &sweeps);
            if (rc == RIGA_EREFINE) status = rc;
            else if (rc) return rc;
            if (iters_out) *iters_out = sweeps;
        }
    }
    enqueue_permute(c, y.ptr, g.ptr, 0, nrhs);
    rc = to_user(c, g.ptr, x, (size_t)N * nrhs);
    if (rc) return rc;
    int dflag = 0;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(&dflag, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (dflag & 2) return set_error(c, RIGA_ETIMEOUT, "a dependency wait of the tree solve gave up");
    return status;
}

int riga_set_eig_options(riga_ctx* c, int slice, int precision, int max_steps, int extra, unsigned long long seed) {
    if (!c) return RIGA_EINVAL;
    if (slice < 0 || max_steps < 0 || extra < 0) return set_error(c, RIGA_EINVAL, "negative option");
    if (precision != RIGA_FP64 && precision != RIGA_FP32 && precision != RIGA_TF32 && precision != RIGA_BF16)
        return set_error(c, RIGA_EINVAL, "unknown precision");
    c->opt_slice = slice;
    c->opt_precision = precision;
    c->opt_max_steps = max_steps;
    c->opt_extra = extra;
    c->opt_seed = seed;
    return RIGA_OK;
}

int riga_set_eig_block(riga_ctx* c, int block) {
    if (!c) return RIGA_EINVAL;
    if (block != 0 && block != 1 && block != 2 && block != 4) return set_error(c, RIGA_EINVAL, "block size must be 0, 1, 2 or 4");
    c->opt_block = block;
    return RIGA_OK;
}

int riga_set_eig_accuracy(riga_ctx* c, int rayleigh) {
    if (!c) return RIGA_EINVAL;
    if (rayleigh != 0 && rayleigh != 1) return set_error(c, RIGA_EINVAL, "rayleigh must be 0 or 1");
    c->opt_rq = rayleigh;
    return RIGA_OK;
}

int riga_set_fp64_update(riga_ctx* c, int mode) {
    if (!c) return RIGA_EINVAL;
    if (mode != 0 && mode != 1) return set_error(c, RIGA_EINVAL, "mode must be 0 (CUDA cores) or 1 (tensor cores)");
    c->fp64_tc = mode;
    return RIGA_OK;
}

int riga_set_reorth(riga_ctx* c, int passes) {
    if (!c) return RIGA_EINVAL;
    if (passes != 1 && passes != 2) return set_error(c, RIGA_EINVAL, "passes must be 1 or 2");
    c->opt_reorth = passes;
    return RIGA_OK;
}

// eigenvalues, residuals rho_i = ||K u - lambda M u|| / (|lambda| ||M u||) and
// eigenvectors (global numbering, sign convention) of the got pairs held in
// c->evals / c->evec_perm, to user arrays (host or device)
static int emit_eigs(riga_ctx* c, int got, double* evals, double* evecs, double* resid) {
    const long long N = c->S.N;
    if (got > 0) {
        if (is_device_ptr(evals)) {
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(evals, c->evals.data(), got * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        } else {
            std::memcpy(evals, c->evals.data(), got * sizeof(double));
        }
    }
    if (resid && got > 0) {
        std::vector<double> rh(got);
        RIGA_CUDA_TRY(c, c->vwork[4].alloc(N));
        RIGA_CUDA_TRY(c, c->vwork[5].alloc(N));
        RIGA_CUDA_TRY(c, c->red.alloc(2 * 304));
        std::vector<double> part(2 * 152);
        for (int q = 0; q < got; ++q) {
            const double* u = c->evec_perm.ptr + (long long)q * N;
            enqueue_spmv(c, 1, u, c->vwork[4].ptr, 0.0);
            enqueue_spmv(c, 0, u, c->vwork[5].ptr, 0.0);
            c->stats.n_matvec--;  // reporting, not part of the iteration count
            { count_launch(c); resid_partial_kernel<<<152, 256, 0, c->stream>>>(N, c->vwork[4].ptr, c->vwork[5].ptr, c->evals[q], c->red.ptr); }
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(part.data(), c->red.ptr, 2 * 152 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            double ra = 0.0, rb = 0.0;
            for (int i = 0; i < 152; ++i) {
                ra += part[2 * i];
                rb += part[2 * i + 1];
            }
            rh[q] = std::sqrt(ra) / (std::fabs(c->evals[q]) * std::sqrt(rb));
        }
        if (is_device_ptr(resid)) {
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(resid, rh.data(), got * sizeof(double), cudaMemcpyHostToDevice, c->stream));
            RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        } else {
            std::memcpy(resid, rh.data(), got * sizeof(double));
        }
    }
    if (evecs && got > 0) {
        DevBuf<double> tmp;
        RIGA_CUDA_TRY(c, tmp.alloc((size_t)N * got));
        enqueue_permute(c, c->evec_perm.ptr, tmp.ptr, 0, got);
        sign_fix(c, tmp.ptr, got);
        int r2 = to_user(c, tmp.ptr, evecs, (size_t)N * got);
        if (r2) return r2;
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    RIGA_CUDA_TRY(c, cudaGetLastError());
    return RIGA_OK;
}

int riga_eigs(riga_ctx* c, int k, double sigma, double tol, double* evals, double* evecs, double* resid, int* nconv) {
    if (!c || !evals) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->assembled) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    if (c->S.dim == 0) return set_error(c, RIGA_ESTATE, "a batch context: use riga_eigs_batch");
    if (!(tol > 0.0)) return set_error(c, RIGA_EINVAL, "tol must be positive");
    if (!std::isfinite(sigma)) return set_error(c, RIGA_EINVAL, "sigma must be finite");
    int got = 0;
    int status = run_eigs(c, k, sigma, tol, &got);
    if (nconv) *nconv = got;
    if (status != RIGA_OK && status != RIGA_ENOCONV) return status;
    int rc = emit_eigs(c, got, evals, evecs, resid);
    return rc ? rc : status;
}

int riga_eigs_interval(riga_ctx* c, double lo, double hi, int kmax, double tol, int m_basis, double* evals,
                       double* evecs, double* resid, int* nfound, int* basis_cols) {
    if (!c || !evals || !nfound || kmax < 0) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->assembled) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    if (c->S.dim == 0) return set_error(c, RIGA_ESTATE, "a batch context: use riga_eigs_batch");
    if (!(tol > 0.0)) return set_error(c, RIGA_EINVAL, "tol must be positive");
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi)) return set_error(c, RIGA_EINVAL, "need finite lo < hi");
    if (m_basis < 0 || m_basis == 1 || m_basis == 2) return set_error(c, RIGA_EINVAL, "m_basis must be 0 or >= 3");
    int got = 0;
    int status = run_eigs_interval(c, lo, hi, kmax, tol, m_basis, &got, basis_cols);
    *nfound = got;
    if (status == RIGA_EINVAL) return status;  // more eigenvalues than kmax: *nfound holds the count
    if (status != RIGA_OK && status != RIGA_ENOCONV) return status;
    int rc = emit_eigs(c, got, evals, evecs, resid);
    return rc ? rc : status;
}

int riga_eig_errors(riga_ctx* c, int nev, const int* modes, int nq, double* everr, double* eferr_l2, double* eferr_e) {
    if (!c || !modes || !everr || !eferr_l2 || !eferr_e || nev < 1 || nq < 0) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (c->S.dim == 0) return set_error(c, RIGA_ESTATE, "a batch context");
    if (c->nev < 1) return set_error(c, RIGA_ESTATE, "riga_eigs or riga_eigs_interval first");
    if (nev > c->nev) return set_error(c, RIGA_EINVAL, "nev exceeds the computed eigenpairs");
    return eig_errors_device(c, nev, modes, nq, everr, eferr_l2, eferr_e);
}

int riga_eig_grad(riga_ctx* c, int k, const double* dL, double* grad_a, double* grad_b) {
    if (!c || !dL || k < 1) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (c->nev < 1) return set_error(c, RIGA_ESTATE, "riga_eigs first");
    if (k > c->nev) return set_error(c, RIGA_EINVAL, "k exceeds the computed eigenpairs");
    const long long ne = c->S.n_elem;
    DevBuf<double> w, ga, gb;
    RIGA_CUDA_TRY(c, w.alloc(k));
    RIGA_CUDA_TRY(c, ga.alloc(ne));
    RIGA_CUDA_TRY(c, gb.alloc(ne));
    int rc = to_device(c, dL, w.ptr, k);
    if (rc) return rc;
    rc = eig_grad_device(c, k, w.ptr, ga.ptr, gb.ptr);
    if (rc) return rc;
    if (grad_a) {
        rc = to_user(c, ga.ptr, grad_a, ne);
        if (rc) return rc;
    }
    if (grad_b) {
        rc = to_user(c, gb.ptr, grad_b, ne);
        if (rc) return rc;
    }
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RIGA_OK;
}

int riga_query(riga_ctx* c, long long* N, long long* nnz, long long* nnzL, double* flops) {
    if (!c) return RIGA_EINVAL;
    if (c->mesh_key.empty() && !c->analyzed_only) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    if (N) *N = c->S.N;
    if (nnz) *nnz = c->S.nnz;
    if (nnzL) *nnzL = c->S.nnzL;
    if (flops) *flops = c->S.flops;
    return RIGA_OK;
}

int riga_get_symbolic(riga_ctx* c, int* n_nodes, long long* total_idx, int* perm, int* node_ptr, int* parent,
                      long long* front_ptr, int* front_idx) {
    if (!c) return RIGA_EINVAL;
    if (c->mesh_key.empty() && !c->analyzed_only) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    const Symbolic& S = c->S;
    if (n_nodes) *n_nodes = S.n_nodes;
    if (total_idx) *total_idx = (long long)S.front_pos.size();
    if (perm) std::memcpy(perm, S.perm.data(), S.perm.size() * sizeof(int));
    if (node_ptr) std::memcpy(node_ptr, S.node_ptr.data(), S.node_ptr.size() * sizeof(int));
    if (parent) std::memcpy(parent, S.parent.data(), S.parent.size() * sizeof(int));
    if (front_ptr) std::memcpy(front_ptr, S.front_ptr.data(), S.front_ptr.size() * sizeof(long long));
    if (front_idx)
        for (size_t i = 0; i < S.front_pos.size(); ++i) front_idx[i] = S.perm[S.front_pos[i]];
    return RIGA_OK;
}

int riga_get_matrices(riga_ctx* c, long long* row_ptr, int* col, double* kval, double* mval) {
    if (!c) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->assembled) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    const Symbolic& S = c->S;
    if (row_ptr) {
        DevBuf<long long> t;
        RIGA_CUDA_TRY(c, t.alloc(S.N + 1));
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(t.ptr, S.glob_rowptr.data(), (S.N + 1) * sizeof(long long), cudaMemcpyHostToDevice, c->stream));
        int rc = to_user(c, t.ptr, row_ptr, S.N + 1);
        if (rc) return rc;
    }
    if (col) {
        DevBuf<int> t;
        RIGA_CUDA_TRY(c, t.alloc(S.nnz));
        { count_launch(c); glob_col_kernel<<<(unsigned)((S.N + 255) / 256), 256, 0, c->stream>>>(S.N, c->rowptr.ptr, c->col.ptr, c->perm.ptr,
                                                                             c->perm_to_glob.ptr, t.ptr); }
        int rc = to_user(c, t.ptr, col, S.nnz);
        if (rc) return rc;
    }
    const double* srcs[2] = {c->Kval.ptr, c->Mval.ptr};
    double* dsts[2] = {kval, mval};
    for (int i = 0; i < 2; ++i) {
        if (!dsts[i]) continue;
        DevBuf<double> t;
        RIGA_CUDA_TRY(c, t.alloc(S.nnz));
        { count_launch(c); scatter_glob_kernel<<<(unsigned)((S.nnz + 255) / 256), 256, 0, c->stream>>>(S.nnz, c->perm_to_glob.ptr, srcs[i], t.ptr); }
        int rc = to_user(c, t.ptr, dsts[i], S.nnz);
        if (rc) return rc;
    }
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RIGA_OK;
}

int riga_get_factor(riga_ctx* c, double* D, long long* Lptr, double* L) {
    if (!c) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->factored) return set_error(c, RIGA_ESTATE, "riga_factor first");
    const Symbolic& S = c->S;
    if (Lptr) {
        long long at = 0;
        for (int f = 0; f < S.n_nodes; ++f) {
            Lptr[f] = at;
            at += (long long)S.n[f] * S.k[f];
        }
        Lptr[S.n_nodes] = at;
    }
    if (D) RIGA_CUDA_TRY(c, cudaMemcpy(D, c->D.ptr, S.N * sizeof(double), cudaMemcpyDeviceToHost));
    if (L) {
        long long at = 0;
        for (int f = 0; f < S.n_nodes; ++f) {
            // first k columns, rows 0..n-1 of the augmented front (leading dimension n + k)
            const long long n = S.n[f], k = S.k[f], ld = S.ld[f];
            const long long cnt = n * k;
            if (c->precision == RIGA_FP64) {
                RIGA_CUDA_TRY(c, cudaMemcpy2D(L + at, n * sizeof(double), c->pool64.ptr + S.front_off[f], ld * sizeof(double),
                                              n * sizeof(double), k, cudaMemcpyDeviceToHost));
            } else {
                std::vector<float> tmp(cnt);
                RIGA_CUDA_TRY(c, cudaMemcpy2D(tmp.data(), n * sizeof(float), c->pool32.ptr + S.front_off[f], ld * sizeof(float),
                                              n * sizeof(float), k, cudaMemcpyDeviceToHost));
                for (long long i = 0; i < cnt; ++i) L[at + i] = tmp[i];
            }
            at += cnt;
        }
    }
    return RIGA_OK;
}

int riga_spmv(riga_ctx* c, int which, const double* x, double* y) {
    if (!c || !x || !y) return RIGA_EINVAL;
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    c->last_error.clear();
    cudaSetDevice(c->device);
    if (!c->assembled) return set_error(c, RIGA_ESTATE, "riga_assemble first");
    if (which < 0 || which > 2) return set_error(c, RIGA_EINVAL, "which must be 0 (M), 1 (K) or 2 (K - sigma M)");
    const long long N = c->S.N;
    for (int i = 0; i < 3; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    int rc = to_device(c, x, c->vwork[0].ptr, N);
    if (rc) return rc;
    enqueue_permute(c, c->vwork[0].ptr, c->vwork[1].ptr, 1, 1);
    rc = enqueue_spmv(c, which, c->vwork[1].ptr, c->vwork[2].ptr, c->sigma);
    if (rc) return rc;
    enqueue_permute(c, c->vwork[2].ptr, c->vwork[0].ptr, 0, 1);
    rc = to_user(c, c->vwork[0].ptr, y, N);
    if (rc) return rc;
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return RIGA_OK;
}

int riga_stats(riga_ctx* c, long long* n_fact, long long* n_solve, long long* n_matvec, long long* steps,
               double* t_fact_ms, double* t_lanczos_ms) {
    if (!c) return RIGA_EINVAL;
    if (n_fact) *n_fact = c->stats.n_fact;
    if (n_solve) *n_solve = c->stats.n_solve;
    if (n_matvec) *n_matvec = c->stats.n_matvec;
    if (steps) *steps = c->stats.steps;
    if (t_fact_ms) *t_fact_ms = c->stats.t_fact_ms;
    if (t_lanczos_ms) *t_lanczos_ms = c->stats.t_lanczos_ms;
    return RIGA_OK;
}

static void resolve_profile(riga_ctx* c) {
    if (c->device >= 0) cudaStreamSynchronize(c->stream);
    for (int p = 0; p < PH_COUNT; ++p) {
        PhaseRec& r = c->prof.ph[p];
        for (auto& e : r.ev) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) r.ms += ms;
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        r.ev.clear();
    }
    cudaGetLastError();
}

int riga_profile(riga_ctx* c, int enable) {
    if (!c) return RIGA_EINVAL;
    resolve_profile(c);
    for (int p = 0; p < PH_COUNT; ++p) c->prof.ph[p] = PhaseRec();
    c->prof.on = enable != 0;
    return RIGA_OK;
}

int riga_profile_get(riga_ctx* c, int phase, const char** name, long long* launches, long long* calls, double* ms,
                     double* bytes, double* flops) {
    static const char* names[PH_COUNT] = {"assemble", "factor", "solve", "reorth", "spmv", "ritz", "other"};
    if (!c) return RIGA_EINVAL;
    if (phase == -1) {
        if (name) *name = "total";
        if (launches) *launches = c->prof.launches;
        return RIGA_OK;
    }
    if (phase < 0 || phase >= PH_COUNT) return set_error(c, RIGA_EINVAL, "phase out of range");
    resolve_profile(c);
    const PhaseRec& r = c->prof.ph[phase];
    if (name) *name = names[phase];
    if (launches) *launches = r.launches;
    if (calls) *calls = r.calls;
    if (ms) *ms = r.ms;
    if (bytes) *bytes = r.bytes;
    if (flops) *flops = r.flops;
    return RIGA_OK;
}

int riga_set_wait_limit(riga_ctx* c, long long limit) {
    if (!c || limit < 0) return RIGA_EINVAL;
    c->wait_limit = limit;
    return RIGA_OK;
}

int riga_check_copies(riga_ctx* c, long long* n_checked) {
    if (!c || !n_checked) return RIGA_EINVAL;
    c->last_error.clear();
    if (c->S.N <= 0) return set_error(c, RIGA_ESTATE, "riga_analyze or riga_assemble first");
    std::string err = check_bulk_copies(c->S, n_checked);
    if (!err.empty()) return set_error(c, RIGA_EINVAL, err);
    return RIGA_OK;
}

int riga_trace_solve(riga_ctx* c, const double* b, int* n_items, long long* trace, int* order) {
    if (!c || !b || !n_items) return RIGA_EINVAL;
    c->last_error.clear();
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    cudaSetDevice(c->device);
    if (!c->factored) return set_error(c, RIGA_ESTATE, "riga_factor first");
    const Symbolic& S = c->S;
    *n_items = (int)S.sitems.size();
    if (!trace) return RIGA_OK;
    const long long N = S.N;
    const size_t nt = 4 * S.sitems.size();
    DevBuf<long long> tb;
    RIGA_CUDA_TRY(c, tb.alloc(nt));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(tb.ptr, 0, nt * sizeof(long long), c->stream));
    for (int i = 0; i < 2; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    int rc = to_device(c, b, c->vwork[0].ptr, N);
    if (rc) return rc;
    enqueue_permute(c, c->vwork[0].ptr, c->vwork[1].ptr, 1, 1);
    c->trace_buf = tb.ptr;
    rc = enqueue_solve(c, c->vwork[1].ptr);
    c->trace_buf = nullptr;
    if (rc) return rc;
    int dflag = 0;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(trace, tb.ptr, nt * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(&dflag, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (order) RIGA_CUDA_TRY(c, cudaMemcpyAsync(order, c->solve_order.ptr, S.sitems.size() * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (dflag & 2) return set_error(c, RIGA_ETIMEOUT, "a dependency wait of the tree solve gave up");
    return RIGA_OK;
}

}  // extern "C"
