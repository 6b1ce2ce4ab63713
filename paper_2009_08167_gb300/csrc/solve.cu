// Forward/backward elimination with the multifrontal factor and FP64 SpMV
// (Sec. 4.2: one f/b elimination and the M mat-vecs per Lanczos step;
// Sec. 5.1 Eq. flopsFb).  Vectors are in elimination order.
//
// fwd_kernel (one CTA per front of a level, leaves to root): the front's
//   local vector w = [b(own); 0] plus the children's update vectors, then
//   L11 z = w(own) by 32-column blocks (warp-shuffle triangle + row updates
//   of every row below), w(border) -= L21 z.  z goes back to the vector, the
//   border part becomes this front's update vector for its parent.
// bwd_kernel (root to leaves): x(own) = L11^{-T} (D^{-1} z - L21^T x(border))
//   by 32-column blocks (warp-per-column dot products + warp-shuffle
//   triangle); x(border) belongs to ancestors and is already final.
// Both read every factor entry exactly once per solve.
#include "ctx.h"

namespace riga {

template <typename T>
__global__ void __launch_bounds__(256) fwd_kernel(const int* __restrict__ nodes, const T* __restrict__ pool,
                                                  const long long* __restrict__ front_off,
                                                  const int* __restrict__ node_ptr, const int* __restrict__ kk,
                                                  const int* __restrict__ nn, const int* __restrict__ child_ptr,
                                                  const int* __restrict__ child_list, const int* __restrict__ rel,
                                                  const long long* __restrict__ rel_ptr,
                                                  const long long* __restrict__ upd_off, double* __restrict__ upd,
                                                  double* __restrict__ y) {
    extern __shared__ unsigned char smem_raw[];
    T* w = reinterpret_cast<T*>(smem_raw);
    const int F = nodes[blockIdx.x];
    const int k = kk[F], n = nn[F], b0 = node_ptr[F];
    const T* L = pool + front_off[F];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n; i += blockDim.x) w[i] = (i < k) ? (T)y[b0 + i] : T(0);
    __syncthreads();
    for (int ci = child_ptr[F]; ci < child_ptr[F + 1]; ++ci) {
        const int c = child_list[ci];
        const int m = nn[c] - kk[c];
        const int* r = rel + rel_ptr[c];
        const double* u = upd + upd_off[c];
        for (int i = tid; i < m; i += blockDim.x) w[r[i]] += (T)u[i];
        __syncthreads();
    }
    for (int jb = 0; jb < k; jb += 32) {
        const int kb = min(32, k - jb);
        if (warp == 0) {
            T v = (lane < kb) ? w[jb + lane] : T(0);
            for (int u = 0; u < kb; ++u) {
                T zu = __shfl_sync(0xffffffffu, v, u);
                if (lane > u && lane < kb) v -= L[(long long)(jb + u) * n + jb + lane] * zu;
            }
            if (lane < kb) w[jb + lane] = v;
        }
        __syncthreads();
        for (int i = jb + kb + tid; i < n; i += blockDim.x) {
            T acc = w[i];
            for (int u = 0; u < kb; ++u) acc -= L[(long long)(jb + u) * n + i] * w[jb + u];
            w[i] = acc;
        }
        __syncthreads();
    }
    for (int i = tid; i < n; i += blockDim.x) {
        if (i < k) y[b0 + i] = (double)w[i];
        else upd[upd_off[F] + i - k] = (double)w[i];
    }
    (void)warp;
}

template <typename T>
__global__ void __launch_bounds__(256) bwd_kernel(const int* __restrict__ nodes, const T* __restrict__ pool,
                                                  const long long* __restrict__ front_off,
                                                  const int* __restrict__ node_ptr, const int* __restrict__ kk,
                                                  const int* __restrict__ nn, const long long* __restrict__ front_ptr,
                                                  const int* __restrict__ front_pos, const double* __restrict__ D,
                                                  double* __restrict__ y) {
    extern __shared__ unsigned char smem_raw[];
    T* w = reinterpret_cast<T*>(smem_raw);
    const int F = nodes[blockIdx.x];
    const int k = kk[F], n = nn[F], b0 = node_ptr[F];
    const T* L = pool + front_off[F];
    const int* idx = front_pos + front_ptr[F];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    for (int i = tid; i < n; i += blockDim.x) w[i] = (i < k) ? (T)(y[b0 + i] / D[b0 + i]) : (T)y[idx[i]];
    __syncthreads();
    const int last = ((k - 1) / 32) * 32;
    for (int jb = last; jb >= 0; jb -= 32) {
        const int kb = min(32, k - jb);
        for (int j = jb + warp; j < jb + kb; j += nwarp) {
            T s = T(0);
            const T* Lc = L + (long long)j * n;
            for (int i = jb + kb + lane; i < n; i += 32) s += Lc[i] * w[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) w[j] -= s;
        }
        __syncthreads();
        if (warp == 0) {
            T v = (lane < kb) ? w[jb + lane] : T(0);
            for (int u = kb - 1; u >= 0; --u) {
                T xu = __shfl_sync(0xffffffffu, v, u);
                if (lane < u) v -= L[(long long)(jb + lane) * n + jb + u] * xu;
            }
            if (lane < kb) w[jb + lane] = v;
        }
        __syncthreads();
    }
    for (int i = tid; i < k; i += blockDim.x) y[b0 + i] = (double)w[i];
}

// y = (A1 - shift A2) x over the permuted CSR, `lanes` threads per row.
// which: 0 -> M, 1 -> K, 2 -> K - shift M.
template <int LANES>
__global__ void spmv_kernel(long long N, const long long* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ Kv, const double* __restrict__ Mv, int which, double shift,
                            const double* __restrict__ x, double* __restrict__ y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = t / LANES;
    const int lane = (int)(t % LANES);
    if (row >= N) return;
    double s = 0.0;
    for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += LANES) {
        double a = which == 0 ? Mv[e] : (which == 1 ? Kv[e] : Kv[e] - shift * Mv[e]);
        s += a * x[col[e]];
    }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);
    if (lane == 0) y[row] = s;
}

// r = b - (K - shift M) x
__global__ void residual_kernel(long long N, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ Kv, const double* __restrict__ Mv, double shift,
                                const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ r) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = t / 16;
    const int lane = (int)(t % 16);
    if (row >= N) return;
    double s = 0.0;
    for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += 16) s += (Kv[e] - shift * Mv[e]) * x[col[e]];
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, 16);
    if (lane == 0) r[row] = b[row] - s;
}

// out[ipos] <-> in[g]: to_perm: out[pos] = in[perm[pos]]; else out[perm[pos]] = in[pos]
__global__ void permute_kernel(long long N, int ncols, const int* __restrict__ perm, const double* __restrict__ in,
                               double* __restrict__ out, int to_perm) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * ncols) return;
    long long col = t / N, pos = t % N;
    long long g = perm[pos];
    if (to_perm) out[col * N + pos] = in[col * N + g];
    else out[col * N + g] = in[col * N + pos];
}

__global__ void axpy_kernel(long long N, double a, const double* __restrict__ x, double* __restrict__ y) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] += a * x[i];
}

// partial sums of squares of two vectors (deterministic two-level reduction)
__global__ void norm2_partial_kernel(long long N, const double* __restrict__ a, const double* __restrict__ b,
                                     double* __restrict__ partial) {
    __shared__ double sa[8], sb[8];
    double xa = 0.0, xb = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        xa += a[i] * a[i];
        xb += b[i] * b[i];
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
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ta += sa[w];
            tb += sb[w];
        }
        partial[2 * blockIdx.x] = ta;
        partial[2 * blockIdx.x + 1] = tb;
    }
}

static size_t level_smem(const LevelPlan& P, size_t elt) { return (size_t)P.max_n * elt; }

template <typename T>
static int enqueue_solve_t(riga_ctx* c, const T* pool, double* y) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    // algorithmic bytes: every factor entry read twice (forward, backward),
    // the vector read and written in each sweep
    PhaseScope scope(c, PH_SOLVE, 2.0 * (double)S.nnzL * sizeof(T) + 4.0 * (double)S.N * sizeof(double));
    for (int l = 0; l < S.n_levels; ++l) {
        const LevelPlan& P = S.levels[l];
        size_t sm = level_smem(P, sizeof(T));
        { count_launch(c); fwd_kernel<T><<<(unsigned)P.nodes.size(), 256, sm, st>>>(
            c->level_nodes.ptr + c->level_nodes_off[l], pool, c->front_off.ptr, c->node_ptr.ptr, c->kk.ptr, c->nn.ptr,
            c->child_ptr.ptr, c->child_list.ptr, c->rel.ptr, c->rel_ptr.ptr, c->upd_off.ptr, c->upd.ptr, y); }
    }
    for (int l = S.n_levels - 1; l >= 0; --l) {
        const LevelPlan& P = S.levels[l];
        size_t sm = level_smem(P, sizeof(T));
        { count_launch(c); bwd_kernel<T><<<(unsigned)P.nodes.size(), 256, sm, st>>>(
            c->level_nodes.ptr + c->level_nodes_off[l], pool, c->front_off.ptr, c->node_ptr.ptr, c->kk.ptr, c->nn.ptr,
            c->front_ptr.ptr, c->front_pos.ptr, c->D.ptr, y); }
    }
    return RIGA_OK;
}

static int configure_smem(riga_ctx* c) {
    static int done_dev = -1;
    if (done_dev == c->device) return RIGA_OK;
    int maxopt = 0;
    RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(fwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxopt));
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxopt));
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxopt));
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxopt));
    done_dev = c->device;
    return RIGA_OK;
}

int enqueue_solve(riga_ctx* c, double* y) {
    if (!c->factored) return set_error(c, RIGA_ESTATE, "no factorization");
    int rc = configure_smem(c);
    if (rc) return rc;
    Symbolic& S = c->S;
    int maxopt = 0;
    cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    size_t elt = c->precision == RIGA_FP64 ? sizeof(double) : sizeof(float);
    for (const LevelPlan& P : S.levels)
        if (level_smem(P, elt) > (size_t)maxopt) return set_error(c, RIGA_EINVAL, "front too large for the shared-memory solve");
    RIGA_CUDA_TRY(c, c->upd.alloc(S.upd_size > 0 ? S.upd_size : 1));
    if (c->precision == RIGA_FP64) rc = enqueue_solve_t<double>(c, c->pool64.ptr, y);
    else rc = enqueue_solve_t<float>(c, c->pool32.ptr, y);
    if (rc) return rc;
    RIGA_CUDA_TRY(c, cudaGetLastError());
    c->stats.n_solve++;
    return RIGA_OK;
}

int enqueue_spmv(riga_ctx* c, int which, const double* x, double* y, double shift) {
    Symbolic& S = c->S;
    long long threads = S.N * 16;
    { count_launch(c); spmv_kernel<16><<<(unsigned)((threads + 255) / 256), 256, 0, c->stream>>>(S.N, c->rowptr.ptr, c->col.ptr,
                                                                               c->Kval.ptr, c->Mval.ptr, which, shift,
                                                                               x, y); }
    RIGA_CUDA_TRY(c, cudaGetLastError());
    if (which == 0) c->stats.n_matvec++;
    return RIGA_OK;
}

void enqueue_permute(riga_ctx* c, const double* in, double* out, int to_perm, int ncols) {
    long long t = c->S.N * ncols;
    { count_launch(c); permute_kernel<<<(unsigned)((t + 255) / 256), 256, 0, c->stream>>>(c->S.N, ncols, c->perm.ptr, in, out, to_perm); }
}

// y := (K - sigma M)^{-1} y (permuted order).  With an FP32 factor, or check
// set, refines: x = 0, r = y; repeat d = solve(r); x += d; r = y - A x.
// check: read ||r|| / ||y|| back after each sweep and stop at tol.
int solve_refined(riga_ctx* c, double* y, double* x, double* r, double tol, int max_sweeps, int check,
                  int* sweeps_out) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    const long long N = S.N;
    const unsigned gb = (unsigned)((N + 255) / 256);
    if (c->precision == RIGA_FP64 && !check) {
        if (sweeps_out) *sweeps_out = 1;
        return enqueue_solve(c, y);
    }
    RIGA_CUDA_TRY(c, c->red.alloc(2 * 304));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(x, 0, N * sizeof(double), st));
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(r, y, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double bnorm = -1.0, best = 1e300;
    int sweeps = 0;
    int status = RIGA_OK;
    std::vector<double> part(2 * 304);
    for (sweeps = 1; sweeps <= max_sweeps; ++sweeps) {
        int rc = enqueue_solve(c, r);  // r := A^{-1} r (correction)
        if (rc) return rc;
        { count_launch(c); axpy_kernel<<<gb, 256, 0, st>>>(N, 1.0, r, x); }
        long long threads = N * 16;
        { count_launch(c); residual_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(N, c->rowptr.ptr, c->col.ptr, c->Kval.ptr,
                                                                            c->Mval.ptr, c->sigma, x, y, r); }
        if (check) {
            { count_launch(c); norm2_partial_kernel<<<304, 256, 0, st>>>(N, r, y, c->red.ptr); }
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(part.data(), c->red.ptr, 2 * 304 * sizeof(double), cudaMemcpyDeviceToHost, st));
            RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
            double rn = 0.0, bn = 0.0;
            for (int i = 0; i < 304; ++i) {
                rn += part[2 * i];
                bn += part[2 * i + 1];
            }
            rn = sqrt(rn);
            bn = sqrt(bn);
            bnorm = bn;
            if (rn <= tol * bnorm) break;
            if (rn >= 0.5 * best && sweeps > 2) {
                status = RIGA_EREFINE;
                break;
            }
            best = rn < best ? rn : best;
        }
    }
    if (sweeps > max_sweeps) {
        sweeps = max_sweeps;
        if (check) status = RIGA_EREFINE;
    }
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(y, x, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (sweeps_out) *sweeps_out = sweeps;
    if (status) return set_error(c, status, "iterative refinement did not reach the tolerance");
    return RIGA_OK;
}

}  // namespace riga
