// Multifrontal LDL^T of A = K - sigma M (Sec. 4.2 and its Remark on inertia),
// fronts in FP64 or FP32, 1x1 pivots without pivoting.
//
// The fronts live side by side in one pool (column-major, lower triangle
// used).  Each front is augmented by k_F extra rows coupled to its own
// variables by the identity (ld_F = n_F + k_F rows): after the own block is
// eliminated, the extra rows' Schur complement holds -A11^{-1} A12 and
// -A11^{-1}, the operators of the GEMV-only tree solve (solve.cu); the
// regular rows, D and the inertia are those of the plain factorization.
// Per assembly-tree level, leaves to root:
//   extend_add_kernel  children's Schur complements into the parents
//                      (child rank 0, then rank 1: deterministic, no atomics);
//   for each panel step s (panel columns [s*nb, s*nb+kb)):
//     diag_kernel      LDL^T of the kb x kb diagonal block in shared memory,
//                      pivots to D and the front diagonal, breakdown flag;
//     trsm_kernel      L21 = A21 L11^{-T} D^{-1}, one thread per row;
//     update_kernel    A22 -= L21 D L21^T on 32x32 (16x16) lower tiles of the
//                      trailing matrix (remaining fully summed part and the
//                      Schur complement); with tensor-core fronts only the
//                      columns of the panel's super-panel, the rest once per
//                      super-panel in tc_update.cu.
// All items of one launch span every front of the level.  The original
// entries are scattered into all fronts once, before the first level.
#include "ctx.h"

namespace riga {

constexpr int NB = 32;    // panel width
constexpr int TILE = 32;  // update tile
constexpr int RB = 64;    // TRSM rows per block

template <typename T>
__global__ void scatter_kernel(long long nnz, const long long* __restrict__ scatter, const double* __restrict__ K,
                               const double* __restrict__ M, double sigma, T* __restrict__ pool) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    long long off = scatter[e];
    if (off >= 0) pool[off] = (T)(K[e] - sigma * M[e]);
}

// batch: per-position shifts (each problem of the forest has its own sigma);
// one warp per row, entry (i, j) with j <= i shares row i's problem
template <typename T>
__global__ void scatter_rows_kernel(long long N, const long long* __restrict__ rowptr,
                                    const long long* __restrict__ scatter, const double* __restrict__ K,
                                    const double* __restrict__ M, const double* __restrict__ sig_pos,
                                    T* __restrict__ pool) {
    const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    const double sg = sig_pos[row];
    for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) {
        const long long off = scatter[e];
        if (off >= 0) pool[off] = (T)(K[e] - sg * M[e]);
    }
}

// batch: negative pivots per problem
__global__ void inertia_prob_kernel(long long N, const double* __restrict__ D, const int* __restrict__ prob,
                                    long long* __restrict__ neg) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        if (D[i] < 0.0) atomicAdd((unsigned long long*)&neg[prob[i]], 1ULL);
}

template <typename T>
__global__ void identity_kernel(int F, const int* __restrict__ kk, const int* __restrict__ nn,
                                const long long* __restrict__ front_off, T* __restrict__ pool) {
    const int f = blockIdx.x;
    if (f >= F) return;
    const int k = kk[f], n = nn[f], ld = n + k;
    T* A = pool + front_off[f];
    for (int r = threadIdx.x; r < k; r += blockDim.x) A[(long long)r * ld + n + r] = T(1);
}

template <typename T>
__global__ void extend_add_kernel(const ExtItem* __restrict__ items, const int* __restrict__ parent,
                                  const long long* __restrict__ front_off, const int* __restrict__ kk,
                                  const int* __restrict__ nn, const int* __restrict__ rel,
                                  const long long* __restrict__ rel_ptr, T* __restrict__ pool) {
    const ExtItem it = items[blockIdx.x];
    const int c = it.child, P = parent[c];
    const int kc = kk[c], nc = nn[c], ldc = nc + kc, ldp = nn[P] + kk[P];
    const int m = nc - kc;
    const T* src = pool + front_off[c] + (long long)kc * ldc + kc;
    T* dst = pool + front_off[P];
    const int* r = rel + rel_ptr[c];
    for (int j = it.c0; j < it.c1; ++j) {
        const long long cj = (long long)r[j] * ldp;
        for (int i = j + threadIdx.x; i < m; i += blockDim.x) dst[cj + r[i]] += src[(long long)j * ldc + i];
    }
}

// LDL^T of one kb x kb diagonal block per front (block of 128 threads).
// Column j stays unscaled while it updates the columns to its right (with
// the reciprocal pivot, one division per column); the columns are scaled by
// their reciprocal pivots when the block is written back.
template <typename T>
__global__ void __launch_bounds__(128) diag_kernel(const PanelItem* __restrict__ items, const int* __restrict__ kk,
                                                   const int* __restrict__ nn, const long long* __restrict__ front_off,
                                                   const int* __restrict__ node_ptr, T* __restrict__ pool,
                                                   double* __restrict__ D, int* __restrict__ flag) {
    __shared__ T Ls[NB][NB + 1];
    __shared__ T inv[NB];
    const PanelItem it = items[blockIdx.x];
    const int F = it.front, k = kk[F], ld = nn[F] + k, j0 = it.r0;
    const int kb = min(NB, k - j0);
    T* A = pool + front_off[F];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, cc = idx / kb;
        Ls[r][cc] = (r >= cc) ? A[(long long)(j0 + cc) * ld + j0 + r] : T(0);
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
        if (threadIdx.x == 0) {
            const T d = Ls[j][j];
            if (!(d != T(0) && isfinite((double)d))) atomicOr(flag, 1);
            inv[j] = T(1) / d;
        }
        __syncthreads();
        // a_rc -= a_rj (a_cj / d_j) over the lower triangle j < c <= r < kb
        const T ij = inv[j];
        const int m = kb - j - 1, tri = m * (m + 1) / 2;
        for (int idx = threadIdx.x; idx < tri; idx += blockDim.x) {
            int rr = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
            while ((rr + 1) * (rr + 2) / 2 <= idx) ++rr;
            while (rr * (rr + 1) / 2 > idx) --rr;
            const int r = j + 1 + rr, cc = j + 1 + idx - rr * (rr + 1) / 2;
            Ls[r][cc] -= Ls[r][j] * (Ls[cc][j] * ij);
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, cc = idx / kb;
        if (r > cc) A[(long long)(j0 + cc) * ld + j0 + r] = Ls[r][cc] * inv[cc];
        else if (r == cc) A[(long long)(j0 + cc) * ld + j0 + r] = Ls[r][r];
    }
    for (int t = threadIdx.x; t < kb; t += blockDim.x) D[node_ptr[F] + j0 + t] = (double)Ls[t][t];
}

// Rows r0..r0+RB-1 of the panel below the diagonal block (blockDim = RB):
// x_t = (a_t - sum_{u<t} x_u d_u l_tu) / d_t with the products d_u l_tu and
// the reciprocal pivots staged in shared memory.
template <typename T>
__global__ void trsm_kernel(const PanelItem* __restrict__ items, int j0, const int* __restrict__ kk,
                            const int* __restrict__ nn, const long long* __restrict__ front_off,
                            T* __restrict__ pool, int plain) {
    __shared__ T LD[NB][NB + 1];
    __shared__ T ds[NB], dinv[NB];
    const PanelItem it = items[blockIdx.x];
    const int F = it.front, k = kk[F], ld = nn[F] + k;
    const int rmax = plain ? nn[F] : ld;  // plain: skip the extra rows
    if (it.r0 >= rmax) return;
    const int kb = min(NB, k - j0);
    T* A = pool + front_off[F];
    for (int t = threadIdx.x; t < kb; t += blockDim.x) {
        const T d = A[(long long)(j0 + t) * ld + j0 + t];
        ds[t] = d;
        dinv[t] = T(1) / d;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, cc = idx / kb;
        if (r > cc) LD[r][cc] = A[(long long)(j0 + cc) * ld + j0 + r] * ds[cc];
    }
    __syncthreads();
    const int r = it.r0 + threadIdx.x;
    if (r >= rmax) return;
    T x[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t)
        if (t < kb) x[t] = A[(long long)(j0 + t) * ld + r];
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        if (t < kb) {
            T s = x[t];
#pragma unroll
            for (int u = 0; u < t; ++u) s -= x[u] * LD[t][u];
            x[t] = s * dinv[t];
        }
    }
#pragma unroll
    for (int t = 0; t < NB; ++t)
        if (t < kb) A[(long long)(j0 + t) * ld + r] = x[t];
}

// last column (exclusive) a tile may update: the front's end, or the tile's
// own limit (the end of the super-panel of a within-super-panel update)
__device__ __forceinline__ int tile_col_end(const TileItem&, int ld) { return ld; }
__device__ __forceinline__ int tile_col_end(const TileItemL& it, int ld) { return min(ld, it.jend); }

// C[i0:i0+TL, j0:j0+TL] -= L[:, panel] D L[:, panel]^T (64 threads, (TL/8)^2 each;
// TL = 32, or 16 on the small trailing blocks where 32x32 tiles pad too much)
template <typename T, int TL, typename Item = TileItem>
__global__ void __launch_bounds__(64) update_kernel(const Item* __restrict__ items, int p0,
                                                    const int* __restrict__ kk, const int* __restrict__ nn,
                                                    const long long* __restrict__ front_off,
                                                    const int* __restrict__ node_ptr, const double* __restrict__ D,
                                                    T* __restrict__ pool, int plain) {
    constexpr int R = TL / 8;  // rows and columns per thread
    __shared__ T As[NB][TL];
    __shared__ T Bs[NB][TL];
    const Item it = items[blockIdx.x];
    const int F = it.front, k = kk[F], n = nn[F], ld = n + k;
    if (plain && (it.i0 >= n || it.j0 >= n)) return;  // plain: tiles touching only extra rows
    const int kb = min(NB, k - p0);
    const int jend = tile_col_end(it, ld);
    T* A = pool + front_off[F];
    const double* d = D + node_ptr[F] + p0;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < NB * TL; idx += 64) {
        int rr = idx % TL, t = idx / TL;
        T a = T(0), b = T(0);
        if (t < kb) {
            int gi = it.i0 + rr, gj = it.j0 + rr;
            if (gi < ld) a = A[(long long)(p0 + t) * ld + gi];
            if (gj < ld) b = A[(long long)(p0 + t) * ld + gj] * (T)d[t];
        }
        As[t][rr] = a;
        Bs[t][rr] = b;
    }
    __syncthreads();
    const int tx = tid % 8, ty = tid / 8;
    T acc[R][R];
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
        for (int b = 0; b < R; ++b) acc[a][b] = T(0);
    for (int t = 0; t < kb; ++t) {
        T av[R], bv[R];
#pragma unroll
        for (int a = 0; a < R; ++a) av[a] = As[t][tx + 8 * a];
#pragma unroll
        for (int b = 0; b < R; ++b) bv[b] = Bs[t][ty + 8 * b];
#pragma unroll
        for (int a = 0; a < R; ++a)
#pragma unroll
            for (int b = 0; b < R; ++b) acc[a][b] += av[a] * bv[b];
    }
#pragma unroll
    for (int b = 0; b < R; ++b) {
        int gj = it.j0 + ty + 8 * b;
        if (gj >= jend) continue;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            int gi = it.i0 + tx + 8 * a;
            // lower triangle, plus the whole extra x extra block
            if (gi < ld && (gi >= gj || (gi >= n && gj >= n)) && !(plain && gi >= n)) A[(long long)gj * ld + gi] -= acc[a][b];
        }
    }
}

// Packs the solve operators from the extra rows E (rows n..n+k of the
// augmented front) into the panels of the solve items:
//   forward item  (columns [lo,hi) of k..n): row-major k x ldp, P[r*ldp + j-lo] = E[r][j];
//   backward item (rows [lo,hi) of 0..k):    column-major ldp x n,
//                 P[jq*ldp + r-lo] = E[r][col(jq)], col(jq) = n + jq (jq < k), jq (jq >= k).
// Padding entries are zero.
template <typename T>
__global__ void pack_q_kernel(const PanelItem* __restrict__ qitems, const SolveItem* __restrict__ sitems, int n_fwd,
                              const int* __restrict__ kk, const int* __restrict__ nn,
                              const long long* __restrict__ front_off, const T* __restrict__ pool,
                              T* __restrict__ Q) {
    const PanelItem pi = qitems[blockIdx.x];
    const SolveItem it = sitems[pi.front];
    const bool fwd = pi.front < n_fwd;
    const int F = it.front, k = kk[F], n = nn[F], ld = n + k;
    const T* E = pool + front_off[F] + n;
    T* q = Q + it.off;
    const long long cnt = (long long)it.ldp * (fwd ? k : n);
    const long long e1 = min(cnt, (long long)pi.r0 + 4096);
    for (long long e = pi.r0 + threadIdx.x; e < e1; e += blockDim.x) {
        T v = T(0);
        if (fwd) {
            const int r = (int)(e / it.ldp), j = it.lo + (int)(e % it.ldp);
            if (j < it.hi) v = E[(long long)j * ld + r];
        } else {
            const int jq = (int)(e / it.ldp), r = it.lo + (int)(e % it.ldp);
            if (r < it.hi) v = E[(long long)(jq < k ? n + jq : jq) * ld + r];
        }
        q[e] = v;
    }
}

__global__ void inertia_kernel(long long N, const double* __restrict__ D, long long* __restrict__ neg) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int local = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        local += (D[i] < 0.0) ? 1 : 0;
    if (local) atomicAdd(&cnt, local);
    __syncthreads();
    if (threadIdx.x == 0 && cnt) atomicAdd((unsigned long long*)neg, (unsigned long long)cnt);
}

template <typename T>
static int enqueue_factor_body(riga_ctx* c, T* pool, T* Q, cudaStream_t st);

// The factorization's launches.  A batch with per-problem shifts (read from
// device memory) replays them as one CUDA graph per mode, captured on the
// first call on a private stream and launched into the ctx's stream; the
// graph is rebuilt when the schedule or a buffer it uses changes.
template <typename T>
static int enqueue_factor_t(riga_ctx* c, T* pool, T* Q) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_FACTOR, 0.0, c->inertia_only ? S.flops : S.flops + S.flops_aug);
    const bool per_problem = (S.dim == 0) && !c->sigma_prob.empty();
    if (per_problem) {
        std::vector<double> sp(S.N);
        for (size_t b = 0; b + 1 < S.prob_pos.size(); ++b)
            for (long long i = S.prob_pos[b]; i < S.prob_pos[b + 1]; ++i) sp[i] = c->sigma_prob[b];
        RIGA_CUDA_TRY(c, c->sig_pos.upload(sp, st));
    }
    // FP64 fronts with tensor-core updates: buffers and attributes before any capture
    const bool oz = sizeof(T) == sizeof(double) && c->fp64_tc;
    if (oz) {
        int rc = prepare_oz(c);
        if (rc) return rc;
    }
    if (!per_problem || sizeof(T) != sizeof(double)) return enqueue_factor_body<T>(c, pool, Q, st);
    riga_ctx::FactorGraph& g = c->fgraph[c->inertia_only ? 1 : 0];
    const void* ptrs[9] = {pool, Q, c->D.ptr, c->flag.ptr, c->neg.ptr, c->sig_pos.ptr,
                           oz ? (const void*)c->ozpack.ptr : nullptr, oz ? (const void*)c->ozexp.ptr : nullptr,
                           oz ? (const void*)c->ozlive.ptr : nullptr};
    bool valid = g.exec && g.gen == c->sched_gen;
    for (int i = 0; i < 9 && valid; ++i) valid = g.ptrs[i] == ptrs[i];
    if (!valid) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        if (!c->cap_stream) RIGA_CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        RIGA_CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        const long long l0 = c->prof.launches;
        int rc = enqueue_factor_body<T>(c, pool, Q, c->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (rc == RIGA_OK && e != cudaSuccess) rc = set_error(c, RIGA_ECUDA, cudaGetErrorString(e));
        if (rc == RIGA_OK && cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
            g.exec = nullptr;
            rc = set_error(c, RIGA_ECUDA, "factorization graph");
        }
        if (graph) cudaGraphDestroy(graph);
        const int launches = (int)(c->prof.launches - l0);
        c->prof.launches = l0;  // counted when the graph runs
        c->prof.ph[PH_FACTOR].launches -= launches;
        if (rc) return rc;
        g.gen = c->sched_gen;
        for (int i = 0; i < 9; ++i) g.ptrs[i] = ptrs[i];
        g.launches = launches;
    }
    RIGA_CUDA_TRY(c, cudaGraphLaunch(g.exec, st));
    c->prof.launches += g.launches;
    c->prof.ph[PH_FACTOR].launches += g.launches;
    return RIGA_OK;
}

template <typename T>
static int enqueue_factor_body(riga_ctx* c, T* pool, T* Q, cudaStream_t st) {
    Symbolic& S = c->S;
    RIGA_CUDA_TRY(c, cudaMemsetAsync(pool, 0, (size_t)S.pool_size * sizeof(T), st));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(c->flag.ptr, 0, sizeof(int), st));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(c->neg.ptr, 0, sizeof(long long), st));
    const int plain = c->inertia_only ? 1 : 0;
    // TF32 / BF16 fronts: the trailing updates on the tensor cores (tc_update.cu)
    const bool tensor = sizeof(T) == sizeof(float) && (c->precision == RIGA_TF32 || c->precision == RIGA_BF16);
    if (tensor) {
        int rc = prepare_tc(c);
        if (rc) return rc;
    }
    // FP64 fronts: the trailing updates on the tensor cores from digit slices
    // (oz_update.cu; prepared in enqueue_factor_t)
    const bool oz = sizeof(T) == sizeof(double) && c->fp64_tc;
    if (!plain) { count_launch(c); identity_kernel<T><<<S.n_nodes, 128, 0, st>>>(S.n_nodes, c->kk.ptr, c->nn.ptr, c->front_off.ptr, pool); }
    const bool per_problem = (S.dim == 0) && !c->sigma_prob.empty();
    if (per_problem) {
        { count_launch(c); scatter_rows_kernel<T><<<(unsigned)((S.N * 32 + 255) / 256), 256, 0, st>>>(
            S.N, c->rowptr.ptr, c->scatter.ptr, c->Kval.ptr, c->Mval.ptr, c->sig_pos.ptr, pool); }
    } else if (S.nnz > 0) {
        { count_launch(c); scatter_kernel<T><<<(unsigned)((S.nnz + 255) / 256), 256, 0, st>>>(S.nnz, c->scatter.ptr, c->Kval.ptr,
                                                                          c->Mval.ptr, c->sigma, pool); }
    }
    for (int l = 0; l < S.n_levels; ++l) {
        const LevelPlan& P = S.levels[l];
        for (int rank = 0; rank < 2; ++rank) {
            int cnt = P.ext_end[rank] - P.ext_begin[rank];
            if (cnt > 0)
                { count_launch(c); extend_add_kernel<T><<<cnt, 128, 0, st>>>(c->eitems.ptr + P.ext_begin[rank], c->parent.ptr,
                                                          c->front_off.ptr, c->kk.ptr, c->nn.ptr, c->rel.ptr,
                                                          c->rel_ptr.ptr, pool); }
        }
        for (const StepRange& R : P.steps) {
            const int j0 = R.s * NB;
            if (R.d_end > R.d_begin)
                { count_launch(c); diag_kernel<T><<<R.d_end - R.d_begin, 128, 0, st>>>(c->pitems.ptr + R.d_begin, c->kk.ptr, c->nn.ptr,
                                                                    c->front_off.ptr, c->node_ptr.ptr, pool, c->D.ptr,
                                                                    c->flag.ptr); }
            if (R.p_end > R.p_begin)
                { count_launch(c); trsm_kernel<T><<<R.p_end - R.p_begin, RB, 0, st>>>(c->pitems.ptr + R.p_begin, j0, c->kk.ptr,
                                                                   c->nn.ptr, c->front_off.ptr, pool, plain); }
            if (tensor) {
                // within the super-panel: this panel's update of the super-panel's
                // remaining columns (CUDA cores); at its last panel: the whole
                // trailing matrix with K = the super-panel (tensor cores)
                if (R.n_end > R.n_begin)
                    { count_launch(c); update_kernel<T, 32, TileItemL><<<R.n_end - R.n_begin, 64, 0, st>>>(c->tcnarrow.ptr + R.n_begin, j0,
                                                                       c->kk.ptr, c->nn.ptr, c->front_off.ptr,
                                                                       c->node_ptr.ptr, c->D.ptr, pool, plain); }
                int rc = enqueue_tc_step(c, R, j0, reinterpret_cast<float*>(pool), plain, st);
                if (rc) return rc;
            } else if (oz) {
                int rc = enqueue_oz_step(c, R, reinterpret_cast<double*>(pool), plain, st);
                if (rc) return rc;
            } else {
                if (R.t_mid > R.t_begin)
                    { count_launch(c); update_kernel<T, 32><<<R.t_mid - R.t_begin, 64, 0, st>>>(c->titems.ptr + R.t_begin, j0,
                                                                       c->kk.ptr, c->nn.ptr, c->front_off.ptr,
                                                                       c->node_ptr.ptr, c->D.ptr, pool, plain); }
                if (R.t_end > R.t_mid)
                    { count_launch(c); update_kernel<T, 16><<<R.t_end - R.t_mid, 64, 0, st>>>(c->titems.ptr + R.t_mid, j0,
                                                                       c->kk.ptr, c->nn.ptr, c->front_off.ptr,
                                                                       c->node_ptr.ptr, c->D.ptr, pool, plain); }
            }
        }
    }
    if (!S.qitems.empty() && !plain)
        { count_launch(c); pack_q_kernel<T><<<(unsigned)S.qitems.size(), 256, 0, st>>>(c->qitems.ptr, c->sitems.ptr, S.n_fwd_items,
                                                                                      c->kk.ptr, c->nn.ptr, c->front_off.ptr,
                                                                                      pool, Q); }
    { count_launch(c); inertia_kernel<<<152, 256, 0, st>>>(S.N, c->D.ptr, c->neg.ptr); }
    if (S.dim == 0) {
        const size_t np = S.prob_pos.size() - 1;
        RIGA_CUDA_TRY(c, cudaMemsetAsync(c->neg.ptr + 1, 0, np * sizeof(long long), st));
        { count_launch(c); inertia_prob_kernel<<<152, 256, 0, st>>>(S.N, c->D.ptr, c->prob_of_pos.ptr, c->neg.ptr + 1); }
    }
    RIGA_CUDA_TRY(c, cudaGetLastError());
    return RIGA_OK;
}

int enqueue_factor(riga_ctx* c) {
    Symbolic& S = c->S;
    if (!c->inertia_only) c->fp64_sweeps = 1;  // a new factor: plain FP64 solves until calibrated
    if (S.nb != NB || S.tile != TILE || S.rowblk != RB) return set_error(c, RIGA_EINVAL, "schedule/kernel tile mismatch");
    RIGA_CUDA_TRY(c, c->D.alloc(S.N));
    RIGA_CUDA_TRY(c, c->flag.alloc(1));
    RIGA_CUDA_TRY(c, c->neg.alloc(S.dim == 0 ? S.prob_pos.size() : 1));
    if (c->precision == RIGA_FP64) {
        if (c->pool64.alloc(S.pool_size) != cudaSuccess) return set_error(c, RIGA_ENOMEM, "front pool (fp64)");
        if (c->q64.alloc(S.q_size + 4) != cudaSuccess) return set_error(c, RIGA_ENOMEM, "solve operators (fp64)");
        return enqueue_factor_t<double>(c, c->pool64.ptr, c->q64.ptr);
    }
    if (c->pool32.alloc(S.pool_size) != cudaSuccess) return set_error(c, RIGA_ENOMEM, "front pool (fp32)");
    if (c->q32.alloc(S.q_size + 4) != cudaSuccess) return set_error(c, RIGA_ENOMEM, "solve operators (fp32)");
    return enqueue_factor_t<float>(c, c->pool32.ptr, c->q32.ptr);
}

int finish_factor(riga_ctx* c) {
    int flag = 0;
    long long neg = 0;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(&flag, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(&neg, c->neg.ptr, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    if (c->S.dim == 0) {
        c->inertia_prob.assign(c->S.prob_pos.size() - 1, 0);
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->inertia_prob.data(), c->neg.ptr + 1, c->inertia_prob.size() * sizeof(long long),
                                         cudaMemcpyDeviceToHost, c->stream));
    }
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->inertia = neg;
    if (flag & 4) {
        c->factored = false;
        return set_error(c, RIGA_ETIMEOUT, "a tensor-core update did not complete within the wait budget");
    }
    if (flag & 1) {
        c->factored = false;
        return set_error(c, RIGA_EPIVOT, "zero or non-finite pivot in LDL^T (shift at an eigenvalue?)");
    }
    c->factored = !c->inertia_only;  // an inertia-only factorization cannot solve
    return RIGA_OK;
}

}  // namespace riga
