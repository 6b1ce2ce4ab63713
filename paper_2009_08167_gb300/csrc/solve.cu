// Forward/backward elimination with the multifrontal factor and FP64 SpMV
// (Sec. 4.2: one f/b elimination and the M mat-vecs per Lanczos step;
// Sec. 5.1 Eq. flopsFb).  Vectors are in elimination order.
//
// tree_solve_kernel: one persistent launch per solve; work items (parts of a
// front's forward or backward sweep) are taken in dependency order (forward
// leaves to root, then backward root to leaves) with bounded waits on
// per-front completed-part counters.
// The factorization leaves in each augmented front's extra rows the block
// elimination operators of the front, -A11^{-1} A12 and -A11^{-1}, so that
// the forward/backward elimination of Sec. 4.2 (L y = b, D, L^T x = z) is,
// front by front, one GEMV each way:
//   forward:  w = [b(own); 0] plus the children's update vectors;
//             u = w(border) - A21 A11^{-1} w(own) is this front's update
//             vector for its parent; w(own) is kept in the vector.
//   backward: x(own) = A11^{-1} w(own) - A11^{-1} A12 x(border), with
//             x(border) owned by ancestors and already final.
// No sequential triangular chain remains inside a front.  The operators are
// packed per front (factor.cu) and stream through shared memory by bulk
// copies (cp.async.bulk + mbarrier, double buffered), issued before the
// item waits on its dependencies; every operator entry is read once per sweep.
#include <algorithm>

#include "ctx.h"

namespace riga {


struct TreeArgs {
    const int* node_ptr;
    const int* kk;
    const int* nn;
    const int* child_ptr;
    const int* child_list;
    const int* parent;
    const int* rel;
    const long long* rel_ptr;
    const long long* upd_off;
    const long long* front_ptr;
    const int* front_pos;
    const int* parts_f;
    const int* parts_b;
    const SolveItem* items;  // forward parts (ascending height), then backward parts
    const ChildRec* crec;    // children records (see Symbolic::crec)
    int n_items, n_fwd;
    int chunk_elems;   // elements per shared-memory chunk buffer (two buffers)
    int max_n;
    double* upd;
    double* y;
    double* w1;        // assembled own right-hand sides (forward -> backward)
    int* done_f;       // completed forward parts per front (zeroed before the launch)
    int* done_b;       // completed backward parts per front
    int* counter;      // next work item (zeroed before the launch)
    int* err;          // bit 1: a dependency or copy wait gave up
    long long spin_limit;  // polls (64 ns back-off each) before a wait gives up
    long long* trace;      // optional: per item {sm, claim ns, deps-ready ns, done ns}
};

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int sm_id() {
    int id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

__device__ __forceinline__ bool wait_count(const int* f, int target, int* err, long long limit) {
    long long it = 0;
    while (*(volatile const int*)f < target) {
        if (++it > limit) {
            atomicOr(err, 2);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// ---- bulk (TMA) copies global -> shared with mbarrier completion (PTX) ----
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with the given parity
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err, long long limit) {
    long long it = 0;
    while (!mbar_test(bar, parity)) {
        if (++it > limit) {
            atomicOr(err, 2);
            return false;
        }
    }
    return true;
}

// acc[q] += sum over units u = ua+g, ua+g+G, ... < ub of P[u-ua][li + NT q] * w[u]
// for the NA output slots of this thread (an exact count: predicated-off FP64
// instructions still occupy GB300's narrow FP64 pipe).
template <typename T, int NA, int NT>
__device__ __forceinline__ void accumulate_chunk(const T* __restrict__ P, int ldp, int ua, int ub, int g, int G,
                                                 int li, int cnt, const T* __restrict__ w, T* acc) {
    for (int u = ua + g; u < ub; u += G) {
        const T* row = P + (long long)(u - ua) * ldp;
        const T x = w[u];
        if (NA == 1) {
            acc[0] += row[li] * x;
        } else {
#pragma unroll
            for (int q2 = 0; q2 < NA; ++q2) {
                const int l = li + q2 * NT;
                if (l < cnt) acc[q2] += row[l] * x;
            }
        }
    }
}

// One persistent launch per solve.  CTAs claim work items in order from a
// global counter; an item waits (bounded) until its dependencies are done:
// forward part: every forward part of every child; backward part: every
// forward part of its own front and every backward part of the parent.
// Dependencies always have lower item indices, so they were claimed by CTAs
// that are already running: no deadlock.  The item's operator panel is
// copied into shared memory by bulk copies issued before the dependency
// wait: in one copy when it fits the whole buffer (the usual case: parts are
// sized for that), else streamed through the two halves of the buffer.  A
// forward part owns border columns [lo,hi): u(j) = w(j) + sum_r P[r][j]
// w1(r); a backward part owns rows [lo,hi) of the front's own variables:
// x(r) = sum_j P[j][r] v(j), v = [-w1; x(border)].  Both are the same loop:
// stream units (forward: rows r; backward: columns j) times a multiplier
// (w1(r), v(j)) accumulated into the part's outputs; threads split the
// outputs and interleave the units, then reduce through shared memory.
// Everything an item needs to know about its front comes packed in the item
// (and, for its children, in one record each), so that few dependent global
// loads separate a claim from the arithmetic.
template <typename T, int NT>
__global__ void __launch_bounds__(NT) tree_solve_kernel(const T* __restrict__ Q, TreeArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* buf[2];
    buf[0] = reinterpret_cast<T*>(smem_raw);
    buf[1] = buf[0] + a.chunk_elems;
    T* w = buf[1] + a.chunk_elems;  // front vector (n)
    T* red = w + a.max_n;           // NT partial sums
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ int s_item, s_ok;
    const int tid = threadIdx.x;
    unsigned parity[2] = {0u, 0u};
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= a.n_items) return;
        const SolveItem it = a.items[item];
        const bool fwd = item < a.n_fwd;
        const int F = it.front, k = it.k, n = it.n, b0 = it.b0;
        const int lo = it.lo, cnt = it.hi - it.lo, ldp = it.ldp;
        const T* q = Q + it.off;
        const int units = fwd ? k : n;  // rows (forward) or columns (backward) of the panel
        // one copy into the whole buffer, or chunks through its halves
        const bool whole = (long long)units * ldp <= 2LL * a.chunk_elems;
        const int upc = whole ? max(1, units) : max(1, a.chunk_elems / ldp);
        const int nchunks = (cnt > 0) ? (units + upc - 1) / upc : 0;
        const int issued = min(2, nchunks);
        if (tid == 0) {
            if (a.trace) {
                a.trace[4 * item] = sm_id();
                a.trace[4 * item + 1] = global_ns();
            }
            for (int c = 0; c < issued; ++c) {
                const int ua = c * upc, un = min(upc, units - ua);
                bulk_load(buf[c], q + (long long)ua * ldp, (unsigned)(un * ldp * sizeof(T)), &mbar[c]);
            }
            bool ok = true;
            if (fwd) {
                for (int ci = it.c0; ci < it.c1 && ok; ++ci) {
                    const ChildRec cr = a.crec[ci];
                    ok = wait_count(&a.done_f[cr.child], cr.parts, a.err, a.spin_limit);
                }
            } else {
                ok = wait_count(&a.done_f[F], it.wait_parts, a.err, a.spin_limit);
                if (ok && it.parent >= 0) ok = wait_count(&a.done_b[it.parent], it.parent_parts, a.err, a.spin_limit);
            }
            __threadfence();
            s_ok = ok;
            if (a.trace) a.trace[4 * item + 2] = global_ns();
        }
        __syncthreads();
        if (!s_ok) {
            // drain the copies in flight (bounded) before leaving
            for (int c = 0; c < issued; ++c) mbar_wait(&mbar[c], parity[c], a.err, a.spin_limit);
            __syncthreads();
            return;
        }
        if (fwd) {
            // w = [b(own); 0] + children's update vectors
            for (int i = tid; i < n; i += NT) w[i] = (i < k) ? (T)__ldcg(&a.y[b0 + i]) : T(0);
            __syncthreads();
            for (int ci = it.c0; ci < it.c1; ++ci) {
                const ChildRec cr = a.crec[ci];
                const int* r = a.rel + cr.rel_off;
                const double* u = a.upd + cr.upd_off;
                for (int i = tid; i < cr.m; i += NT) w[r[i]] += (T)__ldcg(&u[i]);
                __syncthreads();
            }
            if (lo == k)  // the first part keeps w1 = w(own) for the backward sweep
                for (int i = tid; i < k; i += NT) a.w1[b0 + i] = (double)w[i];
        } else {
            const int* idx = a.front_pos + it.fpos;
            for (int i = tid; i < n; i += NT)
                w[i] = (i < k) ? -(T)__ldcg(&a.w1[b0 + i]) : (T)__ldcg(&a.y[idx[i]]);
        }
        __syncthreads();
        // thread layout: outputs l (columns or rows of the part) x unit groups g
        const int cp = max(1, min(cnt, NT));
        const int G = max(1, NT / cp);
        const int li = tid % cp, g = tid / cp;
        const bool active = cnt > 0 && g < G;
        const int na = (cnt + NT - 1) / NT;  // outputs per thread when cnt > NT (G = 1)
        T acc[8];
#pragma unroll
        for (int q2 = 0; q2 < 8; ++q2) acc[q2] = T(0);
        for (int c = 0; c < nchunks; ++c) {
            const int b = c & 1;
            const bool good = mbar_wait(&mbar[b], parity[b], a.err, a.spin_limit);
            if (__syncthreads_or(!good)) {
                // a copy did not complete within the budget: wait once more
                // (bounded) for it and for the next one, then leave
                mbar_wait(&mbar[b], parity[b], a.err, a.spin_limit);
                if (c + 1 < nchunks) mbar_wait(&mbar[b ^ 1], parity[b ^ 1], a.err, a.spin_limit);
                __syncthreads();
                return;
            }
            parity[b] ^= 1u;
            const int ua = c * upc, ub = min(units, ua + upc);
            const T* P = buf[b];
            if (active) {
                switch (na) {
                    case 1: accumulate_chunk<T, 1, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                    case 2: accumulate_chunk<T, 2, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                    case 3: accumulate_chunk<T, 3, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                    case 4: accumulate_chunk<T, 4, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                    case 5: accumulate_chunk<T, 5, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                    case 6: accumulate_chunk<T, 6, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                    case 7: accumulate_chunk<T, 7, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                    default: accumulate_chunk<T, 8, NT>(P, ldp, ua, ub, g, G, li, cnt, w, acc); break;
                }
            }
            __syncthreads();
            if (tid == 0 && c + 2 < nchunks) {
                fence_proxy_async();
                const int u2 = (c + 2) * upc, un2 = min(upc, units - u2);
                bulk_load(buf[b], q + (long long)u2 * ldp, (unsigned)(un2 * ldp * sizeof(T)), &mbar[b]);
            }
        }
        if (cnt > 0) {
            if (G > 1) {
                if (active) red[g * cp + li] = acc[0];
                __syncthreads();
                if (g == 0 && li < cnt) {
                    T s = T(0);
                    for (int g2 = 0; g2 < G; ++g2) s += red[g2 * cp + li];
                    acc[0] = s;
                }
            }
            if (g == 0) {
#pragma unroll
                for (int q2 = 0; q2 < 8; ++q2) {
                    const int l = li + q2 * NT;
                    if (q2 < na && l < cnt) {
                        if (fwd) a.upd[it.upd_off + lo + l - k] = (double)(w[lo + l] + acc[q2]);
                        else a.y[b0 + lo + l] = (double)acc[q2];
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(fwd ? &a.done_f[F] : &a.done_b[F], 1);
            if (a.trace) a.trace[4 * item + 3] = global_ns();
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-per-item variant for batches of many small trees, where the solve is
// bound by how many items are in flight rather than by a critical path:
// every warp is an independent worker with its own front vector in shared
// memory, so that dozens of items per SM overlap their dependency waits and
// gathers.  The item's panel is prefetched into L2 by one bulk prefetch when
// the item is claimed (before its dependency wait) and then read once with
// streaming loads straight into registers.  Parts hold at most 256 outputs
// (8 per lane), in widths that are multiples of 32.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// acc[q] += sum over units u = g, g+G, ... < units of P[u][li + 32 q] * w[u];
// U units per round, so that U * NA loads are in flight per lane
template <typename T, int NA, int U>
__device__ __forceinline__ void warp_accumulate(const T* __restrict__ P, int ldp, int units, int g, int G, int li,
                                                int cnt, const T* __restrict__ w, T* acc) {
    int u = g;
    for (; u + (U - 1) * G < units; u += U * G) {
        T v[U][NA];
#pragma unroll
        for (int s = 0; s < U; ++s) {
            const T* row = P + (long long)(u + s * G) * ldp;
#pragma unroll
            for (int q2 = 0; q2 < NA; ++q2) {
                const int l = li + 32 * q2;
                v[s][q2] = (l < cnt) ? __ldcs(row + l) : T(0);
            }
        }
#pragma unroll
        for (int s = 0; s < U; ++s) {
            const T x = w[u + s * G];
#pragma unroll
            for (int q2 = 0; q2 < NA; ++q2)
                if (li + 32 * q2 < cnt) acc[q2] += v[s][q2] * x;
        }
    }
    for (; u < units; u += G) {
        const T* row = P + (long long)u * ldp;
        const T x = w[u];
#pragma unroll
        for (int q2 = 0; q2 < NA; ++q2) {
            const int l = li + 32 * q2;
            if (l < cnt) acc[q2] += __ldcs(row + l) * x;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(128) tree_solve_warp_kernel(const T* __restrict__ Q, TreeArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    T* w = reinterpret_cast<T*>(smem_raw) + (size_t)(threadIdx.x >> 5) * a.max_n;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= a.n_items) return;
        const SolveItem it = a.items[item];
        const bool fwd = item < a.n_fwd;
        const int F = it.front, k = it.k, n = it.n, b0 = it.b0;
        const int lo = it.lo, cnt = it.hi - it.lo, ldp = it.ldp;
        const T* q = Q + it.off;
        const int units = fwd ? k : n;  // rows (forward) or columns (backward) of the panel
        if (lane == 0) {
            if (a.trace) {
                a.trace[4 * item] = sm_id();
                a.trace[4 * item + 1] = global_ns();
            }
            if (cnt > 0 && units > 0) bulk_prefetch_l2(q, (unsigned)((long long)units * ldp * sizeof(T)));
        }
        // dependency waits: forward, every forward part of every child (one
        // lane per child); backward, this front's forward parts and the
        // parent's backward parts
        bool ok = true;
        if (fwd) {
            for (int ci = it.c0 + lane; ci < it.c1; ci += 32) {
                const ChildRec cr = a.crec[ci];
                ok = ok && wait_count(&a.done_f[cr.child], cr.parts, a.err, a.spin_limit);
            }
        } else if (lane == 0) {
            ok = wait_count(&a.done_f[F], it.wait_parts, a.err, a.spin_limit);
            if (ok && it.parent >= 0) ok = wait_count(&a.done_b[it.parent], it.parent_parts, a.err, a.spin_limit);
        }
        if (!__all_sync(FULL, ok)) return;
        __threadfence();
        if (a.trace && lane == 0) a.trace[4 * item + 2] = global_ns();
        if (fwd) {
            // w = [b(own); 0] + children's update vectors
            for (int i = lane; i < n; i += 32) w[i] = (i < k) ? (T)__ldcg(&a.y[b0 + i]) : T(0);
            __syncwarp();
            for (int ci = it.c0; ci < it.c1; ++ci) {
                const ChildRec cr = a.crec[ci];
                const int* r = a.rel + cr.rel_off;
                const double* u = a.upd + cr.upd_off;
                for (int i = lane; i < cr.m; i += 32) w[r[i]] += (T)__ldcg(&u[i]);
                __syncwarp();
            }
            if (lo == k)  // the first part keeps w1 = w(own) for the backward sweep
                for (int i = lane; i < k; i += 32) a.w1[b0 + i] = (double)w[i];
        } else {
            const int* idx = a.front_pos + it.fpos;
            for (int i = lane; i < n; i += 32)
                w[i] = (i < k) ? -(T)__ldcg(&a.w1[b0 + i]) : (T)__ldcg(&a.y[idx[i]]);
        }
        __syncwarp();
        // lanes: outputs li (cp per unit group) x unit groups g (G = 32 / cp)
        const int cp = cnt > 16 ? 32 : (cnt > 8 ? 16 : (cnt > 4 ? 8 : 4));
        const int G = 32 / cp, li = lane % cp, g = lane / cp;
        const int na = (cnt + 31) / 32;
        T acc[8];
#pragma unroll
        for (int q2 = 0; q2 < 8; ++q2) acc[q2] = T(0);
        if (cnt > 0) {
            switch (na) {
                case 1: warp_accumulate<T, 1, 16>(q, ldp, units, g, G, li, cnt, w, acc); break;
                case 2: warp_accumulate<T, 2, 8>(q, ldp, units, g, G, li, cnt, w, acc); break;
                case 3: warp_accumulate<T, 3, 4>(q, ldp, units, g, G, li, cnt, w, acc); break;
                case 4: warp_accumulate<T, 4, 4>(q, ldp, units, g, G, li, cnt, w, acc); break;
                case 5: warp_accumulate<T, 5, 4>(q, ldp, units, g, G, li, cnt, w, acc); break;
                case 6: warp_accumulate<T, 6, 4>(q, ldp, units, g, G, li, cnt, w, acc); break;
                case 7: warp_accumulate<T, 7, 4>(q, ldp, units, g, G, li, cnt, w, acc); break;
                default: warp_accumulate<T, 8, 4>(q, ldp, units, g, G, li, cnt, w, acc); break;
            }
            for (int o = cp; o < 32; o <<= 1) acc[0] += __shfl_xor_sync(FULL, acc[0], o);
            if (g == 0) {
#pragma unroll
                for (int q2 = 0; q2 < 8; ++q2) {
                    const int l = li + 32 * q2;
                    if (q2 < na && l < cnt) {
                        if (fwd) a.upd[it.upd_off + lo + l - k] = (double)(w[lo + l] + acc[q2]);
                        else a.y[b0 + lo + l] = (double)acc[q2];
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicAdd(fwd ? &a.done_f[F] : &a.done_b[F], 1);
            if (a.trace) a.trace[4 * item + 3] = global_ns();
        }
        __syncwarp();
    }
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

template <typename T>
static int enqueue_solve_t(riga_ctx* c, const T* Q, double* y) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    // algorithmic bytes: the solve operators (k x (n-k) forward, k x n backward)
    // and the vector read and written in each sweep
    PhaseScope scope(c, PH_SOLVE, (2.0 * (double)S.nnzQ - (double)S.nnzL_own2) * sizeof(T) + 4.0 * (double)S.N * sizeof(double));
    int max_n = 0, max_ldp = 0;
    for (int f = 0; f < S.n_nodes; ++f) max_n = std::max(max_n, S.n[f]);
    for (const SolveItem& it : S.sitems) max_ldp = std::max(max_ldp, it.ldp);
    // batches of many small trees: one item per warp (tree_solve_warp_kernel);
    // small fronts: 128 threads and a 32 KiB (FP64) panel buffer per CTA, so
    // that many items per SM overlap their waits; large fronts: 256 threads
    // and two 32 KiB halves
    const int n_items = (int)S.sitems.size();
    int maxopt = 0, nsm = 0, per_sm = 0;
    RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    const int nt = S.solve_mode == SOLVE_CTA256 ? 256 : 128;
    // (small: halves of 2048..3072 elements, so that every part's panel
    // usually arrives in one copy)
    int chunk = S.solve_mode == SOLVE_CTA128
                    ? (int)std::min<long long>(3072, std::max<long long>(2048, (S.max_panel + 1) / 2))
                    : (int)(32768 / sizeof(T));
    chunk = std::max(chunk, max_ldp);
    chunk = (chunk + 3) / 4 * 4;
    const bool warp = S.solve_mode == SOLVE_WARP;
    const size_t smem = warp ? 4 * (size_t)max_n * sizeof(T) : (2 * (size_t)chunk + max_n + nt + 8) * sizeof(T);
    if (smem + 256 > (size_t)maxopt) return set_error(c, RIGA_EINVAL, "front too large for the shared-memory solve");
    auto kern = warp ? tree_solve_warp_kernel<T>
                     : (S.solve_mode == SOLVE_CTA128 ? tree_solve_kernel<T, 128> : tree_solve_kernel<T, 256>);
    if (smem > 48 * 1024)
        RIGA_CUDA_TRY(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    RIGA_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, smem));
    const int per_block = warp ? 4 : 1;  // concurrent items per block
    const int grid = std::max(1, std::min((n_items + per_block - 1) / per_block, std::max(1, per_sm) * nsm));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(c->solve_flags.ptr, 0, (2 * (size_t)S.n_nodes + 1) * sizeof(int), st));
    TreeArgs a;
    a.node_ptr = c->node_ptr.ptr;
    a.kk = c->kk.ptr;
    a.nn = c->nn.ptr;
    a.child_ptr = c->child_ptr.ptr;
    a.child_list = c->child_list.ptr;
    a.parent = c->parent.ptr;
    a.rel = c->rel.ptr;
    a.rel_ptr = c->rel_ptr.ptr;
    a.upd_off = c->upd_off.ptr;
    a.front_ptr = c->front_ptr.ptr;
    a.front_pos = c->front_pos.ptr;
    a.parts_f = c->parts_f.ptr;
    a.parts_b = c->parts_b.ptr;
    a.items = c->sitems.ptr;
    a.crec = c->crec.ptr;
    a.n_items = n_items;
    a.n_fwd = S.n_fwd_items;
    a.chunk_elems = chunk;
    a.max_n = max_n;
    a.upd = c->upd.ptr;
    a.y = y;
    a.w1 = c->w1buf.ptr;
    a.done_f = c->solve_flags.ptr;
    a.done_b = c->solve_flags.ptr + S.n_nodes;
    a.counter = c->solve_flags.ptr + 2 * S.n_nodes;
    a.err = c->flag.ptr;
    a.spin_limit = c->wait_limit;
    a.trace = c->trace_buf;
    { count_launch(c); kern<<<grid, nt, smem, st>>>(Q, a); }
    return RIGA_OK;
}

int enqueue_solve(riga_ctx* c, double* y) {
    if (!c->factored) return set_error(c, RIGA_ESTATE, "no factorization");
    Symbolic& S = c->S;
    RIGA_CUDA_TRY(c, c->upd.alloc(S.upd_size > 0 ? S.upd_size : 1));
    RIGA_CUDA_TRY(c, c->solve_flags.alloc(2 * (size_t)S.n_nodes + 1));
    RIGA_CUDA_TRY(c, c->w1buf.alloc(S.N));
    int rc;
    if (c->precision == RIGA_FP64) rc = enqueue_solve_t<double>(c, c->q64.ptr, y);
    else rc = enqueue_solve_t<float>(c, c->q32.ptr, y);
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
