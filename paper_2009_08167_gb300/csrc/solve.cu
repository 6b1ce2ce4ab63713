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
    int item0;         // first item of this launch (items item0 .. item0 + n_items - 1)
    int n_items, n_fwd;
    int nsplit;        // independent groups of NR right-hand sides, items interleaved
    int n_fronts;      // stride of the per-group completion counters
    long long upd_size;  // stride (per right-hand side) of the update vectors
    int chunk_elems;   // elements per shared-memory chunk buffer (two per slot)
    int nslot;         // 1, or 2: the next item's copies start while the current one runs
    int max_n;
    double* upd;
    double* y;         // NR right-hand sides, column r at y + r * ldy
    long long ldy;
    double* w1;        // assembled own right-hand sides (forward -> backward), stride ldy
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

// Publication of a completed part: the CTA's writes (ordered before by
// __syncthreads) are released at GPU scope by an acquire-release fence, then
// the counter is bumped by a relaxed reduction (no return value); the waiter
// reads the counter and issues the same fence before it reads the data.
__device__ __forceinline__ void release_add(int* p) {
    asm volatile(
        "fence.acq_rel.gpu;\n"
        "red.relaxed.gpu.global.add.s32 [%0], 1;" ::"l"(p)
        : "memory");
}
__device__ __forceinline__ void acquire_fence() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

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

// acc[q][r] += sum over units u = ua+g, ua+g+G, ... < ub of P[u-ua][l0 + li + NT q] * w_r[u]
// for the NA output slots of this thread and the NR right-hand sides (an
// exact count: predicated-off FP64 instructions still occupy GB300's narrow
// FP64 pipe).  Each panel entry read from shared memory serves NR products.
template <typename T, int NA, int NT, int NR>
__device__ __forceinline__ void accumulate_chunk(const T* __restrict__ P, int ldp, int ua, int ub, int g, int G,
                                                 int l0, int li, int cnt, const T* __restrict__ w, int ldw,
                                                 T (*acc)[NR]) {
    for (int u = ua + g; u < ub; u += G) {
        const T* row = P + (long long)(u - ua) * ldp + l0;
        T x[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) x[r] = w[r * ldw + u];
#pragma unroll
        for (int q2 = 0; q2 < NA; ++q2) {
            const int l = li + q2 * NT;
            if (l0 + l < cnt) {
                const T pv = row[l];
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[q2][r] += pv * x[r];
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
// NR right-hand sides (columns of y, w1 and of each front's update vector,
// stride a.ldy / m) go through the same items: one panel read, NR products.
// Everything an item needs to know about its front comes packed in the item
// (and, for its children, in one record each), so that few dependent global
// loads separate a claim from the arithmetic.
template <typename T, int NT, int NR, int MINB = 1>
__global__ void __launch_bounds__(NT, MINB) tree_solve_kernel(const T* __restrict__ Q, TreeArgs a) {
    constexpr int NAMAX = (NR == 1) ? 8 : (NR == 2 ? 4 : 2);  // output slots per thread per pass
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // a.nslot slots of two chunk halves each: slot s = halves 2s, 2s+1
    T* const bufs = reinterpret_cast<T*>(smem_raw);
    T* w = bufs + 2 * a.nslot * a.chunk_elems;  // front vectors (NR x max_n)
    T* red = w + NR * a.max_n;                  // NT x NR partial sums
    const int ldw = a.max_n;
    __shared__ __align__(8) unsigned long long mbar[4];
    __shared__ int s_item, s_next, s_ok;
    __shared__ int s_pend[4];  // per half: a copy issued and not yet waited for
    const int tid = threadIdx.x;
    const int total = a.n_items * a.nsplit;
    unsigned par = 0u;  // bit h: parity of the next phase of mbar[h] (every thread tracks it)
    if (tid == 0) {
        for (int h = 0; h < 4; ++h) {
            mbar_init(&mbar[h], 1);
            s_pend[h] = 0;
        }
        fence_mbar_init();
    }
    __syncthreads();
    // thread 0: issue the first (up to two) chunk copies of claimed work
    // `cw` into slot sl; an item's panel goes in one copy when it fits the
    // slot's two halves, else in chunks through them
    auto issue_first = [&](int cw, int sl) {
        const SolveItem it = a.items[a.item0 + cw / a.nsplit];
        const bool fw = a.item0 + cw / a.nsplit < a.n_fwd;
        const int units = fw ? it.k : it.n, ldp = it.ldp, cnt = it.hi - it.lo;
        const bool whole = (long long)units * ldp <= 2LL * a.chunk_elems;
        const int upc = whole ? max(1, units) : max(1, a.chunk_elems / ldp);
        const int nchunks = (cnt > 0) ? (units + upc - 1) / upc : 0;
        const T* q = Q + it.off;
        fence_proxy_async();  // the slot's previous contents were read by the generic proxy
        for (int c = 0; c < min(2, nchunks); ++c) {
            const int ua = c * upc, un = min(upc, units - ua);
            s_pend[2 * sl + c] = 1;
            bulk_load(bufs + (size_t)(2 * sl + c) * a.chunk_elems, q + (long long)ua * ldp, (unsigned)(un * ldp * sizeof(T)),
                      &mbar[2 * sl + c]);
        }
    };
    // bounded waits for every copy still in flight, then leave
    auto drain = [&]() {
        for (int h = 0; h < 2 * a.nslot; ++h)
            if (s_pend[h]) mbar_wait(&mbar[h], (par >> h) & 1u, a.err, a.spin_limit);
        __syncthreads();
    };
    if (tid == 0) {
        s_item = atomicAdd(a.counter, 1);
        if (s_item < total) issue_first(s_item, 0);
    }
    int cs = 0;  // slot of the current item
    __syncthreads();
    for (;;) {
        const int claimed_local = s_item;
        if (claimed_local >= total) return;  // no copies in flight
        const int claimed = a.item0 * a.nsplit + claimed_local;  // global work index (trace slot)
        const int item = claimed / a.nsplit, grp = claimed - item * a.nsplit;
        double* const y = a.y + (long long)grp * NR * a.ldy;
        double* const w1 = a.w1 + (long long)grp * NR * a.ldy;
        double* const upd = a.upd + (long long)grp * NR * a.upd_size;
        int* const done_f = a.done_f + (long long)grp * a.n_fronts;
        int* const done_b = a.done_b + (long long)grp * a.n_fronts;
        const SolveItem it = a.items[item];
        const bool fwd = item < a.n_fwd;
        const int F = it.front, k = it.k, n = it.n, b0 = it.b0, m = n - k;
        const int lo = it.lo, cnt = it.hi - it.lo, ldp = it.ldp;
        const T* q = Q + it.off;
        const int units = fwd ? k : n;  // rows (forward) or columns (backward) of the panel
        const bool whole = (long long)units * ldp <= 2LL * a.chunk_elems;
        const int upc = whole ? max(1, units) : max(1, a.chunk_elems / ldp);
        const int nchunks = (cnt > 0) ? (units + upc - 1) / upc : 0;
        if (tid == 0) {
            if (a.trace) {
                a.trace[4 * claimed] = sm_id();
                a.trace[4 * claimed + 1] = global_ns();
            }
            // two slots: the next work is claimed now and its copies overlap
            // this item's dependency wait and arithmetic.  Work is still
            // taken in counter order by each CTA, so every dependency of an
            // item is held by a CTA that is running an earlier item.
            if (a.nslot == 2) {
                s_next = atomicAdd(a.counter, 1);
                if (s_next < total) issue_first(s_next, cs ^ 1);
            }
            bool ok = true;
            if (fwd) {
                for (int ci = it.c0; ci < it.c1 && ok; ++ci) {
                    const ChildRec cr = a.crec[ci];
                    ok = wait_count(&done_f[cr.child], cr.parts, a.err, a.spin_limit);
                }
            } else {
                ok = wait_count(&done_f[F], it.wait_parts, a.err, a.spin_limit);
                if (ok && it.parent >= 0) ok = wait_count(&done_b[it.parent], it.parent_parts, a.err, a.spin_limit);
            }
            acquire_fence();
            s_ok = ok;
            if (a.trace) a.trace[4 * claimed + 2] = global_ns();
        }
        // Static data of the item, loaded by every thread while thread 0
        // waits for the dependencies (one right-hand side, fronts of at most
        // PF * NT variables, at most two children): the own right-hand side
        // and the children's relative indices (forward), the border index
        // list (backward).  After the wait one round of loads remains: the
        // children's update vectors, or w1 and the ancestors' solution.
        constexpr int PF = 4;
        T pf_y[PF];
        int pf_ri[2][PF], pf_m[2] = {0, 0}, pf_idx[PF];
        long long pf_uo[2] = {0, 0};
        bool fast = false;
        if (NR == 1) {
            if (fwd) {
                const int nch = it.c1 - it.c0;
                fast = nch <= 2 && n <= PF * NT;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (c < nch && fast) {
                        const ChildRec cr = a.crec[it.c0 + c];
                        pf_m[c] = cr.m;
                        pf_uo[c] = cr.upd_off;
                        fast = cr.m <= PF * NT;
                        const int* rl = a.rel + cr.rel_off;
#pragma unroll
                        for (int q = 0; q < PF; ++q) {
                            const int i = tid + q * NT;
                            pf_ri[c][q] = (fast && i < cr.m) ? __ldg(rl + i) : 0;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < PF; ++q) pf_ri[c][q] = 0;
                    }
                }
                if (fast)
#pragma unroll
                    for (int q = 0; q < PF; ++q) {
                        const int i = tid + q * NT;
                        pf_y[q] = i < k ? (T)__ldcg(&y[b0 + i]) : T(0);
                    }
            } else {
                fast = n <= PF * NT;
                const int* idx = a.front_pos + it.fpos;
#pragma unroll
                for (int q = 0; q < PF; ++q) {
                    const int i = tid + q * NT;
                    pf_idx[q] = (fast && i >= k && i < n) ? __ldg(idx + i) : 0;
                }
            }
        }
        __syncthreads();
        if (!s_ok) {
            drain();
            return;
        }
        if (fast && fwd) {
            // w = [b(own); 0], then child 0's and child 1's update vectors
            // added in that order (as the general path below)
            const int nch = it.c1 - it.c0;
            T uv[2][PF];
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int q = 0; q < PF; ++q) {
                    const int i = tid + q * NT;
                    uv[c][q] = (c < nch && i < pf_m[c]) ? (T)__ldcg(&upd[pf_uo[c] + i]) : T(0);
                }
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                const int i = tid + q * NT;
                if (i < n) w[i] = pf_y[q];
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (c < nch) {
#pragma unroll
                    for (int q = 0; q < PF; ++q) {
                        const int i = tid + q * NT;
                        if (i < pf_m[c]) w[pf_ri[c][q]] += uv[c][q];
                    }
                    __syncthreads();
                }
            }
            if (lo == k)  // the first part keeps w1 = w(own) for the backward sweep
                for (int i = tid; i < k; i += NT) w1[b0 + i] = (double)w[i];
        } else if (fast) {
            T v[PF];
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                const int i = tid + q * NT;
                v[q] = i < k ? -(T)__ldcg(&w1[b0 + i]) : (i < n ? (T)__ldcg(&y[pf_idx[q]]) : T(0));
            }
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                const int i = tid + q * NT;
                if (i < n) w[i] = v[q];
            }
        } else if (fwd) {
            // w = [b(own); 0] + children's update vectors
            for (int r = 0; r < NR; ++r)
                for (int i = tid; i < n; i += NT)
                    w[r * ldw + i] = (i < k) ? (T)__ldcg(&y[(long long)r * a.ldy + b0 + i]) : T(0);
            __syncthreads();
            for (int ci = it.c0; ci < it.c1; ++ci) {
                const ChildRec cr = a.crec[ci];
                const int* rl = a.rel + cr.rel_off;
                const double* u = upd + cr.upd_off * NR;
                for (int r = 0; r < NR; ++r)
                    for (int i = tid; i < cr.m; i += NT) w[r * ldw + rl[i]] += (T)__ldcg(&u[(long long)r * cr.m + i]);
                __syncthreads();
            }
            if (lo == k)  // the first part keeps w1 = w(own) for the backward sweep
                for (int r = 0; r < NR; ++r)
                    for (int i = tid; i < k; i += NT) w1[(long long)r * a.ldy + b0 + i] = (double)w[r * ldw + i];
        } else {
            const int* idx = a.front_pos + it.fpos;
            for (int r = 0; r < NR; ++r)
                for (int i = tid; i < n; i += NT)
                    w[r * ldw + i] = (i < k) ? -(T)__ldcg(&w1[(long long)r * a.ldy + b0 + i])
                                             : (T)__ldcg(&y[(long long)r * a.ldy + idx[i]]);
        }
        __syncthreads();
        // thread layout: outputs l (columns or rows of the part) x unit groups g;
        // outputs beyond NAMAX * NT per thread take further passes over the
        // (then whole) panel in shared memory
        const int cp = max(1, min(cnt, NT));
        const int G = max(1, NT / cp);
        const int li = tid % cp, g = tid / cp;
        const bool active = cnt > 0 && g < G;
        const int npass = nchunks > 1 ? 1 : max(1, (cnt + NAMAX * NT - 1) / (NAMAX * NT));
        for (int pass = 0; pass < npass; ++pass) {
            const int l0 = pass * NAMAX * NT;
            const int cl = min(cnt - l0, (nchunks > 1) ? cnt : NAMAX * NT);  // outputs of this pass
            const int na = (cl + NT - 1) / NT;
            T acc[(NR == 1) ? 8 : NAMAX][NR];
#pragma unroll
            for (int q2 = 0; q2 < ((NR == 1) ? 8 : NAMAX); ++q2)
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[q2][r] = T(0);
            for (int c = 0; c < nchunks; ++c) {
                const int b = 2 * cs + (c & 1);  // half of the current slot
                if (pass == 0) {
                    const bool good = mbar_wait(&mbar[b], (par >> b) & 1u, a.err, a.spin_limit);
                    if (__syncthreads_or(!good)) {
                        // a copy did not complete within the budget: wait once more
                        // (bounded) for every copy in flight, then leave
                        drain();
                        return;
                    }
                    par ^= 1u << b;
                    if (tid == 0) s_pend[b] = 0;
                }
                const int ua = c * upc, ub = min(units, ua + upc);
                const T* P = bufs + (size_t)b * a.chunk_elems;
                if (active) {
                    if (NR == 1) {
                        switch (na) {
                            case 1: accumulate_chunk<T, 1, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                            case 2: accumulate_chunk<T, 2, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                            case 3: accumulate_chunk<T, 3, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                            case 4: accumulate_chunk<T, 4, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                            case 5: accumulate_chunk<T, 5, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                            case 6: accumulate_chunk<T, 6, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                            case 7: accumulate_chunk<T, 7, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                            default: accumulate_chunk<T, 8, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc); break;
                        }
                    } else if (na == 1) {
                        accumulate_chunk<T, 1, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc);
                    } else if (NAMAX >= 2 && na == 2) {
                        accumulate_chunk<T, (NAMAX >= 2 ? 2 : 1), NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc);
                    } else if (NAMAX >= 4) {
                        if (na == 3) accumulate_chunk<T, (NAMAX >= 3 ? 3 : 1), NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc);
                        else accumulate_chunk<T, NAMAX, NT, NR>(P, ldp, ua, ub, g, G, l0, li, cnt, w, ldw, acc);
                    }
                }
                __syncthreads();
                if (pass == 0 && tid == 0 && c + 2 < nchunks) {
                    fence_proxy_async();
                    const int u2 = (c + 2) * upc, un2 = min(upc, units - u2);
                    s_pend[b] = 1;
                    bulk_load(bufs + (size_t)b * a.chunk_elems, q + (long long)u2 * ldp, (unsigned)(un2 * ldp * sizeof(T)),
                              &mbar[b]);
                }
            }
            if (cl > 0) {
                if (G > 1) {
                    if (active)
#pragma unroll
                        for (int r = 0; r < NR; ++r) red[(g * cp + li) * NR + r] = acc[0][r];
                    __syncthreads();
                    if (g == 0 && li < cl)
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            T s2 = T(0);
                            for (int g2 = 0; g2 < G; ++g2) s2 += red[(g2 * cp + li) * NR + r];
                            acc[0][r] = s2;
                        }
                }
                if (g == 0) {
#pragma unroll
                    for (int q2 = 0; q2 < ((NR == 1) ? 8 : NAMAX); ++q2) {
                        const int l = l0 + li + q2 * NT;
                        if (q2 < na && l < cnt) {
#pragma unroll
                            for (int r = 0; r < NR; ++r) {
                                if (fwd) upd[it.upd_off * NR + (long long)r * m + lo + l - k] =
                                             (double)(w[r * ldw + lo + l] + acc[q2][r]);
                                else y[(long long)r * a.ldy + b0 + lo + l] = (double)acc[q2][r];
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (tid == 0) {
            release_add(fwd ? &done_f[F] : &done_b[F]);
            if (a.trace) a.trace[4 * claimed + 3] = global_ns();
            if (a.nslot == 2) {
                s_item = s_next;
            } else {
                s_item = atomicAdd(a.counter, 1);
                if (s_item < total) issue_first(s_item, 0);
            }
        }
        if (a.nslot == 2) cs ^= 1;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Warp-per-item variant for batches of many small trees, where the solve is
// bound by how many items are in flight rather than by a critical path:
// every warp is an independent worker with its own front vectors in shared
// memory, so that dozens of items per SM overlap their dependency waits and
// gathers.  The item's panel is prefetched into L2 by one bulk prefetch when
// the item is claimed (before its dependency wait) and then read once with
// streaming loads straight into registers.  Parts hold at most 128 outputs
// (4 per lane), in widths that are multiples of 32.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// acc[q][r] += sum over units u = g, g+G, ... < units of P[u][li + 32 q] * w_r[u];
// U units per round, so that U * NA loads are in flight per lane
template <typename T, int NA, int U, int NR>
__device__ __forceinline__ void warp_accumulate(const T* __restrict__ P, int ldp, int units, int g, int G, int li,
                                                int cnt, const T* __restrict__ w, int ldw, T (*acc)[NR]) {
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
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const T x = w[r * ldw + u + s * G];
#pragma unroll
                for (int q2 = 0; q2 < NA; ++q2)
                    if (li + 32 * q2 < cnt) acc[q2][r] += v[s][q2] * x;
            }
        }
    }
    for (; u < units; u += G) {
        const T* row = P + (long long)u * ldp;
#pragma unroll
        for (int q2 = 0; q2 < NA; ++q2) {
            const int l = li + 32 * q2;
            if (l < cnt) {
                const T pv = __ldcs(row + l);
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[q2][r] += pv * w[r * ldw + u];
            }
        }
    }
}

// Minimum resident blocks per SM of the warp kernel (a register budget per
// instance): the FP64 single-column instance is held to 64 registers (8
// blocks, 32 items per SM) without spilling; the others get the budgets they
// fit without spilling.
template <typename T, int NR>
constexpr int warp_min_blocks() {
    return sizeof(T) == 8 ? (NR == 1 ? 8 : (NR == 2 ? 5 : 4)) : (NR == 1 ? 10 : (NR == 2 ? 9 : 7));
}

template <typename T, int NR>
__global__ void __launch_bounds__(128, warp_min_blocks<T, NR>()) tree_solve_warp_kernel(const T* __restrict__ Q, TreeArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int ldw = a.max_n;
    T* w = reinterpret_cast<T*>(smem_raw) + (size_t)(threadIdx.x >> 5) * NR * ldw;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        const int claimed = __shfl_sync(FULL, item, 0);
        if (claimed >= a.n_items * a.nsplit) return;
        item = claimed / a.nsplit;
        const int grp = claimed - item * a.nsplit;
        double* const y = a.y + (long long)grp * NR * a.ldy;
        double* const w1 = a.w1 + (long long)grp * NR * a.ldy;
        double* const upd = a.upd + (long long)grp * NR * a.upd_size;
        int* const done_f = a.done_f + (long long)grp * a.n_fronts;
        int* const done_b = a.done_b + (long long)grp * a.n_fronts;
        const SolveItem it = a.items[item];
        const bool fwd = item < a.n_fwd;
        const int F = it.front, k = it.k, n = it.n, b0 = it.b0, m = n - k;
        const int lo = it.lo, cnt = it.hi - it.lo, ldp = it.ldp;
        const T* q = Q + it.off;
        const int units = fwd ? k : n;  // rows (forward) or columns (backward) of the panel
        if (lane == 0) {
            if (a.trace) {
                a.trace[4 * claimed] = sm_id();
                a.trace[4 * claimed + 1] = global_ns();
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
                ok = ok && wait_count(&done_f[cr.child], cr.parts, a.err, a.spin_limit);
            }
        } else if (lane == 0) {
            ok = wait_count(&done_f[F], it.wait_parts, a.err, a.spin_limit);
            if (ok && it.parent >= 0) ok = wait_count(&done_b[it.parent], it.parent_parts, a.err, a.spin_limit);
        }
        if (!__all_sync(FULL, ok)) return;
        __threadfence();
        if (a.trace && lane == 0) a.trace[4 * claimed + 2] = global_ns();
        if (fwd) {
            // w = [b(own); 0] + children's update vectors
            for (int r = 0; r < NR; ++r)
                for (int i = lane; i < n; i += 32)
                    w[r * ldw + i] = (i < k) ? (T)__ldcg(&y[(long long)r * a.ldy + b0 + i]) : T(0);
            __syncwarp();
            for (int ci = it.c0; ci < it.c1; ++ci) {
                const ChildRec cr = a.crec[ci];
                const int* rl = a.rel + cr.rel_off;
                const double* u = upd + cr.upd_off * NR;
                for (int r = 0; r < NR; ++r)
                    for (int i = lane; i < cr.m; i += 32) w[r * ldw + rl[i]] += (T)__ldcg(&u[(long long)r * cr.m + i]);
                __syncwarp();
            }
            if (lo == k)  // the first part keeps w1 = w(own) for the backward sweep
                for (int r = 0; r < NR; ++r)
                    for (int i = lane; i < k; i += 32) w1[(long long)r * a.ldy + b0 + i] = (double)w[r * ldw + i];
        } else {
            const int* idx = a.front_pos + it.fpos;
            for (int r = 0; r < NR; ++r)
                for (int i = lane; i < n; i += 32)
                    w[r * ldw + i] = (i < k) ? -(T)__ldcg(&w1[(long long)r * a.ldy + b0 + i])
                                             : (T)__ldcg(&y[(long long)r * a.ldy + idx[i]]);
        }
        __syncwarp();
        // lanes: outputs li (cp per unit group) x unit groups g (G = 32 / cp)
        const int cp = cnt > 16 ? 32 : (cnt > 8 ? 16 : (cnt > 4 ? 8 : 4));
        const int G = 32 / cp, li = lane % cp, g = lane / cp;
        const int na = (cnt + 31) / 32;
        T acc[4][NR];
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2)
#pragma unroll
            for (int r = 0; r < NR; ++r) acc[q2][r] = T(0);
        if (cnt > 0) {
            switch (na) {
                case 1: warp_accumulate<T, 1, (NR == 1 ? 16 : 8), NR>(q, ldp, units, g, G, li, cnt, w, ldw, acc); break;
                case 2: warp_accumulate<T, 2, (NR == 1 ? 8 : 4), NR>(q, ldp, units, g, G, li, cnt, w, ldw, acc); break;
                case 3: warp_accumulate<T, 3, 4, NR>(q, ldp, units, g, G, li, cnt, w, ldw, acc); break;
                default: warp_accumulate<T, 4, 4, NR>(q, ldp, units, g, G, li, cnt, w, ldw, acc); break;
            }
            for (int o = cp; o < 32; o <<= 1)
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[0][r] += __shfl_xor_sync(FULL, acc[0][r], o);
            if (g == 0) {
#pragma unroll
                for (int q2 = 0; q2 < 4; ++q2) {
                    const int l = li + 32 * q2;
                    if (q2 < na && l < cnt) {
#pragma unroll
                        for (int r = 0; r < NR; ++r) {
                            if (fwd) upd[it.upd_off * NR + (long long)r * m + lo + l - k] =
                                         (double)(w[r * ldw + lo + l] + acc[q2][r]);
                            else y[(long long)r * a.ldy + b0 + lo + l] = (double)acc[q2][r];
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicAdd(fwd ? &done_f[F] : &done_b[F], 1);
            if (a.trace) a.trace[4 * claimed + 3] = global_ns();
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
    double s = 0.0;
    if (row < N)
        for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += LANES) {
            double a = which == 0 ? Mv[e] : (which == 1 ? Kv[e] : Kv[e] - shift * Mv[e]);
            s += a * x[col[e]];
        }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, LANES);  // every lane takes part
    if (row < N && lane == 0) y[row] = s;
}

// r = b - (K - shift M) x (SPMV_TPR lanes per row)
__global__ void residual_kernel(long long N, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ Kv, const double* __restrict__ Mv, double shift,
                                const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ r) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = t / SPMV_TPR;
    const int lane = (int)(t % SPMV_TPR);
    double s = 0.0;
    if (row < N)
        for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) s += (Kv[e] - shift * Mv[e]) * x[col[e]];
    s = group_sum(s);  // every lane of the warp takes part
    if (row < N && lane == 0) r[row] = b[row] - s;
}

// the same residual with a shift per position (a batch: each problem of the
// forest has its own shift; entry (row, col) shares row's problem)
__global__ void residual_pos_kernel(long long N, const long long* __restrict__ rowptr, const int* __restrict__ col,
                                    const double* __restrict__ Kv, const double* __restrict__ Mv,
                                    const double* __restrict__ sig_pos, const double* __restrict__ x,
                                    const double* __restrict__ b, double* __restrict__ r) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long row = t / SPMV_TPR;
    const int lane = (int)(t % SPMV_TPR);
    double s = 0.0;
    const double shift = row < N ? sig_pos[row] : 0.0;
    if (row < N)
        for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) s += (Kv[e] - shift * Mv[e]) * x[col[e]];
    s = group_sum(s);  // every lane of the warp takes part
    if (row < N && lane == 0) r[row] = b[row] - s;
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


// Shared memory of the tree solve (and its chunk size, threads, slots).  The
// NR > 1 kernels take a symbolic analysis only when every part's panel
// arrives in one copy (the extra output passes re-read it from shared
// memory) and the front vectors of NR right-hand sides fit.
// Small fronts (2D trees, 128-thread CTAs): panel slots per CTA and the
// largest chunk half (elements) for one right-hand side.
constexpr int SMALL_SLOTS = 1;
constexpr long long SMALL_CHUNK = 3072;

static size_t solve_smem(const Symbolic& S, int nr, size_t elem, int* chunk_out, int* nt_out, int* nslot_out = nullptr) {
    int max_n = 0, max_ldp = 0;
    for (int f = 0; f < S.n_nodes; ++f) max_n = std::max(max_n, S.n[f]);
    for (const SolveItem& it : S.sitems) max_ldp = std::max(max_ldp, it.ldp);
    const int nt = S.solve_mode == SOLVE_CTA256 ? 256 : 128;
    // small fronts: halves of 2048..3072 elements (NR > 1: as large as the
    // largest panel needs), so that every part's panel arrives in one copy;
    // large fronts: halves of up to 32 KiB, sized so that the CTAs of an SM
    // fit: FP32 panels three CTAs with two slots each (the next item's
    // copies run while the current item computes), FP64 panels (whose front
    // vectors take twice the room) two CTAs with one slot
    const bool large = S.solve_mode == SOLVE_CTA256;
    const int nslot = large ? (elem == 4 ? 2 : 1) : SMALL_SLOTS;
    const int ctas = large && elem == 4 ? 3 : 2;
    const long long fixed = ((long long)nr * max_n + (long long)nt * nr + 8) * (long long)elem;
    const long long budget = 227LL * 1024 / ctas - 2048;
    const long long half_max = std::max<long long>(8192, std::min<long long>(32768, (budget - fixed) / (2 * nslot)));
    long long chunk = S.solve_mode == SOLVE_CTA128
                          ? std::max<long long>(2048, (S.max_panel + 1) / 2)
                          : half_max / (long long)elem;
    if (S.solve_mode == SOLVE_CTA128 && nr == 1) chunk = std::min<long long>(chunk, SMALL_CHUNK);
    chunk = std::max<long long>(chunk, max_ldp);
    chunk = (chunk + 3) / 4 * 4;
    *chunk_out = (int)chunk;
    *nt_out = nt;
    if (nslot_out) *nslot_out = nslot;
    if (S.solve_mode == SOLVE_WARP) return 4 * (size_t)nr * max_n * elem;
    return (2 * (size_t)nslot * chunk + (size_t)nr * max_n + (size_t)nt * nr + 8) * elem;
}

int solve_max_rhs(riga_ctx* c) {
    const Symbolic& S = c->S;
    if (S.solve_mode != SOLVE_WARP) return 4;  // interleaved groups: any count, up to 8 per launch
    int maxopt = 0;
    if (cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device) != cudaSuccess) return 1;
    const size_t elem = sizeof(double);  // the larger of the two front precisions
    for (int nr : {4, 2}) {
        int chunk = 0, nt = 0;
        const size_t smem = solve_smem(S, nr, elem, &chunk, &nt);
        if (smem + 256 <= (size_t)maxopt && (S.solve_mode == SOLVE_WARP || 2LL * chunk >= S.max_panel)) return nr;
    }
    return 1;
}

// chunk half (elements) and resident CTAs per SM (a register budget) of the
// leaf launches of large-front trees
constexpr int LEAF_CHUNK = 2048;
constexpr int LEAF_MINB = 4;

template <typename T, int NR>
static int enqueue_solve_t(riga_ctx* c, const T* Q, double* y, int nsplit) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    // algorithmic bytes of a forward/backward solve with b right-hand sides:
    // the factor L read once per sweep, 2 nnz(L) s_f, plus four FP64 vector
    // passes, 4 N 8 b (the operator panels this design reads instead hold
    // more entries: the difference counts as overhead, not as work)
    // algorithmic flops: one multiply-add per operator entry and right-hand side
    PhaseScope scope(c, PH_SOLVE,
                     2.0 * (double)S.nnzL * sizeof(T) + 4.0 * NR * nsplit * (double)S.N * sizeof(double),
                     2.0 * (2.0 * (double)S.nnzQ - (double)S.nnzL_own2) * NR * nsplit);
    int max_n = 0;
    for (int f = 0; f < S.n_nodes; ++f) max_n = std::max(max_n, S.n[f]);
    const int n_items = (int)S.sitems.size();
    int maxopt = 0, nsm = 0, chunk = 0, nt = 0;
    RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    int nslot = 1;
    const size_t smem = solve_smem(S, NR, sizeof(T), &chunk, &nt, &nslot);
    const bool warp = S.solve_mode == SOLVE_WARP;
    if (smem + 256 > (size_t)maxopt) return set_error(c, RIGA_EINVAL, "front too large for the shared-memory solve");
    if (NR > 1 && (S.solve_mode == SOLVE_CTA256 || (!warp && 2LL * chunk < S.max_panel)))
        return set_error(c, RIGA_EINVAL, "several right-hand sides need whole-panel copies");
    auto kern = warp ? tree_solve_warp_kernel<T, NR>
                     : (S.solve_mode == SOLVE_CTA128 ? tree_solve_kernel<T, 128, NR> : tree_solve_kernel<T, 256, NR>);
    RIGA_CUDA_TRY(c, cudaMemsetAsync(c->solve_flags.ptr, 0, (2 * (size_t)S.n_nodes * nsplit + 3) * sizeof(int), st));
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
    a.item0 = 0;
    a.n_items = n_items;
    a.n_fwd = S.n_fwd_items;
    a.chunk_elems = chunk;
    a.nslot = nslot;
    a.max_n = max_n;
    a.upd = c->upd.ptr;
    a.y = y;
    a.ldy = S.N;
    a.w1 = c->w1buf.ptr;
    a.nsplit = nsplit;
    a.n_fronts = S.n_nodes;
    a.upd_size = S.upd_size;
    a.done_f = c->solve_flags.ptr;
    a.done_b = c->solve_flags.ptr + (size_t)S.n_nodes * nsplit;
    a.counter = c->solve_flags.ptr + 2 * (size_t)S.n_nodes * nsplit;
    a.err = c->flag.ptr;
    a.spin_limit = c->wait_limit;
    a.trace = c->trace_buf;
    // one launch over items [i0, i0 + cnt) with the given configuration and counter
    auto launch = [&](void (*k)(const T*, TreeArgs), int i0, int cnt, size_t sm, int ch, int ns, int mx,
                      int ctr) -> int {
        if (cnt <= 0) return RIGA_OK;
        int occ = 0;
        if (sm > 48 * 1024) RIGA_CUDA_TRY(c, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        RIGA_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nt, sm));
        const int per_block = warp ? 4 : 1;  // concurrent items per block
        const long long work = (long long)cnt * nsplit;
        const int grid = (int)std::max<long long>(1, std::min<long long>((work + per_block - 1) / per_block, std::max(1, occ) * nsm));
        TreeArgs b = a;
        b.item0 = i0;
        b.n_items = cnt;
        b.chunk_elems = ch;
        b.nslot = ns;
        b.max_n = mx;
        b.counter = a.counter + ctr;
        { count_launch(c); k<<<grid, nt, sm, st>>>(Q, b); }
        return RIGA_OK;
    };
    // Trees of large FP64 fronts: the fronts of the lowest levels (forward
    // parts wait only for earlier parts of the same launch, backward parts
    // also for the launch before) run in launches of their own whose short
    // front vectors let four CTAs
    // share an SM (a kernel instance held to 64 registers), so that one
    // CTA's arithmetic covers another's copies, gathers and reductions; the
    // fronts above run in between with the long front vectors, two CTAs per
    // SM.  Chunk 2048 and four CTAs were the best of a sweep on the 64^3
    // p = 2 mesh (one right-hand side: 2.58 ms, against 2.60-2.97 ms for
    // chunks 768-2048 and three or four CTAs).
    int f0 = 0, b0 = 0, leaf_n = 0, lchunk = 0;
    size_t lsmem = 0;
    if (S.solve_mode == SOLVE_CTA256 && sizeof(T) == sizeof(double) && NR == 1) {
        // the lowest levels whose front vectors still let four CTAs share an SM
        // (228 KiB of shared memory per SM, 1 KiB of it reserved per CTA)
        const size_t cap = (size_t)228 * 1024 / LEAF_MINB - 2048;
        for (int hs = 0; hs < S.n_levels; ++hs) {
            int mn = 0, ml = 0;
            for (int i = 0; i < n_items; ++i)
                if (S.height[S.sitems[i].front] <= hs) {
                    mn = std::max(mn, S.n[S.sitems[i].front]);
                    ml = std::max(ml, S.sitems[i].ldp);
                }
            const int ch = std::max(LEAF_CHUNK, (ml + 3) / 4 * 4);
            const size_t sm = (size_t)(2LL * ch + (long long)NR * mn + (long long)nt * NR + 8) * sizeof(T);
            if (sm > cap) break;
            int ff = 0, bb = 0;
            while (ff < S.n_fwd_items && S.height[S.sitems[ff].front] <= hs) ++ff;
            while (bb < n_items - S.n_fwd_items && S.height[S.sitems[n_items - 1 - bb].front] <= hs) ++bb;
            f0 = ff;
            b0 = bb;
            leaf_n = mn;
            lchunk = ch;
            lsmem = sm;
        }
    }
    if (f0 > 0 && b0 > 0 && f0 + b0 < n_items) {
        auto lk = tree_solve_kernel<T, 256, NR, LEAF_MINB>;
        int rc = launch(lk, 0, f0, lsmem, lchunk, 1, leaf_n, 0);
        if (rc == RIGA_OK) rc = launch(kern, f0, n_items - f0 - b0, smem, chunk, nslot, max_n, 1);
        if (rc == RIGA_OK) rc = launch(lk, n_items - b0, b0, lsmem, lchunk, 1, leaf_n, 2);
        return rc;
    }
    return launch(kern, 0, n_items, smem, chunk, nslot, max_n, 0);
}

// y := A^{-1} y for nrhs columns (stride N).  Trees with a critical path
// (one or few problems): the columns run as independent groups of one
// right-hand side interleaved in one launch (up to 8), so that each item
// stays short and the groups share the panels in L2.  Batches of many trees
// (bound by items in flight): up to four columns share each item and each
// panel read.
// Columns that share each item in the 128-thread (2D tree) solve when a
// call carries several right-hand sides (1: interleaved groups instead).
constexpr int SMALL_COMBINED = 1;

int enqueue_solve(riga_ctx* c, double* y, int nrhs) {
    if (!c->factored) return set_error(c, RIGA_ESTATE, "no factorization");
    Symbolic& S = c->S;
    const bool split = S.solve_mode == SOLVE_CTA256 || (S.solve_mode == SOLVE_CTA128 && SMALL_COMBINED == 1);
    const int maxr = split ? 1 : std::min(S.solve_mode == SOLVE_CTA128 ? SMALL_COMBINED : 4, solve_max_rhs(c));
    const int width = split ? std::min(std::max(1, nrhs), 8) : std::min(std::max(1, nrhs), maxr);
    RIGA_CUDA_TRY(c, c->upd.alloc((S.upd_size > 0 ? S.upd_size : 1) * (size_t)width));
    RIGA_CUDA_TRY(c, c->solve_flags.alloc(2 * (size_t)S.n_nodes * width + 3));
    RIGA_CUDA_TRY(c, c->w1buf.alloc((size_t)S.N * width));
    for (int c0 = 0; c0 < nrhs;) {
        const int left = nrhs - c0;
        double* yc = y + (long long)c0 * S.N;
        int rc, used;
        if (split) {
            used = std::min(left, 8);
            rc = c->precision == RIGA_FP64 ? enqueue_solve_t<double, 1>(c, c->q64.ptr, yc, used)
                                           : enqueue_solve_t<float, 1>(c, c->q32.ptr, yc, used);
        } else {
            used = left >= 4 && maxr >= 4 ? 4 : (left >= 2 && maxr >= 2 ? 2 : 1);
            if (c->precision == RIGA_FP64) {
                rc = used == 4 ? enqueue_solve_t<double, 4>(c, c->q64.ptr, yc, 1)
                               : (used == 2 ? enqueue_solve_t<double, 2>(c, c->q64.ptr, yc, 1)
                                            : enqueue_solve_t<double, 1>(c, c->q64.ptr, yc, 1));
            } else {
                rc = used == 4 ? enqueue_solve_t<float, 4>(c, c->q32.ptr, yc, 1)
                               : (used == 2 ? enqueue_solve_t<float, 2>(c, c->q32.ptr, yc, 1)
                                            : enqueue_solve_t<float, 1>(c, c->q32.ptr, yc, 1));
            }
        }
        if (rc) return rc;
        RIGA_CUDA_TRY(c, cudaGetLastError());
        c->stats.n_solve += used;
        c0 += used;
    }
    return RIGA_OK;
}

int enqueue_spmv(riga_ctx* c, int which, const double* x, double* y, double shift) {
    Symbolic& S = c->S;
    long long threads = S.N * SPMV_TPR;
    { count_launch(c); spmv_kernel<SPMV_TPR><<<(unsigned)((threads + 255) / 256), 256, 0, c->stream>>>(S.N, c->rowptr.ptr, c->col.ptr,
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
        // FP64 fronts: plain solves, unless a calibration of this
        // factorization asked for refinement (an interior shift)
        if (c->fp64_sweeps <= 1) {
            if (sweeps_out) *sweeps_out = 1;
            return enqueue_solve(c, y);
        }
        max_sweeps = c->fp64_sweeps;
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
        if (!check && sweeps == max_sweeps) break;  // the last residual is not needed
        long long threads = N * SPMV_TPR;
        if (S.dim == 0 && !c->sigma_prob.empty()) {
            count_launch(c);
            residual_pos_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(N, c->rowptr.ptr, c->col.ptr, c->Kval.ptr,
                                                                                 c->Mval.ptr, c->sig_pos.ptr, x, y, r);
        } else {
            count_launch(c);
            residual_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(N, c->rowptr.ptr, c->col.ptr, c->Kval.ptr,
                                                                             c->Mval.ptr, c->sigma, x, y, r);
        }
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

// y := A^{-1} y for nr columns (stride N) with a low-precision factor: a
// fixed number of refinement sweeps (x = 0, r = y; d = solve(r); x += d;
// r = y - A x), the corrections of all columns in one solve launch per sweep
int solve_refined_multi(riga_ctx* c, double* y, double* x, double* r, int nr, int sweeps) {
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    const long long N = S.N, NN = N * nr;
    if (c->precision == RIGA_FP64) {
        if (c->fp64_sweeps <= 1) return enqueue_solve(c, y, nr);
        sweeps = c->fp64_sweeps;
    }
    RIGA_CUDA_TRY(c, cudaMemsetAsync(x, 0, NN * sizeof(double), st));
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(r, y, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (int s = 1; s <= sweeps; ++s) {
        int rc = enqueue_solve(c, r, nr);
        if (rc) return rc;
        { count_launch(c); axpy_kernel<<<(unsigned)((NN + 255) / 256), 256, 0, st>>>(NN, 1.0, r, x); }
        if (s == sweeps) break;
        const long long threads = N * SPMV_TPR;
        for (int j = 0; j < nr; ++j) {
            count_launch(c);
            residual_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
                N, c->rowptr.ptr, c->col.ptr, c->Kval.ptr, c->Mval.ptr, c->sigma, x + j * N, y + j * N, r + j * N);
        }
    }
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(y, x, NN * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return RIGA_OK;
}

}  // namespace riga
