// Schur-complement update of FP32 fronts on the tensor cores (tcgen05 with
// FP32 accumulation in tensor memory): the dense contraction of the
// multifrontal LDL^T (Sec. 4.2), A22 -= L21 D L21^T, once per super-panel of
// up to TC_KW = 64 columns (two panel steps accumulated in TMEM before the
// trailing tile is reduced once), for every front of a tree level.
//
// Precision.  Each FP32 operand x is split into a head h and a tail
// t = x - h and the tile is accumulated as A_h B_h + A_h B_t + A_t B_h (three
// MMAs per K slice):
//   TF32 mode: h = x with the low 13 mantissa bits cleared (kind::tf32); the
//              dropped A_t B_t term and the tail's own rounding are ~2^-21
//              relative, about FP32 accuracy;
//   BF16 mode: h = bf16(x), t = bf16(x - h) (kind::f16 with BF16 inputs);
//              ~2^-16 relative.  Each packed 128-row block is scaled by a
//              power of two so that its largest magnitude is in [0.5, 1)
//              before the split (the tail of a tiny block stays normal), and
//              the epilogue removes the two blocks' scales exactly.
//
// Data path of one super-panel update:
//   tc_pack_kernel    the trailing rows of each front's super-panel (and the
//                     same times the pivots) in 128-row blocks, one packed
//                     block per 32-column chunk: read once, split once,
//                     written in the MMA's shared-memory layout (K-major 8-row
//                     core matrices, no swizzle), 4 operand arrays per block
//                     (A head, A tail, B head, B tail);
//   tc_update_kernel  persistent, one CTA per SM, 192 threads in three roles:
//     warp 4   producer: for each of the CTA's tiles and each 32-column
//              chunk one bulk copy per operand array (cp.async.bulk, 16-byte
//              aligned, completion counted in bytes on an mbarrier) into one
//              of two shared-memory stages;
//     warp 5   MMA issuer: per chunk 12 (TF32) or 6 (BF16) tcgen05.mma into
//              one of two 128 x 128 FP32 accumulators in tensor memory (256
//              columns) and tcgen05.commit to free the stage; after the
//              tile's last chunk a commit hands the accumulator to the
//              epilogue;
//     warps 0-3 epilogue: tcgen05.ld of the accumulator (warp w reads lanes
//              32w..32w+31 = tile rows), release it, then C -= acc on the
//              front (lower triangle, and the whole extra x extra block of the
//              augmented front) by reductions in L2, coalesced along the rows.
//   Every wait is bounded: on expiry the kernel sets bit 2 of the error word,
//   every role stops, in-flight copies and MMAs are waited for (bounded) and
//   the tensor memory is freed.
#include <cuda_bf16.h>

#include "ctx.h"
#include "tc_common.cuh"

namespace riga {

namespace {

constexpr int KP = 32;                         // panel width (the factorization's NB)
constexpr int ARR = TC_BLK * KP;               // floats per operand array slot (16 KiB)
constexpr int BLK_FLOATS = 4 * ARR;            // one packed block: A head, A tail, B head, B tail
constexpr unsigned STAGE_BYTES = 4u * ARR * 4u;  // 64 KiB per shared-memory stage
constexpr int NSTAGE = 2;
constexpr int UPD_THREADS = 192;
constexpr int TMEM_COLS = 2 * TC_N;            // two accumulators

using namespace tcx;

constexpr unsigned IDESC_TF32 = make_idesc(2, TC_M, TC_N);
constexpr unsigned IDESC_BF16 = make_idesc(1, TC_M, TC_N);

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <int MODE>
__device__ __forceinline__ void mma(unsigned d_tmem, unsigned long long a, unsigned long long b, int acc) {
    if (MODE == 0) mma_tf32(d_tmem, a, b, IDESC_TF32, acc);
    else mma_f16(d_tmem, a, b, IDESC_BF16, acc);
}

// power of two s with s * amax in [0.5, 1) (1 for a zero block)
__device__ __forceinline__ float pow2_scale(float amax) {
    if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
    int e;
    frexpf(amax, &e);  // amax = f 2^e, f in [0.5, 1)
    return ldexpf(1.f, -e);
}

}  // namespace

// One 256-thread block per packed row block: rows r0..r0+127 of the front's
// super-panel (columns p0..p0+kw, kw = min(TC_KW, k - p0)), one packed block
// per 32-column chunk (blocks blk, blk+1, ...), and the same rows times the
// pivots.
// TF32 (MODE 0): float entry (r, k) of an array at
//   ((r >> 3) * (KP / 4) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
// BF16 (MODE 1): bf16 entry (r, k) at
//   ((r >> 3) * (KP / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7)
// (one 8-row x 16-byte core matrix per 32 floats / 64 bf16).  Rows beyond the
// front and columns beyond kw are zero.  BF16: one power-of-two scale for A
// and one for B over all chunks of the row block (the chunks accumulate into
// one tile), scale[2 blk] and scale[2 blk + 1].
template <int MODE>
__global__ void __launch_bounds__(256) tc_pack_kernel(const TcPack* __restrict__ items,
                                                      const int* __restrict__ kk, const int* __restrict__ nn,
                                                      const long long* __restrict__ front_off,
                                                      const int* __restrict__ node_ptr, const double* __restrict__ D,
                                                      const float* __restrict__ pool, float* __restrict__ pack,
                                                      float* __restrict__ scale) {
    __shared__ float Ts[KP][TC_BLK + 1];
    __shared__ float ds[KP];
    __shared__ float red[2][8];
    const TcPack it = items[blockIdx.x];
    const int F = it.front, k = kk[F], ld = nn[F] + k;
    const int kw = min(TC_KW, k - it.p0);
    const int nk = (kw + KP - 1) / KP;
    const float* A = pool + front_off[F];
    const int tid = threadIdx.x;
    float sa = 1.f, sb = 1.f;
    if (MODE == 1) {
        // scales over every chunk of the row block (a first pass over global memory)
        float ma = 0.f, mb = 0.f;
        for (int e = tid; e < kw * TC_BLK; e += 256) {
            const int t = e / TC_BLK, r = e % TC_BLK, gi = it.r0 + r;
            if (gi < ld) {
                const float x = A[(long long)(it.p0 + t) * ld + gi];
                ma = fmaxf(ma, fabsf(x));
                mb = fmaxf(mb, fabsf(x * (float)D[node_ptr[F] + it.p0 + t]));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ma = fmaxf(ma, __shfl_xor_sync(0xffffffffu, ma, o));
            mb = fmaxf(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = ma;
            red[1][tid >> 5] = mb;
        }
        __syncthreads();
        if (tid == 0) {
            float a = 0.f, b = 0.f;
            for (int w = 0; w < 8; ++w) {
                a = fmaxf(a, red[0][w]);
                b = fmaxf(b, red[1][w]);
            }
            red[0][0] = pow2_scale(a);
            red[1][0] = pow2_scale(b);
            scale[2 * it.blk] = red[0][0];
            scale[2 * it.blk + 1] = red[1][0];
        }
        __syncthreads();
        sa = red[0][0];
        sb = red[1][0];
    }
    for (int ch = 0; ch < nk; ++ch) {
        const int p0 = it.p0 + ch * KP;
        const int kb = min(KP, k - p0);
        __syncthreads();  // the previous chunk's reads of Ts are done
        if (tid < KP) ds[tid] = tid < kb ? (float)D[node_ptr[F] + p0 + tid] : 0.f;
        for (int e = tid; e < KP * TC_BLK; e += 256) {
            const int t = e / TC_BLK, r = e % TC_BLK, gi = it.r0 + r;
            Ts[t][r] = (t < kb && gi < ld) ? A[(long long)(p0 + t) * ld + gi] : 0.f;
        }
        __syncthreads();
        float* out = pack + (long long)(it.blk + ch) * BLK_FLOATS;
        if (MODE == 0) {
            for (int q = tid; q < ARR / 4; q += 256) {
                const int r = ((q >> 6) << 3) | (q & 7), k4 = (q >> 3) & 7;
                float ah[4], at[4], bh[4], bt[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float x = Ts[4 * k4 + j][r];
                    const float y = x * ds[4 * k4 + j];
                    ah[j] = tf32_head(x);
                    at[j] = x - ah[j];
                    bh[j] = tf32_head(y);
                    bt[j] = y - bh[j];
                }
                reinterpret_cast<float4*>(out)[q] = make_float4(ah[0], ah[1], ah[2], ah[3]);
                reinterpret_cast<float4*>(out + ARR)[q] = make_float4(at[0], at[1], at[2], at[3]);
                reinterpret_cast<float4*>(out + 2 * ARR)[q] = make_float4(bh[0], bh[1], bh[2], bh[3]);
                reinterpret_cast<float4*>(out + 3 * ARR)[q] = make_float4(bt[0], bt[1], bt[2], bt[3]);
            }
        } else {
            for (int q = tid; q < ARR / 8; q += 256) {  // 16-byte units: 8 bf16 of one row
                const int r = ((q >> 5) << 3) | (q & 7), k8 = (q >> 3) & 3;
                __nv_bfloat16 ah[8], at[8], bh[8], bt[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float x = Ts[8 * k8 + j][r] * sa;
                    const float y = Ts[8 * k8 + j][r] * ds[8 * k8 + j] * sb;
                    ah[j] = __float2bfloat16_rn(x);
                    at[j] = __float2bfloat16_rn(x - __bfloat162float(ah[j]));
                    bh[j] = __float2bfloat16_rn(y);
                    bt[j] = __float2bfloat16_rn(y - __bfloat162float(bh[j]));
                }
                reinterpret_cast<uint4*>(out)[q] = *reinterpret_cast<const uint4*>(ah);
                reinterpret_cast<uint4*>(out + ARR)[q] = *reinterpret_cast<const uint4*>(at);
                reinterpret_cast<uint4*>(out + 2 * ARR)[q] = *reinterpret_cast<const uint4*>(bh);
                reinterpret_cast<uint4*>(out + 3 * ARR)[q] = *reinterpret_cast<const uint4*>(bt);
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(UPD_THREADS, 1) tc_update_kernel(
    const TcTile* __restrict__ tiles, int ntiles, const int* __restrict__ kk, const int* __restrict__ nn,
    const long long* __restrict__ front_off, const float* __restrict__ pack, const float* __restrict__ scale,
    float* __restrict__ pool, int plain, int* __restrict__ err, long long spin_limit) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long full[NSTAGE], empty[NSTAGE], tfull[2], tempty[2], drain;
    __shared__ unsigned s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the dynamic shared memory must start on a 1024-byte boundary (descriptor base offset 0)
    unsigned char* stage0 = sm + ((1024u - (smem_addr(sm) & 1023u)) & 1023u);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 4 * 32);
        }
        mbar_init(&drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    constexpr unsigned ARR_BYTES = MODE == 0 ? ARR * 4u : ARR * 2u;  // bytes of one operand array

    if (warp == 4) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            int it = 0;  // chunks issued
            bool stop = false;
            for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
                const TcTile tl = tiles[t];
                for (int kc = 0; kc < tl.nk; ++kc, ++it) {
                    const int s = it % NSTAGE;
                    const unsigned ph = (unsigned)(it / NSTAGE) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, &s_abort, err, spin_limit)) {
                        stop = true;
                        break;
                    }
                    const float* pa = pack + (long long)(tl.a_blk + kc) * BLK_FLOATS;
                    const float* pb = pack + (long long)(tl.b_blk + kc) * BLK_FLOATS;
                    unsigned char* st = stage0 + (size_t)s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], 4u * ARR_BYTES);
                    bulk_copy(st, pa, ARR_BYTES, &full[s]);
                    bulk_copy(st + ARR * 4, pa + ARR, ARR_BYTES, &full[s]);
                    bulk_copy(st + 2 * ARR * 4, pb + 2 * ARR, ARR_BYTES, &full[s]);
                    bulk_copy(st + 3 * ARR * 4, pb + 3 * ARR, ARR_BYTES, &full[s]);
                }
            }
            // every copy issued has landed before the CTA may exit: wait for
            // the last phase of each stage that was used (bounded)
            for (int q = 0; q < NSTAGE && q < it; ++q) {
                const int last = it - 1 - q;
                const int s = last % NSTAGE;
                long long n = 0;
                while (!mbar_test(&full[s], (unsigned)(last / NSTAGE) & 1u) && ++n <= spin_limit) {
                }
            }
        }
    } else if (warp == 5) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int it = 0, tile_it = 0;  // chunks and tiles consumed
            bool stop = false;
            for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++tile_it) {
                const int nk = tiles[t].nk;
                const int b = tile_it & 1;
                const unsigned pb = (unsigned)(tile_it >> 1) & 1u;
                if (!mbar_wait(&tempty[b], pb ^ 1u, &s_abort, err, spin_limit)) break;
                const unsigned d = tmem + (unsigned)(b * TC_N);
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % NSTAGE;
                    const unsigned ph = (unsigned)(it / NSTAGE) & 1u;
                    if (!mbar_wait(&full[s], ph, &s_abort, err, spin_limit)) {
                        stop = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const unsigned base = smem_addr(stage0 + (size_t)s * STAGE_BYTES);
                    const unsigned ah = base, at = base + ARR * 4, bh = base + 2 * ARR * 4, bt = base + 3 * ARR * 4;
                    if (MODE == 0) {
                        // K = 8 per instruction (two 16-byte cores along K)
                        const unsigned lbo = 128, sbo = (KP / 4) * 128;
#pragma unroll
                        for (int ks = 0; ks < KP / 8; ++ks) {
                            const unsigned off = ks * 256;
                            mma<0>(d, smem_desc(ah + off, lbo, sbo), smem_desc(bh + off, lbo, sbo), kc > 0 || ks > 0);
                            mma<0>(d, smem_desc(ah + off, lbo, sbo), smem_desc(bt + off, lbo, sbo), 1);
                            mma<0>(d, smem_desc(at + off, lbo, sbo), smem_desc(bh + off, lbo, sbo), 1);
                        }
                    } else {
                        // K = 16 per instruction (two 16-byte cores along K)
                        const unsigned lbo = 128, sbo = (KP / 8) * 128;
#pragma unroll
                        for (int ks = 0; ks < KP / 16; ++ks) {
                            const unsigned off = ks * 256;
                            mma<1>(d, smem_desc(ah + off, lbo, sbo), smem_desc(bh + off, lbo, sbo), kc > 0 || ks > 0);
                            mma<1>(d, smem_desc(ah + off, lbo, sbo), smem_desc(bt + off, lbo, sbo), 1);
                            mma<1>(d, smem_desc(at + off, lbo, sbo), smem_desc(bh + off, lbo, sbo), 1);
                        }
                    }
                    mma_commit(&empty[s]);  // the stage is free once these MMAs have read it
                }
                if (stop) break;
                mma_commit(&tfull[b]);  // the accumulator holds the tile's whole super-panel
            }
            // all MMAs issued by this thread have completed (bounded)
            mma_commit(&drain);
            long long n = 0;
            while (!mbar_test(&drain, 0u) && ++n <= spin_limit) {
            }
        }
    } else {
        // ----------------------------------------------- epilogue (warps 0-3)
        int it = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int b = it & 1;
            const unsigned pb = (unsigned)(it >> 1) & 1u;
            // warp-uniform outcome: tcgen05.ld below is a .sync.aligned warp instruction
            const bool ok = mbar_wait(&tfull[b], pb, &s_abort, err, spin_limit);
            if (!__all_sync(0xffffffffu, ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            float acc[TC_N];
            const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(b * TC_N);
#pragma unroll
            for (int ch = 0; ch < TC_N / 32; ++ch) tmem_ld32(taddr + ch * 32, acc + ch * 32);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&tempty[b]);
            const TcTile tl = tiles[t];
            const int F = tl.front, k = kk[F], n = nn[F], ld = n + k;
            if (plain && (tl.i0 >= n || tl.j0 >= n)) continue;  // plain: tiles touching only extra rows
            const float inv = MODE == 0 ? 1.f : 1.f / (scale[2 * tl.a_blk] * scale[2 * tl.b_blk + 1]);
            const int gi = tl.i0 + warp * 32 + lane;
            if (gi >= ld || (plain && gi >= n)) continue;
            // C -= acc as fire-and-forget reductions (red.global.add.f32):
            // every entry receives exactly one addition per panel step (the
            // tiles are disjoint), so the result is that of a read-modify-
            // write, deterministic, without a load latency per column
            float* Af = pool + front_off[F] + gi;
            const int cmax = min(TC_N, ld - tl.j0);
#pragma unroll
            for (int cc = 0; cc < TC_N; ++cc) {
                const int gj = tl.j0 + cc;
                if (cc < cmax && (gi >= gj || (gi >= n && gj >= n))) atomicAdd(Af + (long long)gj * ld, -acc[cc] * inv);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

size_t tc_update_smem() { return (size_t)NSTAGE * STAGE_BYTES + 1024; }
long long tc_pack_floats_per_block() { return BLK_FLOATS; }

// Pack + super-panel update of one panel step (TF32 or BF16 mode) on the
// given stream (the step's narrow update runs before, in factor.cu).
int enqueue_tc_step(riga_ctx* c, const StepRange& R, int p0, float* pool, int plain, cudaStream_t st) {
    const int npack = R.k_end - R.k_begin, ntiles = R.c_end - R.c_begin;
    (void)p0;
    if (ntiles <= 0 || npack <= 0) return RIGA_OK;
    const bool bf16 = c->precision == RIGA_BF16;
    static int nsm = 0;
    if (nsm == 0 && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) nsm = 0;
    const int grid = std::max(1, std::min(ntiles, nsm > 0 ? nsm : 148));
    count_launch(c);
    if (bf16)
        tc_pack_kernel<1><<<npack, 256, 0, st>>>(c->tcpacks.ptr + R.k_begin, c->kk.ptr, c->nn.ptr, c->front_off.ptr,
                                                 c->node_ptr.ptr, c->D.ptr, pool, c->tcpack.ptr, c->tcscale.ptr);
    else
        tc_pack_kernel<0><<<npack, 256, 0, st>>>(c->tcpacks.ptr + R.k_begin, c->kk.ptr, c->nn.ptr, c->front_off.ptr,
                                                 c->node_ptr.ptr, c->D.ptr, pool, c->tcpack.ptr, c->tcscale.ptr);
    count_launch(c);
    if (bf16)
        tc_update_kernel<1><<<grid, UPD_THREADS, tc_update_smem(), st>>>(
            c->tcitems.ptr + R.c_begin, ntiles, c->kk.ptr, c->nn.ptr, c->front_off.ptr, c->tcpack.ptr, c->tcscale.ptr,
            pool, plain, c->flag.ptr, c->wait_limit);
    else
        tc_update_kernel<0><<<grid, UPD_THREADS, tc_update_smem(), st>>>(
            c->tcitems.ptr + R.c_begin, ntiles, c->kk.ptr, c->nn.ptr, c->front_off.ptr, c->tcpack.ptr, c->tcscale.ptr,
            pool, plain, c->flag.ptr, c->wait_limit);
    return RIGA_OK;
}

// Shared-memory size attributes and the packing buffers (once per schedule)
int prepare_tc(riga_ctx* c) {
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(tc_update_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc_update_smem()));
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(tc_update_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc_update_smem()));
    const long long nblk = std::max<long long>(1, c->S.tc_pack_blocks);
    if (c->tcpack.alloc((size_t)nblk * BLK_FLOATS) != cudaSuccess) return set_error(c, RIGA_ENOMEM, "tensor-core panel blocks");
    RIGA_CUDA_TRY(c, c->tcscale.alloc((size_t)2 * nblk));
    return RIGA_OK;
}

}  // namespace riga
