// Schur-complement update of FP32 fronts on the tensor cores (tcgen05, TF32
// inputs, FP32 accumulation in tensor memory): the dense contraction of the
// multifrontal LDL^T (Sec. 4.2), A22 -= L21 D L21^T, one TC_M x TC_N tile of
// the trailing matrix per CTA and one panel step (K = kb <= 32) per launch.
//
// Precision: each FP32 operand x is split into a TF32 head h (x with the low
// 13 mantissa bits cleared) and a tail t = x - h (exact in FP32); the tile is
// accumulated as A_h B_h + A_h B_t + A_t B_h (three MMAs per K slice), which
// keeps the products to about FP32 accuracy (the dropped A_t B_t term and the
// tail's own TF32 rounding are ~2^-21 relative).
//
// Data path per CTA (128 threads, 4 warps):
//   1. warp 0 allocates 64 TMEM columns (D: 128 lanes x 64 FP32 columns);
//   2. the A (128 rows x 32) and B (64 rows x 32, scaled by D) panels are
//      read from the front with coalesced loads and stored to shared memory
//      in the canonical K-major layout without swizzle: 8-row x 16-byte core
//      matrices, core (m, k) at byte (m * 8 + k) * 128 (LBO = 128 B between
//      K-adjacent cores, SBO = 1024 B between 8-row groups);
//   3. one thread issues the MMAs (K = 8 per instruction) and commits them to
//      an mbarrier; everyone waits on it (bounded);
//   4. each warp loads its 32 lanes of D (tcgen05.ld 32x32b.x64) and applies
//      the update to its rows of the front with the lower-triangle /
//      extra-block masks of the CUDA-core kernel.
#include "ctx.h"

namespace riga {

namespace {

constexpr int KP = 32;                  // panel width (the factorization's NB)
constexpr int CORE_BYTES = 128;         // 8 rows x 16 bytes
constexpr int A_BYTES = TC_M * KP * 4;  // 16 KiB per A operand
constexpr int B_BYTES = TC_N * KP * 4;  // 8 KiB per B operand

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a K-major, non-swizzled operand tile
__device__ __forceinline__ int kmajor_off(int row, int k) {
    return ((row >> 3) * (KP / 4) + (k >> 2)) * CORE_BYTES + (row & 7) * 16 + (k & 3) * 4;
}

// shared-memory matrix descriptor: start, LBO, SBO (all >> 4), version 1,
// no swizzle
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major,
// N = TC_N, M = TC_M
constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(TC_N >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mma_tf32(unsigned d_tmem, unsigned long long a, unsigned long long b, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}

}  // namespace

__global__ void __launch_bounds__(128) tc_update_kernel(const TileItem* __restrict__ items, int p0,
                                                        const int* __restrict__ kk, const int* __restrict__ nn,
                                                        const long long* __restrict__ front_off,
                                                        const int* __restrict__ node_ptr, const double* __restrict__ D,
                                                        float* __restrict__ pool, int plain, int* __restrict__ err,
                                                        long long spin_limit) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* Ah = sm;
    unsigned char* At = Ah + A_BYTES;
    unsigned char* Bh = At + A_BYTES;
    unsigned char* Bt = Bh + B_BYTES;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    const TileItem it = items[blockIdx.x];
    const int F = it.front, k = kk[F], n = nn[F], ld = n + k;
    const bool skip = plain && (it.i0 >= n || it.j0 >= n);  // plain: tiles touching only extra rows
    const int kb = min(KP, k - p0);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operands: A rows i0.., B rows j0.. (times the pivots), zero outside
    const float* A = pool + front_off[F];
    const double* d = D + node_ptr[F] + p0;
    for (int e = tid; e < TC_M * KP; e += 128) {
        const int r = e % TC_M, t = e / TC_M;  // consecutive threads: consecutive rows (coalesced)
        const int gi = it.i0 + r;
        const float x = (!skip && t < kb && gi < ld) ? A[(long long)(p0 + t) * ld + gi] : 0.f;
        const float h = tf32_head(x);
        *reinterpret_cast<float*>(Ah + kmajor_off(r, t)) = h;
        *reinterpret_cast<float*>(At + kmajor_off(r, t)) = x - h;
    }
    for (int e = tid; e < TC_N * KP; e += 128) {
        const int r = e % TC_N, t = e / TC_N;
        const int gj = it.j0 + r;
        const float x = (!skip && t < kb && gj < ld) ? A[(long long)(p0 + t) * ld + gj] * (float)d[t] : 0.f;
        const float h = tf32_head(x);
        *reinterpret_cast<float*>(Bh + kmajor_off(r, t)) = h;
        *reinterpret_cast<float*>(Bt + kmajor_off(r, t)) = x - h;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;

    if (tid == 0) {
        const unsigned lbo = CORE_BYTES, sbo = (KP / 4) * CORE_BYTES;
        const unsigned ah = smem_addr(Ah), at = smem_addr(At), bh = smem_addr(Bh), bt = smem_addr(Bt);
        int acc = 0;
        for (int ks = 0; ks < KP / 8; ++ks) {  // K = 8 per instruction: two cores along K
            const unsigned off = ks * 2 * CORE_BYTES;
            mma_tf32(tmem, smem_desc(ah + off, lbo, sbo), smem_desc(bh + off, lbo, sbo), acc);
            acc = 1;
            mma_tf32(tmem, smem_desc(ah + off, lbo, sbo), smem_desc(bt + off, lbo, sbo), 1);
            mma_tf32(tmem, smem_desc(at + off, lbo, sbo), smem_desc(bh + off, lbo, sbo), 1);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_addr(&mbar))
                     : "memory");
    }
    // bounded wait for the MMAs (phase 0)
    {
        long long n_poll = 0;
        unsigned ok = 0;
        while (true) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(ok)
                : "r"(smem_addr(&mbar))
                : "memory");
            if (ok) break;
            if (++n_poll > spin_limit) {
                if (tid == 0) atomicOr(err, 4);
                break;
            }
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w owns TMEM lanes 32w..32w+31 = tile rows 32w + lane
    float acc[TC_N];
    {
        const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16);
        unsigned* r = reinterpret_cast<unsigned*>(acc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
            "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
            "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
            "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
            "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
              "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
              "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
              "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
              "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    }
    if (!skip) {
        float* Af = pool + front_off[F];
        const int gi = it.i0 + warp * 32 + (tid & 31);
        if (gi < ld && !(plain && gi >= n)) {
#pragma unroll 8
            for (int c = 0; c < TC_N; ++c) {
                const int gj = it.j0 + c;
                if (gj < ld && (gi >= gj || (gi >= n && gj >= n))) Af[(long long)gj * ld + gi] -= acc[c];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N) : "memory");
}

size_t tc_update_smem() { return (size_t)2 * A_BYTES + (size_t)2 * B_BYTES + 1024; }

}  // namespace riga
