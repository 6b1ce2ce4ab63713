// FP64-accurate Schur-complement update of FP64 fronts on the tensor cores:
// A22 -= L21 D L21^T of the multifrontal LDL^T (Sec. 4.2), one panel step
// (K = 32) at a time, from exact integer products of 8-bit digit slices (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, here with BF16
// operands and FP32 accumulation in tensor memory).
//
// Balancing.  The operands are L21 |D|^(1/2) and L21 D |D|^(-1/2) rather
// than L21 and L21 D, with |D|^(1/2) rounded to a power of two per column
// (exact scalings whose product is 1): at a shift inside the spectrum a
// near-zero pivot makes its column of L21 huge and leaves that of L21 D
// moderate, and the next pivot the reverse; unbalanced, the row maxima of
// the two operands would come from different columns and their product,
// which sets the error below, would far exceed every product term (a first
// version lost up to 2^9 against FP64 there).  Below, x and y denote the
// balanced entries.
//
// Splitting.  Row i of the panel (32 entries), with e_i the smallest
// integer such that every |x_ik| < 2^e_i, becomes the integer row
// X_ik = round(x_ik 2^(63 - e_i)), |X_ik| < 2^63, written in balanced base
// 256: X_ik = sum_{p=0..7} a_p,ik 256^(7-p), a_0 in [-128, 128], the other
// digits in [-128, 127].  Row j of the other operand likewise (exponent f_j,
// digits b_q,jk).  Then
//   (L21 D L21^T)_ij ~ 2^(e_i + f_j - 126) sum_{p,q} 256^(14-p-q) sum_k a_p,ik b_q,jk.
// Every inner sum is an integer of magnitude at most 32 * 2^14: the BF16
// digits are exact, so are their products, and so is their FP32
// accumulation.  The pairs of one level l = p + q share one accumulator (at
// most 8 pairs: |V_l| <= 8 * 2^19 = 2^22, still exact).  Levels l <= 7 (36
// pairs) are kept.  The dropped levels, the rounding of X and the truncation
// of S below weigh together about 2^-59 of 32 * 2^(e_i + f_j), the bound of
// the entry (an FP64 dot product of length 32 carries up to 32 * 2^-53 of
// it).  Eight levels of 64 columns fill the 512 tensor-memory columns; seven
// (the first version) left 2^-56 and missed residual tolerances of 1e-12 at
// shifts inside the spectrum that the FMA path meets.
//
// Recombination without FP64 arithmetic (GB300 issues FP64 at about 1/60 of
// its FP32 rate): each level sum is read as an integer through one float add
// (V + 1.5 * 2^23 holds V in its low mantissa bits for |V| <= 2^22), the
// eight combine in 64-bit integers to S = floor(sum_l V_l 256^(7-l) / 2^16)
// (|S| < 2^60), and the double -S 2^(e_i + f_j - 54), rounded to nearest
// (ties away from zero), is assembled from S's leading-bit position and the
// two exponents with integer operations, then added to the front by
// red.global.add.f64.
//
// Data path of one panel step:
//   oz_pack_kernel    the trailing rows of each front in 128-row blocks: the
//                     panel's 32 columns read once, the row exponents, the
//                     8 digit slices of L21 and of L21 D written as BF16 in
//                     the MMA's shared-memory layout (K-major 8-row core
//                     matrices, no swizzle; 8 KiB per slice);
//   oz_update_kernel  persistent, one CTA per SM, 576 threads:
//     warp 16  producer: per 128 x 64 tile the A block's 8 slices and the 8
//              slices of the B block's 64-row half (16 bulk copies, 96 KiB)
//              into one of two shared-memory stages;
//     warp 17  MMA issuer: 72 tcgen05.mma (36 digit pairs x K = 32 in two
//              K = 16 instructions) into 8 level accumulators of 128 x 64
//              FP32 (all 512 tensor-memory columns);
//     warps 0-15 epilogue: tcgen05.ld of the 8 levels, 4 columns at a time
//              (warp w: lane quarter w % 4, columns 16 (w / 4) .. + 15),
//              the integer recombination and the FP64 reductions (lower
//              triangle, and the whole extra x extra block of the augmented
//              front).
//   Every wait is bounded: on expiry the kernel sets bit 2 of the error word,
//   every role stops, in-flight copies and MMAs are waited for (bounded) and
//   the tensor memory is freed.
#include "ctx.h"
#include "tc_common.cuh"

namespace riga {

namespace {

using namespace tcx;

constexpr int KP = 32;                                  // panel width
constexpr int NDIG = 8;                                 // digit slices per operand
constexpr unsigned SLICE_BYTES = TC_BLK * KP * 2;       // one slice of a 128-row block (8 KiB of BF16)
constexpr unsigned BLK_BYTES = 2 * NDIG * SLICE_BYTES;  // A slices, then B slices (128 KiB)
constexpr unsigned B_BYTES = OZ_N * KP * 2;             // B slice of a tile: 64 rows (4 KiB)
constexpr unsigned STAGE_BYTES = NDIG * (SLICE_BYTES + B_BYTES);  // 96 KiB
constexpr int NSTAGE = 2;
constexpr int EPI_WARPS = 16;                           // epilogue warps 0..15; producer 16, MMA issuer 17
// accumulator columns per tensor-memory load: 8 levels x 4 columns in
// registers (18 warps of 96 registers: five warps share one SM sub-partition's
// 16K registers)
constexpr int CW = 4;
constexpr int UPD_THREADS = 32 * (EPI_WARPS + 2);
constexpr int NLEV = 8;                                 // levels l = p + q = 0..7
constexpr int TMEM_COLS = 512;                          // NLEV * OZ_N
constexpr unsigned IDESC = make_idesc(1, OZ_M, OZ_N);   // BF16 x BF16 -> FP32, 128 x 64

static_assert(NLEV * OZ_N <= TMEM_COLS, "level accumulators exceed the tensor memory");

// Integer X = round(x 2^(s + 63 - e)) for |x 2^s| < 2^e, from the bits of x
// (no FP64 arithmetic): x = m 2^(E - 1075), m = 2^52 + mantissa.  Zero and
// subnormal x give 0 (an error below 2^-1022); *bad is set for a non-finite x.
__device__ __forceinline__ long long to_fixed(double x, int s, int e, bool* bad) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((u >> 52) & 0x7FF);
    if (E == 0) return 0;
    if (E == 0x7FF) {
        *bad = true;
        return 0;
    }
    const unsigned long long m = (u & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = E + s - 1075 + 63 - e;  // X = m 2^sh, sh <= 10 (X < 2^63)
    long long X;
    if (sh >= 0) X = (long long)(m << sh);
    else if (sh < -54) X = 0;
    else X = (long long)((m + (1ull << (-sh - 1))) >> (-sh));  // round half away from zero
    return (u >> 63) ? -X : X;
}

// BF16 bits of a small integer d (|d| <= 128): the float d is exact after
// one add (magic number 1.5 * 2^23), and its top 16 bits are its BF16 value
__device__ __forceinline__ unsigned bf16_of_int(int d) {
    const float f = __int_as_float(0x4B400000 + d) - 12582912.0f;
    return __float_as_uint(f) >> 16;
}

// An inertia-only factorization (plain) has no extra rows to update: its
// tiles that start in them are skipped by all three roles alike
// Tiles whose A block or B half is all zero (live flags of the pack) are
// skipped the same way.
__device__ __forceinline__ bool skip_tile(const TcTile& tl, const int* nn, const int* live, int plain) {
    if (!(live[tl.a_blk] & 1) || !(live[tl.b_blk] & (2 << tl.nk))) return true;
    if (!plain) return false;
    const int n = nn[tl.front];
    return tl.i0 >= n || tl.j0 >= n;
}

constexpr int NOEXP = -(1 << 20);  // exponent of zero (below every scaled exponent)

// exponent field of x 2^s (x normal), NOEXP for zero and subnormal x
__device__ __forceinline__ int scaled_exp(double x, int s) {
    const int E = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
    return E == 0 ? NOEXP : E + s;
}

// floor(log2 |d| / 2): 2^s is within a factor sqrt(2) of sqrt(|d|); 0 for a
// zero, subnormal or non-finite d (the pivot check reports those)
__device__ __forceinline__ int half_exp(double d) {
    const int E = (int)(((unsigned long long)__double_as_longlong(d) >> 52) & 0x7FF);
    return (E == 0 || E == 0x7FF) ? 0 : (E - 1023) >> 1;
}

}  // namespace

// One 512-thread block per packed row block: rows r0..r0+127 of the front,
// panel columns p0..p0+kb (kb = min(32, k - p0)).  Thread (r, g) holds the 8
// panel entries 8g..8g+7 of row r (one 16-byte BF16 unit per slice).
// Slice s (0..6 for L21, 7..13 for L21 D) of block blk starts at byte
// (blk * 14 + s) * 8192; BF16 entry (r, k) of a slice at element
//   ((r >> 3) * 4 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7).
// expo[256 blk + r] = e_r (L21), expo[256 blk + 128 + r] = f_r (L21 D).
// Rows beyond the front and columns beyond kb are zero.
__global__ void __launch_bounds__(512) oz_pack_kernel(const TcPack* __restrict__ items, const int* __restrict__ kk,
                                                      const int* __restrict__ nn,
                                                      const long long* __restrict__ front_off,
                                                      const int* __restrict__ node_ptr, const double* __restrict__ D,
                                                      const double* __restrict__ pool, unsigned char* __restrict__ pack,
                                                      int* __restrict__ expo, int* __restrict__ live,
                                                      int* __restrict__ err) {
    __shared__ int sexp[2][4][TC_BLK];
    const TcPack it = items[blockIdx.x];
    const int F = it.front, k = kk[F], ld = nn[F] + k;
    const int kb = min(KP, k - it.p0);
    const int r = threadIdx.x & (TC_BLK - 1), g = threadIdx.x >> 7, gi = it.r0 + r;
    const double* A = pool + front_off[F] + gi;
    const double* d = D + node_ptr[F] + it.p0;
    double x[8], y[8];
    int sc[8];
    int ea = NOEXP, eb = NOEXP;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int kc = 8 * g + t;
        const bool in = kc < kb && gi < ld;
        const double dk = kc < kb ? d[kc] : 1.0;
        x[t] = in ? A[(long long)(it.p0 + kc) * ld] : 0.0;
        y[t] = in ? x[t] * dk : 0.0;
        // balanced operands L |D|^(1/2) and (L D) |D|^(-1/2), both scaled by
        // powers of two: the product of the two is unchanged
        sc[t] = half_exp(dk);
        ea = max(ea, scaled_exp(x[t], sc[t]));
        eb = max(eb, scaled_exp(y[t], -sc[t]));
    }
    sexp[0][g][r] = ea;
    sexp[1][g][r] = eb;
    __syncthreads();
    ea = max(max(sexp[0][0][r], sexp[0][1][r]), max(sexp[0][2][r], sexp[0][3][r]));
    eb = max(max(sexp[1][0][r], sexp[1][1][r]), max(sexp[1][2][r], sexp[1][3][r]));
    // every |x 2^s| < 2^(E - 1022) for the largest scaled exponent field E
    const int e = ea - 1022, f = eb - 1022;
    if (g == 0) {
        expo[256 * it.blk + r] = e;
        expo[256 * it.blk + TC_BLK + r] = f;
    }
    // rows of a front that the panel does not reach are zero: a tile whose A
    // block or B half has no nonzero row is skipped by the update
    const int anyA = __syncthreads_or(ea > NOEXP);
    const int anyB0 = __syncthreads_or(eb > NOEXP && r < OZ_N);
    const int anyB1 = __syncthreads_or(eb > NOEXP && r >= OZ_N);
    if (threadIdx.x == 0) live[it.blk] = (anyA ? 1 : 0) | (anyB0 ? 2 : 0) | (anyB1 ? 4 : 0);
    bool bad = false;
    unsigned char* out = pack + (size_t)it.blk * BLK_BYTES + (size_t)((((r >> 3) * 4 + g) * 64 + (r & 7) * 8) * 2);
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        unsigned w[NDIG][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            long long X = side == 0 ? to_fixed(x[t], sc[t], e, &bad) : to_fixed(y[t], -sc[t], f, &bad);
            // balanced base-256 digits, least significant first
#pragma unroll
            for (int p = NDIG - 1; p >= 1; --p) {
                const int dg = (int)((X + 128) & 255) - 128;
                X = (X - dg) >> 8;
                const unsigned b = bf16_of_int(dg);
                if (t & 1) w[p][t >> 1] |= b << 16;
                else w[p][t >> 1] = b;
            }
            const unsigned b = bf16_of_int((int)X);  // top digit, |X| <= 128
            if (t & 1) w[0][t >> 1] |= b << 16;
            else w[0][t >> 1] = b;
        }
#pragma unroll
        for (int p = 0; p < NDIG; ++p)
            *reinterpret_cast<uint4*>(out + (size_t)(side * NDIG + p) * SLICE_BYTES) =
                make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
    }
    if (bad) atomicOr(err, 1);
}

constexpr unsigned MB = 0x4B400000u;  // float bits of 1.5 * 2^23: MB + V are the bits of V + 1.5 * 2^23
// sum of the MB terms of S (mod 2^64): MB (2^40 + 2^32 + 2^24 + 2^16 + 2^8 + 1)
// + (MB 257 mod 2^32) / 2^16 (MB 257 mod 2^32 = 0x8B400000 is a multiple of 2^16)
constexpr unsigned long long KMB =
    ((unsigned long long)MB << 40) + ((unsigned long long)MB << 32) + ((unsigned long long)MB << 24) +
    ((unsigned long long)MB << 16) + ((unsigned long long)MB << 8) + MB + ((MB * 257u) >> 16);

// a * b + c with a 32 x 32 -> 64-bit product (one IMAD.WIDE.U32)
__device__ __forceinline__ unsigned long long mad_wide(unsigned a, unsigned b, unsigned long long c) {
    unsigned long long d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// Phase 1, CW columns of one tile row (this lane): the level sums v[l][cc]
// (exact integers) of column cc combined into the signed 64-bit
//   S = floor((V0 2^56 + V1 2^48 + ... + V7) / 2^16)
//     = sum_{l<6} V_l 2^(40-8l) + floor((V6 2^8 + V7) / 2^16),
// (|S| < 2^60), stored as two 32-bit words.  Accumulated from u_l = MB + V_l
// by 64-bit multiply-adds (mod 2^64; u6 2^8 + u7 = MB 257 + V6 2^8 + V7
// without wrap-around in 32 bits, and MB 257 mod 2^32 is a multiple of 2^16)
// and the constant sum of the MB terms taken off at the end.
__device__ __forceinline__ void oz_sum(const float (&v)[NLEV][CW], unsigned* slo, unsigned* shi) {
    constexpr float MAGIC = 12582912.0f;  // 1.5 * 2^23
#pragma unroll
    for (int cc = 0; cc < CW; ++cc) {
        unsigned u[NLEV];
#pragma unroll
        for (int l = 0; l < NLEV; ++l) u[l] = __float_as_uint(v[l][cc] + MAGIC);
        unsigned long long acc = (u[6] * 256u + u[7]) >> 16;
        acc = mad_wide(u[5], 1u, acc);
        acc = mad_wide(u[4], 1u << 8, acc);
        acc = mad_wide(u[3], 1u << 16, acc);
        acc = mad_wide(u[2], 1u << 24, acc);
        acc += (unsigned long long)(u[0] * 256u + u[1]) << 32;
        unsigned lo = (unsigned)acc, hi = (unsigned)(acc >> 32);
        asm("sub.cc.u32 %0, %0, %2;\n\tsubc.u32 %1, %1, %3;" : "+r"(lo), "+r"(hi) : "r"((unsigned)KMB), "r"((unsigned)(KMB >> 32)));
        slo[cc] = lo;
        shi[cc] = hi;
    }
}

// Phase 2, the warp's 16 columns of one tile row (this lane): the double
// -S 2^(e_i + f_j - 54) added to the front entry col[cc * ld], assembled
// without FP64 arithmetic from |S|, its leading-bit position and the
// exponents.  Results below the normal range are flushed to zero (an error
// below 2^-1022).  CHECK: skip entries outside the front, the lower triangle
// and the extra x extra block.  RANGE: results may fall outside the normal
// range (else known not to).
template <bool CHECK, bool RANGE>
__device__ __forceinline__ void oz_emit(const unsigned (&slo)[16], const unsigned (&shi)[16], int er, int myf,
                                        double* col, int ld, int gi, int gj0, int n, int rmax) {
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
        const int fj = __shfl_sync(0xffffffffu, myf, cc);  // every lane: before any skip
        if (CHECK) {
            const int gj = gj0 + cc;
            if (gi >= rmax || gj >= ld || !(gi >= gj || (gi >= n && gj >= n))) continue;
        }
        unsigned lo = slo[cc], hi = shi[cc];
        const unsigned sg = (unsigned)((int)hi >> 31);  // all ones when S < 0
        lo ^= sg;
        hi ^= sg;
        asm("sub.cc.u32 %0, %0, %2;\n\tsubc.u32 %1, %1, %2;" : "+r"(lo), "+r"(hi) : "r"(sg));  // (hi:lo) = |S|
        const bool big = hi != 0u;
        const unsigned H = big ? hi : lo, L = big ? lo : 0u;  // |S| = (H:L) 2^(big ? 0 : -32)
        const int sh = __clz(H);                              // < 32 unless S = 0
        const int lz = big ? sh : sh + 32;
        // (H:L) << sh: the leading bit at 63; mantissa = bits 63..11, rounded
        // to nearest on bit 10 (a carry into bit 53 raises the exponent by one)
        const unsigned nhi = __funnelshift_l(L, H, sh), nlo = L << (sh & 31);
        unsigned mlo = __funnelshift_r(nlo, nhi, 11), mhi = nhi >> 11;
        asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, 0;" : "+r"(mlo), "+r"(mhi) : "r"((nlo >> 10) & 1u));
        const int be = er + fj - lz;  // biased exponent of the leading bit
        // -S: negative when S > 0
        mhi += ((unsigned)(be - 1) << 20) + (~sg & 0x80000000u);
        unsigned long long bits = ((unsigned long long)mhi << 32) | mlo;
        if (RANGE && (unsigned)(be - 1) >= 2045u)
            bits = (unsigned long long)(~sg & 0x80000000u) << 32 | (be < 1 ? 0ull : 0x7FF0000000000000ull);
        if (H != 0u) atomicAdd(col + (long long)cc * ld, __longlong_as_double((long long)bits));
    }
}

__global__ void __launch_bounds__(UPD_THREADS, 1) oz_update_kernel(
    const TcTile* __restrict__ tiles, int ntiles, const int* __restrict__ kk, const int* __restrict__ nn,
    const long long* __restrict__ front_off, const unsigned char* __restrict__ pack, const int* __restrict__ expo,
    const int* __restrict__ live, double* __restrict__ pool, int plain, int* __restrict__ err, long long spin_limit) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long full[NSTAGE], empty[NSTAGE], tfull, tempty, drain;
    __shared__ unsigned s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
        mbar_init(&tfull, 1);
        mbar_init(&tempty, EPI_WARPS * 32);
        mbar_init(&drain, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;

    if (warp == EPI_WARPS) {
        // ---------------------------------------------------------- producer
        if (lane == 0) {
            int it = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                const TcTile tl = tiles[t];
                if (skip_tile(tl, nn, live, plain)) continue;
                const int s = it % NSTAGE;
                if (!mbar_wait(&empty[s], ((unsigned)(it / NSTAGE) & 1u) ^ 1u, &s_abort, err, spin_limit)) break;
                const unsigned char* pa = pack + (size_t)tl.a_blk * BLK_BYTES;
                const unsigned char* pb = pack + (size_t)tl.b_blk * BLK_BYTES + NDIG * SLICE_BYTES + tl.nk * B_BYTES;
                unsigned char* st = stage0 + (size_t)s * STAGE_BYTES;
                mbar_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll 1
                for (int p = 0; p < NDIG; ++p) {
                    bulk_copy(st + p * SLICE_BYTES, pa + p * SLICE_BYTES, SLICE_BYTES, &full[s]);
                    bulk_copy(st + NDIG * SLICE_BYTES + p * B_BYTES, pb + p * SLICE_BYTES, B_BYTES, &full[s]);
                }
                ++it;
            }
            // every copy issued has landed before the CTA may exit (bounded)
            for (int q = 0; q < NSTAGE && q < it; ++q) {
                const int last = it - 1 - q;
                long long n = 0;
                while (!mbar_test(&full[last % NSTAGE], (unsigned)(last / NSTAGE) & 1u) && ++n <= spin_limit) {
                }
            }
        }
    } else if (warp == EPI_WARPS + 1) {
        // ------------------------------------------------------- MMA issuer
        if (lane == 0) {
            int it = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
                if (skip_tile(tiles[t], nn, live, plain)) continue;
                if (!mbar_wait(&tempty, ((unsigned)it & 1u) ^ 1u, &s_abort, err, spin_limit)) break;
                const int s = it % NSTAGE;
                if (!mbar_wait(&full[s], (unsigned)(it / NSTAGE) & 1u, &s_abort, err, spin_limit)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned a0 = smem_addr(stage0 + (size_t)s * STAGE_BYTES);
                const unsigned b0 = a0 + NDIG * SLICE_BYTES;
                // K-major core matrices: LBO = 128 B (next 8 columns), SBO = 512 B (next 8 rows)
#pragma unroll 1
                for (int p = 0; p < NDIG; ++p)
#pragma unroll 1
                    for (int q = 0; p + q < NLEV; ++q) {
                        const unsigned d = tmem + (unsigned)((p + q) * OZ_N);
#pragma unroll
                        for (int ks = 0; ks < KP / 16; ++ks)
                            mma_f16(d, smem_desc(a0 + p * SLICE_BYTES + ks * 256, 128, 512),
                                    smem_desc(b0 + q * B_BYTES + ks * 256, 128, 512), IDESC, p > 0 || ks > 0);
                    }
                mma_commit(&empty[s]);
                mma_commit(&tfull);
                ++it;
            }
            mma_commit(&drain);
            long long n = 0;
            while (!mbar_test(&drain, 0u) && ++n <= spin_limit) {
            }
        }
    } else {
        // ------------------------------------------ epilogue (warps 0..15)
        // warp w: tile rows 32 (w % 4) .. + 31 (its tensor-memory lane
        // quarter), columns 16 (w / 4) .. + 15.  The next tile's front data
        // and exponents are loaded while the current one's doubles are
        // assembled.
        const int q4 = warp & 3, grp = warp >> 2;
        struct Meta {
            int skip, n, ld, i0, j0, er, myf;
            long long off;
        };
        auto load_meta = [&](int t, Meta& m) {
            if (t >= ntiles) return;
            const TcTile tl = tiles[t];
            const int F = tl.front;
            m.n = nn[F];
            m.ld = m.n + kk[F];
            m.off = front_off[F];
            m.i0 = tl.i0;
            m.j0 = tl.j0;
            m.skip = skip_tile(tl, nn, live, plain);
            // biased exponent of -S 2^(e_i + f_j - 54) is er + f_j - lz(S)
            m.er = expo[256 * tl.a_blk + q4 * 32 + lane] + (1023 - 54 + 63);
            m.myf = expo[256 * tl.b_blk + TC_BLK + tl.nk * OZ_N + grp * 16 + (lane & 15)];
        };
        Meta cur{}, nxt{};
        load_meta(blockIdx.x, cur);
        int it = 0;
        for (int t = blockIdx.x; t < ntiles;) {
            const int tn = t + gridDim.x;
            if (cur.skip) {
                t = tn;
                load_meta(t, cur);
                continue;
            }
            const bool ok = mbar_wait(&tfull, (unsigned)(it++) & 1u, &s_abort, err, spin_limit);
            if (!__all_sync(0xffffffffu, ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int n = cur.n, ld = cur.ld;
            const int rmax = plain ? n : ld;
            const int gi = cur.i0 + q4 * 32 + lane;
            const int gj0 = cur.j0 + grp * 16;
            // no per-entry masks when every row and column exists and every
            // entry is in the lower triangle or the extra x extra block
            const int r0 = cur.i0 + q4 * 32;
            const bool fast = r0 + 32 <= rmax && gj0 + 16 <= ld && (r0 >= gj0 + 15 || (r0 >= n && gj0 >= n));
            // no per-entry exponent-range selects when every possible result
            // of the warp is a normal double (4 <= lz <= 63 as 0 < |S| < 2^60)
            const int fmin = __reduce_min_sync(0xffffffffu, cur.myf), fmax = __reduce_max_sync(0xffffffffu, cur.myf);
            const bool normal = __all_sync(0xffffffffu, cur.er + fmin - 63 >= 1 && cur.er + fmax - 4 <= 2045);
            double* col = pool + cur.off + gi + (long long)gj0 * ld;
            const unsigned taddr = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)(grp * 16);
            // phase 1: the 16 columns' S from four loads of 4 columns x 8
            // levels; the accumulators are released right after, so the next
            // tile's MMAs run while phase 2 assembles and adds the doubles
            unsigned slo[16], shi[16];
#pragma unroll
            for (int ch = 0; ch < 16 / CW; ++ch) {
                float v[NLEV][CW];
#pragma unroll
                for (int l = 0; l < NLEV; ++l) tmem_ld4(taddr + l * OZ_N + ch * CW, v[l]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                oz_sum(v, slo + ch * CW, shi + ch * CW);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&tempty);
            load_meta(tn, nxt);
            // every S of the warp zero (rows or columns the panel does not
            // reach): nothing to add
            unsigned nz = 0;
#pragma unroll
            for (int c = 0; c < 16; ++c) nz |= slo[c] | shi[c];
            if (__any_sync(0xffffffffu, nz != 0u)) {
                if (fast && normal) oz_emit<false, false>(slo, shi, cur.er, cur.myf, col, ld, gi, gj0, n, rmax);
                else if (fast) oz_emit<false, true>(slo, shi, cur.er, cur.myf, col, ld, gi, gj0, n, rmax);
                else oz_emit<true, true>(slo, shi, cur.er, cur.myf, col, ld, gi, gj0, n, rmax);
            }
            t = tn;
            cur = nxt;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

static size_t oz_update_smem() { return (size_t)NSTAGE * STAGE_BYTES + 1024; }

// Pack + update of one panel step of FP64 fronts on the given stream.
int enqueue_oz_step(riga_ctx* c, const StepRange& R, double* pool, int plain, cudaStream_t st) {
    const int npack = R.o_end - R.o_begin, ntiles = R.q_end - R.q_begin;
    if (ntiles <= 0 || npack <= 0) return RIGA_OK;
    static int nsm = 0;
    if (nsm == 0 && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) nsm = 0;
    const int grid = std::max(1, std::min(ntiles, nsm > 0 ? nsm : 148));
    count_launch(c);
    oz_pack_kernel<<<npack, 512, 0, st>>>(c->ozpacks.ptr + R.o_begin, c->kk.ptr, c->nn.ptr, c->front_off.ptr,
                                          c->node_ptr.ptr, c->D.ptr, pool, c->ozpack.ptr, c->ozexp.ptr, c->ozlive.ptr,
                                          c->flag.ptr);
    count_launch(c);
    oz_update_kernel<<<grid, UPD_THREADS, oz_update_smem(), st>>>(c->oztiles.ptr + R.q_begin, ntiles, c->kk.ptr,
                                                                  c->nn.ptr, c->front_off.ptr, c->ozpack.ptr,
                                                                  c->ozexp.ptr, c->ozlive.ptr, pool, plain, c->flag.ptr,
                                                                  c->wait_limit);
    return RIGA_OK;
}

// Shared-memory size attribute and the digit-slice buffers (once per schedule)
int prepare_oz(riga_ctx* c) {
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(oz_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)oz_update_smem()));
    const long long nblk = std::max<long long>(1, c->S.oz_pack_blocks);
    if (c->ozpack.alloc((size_t)nblk * BLK_BYTES) != cudaSuccess)
        return set_error(c, RIGA_ENOMEM, "FP64 tensor-core digit slices");
    RIGA_CUDA_TRY(c, c->ozexp.alloc((size_t)256 * nblk));
    RIGA_CUDA_TRY(c, c->ozlive.alloc((size_t)nblk));
    return RIGA_OK;
}

}  // namespace riga
