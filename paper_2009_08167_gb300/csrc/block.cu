// Block shift-and-invert Lanczos (block size B = 2 or 4) in the M-inner
// product: the recurrence of Sec. 4.1-4.2 with B vectors per step, so that
// one traversal of the factor's tree (a B-right-hand-side solve, solve.cu)
// and one read of M serve B Krylov vectors, and eigenvalues of multiplicity
// up to B appear in a single run.
//
// Per block step j (H = (K - sigma M)^{-1} M, V_j M-orthonormal, MV_j stored):
//   W = H V_j                      one B-RHS solve of the stored M V_j
//   W -= V_{j-1,j} C1              the block three-term recurrence: the
//                                  coefficients against the last two blocks
//                                  (computed, not taken from T)
//   W -= V C2                      one classical Gram-Schmidt pass against
//                                  all columns so far (locked, then run)
//   A_j = (C1 + C2)[block j rows]  diagonal block of T
// The full pass removes what the recurrence leaves along older vectors
// (rounding, loss of orthogonality, the locked vectors' residuals), which is
// tiny next to the new block, so one pass leaves W orthogonal to working
// accuracy.  When it removed more than 100 times the norm that remains (the
// Daniel-Gragg-Kaufman-Stewart test with a loose bound), a flag switches the
// solve to two full passes (CGS2) from then on.
//   W = V_{j+1} B_{j+1}            M-orthonormal QR by Cholesky of W^T M W,
//                                  twice (CholQR2), M W from one block SpMV
// T_m is block tridiagonal (half-bandwidth B) with diagonal blocks A_j and
// sub-diagonal blocks B_{j+1}; its eigenpairs (band.cpp) give the Ritz
// values theta (lambda = sigma + 1/theta) and the residual estimates
// ||B_m s_last||.  A breakdown of the QR (a numerically rank-deficient W)
// ends the run; the converged pairs found so far are kept.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>

#include "lanczos.h"

namespace riga {

constexpr int BLK_MAX = 4;

// Partial dots out[j*B + r] = sum over this chunk's rows of B_j[row] w_r[row]
// (the basis tile staged through shared memory in HR-row pieces, the next
// piece loaded into registers while the current one is summed, as in the
// single-vector kernels; every staged entry serves B products).
template <int B>
__device__ __forceinline__ void bchunk_dots(const double* __restrict__ Bm, long long ld, int J, long long r0, int rows,
                                            const double* __restrict__ ws, double* __restrict__ Vs,
                                            double* __restrict__ red, double* __restrict__ out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (rows <= 0) {  // no rows (the same for the whole block): zero partials
        for (int j = tid; j < J * B; j += blockDim.x) out[j] = 0.0;
        return;
    }
    const int nh = (rows + HR - 1) / HR;         // row pieces per column tile
    const int nst = ((J + TJ - 1) / TJ) * nh;    // stages (column tile, row piece)
    double pre[TJ / 8][HR / 32];                 // the next stage, loaded while this one computes
    auto load = [&](int st) {
        const int j0 = (st / nh) * TJ, h = (st % nh) * HR;
        const int jn = min(TJ, J - j0), hn = min(HR, rows - h);
#pragma unroll
        for (int q = 0; q < TJ / 8; ++q) {
            const int jl = warp + 8 * q;
            const double* col = Bm + (long long)(j0 + jl) * ld + r0 + h;
#pragma unroll
            for (int i = 0; i < HR / 32; ++i) {
                const int r = lane + 32 * i;
                pre[q][i] = (jl < jn && r < hn) ? col[r] : 0.0;
            }
        }
    };
    load(0);
    double s[B];
#pragma unroll
    for (int r = 0; r < B; ++r) s[r] = 0.0;
    for (int st = 0; st < nst; ++st) {
        const int j0 = (st / nh) * TJ, h = (st % nh) * HR;
        const int jn = min(TJ, J - j0), hn = min(HR, rows - h);
#pragma unroll
        for (int q = 0; q < TJ / 8; ++q)
#pragma unroll
            for (int i = 0; i < HR / 32; ++i) Vs[(warp + 8 * q) * (HR + 1) + lane + 32 * i] = pre[q][i];
        __syncthreads();
        if (st + 1 < nst) load(st + 1);
        if (lane < jn) {
            const double* vc = Vs + lane * (HR + 1);
#pragma unroll 4
            for (int i = warp; i < hn; i += 8) {
                const double v = vc[i];
#pragma unroll
                for (int r = 0; r < B; ++r) s[r] += v * ws[r * CH + h + i];
            }
        }
        __syncthreads();
        if (st % nh == nh - 1) {  // last piece of this column tile: sum the 8 row groups
#pragma unroll
            for (int r = 0; r < B; ++r) {
                red[(warp * TJ + lane) * B + r] = s[r];
                s[r] = 0.0;
            }
            __syncthreads();
            if (tid < jn * B) {
                double t = 0.0;
#pragma unroll
                for (int g = 0; g < 8; ++g) t += red[g * TJ * B + tid];
                out[j0 * B + tid] = t;
            }
        }
    }
    __syncthreads();
}

// The tall-skinny kernels split the rows evenly over their blocks (at most
// CH each; the block count a multiple of the SM count), so that every SM gets
// the same share of the FP64 work.
template <int B>
__global__ void __launch_bounds__(256) bdots_kernel(const double* __restrict__ MV, long long ld, int J,
                                                    const double* __restrict__ W, long long N,
                                                    double* __restrict__ partial, int pstride) {
    extern __shared__ double sh[];
    double* ws = sh;                  // B * CH
    double* red = ws + B * CH;        // 8 * TJ * B
    double* Vs = red + 8 * TJ * B;    // TJ * (HR + 1)
    const long long r0 = N * blockIdx.x / gridDim.x;
    const int rows = (int)(N * (blockIdx.x + 1) / gridDim.x - r0);
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < B; ++r) ws[r * CH + tid] = (tid < rows) ? W[r * N + r0 + tid] : 0.0;
    __syncthreads();
    bchunk_dots<B>(MV, ld, J, r0, rows, ws, Vs, red, partial + (long long)blockIdx.x * pstride);
}

// w_r[row] -= sum_j V_j[row] C[j*B + r], the loads issued eight at a time
template <int B>
__device__ __forceinline__ void brow_update(const double* __restrict__ V, long long ld, int J, long long row,
                                            const double* __restrict__ cs, double* v) {
    int j = 0;
    for (; j + 8 <= J; j += 8) {
        double b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = V[(long long)(j + q) * ld + row];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int r = 0; r < B; ++r) v[r] -= b[q] * cs[(j + q) * B + r];
    }
    for (; j < J; ++j) {
        const double b = V[(long long)j * ld + row];
#pragma unroll
        for (int r = 0; r < B; ++r) v[r] -= b * cs[j * B + r];
    }
}

// W -= V[:, 0..Ju) C (this chunk), then partial dots MV[:, 0..Jd)^T W
template <int B>
__global__ void __launch_bounds__(256) bupdate_dots_kernel(const double* __restrict__ V, int Ju,
                                                           const double* __restrict__ C,
                                                           const double* __restrict__ MV, int Jd, long long ld,
                                                           double* __restrict__ W, long long N,
                                                           double* __restrict__ partial, int pstride) {
    extern __shared__ double sh[];
    double* ws = sh;                  // B * CH
    double* red = ws + B * CH;        // 8 * TJ * B
    double* Vs = red + 8 * TJ * B;    // TJ * (HR + 1)
    double* cs = Vs + TJ * (HR + 1);  // Ju * B
    const long long r0 = N * blockIdx.x / gridDim.x;
    const int rows = (int)(N * (blockIdx.x + 1) / gridDim.x - r0);
    const int tid = threadIdx.x;
    for (int t = tid; t < Ju * B; t += blockDim.x) cs[t] = C[t];
    __syncthreads();
    const long long row = r0 + tid;
    double v[B];
#pragma unroll
    for (int r = 0; r < B; ++r) v[r] = 0.0;
    if (tid < rows) {
#pragma unroll
        for (int r = 0; r < B; ++r) v[r] = W[r * N + row];
        brow_update<B>(V, ld, Ju, row, cs, v);
#pragma unroll
        for (int r = 0; r < B; ++r) W[r * N + row] = v[r];
    }
#pragma unroll
    for (int r = 0; r < B; ++r) ws[r * CH + tid] = v[r];
    __syncthreads();
    bchunk_dots<B>(MV, ld, Jd, r0, rows, ws, Vs, red, partial + (long long)blockIdx.x * pstride);
}

// W -= V C; block 0 also stores the squared column norms of C in cn2 (when
// given), the part of each column the pass removed
template <int B>
__global__ void __launch_bounds__(256) bupdate_kernel(const double* __restrict__ V, long long ld, int J,
                                                      const double* __restrict__ C, double* __restrict__ W, long long N,
                                                      double* __restrict__ cn2) {
    extern __shared__ double cs[];
    for (int t = threadIdx.x; t < J * B; t += blockDim.x) cs[t] = C[t];
    __syncthreads();
    if (cn2 && blockIdx.x == 0 && threadIdx.x < 32) {
        double q2[B];
#pragma unroll
        for (int r = 0; r < B; ++r) q2[r] = 0.0;
        for (int q = threadIdx.x; q < J; q += 32)
#pragma unroll
            for (int r = 0; r < B; ++r) q2[r] += cs[q * B + r] * cs[q * B + r];
#pragma unroll
        for (int r = 0; r < B; ++r) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) q2[r] += __shfl_xor_sync(0xffffffffu, q2[r], o);
            if (threadIdx.x == 0) cn2[r] = q2[r];
        }
    }
    const long long r1 = N * (blockIdx.x + 1) / gridDim.x;
    for (long long row = N * blockIdx.x / gridDim.x + threadIdx.x; row < r1; row += blockDim.x) {
        double v[B];
#pragma unroll
        for (int r = 0; r < B; ++r) v[r] = W[r * N + row];
        brow_update<B>(V, ld, J, row, cs, v);
#pragma unroll
        for (int r = 0; r < B; ++r) W[r * N + row] = v[r];
    }
}

// Grid-wide sum of the blocks' CNT-value partials without another launch:
// every block stores its partial, and the last block to arrive (counted on
// `counter`, which it resets) adds them in a fixed order (deterministic).
template <int CNT>
__device__ void tail_reduce(const double* __restrict__ mine, double* __restrict__ partial, int* __restrict__ counter,
                            double* __restrict__ out) {
    __shared__ int s_last;
    __shared__ double sh[256];
    if ((int)threadIdx.x < CNT) partial[(long long)blockIdx.x * CNT + threadIdx.x] = mine[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const int groups = blockDim.x / CNT;  // thread t sums entry t % CNT over blocks t / CNT, t / CNT + groups, ...
    const int e = threadIdx.x % CNT, g = threadIdx.x / CNT;
    double acc = 0.0;
    if (g < groups)
#pragma unroll 8
        for (int i = g; i < (int)gridDim.x; i += groups) acc += __ldcg(&partial[(long long)i * CNT + e]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    if ((int)threadIdx.x < CNT) {
        double t = 0.0;
        for (int q = 0; q < groups; ++q) t += sh[q * CNT + threadIdx.x];
        out[threadIdx.x] = t;
    }
    if (threadIdx.x == 0) *counter = 0;
}

// Coefficients of the block three-term recurrence: out[i B + r] =
// (M v_{u0+i})^T w_r for the JB = B or 2 B columns of the last two blocks
// (grid-stride over rows, reduced by the last block)
template <int B, int JB>
__global__ void __launch_bounds__(256) blocal_dots_kernel(const double* __restrict__ MV, long long ld,
                                                          const double* __restrict__ W, long long N,
                                                          double* __restrict__ partial, int* __restrict__ counter,
                                                          double* __restrict__ out) {
    __shared__ double red[8][JB * B];
    __shared__ double tot[JB * B];
    double acc[JB * B];
#pragma unroll
    for (int e = 0; e < JB * B; ++e) acc[e] = 0.0;
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < N;
         row += (long long)gridDim.x * blockDim.x) {
        double w[B];
#pragma unroll
        for (int r = 0; r < B; ++r) w[r] = W[r * N + row];
#pragma unroll
        for (int i = 0; i < JB; ++i) {
            const double mv = MV[(long long)i * ld + row];
#pragma unroll
            for (int r = 0; r < B; ++r) acc[i * B + r] += mv * w[r];
        }
    }
#pragma unroll
    for (int e = 0; e < JB * B; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int e = 0; e < JB * B; ++e) red[threadIdx.x >> 5][e] = acc[e];
    __syncthreads();
    if (threadIdx.x < JB * B) {
        double t = 0.0;
        for (int g = 0; g < 8; ++g) t += red[g][threadIdx.x];
        tot[threadIdx.x] = t;
    }
    __syncthreads();
    tail_reduce<JB * B>(tot, partial, counter, out);
}

// MW = M W (SPMV_TPR lanes per row, every value of M serving B products) and
// the Gram matrix G = W^T M W (row-major B x B, its entries spread over the
// lanes of the row group, reduced by the last block)
template <int B>
__global__ void __launch_bounds__(256) bspmv_gram_kernel(long long N, const long long* __restrict__ rowptr,
                                                         const int* __restrict__ col, const double* __restrict__ Mv,
                                                         const double* __restrict__ W, double* __restrict__ MW,
                                                         double* __restrict__ partial, int* __restrict__ counter,
                                                         double* __restrict__ G) {
    constexpr int GE = (B * B + SPMV_TPR - 1) / SPMV_TPR;  // Gram entries per lane: lane + SPMV_TPR k
    __shared__ double red[8][B * B];
    __shared__ double tot[B * B];
    const int lane = threadIdx.x & (SPMV_TPR - 1), grp = threadIdx.x / SPMV_TPR;
    double gacc[GE];
#pragma unroll
    for (int k = 0; k < GE; ++k) gacc[k] = 0.0;
    for (long long base = (long long)blockIdx.x * SPMV_RPB; base < N; base += (long long)gridDim.x * SPMV_RPB) {
        const long long row = base + grp;
        double s[B];
#pragma unroll
        for (int r = 0; r < B; ++r) s[r] = 0.0;
        if (row < N) {
            // four entries per lane in flight (their values and columns,
            // then the gathers), summed in the order of the plain loop
            const long long end = rowptr[row + 1];
            for (long long e0 = rowptr[row] + lane; e0 < end; e0 += 4 * SPMV_TPR) {
                double mv[4];
                int cc[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long e = e0 + k * SPMV_TPR;
                    mv[k] = e < end ? Mv[e] : 0.0;
                    cc[k] = e < end ? col[e] : -1;
                }
                double x[4][B];
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int r = 0; r < B; ++r) x[k][r] = cc[k] >= 0 ? W[r * N + cc[k]] : 0.0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (cc[k] >= 0)
#pragma unroll
                        for (int r = 0; r < B; ++r) s[r] += mv[k] * x[k][r];
            }
        }
#pragma unroll
        for (int r = 0; r < B; ++r) s[r] = group_sum(s[r]);
        if (row < N) {
#pragma unroll
            for (int r = 0; r < B; ++r)
                if (lane == r % SPMV_TPR) MW[r * N + row] = s[r];
#pragma unroll
            for (int k = 0; k < GE; ++k) {
                const int e = lane + SPMV_TPR * k;
                if (e < B * B) {
                    const int q = e / B, r = e % B;
                    double sr = s[0];
#pragma unroll
                    for (int rr = 1; rr < B; ++rr)
                        if (r == rr) sr = s[rr];
                    gacc[k] += W[q * N + row] * sr;
                }
            }
        }
    }
    // lanes with the same index in the groups of a warp hold the same entries
#pragma unroll
    for (int k = 0; k < GE; ++k)
#pragma unroll
        for (int o = SPMV_TPR; o < 32; o <<= 1) gacc[k] += __shfl_xor_sync(0xffffffffu, gacc[k], o);
    const int wl = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (wl < SPMV_TPR)
#pragma unroll
        for (int k = 0; k < GE; ++k)
            if (wl + SPMV_TPR * k < B * B) red[warp][wl + SPMV_TPR * k] = gacc[k];
    __syncthreads();
    if (threadIdx.x < B * B) {
        double t2 = 0.0;
        for (int g = 0; g < 8; ++g) t2 += red[g][threadIdx.x];
        tot[threadIdx.x] = t2;
    }
    __syncthreads();
    tail_reduce<B * B>(tot, partial, counter, G);
}

// Cholesky G + s I = R^T R of the symmetrised B x B Gram matrix,
// s = shift_rel * trace(G), and R^{-1}.  A pivot at or below 1e-24 of the
// largest diagonal entry is a breakdown (returned true) and R = I, so that
// the step stays finite.
template <int B>
__device__ bool bcholesky(const double* __restrict__ G, double shift_rel, double (*R)[B], double (*Ri)[B]) {
    double g[B][B];
    double dmax = 0.0, tr = 0.0;
    for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
            g[i][j] = 0.5 * (G[i * B + j] + G[j * B + i]);
            R[i][j] = 0.0;
            Ri[i][j] = 0.0;
        }
    for (int i = 0; i < B; ++i) tr += fmax(g[i][i], 0.0);
    for (int i = 0; i < B; ++i) g[i][i] += shift_rel * tr;
    for (int i = 0; i < B; ++i) dmax = fmax(dmax, g[i][i]);
    bool bad = !(dmax > 0.0);
    for (int i = 0; i < B && !bad; ++i) {
        double d = g[i][i];
        for (int k = 0; k < i; ++k) d -= R[k][i] * R[k][i];
        if (!(d > 1e-24 * dmax)) {
            bad = true;
            break;
        }
        R[i][i] = sqrt(d);
        for (int j = i + 1; j < B; ++j) {
            double v = g[i][j];
            for (int k = 0; k < i; ++k) v -= R[k][i] * R[k][j];
            R[i][j] = v / R[i][i];
        }
    }
    if (bad)
        for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j) R[i][j] = (i == j) ? 1.0 : 0.0;
    for (int j = 0; j < B; ++j) {  // upper-triangular inverse
        Ri[j][j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= j; ++k) s += R[i][k] * Ri[k][j];
            Ri[i][j] = -s / R[i][i];
        }
    }
    return bad;
}

// One QR pass: every block factors the small Gram matrix itself (no separate
// launch), then X[:, l] = sum_{i <= l} Y[:, i] R^{-1}[i][l] for Y = W (into V)
// and Y = M W (into M V), in place when the output aliases the input, and
// (when Gnext is given) the Gram matrix of the new columns for the next pass.
// Block 0 records R (Rout), the accumulated factor Bout = R Rprev, and a
// breakdown (flag bit 0).
template <int B>
__global__ void __launch_bounds__(256) bqr_scale_kernel(long long N, const double* __restrict__ G, double shift_rel,
                                                        const double* __restrict__ Rprev, double* __restrict__ Bout,
                                                        double* __restrict__ Rout, int* __restrict__ flag,
                                                        const double* W, long long ldw, const double* MW, double* V,
                                                        double* MV, long long ldv, double* __restrict__ partial,
                                                        int* __restrict__ counter, double* __restrict__ Gnext,
                                                        const double* __restrict__ cn2) {
    __shared__ double sri[B * B];
    __shared__ double red[8][B * B];
    __shared__ double tot[B * B];
    if (threadIdx.x == 0) {
        double R[B][B], Ri[B][B];
        const bool bad = bcholesky<B>(G, shift_rel, R, Ri);
        for (int i = 0; i < B; ++i)
            for (int j = 0; j < B; ++j) sri[i * B + j] = Ri[i][j];
        if (blockIdx.x == 0) {
            if (bad) atomicOr(flag, 1);
            // the full Gram-Schmidt pass removed more than 100 x the norm left
            if (cn2)
                for (int r = 0; r < B; ++r)
                    if (!(cn2[r] <= 1e4 * G[r * B + r])) atomicOr(flag, 2);
            if (Rout)
                for (int i = 0; i < B; ++i)
                    for (int j = 0; j < B; ++j) Rout[i * B + j] = R[i][j];
            if (Bout)
                for (int i = 0; i < B; ++i)
                    for (int j = 0; j < B; ++j) {
                        double s = 0.0;
                        for (int k = 0; k < B; ++k) s += R[i][k] * (Rprev ? Rprev[k * B + j] : (k == j ? 1.0 : 0.0));
                        Bout[i * B + j] = s;
                    }
        }
    }
    __syncthreads();
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v[B], mv[B];
#pragma unroll
    for (int l = 0; l < B; ++l) v[l] = mv[l] = 0.0;
    if (i < N) {
        double w[B], mw[B];
#pragma unroll
        for (int r = 0; r < B; ++r) {
            w[r] = W[r * ldw + i];
            mw[r] = MW[r * ldw + i];
        }
#pragma unroll
        for (int l = 0; l < B; ++l) {
            double a = 0.0, b = 0.0;
#pragma unroll
            for (int r = 0; r <= l; ++r) {
                a += w[r] * sri[r * B + l];
                b += mw[r] * sri[r * B + l];
            }
            v[l] = a;
            mv[l] = b;
            V[l * ldv + i] = a;
            MV[l * ldv + i] = b;
        }
    }
    if (!Gnext) return;
    double g[B * B];
#pragma unroll
    for (int q = 0; q < B; ++q)
#pragma unroll
        for (int r = 0; r < B; ++r) g[q * B + r] = v[q] * mv[r];
#pragma unroll
    for (int e = 0; e < B * B; ++e)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g[e] += __shfl_xor_sync(0xffffffffu, g[e], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int e = 0; e < B * B; ++e) red[threadIdx.x >> 5][e] = g[e];
    __syncthreads();
    if (threadIdx.x < B * B) {
        double t2 = 0.0;
        for (int w2 = 0; w2 < 8; ++w2) t2 += red[w2][threadIdx.x];
        tot[threadIdx.x] = t2;
    }
    __syncthreads();
    tail_reduce<B * B>(tot, partial, counter, Gnext);
}

// Grid-wide barrier of a cooperative launch (all blocks resident): the
// k-th barrier waits until the arrival counter reaches k * gridDim.x.  The
// wait is bounded: past the poll budget it sets bit 2 of err and reports
// false (the caller returns; the host reads the flag).
__device__ bool grid_barrier(int* arrive, int target, int* err, long long limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(arrive, 1);
        long long it = 0;
        int ok = 1;
        while (*(volatile const int*)arrive < target) {
            if (++it > limit) {
                atomicOr(err, 2);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// The sums below keep FP64 additions few: on GB300 a warp's FP64
// instruction holds its SM's FP64 pipe for 16 clocks whatever its active
// lanes, so a reduction tree that adds every entry at every level costs more
// than the data it sums.  All of them add in a fixed order, so that every
// block obtains bitwise the same result.

// Warp sum of E per-lane values (E a power of two, at most 32): a butterfly
// whose first log2(E) steps halve the entries a lane carries (E - 1
// additions in all), then plain steps on the one value left.  Lane l ends
// with the warp sum of entry ((l >> log2(32 / E)) & (E - 1)); lane
// e * (32 / E) holds entry e.
template <int E>
__device__ __forceinline__ double warp_sum_scatter(double (&v)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int cnt = E, o = 16; cnt > 1; cnt >>= 1, o >>= 1) {
        const int h = cnt / 2;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? v[i] : v[i + h];
            const double keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    double t = v[0];
#pragma unroll
    for (int o = 32 / E / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

// Sum over the warps of a block of the per-warp sums red[w][e] (w < NW):
// lane l adds entry l % E of the warps l / E, l / E + 32 / E, ..., then the
// lanes of one entry combine; the result in out[e] (shared).  Called by one
// whole warp.
template <int E, int NW>
__device__ __forceinline__ void warps_sum(const double (*red)[E], double* out) {
    constexpr int G = 32 / E;
    const int lane = threadIdx.x & 31, e = lane % E, g = lane / E;
    double t = 0.0;
#pragma unroll
    for (int w = g; w < NW; w += G) t += red[w][e];
#pragma unroll
    for (int o = E; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane < E) out[lane] = t;
}

// Block sum of the per-thread Gram contributions g[B * B] into
// part[blockIdx.x * B * B + e]
template <int B, int NT>
__device__ void gram_block_partial(double (&g)[B * B], double (*red)[B * B], double* __restrict__ part,
                                   double* __restrict__ tot) {
    constexpr int E = B * B, G = 32 / E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double t = warp_sum_scatter<E>(g);
    if (lane % G == 0) red[warp][lane / G] = t;
    __syncthreads();
    if (warp == 0) {
        warps_sum<E, NT / 32>(red, tot);
        __syncwarp();
        if (lane < E) part[(long long)blockIdx.x * E + lane] = tot[lane];
    }
}

// Sum of the per-block Gram partials part[i * B * B + e] over the grid by
// one warp (lane l: entry l % E of the blocks l / E, l / E + 32 / E, ...,
// eight loads in flight), into G (shared); the caller synchronizes.
template <int B>
__device__ void gram_from_partials(const double* __restrict__ part, double* __restrict__ G) {
    constexpr int E = B * B, GR = 32 / E;
    const int lane = threadIdx.x & 31, e = lane % E, g = lane / E;
    const int nb = (int)gridDim.x;
    double acc = 0.0;
    for (int i0 = g; i0 < nb; i0 += 8 * GR) {
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = i0 + k * GR;
            v[k] = i < nb ? __ldcg(&part[(long long)i * E + e]) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (i0 + k * GR < nb) acc += v[k];
    }
#pragma unroll
    for (int o = E; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane < E) G[lane] = acc;
}

// The three Cholesky QR passes of bnormalize in one cooperative launch (one
// block of QR_THREADS threads per SM, every block resident), after the block
// SpMV (bspmv_gram_kernel: M W and G0 = W^T M W): the per-block Gram partials
// of the two later passes go to regions of their own, a grid barrier
// separates the passes, and every block sums the partials itself in a fixed
// order and factors the B x B matrix, so that no launch boundary and no
// last-block reduction sits between them.  The same arithmetic as three
// bqr_scale_kernel launches:
//   R1 = chol(G0 + s I), V = W R1^{-1} (and M V); G1 = V^T M V,
//   R2 = chol(G1), V <- V R2^{-1}; G2, R3, V <- V R3^{-1};
//   Bout = R3 R2 R1 (W = V Bout).
// A breakdown of any pass sets flag bit 0, the one-pass test (cn2 given) bit
// 1.  bar[0] counts barrier arrivals, bar[1] exits; the last block to leave
// resets both.
constexpr int QR_THREADS = 512;
template <int B>
__global__ void __launch_bounds__(QR_THREADS, 1) bqr_fused_kernel(long long N, const double* __restrict__ G0,
                                                                  const double* __restrict__ W,
                                                                  const double* __restrict__ MW, long long ldw,
                                                                  double* __restrict__ V, double* __restrict__ MV,
                                                                  long long ldv, double shift_rel,
                                                                  double* __restrict__ part, double* __restrict__ Bout,
                                                                  int* __restrict__ flag, const double* __restrict__ cn2,
                                                                  int* __restrict__ bar, int* __restrict__ err,
                                                                  long long spin_limit) {
    constexpr int E = B * B;
    __shared__ double red[QR_THREADS / 32][E];
    __shared__ double tot[E];
    __shared__ double G[E];
    __shared__ double sri[E];
    __shared__ double Racc[E];  // R_k ... R_1 (block 0)
    const long long gstride = (long long)gridDim.x * E;
    for (int pass = 0; pass < 3; ++pass) {
        if (pass == 0) {
            if ((int)threadIdx.x < E) G[threadIdx.x] = G0[threadIdx.x];
        } else {
            if (!grid_barrier(&bar[0], pass * (int)gridDim.x, err, spin_limit)) return;
            if (threadIdx.x < 32) gram_from_partials<B>(part + (pass - 1) * gstride, G);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double R[B][B], Ri[B][B];
            const bool bad = bcholesky<B>(G, pass == 0 ? shift_rel : 0.0, R, Ri);
            for (int i = 0; i < B; ++i)
                for (int j = 0; j < B; ++j) sri[i * B + j] = Ri[i][j];
            if (blockIdx.x == 0) {
                if (bad) atomicOr(flag, 1);
                // the full Gram-Schmidt pass removed more than 100 x the norm left
                if (pass == 0 && cn2)
                    for (int r = 0; r < B; ++r)
                        if (!(cn2[r] <= 1e4 * G[r * B + r])) atomicOr(flag, 2);
                double P[B][B];
                for (int i = 0; i < B; ++i)
                    for (int j = 0; j < B; ++j) {
                        double t = 0.0;
                        for (int k = 0; k < B; ++k) t += R[i][k] * (pass ? Racc[k * B + j] : (k == j ? 1.0 : 0.0));
                        P[i][j] = t;
                    }
                for (int i = 0; i < B; ++i)
                    for (int j = 0; j < B; ++j) Racc[i * B + j] = P[i][j];
                if (pass == 2)
                    for (int e = 0; e < E; ++e) Bout[e] = Racc[e];
            }
        }
        __syncthreads();
        // every pass maps the same rows to the same thread, so the in-place
        // passes read only what this thread wrote
        const double* X = pass == 0 ? W : V;
        const double* MX = pass == 0 ? MW : MV;
        const long long ldx = pass == 0 ? ldw : ldv;
        double g[E];
#pragma unroll
        for (int e = 0; e < E; ++e) g[e] = 0.0;
        for (long long i = (long long)blockIdx.x * QR_THREADS + threadIdx.x; i < N;
             i += (long long)gridDim.x * QR_THREADS) {
            double x[B], mx[B], v[B], mvv[B];
#pragma unroll
            for (int r = 0; r < B; ++r) {
                x[r] = X[r * ldx + i];
                mx[r] = MX[r * ldx + i];
            }
#pragma unroll
            for (int l = 0; l < B; ++l) {
                double a = 0.0, b = 0.0;
#pragma unroll
                for (int r = 0; r <= l; ++r) {
                    a += x[r] * sri[r * B + l];
                    b += mx[r] * sri[r * B + l];
                }
                v[l] = a;
                mvv[l] = b;
                V[l * ldv + i] = a;
                MV[l * ldv + i] = b;
            }
            if (pass < 2)
#pragma unroll
                for (int q = 0; q < B; ++q)
#pragma unroll
                    for (int r = 0; r < B; ++r) g[q * B + r] += v[q] * mvv[r];
        }
        if (pass < 2) gram_block_partial<B, QR_THREADS>(g, red, part + pass * gstride, tot);
    }
    // leave: the last block out resets the counters for the next launch
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&bar[1], 1) == (int)gridDim.x - 1) {
            bar[0] = 0;
            bar[1] = 0;
            __threadfence();
        }
    }
}

// A_j[i][r] = C1[(cs + i) B + r] + C2[(cs + i) B + r]
template <int B>
__global__ void balpha_kernel(const double* __restrict__ C1, const double* __restrict__ C2, int cs,
                              double* __restrict__ A) {
    const int t = threadIdx.x;
    if (t < B * B) A[t] = C1[(cs + t / B) * B + t % B] + C2[(cs + t / B) * B + t % B];
}

// --------------------------------------------------------------- host side
namespace {

struct BlockWork {
    riga_ctx* c;
    int B;
    long long N, ld;
    int nch;        // row blocks of the tall-skinny kernels
    int cap;
    double* W;      // N x B
    double* MW;     // N x B
    double* X;      // N x B refinement iterate (low-precision fronts)
    double* Rr;     // N x B refinement residual
    double* C1;     // cap * B
    double* C2;
    double* part;   // nch * cap * B, then small partials
    double* small;  // B*B Gram, Rinv, R scratch
    double* cn2;    // B squared norms of the full pass's coefficient columns
    int* flag;
};

size_t dots_smem(int B) { return (size_t)(B * CH + 8 * TJ * B + TJ * (HR + 1)) * sizeof(double); }

// Two full classical Gram-Schmidt passes of W against columns 0..J of V
// (CGS2; the start block, and every step once the one-pass test failed)
template <int B>
int bortho_t(BlockWork& K, int J) {
    riga_ctx* c = K.c;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_REORTH, 4.0 * (double)K.N * J * sizeof(double), 8.0 * (double)K.N * J * B);
    const size_t sm = dots_smem(B);
    const int pstride = K.cap * B;
    { count_launch(c); bdots_kernel<B><<<K.nch, 256, sm, st>>>(c->MV.ptr, K.ld, J, K.W, K.N, K.part, pstride); }
    enqueue_reduce_cols(c, K.part, K.nch, J * B, pstride, K.C1);
    { count_launch(c); bupdate_dots_kernel<B><<<K.nch, 256, sm + (size_t)J * B * sizeof(double), st>>>(
        c->V.ptr, J, K.C1, c->MV.ptr, J, K.ld, K.W, K.N, K.part, pstride); }
    enqueue_reduce_cols(c, K.part, K.nch, J * B, pstride, K.C2);
    { count_launch(c); bupdate_kernel<B><<<K.nch, 256, (size_t)J * B * sizeof(double), st>>>(
        c->V.ptr, K.ld, J, K.C2, K.W, K.N, nullptr); }
    return RIGA_OK;
}

// The block three-term recurrence against columns u0..u0+Ju (the last one
// or two blocks; coefficients into C1 at their column positions), then one
// full pass against columns 0..J (coefficients into C2, squared column
// norms into cn2)
template <int B>
int brecur_t(BlockWork& K, int J, int u0, int Ju) {
    riga_ctx* c = K.c;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_REORTH, (2.0 * J + 2.0 * Ju + 3.0 * B) * (double)K.N * sizeof(double),
                     4.0 * (double)K.N * (J + Ju) * B);
    const size_t sm = dots_smem(B);
    const int pstride = K.cap * B;
    const unsigned gl = (unsigned)std::min<long long>((K.N + 255) / 256, 4 * 152);
    const double* MVu = c->MV.ptr + (long long)u0 * K.ld;
    double* Cl = K.C1 + (size_t)u0 * B;
    int* counter = K.flag + 1;
    count_launch(c);
    if (Ju == 2 * B) blocal_dots_kernel<B, 2 * B><<<gl, 256, 0, st>>>(MVu, K.ld, K.W, K.N, K.part, counter, Cl);
    else blocal_dots_kernel<B, B><<<gl, 256, 0, st>>>(MVu, K.ld, K.W, K.N, K.part, counter, Cl);
    { count_launch(c); bupdate_dots_kernel<B><<<K.nch, 256, sm + (size_t)Ju * B * sizeof(double), st>>>(
        c->V.ptr + (long long)u0 * K.ld, Ju, Cl, c->MV.ptr, J, K.ld, K.W, K.N, K.part, pstride); }
    enqueue_reduce_cols(c, K.part, K.nch, J * B, pstride, K.C2);
    { count_launch(c); bupdate_kernel<B><<<K.nch, 256, (size_t)J * B * sizeof(double), st>>>(
        c->V.ptr, K.ld, J, K.C2, K.W, K.N, K.cn2); }
    return RIGA_OK;
}

// W (N x B) -> M-orthonormal columns col..col+B-1 of V and M V; Bout = the
// triangular factor (W = V_new Bout).  Shifted Cholesky QR, then two plain
// passes (shifted CholeskyQR3): the shift s = 11 (N B + B (B+1)) u trace(W^T M W)
// keeps the first factorization defined however ill-conditioned W is (its
// directions along converged Ritz vectors are tiny), the next two restore
// M-orthonormality, and W = V Bout holds to rounding relative to ||W||.
template <int B>
int bnormalize_t(BlockWork& K, int col, double* Bout, bool one_pass) {
    riga_ctx* c = K.c;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_SPMV, (double)c->S.nnz * 12.0 + (double)K.N * 8.0 * 10.0 * B);
    const unsigned nbs = (unsigned)((K.N + SPMV_RPB - 1) / SPMV_RPB);
    double* G0 = K.small;
    double* G1 = G0 + B * B;
    double* R1 = G1 + B * B;
    double* R2 = R1 + B * B;
    double* V = c->V.ptr + (long long)col * K.ld;
    double* MV = c->MV.ptr + (long long)col * K.ld;
    const unsigned gb = (unsigned)((K.N + 255) / 256);
    const double shift = 11.0 * ((double)K.N * B + (double)B * (B + 1)) * 1.1102230246251565e-16;
    int* counter = K.flag + 1;
    const unsigned nbg = nbs;  // one group of SPMV_TPR lanes per row
    { count_launch(c); bspmv_gram_kernel<B><<<nbg, 256, 0, st>>>(K.N, c->rowptr.ptr, c->col.ptr, c->Mval.ptr, K.W, K.MW,
                                                               K.part, counter, G0); }
    c->stats.n_matvec += B;
    // the three passes in one cooperative launch where the device allows it
    // (one block per SM, every block resident)
    static int coop_blocks = -1;  // blocks per SM of the fused kernel, 0: no cooperative launch
    if (coop_blocks < 0) {
        int coop = 0, occ = 0;
        RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device));
        RIGA_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bqr_fused_kernel<B>, QR_THREADS, 0));
        coop_blocks = coop ? std::min(occ, 1) : 0;
    }
    if (coop_blocks > 0) {
        int nsm = 0;
        RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
        long long n = K.N, ldw = K.N, ldv = K.ld;
        const double* g0 = G0;
        const double* w = K.W;
        const double* mw = K.MW;
        double* part = K.part;
        int* flag = K.flag;
        const double* cn2 = one_pass ? K.cn2 : nullptr;
        int* bar = K.flag + 2;
        int* err = c->flag.ptr;
        long long lim = c->wait_limit;
        double sh = shift;
        void* args[] = {&n, &g0, &w, &mw, &ldw, &V, &MV, &ldv, &sh, &part, &Bout, &flag, &cn2, &bar, &err, &lim};
        const cudaError_t e = cudaLaunchCooperativeKernel((const void*)bqr_fused_kernel<B>,
                                                          dim3((unsigned)(coop_blocks * nsm)), dim3(QR_THREADS), args, 0, st);
        if (e == cudaSuccess) {
            count_launch(c);
            return RIGA_OK;
        }
        if (e != cudaErrorCooperativeLaunchTooLarge && e != cudaErrorNotSupported)
            return set_error(c, RIGA_ECUDA, std::string("cudaLaunchCooperativeKernel: ") + cudaGetErrorString(e));
        // the blocks cannot all be resident here (another process holds SMs):
        // the three separate passes from now on
        cudaGetLastError();
        coop_blocks = 0;
    }
    // shifted pass (W -> V, Gram of V into G1), then two plain passes in place
    { count_launch(c); bqr_scale_kernel<B><<<gb, 256, 0, st>>>(K.N, G0, shift, nullptr, nullptr, R1, K.flag, K.W, K.N,
                                                              K.MW, V, MV, K.ld, K.part, counter, G1,
                                                              one_pass ? K.cn2 : nullptr); }
    { count_launch(c); bqr_scale_kernel<B><<<gb, 256, 0, st>>>(K.N, G1, 0.0, R1, R2, nullptr, K.flag, V, K.ld, MV, V, MV,
                                                              K.ld, K.part, counter, G0, nullptr); }
    { count_launch(c); bqr_scale_kernel<B><<<gb, 256, 0, st>>>(K.N, G0, 0.0, R2, Bout, nullptr, K.flag, V, K.ld, MV, V,
                                                              MV, K.ld, nullptr, nullptr, nullptr, nullptr); }
    return RIGA_OK;
}

int bortho(BlockWork& K, int J) {
    if (J <= 0) return RIGA_OK;
    return K.B == 4 ? bortho_t<4>(K, J) : bortho_t<2>(K, J);
}
int brecur(BlockWork& K, int J, int u0, int Ju) {
    return K.B == 4 ? brecur_t<4>(K, J, u0, Ju) : brecur_t<2>(K, J, u0, Ju);
}
int bnormalize(BlockWork& K, int col, double* Bout, bool one_pass) {
    return K.B == 4 ? bnormalize_t<4>(K, col, Bout, one_pass) : bnormalize_t<2>(K, col, Bout, one_pass);
}

// Eigen-decomposition of a small symmetric c x c matrix (cyclic Jacobi):
// eigenvalues ascending in ev, eigenvectors as the columns of U (c x c,
// column-major).
void jacobi_small(int c, std::vector<double> A, std::vector<double>& ev, std::vector<double>& U) {
    U.assign((size_t)c * c, 0.0);
    for (int i = 0; i < c; ++i) U[(size_t)i * c + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)j * c + i]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < c; ++i)
            for (int j = 0; j < c; ++j) {
                tot += a(i, j) * a(i, j);
                if (i != j) off += a(i, j) * a(i, j);
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < c; ++p)
            for (int q = p + 1; q < c; ++q) {
                if (a(p, q) == 0.0) continue;
                const double tau = (a(q, q) - a(p, p)) / (2.0 * a(p, q));
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < c; ++k) {  // A <- J^T A J
                    const double akp = a(k, p), akq = a(k, q);
                    a(k, p) = cs * akp - sn * akq;
                    a(k, q) = sn * akp + cs * akq;
                }
                for (int k = 0; k < c; ++k) {
                    const double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = cs * apk - sn * aqk;
                    a(q, k) = sn * apk + cs * aqk;
                }
                for (int k = 0; k < c; ++k) {
                    const double ukp = U[(size_t)p * c + k], ukq = U[(size_t)q * c + k];
                    U[(size_t)p * c + k] = cs * ukp - sn * ukq;
                    U[(size_t)q * c + k] = sn * ukp + cs * ukq;
                }
            }
    }
    std::vector<int> ord(c);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return a(x, x) < a(y, y); });
    std::vector<double> U2((size_t)c * c);
    ev.assign(c, 0.0);
    for (int i = 0; i < c; ++i) {
        ev[i] = a(ord[i], ord[i]);
        for (int k = 0; k < c; ++k) U2[(size_t)i * c + k] = U[(size_t)ord[i] * c + k];
    }
    U.swap(U2);
}

// Residual estimates of a cluster of (numerically) equal Ritz values: the
// estimate of a vector s of the cluster's eigenspace is ||B_m s_last||, which
// depends on the basis chosen inside the cluster.  With E = B_m S_last (B x c,
// S_last the cluster's last rows), the eigenvectors of E^T E rotate the basis
// so that the estimates become sqrt of its eigenvalues, ascending: the
// converged directions of the cluster come first.  rot (c x c) is returned.
void cluster_estimates(int B, int c, const double* Bm, const std::vector<double>& last /* B x c */,
                       std::vector<double>& est, std::vector<double>& rot) {
    std::vector<double> E((size_t)B * c, 0.0), G((size_t)c * c, 0.0);
    for (int k = 0; k < c; ++k)
        for (int r = 0; r < B; ++r) {
            double v = 0.0;
            for (int l = 0; l < B; ++l) v += Bm[r * B + l] * last[(size_t)k * B + l];
            E[(size_t)k * B + r] = v;
        }
    for (int i = 0; i < c; ++i)
        for (int j = 0; j < c; ++j) {
            double v = 0.0;
            for (int r = 0; r < B; ++r) v += E[(size_t)i * B + r] * E[(size_t)j * B + r];
            G[(size_t)j * c + i] = v;
        }
    std::vector<double> ev;
    jacobi_small(c, G, ev, rot);
    est.assign(c, 0.0);
    for (int i = 0; i < c; ++i) est[i] = std::sqrt(std::max(ev[i], 0.0));
}

// clusters of acceptable Ritz values that agree to 1e-11 relative (equal
// for the residual tolerance), as [begin, end) ranges of ord (sorted by
// |theta| descending)
std::vector<std::pair<int, int>> ritz_clusters(const std::vector<int>& ord, const std::vector<double>& theta) {
    std::vector<std::pair<int, int>> cl;
    for (int i = 0; i < (int)ord.size();) {
        int j = i + 1;
        while (j < (int)ord.size() &&
               std::fabs(theta[ord[j]] - theta[ord[i]]) <= 1e-11 * std::fabs(theta[ord[i]]))
            ++j;
        cl.push_back({i, j});
        i = j;
    }
    return cl;
}

// the block-tridiagonal T (n = m B) from the diagonal blocks A (row-major
// B x B each, symmetrised) and the sub-diagonal blocks Bs[1..m-1]
void build_T(int m, int B, const double* A, const double* Bs, std::vector<double>& T) {
    const int n = m * B;
    T.assign((size_t)n * n, 0.0);
    for (int j = 0; j < m; ++j) {
        const double* a = A + (size_t)j * B * B;
        for (int i = 0; i < B; ++i)
            for (int l = 0; l < B; ++l) T[(size_t)(j * B + l) * n + j * B + i] = 0.5 * (a[i * B + l] + a[l * B + i]);
        if (j + 1 < m) {
            const double* b = Bs + (size_t)(j + 1) * B * B;  // W_j = V_{j+1} B_{j+1}
            for (int i = 0; i < B; ++i)
                for (int l = 0; l < B; ++l) {
                    T[(size_t)(j * B + l) * n + (j + 1) * B + i] = b[i * B + l];  // T[(j+1)B+i][jB+l]
                    T[(size_t)((j + 1) * B + i) * n + j * B + l] = b[i * B + l];  // symmetric
                }
        }
    }
}

}  // namespace

int block_run(Run& R, int B, int nlock, int want_run, int m_max, double cur_sigma, double sigma0, double tol_est,
              double lock_tol, int lock_cap, uint64_t& seed, std::vector<double>& lam, int* m_out, int* n_locked) {
    static const bool dbg = std::getenv("RIGA_DEBUG") != nullptr;
    riga_ctx* c = R.c;
    cudaStream_t st = c->stream;
    const long long N = R.N;
    *m_out = 0;
    *n_locked = 0;
    if (B != 2 && B != 4) return set_error(c, RIGA_EINVAL, "block size must be 2 or 4");
    const int nblk = std::max(1, m_max / B);
    const int col0 = nlock;
    if (col0 + (nblk + 1) * B > R.cap) return set_error(c, RIGA_ENOMEM, "Lanczos basis capacity");
    BlockWork K;
    K.c = c;
    K.B = B;
    K.N = N;
    K.ld = R.ld;
    int nsm = 0;
    RIGA_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    nsm = std::max(nsm, 1);
    {
        const long long nchunk = (N + CH - 1) / CH;
        K.nch = (int)((nchunk + nsm - 1) / nsm * nsm);  // row blocks: a multiple of the SM count, <= CH rows each
    }
    K.cap = R.cap;
    const unsigned nbs = (unsigned)((N + SPMV_RPB - 1) / SPMV_RPB);
    // the largest user: the dot partials, the last-block reductions, or the
    // fused QR's two Gram regions (one block per SM)
    const size_t part_n = std::max<size_t>({(size_t)K.nch * K.cap * B, (size_t)std::max<unsigned>(nbs, 304) * B * B,
                                            (size_t)4 * 152 * 2 * B * B, (size_t)2 * nsm * B * B});
    const size_t nAB = (size_t)(2 * nblk + 1) * B * B;  // the T blocks: A_0..A_{nblk-1}, B_0..B_nblk
    RIGA_CUDA_TRY(c, c->bwork.alloc((size_t)4 * N * B));
    RIGA_CUDA_TRY(c, c->bcoef.alloc((size_t)2 * K.cap * B));
    RIGA_CUDA_TRY(c, c->bpartial.alloc(part_n));
    RIGA_CUDA_TRY(c, c->bsmall.alloc((size_t)5 * B * B + nAB));
    RIGA_CUDA_TRY(c, c->bflag.alloc(4));
    if (c->bpin_size < nAB + 2) {
        if (c->bpin) cudaFreeHost(c->bpin);
        c->bpin = nullptr;
        c->bpin_size = 0;
        RIGA_CUDA_TRY(c, cudaMallocHost(&c->bpin, (nAB + 2) * sizeof(double)));
        c->bpin_size = nAB + 2;
    }
    K.W = c->bwork.ptr;
    K.MW = c->bwork.ptr + (size_t)N * B;
    K.X = c->bwork.ptr + (size_t)2 * N * B;
    K.Rr = c->bwork.ptr + (size_t)3 * N * B;
    K.C1 = c->bcoef.ptr;
    K.C2 = c->bcoef.ptr + (size_t)K.cap * B;
    K.part = c->bpartial.ptr;
    K.small = c->bsmall.ptr;
    K.flag = c->bflag.ptr;
    K.cn2 = c->bsmall.ptr + 4 * B * B;
    double* dA = c->bsmall.ptr + 5 * B * B;  // nblk diagonal blocks, then nblk + 1 sub-diagonal blocks
    double* dB = dA + (size_t)nblk * B * B;
    double* hA = c->bpin;                   // pinned host copies, same layout
    double* hB = hA + (size_t)nblk * B * B;
    int* hflags = reinterpret_cast<int*>(hA + nAB);  // [0] QR breakdown (1), one-pass test failed (2); [1] solve wait flag
    const size_t smx = dots_smem(B) + (size_t)K.cap * B * sizeof(double);
    if (B == 4) {
        RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bdots_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dots_smem(4)));
        RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bupdate_dots_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx));
        RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bupdate_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)((size_t)K.cap * B * sizeof(double))));
    } else {
        RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bdots_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dots_smem(2)));
        RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bupdate_dots_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx));
        RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bupdate_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)((size_t)K.cap * B * sizeof(double))));
    }
    // breakdown flag, reduction counter, grid-barrier arrivals and exits
    RIGA_CUDA_TRY(c, cudaMemsetAsync(K.flag, 0, 4 * sizeof(int), st));

    // start block: B random vectors, M-orthogonal to the locked ones
    enqueue_start_vector(c, (long long)N * B, seed, K.W);
    int rc = bortho(K, nlock);
    if (rc) return rc;
    rc = bnormalize(K, col0, dB, false);
    if (rc) return rc;

    std::vector<double> T, theta, Zl;
    bool breakdown = false;
    auto acceptable = [&](double th) { return th != 0.0 && cur_sigma + 1.0 / th > sigma0; };
    // copies of the first mm diagonal and mm + 1 sub-diagonal blocks and the
    // flags into pinned memory (asynchronous)
    auto enqueue_fetch = [&](int mm) -> int {
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(hA, dA, (size_t)mm * B * B * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(hB, dB, (size_t)(mm + 1) * B * B * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(hflags, K.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(hflags + 1, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
        return RIGA_OK;
    };
    // Ritz values of T_mm and residual estimates ||B_mm s_last|| for all of them
    auto ritz = [&](int mm, std::vector<double>& est) {
        const int n = mm * B;
        build_T(mm, B, hA, hB, T);
        theta.assign(n, 0.0);
        Zl.assign((size_t)B * n, 0.0);
        band_eig_lastrows(n, B, T.data(), B, theta.data(), Zl.data());
        const double* b = hB + (size_t)mm * B * B;
        est.assign(n, 0.0);
        for (int i = 0; i < n; ++i) {
            double e2 = 0.0;
            for (int r = 0; r < B; ++r) {
                double v = 0.0;
                for (int l = 0; l < B; ++l) v += b[r * B + l] * Zl[(size_t)i * B + l];
                e2 += v * v;
            }
            est[i] = std::sqrt(e2);
        }
    };
    // converged: the want_run acceptable Ritz values of largest |theta| all
    // have estimates below tol_est |theta|
    std::vector<double> est;  // residual estimates of the last Rayleigh-Ritz (check or final)
    auto converged = [&](int mm) {
        ritz(mm, est);
        std::vector<int> ord;
        for (int i = 0; i < mm * B; ++i)
            if (acceptable(theta[i])) ord.push_back(i);
        if (dbg) {  // leading acceptable Ritz values whose estimates meet the bar
            std::vector<int> o2(ord);
            std::sort(o2.begin(), o2.end(), [&](int x, int y) { return std::fabs(theta[x]) > std::fabs(theta[y]); });
            int lead = 0;
            while (lead < (int)o2.size() && est[o2[lead]] <= tol_est * std::fabs(theta[o2[lead]])) ++lead;
            std::fprintf(stderr, "[riga] block check: steps=%d acceptable=%zu leading converged=%d\n", mm * B, o2.size(), lead);
        }
        if ((int)ord.size() < want_run) return false;
        std::sort(ord.begin(), ord.end(), [&](int x, int y) { return std::fabs(theta[x]) > std::fabs(theta[y]); });
        const double* bm = hB + (size_t)mm * B * B;
        int counted = 0;
        for (const auto& cr : ritz_clusters(ord, theta)) {
            const int cn = cr.second - cr.first;
            std::vector<double> last((size_t)B * cn), cest, rot;
            for (int k = 0; k < cn; ++k)
                for (int l = 0; l < B; ++l) last[(size_t)k * B + l] = Zl[(size_t)ord[cr.first + k] * B + l];
            cluster_estimates(B, cn, bm, last, cest, rot);
            for (int k = 0; k < cn && counted < want_run; ++k, ++counted)
                if (!(cest[k] <= tol_est * std::fabs(theta[ord[cr.first]]))) return false;
            if (counted >= want_run) break;
        }
        return counted >= want_run;
    };

    // Checks are lagged: the block copies of step m are queued with an
    // event, the host evaluates them while the GPU runs the next steps, and
    // it never runs more than two block steps ahead of an unevaluated check
    // (a converged check leaves the steps issued after it unused; three
    // steps measured no better on the 2D benchmark: 1 ms less idle, one
    // more block step per run).
    const int ck = std::max(1, 8 / B);  // block steps between checks
    cudaEvent_t ev;
    RIGA_CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    int pending = -1, m = 0, m_conv = 0;
    bool done = false;
    for (int j = 0; j < nblk && !done; ++j) {
        const int cj = col0 + j * B;
        rc = RIGA_OK;
        if (cudaMemcpyAsync(K.W, c->MV.ptr + (long long)cj * R.ld, (size_t)N * B * sizeof(double),
                            cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = set_error(c, RIGA_ECUDA, "block copy");
        if (rc == RIGA_OK) {
            rc = solve_refined_multi(c, K.W, K.X, K.Rr, B, c->ir_sweeps);
        }
        const bool one_pass = !R.cgs2;
        if (rc == RIGA_OK) rc = one_pass ? brecur(K, cj + B, j == 0 ? cj : cj - B, j == 0 ? B : 2 * B) : bortho(K, cj + B);
        if (rc == RIGA_OK) {
            count_launch(c);
            if (B == 4) balpha_kernel<4><<<1, 32, 0, st>>>(K.C1, K.C2, cj, dA + (size_t)j * B * B);
            else balpha_kernel<2><<<1, 32, 0, st>>>(K.C1, K.C2, cj, dA + (size_t)j * B * B);
            rc = bnormalize(K, cj + B, dB + (size_t)(j + 1) * B * B, one_pass);
        }
        if (rc) {
            cudaEventDestroy(ev);
            return rc;
        }
        c->stats.steps += B;
        m = j + 1;
        if (pending >= 0 && (m - pending >= 2 || cudaEventQuery(ev) == cudaSuccess)) {
            cudaEventSynchronize(ev);
            if (hflags[1] & 2) {
                cudaEventDestroy(ev);
                return set_error(c, RIGA_ETIMEOUT, "a dependency wait of the tree solve gave up");
            }
            breakdown = (hflags[0] & 1) != 0;
            if (hflags[0] & 2) R.cgs2 = true;  // two full passes from now on
            done = breakdown;
            if (!done && converged(pending)) {
                done = true;
                m_conv = pending;  // theta, Zl, est, T and hB now hold T_pending's decomposition
            }
            pending = -1;
        }
        if (!done && pending < 0 && m * B >= want_run && m % ck == 0 && m < nblk) {
            rc = enqueue_fetch(m);
            if (rc) {
                cudaEventDestroy(ev);
                return rc;
            }
            cudaEventRecord(ev, st);
            pending = m;
        }
    }
    cudaEventDestroy(ev);
    *m_out = m * B;
    if (m == 0) return RIGA_OK;
    // Rayleigh-Ritz with vectors: every acceptable Ritz pair whose estimate
    // meets the bar, largest |theta| first, up to the locking room.  A run
    // that a check found converged uses that check's T_pending and its
    // decomposition (the blocks V_1 .. V_pending are final; the steps issued
    // after the check only extended the basis), so the host computes no
    // second decomposition while the GPU idles; the flags of those later
    // steps are read after the locking.
    const bool reuse = m_conv > 0;
    if (reuse) {
        m = m_conv;
    } else {
        rc = enqueue_fetch(m);
        if (rc) return rc;
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
        if (hflags[1] & 2) return set_error(c, RIGA_ETIMEOUT, "a dependency wait of the tree solve gave up");
        breakdown = (hflags[0] & 1) != 0;
        if (hflags[0] & 2) R.cgs2 = true;
        ritz(m, est);
    }
    const int n = m * B;
    std::vector<int> ord;
    for (int i = 0; i < n; ++i)
        if (acceptable(theta[i])) ord.push_back(i);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return std::fabs(theta[x]) > std::fabs(theta[y]); });
    // eigenvectors (one inverse-iteration call, so that close Ritz values get
    // orthogonal vectors) of every cluster that may hold a converged
    // direction; per cluster, rotated so that the converged directions
    // separate from the others; keep those whose estimate meets the bar, up
    // to the locking room
    const double* bm = hB + (size_t)m * B * B;
    const int room = std::max(lock_cap - nlock, 0);
    const auto cls = ritz_clusters(ord, theta);
    std::vector<int> keep;  // cluster indices
    std::vector<double> thv;
    for (int ci = 0; ci < (int)cls.size(); ++ci) {
        const auto& cr = cls[ci];
        double best = 1e300;
        for (int k = cr.first; k < cr.second; ++k) best = std::min(best, est[ord[k]]);
        if (cr.second - cr.first == 1 && !(best <= 1e3 * tol_est * std::fabs(theta[ord[cr.first]]))) continue;
        keep.push_back(ci);
        for (int k = cr.first; k < cr.second; ++k) thv.push_back(theta[ord[k]]);
    }
    std::vector<double> Sall((size_t)n * thv.size());
    band_eigvecs(n, B, T.data(), (int)thv.size(), thv.data(), Sall.data());
    std::vector<double> Wsel, lcand;
    size_t col = 0;
    for (int ci : keep) {
        const auto& cr = cls[ci];
        const int cn = cr.second - cr.first;
        const double* Sc = Sall.data() + col * n;
        col += cn;
        if ((int)lcand.size() >= room) continue;
        const double th0 = theta[ord[cr.first]];
        std::vector<double> last((size_t)B * cn), cest, rot;
        for (int k = 0; k < cn; ++k)
            for (int l = 0; l < B; ++l) last[(size_t)k * B + l] = Sc[(size_t)k * n + (n - B) + l];
        cluster_estimates(B, cn, bm, last, cest, rot);
        for (int k = 0; k < cn && (int)lcand.size() < room; ++k) {
            if (!(cest[k] <= tol_est * std::fabs(th0))) break;  // ascending: the rest are worse
            std::vector<double> v(n, 0.0);
            for (int q = 0; q < cn; ++q) {
                const double w = rot[(size_t)k * cn + q];
                for (int i = 0; i < n; ++i) v[i] += w * Sc[(size_t)q * n + i];
            }
            Wsel.insert(Wsel.end(), v.begin(), v.end());
            lcand.push_back(cur_sigma + 1.0 / th0);
        }
    }
    if (dbg)
        std::fprintf(stderr, "[riga] block run: B=%d steps=%d (blocks %d/%d) breakdown=%d cgs2=%d candidates=%zu\n", B,
                     n, m, nblk, (int)breakdown, (int)R.cgs2, lcand.size());
    rc = ritz_lock(R, col0, n, Wsel, lcand, nlock, lock_tol, lam, n_locked);
    if (rc || !reuse) return rc;
    // flags of the steps issued after the converged check (ritz_lock has
    // synchronized the stream)
    RIGA_CUDA_TRY(c, cudaMemcpy(hflags, K.flag, sizeof(int), cudaMemcpyDeviceToHost));
    RIGA_CUDA_TRY(c, cudaMemcpy(hflags + 1, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (hflags[1] & 2) return set_error(c, RIGA_ETIMEOUT, "a dependency wait of the tree solve gave up");
    if (hflags[0] & 2) R.cgs2 = true;
    return RIGA_OK;
}

}  // namespace riga
