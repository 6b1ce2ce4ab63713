// Shift-and-invert Lanczos in the M-inner product (Sec. 4.1-4.2 of arXiv
// 2009.08167) on H = (K - sigma M)^{-1} M, vectors in elimination order.
//
// Per step j (Eq. LanczosAlphaBeta): w = H v_j = A^{-1} (M v_j) with the
// stored M v_j; full reorthogonalization (Sec. 4.2: against all previously
// stored Lanczos vectors) in the M-inner product: the three-term recurrence
// with alpha_j and beta_j computed as inner products against v_j and
// v_{j-1}, then one classical Gram-Schmidt pass against [Y V_j] (Y = locked
// eigenvectors of this and earlier shifts: deflation), or two full passes
// once that pass removed more than 100 times the norm left (or when
// riga_set_reorth asks for them); alpha_j = the recurrence coefficient plus
// its correction; beta_{j+1} = ||w||_M; v_{j+1} = w / beta_{j+1}; M v_{j+1}
// stored from the same SpMV.  Rayleigh-Ritz on T_m (Eq. RitzValues) on the
// host every few steps with the last eigenvector row only (residual
// estimates |beta_{m+1} w_m|), Ritz vectors V_m W by a device GEMM.
// Converged pairs are locked; runs restart from a fresh random vector until
// the Sylvester inertia at a check shift in a spectral gap equals the number
// of locked eigenvalues below it (Remark on inertia); with spectrum slicing
// that check shift becomes the next shift.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <numeric>

#include "lanczos.h"

namespace riga {

// Partial dots out[j] = sum_{r in chunk} B[j][r] ws[r] for j < J over one
// chunk of at most CH rows.  Each 32-column tile is staged through shared
// memory in HR-row pieces by coalesced column loads (the small pieces leave
// room for six blocks per SM); the next piece is loaded into registers while
// the current one is summed;
// thread (column jl, row group g) sums rows g, g+8, ... with one FP64 FMA per
// element (GB300's FP64 pipe is the bound of these tall-skinny products), and
// the 8 row groups are added through shared memory.
__device__ __forceinline__ void chunk_dots(const double* __restrict__ B, long long ld, int J, long long r0, int rows,
                                           const double* __restrict__ ws, double* __restrict__ Vs,
                                           double* __restrict__ red, double* __restrict__ out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (rows <= 0) {  // no rows (the same for the whole block): zero partials
        for (int j = tid; j < J; j += blockDim.x) out[j] = 0.0;
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
            const double* col = B + (long long)(j0 + jl) * ld + r0 + h;
#pragma unroll
            for (int i = 0; i < HR / 32; ++i) {
                const int r = lane + 32 * i;
                pre[q][i] = (jl < jn && r < hn) ? col[r] : 0.0;
            }
        }
    };
    if (nst > 0) load(0);
    double s = 0.0;
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
            const double* wh = ws + h;
#pragma unroll 4
            for (int r = warp; r < hn; r += 8) s += vc[r] * wh[r];
        }
        __syncthreads();
        if (st % nh == nh - 1) {  // last piece of this column tile: sum the 8 row groups
            red[warp * TJ + lane] = s;
            s = 0.0;
            __syncthreads();
            if (tid < jn) {
                double t = 0.0;
#pragma unroll
                for (int gg = 0; gg < 8; ++gg) t += red[gg * TJ + tid];
                out[j0 + tid] = t;
            }
        }
    }
    __syncthreads();
}

// Partial dots of the recurrence over one chunk of CH rows: out[j] = sum of
// B_j[row] w[row] for the JU = 1 or 2 columns of the last two vectors (64
// threads, four rows each, then the block's sum)
template <int JU>
__global__ void __launch_bounds__(64) local_dots_kernel(const double* __restrict__ B, long long ld,
                                                        const double* __restrict__ w, long long N,
                                                        double* __restrict__ partial, int pstride) {
    __shared__ double red[2][JU];
    const long long r0 = (long long)blockIdx.x * CH;
    double acc[JU];
#pragma unroll
    for (int j = 0; j < JU; ++j) acc[j] = 0.0;
#pragma unroll
    for (int i = 0; i < CH / 64; ++i) {
        const long long r = r0 + threadIdx.x + 64 * i;
        if (r < N) {
            const double x = w[r];
#pragma unroll
            for (int j = 0; j < JU; ++j) acc[j] += B[(long long)j * ld + r] * x;
        }
    }
#pragma unroll
    for (int j = 0; j < JU; ++j)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int j = 0; j < JU; ++j) red[threadIdx.x >> 5][j] = acc[j];
    __syncthreads();
    if ((int)threadIdx.x < JU) partial[(long long)blockIdx.x * pstride + threadIdx.x] = red[0][threadIdx.x] + red[1][threadIdx.x];
}

__global__ void __launch_bounds__(256) gemvT_partial_kernel(const double* __restrict__ B, long long ld, int J,
                                                            const double* __restrict__ w, long long N,
                                                            double* __restrict__ partial, int pstride) {
    extern __shared__ double sh[];
    double* ws = sh;                    // CH
    double* red = ws + CH;              // 8 * TJ
    double* Vs = red + 8 * TJ;          // TJ * (HR + 1)
    const long long r0 = (long long)blockIdx.x * CH;
    const int tid = threadIdx.x;
    ws[tid] = (r0 + tid < N) ? w[r0 + tid] : 0.0;
    __syncthreads();
    const int rows = (int)min((long long)CH, N - r0);
    chunk_dots(B, ld, J, r0, rows, ws, Vs, red, partial + (long long)blockIdx.x * pstride);
}

// out[j] = sum over chunks of partial[c][j]: 32 columns per block, 8 chunk
// groups per column, fixed summation order (deterministic)
__global__ void __launch_bounds__(256) reduce_cols_kernel(const double* __restrict__ partial, int nch, int J,
                                                          int pstride, double* __restrict__ out) {
    __shared__ double red[8][33];
    const int jl = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + jl;
    double s = 0.0;
    if (j < J) {
#pragma unroll 4
        for (int c = g; c < nch; c += 8) s += partial[(long long)c * pstride + j];
    }
    red[g][jl] = s;
    __syncthreads();
    if (g == 0 && j < J) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[q][jl];
        out[j] = t;
    }
}

// v - sum_j V[j][r] c[j] with the loads issued eight at a time
__device__ __forceinline__ double row_update(const double* __restrict__ V, long long ld, int J, long long r,
                                             const double* __restrict__ cs, double v) {
    int j = 0;
    for (; j + 8 <= J; j += 8) {
        double b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = V[(long long)(j + q) * ld + r];
#pragma unroll
        for (int q = 0; q < 8; ++q) v -= b[q] * cs[j + q];
    }
    for (; j < J; ++j) v -= V[(long long)j * ld + r] * cs[j];
    return v;
}

// w -= V[:, 0..Ju) c1 on this chunk, then partial dots MV[:, 0..Jd)^T w
__global__ void __launch_bounds__(256) update_gemvT_kernel(const double* __restrict__ V, int Ju,
                                                           const double* __restrict__ c1,
                                                           const double* __restrict__ MV, int Jd, long long ld,
                                                           double* __restrict__ w, long long N,
                                                           double* __restrict__ partial, int pstride) {
    extern __shared__ double sh[];
    double* ws = sh;                    // CH
    double* red = ws + CH;              // 8 * TJ
    double* Vs = red + 8 * TJ;          // TJ * (HR + 1)
    double* cs = Vs + TJ * (HR + 1);    // Ju
    const long long r0 = (long long)blockIdx.x * CH;
    const int tid = threadIdx.x;
    for (int j = tid; j < Ju; j += blockDim.x) cs[j] = c1[j];
    __syncthreads();
    const long long r = r0 + tid;
    double v = 0.0;
    if (r < N) {
        v = row_update(V, ld, Ju, r, cs, w[r]);
        w[r] = v;
    }
    ws[tid] = v;
    __syncthreads();
    const int rows = (int)min((long long)CH, N - r0);
    chunk_dots(MV, ld, Jd, r0, rows, ws, Vs, red, partial + (long long)blockIdx.x * pstride);
}

__global__ void gemv_update_kernel(const double* __restrict__ V, long long ld, int J, const double* __restrict__ c,
                                   double* __restrict__ w, long long N) {
    extern __shared__ double cs[];
    for (int j = threadIdx.x; j < J; j += blockDim.x) cs[j] = c[j];
    __syncthreads();
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    w[r] = row_update(V, ld, J, r, cs, w[r]);
}

// y = M x over the permuted CSR (SPMV_TPR lanes per row) and per-block partial x.y
__global__ void __launch_bounds__(256) spmv_dot_kernel(long long N, const long long* __restrict__ rowptr,
                                                       const int* __restrict__ col, const double* __restrict__ Mv,
                                                       const double* __restrict__ x, double* __restrict__ y,
                                                       double* __restrict__ partial) {
    __shared__ double red[8];
    const long long row = (long long)blockIdx.x * SPMV_RPB + threadIdx.x / SPMV_TPR;
    const int lane = threadIdx.x & (SPMV_TPR - 1);
    double s = 0.0;
    if (row < N)
        for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) s += Mv[e] * x[col[e]];
    s = group_sum(s);
    double d = 0.0;
    if (row < N && lane == 0) {
        y[row] = s;
        d = s * x[row];
    }
    d = warp_sum_groups(d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < 8; ++i) tot += red[i];
        partial[blockIdx.x] = tot;
    }
}

// beta_{j+1} = sqrt(w^T M w) from the SpMV's partials, alpha_j = c1[col1] +
// c2[col]; with one full Gram-Schmidt pass (Jc > 0), bit 2 of *flag when that
// pass removed more than 100 x the norm left (sum of c2[0..Jc)^2 > 1e4 beta^2)
__global__ void finalize_kernel(const double* __restrict__ partial, int nb, const double* __restrict__ c1, int col1,
                                const double* __restrict__ c2, int col, int j, double* __restrict__ alpha,
                                double* __restrict__ beta, int Jc, int* __restrict__ flag) {
    __shared__ double sh[256];
    __shared__ double sq[256];
    double s = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
    for (int i = threadIdx.x; i < Jc; i += blockDim.x) q += c2[i] * c2[i];
    sh[threadIdx.x] = s;
    sq[threadIdx.x] = q;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[threadIdx.x] += sh[threadIdx.x + o];
            sq[threadIdx.x] += sq[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (j >= 0) alpha[j] = c1[col1] + c2[col];
        const double b2 = fmax(sh[0], 0.0);
        beta[j + 1] = sqrt(b2);
        if (Jc > 0 && !(sq[0] <= 1e4 * b2)) atomicOr(flag, 2);
    }
}

__global__ void normalize_kernel(long long N, const double* __restrict__ w, const double* __restrict__ Mw,
                                 const double* __restrict__ bptr, double* __restrict__ v, double* __restrict__ mv) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double b = *bptr;
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    v[r] = w[r] * inv;
    mv[r] = Mw[r] * inv;
}

// U[:, i] = sum_j V[:, j] W[j, i] for i < nsel (rows by threads, 16 outputs each)
__global__ void __launch_bounds__(256) gemm_ritz_kernel(const double* __restrict__ V, long long ld, int J,
                                                        const double* __restrict__ W, int ldw, int nsel,
                                                        double* __restrict__ U, long long ldu, long long N) {
    __shared__ double Ws[128][16];
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i0 = blockIdx.y * 16;
    double acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int j0 = 0; j0 < J; j0 += 128) {
        const int jn = min(128, J - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < 128 * 16; t += blockDim.x) {
            int jj = t / 16, q = t % 16;
            Ws[jj][q] = (jj < jn && i0 + q < nsel) ? W[(long long)(i0 + q) * ldw + j0 + jj] : 0.0;
        }
        __syncthreads();
        if (r < N) {
            for (int jj = 0; jj < jn; ++jj) {
                double v = V[(long long)(j0 + jj) * ld + r];
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] += v * Ws[jj][q];
            }
        }
    }
    if (r < N)
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (i0 + q < nsel) U[(long long)(i0 + q) * ldu + r] = acc[q];
}

// Double-double arithmetic (Knuth's TwoSum, the FMA form of TwoProduct):
// (hi, lo) represents hi + lo with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ void dd_add(double& hi, double& lo, double bh, double bl) {
    const double s = hi + bh;
    const double bb = s - hi;
    double e = (hi - (s - bb)) + (bh - bb);
    e += lo + bl;
    hi = s + e;
    lo = e - (hi - s);
}
__device__ __forceinline__ void dd_add_prod(double& hi, double& lo, double a, double b) {
    const double p = a * b;
    dd_add(hi, lo, p, fma(a, b, -p));
}

// Rayleigh-quotient partial sums per (block, candidate q) in double-double:
// u^T K u = sum_i u_i sum_j K_ij u_j and u^T M u = sum_i u_i (M u)_i, every
// product and sum error-free transformed, so that the quotient carries the
// rounding of the stored u, K and M only (K u cancels heavily for the low
// eigenvalues: its plain FP64 sum would lose ||K|| / lambda ulps).  partial
// holds (uKu_hi, uKu_lo, uMu_hi, uMu_lo) per (q, block).
__global__ void __launch_bounds__(256) rq_cols_kernel(long long N, const long long* __restrict__ rowptr,
                                                      const int* __restrict__ col, const double* __restrict__ Kv,
                                                      const double* __restrict__ U, const double* __restrict__ MU,
                                                      long long ld, double* __restrict__ partial) {
    __shared__ double sh[4][8];
    const int q = blockIdx.y;
    const double* u = U + (long long)q * ld;
    const double* mu = MU + (long long)q * ld;
    const int lane = threadIdx.x & (SPMV_TPR - 1), grp = threadIdx.x / SPMV_TPR;
    double kh = 0.0, kl = 0.0, mh = 0.0, ml = 0.0;
    for (long long it = blockIdx.x; it * SPMV_RPB < N; it += gridDim.x) {
        const long long row = it * SPMV_RPB + grp;
        double sh_ = 0.0, sl_ = 0.0;
        if (row < N)
            for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) dd_add_prod(sh_, sl_, Kv[e], u[col[e]]);
#pragma unroll
        for (int o = SPMV_TPR / 2; o > 0; o >>= 1) {
            const double oh = __shfl_xor_sync(0xffffffffu, sh_, o, SPMV_TPR);
            const double ol = __shfl_xor_sync(0xffffffffu, sl_, o, SPMV_TPR);
            dd_add(sh_, sl_, oh, ol);
        }
        if (lane == 0 && row < N) {
            const double ui = u[row];
            const double p = ui * sh_;
            dd_add(kh, kl, p, fma(ui, sh_, -p) + ui * sl_);
            dd_add_prod(mh, ml, ui, mu[row]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double a = __shfl_xor_sync(0xffffffffu, kh, o), b = __shfl_xor_sync(0xffffffffu, kl, o);
        const double c2 = __shfl_xor_sync(0xffffffffu, mh, o), d = __shfl_xor_sync(0xffffffffu, ml, o);
        dd_add(kh, kl, a, b);
        dd_add(mh, ml, c2, d);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = kh;
        sh[1][threadIdx.x >> 5] = kl;
        sh[2][threadIdx.x >> 5] = mh;
        sh[3][threadIdx.x >> 5] = ml;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double th = 0.0, tl = 0.0, vh = 0.0, vl = 0.0;
        for (int i = 0; i < 8; ++i) {
            dd_add(th, tl, sh[0][i], sh[1][i]);
            dd_add(vh, vl, sh[2][i], sh[3][i]);
        }
        double* out = partial + ((long long)q * gridDim.x + blockIdx.x) * 4;
        out[0] = th;
        out[1] = tl;
        out[2] = vh;
        out[3] = vl;
    }
}

// M u of every candidate q into MU (the matrix and u read once for both
// products), and for q < nres the residual partial sums per block
// ||K u - lam M u||^2 and ||M u||^2 (SPMV_TPR lanes per row; grid-stride
// over groups of rows)
__global__ void __launch_bounds__(256) resid_cols_kernel(long long N, const long long* __restrict__ rowptr,
                                                         const int* __restrict__ col, const double* __restrict__ Kv,
                                                         const double* __restrict__ Mv, const double* __restrict__ U,
                                                         double* __restrict__ MU, long long ld,
                                                         const double* __restrict__ lam, int nres,
                                                         double* __restrict__ partial) {
    __shared__ double sa[8], sb[8];
    const int q = blockIdx.y;
    const bool res = q < nres;
    const double l = res ? lam[q] : 0.0;
    const double* u = U + (long long)q * ld;
    double* mu = MU + (long long)q * ld;
    const int lane = threadIdx.x & (SPMV_TPR - 1), grp = threadIdx.x / SPMV_TPR;
    double sr = 0.0, sm = 0.0;
    for (long long it = blockIdx.x; it * SPMV_RPB < N; it += gridDim.x) {
        const long long row = it * SPMV_RPB + grp;
        double s = 0.0, m = 0.0;
        if (row < N) {
            if (res) {
                for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) {
                    const double x = u[col[e]];
                    s += Kv[e] * x;
                    m += Mv[e] * x;
                }
            } else {
                for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) m += Mv[e] * u[col[e]];
            }
        }
        s = group_sum(s);
        m = group_sum(m);
        if (lane == 0 && row < N) {
            mu[row] = m;
            const double r = s - l * m;
            sr += r * r;
            sm += m * m;
        }
    }
    if (!res) return;
    sr = warp_sum_groups(sr);
    sm = warp_sum_groups(sm);
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = sr;
        sb[threadIdx.x >> 5] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < 8; ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        partial[((long long)q * gridDim.x + blockIdx.x) * 2] = ta;
        partial[((long long)q * gridDim.x + blockIdx.x) * 2 + 1] = tb;
    }
}

// sign convention: largest |u| positive, lowest index on ties (global numbering)
__global__ void sign_fix_kernel(long long N, double* __restrict__ U, long long ldu) {
    __shared__ double bv[256];
    __shared__ long long bi[256];
    double* u = U + (long long)blockIdx.x * ldu;
    double best = -1.0;
    long long idx = 0;
    for (long long i = threadIdx.x; i < N; i += blockDim.x) {
        double a = fabs(u[i]);
        if (a > best) {
            best = a;
            idx = i;
        }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = idx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            double a = bv[threadIdx.x + o];
            long long ia = bi[threadIdx.x + o];
            if (a > bv[threadIdx.x] || (a == bv[threadIdx.x] && ia < bi[threadIdx.x])) {
                bv[threadIdx.x] = a;
                bi[threadIdx.x] = ia;
            }
        }
        __syncthreads();
    }
    const bool flip = u[bi[0]] < 0.0;
    __syncthreads();
    if (flip)
        for (long long i = threadIdx.x; i < N; i += blockDim.x) u[i] = -u[i];
}

__global__ void copy_cols_kernel(long long N, int ncols, const double* __restrict__ src, long long lds,
                                 double* __restrict__ dst, long long ldd) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * ncols) return;
    long long cidx = t / N, r = t % N;
    dst[cidx * ldd + r] = src[cidx * lds + r];
}

// --------------------------------------------------------------- host side
void enqueue_reduce_cols(riga_ctx* c, const double* partial, int nch, int J, int pstride, double* out) {
    count_launch(c);
    reduce_cols_kernel<<<(J + 31) / 32, 256, 0, c->stream>>>(partial, nch, J, pstride, out);
}

uint64_t splitmix(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// w[i] = u(splitmix draw i + 1 after seed0) - 1/2 with u in (0, 1): SplitMix64
// is a counter-based generator (draw i mixes seed0 + (i + 1) * gamma), so the
// device produces the host sequence of splitmix() exactly
__global__ void start_vector_kernel(long long n, unsigned long long seed0, double* __restrict__ w) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed0 + (unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    w[i] = ((double)(z >> 11) + 0.5) / 9007199254740992.0 - 0.5;
}

// n pseudo-random start-vector entries on the device (the values n host
// splitmix() draws would give), the seed advanced past them
void enqueue_start_vector(riga_ctx* c, long long n, uint64_t& seed, double* w) {
    count_launch(c);
    start_vector_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, seed, w);
    seed += (uint64_t)n * 0x9E3779B97F4A7C15ULL;
}

// Two full Gram-Schmidt passes (CGS2) of w against columns col0..col0+J
int ortho_pass(Run& R, int col0, int J, double* w) {
    riga_ctx* c = R.c;
    cudaStream_t st = c->stream;
    if (J <= 0) return RIGA_OK;
    // two Gram-Schmidt passes read MV twice and V twice
    PhaseScope scope(c, PH_REORTH, 4.0 * (double)R.N * J * sizeof(double), 8.0 * (double)R.N * J);
    const size_t sm_dots = (size_t)(CH + 8 * TJ + TJ * (HR + 1)) * sizeof(double);
    { count_launch(c); gemvT_partial_kernel<<<R.nch, 256, sm_dots, st>>>(c->MV.ptr + col0 * R.ld, R.ld, J, w, R.N, c->partial.ptr, R.cap); }
    { count_launch(c); reduce_cols_kernel<<<(J + 31) / 32, 256, 0, st>>>(c->partial.ptr, R.nch, J, R.cap, R.c1); }
    size_t sm = sm_dots + (size_t)J * sizeof(double);
    { count_launch(c); update_gemvT_kernel<<<R.nch, 256, sm, st>>>(c->V.ptr + col0 * R.ld, J, R.c1, c->MV.ptr + col0 * R.ld, J,
                                                                  R.ld, w, R.N, c->partial.ptr, R.cap); }
    { count_launch(c); reduce_cols_kernel<<<(J + 31) / 32, 256, 0, st>>>(c->partial.ptr, R.nch, J, R.cap, R.c2); }
    { count_launch(c); gemv_update_kernel<<<(unsigned)((R.N + 255) / 256), 256, (size_t)J * sizeof(double), st>>>(
        c->V.ptr + col0 * R.ld, R.ld, J, R.c2, w, R.N); }
    return RIGA_OK;
}

// The three-term recurrence against columns u0..u0+Ju (alpha_j and beta_j
// computed as (M v)^T w; coefficients into c1 at their column positions),
// then one full Gram-Schmidt pass against columns 0..J (into c2)
int recur_pass(Run& R, int J, int u0, int Ju, double* w) {
    riga_ctx* c = R.c;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_REORTH, (2.0 * J + 2.0 * Ju + 1.0) * (double)R.N * sizeof(double), 4.0 * (double)R.N * (J + Ju));
    const size_t sm_dots = (size_t)(CH + 8 * TJ + TJ * (HR + 1)) * sizeof(double);
    count_launch(c);
    if (Ju == 2) local_dots_kernel<2><<<R.nch, 64, 0, st>>>(c->MV.ptr + (long long)u0 * R.ld, R.ld, w, R.N, c->partial.ptr, R.cap);
    else local_dots_kernel<1><<<R.nch, 64, 0, st>>>(c->MV.ptr + (long long)u0 * R.ld, R.ld, w, R.N, c->partial.ptr, R.cap);
    { count_launch(c); reduce_cols_kernel<<<1, 256, 0, st>>>(c->partial.ptr, R.nch, Ju, R.cap, R.c1 + u0); }
    size_t sm = sm_dots + (size_t)Ju * sizeof(double);
    { count_launch(c); update_gemvT_kernel<<<R.nch, 256, sm, st>>>(c->V.ptr + (long long)u0 * R.ld, Ju, R.c1 + u0, c->MV.ptr, J,
                                                                  R.ld, w, R.N, c->partial.ptr, R.cap); }
    { count_launch(c); reduce_cols_kernel<<<(J + 31) / 32, 256, 0, st>>>(c->partial.ptr, R.nch, J, R.cap, R.c2); }
    { count_launch(c); gemv_update_kernel<<<(unsigned)((R.N + 255) / 256), 256, (size_t)J * sizeof(double), st>>>(
        c->V.ptr, R.ld, J, R.c2, w, R.N); }
    return RIGA_OK;
}

// w -> M-normalised into column `col` of V / MV; beta slot receives the norm.
// Jc > 0: w came from recur_pass against Jc columns (the one-pass test is
// evaluated, bit 2 of c->bflag[0]).
void normalize_into(Run& R, double* w, int col, int jslot, int Jc) {
    riga_ctx* c = R.c;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_SPMV, (double)c->S.nnz * 12.0 + (double)R.N * 8.0 * 6.0);
    const unsigned nbs = (unsigned)((R.N + SPMV_RPB - 1) / SPMV_RPB);
    { count_launch(c); spmv_dot_kernel<<<nbs, 256, 0, st>>>(R.N, c->rowptr.ptr, c->col.ptr, c->Mval.ptr, w, R.Mw, c->red.ptr); }
    c->stats.n_matvec++;
    { count_launch(c); finalize_kernel<<<1, 256, 0, st>>>(c->red.ptr, (int)nbs, R.c1, col - 1, R.c2, col - 1, jslot, R.alpha,
                                                         R.beta, Jc, c->bflag.ptr); }
    { count_launch(c); normalize_kernel<<<(unsigned)((R.N + 255) / 256), 256, 0, st>>>(R.N, w, R.Mw, R.beta + jslot + 1,
                                                                     c->V.ptr + col * R.ld, c->MV.ptr + col * R.ld); }
}

// Numeric factorization at sigma.  An inertia-only factorization leaves the
// packed solve operators (Q pool) untouched, so the solve state of the
// previous factorization (shift, precision) is restored afterwards.
int factor_at(riga_ctx* c, double sigma, int precision, long long* nu, bool inertia_only) {
    const double keep_sigma = c->sigma;
    const int keep_prec = c->precision;
    const bool keep_factored = c->factored;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    c->sigma = sigma;
    c->precision = precision;
    c->inertia_only = inertia_only;
    cudaEventRecord(e0, c->stream);
    int rc = enqueue_factor(c);
    if (rc == RIGA_OK) {
        cudaEventRecord(e1, c->stream);
        rc = finish_factor(c);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        c->stats.t_fact_ms += ms;
        c->stats.n_fact++;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (nu) *nu = c->inertia;
    if (inertia_only) {
        c->sigma = keep_sigma;
        c->precision = keep_prec;
        c->factored = keep_factored;
    }
    c->inertia_only = false;
    return rc;
}

// FP32 fronts: measure how many refinement sweeps one solve needs to reach a
// relative residual of 1e-13 (a seeded random right-hand side, residuals read
// back after every sweep); Lanczos then runs that many (at least two) without host
// checks.  If refinement stalls, the shift is refactored with FP64 fronts.
int calibrate_refinement(riga_ctx* c, uint64_t seed) {
    const long long N = c->S.N;
    for (int i = 2; i < 6; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    std::vector<double> hb(N);
    uint64_t st = seed ^ 0x5DEECE66DULL;
    for (long long i = 0; i < N; ++i) hb[i] = ((double)(splitmix(st) >> 11) + 0.5) / 9007199254740992.0 - 0.5;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->vwork[4].ptr, hb.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    int sweeps = 0;
    int rc = solve_refined(c, c->vwork[4].ptr, c->vwork[2].ptr, c->vwork[3].ptr, 1e-13, 20, 1, &sweeps);
    if (rc == RIGA_OK) {
        c->ir_sweeps = std::min(std::max(sweeps, 2), 20);
        c->stats.ir_sweeps = c->ir_sweeps;
        return RIGA_OK;
    }
    if (rc != RIGA_EREFINE) return rc;
    c->last_error.clear();
    c->stats.n_fallback++;
    return factor_at(c, c->sigma, RIGA_FP64, nullptr);
}

// FP64 fronts: one seeded solve's relative residual; at most 1e-13 -> plain
// solves (fp64_sweeps = 1), else the sweeps refinement needs to reach it (FP64
// residuals, FP64 corrections), used by every solve until the next factorization
int calibrate_fp64_solve(riga_ctx* c, uint64_t seed) {
    const long long N = c->S.N;
    for (int i = 2; i < 6; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    std::vector<double> hb(N);
    uint64_t st = seed ^ 0x2545F4914F6CDD1DULL;
    for (long long i = 0; i < N; ++i) hb[i] = ((double)(splitmix(st) >> 11) + 0.5) / 9007199254740992.0 - 0.5;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->vwork[4].ptr, hb.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    int sweeps = 0;
    int rc = solve_refined(c, c->vwork[4].ptr, c->vwork[2].ptr, c->vwork[3].ptr, 1e-13, 10, 1, &sweeps);
    if (rc == RIGA_EREFINE) {
        c->last_error.clear();
        sweeps = 10;
    } else if (rc) {
        return rc;
    }
    c->fp64_sweeps = std::max(1, std::min(sweeps, 10));
    return RIGA_OK;
}

// A run that locked nothing with FP64 fronts: its converged candidates (if
// any) missed the true-residual bar, which the accuracy of the plain solves
// limits (the Ritz residual cannot fall much below the solve's backward
// error times ||K|| / lambda).  Later runs on this factorization refine each
// solve once in FP64 (residual b - (K - sigma M) x and a correction solve),
// which takes the solve error to the FP64 residual's rounding level.  A new
// factorization starts again from plain solves.
static void refine_after_fruitless(riga_ctx* c, bool dbg) {
    if (c->precision != RIGA_FP64 || c->fp64_sweeps >= 2) return;
    c->fp64_sweeps = 2;
    if (dbg) std::fprintf(stderr, "[riga] fruitless run: FP64 solves refined once from now on\n");
}

int configure_reorth(riga_ctx* c, int cap) {
    const size_t sm_dots = (size_t)(CH + 8 * TJ + TJ * (HR + 1)) * sizeof(double);
    const size_t sm_upd = sm_dots + (size_t)cap * sizeof(double);
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(gemvT_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_dots));
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(update_gemvT_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_upd));
    return RIGA_OK;
}

// Ritz vectors U = V[:, col0 : col0+m] W (and M U from the stored M V) for the
// candidate pairs, their FP64 residuals ||K u - lam M u|| / (|lam| ||M u||),
// and locking of those at most lock_tol into columns nlock, nlock+1, ... of V
// and M V (eigenvalues appended to lam).
// host double-double addition (the same TwoSum as the device's dd_add)
static void host_dd_add(double& hi, double& lo, double bh, double bl) {
    const double s = hi + bh;
    const double bb = s - hi;
    double e = (hi - (s - bb)) + (bh - bb);
    e += lo + bl;
    hi = s + e;
    lo = e - (hi - s);
}

int ritz_lock(Run& R, int col0, int m, const std::vector<double>& Wsel, const std::vector<double>& lcand,
              int nlock, double lock_tol, std::vector<double>& lam, int* n_locked) {
    riga_ctx* c = R.c;
    cudaStream_t st = c->stream;
    const long long N = R.N;
    const int nsel = (int)lcand.size();
    *n_locked = 0;
    if (nsel == 0) return RIGA_OK;
    // W, then candidate eigenvalues, residual partial sums (304 blocks) and
    // Rayleigh-quotient partial sums (304 blocks)
    RIGA_CUDA_TRY(c, c->Wd.alloc((size_t)m * nsel + nsel + (size_t)6 * 304 * nsel));
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->Wd.ptr, Wsel.data(), (size_t)m * nsel * sizeof(double), cudaMemcpyHostToDevice, st));
    RIGA_CUDA_TRY(c, c->evec_perm.alloc((size_t)N * nsel * 2));
    double* U = c->evec_perm.ptr;
    double* MU = c->evec_perm.ptr + (size_t)N * nsel;
    // algorithmic bytes: V read, U written and read back, M U written, K
    // and M (values and columns) read once
    PhaseScope scope(c, PH_RITZ, (double)N * (m + 3 * nsel) * sizeof(double) + 20.0 * (double)c->S.nnz);
    dim3 g((unsigned)((N + 255) / 256), (unsigned)((nsel + 15) / 16));
    { count_launch(c); gemm_ritz_kernel<<<g, 256, 0, st>>>(c->V.ptr + (long long)col0 * R.ld, R.ld, m, c->Wd.ptr, m, nsel, U, N, N); }
    const int gx = 304;
    double* dlam = c->Wd.ptr + (size_t)m * nsel;
    double* dpart = dlam + nsel;
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(dlam, lcand.data(), nsel * sizeof(double), cudaMemcpyHostToDevice, st));
    double* dpart_rq = dpart + (size_t)2 * gx * nsel;
    // M U by the sparse product (not MV W, a dense product of m columns)
    { count_launch(c); resid_cols_kernel<<<dim3(gx, nsel), 256, 0, st>>>(N, c->rowptr.ptr, c->col.ptr, c->Kval.ptr, c->Mval.ptr, U, MU, N, dlam, nsel, dpart); }
    const bool rq = c->opt_rq != 0;
    if (rq) { count_launch(c); rq_cols_kernel<<<dim3(gx, nsel), 256, 0, st>>>(N, c->rowptr.ptr, c->col.ptr, c->Kval.ptr, U, MU, N, dpart_rq); }
    std::vector<double> part((size_t)(rq ? 6 : 2) * gx * nsel);
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(part.data(), dpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
    const double* prq = part.data() + (size_t)2 * gx * nsel;
    int acc_n = 0;
    for (int q = 0; q < nsel; ++q) {
        double ra = 0.0, rb = 0.0;
        for (int b = 0; b < gx; ++b) {
            ra += part[((size_t)q * gx + b) * 2];
            rb += part[((size_t)q * gx + b) * 2 + 1];
        }
        const double rho = std::sqrt(ra) / (std::fabs(lcand[q]) * std::sqrt(rb));
        if (!(rho <= lock_tol)) continue;
        // the locked eigenvalue: sigma + 1 / theta, which carries the
        // rounding of the Lanczos recurrence (about 1e-15 relative), or with
        // the Rayleigh-quotient option u^T K u / u^T M u of the Ritz vector
        // (its error quadratic in the residual; the double-double sums leave
        // it the rounding of the data alone)
        double lrq = lcand[q], mh = 1.0;
        if (rq) {
            double kh = 0.0, kl = 0.0, ml = 0.0;
            mh = 0.0;
            for (int b = 0; b < gx; ++b) {
                const double* pb = prq + ((size_t)q * gx + b) * 4;
                host_dd_add(kh, kl, pb[0], pb[1]);
                host_dd_add(mh, ml, pb[2], pb[3]);
            }
            lrq = (kh + kl) / (mh + ml);
        }
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->V.ptr + (long long)(nlock + acc_n) * R.ld, U + (long long)q * N,
                                         N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->MV.ptr + (long long)(nlock + acc_n) * R.ld, MU + (long long)q * N,
                                         N * sizeof(double), cudaMemcpyDeviceToDevice, st));
        lam.push_back(std::isfinite(lrq) && mh > 0.0 ? lrq : lcand[q]);
        ++acc_n;
    }
    *n_locked = acc_n;
    return RIGA_OK;
}

// Ritz vectors U = V[:, col0 : col0+J] W and their sparse products M U for
// the nsel columns of W (J x nsel, host, column-major) into U and MU (N x
// nsel, leading dimension N); the FP64 residuals
// ||K u - lam M u|| / (|lam| ||M u||) of the first nres of them into rho.
int ritz_vectors_resid(Run& R, int col0, int J, const std::vector<double>& W, int nsel, double* U, double* MU,
                       const std::vector<double>& lam, int nres, std::vector<double>& rho) {
    riga_ctx* c = R.c;
    cudaStream_t st = c->stream;
    const long long N = R.N;
    rho.assign(nres, 0.0);
    if (nsel <= 0) return RIGA_OK;
    const int gx = 304;
    RIGA_CUDA_TRY(c, c->Wd.alloc((size_t)J * nsel + nsel + (size_t)2 * gx * std::max(nres, 1)));
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->Wd.ptr, W.data(), (size_t)J * nsel * sizeof(double), cudaMemcpyHostToDevice, st));
    PhaseScope scope(c, PH_RITZ, (double)N * (J + 3 * nsel) * sizeof(double) + 20.0 * (double)c->S.nnz);
    dim3 g((unsigned)((N + 255) / 256), (unsigned)((nsel + 15) / 16));
    { count_launch(c); gemm_ritz_kernel<<<g, 256, 0, st>>>(c->V.ptr + (long long)col0 * R.ld, R.ld, J, c->Wd.ptr, J, nsel, U, N, N); }
    double* dlam = c->Wd.ptr + (size_t)J * nsel;
    double* dpart = dlam + nsel;
    if (nres > 0) RIGA_CUDA_TRY(c, cudaMemcpyAsync(dlam, lam.data(), nres * sizeof(double), cudaMemcpyHostToDevice, st));
    // M U by the sparse product, the residuals of the first nres columns
    { count_launch(c); resid_cols_kernel<<<dim3(gx, nsel), 256, 0, st>>>(N, c->rowptr.ptr, c->col.ptr, c->Kval.ptr, c->Mval.ptr, U, MU, N, dlam, nres, dpart); }
    if (nres > 0) {
        std::vector<double> part((size_t)2 * gx * nres);
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(part.data(), dpart, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
        for (int q = 0; q < nres; ++q) {
            double ra = 0.0, rb = 0.0;
            for (int b = 0; b < gx; ++b) {
                ra += part[((size_t)q * gx + b) * 2];
                rb += part[((size_t)q * gx + b) * 2 + 1];
            }
            rho[q] = std::sqrt(ra) / (std::fabs(lam[q]) * std::sqrt(rb));
        }
    }
    return RIGA_OK;
}

int run_eigs(riga_ctx* c, int k, double sigma0, double tol, int* nconv) {
    static const bool dbg = std::getenv("RIGA_DEBUG") != nullptr;
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    const long long N = S.N;
    if (k < 1 || k >= N) return set_error(c, RIGA_EINVAL, "k must be in 1..N-1");
    const int slice = (c->opt_slice > 0 && c->opt_slice < k) ? c->opt_slice : k;
    const int extra = c->opt_extra > 0 ? c->opt_extra : 2;
    const int prec = c->opt_precision;
    const double tol_est = 1e-2 * tol;
    const double lock_tol = 0.5 * tol;  // true-residual bar for locking
    const double gap_rel = 1e-6;
    int wmax = slice + extra;
    int m_cap = c->opt_max_steps > 0 ? c->opt_max_steps : std::max(4 * wmax, wmax + 60);
    m_cap = (int)std::min<long long>(m_cap, N - 1);
    const int lock_cap = k + extra + 64;
    // block size: 2 or 4 when the solve can carry that many right-hand sides
    int B = c->opt_block == 0 ? 4 : c->opt_block;
    if (B > 1) B = std::min(B, solve_max_rhs(c));
    if (B == 3) B = 2;
    if (B < 1 || (long long)(m_cap + 2 * B) >= N) B = 1;
    // block runs converge with the number of block steps: they get 16 more
    // blocks than the single-vector run length (they stop early once converged)
    const int m_extra = B > 1 ? 16 * B : 0;
    if (B > 1 && (long long)(m_cap + m_extra + 2 * B) >= N) B = 1;
    Run R;
    R.c = c;
    R.N = N;
    R.ld = N;
    R.cap = lock_cap + m_cap + (B > 1 ? 16 * B : 0) + 1 + 2 * B;
    R.nch = (int)((N + CH - 1) / CH);
    if (c->V.alloc((size_t)N * R.cap) != cudaSuccess || c->MV.alloc((size_t)N * R.cap) != cudaSuccess)
        return set_error(c, RIGA_ENOMEM, "Lanczos basis");
    RIGA_CUDA_TRY(c, c->partial.alloc((size_t)R.nch * R.cap));
    RIGA_CUDA_TRY(c, c->coef.alloc(2 * (size_t)R.cap));
    RIGA_CUDA_TRY(c, c->ab.alloc(2 * (size_t)m_cap + 4));
    RIGA_CUDA_TRY(c, c->red.alloc((size_t)((N * 16 + 255) / 256) + 1024));
    RIGA_CUDA_TRY(c, c->bflag.alloc(2));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(c->bflag.ptr, 0, 2 * sizeof(int), st));
    for (int i = 0; i < 4; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    R.w = c->vwork[0].ptr;
    R.Mw = c->vwork[1].ptr;
    R.xw = c->vwork[2].ptr;
    R.rw = c->vwork[3].ptr;
    R.c1 = c->coef.ptr;
    R.c2 = c->coef.ptr + R.cap;
    {
        int rc0 = configure_reorth(c, R.cap);
        if (rc0) return rc0;
    }
    R.alpha = c->ab.ptr;
    R.beta = c->ab.ptr + m_cap + 2;
    R.cgs2 = c->opt_reorth == 2;
    c->stats = Stats();

    std::vector<double> lam;      // locked eigenvalues, in column order of V
    int nlock = 0;
    long long nu0 = 0, nu_chk = 0;
    std::map<double, long long> inertia_cache;
    // nu(K - sigma0 M): with homogeneous Dirichlet conditions K and M are
    // symmetric positive definite, every eigenvalue is positive and the
    // inertia at sigma0 <= 0 is 0 without a factorization; otherwise FP64
    // fronts give it (an inertia-only factorization when the run's fronts
    // are of lower precision)
    int rc = RIGA_OK;
    if (prec == RIGA_FP64 || sigma0 > 0.0) {
        rc = factor_at(c, sigma0, RIGA_FP64, &nu0, prec != RIGA_FP64);
        if (rc) return rc;
    }
    inertia_cache[sigma0] = nu0;
    double cur_sigma = sigma0;
    double factored_sigma = (prec == RIGA_FP64) ? sigma0 : std::nan("");
    double calibrated_sigma = std::nan("");
    int confirmed = 0;
    int target = std::min(k, slice);
    int need = target + extra;  // locked pairs above sigma0 wanted before the next check
    uint64_t seed = c->opt_seed ? c->opt_seed : 1;
    int runs = 0, fruitless = 0;
    double missing_shift = std::nan("");  // check shift below which eigenvalues are missing
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    std::vector<double> h_ab, theta, zl, Zf, Wsel;
    int status = RIGA_OK;

    while (true) {
        if (nlock >= need) {
            // completeness check by inertia at a gap after the target count
            std::vector<double> sl(lam);
            std::sort(sl.begin(), sl.end());
            int gi = -1;
            for (int i = std::max(target, 1); i < (int)sl.size(); ++i)
                if (sl[i] - sl[i - 1] > gap_rel * std::fabs(sl[i])) { gi = i; break; }
            if (gi < 0) {
                need = nlock + extra;
                continue;
            }
            const double sp = 0.5 * (sl[gi - 1] + sl[gi]);
            // the inertia that certifies completeness always comes from FP64
            // fronts; it is cached per shift.  The solve operators are only
            // built when this shift may carry the next slice's Lanczos run.
            auto hit = inertia_cache.end();
            for (auto it2 = inertia_cache.begin(); it2 != inertia_cache.end(); ++it2)
                if (std::fabs(it2->first - sp) <= 1e-10 * std::fabs(sp)) hit = it2;
            if (hit != inertia_cache.end()) {
                nu_chk = hit->second;
                rc = RIGA_OK;
            } else {
                const bool reuse = (prec == RIGA_FP64) && (target < k);
                rc = factor_at(c, sp, RIGA_FP64, &nu_chk, !reuse);
                if (rc == RIGA_OK) {
                    inertia_cache[sp] = nu_chk;
                    if (reuse) factored_sigma = sp;
                }
            }
            if (dbg)
                std::fprintf(stderr, "[riga] check: nlock=%d target=%d gap_index=%d shift=%.12g inertia=%lld-%lld found=%d rc=%d cached=%d\n",
                             nlock, target, gi, sp, nu_chk, nu0, gi, rc, (int)(hit != inertia_cache.end()));
            if (rc) { status = rc; break; }
            const long long found = gi;  // locked eigenvalues below sp (all are > sigma0)
            if (nu_chk - nu0 == found) {
                missing_shift = std::nan("");
                confirmed = gi;
                if (confirmed >= k) break;
                target = std::min(k, confirmed + slice);
                need = std::max(need, target + extra);
                cur_sigma = sp;  // next slice starts at the check shift (already factored)
            } else if (nu_chk - nu0 > found) {
                // eigenvalues missing below sp: the next run starts at the
                // current shift; if it locks nothing and the locked values
                // just below sp form a (nearly) degenerate cluster, the runs
                // move to sp, where that cluster's missing copies are the
                // nearest unlocked eigenvalues and their relative separation
                // in theta, |lambda_a - lambda_b| / |lambda - sigma|, is largest
                need = nlock + (int)(nu_chk - nu0 - found);
                // a (nearly) degenerate cluster just below the gap: missing
                // copies are likely its members, next to sp
                if (gi >= 2 && sl[gi - 1] - sl[gi - 2] <= 1e-6 * std::fabs(sl[gi - 1])) missing_shift = sp;
            } else {
                status = set_error(c, RIGA_ENOCONV, "more locked pairs than the inertia allows");
                break;
            }
            continue;
        }
        if (++runs > 60 || fruitless > 4) {
            status = RIGA_ENOCONV;
            break;
        }
        if (fruitless > 0 && !std::isnan(missing_shift) && missing_shift != cur_sigma) cur_sigma = missing_shift;
        if (!(factored_sigma == cur_sigma)) {
            rc = factor_at(c, cur_sigma, prec, nullptr);
            if (rc) { status = rc; break; }
            factored_sigma = cur_sigma;
        }
        if (c->precision != RIGA_FP64 && calibrated_sigma != cur_sigma) {
            rc = calibrate_refinement(c, seed + (uint64_t)runs);
            if (rc) { status = rc; break; }
            calibrated_sigma = cur_sigma;
            if (dbg) std::fprintf(stderr, "[riga] refinement sweeps per solve: %d (precision now %d)\n", c->ir_sweeps, c->precision);
        }
        const int want_run = std::max(need - nlock, 1);
        int m_max = c->opt_max_steps > 0 ? c->opt_max_steps : std::max(4 * want_run, want_run + 60);
        m_max = std::min(m_max, m_cap);
        m_max = (int)std::min<long long>(m_max, N - nlock - 1);
        if (m_max < 1) { status = RIGA_ENOCONV; break; }
        if (nlock + m_max + 1 > R.cap) { status = set_error(c, RIGA_ENOMEM, "Lanczos basis capacity"); break; }
        const int col0 = nlock;
        cudaEventRecord(ev0, st);
        // block runs that stop making progress (a cluster larger than the
        // block, met again and again) hand over to single-vector runs
        if (B > 1 && fruitless < 2) {
            int mb = 0, acc_n = 0;
            const int m_blk = (int)std::min<long long>(m_max + 16 * B, N - nlock - 2 * B);
            rc = block_run(R, B, nlock, want_run, m_blk, cur_sigma, sigma0, tol_est, lock_tol, lock_cap, seed, lam, &mb,
                           &acc_n);
            if (rc) { status = rc; break; }
            nlock += acc_n;
            if (acc_n > 0) fruitless = 0;
            else ++fruitless;
            if (acc_n == 0) refine_after_fruitless(c, dbg);
            if (dbg)
                std::fprintf(stderr, "[riga] run %d: shift=%.12g want=%d block=%d steps=%d/%d locked=%d total=%d\n", runs,
                             cur_sigma, want_run, B, mb, m_max, acc_n, nlock);
            cudaEventRecord(ev1, st);
            RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev0, ev1);
            c->stats.t_lanczos_ms += ms;
            continue;
        }
        // random start vector, M-orthogonal to the locked ones
        enqueue_start_vector(c, N, seed, R.w);
        if (nlock > 0) ortho_pass(R, 0, nlock, R.w);
        normalize_into(R, R.w, col0, -1, 0);
        int m = 0;
        bool converged = false;
        for (int j = 0; j < m_max; ++j) {
            const int col = col0 + j;
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(R.w, c->MV.ptr + (long long)col * R.ld, N * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
            rc = solve_refined(c, R.w, R.xw, R.rw, 0.0, c->ir_sweeps, 0, nullptr);
            if (rc) { status = rc; break; }
            if (R.cgs2) {
                ortho_pass(R, 0, col + 1, R.w);
                normalize_into(R, R.w, col + 1, j, 0);
            } else {
                recur_pass(R, col + 1, j == 0 ? col : col - 1, j == 0 ? 1 : 2, R.w);
                normalize_into(R, R.w, col + 1, j, col + 1);
            }
            c->stats.steps++;
            m = j + 1;
            if (m % 10 == 0 || m == m_max) {
                h_ab.resize(2 * (size_t)m_cap + 4);
                int dflag = 0, rflag = 0;
                RIGA_CUDA_TRY(c, cudaMemcpyAsync(h_ab.data(), c->ab.ptr, h_ab.size() * sizeof(double),
                                                 cudaMemcpyDeviceToHost, st));
                RIGA_CUDA_TRY(c, cudaMemcpyAsync(&dflag, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
                RIGA_CUDA_TRY(c, cudaMemcpyAsync(&rflag, c->bflag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
                RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
                if (dflag & 2) {
                    status = set_error(c, RIGA_ETIMEOUT, "a dependency wait of the tree solve gave up");
                    break;
                }
                if (rflag & 2) R.cgs2 = true;  // two full passes from now on
                const double* a = h_ab.data();
                const double* b = h_ab.data() + m_cap + 2;  // b[i] = beta_i (b[0] = start norm)
                theta.assign(m, 0.0);
                zl.assign(m, 0.0);
                tridiag_eig(m, a, b + 1, theta.data(), zl.data(), false);
                const double bm = b[m];
                // acceptable Ritz values: lambda above sigma0, by decreasing |theta|
                std::vector<int> ord;
                for (int i = 0; i < m; ++i)
                    if (theta[i] != 0.0 && cur_sigma + 1.0 / theta[i] > sigma0) ord.push_back(i);
                std::sort(ord.begin(), ord.end(), [&](int x, int y) { return std::fabs(theta[x]) > std::fabs(theta[y]); });
                int ok = 0;
                bool all = (int)ord.size() >= want_run;
                for (int q = 0; q < (int)ord.size() && q < want_run; ++q) {
                    int i = ord[q];
                    if (std::fabs(bm * zl[i]) <= tol_est * std::fabs(theta[i])) ++ok;
                    else all = false;
                }
                if ((all && ok >= want_run) || bm <= 1e-300) {
                    converged = true;
                    break;
                }
            }
        }
        if (status) break;
        // Rayleigh-Ritz with vectors, select converged acceptable pairs
        h_ab.resize(2 * (size_t)m_cap + 4);
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(h_ab.data(), c->ab.ptr, h_ab.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
        const double* a = h_ab.data();
        const double* b = h_ab.data() + m_cap + 2;
        theta.assign(m, 0.0);
        Zf.assign((size_t)m * m, 0.0);
        tridiag_eig(m, a, b + 1, theta.data(), Zf.data(), true);
        const double bm = b[m];
        std::vector<int> sel;
        for (int i = 0; i < m; ++i) {
            if (theta[i] == 0.0) continue;
            double l = cur_sigma + 1.0 / theta[i];
            if (!(l > sigma0)) continue;
            double est = std::fabs(bm * Zf[(size_t)i * m + (m - 1)]);
            if (est <= tol_est * std::fabs(theta[i])) sel.push_back(i);
        }
        std::sort(sel.begin(), sel.end(), [&](int x, int y) { return std::fabs(theta[x]) > std::fabs(theta[y]); });
        int room = lock_cap - nlock;
        if ((int)sel.size() > room) sel.resize(room);
        const int nsel = (int)sel.size();
        if (nsel > 0) {
            Wsel.assign((size_t)m * nsel, 0.0);
            for (int q = 0; q < nsel; ++q)
                for (int r = 0; r < m; ++r) Wsel[(size_t)q * m + r] = Zf[(size_t)sel[q] * m + r];
            std::vector<double> lcand(nsel);
            for (int q = 0; q < nsel; ++q) lcand[q] = cur_sigma + 1.0 / theta[sel[q]];
            int acc_n = 0;
            rc = ritz_lock(R, col0, m, Wsel, lcand, nlock, lock_tol, lam, &acc_n);
            if (rc) { status = rc; break; }
            nlock += acc_n;
            if (acc_n > 0) fruitless = 0;
            else ++fruitless;
            if (acc_n == 0) refine_after_fruitless(c, dbg);
        } else {
            ++fruitless;
        }
        if (dbg)
            std::fprintf(stderr, "[riga] run %d: shift=%.12g want=%d steps=%d/%d converged=%d locked=%d total=%d\n", runs,
                         cur_sigma, want_run, m, m_max, (int)converged, nsel, nlock);
        cudaEventRecord(ev1, st);
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        c->stats.t_lanczos_ms += ms;
        (void)converged;
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);

    // output: the k smallest locked eigenvalues, ascending, vectors in permuted order
    std::vector<int> ord(nlock);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return lam[x] < lam[y]; });
    const int nout = std::min(k, nlock);
    const int limit = (status == RIGA_OK) ? nout : std::min(nout, confirmed);
    c->evals.assign(limit, 0.0);
    RIGA_CUDA_TRY(c, c->evec_perm.alloc((size_t)N * std::max(limit, 1)));
    for (int q = 0; q < limit; ++q) {
        c->evals[q] = lam[ord[q]];
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->evec_perm.ptr + (long long)q * N, c->V.ptr + (long long)ord[q] * R.ld,
                                         N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    }
    c->nev = limit;
    if (nconv) *nconv = limit;
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
    if (status) {
        if (status == RIGA_ENOCONV && c->last_error.empty()) set_error(c, status, "Lanczos did not converge");
        return status;
    }
    return RIGA_OK;
}

// exported helpers for api.cu
void sign_fix(riga_ctx* c, double* U, int ncols) {
    if (ncols > 0) { count_launch(c); sign_fix_kernel<<<ncols, 256, 0, c->stream>>>(c->S.N, U, c->S.N); }
}

}  // namespace riga
