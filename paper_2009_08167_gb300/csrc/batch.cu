// Batched shift-and-invert Lanczos over many independent eigenproblems
// (Sec. 4.2 applied to each problem of a batch at once).
//
// The problems are merged into one forest (symbolic.cpp merge_symbolic): one
// factorization launch per tree level and one persistent tree solve serve all
// of them, and the SpMV runs on the block-diagonal merged CSR.  Each problem
// keeps its own Lanczos recurrence: all reductions (Gram-Schmidt coefficients,
// M-norms, residuals) are segmented by problem over row chunks that never
// straddle two problems, and every problem has its own alpha, beta, Ritz
// values, locked vectors and completeness check.  Check shifts are per
// problem in one factorization of the forest (per-position shifts), and the
// Sylvester inertia is counted per problem.  FP64 fronts.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <numeric>

#include "ctx.h"

namespace riga {

constexpr int BCH = 256;  // rows per chunk
constexpr int BTJ = 32;   // basis columns per shared-memory tile
constexpr int BHR = 128;  // rows per shared-memory tile (a chunk is staged in BHR-row pieces)

struct Chunks {
    const long long* row0;
    const int* rows;
    const int* prob;
};

// partial dots over one chunk (same scheme as the single-problem kernels)
__device__ __forceinline__ void bchunk_dots(const double* __restrict__ B, long long ld, int J, long long r0, int rows,
                                            const double* __restrict__ ws, double* __restrict__ Vs,
                                            double* __restrict__ red, double* __restrict__ out) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (rows <= 0) {  // no rows (the same for the whole block): zero partials
        for (int j = tid; j < J; j += blockDim.x) out[j] = 0.0;
        return;
    }
    const int nh = (rows + BHR - 1) / BHR;           // row pieces per column tile
    const int nst = ((J + BTJ - 1) / BTJ) * nh;      // stages (column tile, row piece)
    double pre[BTJ / 8][BHR / 32];                   // the next stage, loaded while this one computes
    auto load = [&](int st) {
        const int j0 = (st / nh) * BTJ, h = (st % nh) * BHR;
        const int jn = min(BTJ, J - j0), hn = min(BHR, rows - h);
#pragma unroll
        for (int q = 0; q < BTJ / 8; ++q) {
            const int jl = warp + 8 * q;
            const double* col = B + (long long)(j0 + jl) * ld + r0 + h;
#pragma unroll
            for (int i = 0; i < BHR / 32; ++i) {
                const int r = lane + 32 * i;
                pre[q][i] = (jl < jn && r < hn) ? col[r] : 0.0;
            }
        }
    };
    if (nst > 0) load(0);
    double s = 0.0;
    for (int st = 0; st < nst; ++st) {
        const int j0 = (st / nh) * BTJ, h = (st % nh) * BHR;
        const int jn = min(BTJ, J - j0), hn = min(BHR, rows - h);
#pragma unroll
        for (int q = 0; q < BTJ / 8; ++q)
#pragma unroll
            for (int i = 0; i < BHR / 32; ++i) Vs[(warp + 8 * q) * (BHR + 1) + lane + 32 * i] = pre[q][i];
        __syncthreads();
        if (st + 1 < nst) load(st + 1);
        if (lane < jn) {
            const double* vc = Vs + lane * (BHR + 1);
            const double* wh = ws + h;
#pragma unroll 4
            for (int r = warp; r < hn; r += 8) s += vc[r] * wh[r];
        }
        __syncthreads();
        if (st % nh == nh - 1) {  // last piece of this column tile: sum the 8 row groups
            red[warp * BTJ + lane] = s;
            s = 0.0;
            __syncthreads();
            if (tid < jn) {
                double t = 0.0;
#pragma unroll
                for (int gg = 0; gg < 8; ++gg) t += red[gg * BTJ + tid];
                out[j0 + tid] = t;
            }
        }
    }
    __syncthreads();
}

// Partial dots of the recurrence: out[j] = sum over this chunk's rows of
// B_j[row] w[row] for the JU = 1 or 2 columns of the last two vectors; 64
// threads, four rows each, then the block's sum (every lane does useful
// multiply-adds, unlike the 32-column tiles of the full pass)
template <int JU>
__global__ void __launch_bounds__(64) blocal_dots_kernel(const double* __restrict__ B, long long ld,
                                                         const double* __restrict__ w, Chunks ch,
                                                         double* __restrict__ partial, int pstride) {
    __shared__ double red[2][JU];
    const long long r0 = ch.row0[blockIdx.x];
    const int rows = ch.rows[blockIdx.x];
    double acc[JU];
#pragma unroll
    for (int j = 0; j < JU; ++j) acc[j] = 0.0;
#pragma unroll
    for (int i = 0; i < BCH / 64; ++i) {
        const int rl = (int)threadIdx.x + 64 * i;
        if (rl < rows) {
            const double x = w[r0 + rl];
#pragma unroll
            for (int j = 0; j < JU; ++j) acc[j] += B[(long long)j * ld + r0 + rl] * x;
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

__global__ void __launch_bounds__(256) bgemvT_kernel(const double* __restrict__ B, long long ld, int J,
                                                     const double* __restrict__ w, Chunks ch,
                                                     double* __restrict__ partial, int pstride) {
    extern __shared__ double sh[];
    double* ws = sh;
    double* red = ws + BCH;
    double* Vs = red + 8 * BTJ;
    const long long r0 = ch.row0[blockIdx.x];
    const int rows = ch.rows[blockIdx.x];
    ws[threadIdx.x] = (threadIdx.x < rows) ? w[r0 + threadIdx.x] : 0.0;
    __syncthreads();
    bchunk_dots(B, ld, J, r0, rows, ws, Vs, red, partial + (long long)blockIdx.x * pstride);
}

__device__ __forceinline__ double brow_update(const double* __restrict__ V, long long ld, int J, long long r,
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

// w -= V[:, 0..Ju) c(problem) on this chunk (coefficients at coef + problem *
// cstride), then partial dots MV[:, 0..Jd)^T w
__global__ void __launch_bounds__(256) bupdate_gemvT_kernel(const double* __restrict__ V, int Ju,
                                                            const double* __restrict__ coef, int cstride,
                                                            const double* __restrict__ MV, int Jd, long long ld,
                                                            double* __restrict__ w, Chunks ch,
                                                            double* __restrict__ partial, int pstride) {
    extern __shared__ double sh[];
    double* ws = sh;
    double* red = ws + BCH;
    double* Vs = red + 8 * BTJ;
    double* cs = Vs + BTJ * (BHR + 1);
    const long long r0 = ch.row0[blockIdx.x];
    const int rows = ch.rows[blockIdx.x];
    const double* c = coef + (long long)ch.prob[blockIdx.x] * cstride;
    for (int j = threadIdx.x; j < Ju; j += blockDim.x) cs[j] = c[j];
    __syncthreads();
    double v = 0.0;
    if ((int)threadIdx.x < rows) {
        const long long r = r0 + threadIdx.x;
        v = brow_update(V, ld, Ju, r, cs, w[r]);
        w[r] = v;
    }
    ws[threadIdx.x] = v;
    __syncthreads();
    bchunk_dots(MV, ld, Jd, r0, rows, ws, Vs, red, partial + (long long)blockIdx.x * pstride);
}

__global__ void __launch_bounds__(256) bgemv_update_kernel(const double* __restrict__ V, long long ld, int J,
                                                           const double* __restrict__ coef, double* __restrict__ w,
                                                           Chunks ch) {
    extern __shared__ double cs[];
    const double* c = coef + (long long)ch.prob[blockIdx.x] * J;
    for (int j = threadIdx.x; j < J; j += blockDim.x) cs[j] = c[j];
    __syncthreads();
    if ((int)threadIdx.x < ch.rows[blockIdx.x]) {
        const long long r = ch.row0[blockIdx.x] + threadIdx.x;
        w[r] = brow_update(V, ld, J, r, cs, w[r]);
    }
}

// out[b][j] = sum over problem b's chunks of partial[c][j]
__global__ void __launch_bounds__(256) bseg_reduce_kernel(const double* __restrict__ partial, const int* __restrict__ cbeg,
                                                          const int* __restrict__ cend, int J, int pstride,
                                                          double* __restrict__ out) {
    __shared__ double red[8][33];
    const int b = blockIdx.y;
    const int jl = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int j = blockIdx.x * 32 + jl;
    double s = 0.0;
    if (j < J)
        for (int c = cbeg[b] + g; c < cend[b]; c += 8) s += partial[(long long)c * pstride + j];
    red[g][jl] = s;
    __syncthreads();
    if (g == 0 && j < J) {
        double t = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) t += red[q][jl];
        out[(long long)b * J + j] = t;
    }
}

// y = M x over a chunk (SPMV_TPR lanes per row) and the chunk's partial x.y
__global__ void __launch_bounds__(256) bspmv_dot_kernel(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                                        const double* __restrict__ Mv, const double* __restrict__ x,
                                                        double* __restrict__ y, Chunks ch,
                                                        double* __restrict__ partial) {
    __shared__ double red[8];
    const long long r0 = ch.row0[blockIdx.x];
    const int rows = ch.rows[blockIdx.x];
    const int lane = threadIdx.x & (SPMV_TPR - 1), grp = threadIdx.x / SPMV_TPR;
    double d = 0.0;
    for (int base = 0; base < BCH; base += SPMV_RPB) {
        const int rl = base + grp;
        double s = 0.0;
        if (rl < rows) {
            const long long row = r0 + rl;
            for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) s += Mv[e] * x[col[e]];
        }
        s = group_sum(s);
        if (lane == 0 && rl < rows) {
            const long long row = r0 + rl;
            y[row] = s;
            d += s * x[row];
        }
    }
    d = warp_sum_groups(d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += red[i];
        partial[blockIdx.x] = t;
    }
}

// per problem: alpha[b][j] = c1[b s1 + col1] + c2[b J + col], beta[b][j+1] =
// sqrt(sum of its chunk partials); with one full Gram-Schmidt pass (check),
// bit 2 of *flag when that pass removed more than 100 x the norm left
__global__ void bfinalize_kernel(int P, const double* __restrict__ partial, const int* __restrict__ cbeg,
                                 const int* __restrict__ cend, const double* __restrict__ c1, int s1, int col1,
                                 const double* __restrict__ c2, int J, int col, int j, double* __restrict__ alpha,
                                 double* __restrict__ beta, double* __restrict__ inv, int mstride, bool check,
                                 int* __restrict__ flag) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= P) return;
    double s = 0.0;
    for (int c = cbeg[b]; c < cend[b]; ++c) s += partial[c];
    const double b2 = fmax(s, 0.0), bt = sqrt(b2);
    if (j >= 0) alpha[(long long)b * mstride + j] = c1[(long long)b * s1 + col1] + c2[(long long)b * J + col];
    beta[(long long)b * (mstride + 1) + j + 1] = bt;
    inv[b] = bt > 0.0 ? 1.0 / bt : 0.0;
    if (check) {
        double q = 0.0;
        for (int i = 0; i < J; ++i) q += c2[(long long)b * J + i] * c2[(long long)b * J + i];
        if (!(q <= 1e4 * b2)) atomicOr(flag, 2);
    }
}

__global__ void bnormalize_kernel(long long N, const int* __restrict__ prob, const double* __restrict__ inv,
                                  const double* __restrict__ w, const double* __restrict__ Mw, double* __restrict__ v,
                                  double* __restrict__ mv) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const double s = inv[prob[r]];
    v[r] = w[r] * s;
    mv[r] = Mw[r] * s;
}

// U[r][q] = sum_j V[r][j] W_b[j][q] over a chunk of problem b (W padded to qmax
// columns); QN outputs per thread and pass (qmax rounded up to a multiple of
// 8, at most 32), so that each V entry read serves every candidate
template <int QN>
__global__ void __launch_bounds__(256) bgemm_ritz_kernel(const double* __restrict__ V, long long ld, int J,
                                                         const double* __restrict__ W, int qmax, Chunks ch,
                                                         double* __restrict__ U, long long ldu) {
    __shared__ double Ws[128][QN];
    const int b = ch.prob[blockIdx.x];
    const long long r = ch.row0[blockIdx.x] + threadIdx.x;
    const bool ok = (int)threadIdx.x < ch.rows[blockIdx.x];
    const int i0 = blockIdx.y * QN;
    const double* Wb = W + (long long)b * J * qmax;  // column-major J x qmax per problem
    double acc[QN];
#pragma unroll
    for (int q = 0; q < QN; ++q) acc[q] = 0.0;
    for (int j0 = 0; j0 < J; j0 += 128) {
        const int jn = min(128, J - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < 128 * QN; t += blockDim.x) {
            const int jj = t / QN, q = t % QN;
            Ws[jj][q] = (jj < jn && i0 + q < qmax) ? Wb[(long long)(i0 + q) * J + j0 + jj] : 0.0;
        }
        __syncthreads();
        if (ok)
            for (int jj = 0; jj < jn; ++jj) {
                const double v = V[(long long)(j0 + jj) * ld + r];
#pragma unroll
                for (int q = 0; q < QN; ++q) acc[q] += v * Ws[jj][q];
            }
    }
    if (ok)
#pragma unroll
        for (int q = 0; q < QN; ++q)
            if (i0 + q < qmax) U[(long long)(i0 + q) * ldu + r] = acc[q];
}

// M u of candidate q into MU (the matrix and u read once for both products)
// and the residual partial sums per (chunk, candidate q): ||K u - lam M u||^2,
// ||M u||^2
__global__ void __launch_bounds__(256) bresid_kernel(const long long* __restrict__ rowptr, const int* __restrict__ col,
                                                     const double* __restrict__ Kv, const double* __restrict__ Mv,
                                                     const double* __restrict__ U, double* __restrict__ MU,
                                                     long long ld, const double* __restrict__ lam, int qmax,
                                                     Chunks ch, double* __restrict__ partial) {
    __shared__ double sa[8], sb[8];
    const int q = blockIdx.y;
    const int b = ch.prob[blockIdx.x];
    const double l = lam[(long long)b * qmax + q];
    const double* u = U + (long long)q * ld;
    double* mu = MU + (long long)q * ld;
    const long long r0 = ch.row0[blockIdx.x];
    const int rows = ch.rows[blockIdx.x];
    const int lane = threadIdx.x & (SPMV_TPR - 1), grp = threadIdx.x / SPMV_TPR;
    double sr = 0.0, sm = 0.0;
    for (int base = 0; base < BCH; base += SPMV_RPB) {
        const int rl = base + grp;
        double s = 0.0, m = 0.0;
        if (rl < rows) {
            const long long row = r0 + rl;
            for (long long e = rowptr[row] + lane; e < rowptr[row + 1]; e += SPMV_TPR) {
                const double x = u[col[e]];
                s += Kv[e] * x;
                m += Mv[e] * x;
            }
        }
        s = group_sum(s);
        m = group_sum(m);
        if (lane == 0 && rl < rows) {
            mu[r0 + rl] = m;
            const double rr = s - l * m;
            sr += rr * rr;
            sm += m * m;
        }
    }
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

// dst column dcol[b*qmax + q] (if >= 0) of V / MV receives candidate q of
// problem b, on that problem's rows only
__global__ void bscatter_cols_kernel(long long N, int qmax, const int* __restrict__ prob, const int* __restrict__ dcol,
                                     const double* __restrict__ U, const double* __restrict__ MU, long long ldu,
                                     double* __restrict__ V, double* __restrict__ MV, long long ld) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * qmax) return;
    const int q = (int)(t / N);
    const long long r = t % N;
    const int d = dcol[(long long)prob[r] * qmax + q];
    if (d < 0) return;
    V[(long long)d * ld + r] = U[(long long)q * ldu + r];
    MV[(long long)d * ld + r] = MU[(long long)q * ldu + r];
}

// columns [nlock(problem), L) of V / MV are zero on each problem's rows, so
// that a problem is orthogonalised only against its own locked vectors
__global__ void bzero_tail_kernel(long long N, int L, const int* __restrict__ prob, const int* __restrict__ nlock,
                                  double* __restrict__ V, double* __restrict__ MV, long long ld) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * L) return;
    const int j = (int)(t / N);
    const long long r = t % N;
    if (j < nlock[prob[r]]) return;
    V[(long long)j * ld + r] = 0.0;
    MV[(long long)j * ld + r] = 0.0;
}

// ------------------------------------------------------------------ host side
namespace {

// Start vectors on the device: row r of an active problem takes the
// SplitMix64 output for counter base + r (Steele, Lea and Flood, 2014),
// mapped to a uniform value in (-1/2, 1/2); rows of finished problems are 0.
__global__ void bstart_kernel(long long N, const int* __restrict__ prob, const int* __restrict__ active,
                              unsigned long long base, double* __restrict__ w) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    unsigned long long z = base + (unsigned long long)(r + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    w[r] = active[prob[r]] ? ((double)(z >> 11) + 0.5) / 9007199254740992.0 - 0.5 : 0.0;
}

uint64_t bsplitmix(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct BatchState {
    riga_ctx* c;
    int P;
    long long N, ld;
    int cap;
    int nch;
    Chunks ch;
    DevBuf<long long> ch_row0;
    DevBuf<int> ch_rows, ch_prob, cbeg, cend;
    std::vector<int> h_cbeg, h_cend;
    DevBuf<double> c1, c2, partial, ab_alpha, ab_beta, inv, W, lam, rpart;
    DevBuf<int> dcol, nlock, rflag, active;
    double* pin = nullptr;  // pinned host copies of alpha, beta and the flag (lagged checks)
    cudaEvent_t ev = nullptr;  // marks those copies
    ~BatchState() {
        if (pin) cudaFreeHost(pin);
        if (ev) cudaEventDestroy(ev);
    }
    int mcap;
    bool cgs2 = false;  // two full Gram-Schmidt passes per step (set once one pass was not enough)
};

void bortho(BatchState& B, int J, double* w) {
    riga_ctx* c = B.c;
    cudaStream_t st = c->stream;
    if (J <= 0) return;
    PhaseScope scope(c, PH_REORTH, 4.0 * (double)B.N * J * sizeof(double), 8.0 * (double)B.N * J);
    const size_t sm_dots = (size_t)(BCH + 8 * BTJ + BTJ * (BHR + 1)) * sizeof(double);
    dim3 rg((J + 31) / 32, B.P);
    { count_launch(c); bgemvT_kernel<<<B.nch, 256, sm_dots, st>>>(c->MV.ptr, B.ld, J, w, B.ch, B.partial.ptr, B.cap); }
    { count_launch(c); bseg_reduce_kernel<<<rg, 256, 0, st>>>(B.partial.ptr, B.cbeg.ptr, B.cend.ptr, J, B.cap, B.c1.ptr); }
    { count_launch(c); bupdate_gemvT_kernel<<<B.nch, 256, sm_dots + (size_t)J * sizeof(double), st>>>(
        c->V.ptr, J, B.c1.ptr, J, c->MV.ptr, J, B.ld, w, B.ch, B.partial.ptr, B.cap); }
    { count_launch(c); bseg_reduce_kernel<<<rg, 256, 0, st>>>(B.partial.ptr, B.cbeg.ptr, B.cend.ptr, J, B.cap, B.c2.ptr); }
    { count_launch(c); bgemv_update_kernel<<<B.nch, 256, (size_t)J * sizeof(double), st>>>(c->V.ptr, B.ld, J, B.c2.ptr, w, B.ch); }
}

// Per problem, the three-term recurrence against columns u0..u0+Ju (alpha_j
// and beta_j computed as (M v)^T w, into c1 with stride Ju), then one full
// Gram-Schmidt pass against columns 0..J (into c2)
void brecur(BatchState& B, int J, int u0, int Ju, double* w) {
    riga_ctx* c = B.c;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_REORTH, (2.0 * J + 2.0 * Ju + 1.0) * (double)B.N * sizeof(double), 4.0 * (double)B.N * (J + Ju));
    const size_t sm_dots = (size_t)(BCH + 8 * BTJ + BTJ * (BHR + 1)) * sizeof(double);
    count_launch(c);
    if (Ju == 2) blocal_dots_kernel<2><<<B.nch, 64, 0, st>>>(c->MV.ptr + (long long)u0 * B.ld, B.ld, w, B.ch, B.partial.ptr, B.cap);
    else blocal_dots_kernel<1><<<B.nch, 64, 0, st>>>(c->MV.ptr + (long long)u0 * B.ld, B.ld, w, B.ch, B.partial.ptr, B.cap);
    { count_launch(c); bseg_reduce_kernel<<<dim3(1, B.P), 256, 0, st>>>(B.partial.ptr, B.cbeg.ptr, B.cend.ptr, Ju, B.cap,
                                                                       B.c1.ptr); }
    { count_launch(c); bupdate_gemvT_kernel<<<B.nch, 256, sm_dots + (size_t)Ju * sizeof(double), st>>>(
        c->V.ptr + (long long)u0 * B.ld, Ju, B.c1.ptr, Ju, c->MV.ptr, J, B.ld, w, B.ch, B.partial.ptr, B.cap); }
    dim3 rg((J + 31) / 32, B.P);
    { count_launch(c); bseg_reduce_kernel<<<rg, 256, 0, st>>>(B.partial.ptr, B.cbeg.ptr, B.cend.ptr, J, B.cap, B.c2.ptr); }
    { count_launch(c); bgemv_update_kernel<<<B.nch, 256, (size_t)J * sizeof(double), st>>>(c->V.ptr, B.ld, J, B.c2.ptr, w, B.ch); }
}

// w -> M-normalised per problem into column col of V / MV; beta slot jslot+1.
// Ju > 0: w came from brecur with Ju recurrence columns (alpha from c1's last
// entry, the one-pass test evaluated)
void bnormalize(BatchState& B, double* w, double* Mw, int col, int jslot, int J, int Ju) {
    riga_ctx* c = B.c;
    cudaStream_t st = c->stream;
    PhaseScope scope(c, PH_SPMV, (double)c->S.nnz * 12.0 + (double)B.N * 8.0 * 6.0);
    { count_launch(c); bspmv_dot_kernel<<<B.nch, 256, 0, st>>>(c->rowptr.ptr, c->col.ptr, c->Mval.ptr, w, Mw, B.ch, B.partial.ptr); }
    c->stats.n_matvec++;
    const int s1 = Ju > 0 ? Ju : J, col1 = Ju > 0 ? Ju - 1 : col - 1;
    { count_launch(c); bfinalize_kernel<<<(B.P + 127) / 128, 128, 0, st>>>(
        B.P, B.partial.ptr, B.cbeg.ptr, B.cend.ptr, B.c1.ptr, s1, col1, B.c2.ptr, J, col - 1, jslot, B.ab_alpha.ptr,
        B.ab_beta.ptr, B.inv.ptr, B.mcap, Ju > 0, B.rflag.ptr); }
    { count_launch(c); bnormalize_kernel<<<(unsigned)((B.N + 255) / 256), 256, 0, st>>>(
        B.N, c->prob_of_pos.ptr, B.inv.ptr, w, Mw, c->V.ptr + (long long)col * B.ld, c->MV.ptr + (long long)col * B.ld); }
}

}  // namespace

// Factorization of the whole forest with one shift per problem.  An
// inertia-only factorization (FP64 fronts, no solve operators) leaves the
// solve state of the previous one (precision, per-problem shifts and their
// per-position copy) as it was.
int factor_batch(riga_ctx* c, const std::vector<double>& sig, bool inertia_only, int precision = RIGA_FP64) {
    const std::vector<double> keep_sig = c->sigma_prob;
    const int keep_prec = c->precision;
    const double keep_sigma = c->sigma;
    c->sigma_prob = sig;
    c->sigma = sig.empty() ? 0.0 : sig[0];
    c->precision = inertia_only ? RIGA_FP64 : precision;
    c->inertia_only = inertia_only;
    const bool keep = c->factored;
    int rc = enqueue_factor(c);
    if (rc == RIGA_OK) rc = finish_factor(c);
    if (inertia_only) {
        c->factored = keep;
        if (!keep_sig.empty()) {
            // the shifts of the factorization the solves use
            c->sigma_prob = keep_sig;
            c->precision = keep_prec;
            c->sigma = keep_sigma;
            std::vector<double> sp(c->S.N);
            for (size_t b = 0; b + 1 < c->S.prob_pos.size(); ++b)
                for (long long i = c->S.prob_pos[b]; i < c->S.prob_pos[b + 1]; ++i) sp[i] = c->sigma_prob[b];
            cudaError_t e = c->sig_pos.upload(sp, c->stream);
            if (e != cudaSuccess && rc == RIGA_OK) rc = set_error(c, RIGA_ECUDA, cudaGetErrorString(e));
        }
    }
    c->inertia_only = false;
    c->stats.n_fact++;
    return rc;
}

// Refinement sweeps of a low-precision batch factorization: the sweeps one
// seeded right-hand side over the whole forest needs to reach a relative
// residual of 1e-13 (at least 2); if refinement stalls, the forest is
// refactored with FP64 fronts at the same shifts.
int calibrate_refinement_batch(riga_ctx* c, uint64_t seed, const std::vector<double>& sig) {
    const long long N = c->S.N;
    for (int i = 2; i < 6; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    std::vector<double> hb(N);
    uint64_t st = seed ^ 0x5DEECE66DULL;
    for (long long i = 0; i < N; ++i) hb[i] = ((double)(bsplitmix(st) >> 11) + 0.5) / 9007199254740992.0 - 0.5;
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
    return factor_batch(c, sig, false, RIGA_FP64);
}

// The k smallest eigenvalues above sigma0 of every problem of the batch.
// Outputs in c->batch_evals / batch_resid / batch_nconv (problem-major).
int run_eigs_batch(riga_ctx* c, int k, double sigma0, double tol) {
    static const bool dbg = std::getenv("RIGA_DEBUG") != nullptr;
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t) { return std::chrono::duration<double, std::milli>(clk::now() - t).count(); };
    double t_checks = 0.0, t_rr = 0.0, t_start = 0.0, t_fact = 0.0;
    const clk::time_point t_all = clk::now();
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    const int P = (int)S.prob_pos.size() - 1;
    const long long N = S.N;
    const int extra = c->opt_extra > 0 ? c->opt_extra : 2;
    const int want = k + extra;
    long long minN = N;
    for (int b = 0; b < P; ++b) minN = std::min(minN, S.prob_pos[b + 1] - S.prob_pos[b]);
    if (k < 1 || want >= minN) return set_error(c, RIGA_EINVAL, "k too large for the smallest problem of the batch");
    const double tol_est = 1e-2 * tol, lock_tol = 0.5 * tol, gap_rel = 1e-6;
    int m_cap = c->opt_max_steps > 0 ? c->opt_max_steps : std::max(4 * want, want + 60);
    m_cap = (int)std::min<long long>(m_cap, minN - 1);
    const int lock_cap = want + 32;
    BatchState B;
    B.c = c;
    B.P = P;
    B.N = N;
    B.ld = N;
    B.cap = lock_cap + m_cap + 1;
    B.mcap = m_cap;
    B.cgs2 = c->opt_reorth == 2;
    // row chunks inside problems
    std::vector<long long> r0;
    std::vector<int> rw, pb;
    B.h_cbeg.assign(P, 0);
    B.h_cend.assign(P, 0);
    for (int b = 0; b < P; ++b) {
        B.h_cbeg[b] = (int)r0.size();
        for (long long r = S.prob_pos[b]; r < S.prob_pos[b + 1]; r += BCH) {
            r0.push_back(r);
            rw.push_back((int)std::min<long long>(BCH, S.prob_pos[b + 1] - r));
            pb.push_back(b);
        }
        B.h_cend[b] = (int)r0.size();
    }
    B.nch = (int)r0.size();
    RIGA_CUDA_TRY(c, B.ch_row0.upload(r0, st));
    RIGA_CUDA_TRY(c, B.ch_rows.upload(rw, st));
    RIGA_CUDA_TRY(c, B.ch_prob.upload(pb, st));
    RIGA_CUDA_TRY(c, B.cbeg.upload(B.h_cbeg, st));
    RIGA_CUDA_TRY(c, B.cend.upload(B.h_cend, st));
    B.ch = Chunks{B.ch_row0.ptr, B.ch_rows.ptr, B.ch_prob.ptr};
    if (c->V.alloc((size_t)N * B.cap) != cudaSuccess || c->MV.alloc((size_t)N * B.cap) != cudaSuccess)
        return set_error(c, RIGA_ENOMEM, "batched Lanczos basis");
    RIGA_CUDA_TRY(c, cudaMemsetAsync(c->V.ptr, 0, (size_t)N * B.cap * sizeof(double), st));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(c->MV.ptr, 0, (size_t)N * B.cap * sizeof(double), st));
    RIGA_CUDA_TRY(c, B.partial.alloc((size_t)B.nch * B.cap));
    RIGA_CUDA_TRY(c, B.c1.alloc((size_t)P * B.cap));
    RIGA_CUDA_TRY(c, B.c2.alloc((size_t)P * B.cap));
    RIGA_CUDA_TRY(c, B.ab_alpha.alloc((size_t)P * m_cap));
    RIGA_CUDA_TRY(c, B.ab_beta.alloc((size_t)P * (m_cap + 1)));
    RIGA_CUDA_TRY(c, B.inv.alloc(P));
    RIGA_CUDA_TRY(c, B.rflag.alloc(1));
    RIGA_CUDA_TRY(c, cudaMemsetAsync(B.rflag.ptr, 0, sizeof(int), c->stream));
    RIGA_CUDA_TRY(c, B.active.alloc(P));
    const size_t npin = (size_t)P * m_cap + (size_t)P * (m_cap + 1) + 1;
    RIGA_CUDA_TRY(c, cudaMallocHost(&B.pin, npin * sizeof(double)));
    RIGA_CUDA_TRY(c, cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming));
    cudaEvent_t ev = B.ev;
    RIGA_CUDA_TRY(c, B.dcol.alloc((size_t)P * want));
    for (int i = 0; i < 2; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
    const size_t sm_dots = (size_t)(BCH + 8 * BTJ + BTJ * (BHR + 1)) * sizeof(double);
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bgemvT_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_dots));
    RIGA_CUDA_TRY(c, cudaFuncSetAttribute(bupdate_gemvT_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(sm_dots + (size_t)B.cap * sizeof(double))));
    double* w = c->vwork[0].ptr;
    double* Mw = c->vwork[1].ptr;
    c->stats = Stats();

    // per-problem state
    std::vector<std::vector<double>> lam(P), res(P);
    std::vector<int> nlock(P, 0);
    std::vector<char> done(P, 0);
    std::vector<int> need(P, want);
    std::vector<double> sig0(P, sigma0);
    clk::time_point t0 = clk::now();
    // the run factorization: fronts in the chosen precision.  nu(K - sigma0 M)
    // per problem from FP64 fronts: the run factorization's own inertia on
    // the FP64 path; 0 without a factorization for sigma0 <= 0 (K and M
    // positive definite); an FP64 inertia-only factorization otherwise
    const int prec = c->opt_precision;
    std::vector<long long> nu0(P, 0);
    int rc = RIGA_OK;
    if (prec != RIGA_FP64 && sigma0 > 0.0) {
        rc = factor_batch(c, sig0, true);
        if (rc) return rc;
        nu0 = c->inertia_prob;
    }
    rc = factor_batch(c, sig0, false, prec);
    t_fact += ms_since(t0);
    if (rc) return rc;
    if (prec == RIGA_FP64) nu0 = c->inertia_prob;
    double* xw = nullptr;
    double* rwk = nullptr;
    if (prec != RIGA_FP64) {
        // refinement sweeps per solve for this factorization (a seeded
        // right-hand side over all problems to 1e-13); FP64 fronts if it stalls
        for (int i = 2; i < 4; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
        xw = c->vwork[2].ptr;
        rwk = c->vwork[3].ptr;
        rc = calibrate_refinement_batch(c, c->opt_seed ? c->opt_seed : 1, sig0);
        if (rc) return rc;
    }
    uint64_t seed = c->opt_seed ? c->opt_seed : 1;
    std::vector<double> h_alpha, h_beta;
    int status = RIGA_OK;
    // FP64 fronts: plain solves until a converged candidate misses the
    // true-residual bar (the plain solve's accuracy limits the Ritz
    // residual); from then on each solve is refined once in FP64
    bool refine64 = false;
    for (int run = 1; run <= 4; ++run) {
        int active = 0;
        for (int b = 0; b < P; ++b) active += !done[b];
        if (active == 0) break;
        int Lmax = 0;
        for (int b = 0; b < P; ++b) Lmax = std::max(Lmax, nlock[b]);
        int maxw = 1;
        for (int b = 0; b < P; ++b)
            if (!done[b]) maxw = std::max(maxw, need[b] - nlock[b]);
        int m_max = c->opt_max_steps > 0 ? c->opt_max_steps : std::max(4 * maxw, maxw + 60);
        m_max = std::min(m_max, m_cap);
        if (Lmax + m_max + 1 > B.cap) m_max = B.cap - Lmax - 1;
        if (m_max < 1) {
            status = RIGA_ENOCONV;
            break;
        }
        const int col0 = Lmax;
        if (Lmax > 0) {
            RIGA_CUDA_TRY(c, B.nlock.upload(nlock, st));
            { count_launch(c); bzero_tail_kernel<<<(unsigned)((N * Lmax + 255) / 256), 256, 0, st>>>(
                N, Lmax, c->prob_of_pos.ptr, B.nlock.ptr, c->V.ptr, c->MV.ptr, B.ld); }
        }
        // start vectors: random on active problems, zero on the others
        t0 = clk::now();
        {
            std::vector<int> act(P);
            for (int b = 0; b < P; ++b) act[b] = !done[b];
            RIGA_CUDA_TRY(c, B.active.upload(act, st));
            const unsigned long long base = bsplitmix(seed);
            count_launch(c);
            bstart_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, c->prob_of_pos.ptr, B.active.ptr, base, w);
        }
        if (Lmax > 0) bortho(B, Lmax, w);
        bnormalize(B, w, Mw, col0, -1, Lmax > 0 ? Lmax : 1, 0);
        t_start += ms_since(t0);
        int m = 0, pending = -1;
        for (int j = 0; j < m_max; ++j) {
            const int col = col0 + j;
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(w, c->MV.ptr + (long long)col * B.ld, N * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
            rc = (c->precision == RIGA_FP64 && !refine64) ? enqueue_solve(c, w)
                                                           : solve_refined(c, w, xw, rwk, 0.0, c->ir_sweeps, 0, nullptr);
            if (rc) {
                status = rc;
                break;
            }
            if (B.cgs2) {
                bortho(B, col + 1, w);
                bnormalize(B, w, Mw, col + 1, j, col + 1, 0);
            } else {
                const int Ju = j == 0 ? 1 : 2;
                brecur(B, col + 1, col + 1 - Ju, Ju, w);
                bnormalize(B, w, Mw, col + 1, j, col + 1, Ju);
            }
            c->stats.steps++;
            m = j + 1;
            // lagged checks: the copies of step `pending` are queued with an
            // event, the host evaluates them while the GPU runs on, and it
            // never runs more than two steps ahead of an unevaluated check
            if (pending >= 0 && (m - pending >= 2 || cudaEventQuery(ev) == cudaSuccess)) {
                cudaEventSynchronize(ev);
                const int mc = pending;
                pending = -1;
                const double* pa = B.pin;
                const double* pbeta = B.pin + (size_t)P * m_cap;
                if (reinterpret_cast<const int*>(B.pin + npin - 1)[0] & 2) B.cgs2 = true;  // two full passes from now on
                t0 = clk::now();
                // per problem: are its wanted Ritz values converged?
                std::vector<char> conv(P, 1);
                parallel_for(P, [&](int b) {
                    if (done[b]) return;
                    const double* a = pa + (size_t)b * m_cap;
                    const double* bt = pbeta + (size_t)b * (m_cap + 1);
                    std::vector<double> th(mc), zz(mc);
                    tridiag_eig(mc, a, bt + 1, th.data(), zz.data(), false);
                    const int wb = need[b] - nlock[b];
                    int ok = 0;
                    for (int i = mc - 1; i >= 0 && ok < wb; --i) {
                        if (!(th[i] > 0.0)) break;
                        if (std::fabs(bt[mc] * zz[i]) <= tol_est * th[i]) ++ok;
                        else break;
                    }
                    conv[b] = !(ok < wb && bt[mc] > 1e-300);
                });
                bool all = true;
                for (int b = 0; b < P; ++b) all = all && conv[b];
                t_checks += ms_since(t0);
                if (all) break;
            }
            if (pending < 0 && m % 10 == 0 && m < m_max) {
                RIGA_CUDA_TRY(c, cudaMemcpyAsync(B.pin, B.ab_alpha.ptr, (size_t)P * m_cap * sizeof(double),
                                                 cudaMemcpyDeviceToHost, st));
                RIGA_CUDA_TRY(c, cudaMemcpyAsync(B.pin + (size_t)P * m_cap, B.ab_beta.ptr,
                                                 (size_t)P * (m_cap + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
                RIGA_CUDA_TRY(c, cudaMemcpyAsync(B.pin + npin - 1, B.rflag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
                RIGA_CUDA_TRY(c, cudaEventRecord(ev, st));
                pending = m;
            }
        }
        if (pending >= 0) cudaEventSynchronize(ev);
        if (status) break;
        // Rayleigh-Ritz per problem, candidates = converged largest theta
        h_alpha.resize((size_t)P * m_cap);
        h_beta.resize((size_t)P * (m_cap + 1));
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(h_alpha.data(), B.ab_alpha.ptr, h_alpha.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(h_beta.data(), B.ab_beta.ptr, h_beta.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
        t0 = clk::now();
        const int qmax = want;
        std::vector<double> hW((size_t)P * m * qmax, 0.0), hl((size_t)P * qmax, 0.0);
        std::vector<int> nsel(P, 0);
        parallel_for(P, [&](int b) {
            if (done[b]) return;
            const double* a = h_alpha.data() + (size_t)b * m_cap;
            const double* bt = h_beta.data() + (size_t)b * (m_cap + 1);
            std::vector<double> th(m), Z((size_t)m * m);
            tridiag_eig(m, a, bt + 1, th.data(), Z.data(), true);
            const int room = std::min(qmax, lock_cap - nlock[b]);
            for (int i = m - 1; i >= 0 && nsel[b] < room; --i) {
                if (!(th[i] > 0.0)) break;
                if (std::fabs(bt[m] * Z[(size_t)i * m + m - 1]) > tol_est * th[i]) continue;
                const int q = nsel[b]++;
                for (int r = 0; r < m; ++r) hW[((size_t)b * qmax + q) * m + r] = Z[(size_t)i * m + r];
                hl[(size_t)b * qmax + q] = sigma0 + 1.0 / th[i];
            }
        });
        t_rr += ms_since(t0);
        RIGA_CUDA_TRY(c, B.W.upload(hW, st));
        RIGA_CUDA_TRY(c, B.lam.upload(hl, st));
        RIGA_CUDA_TRY(c, c->evec_perm.alloc((size_t)N * qmax * 2));
        double* U = c->evec_perm.ptr;
        double* MU = c->evec_perm.ptr + (size_t)N * qmax;
        {
            // algorithmic bytes: V read, U written and read back, M U
            // written, K and M (values and columns) read once
            PhaseScope scope(c, PH_RITZ, (double)N * (m + 3 * qmax) * sizeof(double) + 20.0 * (double)S.nnz);
            const int qn = qmax <= 8 ? 8 : (qmax <= 16 ? 16 : (qmax <= 24 ? 24 : 32));
            dim3 g(B.nch, (qmax + qn - 1) / qn);
            auto kern = qn == 8 ? bgemm_ritz_kernel<8>
                                : (qn == 16 ? bgemm_ritz_kernel<16> : (qn == 24 ? bgemm_ritz_kernel<24> : bgemm_ritz_kernel<32>));
            { count_launch(c); kern<<<g, 256, 0, st>>>(c->V.ptr + (long long)col0 * B.ld, B.ld, m, B.W.ptr, qmax, B.ch, U, N); }
            RIGA_CUDA_TRY(c, B.rpart.alloc((size_t)2 * B.nch * qmax));
            // M U by the sparse product (not MV W, a dense product of m columns)
            { count_launch(c); bresid_kernel<<<dim3(B.nch, qmax), 256, 0, st>>>(c->rowptr.ptr, c->col.ptr, c->Kval.ptr, c->Mval.ptr,
                                                                               U, MU, N, B.lam.ptr, qmax, B.ch, B.rpart.ptr); }
        }
        std::vector<double> part((size_t)2 * B.nch * qmax);
        RIGA_CUDA_TRY(c, cudaMemcpyAsync(part.data(), B.rpart.ptr, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
        std::vector<int> dcol((size_t)P * qmax, -1);
        bool rejected = false;
        for (int b = 0; b < P; ++b) {
            for (int q = 0; q < nsel[b]; ++q) {
                double ra = 0.0, rb = 0.0;
                for (int cc = B.h_cbeg[b]; cc < B.h_cend[b]; ++cc) {
                    ra += part[((size_t)q * B.nch + cc) * 2];
                    rb += part[((size_t)q * B.nch + cc) * 2 + 1];
                }
                const double l = hl[(size_t)b * qmax + q];
                const double rho = std::sqrt(ra) / (std::fabs(l) * std::sqrt(rb));
                if (!(rho <= lock_tol)) {
                    rejected = true;
                    continue;
                }
                dcol[(size_t)b * qmax + q] = nlock[b];
                lam[b].push_back(l);
                res[b].push_back(rho);
                ++nlock[b];
            }
        }
        if (rejected && c->precision == RIGA_FP64 && !refine64) {
            for (int i = 2; i < 4; ++i) RIGA_CUDA_TRY(c, c->vwork[i].alloc(N));
            xw = c->vwork[2].ptr;
            rwk = c->vwork[3].ptr;
            c->fp64_sweeps = 2;
            refine64 = true;
            if (dbg) std::fprintf(stderr, "[riga] batch: a candidate missed the residual bar; FP64 solves refined once\n");
        }
        RIGA_CUDA_TRY(c, B.dcol.upload(dcol, st));
        { count_launch(c); bscatter_cols_kernel<<<(unsigned)((N * qmax + 255) / 256), 256, 0, st>>>(
            N, qmax, c->prob_of_pos.ptr, B.dcol.ptr, U, MU, N, c->V.ptr, c->MV.ptr, B.ld); }
        // completeness per problem: check shift in a gap after the k-th eigenvalue
        std::vector<double> sig_chk(P, sigma0);
        std::vector<int> gi(P, -1);
        int checks = 0;
        for (int b = 0; b < P; ++b) {
            if (done[b]) continue;
            std::vector<double> sl(lam[b]);
            std::sort(sl.begin(), sl.end());
            for (int i = k; i < (int)sl.size(); ++i)
                if (sl[i] - sl[i - 1] > gap_rel * std::fabs(sl[i])) {
                    gi[b] = i;
                    break;
                }
            if (gi[b] < 0) {
                need[b] = nlock[b] + extra;
                continue;
            }
            sig_chk[b] = 0.5 * (sl[gi[b] - 1] + sl[gi[b]]);
            ++checks;
        }
        if (checks > 0) {
            t0 = clk::now();
            rc = factor_batch(c, sig_chk, true);
            t_fact += ms_since(t0);
            if (rc) {
                status = rc;
                break;
            }
            for (int b = 0; b < P; ++b) {
                if (done[b] || gi[b] < 0) continue;
                const long long inside = c->inertia_prob[b] - nu0[b];
                if (inside == gi[b]) done[b] = 1;
                else if (inside > gi[b]) need[b] = nlock[b] + (int)(inside - gi[b]);
                else status = set_error(c, RIGA_ENOCONV, "more locked pairs than the inertia allows");
            }
        }
        int nd = 0;
        for (int b = 0; b < P; ++b) nd += done[b];
        if (dbg)
            std::fprintf(stderr,
                         "[riga] batch run %d: steps=%d, problems complete %d/%d; host ms: checks %.1f, "
                         "tridiag RR %.1f, start %.1f, factor calls %.1f, total %.1f\n",
                         run, m, nd, P, t_checks, t_rr, t_start, t_fact, ms_since(t_all));
        if (status) break;
    }
    // outputs: the k smallest locked eigenvalues per problem
    c->batch_evals.assign((size_t)P * k, std::nan(""));
    c->batch_resid.assign((size_t)P * k, std::nan(""));
    c->batch_nconv.assign(P, 0);
    bool all_done = true;
    for (int b = 0; b < P; ++b) {
        std::vector<int> ord(lam[b].size());
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int x, int y) { return lam[b][x] < lam[b][y]; });
        const int nout = done[b] ? std::min(k, (int)ord.size()) : 0;
        for (int q = 0; q < nout; ++q) {
            c->batch_evals[(size_t)b * k + q] = lam[b][ord[q]];
            c->batch_resid[(size_t)b * k + q] = res[b][ord[q]];
        }
        c->batch_nconv[b] = nout;
        all_done = all_done && done[b] && nout == k;
    }
    if (status) return status;
    if (!all_done) return set_error(c, RIGA_ENOCONV, "some problems of the batch did not converge");
    return RIGA_OK;
}

}  // namespace riga

using namespace riga;

extern "C" int riga_assemble_batch(riga_ctx* c, int nprob, const riga_mesh* meshes, const double* const* coefK,
                                   const double* const* coefM) {
    if (!c || nprob < 1 || !meshes) return RIGA_EINVAL;
    c->last_error.clear();
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    cudaSetDevice(c->device);
    c->assembled = false;
    c->factored = false;
    c->nev = 0;
    c->analyzed_only = false;
    // key of the batch's patterns: the symbolic phase is skipped when the
    // meshes repeat (numeric re-assembly only, as for a single problem)
    std::vector<int> key{-1, nprob};
    for (int b = 0; b < nprob; ++b) {
        const riga_mesh* m = &meshes[b];
        if (m->dim < 1 || m->dim > 3 || m->dirichlet != 1 || m->p < 1 || m->p > 6 || m->leaf_extent < 0)
            return set_error(c, RIGA_EINVAL, "bad mesh in the batch: problem " + std::to_string(b));
        key.push_back(m->dim);
        key.push_back(m->p);
        key.push_back(m->leaf_extent > 0 ? m->leaf_extent : 8);
        for (int a = 0; a < m->dim; ++a) {
            if (m->ne[a] < 1 || m->ne[a] > (1 << 20))
                return set_error(c, RIGA_EINVAL, "ne out of range: problem " + std::to_string(b));
            key.push_back(m->ne[a]);
            for (int i = 0; i + 1 < m->ne[a]; ++i) key.push_back(m->mult[a] ? m->mult[a][i] : 1);
        }
    }
    if (key != c->mesh_key) {
        c->mesh_key.clear();
        c->probs.assign(nprob, Symbolic());
        for (int b = 0; b < nprob; ++b) {
            const riga_mesh* m = &meshes[b];
            std::string err = build_symbolic(c->probs[b], m->dim, m->ne, m->p, m->mult, m->leaf_extent);
            if (!err.empty()) return set_error(c, RIGA_EINVAL, "problem " + std::to_string(b) + ": " + err);
        }
        std::string err = merge_symbolic(c->S, c->probs);
        long long nchk = 0;
        if (err.empty()) err = check_bulk_copies(c->S, &nchk);  // every bulk copy aligned and in range
        if (!err.empty()) return set_error(c, RIGA_EINVAL, err);
        int rc0 = upload_symbolic(c);
        if (rc0) return rc0;
        rc0 = prepare_batch_assembly(c);
        if (rc0) return rc0;
        c->mesh_key = key;  // starts with -1: never equal to a single mesh's key
    }
    // coefficients: host pointers, concatenated (NULL per problem = ones)
    bool anyK = false, anyM = false;
    for (int b = 0; b < nprob; ++b) {
        anyK = anyK || (coefK && coefK[b]);
        anyM = anyM || (coefM && coefM[b]);
    }
    c->coefK.clear();
    c->coefM.clear();
    if (anyK) c->coefK.assign(c->S.n_elem, 1.0);
    if (anyM) c->coefM.assign(c->S.n_elem, 1.0);
    for (int b = 0; b < nprob; ++b) {
        const long long e0 = c->S.prob_elem[b], ne = c->probs[b].n_elem;
        for (long long e = 0; e < ne; ++e) {
            if (anyK && coefK[b]) {
                if (!(coefK[b][e] > 0.0) || !std::isfinite(coefK[b][e])) return set_error(c, RIGA_EINVAL, "coefK must be positive");
                c->coefK[e0 + e] = coefK[b][e];
            }
            if (anyM && coefM[b]) {
                if (!(coefM[b][e] > 0.0) || !std::isfinite(coefM[b][e])) return set_error(c, RIGA_EINVAL, "coefM must be positive");
                c->coefM[e0 + e] = coefM[b][e];
            }
        }
    }
    int rc = assemble_device(c);
    if (rc) return rc;
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->assembled = true;
    return RIGA_OK;
}

extern "C" int riga_eigs_batch(riga_ctx* c, int k, double sigma, double tol, double* evals, double* resid, int* nconv) {
    if (!c || !evals) return RIGA_EINVAL;
    c->last_error.clear();
    if (c->device < 0) return set_error(c, RIGA_ESTATE, "host-only context");
    cudaSetDevice(c->device);
    if (!c->assembled || c->S.dim != 0) return set_error(c, RIGA_ESTATE, "riga_assemble_batch first");
    if (!(tol > 0.0) || !std::isfinite(sigma)) return set_error(c, RIGA_EINVAL, "bad tol or sigma");
    int status = run_eigs_batch(c, k, sigma, tol);
    if (status != RIGA_OK && status != RIGA_ENOCONV) return status;
    const size_t P = c->batch_nconv.size();
    std::copy(c->batch_evals.begin(), c->batch_evals.end(), evals);
    if (resid) std::copy(c->batch_resid.begin(), c->batch_resid.end(), resid);
    if (nconv) std::copy(c->batch_nconv.begin(), c->batch_nconv.end(), nconv);
    (void)P;
    return status;
}
