// Every eigenpair in an interval [lo, hi) by dynamic spectrum slicing with
// thick-restart shift-and-invert Lanczos (Sec. 4.1, Sec. 4.2 with
// Eq. LanczosRestart, the Remark on inertia, Sec. 6: Krylov-Schur restarts
// with spectrum slicing).
//
// Counting.  The inertia of K - sigma M (FP64 fronts) gives the number of
// eigenvalues below sigma; nu(hi) - nu(lo) is the number in the interval.
//
// Slices.  A slice starts at a (first lo) with the shift sigma = a; its
// Lanczos runs lock eigenpairs with lambda in [a, hi).  Once `slice` of them
// (plus `extra`) are locked, the slice closes at the midpoint b of the first
// relative gap > 1e-6 after the slice-th locked value; nu(b) - nu(a) must
// equal the number locked in [a, b).  The pairs below b go to the output;
// the next slice starts at a = b, whose factorization (FP64 path) already
// carries the solve operators.  The shifts therefore follow the spectrum's
// own density: each slice ends where its eigenvalues ran out.  Missing
// eigenvalues (copies of a degenerate eigenvalue that one Krylov sequence
// cannot see) are searched by fresh runs that lock only eigenvalues in
// [a, b): first at the slice's shift, then next to the missing ones, which
// inertia counts at midpoints between the locked values locate (bisection).
//
// Bounded memory.  The runs orthogonalize against a window of locked
// vectors: those of the previous slice (the eigenvalues just below a, the
// nearest to the shift on that side) and those locked in the current slice.
// Older slices are not kept; their eigenvalues lie below a and are never
// locked again.  The basis therefore holds at most 2 (slice + extra + 8) + 16
// window vectors plus the m + 1 of a run, whatever the number of pairs.
//
// Thick restart (Wu and Simon's form of Eq. LanczosRestart).  A run builds
// m Lanczos vectors in the M-inner product; at the end of a cycle the
// projected matrix (an arrowhead block of kept Ritz values theta_i with
// couplings b_i, then the tridiagonal alpha / beta of the cycle's steps) is
// diagonalized on the host; converged wanted Ritz pairs are checked by their
// FP64 residual and locked; the keep largest-|theta| unconverged wanted Ritz
// vectors Y, with H Y = Y Theta + v_{m+1} b^T, b_i = beta_m s_{m,i}, and
// v_{m+1} start the next cycle, whose first step orthogonalizes against all
// of them (two Gram-Schmidt passes).  Wanted: lambda = sigma + 1/theta in
// [a, hi), by decreasing |theta|.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <vector>

#include "lanczos.h"

namespace riga {

namespace {

struct Slicer {
    riga_ctx* c;
    Run R;
    int m = 0;          // Lanczos vectors per cycle
    int wcap = 0;       // window capacity
    int nprev = 0;      // window columns [0, nprev): previous slice's pairs
    int nw = 0;         // window columns [nprev, nw): this slice's locked pairs
    std::vector<double> lam_win;  // eigenvalues of the window columns
    double tol_est = 0, lock_tol = 0;
    DevBuf<double> scr;  // Ritz vectors and their M-images of a restart
    uint64_t seed = 1;
};

// dense J x J projected matrix of a cycle: c kept Ritz values (arrowhead with
// couplings bc to local vector c), then the tridiagonal alpha[c..J-1],
// beta[c+1..J-1]
void projected(int c, const std::vector<double>& th, const std::vector<double>& bc, const double* alpha,
               const double* beta, int J, std::vector<double>& T) {
    T.assign((size_t)J * J, 0.0);
    auto t = [&](int i, int j) -> double& { return T[(size_t)j * J + i]; };
    for (int i = 0; i < c && i < J; ++i) {
        t(i, i) = th[i];
        if (c < J) t(i, c) = t(c, i) = bc[i];
    }
    for (int j = c; j < J; ++j) {
        t(j, j) = alpha[j];
        if (j + 1 < J) t(j, j + 1) = t(j + 1, j) = beta[j + 1];
    }
}

// copies columns src (of V / MV, or of the scratch U / MU) to V / MV column dst
int put_col(riga_ctx* c, Run& R, const double* u, const double* mu, int dst) {
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->V.ptr + (long long)dst * R.ld, u, R.N * sizeof(double), cudaMemcpyDeviceToDevice,
                                     c->stream));
    RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->MV.ptr + (long long)dst * R.ld, mu, R.N * sizeof(double),
                                     cudaMemcpyDeviceToDevice, c->stream));
    return RIGA_OK;
}

// One thick-restart run at shift sigma: up to max_cycles cycles of m steps;
// locks (into the window, at most lock_room) converged pairs with lambda in
// [a, hi) until `want` were locked in this run.  *n_locked: pairs locked.
int trlan_run(Slicer& L, int want, int lock_room, double sigma, double a, double hi, int max_cycles, int* n_locked) {
    static const bool dbg = std::getenv("RIGA_DEBUG") != nullptr;
    riga_ctx* c = L.c;
    Run& R = L.R;
    cudaStream_t st = c->stream;
    const long long N = R.N;
    const int m = L.m;
    *n_locked = 0;
    // fresh start vector, M-orthogonal to the window
    enqueue_start_vector(c, N, L.seed, R.w);
    int col0 = L.nw;
    if (L.nw > 0) ortho_pass(R, 0, L.nw, R.w);
    normalize_into(R, R.w, col0, -1, 0);
    int ck = 0;  // kept Ritz vectors at local 0..ck-1, the cycle's start vector at local ck
    std::vector<double> th_keep, b_keep, hab(2 * (size_t)m + 8), T, theta, Z;
    int j = 0;
    for (int cycle = 0; cycle < max_cycles; ++cycle) {
        bool converged = false;
        int J = 0;  // vectors of the projected matrix (local 0..J-1), local J the residual direction
        for (; j < m; ++j) {
            const int col = col0 + j;
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(R.w, c->MV.ptr + (long long)col * R.ld, N * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
            int rc = solve_refined(c, R.w, R.xw, R.rw, 0.0, c->ir_sweeps, 0, nullptr);
            if (rc) return rc;
            if (R.cgs2 || (j == ck && ck > 0)) {
                ortho_pass(R, 0, col + 1, R.w);
                normalize_into(R, R.w, col + 1, j, 0);
            } else {
                recur_pass(R, col + 1, j == ck ? col : col - 1, j == ck ? 1 : 2, R.w);
                normalize_into(R, R.w, col + 1, j, col + 1);
            }
            c->stats.steps++;
            J = j + 1;
            const bool last = (j + 1 == m);
            if (!last && (J - ck) % 10 != 0) continue;
            // convergence test on the projected matrix
            int dflag = 0, rflag = 0;
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(hab.data(), c->ab.ptr, hab.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(&dflag, c->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(&rflag, c->bflag.ptr, sizeof(int), cudaMemcpyDeviceToHost, st));
            RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
            if (dflag & 2) return set_error(c, RIGA_ETIMEOUT, "a dependency wait of the tree solve gave up");
            if (rflag & 2) R.cgs2 = true;
            const double* al = hab.data();
            const double* be = hab.data() + m + 2;
            projected(ck, th_keep, b_keep, al, be, J, T);
            theta.assign(J, 0.0);
            Z.assign((size_t)J * J, 0.0);
            sym_eig_dense(J, T.data(), theta.data(), Z.data());
            const double bJ = be[J];
            std::vector<int> wanted;
            for (int i = 0; i < J; ++i) {
                if (theta[i] == 0.0) continue;
                const double l = sigma + 1.0 / theta[i];
                if (l >= a && l < hi) wanted.push_back(i);
            }
            std::sort(wanted.begin(), wanted.end(), [&](int x, int y) { return std::fabs(theta[x]) > std::fabs(theta[y]); });
            int ok = 0;
            for (int q = 0; q < (int)wanted.size() && q < want; ++q)
                if (std::fabs(bJ * Z[(size_t)wanted[q] * J + (J - 1)]) <= L.tol_est * std::fabs(theta[wanted[q]])) ++ok;
            if ((int)wanted.size() >= want && ok >= want) converged = true;
            if (bJ <= 1e-300) converged = true;
            if (converged || last) break;
        }
        // Rayleigh-Ritz at the end of the cycle (theta, Z of the J x J projection)
        const double* be = hab.data() + m + 2;
        const double bJ = be[J];
        std::vector<int> lockc, keep;
        std::vector<int> wanted;
        for (int i = 0; i < J; ++i) {
            if (theta[i] == 0.0) continue;
            const double l = sigma + 1.0 / theta[i];
            if (l >= a && l < hi) wanted.push_back(i);
        }
        std::sort(wanted.begin(), wanted.end(), [&](int x, int y) { return std::fabs(theta[x]) > std::fabs(theta[y]); });
        const int room = std::min(L.wcap - L.nw, lock_room - *n_locked);
        for (int i : wanted) {
            const bool conv = std::fabs(bJ * Z[(size_t)i * J + (J - 1)]) <= L.tol_est * std::fabs(theta[i]);
            if (conv && (int)lockc.size() < room) lockc.push_back(i);
            else keep.push_back(i);
        }
        // restart size: the best unconverged wanted vectors, up to half the cycle
        const int kmax = std::max(1, std::min(m / 2, m - 8 - (int)lockc.size()));
        if ((int)keep.size() > kmax) keep.resize(kmax);
        const int nl = (int)lockc.size(), nk = converged ? 0 : (int)keep.size();
        const int nsel = nl + nk;
        std::vector<double> W((size_t)J * std::max(nsel, 1)), lam(nl);
        for (int q = 0; q < nl; ++q) {
            std::copy(&Z[(size_t)lockc[q] * J], &Z[(size_t)lockc[q] * J] + J, &W[(size_t)q * J]);
            lam[q] = sigma + 1.0 / theta[lockc[q]];
        }
        for (int q = 0; q < nk; ++q) std::copy(&Z[(size_t)keep[q] * J], &Z[(size_t)keep[q] * J] + J, &W[(size_t)(nl + q) * J]);
        std::vector<double> rho;
        if (nsel > 0) {
            RIGA_CUDA_TRY(c, L.scr.alloc((size_t)N * 2 * nsel));
            int rc = ritz_vectors_resid(R, col0, J, W, nsel, L.scr.ptr, L.scr.ptr + (size_t)N * nsel, lam, nl, rho);
            if (rc) return rc;
        }
        const double* U = L.scr.ptr;
        const double* MU = L.scr.ptr + (size_t)N * nsel;
        // keep the residual direction (local J) before the columns are rearranged
        if (!converged) {
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(R.w, c->V.ptr + (long long)(col0 + J) * R.ld, N * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
            RIGA_CUDA_TRY(c, cudaMemcpyAsync(R.Mw, c->MV.ptr + (long long)(col0 + J) * R.ld, N * sizeof(double),
                                             cudaMemcpyDeviceToDevice, st));
        }
        // lock the candidates that pass the FP64 residual test; the others
        // stay in the restart basis
        std::vector<int> kept_idx;  // indices into the selection (columns of U)
        if (dbg && nl > 0) {
            int failed = 0;
            double worst = 0.0;
            for (int q = 0; q < nl; ++q)
                if (!(rho[q] <= L.lock_tol)) {
                    ++failed;
                    worst = std::max(worst, rho[q]);
                }
            if (failed) std::fprintf(stderr, "[riga] trlan: %d of %d lock candidates failed the residual test (worst %.3g)\n", failed, nl, worst);
        }
        for (int q = 0; q < nl; ++q) {
            if (rho[q] <= L.lock_tol) {
                int rc = put_col(c, R, U + (size_t)q * N, MU + (size_t)q * N, L.nw);
                if (rc) return rc;
                L.lam_win.push_back(lam[q]);
                ++L.nw;
                ++*n_locked;
            } else if (!converged) {
                kept_idx.push_back(q);
            }
        }
        if (converged || *n_locked >= want) return RIGA_OK;
        for (int q = 0; q < nk; ++q) kept_idx.push_back(nl + q);
        if ((int)kept_idx.size() > kmax) kept_idx.resize(kmax);
        // restart: [window][kept Ritz vectors][residual direction]
        col0 = L.nw;
        th_keep.clear();
        b_keep.clear();
        for (int q = 0; q < (int)kept_idx.size(); ++q) {
            const int s = kept_idx[q];
            const int i = s < nl ? lockc[s] : keep[s - nl];
            int rc = put_col(c, R, U + (size_t)s * N, MU + (size_t)s * N, col0 + q);
            if (rc) return rc;
            th_keep.push_back(theta[i]);
            b_keep.push_back(bJ * Z[(size_t)i * J + (J - 1)]);
        }
        ck = (int)kept_idx.size();
        {
            int rc = put_col(c, R, R.w, R.Mw, col0 + ck);
            if (rc) return rc;
        }
        j = ck;
    }
    return RIGA_OK;
}

// Bisection for missing eigenvalues of [a, b): sl[0..below) are the locked
// values in [a, b), ascending; nu(a) = nu_a.  Groups of equal locked values
// (relative 1e-9) are the candidates; an FP64 inertia count at the midpoint
// between two groups tells which side holds more eigenvalues than are
// locked.  *shift: inside the narrowest sub-interval found, just above its
// group (a tenth of the way to the next boundary), so that the missing
// eigenvalues are the nearest unlocked ones.
int locate_missing(riga_ctx* c, double a, double b, long long nu_a, const std::vector<double>& sl, int below,
                   std::map<double, long long>& cache, double* shift) {
    std::vector<double> gval;   // group values
    std::vector<int> gend;      // locked count up to and including the group
    for (int i = 0; i < below; ++i) {
        if (gval.empty() || sl[i] - gval.back() > 1e-9 * std::fabs(sl[i])) gval.push_back(sl[i]);
        else gend.pop_back();
        gend.push_back(i + 1);
    }
    const int G = (int)gval.size();
    if (G == 0) {
        *shift = 0.5 * (a + b);
        return RIGA_OK;
    }
    // invariant: missing eigenvalues in [left, right) with groups lo..hi-1 inside
    int lo = 0, hi = G;
    double left = a, right = b;
    long long nu_left = nu_a;
    int locked_left = 0;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        const double t = 0.5 * (gval[mid - 1] + gval[mid]);
        long long nu_t = 0;
        auto it = cache.find(t);
        if (it != cache.end()) {
            nu_t = it->second;
        } else {
            int rc = factor_at(c, t, RIGA_FP64, &nu_t, true);
            if (rc) return rc;
            cache[t] = nu_t;
        }
        const int locked_t = gend[mid - 1];
        if (nu_t - nu_left > locked_t - locked_left) {
            hi = mid;
            right = t;
        } else {
            lo = mid;
            left = t;
            nu_left = nu_t;
            locked_left = locked_t;
        }
    }
    *shift = gval[lo] + 0.1 * (right - gval[lo]);
    (void)left;
    return RIGA_OK;
}

}  // namespace

int run_eigs_interval(riga_ctx* c, double lo, double hi, int kmax, double tol, int m_basis, int* nfound,
                      int* basis_cols) {
    static const bool dbg = std::getenv("RIGA_DEBUG") != nullptr;
    Symbolic& S = c->S;
    cudaStream_t st = c->stream;
    const long long N = S.N;
    const int slice = c->opt_slice > 0 ? c->opt_slice : 50;
    const int extra = c->opt_extra > 0 ? c->opt_extra : 2;
    const int prec = c->opt_precision;
    const double gap_rel = 1e-6;
    *nfound = 0;
    c->nev = 0;
    c->evals.clear();
    c->stats = Stats();
    // eigenvalue count of the interval from two FP64 inertias (nu(lo) = 0 for
    // lo <= 0: K and M are positive definite)
    long long nu_lo = 0, nu_hi = 0;
    int rc = RIGA_OK;
    if (lo > 0.0) {
        rc = factor_at(c, lo, RIGA_FP64, &nu_lo, true);
        if (rc) return rc;
    }
    rc = factor_at(c, hi, RIGA_FP64, &nu_hi, true);
    if (rc) return rc;
    const long long count = nu_hi - nu_lo;
    if (count > kmax) {
        *nfound = (int)std::min<long long>(count, 2000000000LL);
        return set_error(c, RIGA_EINVAL, "the interval holds more eigenvalues than kmax (count in *nfound)");
    }
    if (count <= 0) return RIGA_OK;
    Slicer L;
    L.c = c;
    L.m = (int)std::min<long long>(m_basis > 0 ? m_basis : std::max(2 * (slice + extra), slice + extra + 40), N - 2);
    L.wcap = 2 * (slice + extra + 8) + 16;
    L.tol_est = 1e-2 * tol;
    L.lock_tol = 0.5 * tol;
    L.seed = c->opt_seed ? c->opt_seed : 1;
    Run& R = L.R;
    R.c = c;
    R.N = N;
    R.ld = N;
    R.cap = L.wcap + L.m + 2;
    R.nch = (int)((N + CH - 1) / CH);
    if (basis_cols) *basis_cols = R.cap;
    if (c->V.alloc((size_t)N * R.cap) != cudaSuccess || c->MV.alloc((size_t)N * R.cap) != cudaSuccess)
        return set_error(c, RIGA_ENOMEM, "Lanczos basis");
    if (c->evec_perm.alloc((size_t)N * count) != cudaSuccess) return set_error(c, RIGA_ENOMEM, "eigenvector output");
    RIGA_CUDA_TRY(c, c->partial.alloc((size_t)R.nch * R.cap));
    RIGA_CUDA_TRY(c, c->coef.alloc(2 * (size_t)R.cap));
    RIGA_CUDA_TRY(c, c->ab.alloc(2 * (size_t)L.m + 8));
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
    R.alpha = c->ab.ptr;
    R.beta = c->ab.ptr + L.m + 2;
    R.cgs2 = c->opt_reorth == 2;
    rc = configure_reorth(c, R.cap);
    if (rc) return rc;
    DevBuf<double> hold;  // window compaction
    double a = lo;
    long long nu_a = nu_lo;
    double sigma = lo > 0.0 ? lo : 0.0;
    double factored = std::nan(""), calibrated = std::nan("");
    long long found = 0;
    int runs = 0, fruitless = 0;
    int target = (int)std::min<long long>(slice, count);
    // the slice end b once chosen, and its inertia; while it is pending the
    // runs lock only eigenvalues in [a, b) (the missing ones)
    bool have_b = false;
    double b = hi;
    long long nu_b = nu_hi;
    std::map<double, long long> inertia_cache;  // FP64 inertia counts of the bisection
    int status = RIGA_OK;
    while (found < count) {
        const long long remaining = count - found;
        const double ub = have_b ? b : hi;
        // this slice's locked pairs (all >= a) sorted, and how many lie below ub
        const int this_cnt = L.nw - L.nprev;
        std::vector<int> ord(this_cnt);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int x, int y) { return L.lam_win[L.nprev + x] < L.lam_win[L.nprev + y]; });
        std::vector<double> sl(this_cnt);
        for (int i = 0; i < this_cnt; ++i) sl[i] = L.lam_win[L.nprev + ord[i]];
        const int below = (int)(std::lower_bound(sl.begin(), sl.end(), ub) - sl.begin());
        int want_run = 0;
        if (!have_b) {
            const int want_slice = (int)std::min<long long>(target, remaining);
            const int need = (int)std::min<long long>(want_slice + extra, remaining);
            if (this_cnt >= need) {
                if (this_cnt >= remaining) {
                    b = hi;
                    nu_b = nu_hi;
                } else {
                    int gi = -1;
                    for (int i = std::max(want_slice, 1); i < this_cnt; ++i)
                        if (sl[i] - sl[i - 1] > gap_rel * std::fabs(sl[i])) {
                            gi = i;
                            break;
                        }
                    if (gi < 0) {  // no gap yet after the slice's pairs: lock more
                        target = this_cnt + 1;
                        continue;
                    }
                    b = 0.5 * (sl[gi - 1] + sl[gi]);
                    const bool reuse = prec == RIGA_FP64;
                    rc = factor_at(c, b, RIGA_FP64, &nu_b, !reuse);
                    if (rc) { status = rc; break; }
                    if (reuse) factored = b;
                }
                have_b = true;
                continue;
            }
            want_run = need - this_cnt;
        } else {
            const long long expected = nu_b - nu_a;
            if (dbg)
                std::fprintf(stderr, "[riga] slice check: a=%.12g b=%.12g locked below b=%d expected=%lld\n", a, b, below,
                             expected);
            if (below == expected) {
                // the slice is complete: its pairs below b to the output
                for (int i = 0; i < below; ++i) {
                    const int colw = L.nprev + ord[i];
                    RIGA_CUDA_TRY(c, cudaMemcpyAsync(c->evec_perm.ptr + (long long)(found + i) * N,
                                                     c->V.ptr + (long long)colw * R.ld, N * sizeof(double),
                                                     cudaMemcpyDeviceToDevice, st));
                    c->evals.push_back(sl[i]);
                }
                found += below;
                // new window: this slice's pairs (below b), then those above b
                const int nkeep = this_cnt;
                RIGA_CUDA_TRY(c, hold.alloc((size_t)2 * N * std::max(nkeep, 1)));
                for (int i = 0; i < nkeep; ++i) {
                    const int colw = L.nprev + ord[i];
                    RIGA_CUDA_TRY(c, cudaMemcpyAsync(hold.ptr + (size_t)i * N, c->V.ptr + (long long)colw * R.ld,
                                                     N * sizeof(double), cudaMemcpyDeviceToDevice, st));
                    RIGA_CUDA_TRY(c, cudaMemcpyAsync(hold.ptr + (size_t)(nkeep + i) * N, c->MV.ptr + (long long)colw * R.ld,
                                                     N * sizeof(double), cudaMemcpyDeviceToDevice, st));
                }
                for (int i = 0; i < nkeep; ++i) {
                    rc = put_col(c, R, hold.ptr + (size_t)i * N, hold.ptr + (size_t)(nkeep + i) * N, i);
                    if (rc) return rc;
                }
                L.nprev = below;
                L.nw = nkeep;
                L.lam_win = sl;
                a = b;
                nu_a = nu_b;
                sigma = b;
                have_b = false;
                inertia_cache.clear();
                target = (int)std::min<long long>(slice, count - found);
                fruitless = 0;
                continue;
            }
            if (below > expected) {
                status = set_error(c, RIGA_ENOCONV, "more locked pairs than the inertia allows");
                break;
            }
            // eigenvalues missing in [a, b) (copies of degenerate eigenvalues
            // that a single Krylov sequence cannot see): fresh runs that lock
            // only in [a, b); the first at the slice's shift, later ones at a
            // shift next to the missing eigenvalues, located by bisecting
            // the locked values with inertia counts
            want_run = (int)(expected - below);
            if (fruitless > 0) {
                double sm = sigma;
                rc = locate_missing(c, a, b, nu_a, sl, below, inertia_cache, &sm);
                if (rc) { status = rc; break; }
                if (dbg) std::fprintf(stderr, "[riga] slice missing %d in [%.12g, %.12g): shift %.12g\n", want_run, a, b, sm);
                sigma = sm;
            }
        }
        if (++runs > 400 || fruitless > 6) {
            status = set_error(c, RIGA_ENOCONV, "spectrum slicing did not converge");
            break;
        }
        if (!(factored == sigma)) {
            rc = factor_at(c, sigma, prec, nullptr);
            if (rc) { status = rc; break; }
            factored = sigma;
        }
        if (!(calibrated == sigma)) {
            // sweeps per solve: low-precision fronts always refine; FP64
            // fronts at an interior shift (an indefinite matrix factored
            // without pivoting can lose accuracy through pivot growth) refine
            // when one solve does not reach a relative residual of 1e-13
            if (c->precision != RIGA_FP64) {
                rc = calibrate_refinement(c, L.seed + (uint64_t)runs);
            } else {
                rc = calibrate_fp64_solve(c, L.seed + (uint64_t)runs);
            }
            if (rc) { status = rc; break; }
            calibrated = sigma;
            if (dbg) std::fprintf(stderr, "[riga] slice shift %.12g: %d solve sweep(s)\n", sigma,
                                  c->precision == RIGA_FP64 ? c->fp64_sweeps : c->ir_sweeps);
        }
        int acc = 0;
        want_run = std::max(want_run, 1);
        rc = trlan_run(L, want_run, want_run + 8, sigma, a, ub, 8, &acc);
        if (rc) { status = rc; break; }
        if (dbg)
            std::fprintf(stderr, "[riga] slice run %d: shift=%.12g a=%.12g ub=%.12g locked=%d window=%d found=%lld/%lld\n",
                         runs, sigma, a, ub, acc, L.nw, found, count);
        if (acc == 0) ++fruitless;
        else fruitless = 0;
    }
    c->nev = (int)found;
    *nfound = (int)found;
    RIGA_CUDA_TRY(c, cudaStreamSynchronize(st));
    return status;
}

}  // namespace riga
