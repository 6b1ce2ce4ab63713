// Shared pieces of the single-vector (lanczos.cu) and block (block.cu)
// shift-and-invert Lanczos drivers.
#pragma once

#include <cstdint>
#include <vector>

#include "ctx.h"

namespace riga {

constexpr int CH = 256;  // rows per chunk of the tall-skinny kernels
constexpr int TJ = 32;   // basis columns per shared-memory tile
constexpr int HR = 128;  // rows per shared-memory tile (a chunk is staged in HR-row pieces)

struct Run {
    riga_ctx* c;
    long long N, ld;
    int cap;       // columns of V / MV
    int nch;       // chunks
    double* w;
    double* Mw;
    double* xw;
    double* rw;
    double* c1;
    double* c2;
    double* alpha;
    double* beta;
    bool cgs2 = false;  // two full Gram-Schmidt passes per step (set once one pass was not enough)
};

uint64_t splitmix(uint64_t& s);
void enqueue_start_vector(riga_ctx* c, long long n, uint64_t& seed, double* w);
// out[j] = sum over nch chunks of partial[c * pstride + j], j < J (fixed order)
void enqueue_reduce_cols(riga_ctx* c, const double* partial, int nch, int J, int pstride, double* out);
int ortho_pass(Run& R, int col0, int J, double* w);
int recur_pass(Run& R, int J, int u0, int Ju, double* w);
void normalize_into(Run& R, double* w, int col, int jslot, int Jc);
int factor_at(riga_ctx* c, double sigma, int precision, long long* nu, bool inertia_only = false);
int calibrate_refinement(riga_ctx* c, uint64_t seed);
int calibrate_fp64_solve(riga_ctx* c, uint64_t seed);  // refinement sweeps FP64 fronts need (1 = none)
int configure_reorth(riga_ctx* c, int cap);  // shared-memory attributes of the reorthogonalization kernels
int ritz_vectors_resid(Run& R, int col0, int J, const std::vector<double>& W, int nsel, double* U, double* MU,
                       const std::vector<double>& lam, int nres, std::vector<double>& rho);
int ritz_lock(Run& R, int col0, int m, const std::vector<double>& Wsel, const std::vector<double>& lcand,
              int nlock, double lock_tol, std::vector<double>& lam, int* n_locked);

// One block Lanczos run of block size B (block.cu): a start block of B
// random vectors M-orthogonal to the nlock locked ones, block steps until the
// want_run largest acceptable Ritz values are converged (or m_max vectors),
// Rayleigh-Ritz and residual-checked locking.  Returns the steps (vectors)
// taken in *m and the pairs locked in *n_locked.
int block_run(Run& R, int B, int nlock, int want_run, int m_max, double cur_sigma, double sigma0, double tol_est,
              double lock_tol, int lock_cap, uint64_t& seed, std::vector<double>& lam, int* m, int* n_locked);

}  // namespace riga
