// Internal context of the riga library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

#include "../../include/riga.h"
#include "symbolic.h"

namespace riga {

// Threads per CSR row in the SpMV kernels.  With about 50 (2D, p = 3) to 350
// (3D) entries per row, four lanes per row keep the FP64 pipe on the
// products: with 16 lanes the partially filled last pass and the cross-lane
// sums (every lane adds) took most of its issue slots.
constexpr int SPMV_TPR = 4;
constexpr int SPMV_RPB = 256 / SPMV_TPR;  // rows per 256-thread block

// Sum of a value held by the first lane of each SPMV_TPR-lane group over the
// warp (the result in lane 0; all lanes take part)
__device__ __forceinline__ double warp_sum_groups(double v) {
#pragma unroll
    for (int o = SPMV_TPR; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Sum over the SPMV_TPR lanes of a row group (the result in all of them)
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
    for (int o = SPMV_TPR / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, SPMV_TPR);
    return v;
}

// Owning device buffer (cudaMalloc/cudaFree).
template <typename T>
struct DevBuf {
    T* ptr = nullptr;
    size_t count = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        count = 0;
    }
    cudaError_t alloc(size_t n) {
        if (ptr && n <= count) return cudaSuccess;  // grow-only
        release();
        if (n == 0) return cudaSuccess;
        cudaError_t e = cudaMalloc((void**)&ptr, n * sizeof(T));
        if (e == cudaSuccess) count = n;
        else ptr = nullptr;
        return e;
    }
    cudaError_t upload(const std::vector<T>& v, cudaStream_t s) {
        cudaError_t e = alloc(v.size());
        if (e != cudaSuccess || v.empty()) return e;
        return cudaMemcpyAsync(ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    }
};

struct Stats {
    long long n_fact = 0, n_solve = 0, n_matvec = 0, steps = 0;
    double t_fact_ms = 0.0, t_lanczos_ms = 0.0;
    int ir_sweeps = 0;        // refinement sweeps per Lanczos solve (FP32 fronts)
    long long n_fallback = 0; // shifts refactored with FP64 fronts after refinement stalled
};

// Per-phase device timing (CUDA events around each phase's launches, only
// while profiling is on), launch counts and algorithmic work.
enum Phase { PH_ASSEMBLE = 0, PH_FACTOR, PH_SOLVE, PH_REORTH, PH_SPMV, PH_RITZ, PH_OTHER, PH_COUNT };
struct PhaseRec {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    long long launches = 0, calls = 0;
    double ms = 0.0, bytes = 0.0, flops = 0.0;
};
struct Profile {
    bool on = false;
    int cur = PH_OTHER;
    long long launches = 0;  // every kernel launch, profiling on or off
    PhaseRec ph[PH_COUNT];
};

}  // namespace riga

namespace riga {
// batch assembly descriptors: one segment per (problem, direction)
struct SegDev {
    int ne, p, ndof, pad;
    long long kv_off, ef_off, ke_off, kb_off;  // into the concatenated 1D arrays
};
struct ProbDev {
    int dim, p, seg0, pad;   // seg0: the problem's first segment
    long long row0, goff;    // first row / first global DOF
    long long e0;            // first element (coefficient offset)
};
}  // namespace riga

struct riga_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;

    // ------------------------------------------------------------ problem
    bool assembled = false;
    bool analyzed_only = false;
    bool factored = false;
    std::vector<int> mesh_key;
    riga::Symbolic S;                  // the problem, or the merged forest of a batch
    std::vector<riga::Symbolic> probs; // batch: the problems (1D data, sizes)
    std::vector<double> coefK, coefM;  // host copies (empty = constant); batch: concatenated
    std::vector<double> sigma_prob;    // batch: per-problem shifts of the next factorization (empty = sigma)

    // symbolic arrays on the device
    riga::DevBuf<riga::SolveItem> sitems;
    riga::DevBuf<riga::ChildRec> crec;
    riga::DevBuf<int> parts_f, parts_b;
    riga::DevBuf<riga::PanelItem> qitems;
    riga::DevBuf<long long> rowptr, front_off, front_ptr, rel_ptr, upd_off, scatter, perm_to_glob, glob_rowptr;
    riga::DevBuf<int> col, perm, ipos, node_ptr, kk, nn, front_pos, child_ptr, child_list, rel, parent;
    riga::DevBuf<riga::PanelItem> pitems;
    riga::DevBuf<riga::TileItem> titems;
    riga::DevBuf<riga::TcTile> tcitems;    // tensor-core update tiles
    riga::DevBuf<riga::TcPack> tcpacks;    // tensor-core panel blocks to pack
    riga::DevBuf<riga::TileItemL> tcnarrow; // within-super-panel update tiles of the tensor-core schedule
    riga::DevBuf<float> tcpack;            // packed panel blocks of one step (operands of the update)
    riga::DevBuf<float> tcscale;           // per packed block: power-of-two operand scale (BF16)
    riga::DevBuf<riga::TcPack> ozpacks;    // FP64 tensor-core schedule: blocks to pack per step
    riga::DevBuf<riga::TcTile> oztiles;    //   its tiles
    riga::DevBuf<unsigned char> ozpack;    //   digit-slice blocks of one step
    riga::DevBuf<int> ozexp;               //   per block: the rows' power-of-two exponents (A, then B)
    riga::DevBuf<int> ozlive;              //   per block: nonzero rows in A (bit 0), B rows 0-63 (1), 64-127 (2)
    int fp64_tc = 1;                       // FP64 fronts: 0 CUDA-core updates, 1 tensor-core digit slices
    riga::DevBuf<riga::ExtItem> eitems;
    // per-direction 1D data
    riga::DevBuf<int> kv[3], elem_first[3];
    riga::DevBuf<double> Ke1[3], Me1[3], Kb1[3], Mb1[3];
    riga::DevBuf<double> dcoefK, dcoefM;
    // batch assembly: concatenated 1D data of all problems
    riga::DevBuf<int> b_kv, b_ef;
    riga::DevBuf<riga::SegDev> b_segs;
    riga::DevBuf<riga::ProbDev> b_probs;
    riga::DevBuf<long long> b_eprefix, b_bprefix;
    riga::DevBuf<double> b_Ke, b_Me, b_Kb, b_Mb;
    int b_nseg = 0;
    long long b_nelem1d = 0, b_nband = 0;

    // matrices in elimination order (CSR of rowptr/col)
    riga::DevBuf<double> Kval, Mval;

    // --------------------------------------------------------------- factor
    int precision = RIGA_FP64;
    double sigma = 0.0;
    bool inertia_only = false;   // next factorization skips the solve operators (extra rows)
    riga::DevBuf<double> pool64;
    riga::DevBuf<float> pool32;
    riga::DevBuf<double> q64;    // packed solve operators (see Symbolic::qoff)
    riga::DevBuf<float> q32;
    riga::DevBuf<double> D;      // pivots in elimination order
    riga::DevBuf<int> flag;      // device error word (bit 0: pivot breakdown)
    riga::DevBuf<long long> neg; // inertia counter(s): one, or one per problem of a batch
    riga::DevBuf<int> prob_of_pos;  // batch: problem of each position
    riga::DevBuf<double> sig_pos;   // batch: shift of each position's problem
    // batch factorization as a CUDA graph (per-position shifts come from
    // sig_pos, so one graph per mode serves every call): [0] with the solve
    // operators, [1] inertia only; valid while the schedule and buffers are
    struct FactorGraph {
        cudaGraphExec_t exec = nullptr;
        long long gen = -1;
        const void* ptrs[9] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        int launches = 0;
    } fgraph[2];
    long long sched_gen = 0;            // bumped whenever the factorization schedule is uploaded
    cudaStream_t cap_stream = nullptr;  // private stream for graph capture
    std::vector<long long> inertia_prob;  // batch: inertia per problem
    long long inertia = -1;

    // ---------------------------------------------------------------- solve
    riga::DevBuf<double> upd;          // forward-solve update vectors
    riga::DevBuf<int> solve_order;     // 2F work items of the persistent solve
    riga::DevBuf<int> solve_flags;     // per-front completed parts, forward then backward
    riga::DevBuf<double> w1buf;        // assembled own right-hand sides of the forward sweep
    long long wait_limit = 1LL << 24;  // device dependency-wait budget (polls)
    long long* trace_buf = nullptr;    // device trace of the next solve (riga_trace_solve)
    riga::DevBuf<double> vwork[6];     // N-vectors (permuted order)
    riga::DevBuf<double> red;          // reduction scratch
    int ir_sweeps = 4;                 // refinement sweeps per solve inside Lanczos (FP32 factor)
    int fp64_sweeps = 1;               // FP64 factor: sweeps per solve (1 = plain; set by a calibration, reset by a factorization)

    // -------------------------------------------------------------- Lanczos
    int opt_slice = 0, opt_precision = RIGA_FP64, opt_max_steps = 0, opt_extra = 2;
    int opt_block = 1;                 // Lanczos block size (1, 2, 4; 0 = automatic)
    int opt_reorth = 1;                // 1: recurrence + one full Gram-Schmidt pass; 2: two full passes
    int opt_rq = 0;                    // 1: locked eigenvalues are double-double Rayleigh quotients
    riga::DevBuf<double> bwork, bcoef, bpartial, bsmall;  // block Lanczos workspace
    riga::DevBuf<int> bflag;
    double* bpin = nullptr;            // pinned host copies of the block-tridiagonal T
    size_t bpin_size = 0;
    unsigned long long opt_seed = 1;
    riga::DevBuf<double> V, MV;        // basis storage: locked vectors, then the run's vectors
    riga::DevBuf<double> coef;         // Gram-Schmidt coefficients
    riga::DevBuf<double> partial;      // per-chunk partial dots
    riga::DevBuf<double> ab;           // alpha / beta of the current run
    riga::DevBuf<double> Wd;           // Ritz coefficient matrix
    riga::DevBuf<double> evec_perm;    // final eigenvectors, permuted order, N x nev
    std::vector<double> evals;         // final eigenvalues
    std::vector<double> batch_evals, batch_resid;  // batch: k per problem, problem-major
    std::vector<int> batch_nconv;
    int nev = 0;
    riga::Stats stats;
    riga::Profile prof;
};

namespace riga {

// error helpers
int set_error(riga_ctx* c, int code, const std::string& msg);
#define RIGA_CUDA_TRY(ctx, call)                                                                 \
    do {                                                                                         \
        cudaError_t _e = (call);                                                                 \
        if (_e != cudaSuccess)                                                                   \
            return ::riga::set_error((ctx), RIGA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

// f(i) for i in [0, n) on up to 16 host threads (independent iterations)
template <typename Fn>
void parallel_for(int n, Fn f) {
    int nt = (int)std::thread::hardware_concurrency();
    nt = std::max(1, std::min({nt, 16, n / 8}));
    if (nt <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; ++t) {
        auto part = [=]() {
            for (int i = t; i < n; i += nt) f(i);
        };
        try {
            th.emplace_back(part);
        } catch (...) {  // no thread to be had: run this share here (no exception leaves the library)
            part();
        }
    }
    for (std::thread& x : th) x.join();
}

// one kernel launch, attributed to the current phase
inline void count_launch(riga_ctx* c) {
    c->prof.launches++;
    c->prof.ph[c->prof.cur].launches++;
}
// RAII phase scope: events around the enclosed launches when profiling is on
struct PhaseScope {
    riga_ctx* c;
    int prev;
    int p;
    cudaEvent_t a = nullptr;
    PhaseScope(riga_ctx* c_, int p_, double bytes = 0.0, double flops = 0.0) : c(c_), prev(c_->prof.cur), p(p_) {
        c->prof.cur = p;
        PhaseRec& r = c->prof.ph[p];
        r.calls++;
        r.bytes += bytes;
        r.flops += flops;
        if (c->prof.on) {
            cudaEventCreate(&a);
            cudaEventRecord(a, c->stream);
        }
    }
    ~PhaseScope() {
        if (c->prof.on && a) {
            cudaEvent_t b;
            cudaEventCreate(&b);
            cudaEventRecord(b, c->stream);
            c->prof.ph[p].ev.push_back({a, b});
        }
        c->prof.cur = prev;
    }
};

// api.cu
int upload_symbolic(riga_ctx* c);  // symbolic arrays of c->S to the device
// assemble.cu
int assemble_device(riga_ctx* c);
int prepare_batch_assembly(riga_ctx* c);  // once per batch pattern
// tc_update.cu: tensor-core Schur updates of FP32 fronts (TF32 or BF16 operands)
int prepare_tc(riga_ctx* c);  // kernel attributes and packing buffers for the current schedule
int enqueue_tc_step(riga_ctx* c, const StepRange& R, int p0, float* pool, int plain, cudaStream_t st);
// oz_update.cu: FP64-accurate Schur updates of FP64 fronts on the tensor cores
int prepare_oz(riga_ctx* c);
int enqueue_oz_step(riga_ctx* c, const StepRange& R, double* pool, int plain, cudaStream_t st);
// factor.cu
int enqueue_factor(riga_ctx* c);  // enqueue numeric LDL^T (no sync)
int finish_factor(riga_ctx* c);   // sync, read flag and inertia
// solve.cu
int enqueue_solve(riga_ctx* c, double* y, int nrhs = 1);  // y := A^{-1} y (nrhs columns, stride N), permuted order
int solve_max_rhs(riga_ctx* c);  // right-hand sides one tree traversal can carry (1, 2 or 4)
int enqueue_spmv(riga_ctx* c, int which, const double* x, double* y, double alpha_shift);
void enqueue_permute(riga_ctx* c, const double* in, double* out, int to_perm, int ncols);
int solve_refined(riga_ctx* c, double* y, double* work_x, double* work_r, double tol, int max_sweeps,
                  int check, int* sweeps_out);
int solve_refined_multi(riga_ctx* c, double* y, double* work_x, double* work_r, int nr, int sweeps);
// lanczos.cu
int run_eigs(riga_ctx* c, int k, double sigma, double tol, int* nconv);
// slicing.cu: every eigenpair in [lo, hi) by spectrum slicing with thick-restart Lanczos
int run_eigs_interval(riga_ctx* c, double lo, double hi, int kmax, double tol, int m_basis, int* nfound,
                      int* basis_cols);
// batch.cu
int run_eigs_batch(riga_ctx* c, int k, double sigma, double tol);
// accuracy.cu: EVerr, EFerr_L2, EFerr_E of the context's first nev eigenpairs
int eig_errors_device(riga_ctx* c, int nev, const int* modes_host, int nq, double* everr, double* efl2, double* efe);
// adjoint.cu
int eig_grad_device(riga_ctx* c, int k, const double* w_dev, double* ga_dev, double* gb_dev);
// tridiag.cpp
void tridiag_eig(int m, const double* alpha, const double* beta, double* theta, double* Z, bool vectors);
void tridiag_eig_rows(int m, const double* alpha, const double* beta, double* theta, int zr, const double* z0,
                      double* Zout);
// band.cpp: symmetric band matrix (dense n x n column-major, half-bandwidth b)
void band_eigvals(int n, int b, const double* T, double* theta);                      // ascending
// eigenvalues and the last r rows of all eigenvectors (Zlast: r x n column-major)
void band_eig_lastrows(int n, int b, const double* T, int r, double* theta, double* Zlast);
void band_eigvecs(int n, int b, const double* T, int q, const double* th, double* S);  // S: n x q
void sym_eig_dense(int n, const double* A, double* theta, double* Z);  // dense symmetric: all eigenpairs

}  // namespace riga
