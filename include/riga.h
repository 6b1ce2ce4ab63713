/*
 * riga.h -- C ABI of the GB300 shift-and-invert eigensolver for B-spline (IGA)
 * and refined-IGA (rIGA) discretizations of the Laplace eigenproblem.
 *
 * Problem (Sec. 2.1, Eq. helmholtz / Eq. GHEP of arXiv 2009.08167): find
 * (lambda, u) with K u = lambda M u, K and M the stiffness and mass matrices
 * of a tensor-product B-spline space of degree p on (0,1)^d with homogeneous
 * Dirichlet conditions.  The solution path is the paper's (Sec. 4): an LDL^T
 * factorization of K - sigma M (multifrontal, in the nested-dissection order
 * whose separators are the rIGA C0 hyperplanes of Sec. 3.2), forward/backward
 * solves and M mat-vecs inside a Lanczos iteration in the M-inner product
 * (Eq. LanczosAlphaBeta), Rayleigh-Ritz on T_m (Eq. RitzValues), and the
 * Sylvester inertia of D (Remark on inertia) to place shifts and to confirm
 * that no eigenvalue was missed.
 *
 * Conventions for every entry point
 *  - Return value: RIGA_OK (0) or a negative RIGA_E* code; no exception or
 *    signal crosses the ABI.  riga_strerror() names a code;
 *    riga_last_error() gives a human-readable message for the last failing
 *    call on a context.
 *  - Arrays are owned by the caller.  A pointer argument may address host or
 *    device memory of the context's device; the library detects which.
 *    Device arrays are accessed on the context's stream in stream order; host
 *    arrays are copied synchronously (the call returns after the copy).
 *  - The context owns its internal device allocations (matrices, fronts,
 *    Lanczos basis) until riga_destroy().
 *  - Global DOF numbering is x-fastest: g = i + n_x (j + n_y k), where n_a is
 *    the number of DOFs in direction a after the two Dirichlet functions of
 *    each direction are removed (Eq. dofs).  Element numbering is x-fastest
 *    likewise: e = e_x + ne_x (e_y + ne_y e_z).
 *  - Vectors and matrices of several columns are column-major with leading
 *    dimension N (one eigenvector per column).
 */
#ifndef RIGA_H
#define RIGA_H

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- status */
#define RIGA_OK 0
#define RIGA_EINVAL (-1)   /* bad argument (sizes, NULL pointer, unsupported option) */
#define RIGA_ESTATE (-2)   /* call order (e.g. riga_solve before riga_factor) */
#define RIGA_EPIVOT (-3)   /* zero or non-finite pivot in LDL^T (sigma at an eigenvalue) */
#define RIGA_ENOCONV (-4)  /* Lanczos did not converge; outputs valid for *nconv pairs */
#define RIGA_EREFINE (-5)  /* iterative refinement stagnated above the tolerance */
#define RIGA_ETIMEOUT (-6) /* a bounded device-side wait expired */
#define RIGA_ECUDA (-7)    /* a CUDA runtime call failed */
#define RIGA_ENOMEM (-8)   /* device allocation failed */

/* ---------------------------------------------------- factor precisions */
#define RIGA_FP64 0 /* fronts in FP64 */
#define RIGA_FP32 1 /* fronts in FP32, solves refined to FP64 accuracy */
#define RIGA_TF32 2 /* fronts in FP32, trailing updates on the tensor cores (TF32 head + tail
                       products, about FP32 accuracy), solves refined to FP64 accuracy */
#define RIGA_BF16 3 /* fronts in FP32, trailing updates on the tensor cores with BF16 operands
                       (BF16 head + tail products, FP32 accumulation, every 128-row operand
                       block scaled by a power of two; about 2^-16 relative), solves refined
                       to FP64 accuracy where the refinement converges */

typedef struct riga_ctx riga_ctx;

/*
 * Mesh description (Sec. 3.1 Eq. U, Sec. 3.2): uniform open knot vectors on
 * [0,1] with ne[a] elements in direction a and degree p in every direction.
 * mult[a] points to ne[a]-1 interior knot multiplicities in 1..p (p makes the
 * knot a C0 separator, Fig. 2); NULL means all 1 (maximum continuity C^{p-1}).
 * dirichlet must be 1 (homogeneous Dirichlet on all faces, Eq. helmholtz).
 * leaf_extent bounds the DOF extent of a leaf box of the nested dissection
 * (0 selects 8); see riga_assemble.
 */
typedef struct {
    int dim;         /* 1, 2 or 3 */
    int ne[3];       /* elements per direction, >= 1 */
    int p;           /* degree, 1..6 */
    const int* mult[3];
    int dirichlet;   /* must be 1 */
    int leaf_extent; /* >= 1, or 0 for the default 8 */
} riga_mesh;

/*
 * riga_create: make a context on CUDA device `device` that issues all work on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * stream must outlive the context.  Errors: RIGA_EINVAL, RIGA_ECUDA.
 */
int riga_create(riga_ctx** out, int device, void* cuda_stream);

/*
 * riga_create with device = -1 makes a host-only context: it accepts
 * riga_analyze, riga_query, riga_get_symbolic, riga_strerror and
 * riga_last_error (no CUDA call is made); every other call returns
 * RIGA_ESTATE.
 */

/* riga_destroy: free every device allocation of the context.  NULL is a no-op. */
void riga_destroy(riga_ctx* ctx);

/*
 * riga_assemble: build K and M (Eq. 1Dmatrix, Eq. 2Dmatrix) on the device.
 *  - Symbolic analysis (host, integer, once per mesh pattern): C0 DOFs,
 *    nested-dissection order (separators = C0 hyperplanes first, then p-thick
 *    slabs down to leaf boxes of extent <= max(leaf_extent, p+1)), assembly
 *    tree, fronts, scatter and extend-add maps.  A second call with the same
 *    mesh reuses it and only recomputes values.
 *  - Numeric assembly (device): Cox-de Boor basis and derivatives at p+1
 *    Gauss points per element, 1D element matrices, then CSR values of K and
 *    M in elimination order.
 *  coefK, coefM: NULL for constant coefficients (Kronecker construction of
 *    Eq. 2Dmatrix), else n_elem factors c_e so that K = sum_e coefK[e] K_e and
 *    M = sum_e coefM[e] M_e (either may be NULL = all ones).
 * Errors: RIGA_EINVAL (bad mesh), RIGA_ENOMEM, RIGA_ECUDA.  Invalidates any
 * factorization held by the context.
 */
int riga_assemble(riga_ctx* ctx, const riga_mesh* mesh, const double* coefK, const double* coefM);

/*
 * riga_assemble_log: riga_assemble with per-element LOG-coefficients,
 * K = sum_e exp(logK[e]) K_e and M = sum_e exp(logM[e]) M_e (the
 * parametrisation in which riga_eig_grad differentiates).  The exponentials
 * are taken on the device.  logK, logM: n_elem values each, host or device
 * pointers, NULL = all zeros (unit coefficients).  Errors as riga_assemble;
 * RIGA_EINVAL also when an exponential is zero or not finite.
 */
int riga_assemble_log(riga_ctx* ctx, const riga_mesh* mesh, const double* logK, const double* logM);

/*
 * riga_analyze: the symbolic half of riga_assemble alone (host, integer):
 * C0 DOFs, elimination order, assembly tree and fronts for `mesh`, without
 * touching a device.  Makes riga_query and riga_get_symbolic available.
 * Errors: RIGA_EINVAL (bad mesh).
 */
int riga_analyze(riga_ctx* ctx, const riga_mesh* mesh);

/*
 * riga_factor: numeric LDL^T of A = K - sigma M in the context's elimination
 * order (Sec. 4.2 and its Remark on inertia), 1x1 pivots without pivoting.
 * precision: RIGA_FP64, RIGA_FP32 (fronts stored and updated in FP32; the
 *   assembled A is rounded from FP64), RIGA_BF16 (FP32 fronts whose Schur
 *   updates take BF16 head + tail operands on the tensor cores) or RIGA_TF32 (FP32 fronts whose Schur
 *   updates run on the tensor cores: each operand split into a TF32 head and
 *   tail, three products accumulated in FP32).
 * n_neg (may be NULL): receives the inertia nu(K - sigma M), the number of
 *   negative entries of D = the number of eigenvalues below sigma (Sylvester).
 * Errors: RIGA_ESTATE (no riga_assemble), RIGA_EPIVOT (a zero or non-finite
 * pivot: sigma is at, or numerically indistinguishable from, an eigenvalue),
 * RIGA_EINVAL, RIGA_ECUDA.
 */
int riga_factor(riga_ctx* ctx, double sigma, int precision, long long* n_neg);

/*
 * riga_solve: x = (K - sigma M)^{-1} b for nrhs right-hand sides (columns of
 * length N, x-fastest numbering) with the last factorization: forward
 * elimination, D^{-1}, backward elimination over the assembly tree.  Several
 * columns share one launch (up to 8 as independent interleaved traversals,
 * or, for batches of many problems, up to 4 per work item sharing each
 * operator panel read); the result of a column does not depend on how the
 * columns are grouped.  With an
 * FP32 factor (or tol > 0) the FP64 residual b - (K - sigma M) x drives
 * iterative refinement until ||r||_2 <= tol ||b||_2 (tol <= 0 with an FP32
 * factor selects 1e-13); iters_out (may be NULL) receives the refinement
 * sweeps of the last column.  b and x may alias.  Errors: RIGA_ESTATE,
 * RIGA_EREFINE (no progress, x holds the best iterate), RIGA_EINVAL, RIGA_ECUDA.
 */
int riga_solve(riga_ctx* ctx, const double* b, double* x, int nrhs, double tol, int* iters_out);

/*
 * riga_eigs: the k smallest eigenvalues lambda > sigma of K u = lambda M u
 * and M-orthonormal eigenvectors, by shift-and-invert Lanczos (Sec. 4).
 *  - The first shift is sigma.  When slice > 0 and slice < k, the interval is
 *    covered by spectrum slicing: after each shift's `slice` pairs are
 *    accepted, the next shift is placed midway between the last accepted
 *    eigenvalue and the next Ritz value (Sec. 4.1, Remark on inertia).
 *  - Each shift: factorization at `precision`, Lanczos with full
 *    reorthogonalization against the basis and all locked vectors (the
 *    recurrence plus one classical Gram-Schmidt pass, or two passes: see
 *    riga_set_reorth), Rayleigh-Ritz on T_m, locking of pairs
 *    whose residual estimate is below tol, restarts from a fresh random vector
 *    M-orthogonal to the locked ones until the inertia difference between the
 *    shift and a check shift confirms the count (degenerate eigenvalues).
 *  - evals[k] ascending; evecs (N x k, may be NULL) M-normalised, sign fixed
 *    so that the entry of largest magnitude is positive (lowest index on
 *    ties); resid[k] (may be NULL) the residuals
 *    ||K u - lambda M u||_2 / (|lambda| ||M u||_2) evaluated in FP64.
 *  - nconv (may be NULL): pairs delivered.
 * Errors: RIGA_ESTATE, RIGA_ENOCONV (first *nconv outputs valid), RIGA_EPIVOT,
 * RIGA_EINVAL, RIGA_ECUDA.
 */
int riga_eigs(riga_ctx* ctx, int k, double sigma, double tol, double* evals, double* evecs,
              double* resid, int* nconv);

/*
 * riga_eigs_interval: every eigenpair with lo <= lambda < hi, by dynamic
 * spectrum slicing with thick-restart shift-and-invert Lanczos (Sec. 4.1;
 * Sec. 4.2, Eq. LanczosRestart read as Wu and Simon's thick restart; the
 * Remark on inertia; Sec. 6, Krylov-Schur with spectrum slicing, where the
 * paper computes up to N0 = 4096 pairs).
 *  - The count nu(K - hi M) - nu(K - lo M) comes from two FP64 inertias
 *    (nu = 0 for lo <= 0).  More than kmax: RIGA_EINVAL with *nfound = the
 *    count (allocate and call again).
 *  - Slices of riga_set_eig_options' `slice` pairs (default 50) and `extra`
 *    (default 2): each slice's shift is the previous slice's end, placed in
 *    the first relative gap > 1e-6 after its pairs and certified by inertia.
 *  - m_basis: Lanczos vectors per thick-restart cycle (0 = max(2 (slice +
 *    extra), slice + extra + 40)).  The basis holds at most
 *    2 (slice + extra + 8) + 16 + m_basis + 2 vectors whatever the number of
 *    pairs; *basis_cols (may be NULL) receives that capacity.
 *  - precision (riga_set_eig_options) applies to the run factorizations;
 *    inertias always use FP64 fronts.
 *  - evals[kmax], evecs (N x kmax column-major, may be NULL), resid[kmax]
 *    (may be NULL): host or device, filled with the *nfound pairs ascending,
 *    vectors M-normalised as riga_eigs's.
 *  - lo and hi must not be eigenvalues (zero pivot: RIGA_EPIVOT).
 * Errors: RIGA_EINVAL, RIGA_ESTATE, RIGA_EPIVOT, RIGA_ENOCONV (the pairs of
 * the completed slices are returned), RIGA_ENOMEM, RIGA_ECUDA.
 */
int riga_eigs_interval(riga_ctx* ctx, double lo, double hi, int kmax, double tol, int m_basis, double* evals,
                       double* evecs, double* resid, int* nfound, int* basis_cols);

/*
 * riga_set_eig_options: options of riga_eigs and riga_eigs_batch, kept
 * separate so that their signatures stay short.
 *  slice      eigenpairs accepted per shift (0 = k, a single shift);
 *  precision  RIGA_FP64, RIGA_FP32, RIGA_TF32 or RIGA_BF16 factor inside riga_eigs;
 *  max_steps  Lanczos steps per run (0 = automatic: min(N, max(3 w, w + 40))
 *             for w wanted pairs);
 *  extra      additional pairs computed beyond the wanted ones so that the
 *             completeness check shift can sit in a gap (0 selects 2);
 *  seed       start-vector seed (SplitMix64 stream).
 */
int riga_set_eig_options(riga_ctx* ctx, int slice, int precision, int max_steps, int extra,
                         unsigned long long seed);

/*
 * riga_assemble_batch: assembles nprob independent problems (each a mesh as
 * in riga_assemble, Sec. 2-3; meshes may differ in dim, p, elements and
 * separators) into one context.  Their elimination trees (Sec. 4.2) are merged
 * into a forest: every later factorization processes one tree level of all
 * problems per launch, and one persistent solve serves all of them.
 *  coefK[b], coefM[b] (the arrays themselves and each entry may be NULL):
 *    HOST arrays of per-element coefficients of problem b as in
 *    riga_assemble; NULL selects constant coefficients.
 * The context then holds a batch: riga_eigs and riga_eig_grad answer
 * RIGA_ESTATE, riga_factor factors all problems at one shift (n_neg = the
 * inertia summed over the problems), riga_solve and riga_spmv act on the
 * concatenated vectors (problem b's rows follow problem b-1's), and
 * riga_get_matrices returns the block-diagonal K and M.  A later
 * riga_assemble replaces the batch by a single problem.
 * Errors: RIGA_EINVAL (bad mesh, with its index in riga_last_error),
 * RIGA_ENOMEM, RIGA_ECUDA.
 */
int riga_assemble_batch(riga_ctx* ctx, int nprob, const riga_mesh* meshes, const double* const* coefK,
                        const double* const* coefM);

/*
 * riga_eigs_batch: for every problem of the batch, the k smallest eigenvalues
 * lambda > sigma of K u = lambda M u by shift-and-invert Lanczos (Sec. 4),
 * all problems advancing together: one factorization of the forest, one
 * persistent solve and one M-SpMV per Lanczos step for the whole batch, with
 * each problem's recurrence, reorthogonalisation, Rayleigh-Ritz step, locking
 * and inertia-certified completeness check (its own check shift, in one
 * factorization of the forest with per-problem shifts) kept separate.
 *  evals[nprob * k]: HOST, problem-major, ascending within each problem;
 *    NaN where a problem did not converge.
 *  resid[nprob * k] (may be NULL): HOST, FP64 residuals
 *    ||K u - lambda M u||_2 / (|lambda| ||M u||_2) of the accepted pairs.
 *  nconv[nprob] (may be NULL): HOST, pairs delivered per problem (k or 0).
 * Uses the slice-free options of riga_set_eig_options (precision, max_steps,
 * extra, seed).  precision RIGA_FP32 / RIGA_TF32 / RIGA_BF16: the run
 * factorization's fronts in that precision (per-problem shifts), every
 * Lanczos solve refined to FP64 accuracy with FP64 residuals of each
 * problem's own shifted matrix (the number of sweeps calibrated once per
 * factorization on a seeded right-hand side; FP64 fronts if refinement
 * stalls); the Lanczos recurrence, reorthogonalisation, residuals and the
 * inertia checks stay FP64.
 * Errors: RIGA_ESTATE (no riga_assemble_batch), RIGA_EINVAL (k too large for
 * the smallest problem), RIGA_ENOCONV (outputs of the converged problems
 * valid), RIGA_EPIVOT, RIGA_ENOMEM, RIGA_ECUDA.
 */
int riga_eigs_batch(riga_ctx* ctx, int k, double sigma, double tol, double* evals, double* resid, int* nconv);

/*
 * riga_band_eig: the Rayleigh-Ritz step of block Lanczos on the host (the
 * block form of Eq. LanczosTm and Eq. RitzValues): all eigenvalues of a real
 * symmetric band matrix, and eigenvectors for chosen ones.  Needs no context
 * and no GPU.
 *  T[n*n]: HOST, column-major, symmetric; entries with |i - j| > b are
 *    ignored (taken as zero).  b >= 0 is the half-bandwidth (the Lanczos
 *    block size).
 *  theta[n]: HOST out, all eigenvalues ascending.
 *  which[q]: HOST, indices into theta of the wanted eigenvectors; S[n*q]:
 *    HOST out, column-major, orthonormal eigenvectors (sign unspecified).
 *  r, Zlast[r*n] (r may be 0, then Zlast NULL): HOST out, the last r rows of
 *    ALL eigenvectors, column i for theta[i] (column-major r x n): what the
 *    block Lanczos residual estimates need.
 * Band reduction to tridiagonal form by Givens rotations (tracking the last r
 * rows of the accumulated rotation), implicit QL, and inverse iteration with
 * a pivoted band LU, orthogonalised within clusters.
 * Errors: RIGA_EINVAL (bad sizes or indices).
 */
int riga_band_eig(int n, int b, const double* T, double* theta, int q, const int* which, double* S, int r,
                  double* Zlast);

/*
 * riga_sym_eig: all eigenpairs of a dense symmetric n x n matrix A (host, no
 * context, no GPU): the Rayleigh-Ritz step of thick-restart Lanczos, whose
 * projected matrix (Sec. 4.2, Eq. LanczosRestart read as Wu and Simon's
 * thick restart) is an arrowhead block followed by a tridiagonal one.
 * Householder reduction to tridiagonal form, then the implicit QR iteration.
 *  - A: n x n column-major (only symmetric input is meaningful; both
 *    triangles are read).  theta[n]: eigenvalues ascending.  Z: n x n
 *    column-major, column i the unit eigenvector of theta[i].  All host
 *    arrays owned by the caller.
 * Errors: RIGA_EINVAL (n < 1 or a NULL pointer).
 */
int riga_sym_eig(int n, const double* A, double* theta, double* Z);

/*
 * riga_set_eig_block: Lanczos block size of riga_eigs.  1 (the default) is
 * the single-vector recurrence of Sec. 4.1-4.2; 2 or 4 run block Lanczos:
 * each step applies the shift-inverted operator to a block of vectors with
 * one traversal of the factor (riga_solve's grouping), orthogonalises the
 * block against all previous vectors in the M-inner product (as set by
 * riga_set_reorth) and M-orthonormalises it (shifted Cholesky QR, three
 * passes); the Rayleigh-Ritz step uses the block-tridiagonal T_m
 * (riga_band_eig).
 * Eigenvalues of multiplicity up to the block size appear in one run.  0
 * selects 4.  When a batch's solve kernel cannot carry that many right-hand
 * sides per item, the size falls back to what it can (possibly 1).
 * Errors: RIGA_EINVAL.
 */
int riga_set_eig_block(riga_ctx* ctx, int block);

/*
 * riga_autotune: choose the factorization's update-tile shapes for the
 * assembled pattern (a single problem or a batch) by measurement.  Trailing
 * blocks of at most T rows are updated in 16x16 tiles and larger ones in
 * 32x32 tiles; for T in {0, 128, 256, 512, 1024, 4096} the FP64
 * factorization at sigma = 0 (with the solve operators) is run four times,
 * the last three timed with CUDA events on the ctx's stream, and the T of the
 * smallest median is kept for later factorizations of this pattern (a new
 * pattern starts again from T = 1024, the default).  The tile shape changes
 * no result: every entry's update sums the same products in the same order.
 *  small_trail_out (may be NULL): HOST out, the chosen T.
 *  ms_out[6] (may be NULL): HOST out, the median time for each T in the
 *    order above.
 * On return the ctx holds the FP64 factorization at sigma = 0 (as after
 * riga_factor(ctx, 0, RIGA_FP64, ...)).
 * Errors: RIGA_EINVAL (ctx NULL), RIGA_ESTATE (nothing assembled), and the
 * errors of riga_factor.
 */
int riga_autotune(riga_ctx* ctx, int* small_trail_out, double* ms_out);

/*
 * riga_set_eig_accuracy: how riga_eigs forms the eigenvalues of the pairs it
 * locks (Eq. RitzValues gives lambda = sigma + 1/theta).
 *  rayleigh = 0 (the default): lambda = sigma + 1/theta of the converged Ritz
 *    pair; it carries the rounding of the Lanczos recurrence, about 1e-15
 *    relative for the lowest eigenvalues.
 *  rayleigh = 1: lambda = u^T K u / u^T M u of the Ritz vector u, each sum
 *    (including every row of K u, which cancels heavily for the low
 *    eigenvalues) accumulated in double-double with error-free products;
 *    the error is quadratic in the residual plus the rounding of the stored
 *    u, K and M.  For derivative checks by finite differences at small steps
 *    (an eigenvalue noise delta becomes delta / h).  It costs one pass over
 *    K per locked candidate at several FP64 operations per entry (C2: about
 *    10 ms per 50 pairs).
 * The setting holds for later riga_eigs calls on ctx.
 * Errors: RIGA_EINVAL (ctx NULL, rayleigh not 0 or 1).
 */
int riga_set_eig_accuracy(riga_ctx* ctx, int rayleigh);

/*
 * riga_set_fp64_update: where the Schur-complement updates of FP64 fronts
 * (A22 -= L21 D L21^T of each panel step, Sec. 4.2) run, for every later
 * FP64 factorization on ctx (riga_factor with RIGA_FP64, the factorizations
 * and inertia checks inside riga_eigs, riga_eigs_interval and
 * riga_eigs_batch):
 *  mode = 0: CUDA cores, FP64 fused multiply-adds;
 *  mode = 1 (the default): tensor cores.  The panel operands L21 |D|^(1/2) and
 *    L21 D |D|^(-1/2) (|D|^(1/2) rounded to powers of two per column: exact
 *    scalings that keep the row maxima of the two operands in the same
 *    columns next to near-zero pivots at shifts inside the spectrum) are
 *    scaled by a power of two per row, rounded to 55-bit integers and split
 *    into seven balanced 8-bit digits (BF16); the 28 digit products with
 *    weight above FP64 rounding are accumulated exactly in FP32 tensor
 *    memory and recombined in 64-bit integers (splitting of Ozaki, Ogita,
 *    Oishi and Rump).  The error of an updated entry is about
 *    2^-53 * 32 * 2^(e_i + f_j), where 2^e_i and 2^f_j bound the two
 *    operands' panel rows: the rounding level of FP64 arithmetic, normwise
 *    per row pair instead of per product.
 * FP32, TF32 and BF16 fronts are unaffected.
 * Errors: RIGA_EINVAL (ctx NULL, mode not 0 or 1).
 */
int riga_set_fp64_update(riga_ctx* ctx, int mode);

/*
 * riga_set_reorth: how riga_eigs and riga_eigs_batch orthogonalise each new
 * Lanczos vector (block) against all stored ones, in the M-inner product
 * (Sec. 4.2: orthogonalisation against all previously stored vectors).
 *  passes = 1 (the default): the three-term recurrence with its
 *    coefficients computed against the last two vectors (blocks), then one
 *    classical Gram-Schmidt pass against every stored vector; when that pass
 *    removes more than 100 times the norm that remains, the eigensolution
 *    switches to passes = 2 by itself.
 *  passes = 2: two full classical Gram-Schmidt passes (CGS2) every step
 *    (twice the FP64 work of the orthogonalisation).
 * The setting holds for later riga_eigs / riga_eigs_batch calls on ctx.
 * Errors: RIGA_EINVAL (ctx NULL, passes not 1 or 2).
 */
int riga_set_reorth(riga_ctx* ctx, int passes);

/*
 * riga_eig_errors: errors of the first nev eigenpairs of the last riga_eigs /
 * riga_eigs_interval against the exact eigenpairs of the Laplacian on the
 * unit interval, square or cube (Sec. 2, Eq. exact and Eq. eigerrors; the
 * accuracy study of Sec. 8):
 *   everr[i]    = (lambda_h - lambda) / lambda,
 *   eferr_l2[i] = ||s u_h - u||_{L2}^2,
 *   eferr_e[i]  = a(s u_h - u, s u_h - u) / lambda,
 * with lambda = pi^2 (m_1^2 + .. + m_d^2), u = 2^{d/2} prod_a sin(m_a pi x_a),
 * u_h the M-normalised computed eigenvector and s = sign (u_h, u).  Meaningful
 * for constant coefficients; Eq. Pythagorean (eferr_e = everr + eferr_l2)
 * holds for converged pairs.  Computed on the device: B-spline tables at nq
 * Gauss points per element and direction, one pass over the tensor grid of
 * points per eigenpair for the sign and one for the errors.
 *  - modes: HOST array nev x dim, the 1-based mode index per direction of
 *    eigenpair i at modes[i * dim + a] (x first).  A pair inside a degenerate
 *    eigenspace is compared with the one mode named (the paper compares the
 *    diagonal modes of the square only).
 *  - nq: 0 = p + 6 (u_h is a piecewise polynomial of degree p), at most 16.
 *  - everr, eferr_l2, eferr_e: HOST arrays of nev.
 * Errors: RIGA_EINVAL, RIGA_ESTATE (no eigenpairs; a batch context), RIGA_ECUDA.
 */
int riga_eig_errors(riga_ctx* ctx, int nev, const int* modes, int nq, double* everr, double* eferr_l2,
                    double* eferr_e);

/*
 * riga_eig_grad: gradient of L = sum_i dL_dlambda[i] lambda_i over the k
 * eigenpairs of the last riga_eigs with respect to the log-coefficients a_e,
 * b_e (coefK[e] = exp(a_e), coefM[e] = exp(b_e) of riga_assemble):
 *   dL/da_e =  sum_i w_i coefK[e] u_ie^T K_e u_ie,
 *   dL/db_e = -sum_i w_i lambda_i coefM[e] u_ie^T M_e u_ie,
 * with K_e, M_e the unit-coefficient element matrices (tensor products of 1D
 * element matrices) and u_ie the element's coefficients of eigenvector i.
 * Not in the paper; valid for simple eigenvalues (or symmetric functions of a
 * complete degenerate set).  grad_a, grad_b: n_elem each (either may be NULL).
 * Errors: RIGA_ESTATE (no eigenpairs), RIGA_EINVAL (k larger than computed),
 * RIGA_ECUDA.
 */
int riga_eig_grad(riga_ctx* ctx, int k, const double* dL_dlambda, double* grad_a, double* grad_b);

/*
 * riga_query: sizes of the current problem (any pointer may be NULL):
 * N DOFs, nnz of K (= nnz of M, full symmetric pattern), nnzL entries held by
 * the dense fronts' factor (lower trapezoids incl. diagonal), flops_fact the
 * factorization flop count sum_F sum_{i<k_F} (n_F-i)(n_F-i-1).
 */
int riga_query(riga_ctx* ctx, long long* N, long long* nnz, long long* nnzL, double* flops_fact);

/*
 * riga_get_symbolic: the elimination order and assembly tree (integers,
 * bit-exact comparable).  Query sizes first with all arrays NULL:
 *  n_nodes, total_idx (sum of front sizes).
 *  perm[N]: perm[pos] = global DOF eliminated at position pos;
 *  node_ptr[n_nodes+1]: node F owns positions node_ptr[F]..node_ptr[F+1]-1;
 *  parent[n_nodes]: parent node (-1 for a root), nodes are post-ordered;
 *  front_ptr[n_nodes+1], front_idx[total_idx]: the front of F as global DOFs,
 *  own variables first then the border in elimination order.
 * Host arrays only.  Errors: RIGA_ESTATE, RIGA_EINVAL.
 */
int riga_get_symbolic(riga_ctx* ctx, int* n_nodes, long long* total_idx, int* perm, int* node_ptr,
                      int* parent, long long* front_ptr, int* front_idx);

/*
 * riga_get_matrices: CSR of K and M in global (x-fastest) numbering, rows and
 * columns ascending: row_ptr[N+1], col[nnz], kval[nnz], mval[nnz] (any may be
 * NULL).  Host or device arrays.  Errors: RIGA_ESTATE, RIGA_ECUDA.
 */
int riga_get_matrices(riga_ctx* ctx, long long* row_ptr, int* col, double* kval, double* mval);

/*
 * riga_get_factor: D[N] (in elimination order) of the last factorization and,
 * if L is non-NULL, the dense-front factor: for node F the column-major
 * n_F x k_F block of L (unit diagonal implied, strictly lower part valid)
 * stored at L + Lptr[F] with leading dimension n_F, Lptr[n_nodes+1] the
 * offsets (query with L = NULL first).  Values are converted to double.
 * Host arrays only.  Errors: RIGA_ESTATE, RIGA_ECUDA.
 */
int riga_get_factor(riga_ctx* ctx, double* D, long long* Lptr, double* L);

/*
 * riga_spmv: y = A x with A = M (which = 0), K (1) or K - sigma M (2, sigma of
 * the last factorization), x and y of length N in global numbering, FP64.
 * Host or device arrays.  Errors: RIGA_ESTATE, RIGA_EINVAL, RIGA_ECUDA.
 */
int riga_spmv(riga_ctx* ctx, int which, const double* x, double* y);

/*
 * riga_stats: counters of the last riga_eigs (any may be NULL):
 * n_fact factorizations (N_fa of Table 1), n_solve f/b eliminations (N_fb),
 * n_matvec M mat-vecs (N_mv), lanczos_steps total steps over all runs,
 * t_fact_ms / t_solve_ms device time in factorizations / Lanczos loops.
 */
int riga_stats(riga_ctx* ctx, long long* n_fact, long long* n_solve, long long* n_matvec,
               long long* lanczos_steps, double* t_fact_ms, double* t_lanczos_ms);

/*
 * riga_profile: enable (1) or disable (0) device timing of the library's
 * phases and reset all phase counters (launch counts keep running).  While
 * enabled, every phase invocation is bracketed by CUDA events on the
 * context's stream (a small per-invocation cost).
 */
int riga_profile(riga_ctx* ctx, int enable);

/*
 * riga_profile_get: counters of phase `phase` since the last riga_profile
 * call: 0 assemble, 1 factor (numeric LDL^T), 2 solve (one forward/backward
 * elimination), 3 reorth (Gram-Schmidt passes), 4 spmv (M mat-vec and
 * normalisation), 5 ritz (Ritz-vector GEMM), 6 other.  phase = -1 gives the
 * total kernel launches since riga_create in *launches.  Outputs (any may be
 * NULL): name (static string), launches (kernel launches), calls (phase
 * invocations), ms (summed device time, profiling on), bytes and flops
 * (algorithmic work: factor entries read twice per solve, basis columns read
 * four times per reorthogonalization, and so on).  Synchronizes the stream.
 */
int riga_profile_get(riga_ctx* ctx, int phase, const char** name, long long* launches, long long* calls,
                     double* ms, double* bytes, double* flops);

/*
 * riga_set_wait_limit: budget of every device-side wait, in polls (default
 * 2^24): the dependency waits of the persistent tree solve (polls of about
 * 64 ns: about a second), the pipeline waits of the tensor-core Schur updates
 * and the grid barriers of the block-Lanczos QR (shorter polls).  A wait that
 * exhausts it sets the context's device error word, the kernel returns, and
 * the next host check reports RIGA_ETIMEOUT; the context stays usable.
 * limit >= 0.  Errors: RIGA_EINVAL.
 */
int riga_set_wait_limit(riga_ctx* ctx, long long limit);

/*
 * riga_check_copies: host check (no GPU; a host-only context after
 * riga_analyze works) of every bulk copy the kernels issue for the current
 * schedule: the tree solve's operator panels (cp.async.bulk: 16-byte aligned
 * source, size a multiple of 16 bytes, inside the operator pool) and the
 * tensor-core update's packed panel blocks (block indices inside the packing
 * buffer and belonging to the tile's front and panel step).  *n_checked
 * receives the number of copies and references verified.  The library runs
 * no kernel on a schedule this check would reject (riga_assemble runs it).
 * Errors: RIGA_EINVAL (a violation; riga_last_error names it), RIGA_ESTATE.
 */
int riga_check_copies(riga_ctx* ctx, long long* n_checked);

/*
 * riga_trace_solve: one forward/backward elimination of b (as riga_solve with
 * tol = 0, FP64 or FP32 factor, no refinement) that also records, for each
 * work item of the persistent tree solve (forward parts in ascending tree
 * height, then backward parts in descending height; *n_items of them), four
 * int64 values in trace[4*item ..]: the SM that ran it, the global-timer
 * nanoseconds when it was claimed, when its dependencies were satisfied, and
 * when it completed.  Call with trace = NULL first to get *n_items.
 * trace: host array of 4 *n_items int64; order (may be NULL): host array of
 * *n_items ints receiving the node of each item.
 * Errors: RIGA_ESTATE, RIGA_ETIMEOUT, RIGA_ECUDA.
 */
int riga_trace_solve(riga_ctx* ctx, const double* b, int* n_items, long long* trace, int* order);

/*
 * riga_spmv_dot_noalloc: y = A x and *xy = x^T y for a CSR matrix A, without
 * allocating any device memory.  The paper has no counterpart: this is an
 * allocation-free variant of the SpMV + inner-product kernel of the Lanczos
 * step, for callers that cannot allocate device memory, such as code that
 * runs inside a host framework which owns the whole device-memory budget (a
 * pool or a fixed reservation) and forbids cudaMalloc, or a long-running
 * service that must not grow its device footprint after start-up.
 *  - rowptr[N+1] (int64), col[nnz] (int32, ascending within a row), val[nnz],
 *    x[N], y[N], xy[1]: DEVICE pointers of the CURRENT device, owned by the
 *    caller; 1 <= N <= 2^20.  Every pointer is checked
 *    (cudaPointerGetAttributes) before anything is launched: a host pointer
 *    or memory of another device returns RIGA_EINVAL.  Preconditions the
 *    call cannot check without reading device memory: rowptr[0] = 0,
 *    rowptr non-decreasing, 0 <= col[e] < N for every entry, and col and
 *    val hold rowptr[N] entries.
 *  - The per-block partial sums live in a fixed 512 KiB array in device
 *    memory that every GPU which loads this library holds until the process
 *    exits.  The first call on a device looks that array's address up
 *    (cudaGetSymbolAddress, with the device current) and caches it: make the
 *    first call on each device before any stream capture.  The cached
 *    address is valid for the lifetime of the device's primary context; do
 *    not call this function again after cudaDeviceReset in the same process.
 *  - Every call uses the same array, which keeps the last call's contents;
 *    nothing in it has to start at zero (each call writes every entry it
 *    reads).  Calls that overlap on the GPU (other streams, or host threads
 *    without ordering between them) race on it.
 *  - Work is enqueued on cuda_stream (NULL = legacy default stream); the call
 *    returns without synchronizing.
 * Errors: RIGA_EINVAL (NULL pointer, a pointer that is not device memory of
 * the current device, N < 1 or N > 2^20), RIGA_ECUDA.
 */
int riga_spmv_dot_noalloc(const long long* rowptr, const int* col, const double* val, long long N,
                          const double* x, double* y, double* xy, void* cuda_stream);

/* riga_strerror: static name of a status code. */
const char* riga_strerror(int status);

/* riga_last_error: message of the last failing call on ctx ("" if none). */
const char* riga_last_error(riga_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RIGA_H */
