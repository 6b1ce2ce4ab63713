// Host-side symbolic analysis: B-spline index structure, separator-induced
// nested dissection, assembly tree, fronts and all integer maps the device
// kernels consume.  Integer only; computed once per mesh pattern.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace riga {

// One direction of the tensor-product space (Sec. 3.1 Eq. U, Sec. 3.2).
struct Dir1D {
    int ne = 0, p = 0;
    std::vector<int> mult;      // interior knot multiplicities (ne-1)
    std::vector<int> kv;        // knot vector in element units (value * ne)
    int nfun = 0;               // functions before Dirichlet removal
    int ndof = 0;               // nfun - 2
    std::vector<int> elem_first;  // first non-zero function on element e (pre-Dirichlet)
    std::vector<int> c0;        // C0 DOFs (after Dirichlet removal), ascending
    // adjacency of DOFs: adj_ptr[a]..adj_ptr[a+1] in adj (ascending)
    std::vector<int> adj_ptr, adj;
};

// Factorization work items (precomputed per level and panel step).
struct PanelItem { int front; int r0; };            // TRSM row block of a front
struct TileItem { int front; int i0; int j0; };     // trailing-update tile
struct TileItemL { int front; int i0; int j0; int jend; };  // tile whose columns stop at jend (exclusive)
constexpr int TC_M = 128, TC_N = 128;               // tensor-core update tile (rows x columns)
constexpr int TC_BLK = 128;                          // rows of one packed panel block
// Columns of a super-panel (K of one tensor-core update): 64.  The TF32
// head/tail products accumulate in the FP32 tensor-memory accumulator; at
// K = 128 (48 MMAs per tile) the factor's error let the three calibrated
// refinement sweeps fall short on the Lanczos vectors of the 3D mesh (800
// Lanczos steps instead of 324), at K = 64 (24 MMAs) it does not, and the
// tile traffic is half that of K = 32.
constexpr int TC_KW = 64;
// Tensor-core update of the trailing matrix once per super-panel (up to
// TC_KW / 32 panel steps): the super-panel's columns of the trailing rows are
// packed into 128-row blocks, one packed block per 32-column chunk (operands
// in the MMA's shared-memory layout; the chunks of a row block are
// consecutive block numbers).  A tile reads the nk chunk blocks starting at
// a_blk as its A operand (rows i0..) and at b_blk as its B operand (rows j0..).
struct TcPack { int front; int r0; int blk; int p0; };  // rows r0..r0+127, super-panel columns from p0, chunks from blk
struct TcTile { int front; int i0; int j0; int a_blk; int b_blk; int nk; };
// FP64-accurate tensor-core update (oz_update.cu), one panel step: trailing
// rows packed per 128-row block as 8-bit digit slices; tiles of OZ_M x OZ_N,
// B rows j0.. in half b_half of block b_blk (TcTile.nk holds b_half)
constexpr int OZ_M = 128, OZ_N = 64;
struct ExtItem { int child; int c0; int c1; };      // extend-add columns [c0,c1) of a child

// tree-solve kernel shapes: 256-thread CTAs per item (large fronts),
// 128-thread CTAs (small fronts, few trees), one warp per item (small fronts,
// a batch of many trees)
enum { SOLVE_CTA256 = 0, SOLVE_CTA128 = 1, SOLVE_WARP = 2 };

struct SolveItem {   // one work item of the persistent tree solve
    int front;
    int lo, hi;       // forward: border columns [lo,hi) (front numbering, k <= lo); backward: own rows [lo,hi)
    int ldp;          // panel leading dimension, multiple of 4
    long long off;    // panel offset in the Q pool (elements, multiple of 4)
    // the front's data the item needs, packed so that one load fetches it
    int k, n, b0;     // own / front size, first own position
    int wait_parts;   // backward: forward parts of this front to wait for
    long long upd_off, fpos;  // update-vector offset, index-list offset of the front
    int c0, c1;       // forward: the front's children, records [c0, c1) of Symbolic::crec
    int parent, parent_parts;  // backward: parent front (-1: root) and its backward parts
};

struct ChildRec {    // one child of a front, as the forward solve reads it
    int child;       // child front
    int parts;       // its forward parts (all must be done)
    int m;           // its update-vector length n - k
    int pad;
    long long rel_off, upd_off;  // its relative indices and update vector
};

struct StepRange {   // one panel step of one level
    int s;           // step index (panel columns s*nb .. )
    int d_begin, d_end;   // PanelItem range: one diagonal-block item per active front (r0 = s*nb)
    int p_begin, p_end;   // PanelItem range: row blocks below the diagonal block
    int c_begin, c_end;   // TcTile range of Symbolic::tc_tiles (tensor-core update tiles)
    int k_begin, k_end;   // TcPack range of Symbolic::tc_packs (blocks packed before the update)
    int o_begin, o_end;   // TcPack range of Symbolic::oz_packs (FP64 digit-slice blocks of this step)
    int q_begin, q_end;   // TcTile range of Symbolic::oz_tiles
    int n_begin, n_end;   // TileItem range of Symbolic::tc_narrow: 32x32 tiles of the panel's update
                          // restricted to the columns of its super-panel (tensor-core schedule)
    int t_begin, t_end;   // TileItem range: [t_begin, t_mid) 32x32 tiles, [t_mid, t_end) 16x16 tiles
    int t_mid;
};

struct LevelPlan {
    std::vector<int> nodes;          // nodes of this level
    int max_n = 0, max_k = 0;
    int ext_begin[2], ext_end[2];    // ExtItem ranges per child rank
    std::vector<StepRange> steps;
};

struct Symbolic {
    int dim = 0, p = 0, leaf_extent = 8;
    Dir1D dir[3];
    int n1[3] = {1, 1, 1};
    long long N = 0;

    // elimination order
    std::vector<int> perm;  // perm[pos] = global DOF
    std::vector<int> ipos;  // ipos[g] = pos

    // nodes, post-ordered
    int n_nodes = 0;
    std::vector<int> node_ptr;     // own positions [node_ptr[F], node_ptr[F+1])
    std::vector<int> parent;
    std::vector<int> child_ptr, child_list;  // children in order (left, right)
    std::vector<int> node_of;      // node_of[pos]
    std::vector<int> k, n;         // fully summed / front size (own + border)
    std::vector<int> ld;           // rows of the augmented front: n + k
    std::vector<long long> front_ptr;  // index lists (positions) at front_ptr[F]
    std::vector<int> front_pos;        // own positions then border positions
    std::vector<int> height;
    int n_levels = 0;

    // CSR pattern in elimination order (row = pos, cols = pos ascending)
    std::vector<long long> rowptr;
    std::vector<int> col;
    long long nnz = 0;
    // the same entries in global numbering: csr_perm_to_glob[e] = index of
    // entry e of the permuted CSR inside the global CSR (rows/cols ascending)
    std::vector<long long> glob_rowptr;
    std::vector<long long> perm_to_glob;

    // front pool (column-major, leading dimension ld_F = n_F + k_F)
    std::vector<long long> front_off;
    long long pool_size = 0;
    std::vector<long long> scatter;   // per permuted CSR entry: pool offset or -1 (upper)
    std::vector<int> rel;             // extend-add: local index in parent, per border entry
    std::vector<long long> rel_ptr;   // rel of node F at rel_ptr[F] (length n_F - k_F)
    std::vector<long long> upd_off;   // solve update vector offsets (length n_F - k_F)
    // Tree-solve work items and their packed operator panels.  A front's
    // forward sweep is split into parts by border columns, its backward sweep
    // by own rows; every part has one panel in the Q pool (16-byte aligned):
    //   forward part  [lo,hi) of columns k..n: row-major k x ldp panel of
    //                 -A11^{-1} A12 (ldp = hi-lo rounded up to 4);
    //   backward part [lo,hi) of rows 0..k: column-major ldp x n panel of
    //                 [-A11^{-1} | -A11^{-1} A12] (ldp = hi-lo rounded up to 4).
    std::vector<TcTile> tc_tiles;     // update tiles of TC_M x TC_N for the tensor-core update kernel
    std::vector<TcPack> tc_packs;     // panel blocks packed for it, per step
    std::vector<TileItemL> tc_narrow; // within-super-panel updates (CUDA cores, columns < the super-panel's end)
    std::vector<TcPack> oz_packs;     // FP64 tensor-core schedule: blocks packed per panel step
    std::vector<TcTile> oz_tiles;     //   and its OZ_M x OZ_N tiles
    long long oz_pack_blocks = 0;     //   packed blocks of the largest step
    long long tc_pack_blocks = 0;     // packed blocks of the largest step
    std::vector<SolveItem> sitems;    // forward items (ascending height), then backward (descending)
    std::vector<ChildRec> crec;       // per child_list entry
    int solve_mode = 0;               // SOLVE_CTA256 / SOLVE_CTA128 / SOLVE_WARP (finish_symbolic)
    long long max_panel = 0;          // largest solve-item panel (elements)
    int n_fwd_items = 0;
    std::vector<int> parts_f, parts_b;
    long long q_size = 0;
    std::vector<PanelItem> qitems;    // pack work: (solve item, first element) per 4096 elements
    long long upd_size = 0;

    // factorization schedule
    int nb = 32, tile = 32, rowblk = 64;
    int small_trail = 1024;            // trailing blocks of at most this many rows take 16x16 update tiles
    std::vector<LevelPlan> levels;
    std::vector<PanelItem> pitems;
    std::vector<TileItem> titems;
    std::vector<ExtItem> eitems;

    // element structure (for assembly with coefficients and the adjoint)
    long long n_elem = 0;

    // batch (merged forest of independent problems): per-problem offsets of
    // positions / DOFs, CSR entries, elements and nodes (size problems + 1)
    std::vector<long long> prob_pos, prob_nnz, prob_elem;
    std::vector<int> prob_node;
    std::vector<int> prob_of_pos;   // problem of each position

    long long nnzL = 0;   // factor entries (lower trapezoids of the n x k panels)
    long long nnzQ = 0;   // solve-operator entries (k x n extra-row blocks)
    long long nnzL_own2 = 0;  // sum k^2: the -A11^{-1} part, read only by the backward sweep
    double flops = 0.0;   // LDL^T flops of the fronts
    double flops_aug = 0.0;  // additional flops of the extra rows
};

// Builds everything above.  Returns an empty string on success, else a message.
std::string build_symbolic(Symbolic& S, int dim, const int* ne, int p, const int* const* mult,
                           int leaf_extent);
// Heights, counts, schedule and solve items from nodes, fronts and maps.
std::string finish_symbolic(Symbolic& S);
void build_schedule(Symbolic& S);  // the factorization's level schedule (after finish_symbolic)
// Host check of the alignment and range of every bulk copy of the schedule.
std::string check_bulk_copies(const Symbolic& S, long long* checked);
// Merges independent problems into one forest (dim = 0 marks a batch).
std::string merge_symbolic(Symbolic& M, const std::vector<Symbolic>& P);

}  // namespace riga
