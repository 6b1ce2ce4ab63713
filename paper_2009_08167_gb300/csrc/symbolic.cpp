// Host symbolic analysis (integer only, once per mesh pattern).
//
// * Knot vectors in element units and C0 DOFs (Sec. 3.1 Eq. U, Sec. 3.2).
// * Nested dissection whose first cuts are the rIGA C0 hyperplanes and whose
//   remaining cuts are p-thick slabs (a reading of the "blocks first, then
//   separators" cost model of Sec. 5.1 Eq. flopsFact; the paper itself orders
//   with METIS, Sec. 6).  Rule, per box of DOF intervals [lo,hi):
//     leaf        if every extent <= max(leaf_extent, p+1);
//     C0 cut      else if a direction has a C0 DOF c with lo < c < hi-1: the
//                 direction of largest extent among those (lowest axis on
//                 ties), the c minimising |2c-(lo+hi-1)| (lower c on ties),
//                 separator [c, c+1);
//     p-thick cut else: direction of largest extent (lowest axis on ties),
//                 separator [s, s+p), s = lo + floor((hi-lo-p)/2).
//   Post-order: left subtree, right subtree, separator; DOFs inside a node
//   ascending in global (x-fastest) numbering.
// * Multifrontal structure: each node's front = own DOFs + border (later DOFs
//   adjacent to the node's DOFs or in a child's border), scatter map of A's
//   lower entries into fronts, extend-add maps, solve update offsets, and the
//   per-level panel/tile work lists of the blocked partial LDL^T.
#include "symbolic.h"

#include <algorithm>
#include <cstdio>
#include <functional>

namespace riga {

static std::string build_dir(Dir1D& D, int ne, int p, const int* mult) {
    if (ne < 1) return "ne must be >= 1";
    D.ne = ne;
    D.p = p;
    D.mult.assign(ne > 1 ? ne - 1 : 0, 1);
    if (mult) {
        for (int i = 0; i < ne - 1; ++i) {
            if (mult[i] < 1 || mult[i] > p) return "knot multiplicity outside 1..p";
            D.mult[i] = mult[i];
        }
    }
    D.kv.clear();
    for (int i = 0; i <= p; ++i) D.kv.push_back(0);
    for (int t = 1; t < ne; ++t)
        for (int m = 0; m < D.mult[t - 1]; ++m) D.kv.push_back(t);
    for (int i = 0; i <= p; ++i) D.kv.push_back(ne);
    D.nfun = (int)D.kv.size() - p - 1;
    D.ndof = D.nfun - 2;
    if (D.ndof < 1) return "fewer than one interior DOF in a direction";
    // first non-zero function on each element: the span index sp with
    // kv[sp] <= e < kv[sp+1], minus p
    D.elem_first.assign(ne, 0);
    for (int e = 0; e < ne; ++e) {
        int sp = -1;
        for (int i = 0; i + 1 < (int)D.kv.size(); ++i)
            if (D.kv[i] <= e && e < D.kv[i + 1]) sp = i;
        if (sp < p) return "internal: bad span";
        D.elem_first[e] = sp - p;
    }
    // C0 DOFs: the function B_{s-1}, s the first occurrence of a knot of
    // multiplicity p; after removing function 0 its DOF index is s-2
    D.c0.clear();
    for (int t = 1; t < ne; ++t) {
        if (D.mult[t - 1] != p) continue;
        int s = -1;
        for (int i = 0; i < (int)D.kv.size(); ++i)
            if (D.kv[i] == t) { s = i; break; }
        D.c0.push_back(s - 2);
    }
    // DOF adjacency: supports [kv[f], kv[f+p+1]) share an element
    D.adj_ptr.assign(D.ndof + 1, 0);
    D.adj.clear();
    for (int a = 0; a < D.ndof; ++a) {
        int f = a + 1;
        for (int b = std::max(0, a - p); b <= std::min(D.ndof - 1, a + p); ++b) {
            int g = b + 1;
            int lo = std::max(D.kv[f], D.kv[g]);
            int hi = std::min(D.kv[f + p + 1], D.kv[g + p + 1]);
            if (lo < hi) D.adj.push_back(b);
        }
        D.adj_ptr[a + 1] = (int)D.adj.size();
    }
    return "";
}

namespace {
struct Box {
    int lo[3], hi[3];
};
}  // namespace


// Heights, counts, factorization schedule and tree-solve items of a
// (possibly merged) symbolic structure whose nodes, fronts and maps are set.
std::string finish_symbolic(Symbolic& S) {
    const int F = S.n_nodes;
    // heights and counts
    S.height.assign(F, 0);
    int maxh = 0;
    for (int f = 0; f < F; ++f) {
        int h = 0;
        for (int ci = S.child_ptr[f]; ci < S.child_ptr[f + 1]; ++ci)
            h = std::max(h, S.height[S.child_list[ci]] + 1);
        S.height[f] = h;
        maxh = std::max(maxh, h);
    }
    S.n_levels = maxh + 1;
    S.nnzL = 0;
    S.nnzQ = 0;
    S.nnzL_own2 = 0;
    S.flops = 0.0;
    S.flops_aug = 0.0;
    for (int f = 0; f < F; ++f) {
        long long kk = S.k[f], nn = S.n[f];
        S.nnzL += kk * (kk + 1) / 2 + kk * (nn - kk);
        S.nnzQ += kk * nn;
        S.nnzL_own2 += kk * kk;
        for (long long i = 0; i < kk; ++i) {
            S.flops += (double)(nn - i) * (double)(nn - i - 1);
            S.flops_aug += (double)(nn + kk - i) * (double)(nn + kk - i - 1) - (double)(nn - i) * (double)(nn - i - 1);
        }
    }

    // ------------------------------------------------------- solve items
    // Parts of about part_fma multiply-adds each (at most 32 per sweep for 2D
    // trees, 256 for large fronts), of at
    // most 8 outputs per thread of the solve CTA (4 per lane for the warp
    // kernel).  When every front has at most SMALL_MAX_N variables (2D
    // meshes), parts are smaller, so that the fronts near the root (the
    // critical path of the solve) spread over more SMs and each part's panel
    // fits one shared-memory copy; a forest of many such trees (a batch) is
    // solved one warp per item.
    const int SMALL_MAX_N = 1536;
    int max_n = 0;
    for (int f = 0; f < F; ++f) max_n = std::max(max_n, S.n[f]);
    int n_trees = 0;
    for (int f = 0; f < F; ++f) n_trees += S.parent[f] < 0;
    S.solve_mode = max_n > SMALL_MAX_N ? SOLVE_CTA256 : (n_trees >= 16 ? SOLVE_WARP : SOLVE_CTA128);
    const bool warp = S.solve_mode == SOLVE_WARP;
    const long long part_fma = S.solve_mode == SOLVE_CTA256 ? 12288 : 4096;
    const long long max_width = warp ? 128 : (S.solve_mode == SOLVE_CTA128 ? 8 * 128 : 8 * 256);
    // split `len` outputs into at least `want` parts of at most max_width
    // (warp kernel: widths a multiple of 32 except the last)
    auto split = [&](long long len, long long want) -> long long {
        long long P = std::max({1LL, want, (len + max_width - 1) / max_width});
        if (warp && len > 32) {
            const long long wdt = ((len + P - 1) / P + 31) / 32 * 32;
            P = (len + wdt - 1) / wdt;
        }
        return P;
    };
    // Large fronts (3D) near the root take up to 256 parts, so that the top
    // separators of the tree spread over every SM; each part also gathers its
    // front's vector (n values, plus the children's update vectors going
    // forward), so a part keeps at least two multiply-adds per gathered value.
    const bool large = S.solve_mode == SOLVE_CTA256;
    const long long max_parts = large ? 256 : 32;
    S.parts_f.assign(F, 1);
    S.parts_b.assign(F, 1);
    for (int f = 0; f < F; ++f) {
        const long long kk = S.k[f], mm = S.n[f] - S.k[f], nn = S.n[f];
        long long gat_f = nn;
        for (int ci = S.child_ptr[f]; ci < S.child_ptr[f + 1]; ++ci) {
            const int c = S.child_list[ci];
            gat_f += S.n[c] - S.k[c];
        }
        const long long unit_f = large ? std::max(part_fma, 2 * gat_f) : part_fma;
        const long long unit_b = large ? std::max(part_fma, 2 * nn) : part_fma;
        long long pf = (kk * mm + unit_f - 1) / unit_f;
        pf = std::max(1LL, std::min({pf, max_parts, std::max(1LL, mm)}));
        pf = split(mm, pf);
        long long pb = (kk * nn + unit_b - 1) / unit_b;
        pb = std::max(1LL, std::min({pb, max_parts, std::max(1LL, kk / 8)}));
        pb = split(kk, pb);
        if (pf > 4 * max_parts || pb > 4 * max_parts) return "front too large for the tree solve";
        S.parts_f[f] = (int)pf;
        S.parts_b[f] = (int)pb;
    }
    // part q of P over len outputs: [bound(q), bound(q+1))
    auto bound = [&](long long len, long long P, long long q) -> int {
        if (warp && len > 32) {
            const long long wdt = ((len + P - 1) / P + 31) / 32 * 32;
            return (int)std::min(len, wdt * q);
        }
        return (int)(len * q / P);
    };
    S.crec.resize(S.child_list.size());
    for (int f = 0; f < F; ++f)
        for (int ci = S.child_ptr[f]; ci < S.child_ptr[f + 1]; ++ci) {
            const int c = S.child_list[ci];
            S.crec[ci] = ChildRec{c, S.parts_f[c], S.n[c] - S.k[c], 0, S.rel_ptr[c], S.upd_off[c]};
        }
    {
        std::vector<int> byh(F);
        for (int f = 0; f < F; ++f) byh[f] = f;
        std::stable_sort(byh.begin(), byh.end(), [&](int a, int b) { return S.height[a] < S.height[b]; });
        S.sitems.clear();
        S.qitems.clear();
        S.max_panel = 0;
        long long off = 0;
        auto add = [&](int f, int lo, int hi, long long elems_per_ld_unit) {
            SolveItem it{};
            it.front = f;
            it.lo = lo;
            it.hi = hi;
            it.ldp = std::max(4, (hi - lo + 3) / 4 * 4);
            it.off = off;
            it.k = S.k[f];
            it.n = S.n[f];
            it.b0 = S.node_ptr[f];
            it.wait_parts = S.parts_f[f];
            it.upd_off = S.upd_off[f];
            it.fpos = S.front_ptr[f];
            it.c0 = S.child_ptr[f];
            it.c1 = S.child_ptr[f + 1];
            it.parent = S.parent[f];
            it.parent_parts = S.parent[f] >= 0 ? S.parts_b[S.parent[f]] : 0;
            const long long cnt = (long long)it.ldp * elems_per_ld_unit;
            S.max_panel = std::max(S.max_panel, cnt);
            const int idx = (int)S.sitems.size();
            for (long long e0 = 0; e0 < cnt; e0 += 4096) S.qitems.push_back({idx, (int)e0});
            off += cnt;
            S.sitems.push_back(it);
        };
        for (int f : byh) {  // forward, ascending height
            const int kk = S.k[f], mm = S.n[f] - S.k[f], P = S.parts_f[f];
            for (int q = 0; q < P; ++q) add(f, kk + bound(mm, P, q), kk + bound(mm, P, q + 1), kk);
        }
        S.n_fwd_items = (int)S.sitems.size();
        for (int i = F - 1; i >= 0; --i) {  // backward, descending height
            const int f = byh[i], kk = S.k[f], P = S.parts_b[f];
            for (int q = 0; q < P; ++q) add(f, bound(kk, P, q), bound(kk, P, q + 1), S.n[f]);
        }
        S.q_size = off;
    }

    build_schedule(S);
    return "";
}

// Host check of every bulk copy the kernels will issue for this schedule
// (cp.async.bulk wants 16-byte aligned source and destination and a size
// that is a multiple of 16 bytes, for 4- and 8-byte elements alike):
//  - tree solve: each work item's panel starts at element it.off of the Q
//    pool and is copied in chunks of whole ldp-element rows/columns: off and
//    ldp must be multiples of 4 and the panel (ldp x units) must end inside
//    the pool (q_size elements);
//  - tensor-core update: every packed block index of a step lies below the
//    packing buffer's block count, every tile's blocks belong to its front
//    and step, and the front rows it covers start inside the front.
// Returns "" or a description of the first violation; *checked counts the
// copies (and tile references) verified.
std::string check_bulk_copies(const Symbolic& S, long long* checked) {
    long long n = 0;
    for (size_t i = 0; i < S.sitems.size(); ++i) {
        const SolveItem& it = S.sitems[i];
        const bool fwd = (int)i < S.n_fwd_items;
        const long long units = fwd ? it.k : it.n;
        if (it.off % 4 != 0 || it.ldp % 4 != 0 || it.ldp < it.hi - it.lo)
            return "solve item " + std::to_string(i) + ": panel offset or width not a multiple of 4 elements";
        if (it.off < 0 || it.off + (long long)it.ldp * units > S.q_size)
            return "solve item " + std::to_string(i) + ": panel outside the operator pool";
        ++n;
    }
    for (const LevelPlan& P : S.levels)
        for (const StepRange& R : P.steps) {
            std::vector<int> blk_front;
            for (int q = R.k_begin; q < R.k_end; ++q) {
                const TcPack& pk = S.tc_packs[q];
                const int kw = std::min(TC_KW, S.k[pk.front] - pk.p0);
                const int nk = (kw + 31) / 32;
                if (kw <= 0 || pk.blk < 0 || pk.blk + nk > S.tc_pack_blocks || pk.r0 < 0 || pk.r0 >= S.ld[pk.front])
                    return "tensor-core pack item " + std::to_string(q) + " out of range";
                if ((int)blk_front.size() < pk.blk + nk) blk_front.resize(pk.blk + nk, -1);
                for (int cidx = 0; cidx < nk; ++cidx) blk_front[pk.blk + cidx] = pk.front;
                ++n;
            }
            for (int t = R.c_begin; t < R.c_end; ++t) {
                const TcTile& tl = S.tc_tiles[t];
                const int nb = (int)blk_front.size();
                if (tl.nk < 1 || tl.nk > TC_KW / 32 || tl.a_blk < 0 || tl.b_blk < 0 || tl.a_blk + tl.nk > nb ||
                    tl.b_blk + tl.nk > nb || tl.i0 >= S.ld[tl.front] || tl.j0 >= S.ld[tl.front])
                    return "tensor-core tile " + std::to_string(t) + " references blocks out of range";
                for (int cidx = 0; cidx < tl.nk; ++cidx)
                    if (blk_front[tl.a_blk + cidx] != tl.front || blk_front[tl.b_blk + cidx] != tl.front)
                        return "tensor-core tile " + std::to_string(t) + " references a block of another front or step";
                ++n;
            }
        }
    for (const LevelPlan& P : S.levels)
        for (const StepRange& R : P.steps) {
            std::vector<int> blk_front;
            for (int q = R.o_begin; q < R.o_end; ++q) {
                const TcPack& pk = S.oz_packs[q];
                if (pk.blk < 0 || pk.blk >= S.oz_pack_blocks || pk.r0 < 0 || pk.r0 >= S.ld[pk.front])
                    return "FP64 tensor-core pack item " + std::to_string(q) + " out of range";
                if ((int)blk_front.size() <= pk.blk) blk_front.resize(pk.blk + 1, -1);
                blk_front[pk.blk] = pk.front;
                ++n;
            }
            for (int t = R.q_begin; t < R.q_end; ++t) {
                const TcTile& tl = S.oz_tiles[t];
                const int nb = (int)blk_front.size();
                if (tl.a_blk < 0 || tl.b_blk < 0 || tl.a_blk >= nb || tl.b_blk >= nb || tl.nk < 0 || tl.nk > 1 ||
                    blk_front[tl.a_blk] != tl.front || blk_front[tl.b_blk] != tl.front || tl.i0 >= S.ld[tl.front] ||
                    tl.j0 >= S.ld[tl.front])
                    return "FP64 tensor-core tile " + std::to_string(t) + " references a block of another front or step";
                ++n;
            }
        }
    if (checked) *checked = n;
    return "";
}

// Level schedule of the blocked partial LDL^T: per tree level the extend-add
// items, and per panel step the diagonal-block, row-block and trailing-update
// tile items (the update tiles' shape follows S.small_trail).
void build_schedule(Symbolic& S) {
    const int F = S.n_nodes;
    S.levels.assign(S.n_levels, LevelPlan());
    for (int f = 0; f < F; ++f) S.levels[S.height[f]].nodes.push_back(f);
    S.pitems.clear();
    S.titems.clear();
    S.tc_tiles.clear();
    S.tc_packs.clear();
    S.tc_narrow.clear();
    S.tc_pack_blocks = 0;
    S.oz_packs.clear();
    S.oz_tiles.clear();
    S.oz_pack_blocks = 0;
    S.eitems.clear();
    const int nb = S.nb, tile = S.tile, rb = S.rowblk;
    const int SMALL_TRAIL = S.small_trail;
    const int ext_cols = 32;
    for (int l = 0; l < S.n_levels; ++l) {
        LevelPlan& P = S.levels[l];
        for (int f : P.nodes) {
            P.max_n = std::max(P.max_n, S.n[f]);
            P.max_k = std::max(P.max_k, S.k[f]);
        }
        for (int rank = 0; rank < 2; ++rank) {
            P.ext_begin[rank] = (int)S.eitems.size();
            for (int f : P.nodes) {
                int nc = S.child_ptr[f + 1] - S.child_ptr[f];
                if (rank >= nc) continue;
                int c = S.child_list[S.child_ptr[f] + rank];
                int m = S.n[c] - S.k[c];
                for (int c0 = 0; c0 < m; c0 += ext_cols)
                    S.eitems.push_back({c, c0, std::min(m, c0 + ext_cols)});
            }
            P.ext_end[rank] = (int)S.eitems.size();
        }
        for (int s = 0; s * nb < P.max_k; ++s) {
            StepRange R;
            R.s = s;
            R.d_begin = (int)S.pitems.size();
            for (int f : P.nodes)
                if (S.k[f] > s * nb) S.pitems.push_back({f, s * nb});
            R.d_end = (int)S.pitems.size();
            R.p_begin = (int)S.pitems.size();
            // Rows and columns of the augmented front beyond n + c0 (c0 = the
            // end of the panel) are extra rows of pivots after the panel:
            // they start as identity rows and stay exactly zero in every
            // column before their own pivot, so the panel's row solve and
            // trailing update skip them (their products are exact zeros)
            for (int f : P.nodes) {
                int kf = S.k[f], nf = S.n[f], lf = S.ld[f];
                if (kf <= s * nb) continue;
                int kb = std::min(nb, kf - s * nb);
                const int le = std::min(lf, nf + s * nb + kb);
                for (int r0 = s * nb + kb; r0 < le; r0 += rb) S.pitems.push_back({f, r0});
            }
            R.p_end = (int)S.pitems.size();
            // trailing update: lower tiles of the augmented front, plus the
            // upper tiles of the extra x extra block so that -A11^{-1} is
            // stored in full.  Trailing blocks of at most S.small_trail rows
            // take 16x16 tiles (less padding on the diagonal and the edges of
            // small fronts), larger ones 32x32 tiles.
            R.t_begin = (int)S.titems.size();
            for (int pass = 0; pass < 2; ++pass) {
                if (pass == 1) R.t_mid = (int)S.titems.size();
                for (int f : P.nodes) {
                    int kf = S.k[f], nf = S.n[f], lf = S.ld[f];
                    if (kf <= s * nb) continue;
                    const int c0 = s * nb + std::min(nb, kf - s * nb);
                    const int le = std::min(lf, nf + c0);
                    const int tl = (le - c0 <= SMALL_TRAIL) ? 16 : tile;
                    if ((pass == 0) != (tl == tile)) continue;
                    const int T = (le - c0 + tl - 1) / tl;
                    for (int bi = 0; bi < T; ++bi)
                        for (int bj = 0; bj < T; ++bj) {
                            int i0 = c0 + bi * tl, j0 = c0 + bj * tl;
                            bool lower = bj <= bi;
                            bool extra_upper = (i0 + tl > nf) && (j0 + tl > nf);
                            if (lower || extra_upper) S.titems.push_back({f, i0, j0});
                        }
                }
            }
            R.t_end = (int)S.titems.size();
            // the tensor-core schedule of the same step.  Super-panels of
            // TC_KW columns: a step that does not end its front's current
            // super-panel updates only the super-panel's remaining columns
            // (all rows below them), on 32x32 CUDA-core tiles; the step that
            // ends it updates everything to the right of the super-panel at
            // once, K = its width, in TC_M x TC_N tensor-core tiles over packed
            // 128-row blocks (one per 32-column chunk of the super-panel)
            R.n_begin = (int)S.tc_narrow.size();
            R.k_begin = (int)S.tc_packs.size();
            R.c_begin = (int)S.tc_tiles.size();
            int nblk_step = 0;
            for (int f : P.nodes) {
                int kf = S.k[f], nf = S.n[f], lf = S.ld[f];
                if (kf <= s * nb) continue;
                const int c0 = s * nb + std::min(nb, kf - s * nb);
                const int le = std::min(lf, nf + c0);
                const int S0 = (s * nb) / TC_KW * TC_KW, S1 = std::min(S0 + TC_KW, kf);
                if (c0 < S1) {
                    // narrow update: columns [c0, S1), rows j0..le
                    for (int j0 = c0; j0 < S1; j0 += nb)
                        for (int i0 = j0; i0 < le; i0 += nb) S.tc_narrow.push_back({f, i0, j0, S1});
                    continue;
                }
                const int nk = (S1 - S0 + nb - 1) / nb;
                const int blk0 = nblk_step;
                for (int r0 = c0; r0 < le; r0 += TC_BLK) {
                    S.tc_packs.push_back({f, r0, nblk_step, S0});
                    nblk_step += nk;
                }
                for (int i0 = c0, bi = 0; i0 < le; i0 += TC_M, ++bi)
                    for (int j0 = c0, bj = 0; j0 < le; j0 += TC_N, ++bj) {
                        const bool lower = j0 <= i0;
                        const bool extra = (i0 + TC_M > nf) && (j0 + TC_N > nf);
                        if (lower || extra) S.tc_tiles.push_back({f, i0, j0, blk0 + bi * nk, blk0 + bj * nk, nk});
                    }
            }
            S.tc_pack_blocks = std::max<long long>(S.tc_pack_blocks, nblk_step);
            R.n_end = (int)S.tc_narrow.size();
            // the FP64 tensor-core schedule of the step (K = 32, the panel):
            // digit-slice blocks of the trailing rows, lower 128 x 64 tiles
            // plus those of the extra x extra block
            R.o_begin = (int)S.oz_packs.size();
            R.q_begin = (int)S.oz_tiles.size();
            int oblk = 0;
            for (int f : P.nodes) {
                int kf = S.k[f], nf = S.n[f], lf = S.ld[f];
                if (kf <= s * nb) continue;
                const int c0 = s * nb + std::min(nb, kf - s * nb);
                const int le = std::min(lf, nf + c0);
                const int blk0 = oblk;
                for (int r0 = c0; r0 < le; r0 += TC_BLK) S.oz_packs.push_back({f, r0, oblk++, s * nb});
                for (int i0 = c0; i0 < le; i0 += OZ_M)
                    for (int j0 = c0; j0 < le; j0 += OZ_N) {
                        const bool lower = j0 <= i0 + OZ_M - 1;
                        const bool extra = (i0 + OZ_M > nf) && (j0 + OZ_N > nf);
                        if (!(lower || extra)) continue;
                        const int bj = (j0 - c0) / TC_BLK, half = ((j0 - c0) % TC_BLK) / OZ_N;
                        S.oz_tiles.push_back({f, i0, j0, blk0 + (i0 - c0) / TC_BLK, blk0 + bj, half});
                    }
            }
            S.oz_pack_blocks = std::max<long long>(S.oz_pack_blocks, oblk);
            R.o_end = (int)S.oz_packs.size();
            R.q_end = (int)S.oz_tiles.size();
            R.k_end = (int)S.tc_packs.size();
            R.c_end = (int)S.tc_tiles.size();
            P.steps.push_back(R);
        }
    }
}

std::string build_symbolic(Symbolic& S, int dim, const int* ne, int p, const int* const* mult,
                           int leaf_extent) {
    if (dim < 1 || dim > 3) return "dim must be 1, 2 or 3";
    if (p < 1 || p > 6) return "p must be in 1..6";
    S = Symbolic();
    S.dim = dim;
    S.p = p;
    S.leaf_extent = leaf_extent > 0 ? leaf_extent : 8;
    S.N = 1;
    S.n_elem = 1;
    for (int a = 0; a < 3; ++a) S.n1[a] = 1;
    for (int a = 0; a < dim; ++a) {
        std::string err = build_dir(S.dir[a], ne[a], p, mult ? mult[a] : nullptr);
        if (!err.empty()) return err;
        S.n1[a] = S.dir[a].ndof;
        S.N *= S.n1[a];
        S.n_elem *= ne[a];
    }
    if (S.N > 2000000000LL) return "problem too large for 32-bit DOF indices";
    const int N = (int)S.N;
    const int nx = S.n1[0], ny = S.n1[1];

    // ------------------------------------------------------------ dissection
    std::vector<std::vector<int>> own;
    std::vector<std::vector<int>> kids;
    const int limit = std::max(S.leaf_extent, p + 1);
    auto box_vars = [&](const Box& b) {
        std::vector<int> v;
        for (int z = b.lo[2]; z < b.hi[2]; ++z)
            for (int y = b.lo[1]; y < b.hi[1]; ++y)
                for (int x = b.lo[0]; x < b.hi[0]; ++x) v.push_back(x + nx * (y + ny * z));
        return v;
    };
    std::function<int(const Box&)> rec = [&](const Box& b) -> int {
        int ext[3], maxext = 0;
        for (int a = 0; a < 3; ++a) {
            ext[a] = b.hi[a] - b.lo[a];
            if (a < dim) maxext = std::max(maxext, ext[a]);
        }
        if (maxext <= limit) {
            own.push_back(box_vars(b));
            kids.push_back({});
            return (int)own.size() - 1;
        }
        int axis = -1;
        for (int a = 0; a < dim; ++a) {
            bool has = false;
            for (int c : S.dir[a].c0)
                if (b.lo[a] < c && c < b.hi[a] - 1) has = true;
            if (has && (axis < 0 || ext[a] > ext[axis])) axis = a;
        }
        int s, t;
        if (axis >= 0) {
            const int lo = b.lo[axis], hi = b.hi[axis];
            int best = -1;
            long long bestd = 0;
            for (int c : S.dir[axis].c0) {
                if (!(lo < c && c < hi - 1)) continue;
                long long d = std::llabs(2LL * c - (lo + hi - 1));
                if (best < 0 || d < bestd) { best = c; bestd = d; }
            }
            s = best;
            t = best + 1;
        } else {
            axis = 0;
            for (int a = 1; a < dim; ++a)
                if (ext[a] > ext[axis]) axis = a;
            s = b.lo[axis] + (ext[axis] - p) / 2;
            t = s + p;
        }
        Box L = b, R = b, Sep = b;
        L.hi[axis] = s;
        R.lo[axis] = t;
        Sep.lo[axis] = s;
        Sep.hi[axis] = t;
        int l = rec(L);
        int r = rec(R);
        own.push_back(box_vars(Sep));
        kids.push_back({l, r});
        return (int)own.size() - 1;
    };
    Box root;
    for (int a = 0; a < 3; ++a) {
        root.lo[a] = 0;
        root.hi[a] = S.n1[a];
    }
    rec(root);

    const int F = (int)own.size();
    S.n_nodes = F;
    S.node_ptr.assign(F + 1, 0);
    S.perm.clear();
    S.perm.reserve(N);
    for (int f = 0; f < F; ++f) {
        S.node_ptr[f] = (int)S.perm.size();
        for (int g : own[f]) S.perm.push_back(g);
    }
    S.node_ptr[F] = (int)S.perm.size();
    if ((int)S.perm.size() != N) return "internal: dissection does not cover all DOFs";
    S.ipos.assign(N, -1);
    for (int i = 0; i < N; ++i) S.ipos[S.perm[i]] = i;
    for (int g = 0; g < N; ++g)
        if (S.ipos[g] < 0) return "internal: dissection repeats a DOF";
    S.node_of.assign(N, 0);
    for (int f = 0; f < F; ++f)
        for (int i = S.node_ptr[f]; i < S.node_ptr[f + 1]; ++i) S.node_of[i] = f;
    S.parent.assign(F, -1);
    S.child_ptr.assign(F + 1, 0);
    S.child_list.clear();
    for (int f = 0; f < F; ++f) {
        S.child_ptr[f] = (int)S.child_list.size();
        for (int c : kids[f]) {
            S.child_list.push_back(c);
            S.parent[c] = f;
        }
    }
    S.child_ptr[F] = (int)S.child_list.size();

    // ------------------------------------------------------- CSR patterns
    // global numbering first (rows and columns ascending)
    S.glob_rowptr.assign(N + 1, 0);
    std::vector<int> gcol;
    gcol.reserve((size_t)N * 27);
    {
        const Dir1D& X = S.dir[0];
        for (int g = 0; g < N; ++g) {
            int ix = g % nx, rem = g / nx;
            int iy = dim > 1 ? rem % ny : 0;
            int iz = dim > 2 ? rem / ny : 0;
            int zb = 0, ze = 1, yb = 0, ye = 1;
            const int* zadj = nullptr;
            const int* yadj = nullptr;
            if (dim > 2) { zb = S.dir[2].adj_ptr[iz]; ze = S.dir[2].adj_ptr[iz + 1]; zadj = S.dir[2].adj.data(); }
            if (dim > 1) { yb = S.dir[1].adj_ptr[iy]; ye = S.dir[1].adj_ptr[iy + 1]; yadj = S.dir[1].adj.data(); }
            for (int zz = zb; zz < ze; ++zz) {
                int jz = zadj ? zadj[zz] : 0;
                for (int yy = yb; yy < ye; ++yy) {
                    int jy = yadj ? yadj[yy] : 0;
                    for (int xx = X.adj_ptr[ix]; xx < X.adj_ptr[ix + 1]; ++xx)
                        gcol.push_back(X.adj[xx] + nx * (jy + ny * jz));
                }
            }
            S.glob_rowptr[g + 1] = (long long)gcol.size();
        }
    }
    S.nnz = (long long)gcol.size();
    // permuted CSR: row = pos, columns = positions ascending
    S.rowptr.assign(N + 1, 0);
    S.col.resize(S.nnz);
    S.perm_to_glob.resize(S.nnz);
    {
        std::vector<std::pair<int, long long>> tmp;
        long long at = 0;
        for (int i = 0; i < N; ++i) {
            int g = S.perm[i];
            tmp.clear();
            for (long long e = S.glob_rowptr[g]; e < S.glob_rowptr[g + 1]; ++e)
                tmp.push_back({S.ipos[gcol[e]], e});
            std::sort(tmp.begin(), tmp.end());
            for (auto& pr : tmp) {
                S.col[at] = pr.first;
                S.perm_to_glob[at] = pr.second;
                ++at;
            }
            S.rowptr[i + 1] = at;
        }
    }

    // ------------------------------------------------------------- fronts
    S.k.assign(F, 0);
    S.n.assign(F, 0);
    S.front_ptr.assign(F + 1, 0);
    S.front_pos.clear();
    std::vector<int> stamp(N, -1);
    std::vector<int> cand;
    for (int f = 0; f < F; ++f) {
        const int b0 = S.node_ptr[f], b1 = S.node_ptr[f + 1];
        cand.clear();
        for (int i = b0; i < b1; ++i)
            for (long long e = S.rowptr[i]; e < S.rowptr[i + 1]; ++e) {
                int q = S.col[e];
                if (q >= b1 && stamp[q] != f) { stamp[q] = f; cand.push_back(q); }
            }
        for (int ci = S.child_ptr[f]; ci < S.child_ptr[f + 1]; ++ci) {
            int c = S.child_list[ci];
            for (long long e = S.front_ptr[c] + S.k[c]; e < S.front_ptr[c] + S.n[c]; ++e) {
                int q = S.front_pos[e];
                if (q < b0) return "internal: child border precedes parent";
                if (q >= b1 && stamp[q] != f) { stamp[q] = f; cand.push_back(q); }
            }
        }
        std::sort(cand.begin(), cand.end());
        S.front_ptr[f] = (long long)S.front_pos.size();
        for (int i = b0; i < b1; ++i) S.front_pos.push_back(i);
        for (int q : cand) S.front_pos.push_back(q);
        S.k[f] = b1 - b0;
        S.n[f] = S.k[f] + (int)cand.size();
    }
    S.front_ptr[F] = (long long)S.front_pos.size();

    auto local_index = [&](int f, int q) -> int {
        if (q >= S.node_ptr[f] && q < S.node_ptr[f + 1]) return q - S.node_ptr[f];
        const int* bb = S.front_pos.data() + S.front_ptr[f] + S.k[f];
        const int* be = S.front_pos.data() + S.front_ptr[f + 1];
        const int* it = std::lower_bound(bb, be, q);
        if (it == be || *it != q) return -1;
        return S.k[f] + (int)(it - bb);
    };

    // Augmented fronts: k extra rows below the n front rows, coupled to the own
    // variables by the identity.  Eliminating the own block leaves -A11^{-1} A12
    // and -A11^{-1} in the extra rows' Schur complement: the solve operators.
    S.ld.assign(F, 0);
    for (int f = 0; f < F; ++f) S.ld[f] = S.n[f] + S.k[f];
    S.front_off.assign(F + 1, 0);
    for (int f = 0; f < F; ++f) S.front_off[f + 1] = S.front_off[f] + (long long)S.ld[f] * S.ld[f];
    S.pool_size = S.front_off[F];

    S.scatter.assign(S.nnz, -1);
    for (int i = 0; i < N; ++i)
        for (long long e = S.rowptr[i]; e < S.rowptr[i + 1]; ++e) {
            int j = S.col[e];
            if (j > i) continue;
            int f = S.node_of[j];
            int lc = j - S.node_ptr[f];
            int lr = local_index(f, i);
            if (lr < 0) return "internal: matrix entry outside its front";
            S.scatter[e] = S.front_off[f] + (long long)lc * S.ld[f] + lr;
        }

    S.rel_ptr.assign(F + 1, 0);
    S.upd_off.assign(F + 1, 0);
    S.rel.clear();
    for (int f = 0; f < F; ++f) {
        S.rel_ptr[f] = (long long)S.rel.size();
        S.upd_off[f + 1] = S.upd_off[f] + (S.n[f] - S.k[f]);
        int par = S.parent[f];
        for (long long e = S.front_ptr[f] + S.k[f]; e < S.front_ptr[f + 1]; ++e) {
            if (par < 0) return "internal: root front with a border";
            int li = local_index(par, S.front_pos[e]);
            if (li < 0) return "internal: child border not in parent front";
            S.rel.push_back(li);
        }
    }
    S.rel_ptr[F] = (long long)S.rel.size();
    S.upd_size = S.upd_off[F];

    // (solve items are built after the heights, below)

    return finish_symbolic(S);
}


// Concatenates independent problems into one forest: positions, DOFs, nodes,
// CSR entries, fronts and maps are offset per problem; the schedule and the
// solve items are then built for the whole forest (one launch per level and
// one persistent solve serve every problem).
std::string merge_symbolic(Symbolic& M, const std::vector<Symbolic>& P) {
    M = Symbolic();
    M.dim = 0;  // a batch: per-problem data stay in P
    long long N = 0, nnz = 0, pool = 0, fpos = 0, rel = 0, upd = 0, nel = 0;
    int F = 0, nch = 0;
    for (const Symbolic& S : P) {
        N += S.N;
        nnz += S.nnz;
        F += S.n_nodes;
    }
    if (N > 2000000000LL) return "batch too large for 32-bit DOF indices";
    M.N = N;
    M.nnz = nnz;
    M.n_nodes = F;
    M.perm.reserve(N);
    M.ipos.reserve(N);
    M.node_of.reserve(N);
    M.rowptr.assign(1, 0);
    M.glob_rowptr.assign(1, 0);
    M.node_ptr.clear();
    M.front_ptr.clear();
    M.child_ptr.clear();
    M.rel_ptr.clear();
    M.upd_off.clear();
    M.front_off.clear();
    long long pos0 = 0;
    int node0 = 0;
    for (const Symbolic& S : P) {
        M.prob_pos.push_back(pos0);
        M.prob_nnz.push_back(M.col.size());
        M.prob_elem.push_back(nel);
        M.prob_node.push_back(node0);
        for (int i = 0; i < S.N; ++i) {
            M.perm.push_back((int)(S.perm[i] + pos0));
            M.ipos.push_back((int)(S.ipos[i] + pos0));
            M.node_of.push_back(S.node_of[i] + node0);
            M.prob_of_pos.push_back((int)M.prob_pos.size() - 1);
        }
        const long long e0 = (long long)M.col.size();
        for (int i = 0; i < S.N; ++i) {
            M.rowptr.push_back(S.rowptr[i + 1] + e0);
            M.glob_rowptr.push_back(S.glob_rowptr[i + 1] + e0);
        }
        for (long long e = 0; e < S.nnz; ++e) {
            M.col.push_back((int)(S.col[e] + pos0));
            M.perm_to_glob.push_back(S.perm_to_glob[e] + e0);
            M.scatter.push_back(S.scatter[e] >= 0 ? S.scatter[e] + pool : -1);
        }
        for (int f = 0; f < S.n_nodes; ++f) {
            M.node_ptr.push_back((int)(S.node_ptr[f] + pos0));
            M.parent.push_back(S.parent[f] >= 0 ? S.parent[f] + node0 : -1);
            M.child_ptr.push_back((int)M.child_list.size() + S.child_ptr[f] - S.child_ptr[0]);
            M.k.push_back(S.k[f]);
            M.n.push_back(S.n[f]);
            M.ld.push_back(S.ld[f]);
            M.front_ptr.push_back(S.front_ptr[f] + fpos);
            M.front_off.push_back(S.front_off[f] + pool);
            M.rel_ptr.push_back(S.rel_ptr[f] + rel);
            M.upd_off.push_back(S.upd_off[f] + upd);
        }
        for (int c : S.child_list) M.child_list.push_back(c + node0);
        for (int q : S.front_pos) M.front_pos.push_back((int)(q + pos0));
        for (int r : S.rel) M.rel.push_back(r);
        pos0 += S.N;
        node0 += S.n_nodes;
        pool += S.pool_size;
        fpos += (long long)S.front_pos.size();
        rel += (long long)S.rel.size();
        upd += S.upd_size;
        nel += S.n_elem;
        ++nch;
    }
    M.node_ptr.push_back((int)N);
    M.front_ptr.push_back(fpos);
    M.front_off.push_back(pool);
    M.child_ptr.push_back((int)M.child_list.size());
    M.rel_ptr.push_back(rel);
    M.upd_off.push_back(upd);
    M.prob_pos.push_back(N);
    M.prob_nnz.push_back((long long)M.col.size());
    M.prob_elem.push_back(nel);
    M.prob_node.push_back(F);
    M.pool_size = pool;
    M.upd_size = upd;
    M.n_elem = nel;
    (void)nch;
    return finish_symbolic(M);
}

}  // namespace riga
