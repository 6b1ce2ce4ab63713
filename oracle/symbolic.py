"""Separator-induced elimination order and multifrontal structure (oracle; test infrastructure only).

The paper orders with METIS (Sec. 6) and explains the cost of rIGA by
eliminating the macro-element blocks first and the C0 separators last
(Sec. 3.2, Fig. 2-3; Sec. 5.1, Eq. flopsFact).  The order used here is a
nested dissection whose cuts are those C0 separators, refined by p-thick
slabs inside blocks that are still larger than a leaf.  The rule (a reading;
the paper leaves the ordering to METIS):

* a box is a product of per-direction DOF intervals [lo, hi);
* leaf: every extent <= max(leaf_extent, p+1);
* C0 cut: otherwise, if some direction has a C0 DOF c with lo < c < hi-1,
  take among those directions the one with the largest extent (tie: lowest
  axis, x < y < z) and in it the c minimising |2c - (lo+hi-1)| (tie: lower
  c); the separator is the 1-DOF slab [c, c+1);
* p-thick cut: otherwise take the direction of largest extent (tie: lowest
  axis) and the slab [s, s+p) with s = lo + floor((hi-lo-p)/2);
* post-order: left child, right child, separator; inside a node the DOFs are
  lexicographic with x fastest (i.e. ascending global index).

A p-thick slab separates because two B-splines share an element only if
their indices differ by at most p; a C0 DOF separates because no other
function's support crosses its knot (Fig. 3).
"""
import numpy as np


def build_tree(n1, c0, p, leaf_extent):
    """Nested dissection of the DOF grid ``n1`` (per-direction counts, x first).

    ``c0[a]`` lists the C0 DOF indices in direction a.  Returns
    (nodes, perm): ``nodes`` is a post-ordered list of dicts with keys
    'vars' (global DOFs in elimination order) and 'children' (node ids);
    ``perm[pos] = global DOF`` eliminated at position pos.
    """
    dim = len(n1)
    c0s = [sorted(set(int(c) for c in c0[a])) for a in range(dim)]
    limit = max(leaf_extent, p + 1)
    nodes = []

    def box_vars(box):
        axes = [np.arange(lo, hi) for lo, hi in box]
        g = np.zeros(1, dtype=np.int64)
        for a in reversed(range(dim)):
            stride = int(np.prod(n1[:a])) if a > 0 else 1
            g = (g[:, None] + axes[a][None, :] * stride).ravel()
        return np.sort(g)

    def rec(box):
        ext = [hi - lo for lo, hi in box]
        if max(ext) <= limit:
            nodes.append({"vars": box_vars(box), "children": [], "box": box})
            return len(nodes) - 1
        cand = []
        for a in range(dim):
            lo, hi = box[a]
            if any(lo < c < hi - 1 for c in c0s[a]):
                cand.append(a)
        if cand:
            best = max(ext[a] for a in cand)
            a = min(a for a in cand if ext[a] == best)
            lo, hi = box[a]
            cs = [c for c in c0s[a] if lo < c < hi - 1]
            c = min(cs, key=lambda c: (abs(2 * c - (lo + hi - 1)), c))
            s, t = c, c + 1
        else:
            best = max(ext)
            a = min(a for a in range(dim) if ext[a] == best)
            lo, hi = box[a]
            s = lo + (hi - lo - p) // 2
            t = s + p
        left = list(box)
        left[a] = (lo, s)
        right = list(box)
        right[a] = (t, hi)
        sep = list(box)
        sep[a] = (s, t)
        kids = [rec(left), rec(right)]
        nodes.append({"vars": box_vars(sep), "children": kids, "box": sep})
        return len(nodes) - 1

    rec([(0, n) for n in n1])
    perm = np.concatenate([nd["vars"] for nd in nodes])
    return nodes, perm


def fronts(nodes, perm, pattern):
    """Front index lists of the multifrontal LDL^T (Sec. 5.1 cost basis).

    For node F: own variables (fully summed) followed by the border, i.e. the
    later-eliminated variables adjacent to F's own variables or contained in a
    child's border.  ``pattern`` is a CSR matrix (indptr, indices) of the
    symmetric sparsity of A = K - sigma M in original numbering.  Returns a
    list of (own, border) arrays in original numbering; border sorted by
    elimination position.
    """
    N = perm.size
    pos = np.empty(N, dtype=np.int64)
    pos[perm] = np.arange(N)
    indptr, indices = pattern
    out = []
    for F, nd in enumerate(nodes):
        own = nd["vars"]
        last = pos[own].max()
        cand = set()
        for v in own:
            cand.update(indices[indptr[v]:indptr[v + 1]].tolist())
        for c in nd["children"]:
            cand.update(out[c][1].tolist())
        border = np.array(sorted((u for u in cand if pos[u] > last), key=lambda u: pos[u]), dtype=np.int64)
        own_set = set(own.tolist())
        assert not any(u in own_set for u in border.tolist())
        out.append((own, border))
    return out


def parents(nodes):
    """Parent node id of every node (-1 for the root)."""
    par = [-1] * len(nodes)
    for F, nd in enumerate(nodes):
        for c in nd["children"]:
            par[c] = F
    return par


def etree_liu(pattern, perm):
    """Elimination tree of P A P^T by Liu's algorithm with path compression
    (virtual ancestors).  Returns parent[j] in permuted numbering (-1 root)."""
    N = perm.size
    pos = np.empty(N, dtype=np.int64)
    pos[perm] = np.arange(N)
    indptr, indices = pattern
    parent = -np.ones(N, dtype=np.int64)
    anc = -np.ones(N, dtype=np.int64)
    for j in range(N):
        v = perm[j]
        for u in indices[indptr[v]:indptr[v + 1]]:
            i = pos[u]
            while i != -1 and i < j:
                nxt = anc[i]
                anc[i] = j
                if nxt == -1:
                    parent[i] = j
                i = nxt
    return parent


def symbolic_elimination(pattern, perm):
    """Brute-force symbolic Cholesky: eliminate the permuted graph vertex by
    vertex, turning each vertex's later neighbours into a clique.  Returns
    (struct, parent): struct[j] is the sorted array of rows i > j with
    L_ij structurally non-zero (permuted numbering); parent[j] = min struct[j]."""
    N = perm.size
    pos = np.empty(N, dtype=np.int64)
    pos[perm] = np.arange(N)
    indptr, indices = pattern
    adj = [set() for _ in range(N)]
    for v in range(N):
        for u in indices[indptr[v]:indptr[v + 1]]:
            if u != v:
                adj[pos[v]].add(int(pos[u]))
    struct = []
    parent = -np.ones(N, dtype=np.int64)
    for j in range(N):
        later = sorted(i for i in adj[j] if i > j)
        struct.append(np.array(later, dtype=np.int64))
        if later:
            parent[j] = later[0]
        for a in later:
            adj[a].update(later)
            adj[a].discard(a)
    return struct, parent


def front_nnz_and_flops(fr):
    """Entries of L held by dense fronts (lower trapezoid incl. diagonal) and
    the factorization flop count sum_F sum_{i<k} (n-i)(n-i-1) (a multiply-add
    counted as 2 flops, lower triangle only)."""
    nnz = 0
    flops = 0
    for own, border in fr:
        k = own.size
        n = k + border.size
        nnz += k * (k + 1) // 2 + k * (n - k)
        for i in range(k):
            flops += (n - i) * (n - i - 1)
    return nnz, flops


def riga_c0_lists(dim, ne, p, mults):
    """C0 DOF indices per direction (after Dirichlet removal)."""
    from . import bspline
    return [bspline.c0_dofs(ne[a], p, None if mults is None else mults[a]) for a in range(dim)]
