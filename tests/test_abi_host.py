"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and
its host-side symbolic analysis (riga_analyze, no device) matches the
oracle's separator-induced ordering and fronts bit for bit."""
import os
import re

import numpy as np
import pytest

from oracle import assembly, bspline, symbolic
from paper_2009_08167_gb300.inputs import Mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "riga.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2009_08167_gb300 import riga
    if not os.path.exists(riga.LIB_PATH):
        from paper_2009_08167_gb300.build import build
        build()
    return riga.load_library()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(riga_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("riga_create", "riga_assemble", "riga_factor", "riga_solve", "riga_eigs", "riga_eig_grad",
                 "riga_query", "riga_destroy", "riga_strerror"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_strerror_names(lib):
    assert lib.riga_strerror(0) == b"RIGA_OK"
    assert lib.riga_strerror(-3) == b"RIGA_EPIVOT"
    assert lib.riga_strerror(-99) == b"RIGA_UNKNOWN"


def _host_ctx():
    from paper_2009_08167_gb300.riga import Riga
    return Riga(device=-1)


def _oracle_symbolic(mesh):
    mults = mesh.mults
    n1, N = assembly.dof_count(mesh.dim, mesh.ne, mesh.p, mults)
    c0 = symbolic.riga_c0_lists(mesh.dim, mesh.ne, mesh.p, mults)
    nodes, perm = symbolic.build_tree(n1, c0, mesh.p, mesh.leaf_extent)
    return n1, N, nodes, perm


CASES = [
    Mesh(2, 16, 2, None, 8),          # 16x16 p=2 maximum continuity
    Mesh(2, 32, 3, 8, 8),             # rIGA blocks of 8, inner dissection
    Mesh(2, [13, 9], 2, 4, 4),        # ragged, partial last block
    Mesh(2, 24, 3, 8, 11),            # block interiors are the leaves
    Mesh(1, 40, 3, 8, 8),
    Mesh(3, [6, 5, 7], 2, None, 3),
    Mesh(3, 8, 2, 4, 8),
    Mesh(2, 10, 1, None, 4),          # p = 1: every knot is C0
    Mesh(2, 3, 4, None, 2),           # fewer elements than the degree
    Mesh(3, [7, 9, 5], 2, 3, 4),      # 3D rIGA, ragged last blocks in every direction
    Mesh(3, [10, 6, 8], 3, 4, 5),     # 3D rIGA p = 3, uneven extents
    Mesh(2, [37, 23], 4, 8, 8),       # p = 4, ragged blocks
    Mesh(2, 20, 5, 6, 12),            # p = 5, leaves larger than the blocks
    Mesh(1, 57, 2, 5, 6),             # 1D rIGA, ragged last block
    Mesh(2, [5, 40], 2, 16, 3),       # one direction without a C0 line
    Mesh(3, 6, 1, None, 2),           # 3D p = 1
]


@pytest.mark.parametrize("mesh", CASES, ids=[repr(m) for m in CASES])
def test_symbolic_bit_exact(mesh):
    r = _host_ctx()
    r.analyze(mesh)
    got = r.get_symbolic()
    q = r.query()
    n1, N, nodes, perm = _oracle_symbolic(mesh)
    assert q["N"] == N
    assert np.array_equal(got["perm"], perm)
    node_ptr = np.cumsum([0] + [nd["vars"].size for nd in nodes])
    assert np.array_equal(got["node_ptr"], node_ptr)
    par = symbolic.parents(nodes)
    assert np.array_equal(got["parent"], par)
    if N <= 5000:
        K, M = assembly.assemble_kron(mesh.dim, mesh.ne, mesh.p, mesh.mults)
        assert q["nnz"] == K.nnz
        fr = symbolic.fronts(nodes, perm, (K.indptr, K.indices))
        fp = got["front_ptr"]
        for F, (own, border) in enumerate(fr):
            idx = got["front_idx"][fp[F]:fp[F + 1]]
            assert np.array_equal(idx, np.concatenate([own, border])), F
        nnzL, flops = symbolic.front_nnz_and_flops(fr)
        assert q["nnzL"] == nnzL
        assert q["flops_fact"] == float(flops)


def test_symbolic_full_size_c2_riga_perm():
    # the 256^2 p=3 rIGA mesh with C0 lines every 16 elements (82,369 DOFs)
    mesh = Mesh(2, 256, 3, 16, 8)
    r = _host_ctx()
    r.analyze(mesh)
    got = r.get_symbolic()
    n1, N, nodes, perm = _oracle_symbolic(mesh)
    assert N == 82369 and n1 == [287, 287]
    assert np.array_equal(got["perm"], perm)
    assert np.array_equal(got["parent"], symbolic.parents(nodes))


def test_analyze_rejects_bad_mesh():
    from paper_2009_08167_gb300.riga import RigaError
    r = _host_ctx()
    with pytest.raises(RigaError):
        r.analyze(Mesh(4 if False else 2, 8, 0, None))  # p = 0
    m = Mesh(2, 8, 2, None)
    m.mults[0][3] = 5  # multiplicity above p
    with pytest.raises(RigaError):
        r.analyze(m)


def test_host_context_refuses_device_calls():
    from paper_2009_08167_gb300.riga import RigaError, RIGA_ESTATE
    r = _host_ctx()
    r.analyze(Mesh(2, 8, 2, None))
    with pytest.raises(RigaError) as e:
        r.factor(0.0)
    assert e.value.code == RIGA_ESTATE


def test_host_context_options_and_autotune():
    """riga_set_reorth validates its argument on any context; riga_autotune
    needs a device context (RIGA_ESTATE on a host-only one)."""
    from paper_2009_08167_gb300.riga import RigaError, RIGA_EINVAL, RIGA_ESTATE
    r = _host_ctx()
    r.analyze(Mesh(2, 8, 2, None))
    r.set_reorth(1)
    r.set_reorth(2)
    for bad in (0, 3):
        with pytest.raises(RigaError) as e:
            r.set_reorth(bad)
        assert e.value.code == RIGA_EINVAL
    with pytest.raises(RigaError) as e:
        r.autotune()
    assert e.value.code == RIGA_ESTATE


@pytest.mark.parametrize("mesh", [Mesh(2, 256, 3, 16, 8), Mesh(2, 256, 3, None, 8), Mesh(3, 64, 2, 8, 8),
                                  Mesh(3, 32, 2, 8, 8), Mesh(1, 33, 4, 8), Mesh(2, [13, 9], 3, 4, 4)],
                         ids=["c2_riga", "c2_iga", "c3", "3d_32", "1d", "2d_ragged"])
def test_bulk_copies_aligned_and_in_range(lib, mesh):
    """Host check of every bulk copy of the schedule (riga_check_copies, also
    run by riga_assemble): the tree solve's operator panels start on
    16-byte boundaries with sizes in whole 16-byte units inside the operator
    pool, and every tensor-core tile's packed blocks exist and belong to its
    own front and panel step."""
    from paper_2009_08167_gb300 import riga
    r = riga.Riga(-1)
    r.analyze(mesh)
    n = r.check_copies()
    assert n > 0
    r.close()
