"""Thin ctypes binding of libriga.so (include/riga.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
only converts Python arguments to pointers and sizes.  Arrays may be numpy
arrays (host memory) or CUDA torch tensors (device memory, float64,
contiguous); outputs are returned in the kind of memory the caller asks for.
The library must have been built (``python -m paper_2009_08167_gb300.build``);
importing fails loudly otherwise: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from .inputs import Mesh

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libriga.so")

RIGA_OK = 0
RIGA_EINVAL = -1
RIGA_ESTATE = -2
RIGA_EPIVOT = -3
RIGA_ENOCONV = -4
RIGA_EREFINE = -5
RIGA_ETIMEOUT = -6
RIGA_ECUDA = -7
RIGA_ENOMEM = -8
RIGA_FP64 = 0
RIGA_FP32 = 1
RIGA_TF32 = 2
RIGA_BF16 = 3

EXPORTED = [
    "riga_create", "riga_destroy", "riga_analyze", "riga_assemble", "riga_assemble_log", "riga_factor", "riga_solve", "riga_eigs",
    "riga_eigs_interval", "riga_eig_errors",
    "riga_set_eig_options", "riga_eig_grad", "riga_query", "riga_get_symbolic", "riga_get_matrices",
    "riga_get_factor", "riga_spmv", "riga_stats", "riga_profile", "riga_profile_get", "riga_set_wait_limit",
    "riga_trace_solve", "riga_check_copies", "riga_spmv_dot_noalloc", "riga_sym_eig", "riga_strerror",
    "riga_last_error",
]
PHASES = ["assemble", "factor", "solve", "reorth", "spmv", "ritz", "other"]


class RigaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} ({code})")
        self.code = code


class _MeshC(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("ne", ctypes.c_int * 3),
        ("p", ctypes.c_int),
        ("mult", ctypes.POINTER(ctypes.c_int) * 3),
        ("dirichlet", ctypes.c_int),
        ("leaf_extent", ctypes.c_int),
    ]


_lib = None


def load_library(path=LIB_PATH):
    """Load libriga.so and declare the C signatures.  Raises if missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libriga.so not built at {path}: run python -m paper_2009_08167_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    LL = ctypes.c_longlong
    lib.riga_create.argtypes = [ctypes.POINTER(P), I, P]
    lib.riga_destroy.argtypes = [P]
    lib.riga_destroy.restype = None
    lib.riga_assemble.argtypes = [P, ctypes.POINTER(_MeshC), P, P]
    lib.riga_assemble_log.argtypes = [P, ctypes.POINTER(_MeshC), P, P]
    lib.riga_analyze.argtypes = [P, ctypes.POINTER(_MeshC)]
    lib.riga_factor.argtypes = [P, D, I, ctypes.POINTER(LL)]
    lib.riga_solve.argtypes = [P, P, P, I, D, ctypes.POINTER(I)]
    lib.riga_eigs.argtypes = [P, I, D, D, P, P, P, ctypes.POINTER(I)]
    lib.riga_set_eig_options.argtypes = [P, I, I, I, I, ctypes.c_ulonglong]
    lib.riga_eig_grad.argtypes = [P, I, P, P, P]
    lib.riga_assemble_batch.argtypes = [P, I, ctypes.POINTER(_MeshC), P, P]
    lib.riga_band_eig.argtypes = [I, I, P, P, I, P, P, I, P]
    lib.riga_set_eig_block.argtypes = [P, I]
    lib.riga_set_reorth.argtypes = [P, I]
    lib.riga_set_fp64_update.argtypes = [P, I]
    lib.riga_set_eig_accuracy.argtypes = [P, I]
    lib.riga_autotune.argtypes = [P, P, P]
    lib.riga_eigs_batch.argtypes = [P, I, D, D, P, P, P]
    lib.riga_query.argtypes = [P, ctypes.POINTER(LL), ctypes.POINTER(LL), ctypes.POINTER(LL), ctypes.POINTER(D)]
    lib.riga_get_symbolic.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(LL), P, P, P, P, P]
    lib.riga_get_matrices.argtypes = [P, P, P, P, P]
    lib.riga_get_factor.argtypes = [P, P, P, P]
    lib.riga_spmv.argtypes = [P, I, P, P]
    lib.riga_stats.argtypes = [P] + [ctypes.POINTER(LL)] * 4 + [ctypes.POINTER(D)] * 2
    lib.riga_profile.argtypes = [P, I]
    lib.riga_set_wait_limit.argtypes = [P, LL]
    lib.riga_trace_solve.argtypes = [P, P, ctypes.POINTER(I), P, P]
    lib.riga_spmv_dot_noalloc.argtypes = [P, P, P, LL, P, P, P, P]
    lib.riga_sym_eig.argtypes = [I, P, P, P]
    lib.riga_check_copies.argtypes = [P, ctypes.POINTER(LL)]
    lib.riga_eigs_interval.argtypes = [P, D, D, I, D, I, P, P, P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.riga_eig_errors.argtypes = [P, I, P, I, P, P, P]
    lib.riga_profile_get.argtypes = [P, I, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(LL), ctypes.POINTER(LL),
                                     ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.riga_strerror.argtypes = [I]
    lib.riga_strerror.restype = ctypes.c_char_p
    lib.riga_last_error.argtypes = [P]
    lib.riga_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"] or a.flags["F_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def _is_torch(a):
    return a is not None and not isinstance(a, np.ndarray) and hasattr(a, "data_ptr")


class Riga:
    """One library context on one CUDA device and stream (C: riga_ctx)."""

    def __init__(self, device=0, stream=None):
        self.lib = load_library()
        self.ctx = ctypes.c_void_p()
        s = None
        if stream is not None:
            s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._check(self.lib.riga_create(ctypes.byref(self.ctx), int(device), s))
        self.mesh = None
        self._mult_keep = None

    def close(self):
        if self.ctx:
            self.lib.riga_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != RIGA_OK:
            msg = self.lib.riga_strerror(rc).decode()
            if getattr(self, "ctx", None):
                extra = self.lib.riga_last_error(self.ctx).decode()
                if extra:
                    msg += ": " + extra
            raise RigaError(rc, msg)
        return rc

    # ------------------------------------------------------------ riga_assemble
    @staticmethod
    def _mesh_c(mesh):
        m = _MeshC()
        m.dim = mesh.dim
        for a in range(3):
            m.ne[a] = mesh.ne[a] if a < mesh.dim else 1
        m.p = mesh.p
        keep = []
        for a in range(mesh.dim):
            arr = np.ascontiguousarray(mesh.mults[a], dtype=np.int32)
            keep.append(arr)
            m.mult[a] = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if arr.size else None
        m.dirichlet = 1
        m.leaf_extent = mesh.leaf_extent
        return m, keep

    def analyze(self, mesh: Mesh):
        m, keep = self._mesh_c(mesh)
        self._check(self.lib.riga_analyze(self.ctx, ctypes.byref(m)))
        self.mesh = mesh

    def assemble(self, mesh: Mesh, coefK=None, coefM=None, log=False):
        """K and M of `mesh`; coefK / coefM: per-element coefficients (or, with
        log=True, their logarithms, exponentiated by the library)."""
        m = _MeshC()
        m.dim = mesh.dim
        for a in range(3):
            m.ne[a] = mesh.ne[a] if a < mesh.dim else 1
        m.p = mesh.p
        keep = []
        for a in range(mesh.dim):
            arr = np.ascontiguousarray(mesh.mults[a], dtype=np.int32)
            keep.append(arr)
            m.mult[a] = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if arr.size else None
        m.dirichlet = 1
        m.leaf_extent = mesh.leaf_extent
        if coefK is not None and isinstance(coefK, np.ndarray):
            coefK = np.ascontiguousarray(coefK, dtype=np.float64)
        if coefM is not None and isinstance(coefM, np.ndarray):
            coefM = np.ascontiguousarray(coefM, dtype=np.float64)
        fn = self.lib.riga_assemble_log if log else self.lib.riga_assemble
        self._check(fn(self.ctx, ctypes.byref(m), _ptr(coefK), _ptr(coefM)))
        self.mesh = mesh
        self._mult_keep = keep

    def assemble_batch(self, meshes, coefK=None, coefM=None):
        """Assembles independent problems into one batch context; coefK /
        coefM: None or a list with one array (or None) per problem."""
        n = len(meshes)
        arr = (_MeshC * n)()
        keep = []
        for b, mesh in enumerate(meshes):
            m, kp = self._mesh_c(mesh)
            arr[b] = m
            keep.append(kp)
        ptrs = []
        for coefs in (coefK, coefM):
            if coefs is None:
                ptrs.append((None, None))
                continue
            hold = [None if c is None else np.ascontiguousarray(c, dtype=np.float64) for c in coefs]
            pa = (ctypes.c_void_p * n)(*[None if h is None else h.ctypes.data for h in hold])
            ptrs.append((pa, hold))
        self._check(self.lib.riga_assemble_batch(self.ctx, n, arr, ptrs[0][0], ptrs[1][0]))
        self.meshes = list(meshes)
        self.mesh = None
        self._mult_keep = keep

    def eigs_batch(self, k, sigma=0.0, tol=1e-10, check=True):
        """(evals, resid, nconv) of every problem of the batch: arrays of
        shape (nprob, k), (nprob, k), (nprob,)."""
        n = len(self.meshes)
        ev = np.zeros((n, k))
        rs = np.zeros((n, k))
        nc = np.zeros(n, dtype=np.int32)
        rc = self.lib.riga_eigs_batch(self.ctx, int(k), float(sigma), float(tol), _ptr(ev), _ptr(rs), _ptr(nc))
        if check or rc != RIGA_ENOCONV:
            self._check(rc)
        return ev, rs, nc

    # ------------------------------------------------------------ riga_factor
    def factor(self, sigma, precision=RIGA_FP64):
        nneg = ctypes.c_longlong(0)
        self._check(self.lib.riga_factor(self.ctx, float(sigma), int(precision), ctypes.byref(nneg)))
        return nneg.value

    def query(self):
        N, nnz, nnzL = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        fl = ctypes.c_double()
        self._check(self.lib.riga_query(self.ctx, ctypes.byref(N), ctypes.byref(nnz), ctypes.byref(nnzL), ctypes.byref(fl)))
        return dict(N=N.value, nnz=nnz.value, nnzL=nnzL.value, flops_fact=fl.value)

    # ------------------------------------------------------------ riga_solve
    def solve(self, b, tol=0.0, out=None):
        """x = (K - sigma M)^{-1} b; b of shape (N,) or (N, nrhs) column-major."""
        N = self.query()["N"]
        if isinstance(b, np.ndarray):
            bb = np.asfortranarray(b, dtype=np.float64)
            nrhs = 1 if bb.ndim == 1 else bb.shape[1]
            x = np.zeros_like(bb) if out is None else out
        else:
            bb = b
            nrhs = 1 if b.dim() == 1 else b.shape[1]
            x = b.new_zeros(b.shape) if out is None else out
        assert bb.shape[0] == N
        it = ctypes.c_int(0)
        self._check(self.lib.riga_solve(self.ctx, _ptr(bb), _ptr(x), nrhs, float(tol), ctypes.byref(it)))
        return x, it.value

    def set_eig_options(self, slice=0, precision=RIGA_FP64, max_steps=0, extra=2, seed=1):
        self._check(self.lib.riga_set_eig_options(self.ctx, int(slice), int(precision), int(max_steps), int(extra), int(seed)))

    def set_eig_block(self, block):
        self._check(self.lib.riga_set_eig_block(self.ctx, int(block)))

    def autotune(self):
        """Measured choice of the factorization's update-tile shapes for the
        assembled pattern; returns (chosen cut-off, [ms per candidate 0, 128,
        256, 512, 1024, 4096]).  Leaves the FP64 factorization at sigma = 0."""
        t = ctypes.c_int(0)
        ms = (ctypes.c_double * 6)()
        self._check(self.lib.riga_autotune(self.ctx, ctypes.byref(t), ms))
        return t.value, list(ms)

    def set_eig_accuracy(self, rayleigh):
        """0: eigenvalues sigma + 1/theta (default); 1: double-double Rayleigh
        quotients of the Ritz vectors (for finite-difference checks)."""
        self._check(self.lib.riga_set_eig_accuracy(self.ctx, int(rayleigh)))

    def set_fp64_update(self, mode):
        """Schur updates of FP64 fronts: 0 on the CUDA cores (FP64 FMA), 1 (the
        default) on the tensor cores from exact 8-bit digit-slice products."""
        self._check(self.lib.riga_set_fp64_update(self.ctx, int(mode)))

    def set_reorth(self, passes):
        """1: recurrence + one full Gram-Schmidt pass (switching to 2 by itself
        when one pass is not enough); 2: two full passes every step."""
        self._check(self.lib.riga_set_reorth(self.ctx, int(passes)))

    # ------------------------------------------------------------ riga_eigs
    def eigs(self, k, sigma=0.0, tol=1e-10, vectors=True, device_out=False):
        N = self.query()["N"]
        if device_out:
            import torch
            ev = torch.zeros(k, dtype=torch.float64, device="cuda")
            U = torch.zeros((k, N), dtype=torch.float64, device="cuda") if vectors else None
            rs = torch.zeros(k, dtype=torch.float64, device="cuda")
        else:
            ev = np.zeros(k)
            U = np.zeros((k, N)) if vectors else None  # row i = eigenvector i (column-major N x k)
            rs = np.zeros(k)
        nconv = ctypes.c_int(0)
        rc = self.lib.riga_eigs(self.ctx, int(k), float(sigma), float(tol), _ptr(ev), _ptr(U), _ptr(rs), ctypes.byref(nconv))
        if rc not in (RIGA_OK,):
            self._check(rc)
        U = U.T if U is not None else None
        return ev, U, rs

    def eigs_interval(self, lo, hi, kmax, tol=1e-10, m_basis=0, vectors=True):
        """Every eigenpair with lo <= lambda < hi (riga_eigs_interval):
        (evals, U (N x n) or None, resid, basis_cols); raises RigaError
        RIGA_EINVAL with .count when the interval holds more than kmax."""
        N = self.query()["N"]
        ev = np.zeros(max(kmax, 1))
        U = np.zeros((max(kmax, 1), N)) if vectors else None
        rs = np.zeros(max(kmax, 1))
        nf = ctypes.c_int(0)
        bc = ctypes.c_int(0)
        rc = self.lib.riga_eigs_interval(self.ctx, float(lo), float(hi), int(kmax), float(tol), int(m_basis), _ptr(ev),
                                         _ptr(U), _ptr(rs), ctypes.byref(nf), ctypes.byref(bc))
        if rc != RIGA_OK:
            err = RigaError(rc, self.lib.riga_strerror(rc).decode() + ": " + self.lib.riga_last_error(self.ctx).decode())
            err.count = nf.value
            raise err
        n = nf.value
        return ev[:n], (U[:n].T if U is not None else None), rs[:n], bc.value

    def eig_errors(self, modes, nq=0):
        """(EVerr, EFerr_L2, EFerr_E) of the first len(modes) computed
        eigenpairs against the exact Laplace modes (1-based index tuples, x
        first), riga_eig_errors."""
        md = np.ascontiguousarray(modes, dtype=np.int32)
        if md.ndim == 1:
            md = md[:, None]
        n = md.shape[0]
        out = [np.zeros(n) for _ in range(3)]
        self._check(self.lib.riga_eig_errors(self.ctx, n, _ptr(md), int(nq), *[_ptr(o) for o in out]))
        return tuple(out)

    def eig_grad(self, k, weights):
        """Gradients (grad_a, grad_b) of sum_i weights[i] lambda_i; numpy in ->
        numpy out, CUDA tensor in -> CUDA tensors out."""
        ne = self.mesh.n_elem
        if _is_torch(weights):
            w = weights.contiguous()
            ga = w.new_zeros(ne)
            gb = w.new_zeros(ne)
        else:
            w = np.ascontiguousarray(weights, dtype=np.float64)
            ga = np.zeros(ne)
            gb = np.zeros(ne)
        self._check(self.lib.riga_eig_grad(self.ctx, int(k), _ptr(w), _ptr(ga), _ptr(gb)))
        return ga, gb

    # ------------------------------------------------------------ inspection
    def check_copies(self):
        """Number of bulk copies of the current schedule verified on the host
        (riga_check_copies); raises RigaError on a violation."""
        n = ctypes.c_longlong(0)
        self._check(self.lib.riga_check_copies(self.ctx, ctypes.byref(n)))
        return n.value

    def get_symbolic(self):
        nn = ctypes.c_int()
        tot = ctypes.c_longlong()
        self._check(self.lib.riga_get_symbolic(self.ctx, ctypes.byref(nn), ctypes.byref(tot), None, None, None, None, None))
        N = self.query()["N"]
        perm = np.zeros(N, dtype=np.int32)
        node_ptr = np.zeros(nn.value + 1, dtype=np.int32)
        parent = np.zeros(nn.value, dtype=np.int32)
        front_ptr = np.zeros(nn.value + 1, dtype=np.int64)
        front_idx = np.zeros(tot.value, dtype=np.int32)
        self._check(self.lib.riga_get_symbolic(self.ctx, ctypes.byref(nn), ctypes.byref(tot), _ptr(perm), _ptr(node_ptr),
                                               _ptr(parent), _ptr(front_ptr), _ptr(front_idx)))
        return dict(perm=perm, node_ptr=node_ptr, parent=parent, front_ptr=front_ptr, front_idx=front_idx)

    def get_matrices(self):
        q = self.query()
        N, nnz = q["N"], q["nnz"]
        rp = np.zeros(N + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        kv = np.zeros(nnz)
        mv = np.zeros(nnz)
        self._check(self.lib.riga_get_matrices(self.ctx, _ptr(rp), _ptr(col), _ptr(kv), _ptr(mv)))
        return rp, col, kv, mv

    def get_factor(self, with_L=False):
        sym = self.get_symbolic()
        N = self.query()["N"]
        nn = sym["node_ptr"].size - 1
        D = np.zeros(N)
        Lptr = np.zeros(nn + 1, dtype=np.int64)
        self._check(self.lib.riga_get_factor(self.ctx, _ptr(D), _ptr(Lptr), None))
        L = None
        if with_L:
            L = np.zeros(int(Lptr[-1]))
            self._check(self.lib.riga_get_factor(self.ctx, None, _ptr(Lptr), _ptr(L)))
        return D, Lptr, L

    def spmv(self, which, x):
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
            y = np.zeros_like(x)
        else:
            y = x.new_zeros(x.shape)
        self._check(self.lib.riga_spmv(self.ctx, int(which), _ptr(x), _ptr(y)))
        return y

    def stats(self):
        v = [ctypes.c_longlong() for _ in range(4)] + [ctypes.c_double() for _ in range(2)]
        self._check(self.lib.riga_stats(self.ctx, *[ctypes.byref(t) for t in v]))
        keys = ["n_fact", "n_solve", "n_matvec", "lanczos_steps", "t_fact_ms", "t_lanczos_ms"]
        return {k: t.value for k, t in zip(keys, v)}

    def trace_solve(self, b):
        """One traced solve: per work item (sm, claim ns, ready ns, done ns) and its node."""
        bb = np.ascontiguousarray(b, dtype=np.float64) if isinstance(b, np.ndarray) else b
        ni = ctypes.c_int(0)
        self._check(self.lib.riga_trace_solve(self.ctx, _ptr(bb), ctypes.byref(ni), None, None))
        tr = np.zeros((ni.value, 4), dtype=np.int64)
        order = np.zeros(ni.value, dtype=np.int32)
        self._check(self.lib.riga_trace_solve(self.ctx, _ptr(bb), ctypes.byref(ni), _ptr(tr), _ptr(order)))
        return tr, order

    def set_wait_limit(self, limit):
        self._check(self.lib.riga_set_wait_limit(self.ctx, int(limit)))

    # ------------------------------------------------------------ profiling
    def profile(self, enable=True):
        self._check(self.lib.riga_profile(self.ctx, 1 if enable else 0))

    def launches(self):
        n = ctypes.c_longlong()
        self._check(self.lib.riga_profile_get(self.ctx, -1, None, ctypes.byref(n), None, None, None, None))
        return n.value

    def profile_get(self):
        out = {}
        for i, name in enumerate(PHASES):
            la, ca = ctypes.c_longlong(), ctypes.c_longlong()
            ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            self._check(self.lib.riga_profile_get(self.ctx, i, None, ctypes.byref(la), ctypes.byref(ca), ctypes.byref(ms),
                                                  ctypes.byref(by), ctypes.byref(fl)))
            out[name] = dict(launches=la.value, calls=ca.value, ms=ms.value, bytes=by.value, flops=fl.value)
        return out


def band_eig(T, b, which=(), last_rows=0):
    """Eigenvalues (ascending) of the symmetric band matrix T (half-bandwidth
    b), the eigenvectors of the eigenvalues with indices `which`, and (when
    last_rows > 0) the last rows of all eigenvectors; host only."""
    lib = load_library()
    T = np.asfortranarray(T, dtype=np.float64)
    n = T.shape[0]
    theta = np.zeros(n)
    wh = np.ascontiguousarray(which, dtype=np.int32)
    S = np.zeros((n, max(1, wh.size)), order="F")
    Z = np.zeros((max(1, last_rows), n), order="F")
    rc = lib.riga_band_eig(n, int(b), _ptr(T), _ptr(theta), int(wh.size), _ptr(wh) if wh.size else None,
                           _ptr(S) if wh.size else None, int(last_rows), _ptr(Z) if last_rows else None)
    if rc != RIGA_OK:
        raise RigaError(rc, lib.riga_strerror(rc).decode())
    if last_rows:
        return theta, S[:, :wh.size], Z
    return theta, S[:, :wh.size]


def sym_eig(A):
    """All eigenpairs (ascending eigenvalues, eigenvectors as columns) of a
    dense symmetric matrix; host only (riga_sym_eig)."""
    lib = load_library()
    A = np.asfortranarray(A, dtype=np.float64)
    n = A.shape[0]
    theta = np.zeros(n)
    Z = np.zeros((n, n), order="F")
    rc = lib.riga_sym_eig(n, _ptr(A), _ptr(theta), _ptr(Z))
    if rc != RIGA_OK:
        raise RigaError(rc, lib.riga_strerror(rc).decode())
    return theta, Z


def spmv_dot_noalloc(rowptr, col, val, x, y, xy, stream=None):
    """y = A x and xy[0] = x^T y through riga_spmv_dot_noalloc (no device
    allocation).  All arguments are CUDA torch tensors (int64 rowptr, int32
    col, float64 val/x/y/xy); work is enqueued on ``stream`` (a torch stream,
    default the current one) and not synchronized."""
    import torch
    lib = load_library()
    n = x.numel()
    want = [("rowptr", rowptr, torch.int64, n + 1), ("col", col, torch.int32, None), ("val", val, torch.float64, None),
            ("x", x, torch.float64, n), ("y", y, torch.float64, n), ("xy", xy, torch.float64, 1)]
    for name, t, dt, size in want:
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if size is not None and t.numel() != size:
            raise ValueError(f"{name} must have {size} entries, got {t.numel()}")
        if t.device != x.device:
            raise ValueError(f"{name} is on {t.device}, x on {x.device}")
    if col.numel() != val.numel():
        raise ValueError("col and val must have the same length")
    with torch.cuda.device(x.device):
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        rc = lib.riga_spmv_dot_noalloc(_ptr(rowptr), _ptr(col), _ptr(val), int(n), _ptr(x), _ptr(y), _ptr(xy),
                                       ctypes.c_void_p(s.cuda_stream))
    if rc != RIGA_OK:
        raise RigaError(rc, lib.riga_strerror(rc).decode())
