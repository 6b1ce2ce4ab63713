"""The allocation-free SpMV + inner product (riga_spmv_dot_noalloc) against
the regular entry point (riga_spmv with the context's own scratch).

Callers that cannot allocate device memory use the no-alloc variant; it keeps
its partial sums in a fixed device array shared by every call.  Two calls in
a row must both agree with the regular path (the second one reuses the
array's previous contents), also when both are queued on one stream with no
synchronization between them.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _matrix():
    import torch

    from paper_2009_08167_gb300.inputs import Mesh
    from tests.gpu_helpers import riga_ctx

    R = riga_ctx()
    R.assemble(Mesh(2, 64, 3, 16, 8))
    rp, col, kv, mv = R.get_matrices()
    dev = torch.device("cuda", 0)
    return R, rp, torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev), torch.from_numpy(mv).to(dev)


def test_spmv_dot_noalloc_matches_regular_path_twice():
    import torch

    from paper_2009_08167_gb300 import riga

    R, rp, rp_d, col_d, mv_d = _matrix()
    N = rp.size - 1
    dev = rp_d.device
    rng = np.random.default_rng(17)
    for call in range(2):
        x = rng.normal(size=N)
        x_d = torch.from_numpy(x).to(dev)
        y_d = torch.zeros(N, dtype=torch.float64, device=dev)
        xy_d = torch.zeros(1, dtype=torch.float64, device=dev)
        riga.spmv_dot_noalloc(rp_d, col_d, mv_d, x_d, y_d, xy_d)
        torch.cuda.synchronize()
        y_ref = R.spmv(0, x)  # regular entry point: y = M x
        y = y_d.cpu().numpy()
        assert np.allclose(y, y_ref, rtol=1e-13, atol=1e-15), call
        xy_ref = float(x @ y_ref)
        assert abs(float(xy_d.item()) - xy_ref) <= 1e-12 * abs(xy_ref), call
    R.close()


def test_spmv_dot_noalloc_two_calls_queued_on_one_stream():
    """Both calls on one non-default stream, no synchronization in between:
    stream order keeps the second call's use of the shared array after the
    first call's reduction has read it."""
    import torch

    from paper_2009_08167_gb300 import riga

    R, rp, rp_d, col_d, mv_d = _matrix()
    N = rp.size - 1
    dev = rp_d.device
    rng = np.random.default_rng(23)
    xs = [rng.normal(size=N) for _ in range(2)]
    st = torch.cuda.Stream(device=dev)
    st.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(st):
        x_d = [torch.from_numpy(x).to(dev, non_blocking=False) for x in xs]
        y_d = [torch.zeros(N, dtype=torch.float64, device=dev) for _ in xs]
        xy_d = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in xs]
    for i in range(2):
        riga.spmv_dot_noalloc(rp_d, col_d, mv_d, x_d[i], y_d[i], xy_d[i], stream=st)
    st.synchronize()
    for i, x in enumerate(xs):
        y_ref = R.spmv(0, x)
        assert np.allclose(y_d[i].cpu().numpy(), y_ref, rtol=1e-13, atol=1e-15), i
        xy_ref = float(x @ y_ref)
        assert abs(float(xy_d[i].item()) - xy_ref) <= 1e-12 * abs(xy_ref), i
    R.close()


def test_spmv_dot_noalloc_rejects_host_pointer():
    """A host array among the arguments is refused by the C entry point
    itself (RIGA_EINVAL) before anything is launched."""
    import torch

    from paper_2009_08167_gb300 import riga

    lib = riga.load_library()
    R, rp, rp_d, col_d, mv_d = _matrix()
    N = rp.size - 1
    dev = rp_d.device
    x_h = np.ones(N)
    y_d = torch.zeros(N, dtype=torch.float64, device=dev)
    xy_d = torch.zeros(1, dtype=torch.float64, device=dev)
    P = ctypes.c_void_p
    rc = lib.riga_spmv_dot_noalloc(P(rp_d.data_ptr()), P(col_d.data_ptr()), P(mv_d.data_ptr()), N,
                                   P(x_h.ctypes.data), P(y_d.data_ptr()), P(xy_d.data_ptr()), None)
    assert rc == riga.RIGA_EINVAL
    rp_h = np.ascontiguousarray(rp)
    rc = lib.riga_spmv_dot_noalloc(P(rp_h.ctypes.data), P(col_d.data_ptr()), P(mv_d.data_ptr()), N,
                                   P(y_d.data_ptr()), P(y_d.data_ptr()), P(xy_d.data_ptr()), None)
    assert rc == riga.RIGA_EINVAL
    torch.cuda.synchronize()
    assert float(xy_d.item()) == 0.0  # nothing ran
    # the Python wrapper refuses CPU tensors and wrong dtypes before the call
    with pytest.raises(ValueError):
        riga.spmv_dot_noalloc(rp_d, col_d, mv_d, torch.from_numpy(x_h), y_d, xy_d)
    with pytest.raises(ValueError):
        riga.spmv_dot_noalloc(rp_d, col_d.to(torch.int64), mv_d, y_d, y_d, xy_d)
    R.close()


def test_spmv_dot_noalloc_rejects_oversize():
    import torch

    from paper_2009_08167_gb300 import riga

    dev = torch.device("cuda", 0)
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    col = torch.zeros(1, dtype=torch.int32, device=dev)
    val = torch.zeros(1, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    y = torch.zeros(n, dtype=torch.float64, device=dev)
    xy = torch.zeros(1, dtype=torch.float64, device=dev)
    with pytest.raises(riga.RigaError) as e:
        riga.spmv_dot_noalloc(rp, col, val, x, y, xy)
    assert e.value.code == riga.RIGA_EINVAL
