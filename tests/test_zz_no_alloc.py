"""The allocation-free SpMV + inner product (riga_spmv_dot_noalloc) against
the regular entry point (riga_spmv with the context's own scratch).

Callers that cannot allocate device memory use the no-alloc variant; it keeps
its partial sums in a fixed device array shared by every call.  Two calls in
a row must both agree with the regular path (the second one reuses the
array's previous contents).  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_spmv_dot_noalloc_matches_regular_path_twice():
    import torch

    from paper_2009_08167_gb300 import riga
    from paper_2009_08167_gb300.inputs import Mesh
    from tests.gpu_helpers import riga_ctx

    R = riga_ctx()
    R.assemble(Mesh(2, 64, 3, 16, 8))
    rp, col, kv, mv = R.get_matrices()
    N = rp.size - 1
    dev = torch.device("cuda", 0)
    rp_d = torch.from_numpy(rp).to(dev)
    col_d = torch.from_numpy(col).to(dev)
    mv_d = torch.from_numpy(mv).to(dev)
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
