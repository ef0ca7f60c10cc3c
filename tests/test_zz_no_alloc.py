"""The allocation-free solve entry point, checked against the scene solve.

tursca_csr_solve_noalloc serves callers that may not allocate device memory
while they solve (a program whose device memory belongs to its own allocator,
or a loop where cudaMalloc's device-wide synchronisation is not allowed).  It
must give the same x as the library's regular refined Neumann solve on the
same matrix and source, call after call, although every call reuses the same
fixed scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2503_16037_gb300 import scenes
from paper_2503_16037_gb300 import tursca as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_16037_gb300 import build
    build.build()


@pytest.mark.parametrize("shape", [(24, 20, 12), (32, 32, 16)])
def test_noalloc_solve_matches_scene_solve_twice(shape):
    # 32 x 32 x 16 has 17,408 nodes: the residual pass's grid (capped at 1024
    # blocks of 8 warps) then walks its rows more than once per warp
    sc = scenes.make_plume(nx=shape[0], ny=shape[1], nz=shape[2])
    rn = T.Runner(sc, T.FP32_REFINE)
    mu_a, mu_s = rn.fields("cuda")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    rn.solve(rtol=1e-12, solver=T.SOLVER_NEUMANN)
    st = rn.stats
    n = st.n_nodes
    x_ref = rn.get(T.F_X, n, torch.float64)
    dev = "cuda"
    row_ptr = torch.from_numpy(rn.get(T.F_ROW_PTR, n + 1, torch.int32)).to(dev)
    col = torch.from_numpy(rn.get(T.F_COL, st.nnz, torch.int32)).to(dev)
    val = torch.from_numpy(rn.get(T.F_VAL, st.nnz, torch.float32)).to(dev)
    s = torch.from_numpy(rn.get(T.F_S, n, torch.float32)).to(dev)
    s2 = float((s.double() ** 2).sum())
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        r2 = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        T.tursca_csr_solve_noalloc(row_ptr, col, val, n, s, x, 30, 6, r2, stream)
        torch.cuda.synchronize()
        xs = x.cpu().numpy()
        # the same bound the parity tests put on x (1e-10 of its largest entry)
        assert np.abs(xs - x_ref).max() <= 1e-10 * np.abs(x_ref).max(), call
        assert 0.0 <= float(r2.item()) <= (1e-12 ** 2) * s2, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(T.TurscaError) as ei:
        T.tursca_csr_solve_noalloc(dummy, dummy, dummy, (1 << 20) + 1, dummy, dummy, 4, 1, None, 0)
    assert ei.value.status == T.E_INVALID
    # more than 10^6 launches in one call
    with pytest.raises(T.TurscaError) as ei:
        T.tursca_csr_solve_noalloc(dummy, dummy, dummy, 8, dummy, dummy, 100000, 1000, None, 0)
    assert ei.value.status == T.E_INVALID
