"""GPU adjoint: the gradient of J = sum_p L_p^2 with respect to the absorption
coefficient of every voxel, through the library's hand-written adjoint (K^T
solve and reverse edge march), checked against central finite differences of
the FP64 forward: the GPU FP64 path, and the FP64 CPU oracle on a small scene.

Finite differences use h = 1e-3 mu_a + 1e-6 km^-1 (central), on voxels drawn
with a fixed seed among those with mu_a > 1e-3 km^-1.  Tolerances:
  * FP64 adjoint vs FP64 differences: 1e-6 relative (the differences carry
    O(h^2) truncation, far below that);
  * FP32 adjoint (FP32 assembly and K^T solve) vs FP64 differences: 1e-3
    relative on every compared voxel (no floor).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_16037_gb300 import scenes
from paper_2503_16037_gb300 import tursca as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_16037_gb300 import build
    build.build()
    torch.cuda.init()


def pick_voxels(sc, n, seed=0, thresh=1e-3):
    rng = np.random.default_rng(seed)
    cand = np.flatnonzero(np.asarray(sc.mu_a).ravel() > thresh)
    return np.sort(rng.choice(cand, size=min(n, cand.size), replace=False))


def step(v):
    return 1e-3 * v + 1e-6


def fd_gpu(sc, vox, precision=T.FP64, rtol=1e-13):
    rn = T.Runner(sc, precision)
    mu_a, mu_s = rn.fields("cuda")
    flat = mu_a.view(-1)
    out = []
    for v in vox:
        v0 = float(flat[v])
        h = step(v0)
        js = []
        for sgn in (1.0, -1.0):
            flat[v] = v0 + sgn * h
            rn.run(mu_a, mu_s, rtol=rtol)
            torch.cuda.synchronize()
            js.append(float((rn.rad.double() ** 2).sum()))
        flat[v] = v0
        out.append((js[0] - js[1]) / (2 * h))
    rn.close()
    return np.array(out)


def adjoint_grad(sc, precision, rtol):
    rn = T.Runner(sc, precision)
    mu_a, mu_s = rn.fields("cuda")
    mu_a.requires_grad_(True)
    rad = T.render(mu_a, rn, mu_s, rtol)
    J = (rad.double() ** 2).sum()
    J.backward()
    g = mu_a.grad.detach().cpu().numpy().astype(np.float64).ravel()
    rn.close()
    return g


def compare(g, ref, rel, floor_frac):
    floor = floor_frac * np.abs(ref).max()
    err = np.abs(g - ref) / np.maximum(np.abs(ref), floor)
    return err.max()


def test_adjoint_fp64_matches_finite_differences():
    sc = scenes.make_plume(nx=16, ny=16, nz=8)
    vox = pick_voxels(sc, 16)
    g = adjoint_grad(sc, T.FP64, 1e-13)[vox]
    ref = fd_gpu(sc, vox)
    assert np.abs(ref).max() > 0
    err = compare(g, ref, 1e-6, 1e-3)
    print("fp64 adjoint vs fd: max rel err %.2e" % err)
    assert err < 1e-6


def test_adjoint_fp64_matches_oracle_finite_differences():
    """The oracle gradient: central differences of the FP64 CPU oracle."""
    sc = scenes.make_plume(nx=10, ny=10, nz=6)
    vox = pick_voxels(sc, 6, seed=1)
    g = adjoint_grad(sc, T.FP64, 1e-13)[vox]
    ref = []
    base = np.asarray(sc.mu_a, dtype=np.float64)
    for v in vox:
        h = step(float(base.ravel()[v]))
        js = []
        for sgn in (1.0, -1.0):
            m = base.copy()
            m.ravel()[v] += sgn * h
            js.append(float((O.run(sc.replace(mu_a=m))["rad"] ** 2).sum()))
        ref.append((js[0] - js[1]) / (2 * h))
    ref = np.array(ref)
    err = compare(g, ref, 1e-6, 1e-3)
    print("fp64 adjoint vs oracle fd: max rel err %.2e" % err)
    assert err < 1e-6


def oracle_fd(sc, vox):
    """Central differences of J = sum_p L_p^2 from the FP64 CPU oracle (all
    host cores), one pair of oracle runs per voxel."""
    import os
    base = np.asarray(sc.mu_a, dtype=np.float64)
    out = []
    for v in vox:
        h = step(float(base.ravel()[v]))
        js = []
        for sgn in (1.0, -1.0):
            m = base.copy()
            m.ravel()[v] += sgn * h
            js.append(float((O.run(sc.replace(mu_a=m, precision=0), threads=os.cpu_count() or 1)["rad"] ** 2)
                            .sum()))
        out.append((js[0] - js[1]) / (2 * h))
    return np.array(out)


def test_adjoint_fp32_plume_48x48x32():
    """The adjoint configuration: plume generator at 48 x 48 x 32, FP32 +
    refinement, 64 voxels against FP64 finite differences of the GPU path,
    and 16 of them against finite differences of the FP64 oracle; 1e-3
    relative on every voxel, no floor."""
    sc = scenes.make_plume(nx=48, ny=48, nz=32)
    vox = pick_voxels(sc, 64)
    g = adjoint_grad(sc, T.FP32_REFINE, 1e-10)[vox]
    ref = fd_gpu(sc, vox, T.FP64, 1e-12)
    assert np.all(ref != 0.0)
    err = np.abs(g - ref) / np.abs(ref)
    print("fp32 adjoint vs fp64 gpu fd (64 voxels): max rel err %.2e, |grad| %.2e .. %.2e"
          % (err.max(), np.abs(ref).min(), np.abs(ref).max()))
    assert err.max() < 1e-3
    # the oracle gradient on 16 of the 64 voxels (a seeded choice)
    sub = np.sort(np.random.default_rng(4).choice(len(vox), size=16, replace=False))
    ref_o = oracle_fd(sc, vox[sub])
    err_o = np.abs(g[sub] - ref_o) / np.abs(ref_o)
    print("fp32 adjoint vs fp64 oracle fd (16 voxels): max rel err %.2e" % err_o.max())
    assert err_o.max() < 1e-3
    # the two difference quotients agree well below the tolerance
    assert np.abs(ref[sub] - ref_o).max() <= 1e-4 * np.abs(ref_o).max()


def test_adjoint_linear_in_dJdL_and_state_checks():
    sc = scenes.make_plume(nx=12, ny=12, nz=6)
    rn = T.Runner(sc, T.FP64)
    mu_a, mu_s = rn.fields("cuda")
    with pytest.raises(T.TurscaError) as e:
        rn.adjoint(torch.ones_like(rn.rad))
    assert e.value.status == T.E_STATE
    rn.run(mu_a, mu_s, rtol=1e-13)
    a = torch.randn_like(rn.rad)
    b = torch.randn_like(rn.rad)
    ga, gb, gab = rn.adjoint(a), rn.adjoint(b), rn.adjoint(2.0 * a - b)
    lin = (2.0 * ga - gb - gab).abs().max().item()
    assert lin <= 1e-10 * max(ga.abs().max().item(), gb.abs().max().item())
    assert rn.adjoint(torch.zeros_like(rn.rad)).abs().max().item() == 0.0
    rn.close()


def test_adjoint_gather_tile_identical():
    """The K^T passes of the FP32 adjoint gather from a shared-memory tile or
    from global memory; both add the same products in the same order.  The
    reverse edge march scatters with atomics (order not fixed), so the
    gradients are compared to 1e-5 of their largest entry."""
    sc = scenes.make_plume(nx=24, ny=20, nz=12)
    grads = []
    for tile in (0, 1):
        rn = T.Runner(sc, T.FP32_REFINE)
        T.tursca_set_option(rn.handle, T.OPT_GATHER_TILE, tile)
        mu_a, mu_s = rn.fields("cuda")
        rn.run(mu_a, mu_s, rtol=1e-10)
        g = rn.adjoint(2.0 * rn.rad)
        torch.cuda.synchronize()
        grads.append(g.cpu().numpy().copy())
        rn.close()
    scale = np.abs(grads[0]).max()
    assert scale > 0
    assert np.abs(grads[0] - grads[1]).max() <= 1e-5 * scale


def test_adjoint_dot_product_over_every_voxel():
    """Dot-product test of the whole adjoint: for a random direction d over
    all voxels (scaled to the local absorption) and a random weighting w of
    the pixels, <dL/dmu_a d, w> from central differences of the FP64 forward
    equals <d, adjoint(w)>."""
    sc = scenes.make_plume(nx=16, ny=14, nz=8)
    rn = T.Runner(sc, T.FP64)
    mu_a, mu_s = rn.fields("cuda")
    gen = torch.Generator(device="cpu").manual_seed(5)
    d = (torch.rand(mu_a.shape, generator=gen, dtype=torch.float64) - 0.5).to(mu_a.device) * mu_a
    w = torch.randn(rn.rad.shape, generator=gen, dtype=torch.float64).to(mu_a.device)
    rn.run(mu_a, mu_s, rtol=1e-13)
    lhs_adj = float((rn.adjoint(w) * d).sum())
    h = 1e-4
    js = []
    for sgn in (1.0, -1.0):
        rn.run(mu_a + sgn * h * d, mu_s, rtol=1e-13)
        torch.cuda.synchronize()
        js.append(float((rn.rad * w).sum()))
    fd = (js[0] - js[1]) / (2 * h)
    rn.close()
    print("dot-product test: adjoint %.12e, differences %.12e" % (lhs_adj, fd))
    assert abs(fd) > 0
    assert abs(lhs_adj - fd) <= 1e-7 * abs(fd)
