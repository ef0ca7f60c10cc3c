"""GPU coupling selection (c_min > 0) against the FP64 oracle.

The selection decision C > c_min is taken in FP64 on both sides from the same
inputs (the oracle gets the FP32 scene's fields rounded to FP32), so the set
of zeroed chains must agree exactly.  Values: FP64 1e-10 relative (as the full
path), FP32 + refinement 1e-4 relative on every radiance, K entries at the
FP32-derived bound of the full path (2e-5 relative).
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


def fp32_inputs(sc):
    """The scene with its fields rounded to FP32 (what an FP32 scene sees)."""
    return sc.replace(mu_a=sc.mu_a.astype(np.float32).astype(np.float64),
                      mu_s=sc.mu_s.astype(np.float32).astype(np.float64))


def run_gpu(sc, precision, rtol):
    rn = T.Runner(sc, precision)
    mu_a, mu_s = rn.fields("cuda")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    rn.solve(rtol=rtol)
    rad, _ = rn.render()
    torch.cuda.synchronize()
    return rn, rad.cpu().numpy().astype(np.float64)


def gpu_vs_oracle_slots(rn, r):
    st = rn.stats
    rp = rn.get(T.F_ROW_PTR, st.n_nodes + 1, torch.int32)
    col = rn.get(T.F_COL, st.nnz, torch.int32)
    dr = rn.get(T.F_SLOT_DIR, st.nnz, torch.int16)
    k = rn.get(T.F_SLOT_K, st.nnz, torch.int8)
    val = rn.get(T.F_VAL, st.nnz, rn.dtype)
    rows = np.repeat(np.arange(st.n_nodes), np.diff(rp))
    kg = np.stack([rows, col, dr.astype(np.int64), k.astype(np.int64)], 1)
    ko = np.stack([r["slot_row"], r["slot_col"], r["slot_dir"], r["slot_k"]], 1)
    ig = np.lexsort(kg.T[::-1])
    io = np.lexsort(ko.T[::-1])
    assert np.array_equal(kg[ig], ko[io])
    return val[ig].astype(np.float64), r["slot_val"][io]


CASES = {
    "random_R2_cmin3": (lambda: scenes.make_random(21, 19, 9, seed=7, S=2, R=2, M=2048), 3.0),
    "random_R2_cmin8": (lambda: scenes.make_random(21, 19, 9, seed=7, S=2, R=2, M=2048), 8.0),
    "random_R1_3species": (lambda: scenes.make_random(13, 11, 7, seed=8, S=3, R=1, M=1024, sza=20.0, vza=55.0), 8.0),
    "random_4species": (lambda: scenes.make_random(12, 11, 6, seed=10, S=4, R=2, M=1024), 5.0),
    "plume_small": (lambda: scenes.make_plume(nx=24, ny=20, nz=12), 2.0),
    "random_R2_all_dropped": (lambda: scenes.make_random(12, 11, 6, seed=11, S=2, R=2, M=1024), 1e30),
    # only the 9 upward chains that leave through the TOA stay (a short kept list)
    "random_R1_all_dropped": (lambda: scenes.make_random(10, 9, 5, seed=12, S=2, R=1, M=2048), 1e30),
    "random_R1_few_kept": (lambda: scenes.make_random(10, 9, 5, seed=13, S=1, R=1, M=2048), 9.0),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_selection_parity(name, prec):
    make, c_min = CASES[name]
    sc = make().replace(c_min=c_min)
    ref = sc if prec == "fp64" else fp32_inputs(sc)
    r = O.run(ref)
    full = O.run(ref.replace(c_min=0.0), flags=O.NO_SOLVE)
    dropped = (full["slot_val"] != 0).sum() - (r["slot_val"] != 0).sum()
    assert dropped > 0
    rn, rad = run_gpu(sc, T.FP64 if prec == "fp64" else T.FP32_REFINE, 1e-13 if prec == "fp64" else 1e-10)
    vg, vo = gpu_vs_oracle_slots(rn, r)
    # the same chains are zeroed on both sides
    assert np.array_equal(vg == 0, vo == 0)
    kt = 1e-11 if prec == "fp64" else 2e-5
    floor = (1e-14 if prec == "fp64" else 1e-6) * vo.max()
    assert (np.abs(vg - vo) / np.maximum(np.abs(vo), floor)).max() < kt
    st = rn.stats
    s = rn.get(T.F_S, st.n_nodes, rn.dtype)
    assert np.abs(s - r["s"]).max() <= kt * np.abs(r["s"]).max()
    tol = 1e-10 if prec == "fp64" else 1e-4
    err = (np.abs(rad - r["rad"]) / np.abs(r["rad"])).max()
    print("%s %s: %d chains' slots zeroed, radiance max rel err %.2e" % (name, prec, dropped, err))
    assert err < tol


def test_selection_toggle():
    """Switching the threshold on and off on one scene: the full path gives the
    same radiance bit for bit afterwards, and a negative threshold is
    rejected."""
    sc = scenes.make_plume(nx=24, ny=20, nz=12)
    rn, full0 = run_gpu(sc, T.FP32_REFINE, 1e-10)
    mu_a, mu_s = rn.fields("cuda")
    T.tursca_set_option(rn.handle, T.OPT_COUPLING_MIN, 0.5)
    rn.run(mu_a, mu_s, rtol=1e-10)
    sel = rn.rad.cpu().numpy().astype(np.float64)
    T.tursca_set_option(rn.handle, T.OPT_COUPLING_MIN, 0.0)
    rn.run(mu_a, mu_s, rtol=1e-10)
    torch.cuda.synchronize()
    full1 = rn.rad.cpu().numpy().astype(np.float64)
    assert np.array_equal(full0, full1)
    assert not np.array_equal(sel, full0)
    with pytest.raises(T.TurscaError) as e:
        T.tursca_set_option(rn.handle, T.OPT_COUPLING_MIN, -1.0)
    assert e.value.status == T.E_INVALID


def test_selection_adjoint_matches_oracle_finite_differences():
    """The gradient of J = sum_p L_p^2 with respect to absorption under
    coupling selection (the kept sets and weights depend on the scattering
    coefficients only): the FP64 adjoint against central differences of the
    FP64 oracle with the same threshold, and the FP32 adjoint at 1e-3."""
    sc = scenes.make_plume(nx=10, ny=10, nz=6).replace(c_min=3.0)
    base = np.asarray(sc.mu_a, dtype=np.float64)
    vox = np.sort(np.random.default_rng(3).choice(np.flatnonzero(base.ravel() > 1e-3), 6, replace=False))
    ref = []
    for v in vox:
        h = 1e-3 * float(base.ravel()[v]) + 1e-6
        js = []
        for sgn in (1.0, -1.0):
            m = base.copy()
            m.ravel()[v] += sgn * h
            js.append(float((O.run(sc.replace(mu_a=m))["rad"] ** 2).sum()))
        ref.append((js[0] - js[1]) / (2 * h))
    ref = np.array(ref)
    assert np.abs(ref).max() > 0
    for prec, tol in ((T.FP64, 1e-6), (T.FP32_REFINE, 1e-3)):
        rn = T.Runner(sc, prec)
        mu_a, mu_s = rn.fields("cuda")
        mu_a.requires_grad_(True)
        rad = T.render(mu_a, rn, mu_s, 1e-13 if prec == T.FP64 else 1e-10)
        (rad.double() ** 2).sum().backward()
        g = mu_a.grad.detach().cpu().numpy().astype(np.float64).ravel()[vox]
        rn.close()
        err = (np.abs(g - ref) / np.maximum(np.abs(ref), 1e-2 * np.abs(ref).max())).max()
        print("selection adjoint (precision %d) vs oracle fd: max rel err %.2e" % (prec, err))
        assert err < tol


# The preselected maximum number of couplings (Sec. 3): the GPU finds the
# (K + 1)-th largest FP64 coupling by a radix select and must reproduce the
# oracle's sorted threshold bit for bit, hence the same kept chains.
TOPK_CASES = {
    "random_R2": (lambda: scenes.make_random(21, 19, 9, seed=7, S=2, R=2, M=2048), 0.3),
    "random_R1_3species": (lambda: scenes.make_random(13, 11, 7, seed=8, S=3, R=1, M=1024, sza=20.0, vza=55.0), 0.5),
    "plume_small": (lambda: scenes.make_plume(nx=24, ny=20, nz=12), 0.1),
    # non-scattering voxels: zero couplings at the boundary (threshold: the smallest positive double)
    "zero_couplings": (lambda: scenes.make_random(12, 11, 6, seed=14, S=1, R=2, M=1024, zero_frac=0.3), None),
}


@pytest.mark.parametrize("name", list(TOPK_CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_topk_parity(name, prec):
    make, frac = TOPK_CASES[name]
    sc0 = make()
    ref0 = sc0 if prec == "fp64" else fp32_inputs(sc0)
    full = O.run(ref0, flags=O.NO_SOLVE)
    n = full["n_couplings"]
    if frac is None:
        # keep exactly the positive couplings (with K = n - 1 the threshold is
        # the smallest coupling, 0, so what stays is every positive one)
        K = int(O.run(ref0.replace(max_couplings=n - 1), flags=O.NO_SOLVE)["n_kept"])
        assert 0 < K < n - 1
    else:
        K = int(frac * n)
    sc = sc0.replace(max_couplings=K)
    r = O.run(ref0.replace(max_couplings=K))
    if frac is None:
        assert 0.0 < r["c_min_used"] < 1e-300 and r["n_kept"] == K
    rn, rad = run_gpu(sc, T.FP64 if prec == "fp64" else T.FP32_REFINE, 1e-13 if prec == "fp64" else 1e-10)
    info = T.tursca_selection_info(rn.handle)
    assert info["threshold"] == r["c_min_used"]
    assert info["n_couplings"] == r["n_couplings"] and info["n_kept"] == r["n_kept"]
    vg, vo = gpu_vs_oracle_slots(rn, r)
    assert np.array_equal(vg == 0, vo == 0)
    kt = 1e-11 if prec == "fp64" else 2e-5
    floor = (1e-14 if prec == "fp64" else 1e-6) * vo.max()
    assert (np.abs(vg - vo) / np.maximum(np.abs(vo), floor)).max() < kt
    tol = 1e-10 if prec == "fp64" else 1e-4
    err = (np.abs(rad - r["rad"]) / np.abs(r["rad"])).max()
    print("%s %s: K = %d of %d, kept %d, threshold %.6e, radiance max rel err %.2e"
          % (name, prec, K, n, info["n_kept"], info["threshold"], err))
    assert err < tol


def test_topk_edges_and_errors():
    """K at or above the number of couplings is the full stencil (bit for
    bit); c_min and K together, and a negative or fractional K, are
    rejected."""
    sc = scenes.make_plume(nx=24, ny=20, nz=12)
    rn, full0 = run_gpu(sc, T.FP32_REFINE, 1e-10)
    mu_a, mu_s = rn.fields("cuda")
    n = O.run(fp32_inputs(sc), flags=O.NO_SOLVE)["n_couplings"]
    for K in (n, 10 ** 12):
        T.tursca_set_option(rn.handle, T.OPT_MAX_COUPLINGS, K)
        rn.run(mu_a, mu_s, rtol=1e-10)
        torch.cuda.synchronize()
        assert np.array_equal(rn.rad.cpu().numpy().astype(np.float64), full0)
        info = T.tursca_selection_info(rn.handle)
        assert info["threshold"] == 0.0 and info["n_couplings"] == n and info["n_kept"] == n
    T.tursca_set_option(rn.handle, T.OPT_COUPLING_MIN, 1.0)
    with pytest.raises(T.TurscaError) as e:
        rn.run(mu_a, mu_s, rtol=1e-10)
    assert e.value.status == T.E_INVALID
    T.tursca_set_option(rn.handle, T.OPT_COUPLING_MIN, 0.0)
    for bad in (-1.0, 2.5):
        with pytest.raises(T.TurscaError) as e:
            T.tursca_set_option(rn.handle, T.OPT_MAX_COUPLINGS, bad)
        assert e.value.status == T.E_INVALID
    rn.close()
