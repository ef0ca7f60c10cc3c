"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances:
  * FP64 mode: 1e-10 relative on every radiance and on the intermediates.
  * FP32 + FP64 refinement: 1e-4 relative on every radiance (the accuracy
    the method targets); intermediates are checked at FP32-derived bounds:
    each K entry is a product of a few correctly rounded FP32 factors, an
    exp/expm1 and a tap sum of at most ~150 terms, so its relative error is
    below ~2e-5; sums over a row (s, E) carry the same bound.
Integer and index work (CSR structure, slot directions) is compared exactly.
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


def run_gpu(sc, precision=None, rtol=1e-11, solver=T.SOLVER_AUTO, host=False):
    rn = T.Runner(sc, precision)
    dev = "cpu" if host else "cuda"
    mu_a, mu_s = rn.fields(dev)
    if host:
        mu_a, mu_s = mu_a.pin_memory(), mu_s.pin_memory()
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    rn.solve(rtol=rtol, solver=solver)
    if host:
        rad = torch.empty((sc.npy, sc.npx), dtype=rn.dtype).pin_memory()
        refl = torch.empty((sc.npy, sc.npx), dtype=rn.dtype).pin_memory()
        rn.render(rad, refl)
    else:
        rad, refl = rn.render()
    torch.cuda.synchronize()
    return rn, rad.cpu().numpy().astype(np.float64), refl.cpu().numpy().astype(np.float64)


def gpu_slots(rn):
    st = rn.stats
    rp = rn.get(T.F_ROW_PTR, st.n_nodes + 1, torch.int32)
    col = rn.get(T.F_COL, st.nnz, torch.int32)
    dr = rn.get(T.F_SLOT_DIR, st.nnz, torch.int16)
    k = rn.get(T.F_SLOT_K, st.nnz, torch.int8)
    val = rn.get(T.F_VAL, st.nnz, rn.dtype)
    rows = np.repeat(np.arange(st.n_nodes), np.diff(rp))
    return rp, rows, col, dr, k, val


def match_slots(rn, r):
    rp, rows, col, dr, k, val = gpu_slots(rn)
    kg = np.stack([rows, col, dr.astype(np.int64), k.astype(np.int64)], 1)
    ko = np.stack([r["slot_row"], r["slot_col"], r["slot_dir"], r["slot_k"]], 1)
    ig = np.lexsort(kg.T[::-1])
    io = np.lexsort(ko.T[::-1])
    assert np.array_equal(kg[ig], ko[io])
    return val[ig].astype(np.float64), r["slot_val"][io]


def rel_err(a, b, floor=0.0):
    return np.abs(a - b) / np.maximum(np.abs(b), floor)


SMALL = {
    "plain8_fp64": lambda: scenes.make_plain(),
    "random_R2_ragged": lambda: scenes.make_random(21, 19, 9, seed=7, S=2, R=2, M=2048),
    "random_R1_3species": lambda: scenes.make_random(13, 11, 7, seed=8, S=3, R=1, M=1024, sza=20.0, vza=55.0),
    "thin_nz_eq_R": lambda: scenes.make_random(9, 10, 2, seed=9, S=2, R=2, M=1024),
    "plume_small": lambda: scenes.make_plume(nx=24, ny=20, nz=12),
    "random_4species": lambda: scenes.make_random(12, 11, 6, seed=10, S=4, R=2, M=1024),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_fp64_parity_all_stages(name):
    sc = SMALL[name]()
    r = O.run(sc)
    rn, rad, refl = run_gpu(sc, precision=T.FP64, rtol=1e-13)
    st = rn.stats
    nn, na = st.n_nodes, st.n_atm
    np.testing.assert_allclose(rn.get(T.F_TSUN, nn, torch.float64), r["tsun"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(rn.get(T.F_E1, nn, torch.float64), r["e1"], rtol=1e-11, atol=1e-300)
    qs = rn.get(T.F_Q_SUN, sc.n_species * st.n_dirs, torch.float64).reshape(sc.n_species, -1)
    np.testing.assert_allclose(qs, r["q_sun"], rtol=1e-12, atol=1e-16)
    vg, vo = match_slots(rn, r)
    assert rel_err(vg, vo, 1e-14 * vo.max()).max() < 1e-11
    np.testing.assert_allclose(rn.get(T.F_S, nn, torch.float64), r["s"], rtol=1e-11, atol=1e-14 * r["s"].max())
    x = rn.get(T.F_X, nn, torch.float64)
    assert np.abs(x - r["x"]).max() <= 1e-10 * np.abs(r["x"]).max()
    em = rn.get(T.F_EMIS, na, torch.float64)
    assert np.abs(em - r["emis"]).max() <= 1e-10 * np.abs(r["emis"]).max()
    assert rel_err(rad, r["rad"]).max() < 1e-10
    assert rel_err(refl, r["refl"]).max() < 1e-10
    assert rn.info.rel_resid64 <= 1e-13


@pytest.mark.parametrize("name", ["random_R2_ragged", "random_R1_3species", "thin_nz_eq_R", "plume_small",
                                  "random_4species"])
def test_fp32_refined_parity(name):
    sc = SMALL[name]()
    r = O.run(sc)
    rn, rad, refl = run_gpu(sc, precision=T.FP32_REFINE, rtol=1e-10)
    st = rn.stats
    vg, vo = match_slots(rn, r)
    assert rel_err(vg, vo, 1e-6 * vo.max()).max() < 2e-5
    s = rn.get(T.F_S, st.n_nodes, torch.float32)
    assert np.abs(s - r["s"]).max() <= 2e-5 * np.abs(r["s"]).max()
    assert rn.info.rel_resid64 <= 1e-10
    err = rel_err(rad, r["rad"])
    assert err.max() < 1e-4, err.max()
    assert rel_err(refl, r["refl"]).max() < 1e-4


def test_device_structure_equals_host_structure():
    sc = SMALL["random_R2_ragged"]()
    rn = T.Runner(sc, T.FP32_REFINE)
    rp_h, col_h, dr_h, k_h = T.tursca_graph_structure(rn.desc)
    st = rn.stats
    assert np.array_equal(rn.get(T.F_ROW_PTR, st.n_nodes + 1, torch.int32), rp_h)
    assert np.array_equal(rn.get(T.F_COL, st.nnz, torch.int32), col_h)
    assert np.array_equal(rn.get(T.F_SLOT_DIR, st.nnz, torch.int16), dr_h)
    assert np.array_equal(rn.get(T.F_SLOT_K, st.nnz, torch.int8), k_h)


@pytest.mark.parametrize("solver", [T.SOLVER_NEUMANN, T.SOLVER_GMRES, T.SOLVER_CHEBYSHEV])
def test_solvers_agree(solver):
    sc = SMALL["plume_small"]()
    r = O.run(sc)
    rn, rad, _ = run_gpu(sc, precision=T.FP32_REFINE, rtol=1e-10, solver=solver)
    assert rn.info.solver == solver
    assert rel_err(rad, r["rad"]).max() < 1e-4


def test_cloud_high_albedo_fp32():
    """Broken cloud (omega 0.999, largest eigenvalue of K near 1): the automatic
    solver must reach the FP64 tolerance and match the oracle to 1e-4."""
    sc = scenes.make_cloud(nx=32, ny=32, nz=40)
    r = O.run(sc)
    rn, rad, _ = run_gpu(sc, precision=T.FP32_REFINE, rtol=1e-10)
    print("cloud 32x32x40: iters %d refinements %d rho %.4f solver %d" % (rn.info.iters, rn.info.refinements,
                                                                        rn.info.rho_est, rn.info.solver))
    assert rn.info.rel_resid64 <= 1e-10
    assert rel_err(rad, r["rad"]).max() < 1e-4


def test_fp32_pair_residual_matches_fp64_residual():
    """The refinement residual in FP32-pair arithmetic and in FP64 arithmetic
    give the same solution (both converge to the solution of the FP32 K)."""
    sc = SMALL["plume_small"]()
    xs = []
    for opt in (0, 1):
        rn = T.Runner(sc, T.FP32_REFINE)
        T.tursca_set_option(rn.handle, T.OPT_RESIDUAL_FP64, opt)
        mu_a, mu_s = rn.fields("cuda")
        rn.run(mu_a, mu_s, rtol=1e-12)
        assert rn.info.rel_resid64 <= 1e-12
        xs.append(rn.get(T.F_X, rn.stats.n_nodes, torch.float64))
    assert np.abs(xs[0] - xs[1]).max() <= 1e-10 * np.abs(xs[1]).max()


@pytest.mark.parametrize("name", ["random_R2_ragged", "plume_small"])
def test_staged_values_identical(name):
    """Streaming the values through shared memory (persistent pipelined
    passes) changes where the warps read them, not what they add: both
    drivers sum the same products in the same order, so x and the radiance
    are bit-identical with and without it, for every warp count."""
    sc = SMALL[name]()
    ref = None
    for wq in (4, 8, 16):
        for stage in (0, 1):
            rn = T.Runner(sc, T.FP32_REFINE)
            T.tursca_set_option(rn.handle, T.OPT_GROUP_WARPS, wq)
            T.tursca_set_option(rn.handle, T.OPT_STAGE_VALUES, stage)
            mu_a, mu_s = rn.fields("cuda")
            rad, _ = rn.run(mu_a, mu_s, rtol=1e-11)
            torch.cuda.synchronize()
            x = rn.get(T.F_X, rn.stats.n_nodes, torch.float64)
            got = (x, rad.cpu().numpy(), rn.info.iters)
            rn.close()
            if ref is None:
                ref = (wq, got)
            elif wq == ref[0]:
                assert got[2] == ref[1][2]
                assert np.array_equal(got[0], ref[1][0])
                assert np.array_equal(got[1], ref[1][1])
            if stage == 1:
                ref = None


@pytest.mark.parametrize("solver", [T.SOLVER_NEUMANN, T.SOLVER_GMRES, T.SOLVER_CHEBYSHEV])
@pytest.mark.parametrize("name", ["random_R2_ragged", "random_R1_3species", "thin_nz_eq_R", "plume_small"])
def test_gather_tile_and_l2_residency_identical(name, solver):
    """Gathering the source vector from a shared-memory tile, and keeping the
    values of K resident in L2, change where the passes read their operands,
    not the products or their order: x and the radiance are bit-identical to
    those of the passes that gather from global memory, for every solver."""
    sc = SMALL[name]()
    outs = []
    for tile, l2 in ((0, 0), (1, 0), (1, 1), (0, 1)):
        rn = T.Runner(sc, T.FP32_REFINE)
        T.tursca_set_option(rn.handle, T.OPT_GATHER_TILE, tile)
        T.tursca_set_option(rn.handle, T.OPT_L2_RESIDENT, l2)
        mu_a, mu_s = rn.fields("cuda")
        rad, _ = rn.run(mu_a, mu_s, rtol=1e-11, solver=solver)
        torch.cuda.synchronize()
        x = rn.get(T.F_X, rn.stats.n_nodes, torch.float64)
        outs.append((x, rad.cpu().numpy(), rn.info.iters))
        rn.close()
    for got in outs[1:]:
        assert got[2] == outs[0][2]
        assert np.array_equal(got[0], outs[0][0])
        assert np.array_equal(got[1], outs[0][1])


def test_host_pointers_end_to_end():
    sc = SMALL["plume_small"]()
    r = O.run(sc)
    _, rad, refl = run_gpu(sc, precision=T.FP32_REFINE, rtol=1e-10, host=True)
    assert rel_err(rad, r["rad"]).max() < 1e-4


def test_edge_cases_geometry_and_medium():
    # nadir sun and view, no coupling, black surface, detector finer than the grid
    base = scenes.make_random(10, 9, 5, seed=11, S=1, R=2, M=1024, sza=0.0, vza=0.0, albedo=0.0, npx=20, npy=9)
    cases = [base, base.replace(coupling=0), base.replace(npx=5, npy=3, vza=45.0, vaa=10.0, sza=75.0)]
    vac = base.copy()
    vac.mu_s[:, 2] = 0.0          # a layer with no scattering at all
    vac.mu_a[1] = 0.0
    vac.mu_s[:, 1] = 0.0          # and a vacuum layer
    cases.append(vac)
    for sc in cases:
        r = O.run(sc)
        _, rad, _ = run_gpu(sc, precision=T.FP64, rtol=1e-13)
        assert rel_err(rad, r["rad"], 1e-300).max() < 1e-10


def test_out_of_order_and_invalid_fields():
    sc = SMALL["plume_small"]()
    rn = T.Runner(sc, T.FP32_REFINE)
    with pytest.raises(T.TurscaError) as ei:
        T.tursca_assemble_flux(rn.handle, rn.geom)
    assert ei.value.status == T.E_STATE
    mu_a, mu_s = rn.fields("cuda")
    mu_a[0, 0, 0] = float("nan")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    with pytest.raises(T.TurscaError) as ei:
        rn.solve()
    assert ei.value.status == T.E_INVALID
    with pytest.raises(T.TurscaError) as ei:
        T.tursca_adjoint(rn.handle, None, None)
    assert ei.value.status == T.E_INVALID
    # a valid medium afterwards works on the same scene
    mu_a, mu_s = rn.fields("cuda")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    rn.solve()
    rn.render()


def test_plume_full_size_bench_configuration():
    """64x64x32, R = 2, FP32 + FP64 refinement, exactly as the benchmark runs it."""
    sc = scenes.make_plume()
    r = O.run(sc)
    rn, rad, refl = run_gpu(sc, precision=T.FP32_REFINE, rtol=1e-10)
    err = rel_err(rad, r["rad"])
    print("plume 64x64x32: max rel err %.3e  mean %.3e  solve iters %d refinements %d rho %.3f"
          % (err.max(), err.mean(), rn.info.iters, rn.info.refinements, rn.info.rho_est))
    assert err.max() < 1e-4
    assert rel_err(refl, r["refl"]).max() < 1e-4
    # sampled K entries against the oracle
    vg, vo = match_slots(rn, r)
    idx = np.random.default_rng(0).choice(len(vo), 200000, replace=False)
    assert rel_err(vg[idx], vo[idx], 1e-6 * vo.max()).max() < 2e-5


def test_cloud_full_size_configuration():
    """The broken-cloud configuration at full size (128 x 128 x 40, R = 2,
    about 81M edges; omega 0.999, largest eigenvalue of K near 0.99, so the
    solver hands over to GMRES), FP32 + FP64 refinement, every radiance
    against the FP64 oracle."""
    sc = scenes.make_cloud()
    r = O.run(sc)
    rn, rad, refl = run_gpu(sc, precision=T.FP32_REFINE, rtol=1e-10)
    err = rel_err(rad, r["rad"])
    print("cloud 128x128x40: max rel err %.3e  mean %.3e  iters %d refinements %d solver %d"
          % (err.max(), err.mean(), rn.info.iters, rn.info.refinements, rn.info.solver))
    assert rn.info.rel_resid64 <= 1e-10
    assert err.max() < 1e-4
    assert rel_err(refl, r["refl"]).max() < 1e-4



@pytest.mark.parametrize("precision", [T.FP32_REFINE, T.FP64])
def test_repeated_runs_on_one_runner_identical(precision):
    """A Runner re-assembles, re-solves and re-renders with its geometry
    buffers kept from the first run: every run must give the same bits."""
    sc = SMALL["plume_small"]()
    rn = T.Runner(sc, precision)
    mu_a, mu_s = rn.fields("cuda")
    rads = []
    for _ in range(3):
        rad, refl = rn.run(mu_a, mu_s, rtol=1e-10 if precision == T.FP32_REFINE else 1e-13)
        torch.cuda.synchronize()
        rads.append((rad.cpu().numpy().copy(), refl.cpu().numpy().copy()))
    rn.close()
    for r in rads[1:]:
        assert np.array_equal(r[0], rads[0][0])
        assert np.array_equal(r[1], rads[0][1])


@pytest.mark.parametrize("precision", [T.FP32_REFINE, T.FP64])
def test_run_in_one_call_equals_the_four_calls(precision):
    """tursca_run (set_medium, assemble_flux, solve, render in one call)
    gives the bits of the four calls made one by one, with device and with
    pinned host buffers, and reports the errors of its steps."""
    sc = SMALL["random_R2_ragged"]()
    rtol = 1e-10 if precision == T.FP32_REFINE else 1e-13
    rn = T.Runner(sc, precision)
    mu_a, mu_s = rn.fields("cuda")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    info1 = rn.solve(rtol=rtol)
    rad1, refl1 = rn.render()
    torch.cuda.synchronize()
    ref = (rad1.cpu().numpy().copy(), refl1.cpu().numpy().copy())
    rad2, refl2 = rn.run(mu_a, mu_s, rtol=rtol)
    torch.cuda.synchronize()
    assert np.array_equal(rad2.cpu().numpy(), ref[0]) and np.array_equal(refl2.cpu().numpy(), ref[1])
    assert rn.info.iters == info1.iters and rn.info.refinements == info1.refinements
    # pinned host buffers through the same call
    dt = torch.float32 if precision == T.FP32_REFINE else torch.float64
    rad_h = torch.empty((sc.npy, sc.npx), dtype=dt).pin_memory()
    refl_h = torch.empty((sc.npy, sc.npx), dtype=dt).pin_memory()
    T.tursca_run(rn.handle, mu_a.cpu().pin_memory(), mu_s.cpu().pin_memory(), list(sc.g), sc.albedo, rn.geom,
                 T.SOLVER_AUTO, rtol, 5000, rad_h, refl_h)
    assert np.array_equal(rad_h.numpy(), ref[0]) and np.array_equal(refl_h.numpy(), ref[1])
    # an invalid field value is reported by the call
    bad = mu_a.clone()
    bad.view(-1)[0] = float("nan")
    with pytest.raises(T.TurscaError) as ei:
        rn.run(bad, mu_s, rtol=rtol)
    assert ei.value.status == T.E_INVALID
    rn.close()
