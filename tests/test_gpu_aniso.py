"""GPU anisotropic multiple scattering (the edge unknowns of Eq. flux_system,
TURSCA_OPT_ANISO) against the FP64 oracle's edge form.

Tolerances as for the node form: FP64 1e-10 relative on every radiance,
FP32 (FP32 series, then refinement with the FP64 residual; the dense
per-node contraction on the tensor cores, or with TURSCA_OPT_ANISO = 2 on
the CUDA cores) 1e-4.
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


def run_aniso(sc, prec, aniso=1):
    rn = T.Runner(sc, prec)
    T.tursca_set_option(rn.handle, T.OPT_ANISO, aniso)
    mu_a, mu_s = rn.fields("cuda")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    rn.solve(rtol=1e-13 if prec == T.FP64 else 1e-10, max_iter=20000)
    rad, _ = rn.render()
    torch.cuda.synchronize()
    return rn, rad.cpu().numpy().astype(np.float64)


CASES = {
    "random_R2_2species": lambda: scenes.make_random(12, 11, 6, seed=51, S=2, R=2, M=1024),
    "random_R1_3species": lambda: scenes.make_random(13, 11, 7, seed=52, S=3, R=1, M=1024, sza=20.0, vza=55.0),
    "plume_12x12x6": lambda: scenes.make_plume(nx=12, ny=12, nz=6),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_cuda_cores"])
def test_aniso_parity(name, prec):
    sc = CASES[name]()
    r = O.run(sc, flags=O.ANISO)
    rn, rad = run_aniso(sc, T.FP64 if prec == "fp64" else T.FP32_REFINE, aniso=2 if prec == "fp32_cuda_cores" else 1)
    tol = 1e-10 if prec == "fp64" else 1e-4
    st = rn.stats
    x = rn.get(T.F_X, st.n_nodes, torch.float64)
    assert np.abs(x - r["x"]).max() <= tol * np.abs(r["x"]).max()
    err = (np.abs(rad - r["rad"]) / np.abs(r["rad"])).max()
    node = O.run(sc)["rad"]
    print("%s %s: %d terms, %d residuals (%.1e), radiance max rel err %.2e (edge vs node form differ by %.2e)"
          % (name, prec, rn.info.iters, rn.info.refinements, rn.info.rel_resid64, err,
             (np.abs(r["rad"] - node) / node).max()))
    assert err < tol
    if prec != "fp64":
        assert rn.info.refinements >= 1 and rn.info.rel_resid64 <= 1e-10


@pytest.mark.parametrize("name", ["random_R2_2species", "random_R1_3species"])
def test_aniso_contractions_tensor_cores_match_cuda_cores(name):
    """The tcgen05 kernel (TF32 high/low split, FP32 accumulation in tensor
    memory) against the CUDA-core FP32 kernel on the same tables, every
    output of the per-term contraction; the per-assembly one runs on the
    CUDA cores only."""
    sc = CASES[name]()
    rn = T.Runner(sc, T.FP32_REFINE)
    T.tursca_set_option(rn.handle, T.OPT_ANISO, 1)
    mu_a, mu_s = rn.fields("cuda")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    st = rn.stats
    nin = st.n_dirs + st.n_gdirs
    g = torch.Generator(device="cpu").manual_seed(7)
    X = torch.rand((nin, st.n_nodes), generator=g, dtype=torch.float32).cuda()
    out = torch.zeros((nin, st.n_atm), dtype=torch.float32, device="cuda")
    with pytest.raises(T.TurscaError) as e:
        T.tursca_selftest_aniso_contract(rn.handle, 1, True, X, out)
    assert e.value.status == T.E_UNSUPPORTED
    for which, N in ((0, st.n_dirs),):
        outs = []
        for mma in (True, False):
            out = torch.full((N, st.n_atm), float("nan"), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            T.tursca_selftest_aniso_contract(rn.handle, which, mma, X, out)
            outs.append(out.double().cpu().numpy())
        a, b = outs
        assert np.isfinite(a).all() and np.isfinite(b).all()
        scale = np.abs(b).max(axis=0, keepdims=True) + 1e-30
        err = (np.abs(a - b) / scale).max()
        print("%s contraction %d: max rel err %.2e" % (name, which, err))
        # hi*hi + hi*lo + lo*hi leaves 2^-22 of each product; the tensor
        # memory's FP32 accumulation over the 3 K / 8 MMAs adds a few 1e-6
        assert err < 2e-5


def test_aniso_terms_are_deterministic():
    sc = CASES["plume_12x12x6"]()
    _, a = run_aniso(sc, T.FP32_REFINE)
    _, b = run_aniso(sc, T.FP32_REFINE)
    assert np.array_equal(a, b)


def test_aniso_isotropic_phase_equals_node_form_on_gpu():
    sc = scenes.make_random(12, 11, 6, seed=53, S=2, R=2, M=1024).replace(g=np.zeros(2))
    _, a = run_aniso(sc, T.FP64)
    _, n = run_aniso(sc, T.FP64, aniso=0)
    assert (np.abs(a - n) / n).max() < 1e-11


def test_aniso_combinations_and_toggle():
    sc = scenes.make_plume(nx=12, ny=12, nz=6)
    rn, full0 = run_aniso(sc, T.FP32_REFINE, aniso=0)
    mu_a, mu_s = rn.fields("cuda")
    T.tursca_set_option(rn.handle, T.OPT_ANISO, 1)
    rn.run(mu_a, mu_s, rtol=1e-10)
    with pytest.raises(T.TurscaError) as e:
        rn.adjoint(torch.ones_like(rn.rad))
    assert e.value.status == T.E_UNSUPPORTED
    with pytest.raises(T.TurscaError) as e:
        rn.get(T.F_VAL, rn.stats.nnz, rn.dtype)
    assert e.value.status == T.E_STATE
    for opt in (T.OPT_SINGLE_SCATTER, T.OPT_COUPLING_MIN):
        T.tursca_set_option(rn.handle, opt, 1)
        with pytest.raises(T.TurscaError) as e:
            rn.assemble()
        assert e.value.status == T.E_INVALID
        T.tursca_set_option(rn.handle, opt, 0)
    T.tursca_set_option(rn.handle, T.OPT_ANISO, 0)
    rn.run(mu_a, mu_s, rtol=1e-10)
    torch.cuda.synchronize()
    assert np.array_equal(rn.rad.cpu().numpy().astype(np.float64), full0)


def _sample_rows(sc, n_per_layer=12, seed=3):
    """Rows spread over the layers that differ: the bottom and top layers
    (ground hits, directions without a receiver), the middle, and the ground."""
    rng = np.random.default_rng(seed)
    nxy = sc.nx * sc.ny
    layers = sorted({0, 1, sc.nz // 2, sc.nz - 2, sc.nz - 1, sc.nz})  # nz: the ground nodes
    rows = [z * nxy + int(c) for z in layers for c in rng.choice(nxy, n_per_layer, replace=False)]
    return np.array(rows, dtype=np.int32)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_aniso_full_plume_is_a_fixed_point_of_the_oracle_map(prec):
    """The full 64x64x32 plume (the bench's edge-form workload): the GPU's
    solved X(i, w) satisfies the oracle's own edge-form map, F_oracle(X) = X,
    at rows sampled over the layers that differ (the whole series does not
    fit the oracle at this size).  FP64: to rounding.  FP32 + refinement: to
    the FP32 rounding of the coefficients the GPU operator stores."""
    sc = scenes.make_plume()
    P = T.FP64 if prec == "fp64" else T.FP32_REFINE
    rn, rad = run_aniso(sc, P)
    st = rn.stats
    nin = st.n_dirs + st.n_gdirs
    X = rn.get(T.F_ANISO_X, nin * st.n_nodes, torch.float64).reshape(nin, st.n_nodes).T.copy()
    rows = _sample_rows(sc)
    F = O.aniso_rows(sc, X, rows)
    scale = np.abs(X[rows]).max(axis=1) + 1e-300
    err = (np.abs(F - X[rows]).max(axis=1) / scale).max()
    print("plume 64x64x32 %s: %d terms, %d residuals (%.1e); max row-relative |F(X) - X| = %.2e over %d rows"
          % (prec, rn.info.iters, rn.info.refinements, rn.info.rel_resid64, err, len(rows)))
    assert np.isfinite(rad).all() and (rad > 0).all()
    assert err < (1e-11 if prec == "fp64" else 5e-6)
