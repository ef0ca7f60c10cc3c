"""GPU anisotropic multiple scattering (the edge unknowns of Eq. flux_system,
TURSCA_OPT_ANISO) against the FP64 oracle's edge form.

Tolerances as for the node form: FP64 1e-10 relative on every radiance,
FP32 (series in FP32 to a relative change of 1e-6) 1e-4.
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
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_aniso_parity(name, prec):
    sc = CASES[name]()
    r = O.run(sc, flags=O.ANISO)
    rn, rad = run_aniso(sc, T.FP64 if prec == "fp64" else T.FP32_REFINE)
    tol = 1e-10 if prec == "fp64" else 1e-4
    st = rn.stats
    x = rn.get(T.F_X, st.n_nodes, torch.float64)
    assert np.abs(x - r["x"]).max() <= tol * np.abs(r["x"]).max()
    err = (np.abs(rad - r["rad"]) / np.abs(r["rad"])).max()
    node = O.run(sc)["rad"]
    print("%s %s: %d terms, radiance max rel err %.2e (edge vs node form differ by %.2e)"
          % (name, prec, rn.info.iters, err, (np.abs(r["rad"] - node) / node).max()))
    assert err < tol


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
