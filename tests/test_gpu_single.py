"""GPU first-order (single-scattering) path against the oracle's first-order
mode and against the discrete single-scattering closed form of a homogeneous
periodic slab.

Tolerances: FP64 1e-10 relative on every radiance (as for the full path);
FP32 1e-4 relative against the oracle, 2e-5 against the closed form (the
first order is a product of a few FP32 factors and one optical-depth sum
per ray, so its relative error stays near 1e-6).
"""
import math

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


def run_single(rn, single=True):
    T.tursca_set_option(rn.handle, T.OPT_SINGLE_SCATTER, 1 if single else 0)
    mu_a, mu_s = rn.fields("cuda")
    rn.set_medium(mu_a, mu_s)
    rn.assemble()
    rn.solve(rtol=1e-13 if rn.dtype == torch.float64 else 1e-10)
    rad, refl = rn.render()
    torch.cuda.synchronize()
    return rad.cpu().numpy().astype(np.float64), refl.cpu().numpy().astype(np.float64)


def rel_err(a, b):
    return np.abs(a - b) / np.abs(b)


SCENES = {
    "random_R2_ragged": lambda: scenes.make_random(21, 19, 9, seed=7, S=2, R=2, M=2048),
    "random_R1_3species": lambda: scenes.make_random(13, 11, 7, seed=8, S=3, R=1, M=1024, sza=20.0, vza=55.0),
    "plume_small": lambda: scenes.make_plume(nx=24, ny=20, nz=12),
    "random_4species": lambda: scenes.make_random(12, 11, 6, seed=10, S=4, R=2, M=1024),
}


@pytest.mark.parametrize("name", list(SCENES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_scatter_parity(name, prec):
    sc = SCENES[name]()
    r = O.run(sc, flags=O.SINGLE_SCATTER)
    rn = T.Runner(sc, T.FP64 if prec == "fp64" else T.FP32_REFINE)
    rad, refl = run_single(rn)
    st = rn.stats
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert rn.info.iters == 0 and rn.info.refinements == 0
    assert not np.any(rn.get(T.F_S, st.n_nodes, rn.dtype))
    assert not np.any(rn.get(T.F_X, st.n_nodes, torch.float64))
    e1 = rn.get(T.F_E1, st.n_nodes, rn.dtype)
    assert np.abs(e1 - r["e1"]).max() <= tol * np.abs(r["e1"]).max()
    em = rn.get(T.F_EMIS, st.n_atm, rn.dtype)
    assert np.abs(em - r["emis"]).max() <= tol * np.abs(r["emis"]).max()
    assert rel_err(rad, r["rad"]).max() < tol
    assert rel_err(refl, r["refl"]).max() < tol
    print("%s %s: first-order radiance max rel err %.2e" % (name, prec, rel_err(rad, r["rad"]).max()))


def l_ss_discrete(omega, g, sza, vza, mu_e, hz, nz, cosang):
    """First-order radiance (units of f0) of a homogeneous periodic slab over
    a black surface on the voxel lattice: each layer contributes
    omega mu0 Theta(cosang) (1 - e^{-dt/mu0}) (1 - e^{-dt/muv}) / dt, dimmed
    by e^{-k dt (1/mu0 + 1/muv)} for the k layers above it; the layer sum is
    geometric."""
    mu0, muv = math.cos(math.radians(sza)), math.cos(math.radians(vza))
    hgv = (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * cosang) ** 1.5)
    dt = mu_e * hz
    a = 1 / mu0 + 1 / muv
    return (omega * mu0 * hgv * (1 - math.exp(-dt / mu0)) * (1 - math.exp(-dt / muv)) / dt
            * (1 - math.exp(-nz * dt * a)) / (1 - math.exp(-dt * a)))


def unit(zen, az):
    z, a = math.radians(zen), math.radians(az)
    return np.array([math.sin(z) * math.cos(a), math.sin(z) * math.sin(a), math.cos(z)])


@pytest.mark.parametrize("R,sza,saa,vza,vaa", [(1, 30, 0, 0, 0), (2, 55, 40, 35, 300), (2, 10, 180, 50, 90)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_scatter_closed_form(R, sza, saa, vza, vaa, prec):
    nz, mu_e, om, g = 9, 0.8, 0.7, 0.6
    sc = scenes.make_layered(6, 6, nz, [mu_e] * nz, [om], g=(g,), albedo=0.0, R=R, sza=sza, saa=saa,
                             vza=vza, vaa=vaa, h=(0.1, 0.12, 0.07), M=1024)
    rn = T.Runner(sc, T.FP64 if prec == "fp64" else T.FP32_REFINE)
    rad, _ = run_single(rn)
    # sunlight travels along -unit(sza, saa) and leaves toward the instrument
    # along unit(vza, vaa): the scattering angle's cosine is their product
    ref = l_ss_discrete(om, g, sza, vza, mu_e, sc.hz, nz, float(-unit(sza, saa) @ unit(vza, vaa)))
    assert rel_err(rad, ref).max() < (1e-12 if prec == "fp64" else 2e-5)


def test_single_scatter_toggle_leaves_full_path_unchanged():
    """Switching the first-order mode on and off on one scene: the full path
    gives the same radiance bit for bit before and after, the first-order
    radiance lies below it (the higher orders add light), and the adjoint and
    the matrix values are refused after a first-order assembly."""
    sc = scenes.make_plume(nx=24, ny=20, nz=12)
    rn = T.Runner(sc, T.FP32_REFINE)
    full0, _ = run_single(rn, single=False)
    ss, _ = run_single(rn, single=True)
    with pytest.raises(T.TurscaError) as e:
        rn.adjoint(torch.ones_like(rn.rad))
    assert e.value.status == T.E_STATE
    with pytest.raises(T.TurscaError) as e:
        rn.get(T.F_VAL, rn.stats.nnz, rn.dtype)
    assert e.value.status == T.E_STATE
    full1, _ = run_single(rn, single=False)
    assert np.array_equal(full0, full1)
    assert np.all(ss <= full0) and (ss < full0).mean() > 0.9
    r = O.run(sc, flags=O.SINGLE_SCATTER)
    assert rel_err(ss, r["rad"]).max() < 1e-4
