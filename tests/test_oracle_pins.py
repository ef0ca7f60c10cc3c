"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a textbook special case or brute force on tiny inputs.
Citations name the section / equation of Mikkonen et al. (scattering graph
method) that the checked function implements.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_16037_gb300 import scenes


def hg(g, mu):
    return (1 - g * g) / (4 * math.pi * (1 + g * g - 2 * g * mu) ** 1.5)


def hg_vec(g, mu):
    return (1 - g * g) / (4 * np.pi * (1 + g * g - 2 * g * mu) ** 1.5)


def sun_vec(sza, saa):
    t, p = math.radians(sza), math.radians(saa)
    return -np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])


def view_vec(vza, vaa):
    t, p = math.radians(vza), math.radians(vaa)
    return np.array([math.sin(t) * math.cos(p), math.sin(t) * math.sin(p), math.cos(t)])


# --------------------------------------------------------------------------
# Directions and stencil (Sec. 2 coupling graph restricted to a voxel stencil)

@pytest.mark.parametrize("R,n,up,hor,down,ng,nmem", [(1, 26, 9, 8, 9, 9, 9), (2, 98, 41, 16, 41, 49, 50)])
def test_direction_counts(R, n, up, hor, down, ng, nmem):
    sc = scenes.make_layered(6, 6, 4, [0.1] * 4, [0.5], R=R, M=512)
    r = O.run(sc, flags=O.NO_SOLVE)
    d = r["dirs"]
    assert r["n_dirs"] == n
    assert (d[:, 2] > 0).sum() == up and (d[:, 2] == 0).sum() == hor and (d[:, 2] < 0).sum() == down
    assert r["n_gdirs"] == ng and r["gdir_nmem"].sum() == nmem
    # the stencil offsets k*u cover the Chebyshev ball exactly once
    offs = set()
    for u, km in zip(d, r["kmax"]):
        for k in range(1, km + 1):
            o = tuple(int(v) for v in k * u)
            assert o not in offs
            offs.add(o)
    assert len(offs) == (2 * R + 1) ** 3 - 1


# --------------------------------------------------------------------------
# P1: voxel traversal (Beer-Lambert optical depth, Eq. radiance_effectuality)

def brute_tau(mu_e, n, P, V, tend, lphys):
    """Exact rational traversal: all plane crossings, midpoint cell of each piece."""
    nz, ny, nx = n
    ts = {Fraction(0), Fraction(tend)}
    for a in range(3):
        if V[a] == 0:
            continue
        lo, hi = sorted([P[a], P[a] + V[a] * tend])
        for b in range(math.floor(lo), math.ceil(hi) + 1):
            t = (Fraction(b) - P[a]) / V[a]
            if 0 < t < tend:
                ts.add(t)
    ts = sorted(ts)
    tau = Fraction(0)
    for t0, t1 in zip(ts[:-1], ts[1:]):
        tm = (t0 + t1) / 2
        c = [math.floor(P[a] + V[a] * tm) for a in range(3)]
        cell = (c[2] * ny + c[1] % ny) * nx + c[0] % nx
        tau += Fraction(mu_e[cell]) * (t1 - t0)
    return float(tau) * lphys


def test_p1_dda_brute_force():
    rng = np.random.default_rng(1)
    nx, ny, nz = 3, 4, 5
    sc = scenes.make_layered(nx, ny, nz, [0.1] * nz, [0.5])
    mu_e = rng.lognormal(0, 1, nx * ny * nz)
    worst = 0.0
    for trial in range(300):
        # dyadic rationals: exact in FP64 and in Fractions
        P = [Fraction(int(rng.integers(0, 64 * nx)), 64), Fraction(int(rng.integers(0, 64 * ny)), 64),
             Fraction(int(rng.integers(1, 64 * nz - 1)), 64)]
        if trial % 3 == 0:  # lattice-like: centres and integer directions (corner ties)
            P = [Fraction(int(rng.integers(0, nx))) + Fraction(1, 2), Fraction(int(rng.integers(0, ny))) + Fraction(1, 2),
                 Fraction(int(rng.integers(0, nz))) + Fraction(1, 2)]
            V = [Fraction(int(v)) for v in rng.integers(-2, 3, 3)]
        else:
            V = [Fraction(int(v), 8) for v in rng.integers(-24, 25, 3)]
        if V[2] == 0 and V[0] == 0 and V[1] == 0:
            continue
        # stay inside the slab vertically
        if V[2] > 0:
            tmax = (nz - P[2]) / V[2]
        elif V[2] < 0:
            tmax = P[2] / -V[2]
        else:
            tmax = Fraction(7)
        tend = min(tmax, Fraction(int(rng.integers(1, 40)), 8))
        lphys = 0.37
        ref = brute_tau(mu_e, (nz, ny, nx), P, V, tend, lphys)
        got = O.tau_segment(sc, mu_e, [float(p) for p in P], [float(v) for v in V], float(tend), lphys)
        if ref > 0:
            worst = max(worst, abs(got - ref) / ref)
        else:
            assert got == 0.0
    assert worst < 1e-14


def test_p1_dda_homogeneous_length():
    rng = np.random.default_rng(2)
    nx, ny, nz = 5, 4, 6
    sc = scenes.make_layered(nx, ny, nz, [0.1] * nz, [0.5], h=(0.07, 0.05, 0.11))
    mu_e = np.full(nx * ny * nz, 0.731)
    for _ in range(200):
        P = rng.uniform([0, 0, 0.01], [nx, ny, nz - 0.01])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        V = d / np.array([sc.hx, sc.hy, sc.hz])  # cell units per km
        tmax = (nz - P[2]) / V[2] if V[2] > 0 else P[2] / -V[2]
        L = min(tmax, rng.uniform(0.01, 3.0))
        tau = O.tau_segment(sc, mu_e, P, V, L, 1.0)
        assert abs(tau - 0.731 * L) <= 1e-14 * 0.731 * L


# --------------------------------------------------------------------------
# P2: Beer-Lambert slab closed form (no scattering, Lambertian ground)

@pytest.mark.parametrize("R", [1, 2])
def test_p2_beer_lambert_slab(R):
    nz = 7
    me = [0.3, 0.1, 0.25, 0.6, 0.05, 0.2, 0.4]
    for A in (0.3, 0.0):
        sc = scenes.make_layered(6, 5, nz, me, [0.0], albedo=A, R=R, sza=40.0, saa=33.0, vza=25.0, vaa=250.0,
                                 h=(0.08, 0.1, 0.12), M=1024)
        r = O.run(sc)
        tau = sum(me) * sc.hz
        mu0, muv = math.cos(math.radians(40.0)), math.cos(math.radians(25.0))
        L = A * mu0 / math.pi * math.exp(-tau / mu0) * math.exp(-tau / muv)
        if A > 0:
            np.testing.assert_allclose(r["rad"], L, rtol=1e-14, atol=0)
            np.testing.assert_allclose(r["refl"], math.pi * L / mu0, rtol=1e-14)
        else:
            assert np.all(r["rad"] == 0.0)


# --------------------------------------------------------------------------
# P3: discrete single-scattering closed form (homogeneous periodic slab)

def l_ss_discrete(omega, g, sza, vza, mu_e, hz, nz, cosang):
    mu0, muv = math.cos(math.radians(sza)), math.cos(math.radians(vza))
    dt = mu_e * hz
    a = 1 / mu0 + 1 / muv
    return (omega * mu0 * hg(g, cosang) * (1 - math.exp(-dt / mu0)) * (1 - math.exp(-dt / muv)) / dt
            * (1 - math.exp(-nz * dt * a)) / (1 - math.exp(-dt * a)))


@pytest.mark.parametrize("R,sza,saa,vza,vaa", [(1, 30, 0, 0, 0), (2, 55, 40, 35, 300), (2, 10, 180, 50, 90)])
def test_p3_single_scatter_closed_form(R, sza, saa, vza, vaa):
    nz, mu_e, om, g = 9, 0.8, 0.7, 0.6
    sc = scenes.make_layered(6, 6, nz, [mu_e] * nz, [om], g=(g,), albedo=0.0, R=R, sza=sza, saa=saa,
                             vza=vza, vaa=vaa, h=(0.1, 0.12, 0.07), M=1024)
    r = O.run(sc, flags=O.SINGLE_SCATTER)
    ca = float(sun_vec(sza, saa) @ view_vec(vza, vaa))
    ref = l_ss_discrete(om, g, sza, vza, mu_e, sc.hz, nz, ca)
    np.testing.assert_allclose(r["rad"], ref, rtol=1e-13)


# --------------------------------------------------------------------------
# P4: single-scattering limits

def test_p4_ms_vanishes_linearly_in_omega():
    nz = 6
    rel = []
    oms = [4e-3, 2e-3, 1e-3]
    for om in oms:
        sc = scenes.make_layered(6, 6, nz, [0.5] * nz, [om], g=(0.5,), albedo=0.0, R=1, sza=35, vza=20,
                                 saa=0, vaa=90, M=1024)
        full = O.run(sc)["rad"].mean()
        ss = O.run(sc, flags=O.SINGLE_SCATTER)["rad"].mean()
        rel.append((full - ss) / ss)
    slope = np.polyfit(np.log(oms), np.log(rel), 1)[0]
    assert abs(slope - 1.0) < 0.05


def test_p4_single_scatter_continuum_limit():
    sza, vza, g, om, tau = 40.0, 20.0, 0.5, 0.8, 0.9
    mu0, muv = math.cos(math.radians(sza)), math.cos(math.radians(vza))
    ca = float(sun_vec(sza, 0) @ view_vec(vza, 0))
    cont = om * hg(g, ca) * mu0 / (mu0 + muv) * (1 - math.exp(-tau * (1 / mu0 + 1 / muv)))
    errs, hs = [], []
    for nz in (4, 8, 16):
        hz = 1.0 / nz
        sc = scenes.make_layered(4, 4, nz, [tau] * nz, [om], g=(g,), albedo=0.0, R=1, sza=sza, vza=vza,
                                 h=(0.25, 0.25, hz), M=512)
        L = O.run(sc, flags=O.SINGLE_SCATTER)["rad"].mean()
        errs.append(abs(L - cont))
        hs.append(hz)
    order = np.polyfit(np.log(hs), np.log(errs), 1)[0]
    assert abs(order - 2.0) < 0.1


# --------------------------------------------------------------------------
# P5: energy conservation at omega = 1 with a black surface

@pytest.mark.parametrize("R,sza,saa", [(1, 35.0, 10.0), (2, 62.0, 130.0)])
def test_p5_energy_conservation(R, sza, saa):
    nx, ny, nz = 6, 5, 7
    rng = np.random.default_rng(5)
    me = rng.uniform(0.1, 2.0, nz)
    sc = scenes.make_layered(nx, ny, nz, me, [1.0], g=(0.6,), albedo=0.0, R=R, sza=sza, saa=saa,
                             vza=10, h=(0.1, 0.08, 0.12), M=2048)
    r = O.run(sc, gmres_tol=1e-15)
    na = r["n_atm"]
    mu0 = math.cos(math.radians(sza))
    incident = nx * ny * mu0 * sc.hx * sc.hy
    escape = float(r["e1"] @ r["esc_sun"] + r["x"] @ r["esc_iso"])
    direct_ground = float(mu0 * sc.hx * sc.hy * r["tsun"][na:].sum())
    row, col = r["slot_row"], r["slot_col"]
    gnd = row >= na
    deposited_ground = float((r["slot_depsun"][gnd] * r["e1"][col[gnd]]).sum()
                             + (r["slot_dep"][gnd] * r["x"][col[gnd]]).sum())
    total = escape + direct_ground + deposited_ground
    assert abs(total - incident) <= 1e-12 * incident


@pytest.mark.parametrize("R,sza,saa,A", [(1, 35.0, 10.0, 0.3), (2, 62.0, 130.0, 0.8), (2, 20.0, 250.0, 0.5)])
def test_p5_energy_conservation_with_a_reflecting_ground(R, sza, saa, A):
    """omega = 1 and a Lambertian ground of albedo A: the ground re-emits the
    fraction A of what reaches it (e1_c + x_c, routed by the Lambertian
    weights q^lamb over the ground chains) and absorbs the rest, so
    incident = TOA escape + (1 - A) (direct + diffuse power reaching the ground)."""
    nx, ny, nz = 6, 5, 7
    rng = np.random.default_rng(7)
    me = rng.uniform(0.1, 2.0, nz)
    sc = scenes.make_layered(nx, ny, nz, me, [1.0], g=(0.6,), albedo=A, R=R, sza=sza, saa=saa,
                             vza=10, h=(0.1, 0.08, 0.12), M=2048)
    r = O.run(sc, gmres_tol=1e-15)
    na = r["n_atm"]
    mu0 = math.cos(math.radians(sza))
    incident = nx * ny * mu0 * sc.hx * sc.hy
    escape = float(r["e1"] @ r["esc_sun"] + r["x"] @ r["esc_iso"])
    direct_ground = float(mu0 * sc.hx * sc.hy * r["tsun"][na:].sum())
    row, col = r["slot_row"], r["slot_col"]
    gnd = row >= na
    diffuse_ground = float((r["slot_depsun"][gnd] * r["e1"][col[gnd]]).sum()
                           + (r["slot_dep"][gnd] * r["x"][col[gnd]]).sum())
    # what the ground re-emits is A times what reaches it
    np.testing.assert_allclose(r["e1"][na:], A * mu0 * sc.hx * sc.hy * r["tsun"][na:], rtol=1e-14)
    reemitted = float(r["e1"][na:].sum() + r["x"][na:].sum())
    assert abs(reemitted - A * (direct_ground + diffuse_ground)) <= 1e-12 * incident
    # the ground's own chains carry part of the escape
    assert float(r["e1"][na:] @ r["esc_sun"][na:] + r["x"][na:] @ r["esc_iso"][na:]) > 0.01 * escape
    total = escape + (1.0 - A) * (direct_ground + diffuse_ground)
    assert abs(total - incident) <= 1e-12 * incident


# --------------------------------------------------------------------------
# P6: horizontal translation invariance / equivariance (periodic x, y)

@pytest.mark.parametrize("R", [1, 2])
def test_p6_translation_invariance(R):
    nz = 6
    rng = np.random.default_rng(6)
    sc = scenes.make_layered(6, 6, nz, rng.uniform(0.2, 1.5, nz), rng.uniform(0.5, 0.95, nz), g=(0.7,),
                             albedo=0.25, R=R, sza=50, saa=20, vza=30, vaa=200, M=2048)
    r = O.run(sc)
    L = r["rad"]
    assert (L.max() - L.min()) <= 1e-13 * L.mean()
    x = r["x"][: r["n_atm"]].reshape(nz, 6, 6)
    spread = (x.max(axis=(1, 2)) - x.min(axis=(1, 2))) / x.mean(axis=(1, 2))
    assert spread.max() <= 1e-13


def test_p6_shift_equivariance():
    sc = scenes.make_random(6, 5, 4, seed=3, S=2, R=2, M=1024)
    r0 = O.run(sc)
    sh = sc.copy()
    sh.mu_a = np.roll(sc.mu_a, (2, 1), axis=(2, 1))
    sh.mu_s = np.roll(sc.mu_s, (2, 1), axis=(3, 2))
    r1 = O.run(sh)
    np.testing.assert_allclose(r1["rad"], np.roll(r0["rad"], (1, 2), axis=(0, 1)), rtol=1e-12)


def test_p9_mirror_single_scatter():
    # y-mirror with sun and sensor in the x-z plane: the single-scattered and
    # surface-reflected image mirrors exactly (the Fibonacci lattice is not
    # mirror symmetric, so orders >= 2 are excluded)
    sc = scenes.make_random(6, 6, 4, seed=9, S=2, R=2, M=1024, saa=0.0, vaa=0.0, vza=30.0, sza=50.0)
    r0 = O.run(sc, flags=O.SINGLE_SCATTER)
    mi = sc.copy()
    mi.mu_a = sc.mu_a[:, ::-1, :].copy()
    mi.mu_s = sc.mu_s[:, :, ::-1, :].copy()
    r1 = O.run(mi, flags=O.SINGLE_SCATTER)
    np.testing.assert_allclose(r1["rad"], r0["rad"][::-1, :], rtol=1e-13)


# --------------------------------------------------------------------------
# P7: the solve of Eq. flux_system against a dense direct solve; the series
# of Eq. fs_sum increases monotonically to the same x

@pytest.mark.parametrize("maker", [
    lambda: scenes.make_plain(),
    lambda: scenes.make_random(4, 4, 4, seed=1, R=1, M=512),
    lambda: scenes.make_random(5, 5, 4, seed=2, R=2, M=512),
])
def test_p7_dense_solve_and_series(maker):
    sc = maker()
    r = O.run(sc)
    K = O.dense(r)
    n = K.shape[0]
    x = np.linalg.solve(np.eye(n) - K, r["s"])
    np.testing.assert_allclose(r["x"], x, rtol=1e-12, atol=1e-12 * np.abs(x).max())
    part = r["s"].copy()
    term = r["s"].copy()
    for _ in range(60):
        term = K @ term
        nxt = part + term
        assert np.all(nxt >= part)
        part = nxt
    assert np.abs(part - x).max() <= 1e-6 * np.abs(x).max()
    assert max(abs(np.linalg.eigvals(K))) < 1.0


# --------------------------------------------------------------------------
# P8: every unit of power leaving a node is deposited or escapes

@pytest.mark.parametrize("maker", [
    lambda: scenes.make_plain(),
    lambda: scenes.make_random(5, 6, 5, seed=4, R=2, M=1024),
    lambda: scenes.make_random(5, 5, 2, seed=5, R=2, M=1024),   # thinner than the stencil
])
def test_p8_column_identity(maker):
    sc = maker()
    r = O.run(sc, flags=O.NO_SOLVE)
    nn = r["n_nodes"]
    for dep, esc in (("slot_dep", "esc_iso"), ("slot_depsun", "esc_sun")):
        tot = np.zeros(nn)
        np.add.at(tot, r["slot_col"], r[dep])
        np.testing.assert_allclose(tot + r[esc], 1.0, atol=1e-14)
    # sum_u q c = 1 expressed through the normalisers: z = sum qC / sum q
    assert np.all(r["z_iso"] > 0)


# --------------------------------------------------------------------------
# Chain deposits in a homogeneous medium: closed forms of the three cases

def test_chain_cases_closed_form():
    nx, ny, nz, me = 6, 6, 5, 0.9
    sc = scenes.make_layered(nx, ny, nz, [me] * nz, [0.5], albedo=0.3, R=1, h=(0.1, 0.1, 0.1), M=2048,
                             coupling=0)
    r = O.run(sc, flags=O.NO_SOLVE)
    dirs = [tuple(d) for d in r["dirs"]]
    q = r["q_iso"]
    na = r["n_atm"]
    row, col, dr, k, dep = r["slot_row"], r["slot_col"], r["slot_dir"], r["slot_k"], r["slot_dep"]

    def node(ix, iy, iz):
        return (iz * ny + iy % ny) * nx + ix % nx

    def slots(j, u):
        m = (col == j) & (dr == u)
        return {(int(a), int(b)): float(v) for a, b, v in zip(row[m], k[m], dep[m])}

    h = 0.1
    # (c) diagonal down from the bottom layer: the ground is hit at a corner
    u = dirs.index((1, 1, -1))
    j = node(2, 3, 0)
    L = h * math.sqrt(3)
    s = slots(j, u)
    Th = math.exp(-me * L / 2)
    assert abs(s[(j, O.K_SELF)] - q[u] * (1 - Th)) < 1e-15
    cols = [na + (3 + dy) * nx + (2 + dx) for dx in (0, 1) for dy in (0, 1)]
    for c in cols:
        assert abs(s[(c, O.K_GROUND)] - q[u] * Th / 4) < 1e-15
    # (b) up from the top layer: self-deposit and escape
    u = dirs.index((0, 1, 1))
    j = node(1, 1, nz - 1)
    L = h * math.sqrt(2)
    s = slots(j, u)
    assert abs(s[(j, O.K_SELF)] - q[u] * (1 - math.exp(-me * L / 2))) < 1e-15
    # (a) up from an interior voxel: p1 gets its segment plus the extinction
    # beyond the stencil up to the TOA; horizontal: p1 takes everything
    u = dirs.index((1, 0, 1))
    j = node(0, 0, 1)
    L = h * math.sqrt(2)
    s = slots(j, u)
    p1 = node(1, 0, 2)
    dist_top = (nz - 2.5) * L  # from the centre of layer 2 to the TOA along u
    expect = (1 - math.exp(-me * L)) + math.exp(-me * L) * (1 - math.exp(-me * dist_top))
    assert abs(s[(p1, 1)] - q[u] * expect) < 1e-15
    u = dirs.index((-1, 0, 0))
    s = slots(j, u)
    assert abs(s[(node(-1, 0, 1), 1)] - q[u]) < 1e-15


def test_coupling_weight_eq_scatt_coup():
    """Eq. scatt_coup through the assembled matrix: with uniform extinction,
    the horizontal chains of one source deposit everything at their first
    node, so deposit ratios of opposite / perpendicular neighbours equal the
    coupling ratio sqrt(mu_s(n) mu_s(j)) / |r_n - r_j|."""
    nx, ny, nz = 6, 6, 3
    rng = np.random.default_rng(8)
    me = 1.2
    mus = rng.uniform(0.1, 1.1, (nz, ny, nx))
    sc = scenes.Scene(nx, ny, nz, 0.07, 0.11, 0.1, mu_a=me - mus, mu_s=mus[None], g=np.array([0.3]),
                      albedo=0.2, R=1, M=4096)
    r = O.run(sc, flags=O.NO_SOLVE)
    dirs = [tuple(d) for d in r["dirs"]]
    q = r["q_iso"]
    row, col, dr, dep = r["slot_row"], r["slot_col"], r["slot_dir"], r["slot_dep"]
    j = (1 * ny + 2) * nx + 3
    flat = mus.ravel()

    def d_of(u):
        m = (col == j) & (dr == dirs.index(u))
        assert m.sum() == 1
        return float(dep[m][0]), int(row[m][0])

    (dp, np_), (dm, nm) = d_of((1, 0, 0)), d_of((-1, 0, 0))
    (dyp, nyp) = d_of((0, 1, 0))
    qp, qm, qy = q[dirs.index((1, 0, 0))], q[dirs.index((-1, 0, 0))], q[dirs.index((0, 1, 0))]
    np.testing.assert_allclose((dp / qp) / (dm / qm), math.sqrt(flat[np_] / flat[nm]), rtol=1e-13)
    np.testing.assert_allclose((dp / qp) / (dyp / qy), math.sqrt(flat[np_] / flat[nyp]) * 0.11 / 0.07, rtol=1e-13)
    # invariance: scaling every mu_s by a constant at fixed extinction leaves
    # the routing weights unchanged
    sc2 = sc.copy()
    sc2.mu_s = 0.5 * sc.mu_s
    sc2.mu_a = me - sc2.mu_s[0]
    r2 = O.run(sc2, flags=O.NO_SOLVE)
    np.testing.assert_allclose(r2["slot_dep"], r["slot_dep"], rtol=1e-13, atol=1e-17)
    # no coupling: every direction keeps its quadrature weight
    sc3 = sc.replace(coupling=0)
    r3 = O.run(sc3, flags=O.NO_SOLVE)
    assert np.all(r3["z_iso"] == 1.0)


# --------------------------------------------------------------------------
# P10: quadrature of Eq. F_term_phase on the Fibonacci lattice

def test_p10_quadrature_sums_and_hg_normalisation():
    for R in (1, 2):
        sc = scenes.make_random(5, 5, 3, seed=1, S=2, R=R, M=8192)
        r = O.run(sc, flags=O.NO_SOLVE)
        assert abs(r["q_iso"].sum() - 1) < 1e-14
        assert abs(r["q_lamb"].sum() - 1) < 1e-14
        np.testing.assert_allclose(r["q_sun"].sum(axis=1), 1.0, atol=1e-14)
    pts = O.fibonacci(8192)
    np.testing.assert_allclose(np.linalg.norm(pts, axis=1), 1.0, atol=1e-15)
    assert abs(pts.mean(axis=0)).max() < 1e-3
    for g in (0.0, 0.3, 0.65, 0.85):
        for s0 in (np.array([0, 0, -1.0]), sun_vec(63, 27)):
            val = np.array([hg(g, mu) for mu in pts @ s0]).sum() * 4 * math.pi / 8192
            assert abs(val - 1) < 1e-3


def test_p10_cells_converge_to_spherical_voronoi():
    sv_mod = pytest.importorskip("scipy.spatial")
    for R, h in ((1, (0.1, 0.1, 0.1)), (2, (0.05, 0.05, 0.1))):
        sc = scenes.make_layered(5, 5, 3, [0.1] * 3, [0.5], R=R, h=h, M=8192)
        r8 = O.run(sc, flags=O.NO_SOLVE)
        u = r8["dirs"] * np.array(h)
        u = u / np.linalg.norm(u, axis=1, keepdims=True)
        sv = sv_mod.SphericalVoronoi(u, radius=1.0)
        area = sv.calculate_areas() / (4 * math.pi)
        e8 = np.abs(r8["q_iso"] - area).max()
        rb = O.run(sc.replace(M=262144), flags=O.NO_SOLVE)
        eb = np.abs(rb["q_iso"] - area).max()
        assert eb < 2.5e-4 and eb < e8


# Per-cell weights of Eq. F_term_phase, pinned to integrals over the exact
# spherical-Voronoi cells of the directions (Sec. 3: each lattice point belongs
# to its nearest coupled direction, so as M grows a cell's lattice sum tends
# to the integral over that direction's Voronoi cell).  The cells come from
# SciPy; the integrals are computed here, independently of the lattice: HG by
# recursive subdivision of each cell into small spherical triangles (exact
# areas, edge-midpoint rule), the cosine weight of the Lambertian ground in
# closed form from the polygon's first moment.

def _nrm(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _moment(poly):
    """First moment (integral of the unit vector) of a spherical polygon whose
    vertices run counter-clockwise seen from outside: half the sum over the
    edges of the arc angle times the unit normal of the edge's plane (the
    divergence theorem on the cone over the polygon)."""
    m = np.zeros(3)
    for a, b in zip(poly, np.roll(poly, -1, axis=0)):
        c = np.cross(a, b)
        s = np.linalg.norm(c)
        if s > 0.0:
            m += 0.5 * math.atan2(s, float(a @ b)) * c / s
    return m


def _voronoi_cells(gen):
    """Vertex loops of the spherical-Voronoi cells of unit vectors gen,
    oriented counter-clockwise seen from outside (the cell's moment points
    toward its generator)."""
    sv_mod = pytest.importorskip("scipy.spatial")
    sv = sv_mod.SphericalVoronoi(gen, radius=1.0)
    sv.sort_vertices_of_regions()
    out = []
    for k, reg in enumerate(sv.regions):
        poly = sv.vertices[reg]
        out.append(poly if _moment(poly) @ gen[k] > 0 else poly[::-1])
    return out


def _tri_area(a, b, c):
    num = np.abs(np.einsum("ij,ij->i", a, np.cross(b, c)))
    den = 1.0 + (a * b).sum(1) + (b * c).sum(1) + (c * a).sum(1)
    return 2.0 * np.arctan2(num, den)  # Van Oosterom & Strackee


def _cell_integral(gen, poly, f, level=5):
    """Integral of f over the convex spherical polygon poly containing gen:
    the fan of triangles (gen, v_k, v_k+1), each split 4**level times."""
    A = np.repeat(gen[None], len(poly), 0)
    B, C = poly, np.roll(poly, -1, axis=0)
    for _ in range(level):
        ab, bc, ca = _nrm(A + B), _nrm(B + C), _nrm(C + A)
        A, B, C = (np.concatenate(t) for t in ((A, ab, ca, ab), (ab, B, bc, bc), (ca, bc, C, ca)))
    mid = (f(_nrm(A + B)) + f(_nrm(B + C)) + f(_nrm(C + A))) / 3.0
    return float((_tri_area(A, B, C) * mid).sum())


def _clip_upper(poly):
    """The part z >= 0 of a convex spherical polygon (great-circle clipping)."""
    out = []
    for P, Q in zip(poly, np.roll(poly, -1, axis=0)):
        if P[2] >= 0.0:
            out.append(P)
        if (P[2] >= 0.0) != (Q[2] >= 0.0):
            out.append(_nrm(abs(Q[2]) * P + abs(P[2]) * Q))
    return np.array(out)


def test_p10_hg_helper_has_unit_norm_and_mean_cosine_g():
    """The textbook HG used by these pins: unit integral over the sphere and
    mean cosine g (Gauss-Legendre in mu, exact to rounding here)."""
    x, w = np.polynomial.legendre.leggauss(400)
    for g in (0.0, 0.3, 0.65, 0.85):
        f = np.array([hg(g, mu) for mu in x])
        assert abs(2 * math.pi * (w * f).sum() - 1.0) < 1e-11
        assert abs(2 * math.pi * (w * f * x).sum() - g) < 1e-11


@pytest.mark.parametrize("R,sza,saa", [(1, 30.0, 0.0), (1, 63.0, 27.0), (2, 30.0, 0.0), (2, 63.0, 27.0)])
def test_p10_sun_weights_converge_to_hg_over_voronoi_cells(R, sza, saa):
    """q^sun[s, u] tends to the integral of HG_g(s0 . s) over the Voronoi cell
    of u (s0 the sun's propagation direction), for g = 0.3 and 0.85."""
    h = (0.1, 0.1, 0.1) if R == 1 else (0.05, 0.05, 0.1)
    sc = scenes.make_random(5, 5, 3, seed=3, S=2, R=R, h=h, sza=sza, saa=saa, M=8192, precision=0)
    sc = sc.replace(g=np.array([0.3, 0.85]))
    r8 = O.run(sc, flags=O.NO_SOLVE)
    rb = O.run(sc.replace(M=1 << 20), flags=O.NO_SOLVE)
    gen = _unit_dirs(r8, h)
    cells = _voronoi_cells(gen)
    s0 = sun_vec(sza, saa)
    for sp, g in enumerate(sc.g):
        ref = np.array([_cell_integral(gen[u], cells[u], lambda s: hg_vec(g, s @ s0)) for u in range(len(gen))])
        assert abs(ref.sum() - 1.0) < 1e-6  # the subdivision integrates the whole sphere
        e8 = np.abs(r8["q_sun"][sp] - ref).max()
        eb = np.abs(rb["q_sun"][sp] - ref).max()
        assert eb < 4e-4 and eb < e8 / 8, (g, e8, eb)


@pytest.mark.parametrize("R,h", [(1, (0.1, 0.1, 0.1)), (2, (0.05, 0.05, 0.1)), (2, (0.1, 0.08, 0.12))])
def test_p10_lambertian_weights_converge_to_cosine_over_voronoi_cells(R, h):
    """q^lamb[u] tends to (1/pi) times the integral of cos(theta) over the
    upper half of the Voronoi cell of ground direction u.  The cells are those
    of the ground directions plus the nadir, whose cell lies below the horizon
    (the bisector of the nadir and a direction at elevation e sits at (e - 90)/2)
    and keeps the set from lying in one hemisphere."""
    sc = scenes.make_layered(5, 5, 3, [0.1] * 3, [0.5], R=R, h=h, M=8192)
    r8 = O.run(sc, flags=O.NO_SOLVE)
    rb = O.run(sc.replace(M=1 << 20), flags=O.NO_SOLVE)
    m = r8["gdir_mem"][:, 0, :].astype(np.float64)
    gen = _nrm(np.stack([m[:, 0] * h[0], m[:, 1] * h[1], (m[:, 2] - 0.5) * h[2]], axis=1))
    cells = _voronoi_cells(np.vstack([gen, [[0.0, 0.0, -1.0]]]))
    assert np.all(cells[-1][:, 2] < 0.0)
    ref = np.array([_moment(_clip_upper(cells[u]))[2] / math.pi for u in range(len(gen))])
    assert abs(ref.sum() - 1.0) < 1e-13  # the upper hemisphere's cosine integral is pi
    e8 = np.abs(r8["q_lamb"] - ref).max()
    eb = np.abs(rb["q_lamb"] - ref).max()
    assert eb < 1e-4 and eb < e8 / 8, (e8, eb)


@pytest.mark.parametrize("sza,saa", [(20.0, 0.0), (40.0, 10.0), (45.0, 60.0), (63.0, 27.0), (75.0, 200.0)])
def test_p10_sun_weights_peak_forward(sza, saa):
    """Sign of the scattering angle: for a forward-peaked phase function
    (g = 0.85, forward / backward HG ratio ((1 + g) / (1 - g))^3 = 1876) the
    mean HG over a cell (q^sun / q^iso) peaks among the directions nearest
    the sun's propagation direction s0 and bottoms out among those nearest
    -s0 (the cells' shapes decide between near neighbours)."""
    h = (0.05, 0.05, 0.1)
    sc = scenes.make_random(5, 5, 3, seed=3, S=1, R=2, h=h, sza=sza, saa=saa, M=8192, precision=0)
    r = O.run(sc.replace(g=np.array([0.85])), flags=O.NO_SOLVE)
    u = _unit_dirs(r, h)
    s0 = sun_vec(sza, saa)
    mean_hg = r["q_sun"][0] / r["q_iso"]
    fwd, back = np.argsort(-(u @ s0))[:3], np.argsort(u @ s0)[:3]
    assert np.argmax(mean_hg) in fwd and np.argmin(mean_hg) in back
    assert mean_hg[fwd[0]] > 100.0 * mean_hg[back[0]]


# --------------------------------------------------------------------------
# P11: coupling selection (scattering graph with C > c_min, Sec. 2) and the
# re-partition of the lattice among the kept directions

def _unit_dirs(r, h):
    u = r["dirs"] * np.array(h)
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def test_p11_threshold_below_every_coupling_is_the_full_stencil():
    """Every voxel scatters and the surface reflects, so every coupling is
    positive: a threshold below all of them keeps the full stencil.  With
    non-scattering voxels the zero couplings go at any c_min > 0."""
    sc = scenes.make_random(9, 8, 5, seed=21, S=2, R=2, M=1024, zero_frac=0.0)
    r0 = O.run(sc)
    r1 = O.run(sc.replace(c_min=1e-300))
    for k in ("slot_val", "slot_valsun", "x", "rad"):
        assert np.array_equal(r0[k], r1[k]), k
    sz = scenes.make_random(9, 8, 5, seed=21, S=1, R=2, M=1024, zero_frac=0.1)
    z0, z1 = O.run(sz, flags=O.NO_SOLVE), O.run(sz.replace(c_min=1e-300), flags=O.NO_SOLVE)
    assert (z1["slot_val"] != 0).sum() < (z0["slot_val"] != 0).sum()


def test_p11_partition_with_every_direction_kept_is_the_global_quadrature():
    sc = scenes.make_random(5, 5, 3, seed=1, S=2, R=2, M=4096)
    r = O.run(sc, flags=O.NO_SOLVE)
    qi, qs = O.partition(sc, np.ones(r["n_dirs"], dtype=int))
    assert np.array_equal(qi, r["q_iso"]) and np.array_equal(qs, r["q_sun"])
    assert np.array_equal(O.partition(sc, np.ones(r["n_gdirs"], dtype=int), ground=True), r["q_lamb"])


@pytest.mark.parametrize("R", [1, 2])
def test_p11_partition_conserves_the_sphere(R):
    """Dropped cells hand all their points to kept directions: the weights
    still sum to one, dropped directions get nothing, kept cells only grow."""
    sc = scenes.make_random(5, 5, 3, seed=2, S=3, R=R, M=4096)
    r = O.run(sc, flags=O.NO_SOLVE)
    rng = np.random.default_rng(R)
    for frac in (0.2, 0.6, 0.95):
        kept = rng.random(r["n_dirs"]) > frac
        kept[rng.integers(r["n_dirs"])] = True
        qi, qs = O.partition(sc, kept.astype(int))
        assert abs(qi.sum() - 1) < 1e-14
        np.testing.assert_allclose(qs.sum(axis=1), 1.0, atol=1e-13)
        assert not qi[~kept].any() and not qs[:, ~kept].any()
        assert np.all(qi[kept] >= r["q_iso"][kept]) and np.all(qs[:, kept] >= r["q_sun"][:, kept])
        kg = rng.random(r["n_gdirs"]) > frac
        kg[rng.integers(r["n_gdirs"])] = True
        ql = O.partition(sc, kg.astype(int), ground=True)
        assert abs(ql.sum() - 1) < 1e-14 and not ql[~kg].any() and np.all(ql[kg] >= r["q_lamb"][kg])
    none = O.partition(sc, np.zeros(r["n_dirs"], dtype=int))
    assert not none[0].any() and not none[1].any()


def test_p11_kept_cells_converge_to_the_spherical_voronoi_of_the_kept_set():
    sv_mod = pytest.importorskip("scipy.spatial")
    h = (0.05, 0.05, 0.1)
    sc = scenes.make_layered(5, 5, 3, [0.1] * 3, [0.5], R=2, h=h, M=8192)
    r = O.run(sc, flags=O.NO_SOLVE)
    kept = np.random.default_rng(11).random(r["n_dirs"]) < 0.4
    u = _unit_dirs(r, h)[kept]
    area = sv_mod.SphericalVoronoi(u, radius=1.0).calculate_areas() / (4 * math.pi)
    e8 = np.abs(O.partition(sc, kept.astype(int))[0][kept] - area).max()
    eb = np.abs(O.partition(sc.replace(M=262144), kept.astype(int))[0][kept] - area).max()
    assert eb < 2.5e-4 and eb < e8


def test_p11_kept_set_of_a_homogeneous_medium_is_the_short_directions():
    """In a homogeneous medium C = mu_s / |r' - r|, so a source keeps exactly
    the directions shorter than mu_s / c_min (plus those leaving the domain
    without a receiver)."""
    h = (0.1, 0.08, 0.12)
    mus = 1.3
    sc = scenes.make_layered(7, 6, 6, [2.0] * 6, [mus / 2.0], g=(0.5,), albedo=0.3, R=2, h=h, M=2048)
    r0 = O.run(sc, flags=O.NO_SOLVE)

    def length(v):  # physical length of a lattice vector, summed in x, y, z order
        p = [v[0] * h[0], v[1] * h[1], v[2] * h[2]]
        return math.sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2])

    L = np.array([length(v) for v in r0["dirs"].tolist()])
    # the threshold equals the coupling of the sixth-shortest length exactly:
    # those directions go too (the graph keeps C > c_min)
    c_min = mus / np.unique(L)[5]
    r = O.run(sc.replace(c_min=c_min), flags=O.NO_SOLVE)
    nx, ny = sc.nx, sc.ny
    j = (3 * ny + 2) * nx + 3  # an interior source: every chain has a voxel receiver
    want = {u for u in range(r["n_dirs"]) if mus / L[u] > c_min}
    assert 0 < len(want) < r["n_dirs"]
    for w in ("slot_dep", "slot_depsun"):
        sel = (r["slot_col"] == j) & (r[w] != 0)
        assert set(r["slot_dir"][sel].tolist()) == want, w


def test_p11_nonzero_couplings_shrink_as_the_threshold_grows():
    sc = scenes.make_random(8, 7, 5, seed=22, S=2, R=2, M=1024)
    prev = None
    for c_min in (0.0, 1.0, 3.0, 8.0, 1e300):
        r = O.run(sc.replace(c_min=c_min), flags=O.NO_SOLVE)
        nz = r["slot_val"] != 0
        key = set(zip(r["slot_row"][nz].tolist(), r["slot_col"][nz].tolist(), r["slot_dir"][nz].tolist(),
                      r["slot_k"][nz].tolist()))
        if prev is not None:
            assert key < prev
        prev = key
    # only chains without a receiver are left: they deposit on their source
    assert all(row == col for row, col, _, _ in prev)


def test_p11_ground_sources_share_one_quadrature_for_sun_and_diffuse_light():
    """A Lambertian source re-emits without memory of the incoming direction,
    so its sun-lit and diffusely lit deposits are equal, with and without
    coupling selection."""
    sc = scenes.make_random(9, 8, 5, seed=23, S=2, R=2, M=1024, albedo=0.4)
    for c_min in (0.0, 3.0, 8.0):
        r = O.run(sc.replace(c_min=c_min), flags=O.NO_SOLVE)
        g = r["slot_col"] >= r["n_atm"]
        assert np.array_equal(r["slot_depsun"][g], r["slot_dep"][g])
        assert np.array_equal(r["esc_sun"][r["n_atm"]:], r["esc_iso"][r["n_atm"]:])


@pytest.mark.parametrize("R,sza,saa", [(1, 35.0, 10.0), (2, 62.0, 130.0)])
def test_p11_energy_conservation_with_selection(R, sza, saa):
    """P5 with c_min > 0: with omega = 1 and a black surface every photon
    leaves through the TOA or reaches the ground, as long as each source keeps
    a direction (here: every axis neighbour stays coupled)."""
    nx, ny, nz = 6, 5, 7
    h = (0.1, 0.08, 0.12)
    me = np.random.default_rng(5).uniform(0.5, 2.0, nz)
    c_min = 0.99 * me.min() / max(h)
    sc = scenes.make_layered(nx, ny, nz, me, [1.0], g=(0.6,), albedo=0.0, R=R, sza=sza, saa=saa,
                             vza=10, h=h, M=2048).replace(c_min=c_min)
    r = O.run(sc, gmres_tol=1e-15)
    full = O.run(sc.replace(c_min=0.0), flags=O.NO_SOLVE)
    assert (r["slot_val"] != 0).sum() < (full["slot_val"] != 0).sum()
    na = r["n_atm"]
    mu0 = math.cos(math.radians(sza))
    incident = nx * ny * mu0 * sc.hx * sc.hy
    escape = float(r["e1"] @ r["esc_sun"] + r["x"] @ r["esc_iso"])
    direct_ground = float(mu0 * sc.hx * sc.hy * r["tsun"][na:].sum())
    row, col = r["slot_row"], r["slot_col"]
    gnd = row >= na
    deposited_ground = float((r["slot_depsun"][gnd] * r["e1"][col[gnd]]).sum()
                             + (r["slot_dep"][gnd] * r["x"][col[gnd]]).sum())
    total = escape + direct_ground + deposited_ground
    assert abs(total - incident) <= 1e-12 * incident


# P11 (top-K): the preselected maximum number of couplings of Sec. 3

def _all_couplings(sc, r):
    """Every chain's coupling C = sqrt(mu_s(source) mu_s(first receiver)) / d
    (Eq. scatt_coup), computed here from the grid and the fields: atmospheric
    sources along each direction u (first receiver j + u, or the ground when
    the chain crosses z = 0 first, none when it leaves through the TOA),
    ground sources along each ground chain (first member voxel)."""
    nx, ny, nz = sc.nx, sc.ny, sc.nz
    mus = np.zeros((nz, ny, nx))
    for sp in range(sc.n_species):
        mus = mus + np.asarray(sc.mu_s[sp], dtype=np.float64)
    mus_lamb = sc.albedo * float(mus.max())
    h = (sc.hx, sc.hy, sc.hz)
    out = []
    for (ux, uy, uz) in r["dirs"]:
        p0, p1, p2 = ux * h[0], uy * h[1], uz * h[2]
        L = math.sqrt(p0 * p0 + p1 * p1 + p2 * p2)
        for z in range(nz):
            rz = z + uz
            if rz >= nz:
                continue
            for y in range(ny):
                for x in range(nx):
                    if rz >= 0:
                        mn, d = float(mus[rz, (y + uy) % ny, (x + ux) % nx]), L
                    else:
                        mn, d = mus_lamb, (z + 0.5) / -uz * L
                    out.append(math.sqrt(float(mus[z, y, x]) * mn) / d)
    for mem in r["gdir_mem"][: r["n_gdirs"]]:
        m0, m1, m2 = (int(v) for v in mem[0])
        p0, p1, p2 = m0 * h[0], m1 * h[1], (m2 - 0.5) * h[2]
        L = math.sqrt(p0 * p0 + p1 * p1 + p2 * p2)
        for y in range(ny):
            for x in range(nx):
                out.append(math.sqrt(mus_lamb * float(mus[m2 - 1, (y + m1) % ny, (x + m0) % nx])) / L)
    return np.array(out)


@pytest.mark.parametrize("R", [1, 2])
def test_p11_topk_threshold_is_the_k_plus_first_largest_coupling(R):
    """Keeping the K largest couplings is the threshold rule C > c_min with
    c_min the (K + 1)-th largest coupling (brute force over every chain);
    couplings tie in pairs (a chain and its reverse), so a boundary inside a
    tied group keeps fewer than K."""
    sc = scenes.make_random(7, 6, 4, seed=31, S=2, R=R, M=512, zero_frac=0.0, albedo=0.3)
    r0 = O.run(sc, flags=O.NO_SOLVE)
    C = np.sort(_all_couplings(sc, r0))[::-1]
    assert r0["n_couplings"] == C.size and r0["n_kept"] == C.size and r0["c_min_used"] == 0.0
    for K in (1, 2, 3, C.size // 3, C.size // 3 + 1, C.size // 2, C.size - 1):
        r = O.run(sc.replace(max_couplings=int(K)), flags=O.NO_SOLVE)
        assert r["c_min_used"] == C[K], K
        assert r["n_kept"] == int((C > C[K]).sum()) <= K, K
    assert r["n_kept"] == C.size - 1 or C[-1] == C[-2]


def test_p11_topk_at_or_above_the_count_is_the_full_stencil():
    sc = scenes.make_random(9, 8, 5, seed=21, S=2, R=2, M=1024, zero_frac=0.0)
    r0 = O.run(sc)
    for K in (r0["n_couplings"], 10 ** 9):
        r1 = O.run(sc.replace(max_couplings=K))
        assert r1["c_min_used"] == 0.0 and r1["n_kept"] == r0["n_couplings"]
        for k in ("slot_val", "slot_valsun", "x", "rad"):
            assert np.array_equal(r0[k], r1[k]), k


def test_p11_topk_equals_the_threshold_rule_and_nests():
    """Top-K reproduces the c_min selection at its threshold bit for bit, and
    the kept edges shrink as K does; zero couplings (non-scattering voxels)
    go first."""
    sc = scenes.make_random(8, 7, 5, seed=22, S=2, R=2, M=1024, zero_frac=0.1)
    full = O.run(sc, flags=O.NO_SOLVE)
    prev = None
    for frac in (0.9, 0.6, 0.3, 0.1):
        K = int(frac * full["n_couplings"])
        rk = O.run(sc.replace(max_couplings=K))
        rc = O.run(sc.replace(c_min=rk["c_min_used"]))
        for k in ("slot_val", "slot_valsun", "x", "rad"):
            assert np.array_equal(rk[k], rc[k]), (frac, k)
        nz_now = set(zip(rk["slot_row"][rk["slot_val"] != 0], rk["slot_col"][rk["slot_val"] != 0],
                         rk["slot_dir"][rk["slot_val"] != 0]))
        if prev is not None:
            assert nz_now < prev
        prev = nz_now
    zero = _all_couplings(sc, full) == 0.0
    assert zero.any()
    K = int((~zero).sum())  # exactly the positive couplings survive
    rz = O.run(sc.replace(max_couplings=K), flags=O.NO_SOLVE)
    assert rz["c_min_used"] > 0.0 and rz["c_min_used"] < 1e-300 and rz["n_kept"] == K


@pytest.mark.parametrize("R,A", [(1, 0.0), (2, 0.4)])
def test_p11_energy_conservation_with_topk(R, A):
    """Energy balance with a quarter of the couplings kept.  Sources that keep
    no direction scatter their power out of the graph ("lost"), and with
    omega = 1 a set of sources that keep only directions among themselves
    (horizontal chains deposit everything) would trap power (rho(K) = 1), so
    the layers absorb a little (omega = 0.97): incident = TOA escape + ground
    absorption + voxel absorption (of the direct beam and of what arrives) +
    lost."""
    nx, ny, nz = 6, 5, 6
    om = 0.97
    rng = np.random.default_rng(9)
    sc = scenes.make_layered(nx, ny, nz, rng.uniform(0.1, 2.0, nz), [om], g=(0.6,), albedo=A, R=R, sza=40.0,
                             saa=70.0, vza=10, h=(0.1, 0.08, 0.12), M=1024)
    n = O.run(sc, flags=O.NO_SOLVE)["n_couplings"]
    r = O.run(sc.replace(max_couplings=n // 4), gmres_tol=1e-15)
    assert 0 < r["n_kept"] <= n // 4 and r["rel_resid"] < 1e-14
    na, nn = r["n_atm"], r["n_nodes"]
    mu0 = math.cos(math.radians(40.0))
    incident = nx * ny * mu0 * sc.hx * sc.hy
    e1, x = r["e1"], r["x"]
    escape = float(e1 @ r["esc_sun"] + x @ r["esc_iso"])
    direct = float(mu0 * sc.hx * sc.hy * r["tsun"][na:].sum())
    row, col = r["slot_row"], r["slot_col"]
    gnd = row >= na
    diffuse = float((r["slot_depsun"][gnd] * e1[col[gnd]]).sum() + (r["slot_dep"][gnd] * x[col[gnd]]).sum())
    dep_iso = np.zeros(nn)
    np.add.at(dep_iso, col, r["slot_dep"])
    dep_sun = np.zeros(nn)
    np.add.at(dep_sun, col, r["slot_depsun"])
    lost = float(e1 @ (1.0 - dep_sun - r["esc_sun"]) + x @ (1.0 - dep_iso - r["esc_iso"]))
    assert lost > 0.0
    # voxels: e1 = omega x (beam extinction), x = omega x (power arriving)
    absorbed = (1.0 - om) / om * float(e1[:na].sum() + x[:na].sum())
    total = escape + (1.0 - A) * (direct + diffuse) + absorbed + lost
    assert abs(total - incident) <= 1e-12 * incident


# --------------------------------------------------------------------------
# P12: anisotropic multiple scattering, the edge unknowns of Eq. flux_system
# (the arrival direction kept into every scattering)

@pytest.mark.parametrize("R,S", [(1, 1), (2, 2), (2, 3)])
def test_p12_isotropic_phase_reduces_to_the_node_form(R, S):
    """With g = 0 the re-emission does not depend on the arrival direction,
    so the edge form gives the node-collapsed solution."""
    sc = scenes.make_random(8, 7, 4, seed=30 + R + S, S=S, R=R, M=1024)
    sc = sc.replace(g=np.zeros(S))
    a, i = O.run(sc, flags=O.ANISO), O.run(sc)
    assert np.abs(a["x"] - i["x"]).max() <= 1e-12 * np.abs(i["x"]).max()
    assert np.abs(a["X"].sum(axis=1) - i["x"]).max() <= 1e-12 * np.abs(i["x"]).max()
    assert (np.abs(a["rad"] - i["rad"]) / i["rad"]).max() < 1e-12


def test_p12_phase_quadrature_rows_peak_forward_and_reduce_to_cells():
    sc = scenes.make_random(5, 5, 3, seed=1, S=3, R=2, M=4096).replace(g=np.array([0.0, 0.5, 0.85]))
    Q = O.phase_quadrature(sc)
    r = O.run(sc, flags=O.NO_SOLVE)
    nd, ngd = r["n_dirs"], r["n_gdirs"]
    assert Q.shape == (3, nd + ngd, nd)
    np.testing.assert_allclose(Q.sum(axis=2), 1.0, atol=1e-13)
    # g = 0: the cells' shares of the lattice for every arrival direction
    np.testing.assert_allclose(Q[0], np.broadcast_to(r["q_iso"], (nd + ngd, nd)), rtol=1e-12)
    # forward scattering: the mean of HG over a cell (Q / the cell's share)
    # peaks at the cell of the arrival direction itself; a ground chain's
    # direction peaks at the cell that holds it
    u = r["dirs"] * np.array([sc.hx, sc.hy, sc.hz])
    u = u / np.linalg.norm(u, axis=1, keepdims=True)
    gm = r["gdir_mem"][:, 0, :].astype(float) - np.array([0.0, 0.0, 0.5])
    gu = gm * np.array([sc.hx, sc.hy, sc.hz])
    gu = gu / np.linalg.norm(gu, axis=1, keepdims=True)
    for sp in (1, 2):
        dens = Q[sp] / r["q_iso"]
        assert np.array_equal(dens[:nd].argmax(axis=1), np.arange(nd))
        assert np.array_equal(dens[nd:].argmax(axis=1), (gu @ u.T).argmax(axis=1))


@pytest.mark.parametrize("R,sza,saa,g", [(1, 35.0, 10.0, 0.6), (2, 62.0, 130.0, 0.85)])
def test_p12_energy_conservation(R, sza, saa, g):
    """P5 for the edge form: with omega = 1 and a black surface all incident
    power leaves through the TOA or reaches the ground."""
    nx, ny, nz = 6, 5, 7
    me = np.random.default_rng(5).uniform(0.1, 2.0, nz)
    sc = scenes.make_layered(nx, ny, nz, me, [1.0], g=(g,), albedo=0.0, R=R, sza=sza, saa=saa,
                             vza=10, h=(0.1, 0.08, 0.12), M=2048)
    r = O.run(sc, flags=O.ANISO)
    na = r["n_atm"]
    mu0 = math.cos(math.radians(sza))
    incident = nx * ny * mu0 * sc.hx * sc.hy
    direct_ground = mu0 * sc.hx * sc.hy * r["tsun"][na:].sum()
    total = r["esc_out"].sum() + direct_ground + r["arrive"][na:].sum()
    assert abs(total - incident) <= 1e-12 * incident


def test_p12_forward_peaked_light_penetrates_deeper():
    """Strong forward scattering keeps multiply scattered light moving away
    from the sun: against the node form (isotropic re-emission after the
    first scattering), the edge form sends more light to a black ground under
    a thick scattering layer and less back to space."""
    nx, ny, nz = 6, 6, 8
    sc = scenes.make_layered(nx, ny, nz, [1.5] * nz, [1.0], g=(0.85,), albedo=0.0, R=2, sza=30, vza=0,
                             h=(0.1, 0.1, 0.1), M=2048)
    a, i = O.run(sc, flags=O.ANISO), O.run(sc)
    na = a["n_atm"]
    gnd_a = a["arrive"][na:].sum()
    gnd_i = float((i["slot_depsun"][i["slot_row"] >= na] * i["e1"][i["slot_col"][i["slot_row"] >= na]]).sum()
                  + (i["slot_dep"][i["slot_row"] >= na] * i["x"][i["slot_col"][i["slot_row"] >= na]]).sum())
    assert gnd_a > gnd_i
    assert a["rad"].mean() < i["rad"].mean()


def test_p12_a_species_that_never_scatters_has_no_effect():
    """The per-node phase quadrature mixes the species by their share of
    mu_s: a second species with mu_s = 0 everywhere (whatever its g) leaves
    the edge form's solution unchanged."""
    one = scenes.make_random(7, 6, 4, seed=41, S=1, R=2, M=1024).replace(g=np.array([0.7]))
    two = one.replace(mu_s=np.concatenate([one.mu_s, np.zeros_like(one.mu_s)]), g=np.array([0.7, -0.5]))
    a1, a2 = O.run(one, flags=O.ANISO), O.run(two, flags=O.ANISO)
    assert (np.abs(a2["rad"] - a1["rad"]) / a1["rad"]).max() < 1e-13


def test_p12_rejects_coupling_selection():
    sc = scenes.make_random(5, 5, 3, seed=1, S=1, R=1, M=512).replace(c_min=1.0)
    with pytest.raises(ValueError):
        O.run(sc, flags=O.ANISO)


def read_flux_matrix_example():
    """The worked example of Sec. 2 (four nodes, six edges, the printed
    pattern of F), from tests/golden/flux_matrix_example.txt."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "flux_matrix_example.txt")
    edges, pattern, in_pattern = {}, [], False
    for line in open(path):
        line = line.split("#", 1)[0].split()
        if not line:
            continue
        if line[0] == "edge":
            edges[int(line[1])] = (int(line[2]), int(line[3]))
        elif line[0] == "pattern":
            in_pattern = True
        elif in_pattern:
            pattern.append([int(v) for v in line])
    return [edges[k] for k in sorted(edges)], np.array(pattern, dtype=np.int64)


def test_p12_worked_example_pattern_is_head_to_tail():
    """F_ab is nonzero exactly where edge a ends at the node where edge b
    starts (light that arrives along a scatters there into b): that rule,
    applied to the example's six edges, gives the pattern the paper prints,
    and its transpose does not."""
    edges, printed = read_flux_matrix_example()
    assert printed.shape == (6, 6)
    rule = np.array([[int(a[1] == b[0]) for b in edges] for a in edges])
    assert (rule == printed).all()
    assert (rule.T != printed).any()


@pytest.mark.parametrize("make", [
    lambda: scenes.make_random(5, 4, 3, seed=71, S=2, R=1, M=512, zero_frac=0.0),
    lambda: scenes.make_random(6, 5, 3, seed=72, S=1, R=2, M=512, sza=35.0, albedo=0.4, zero_frac=0.0),
])
def test_p12_edge_form_couples_head_to_tail(make):
    """The oracle's edge-form operator has the worked example's structure
    (Sec. 2, the flux matrix example, with the edges arriving at a node along
    one direction merged into one unknown): X(i, w) depends on X(j, w')
    exactly when an edge from j reaches i along w, for every arrival
    direction w' of j.  A seeded sample of the operator's columns is probed
    with a single large entry at X = 0 (the map is affine, and a term with no
    dependence adds exact zeros); a term that ran over the receiver's edges
    instead of the source's, or kept the wrong arrival direction, moves the
    pattern.  Every voxel of these scenes scatters (an element carries the
    receiver's mu_s, so a voxel without scattering would zero the elements
    of its edges)."""
    sc = make()
    r = O.run(sc, flags=O.ANISO)
    nn, nin = r["n_nodes"], r["n_dirs"] + r["n_gdirs"]
    rows = np.arange(nn, dtype=np.int32)
    srow, scol, sdir = r["slot_row"], r["slot_col"], r["slot_dir"]
    # the unknowns that are edges' heads: some edge arrives at i along w
    arrives = np.zeros((nn, nin), dtype=bool)
    arrives[srow, sdir] = True
    feeds = {}  # source j -> the unknowns (i, w) of the edges that leave j
    for i, j, w in zip(srow.tolist(), scol.tolist(), sdir.tolist()):
        feeds.setdefault(j, set()).add((i, w))
    X0 = np.zeros((nn, nin))
    F0 = O.aniso_rows(sc, X0, rows)
    cols = np.argwhere(arrives)
    assert len(cols) > 0
    if len(cols) > 500:  # a seeded sample of the columns keeps the R = 2 case to a few seconds
        cols = cols[np.random.default_rng(9).choice(len(cols), 500, replace=False)]
    for j, wp in cols.tolist():
        X = X0.copy()
        X[j, wp] = 1e10
        d = O.aniso_rows(sc, X, rows) - F0
        assert set(map(tuple, np.argwhere(d != 0).tolist())) == feeds.get(j, set()), (j, wp)


# --------------------------------------------------------------------------
# Emission toward the instrument (final radiance sum of Sec. 2)

def test_isotropic_emission_identity():
    """With isotropic phase functions every in-edge is weighted by 1/(4 pi):
    E_i = (e1_i + x_i) / (4 pi), because the in-edge deposits of a receiver
    sum to x_i = s_i + (K x)_i."""
    sc = scenes.make_random(5, 6, 4, seed=11, S=2, R=2, M=1024)
    sc.g = np.zeros(2)
    r = O.run(sc)
    na = r["n_atm"]
    np.testing.assert_allclose(r["emis"], (r["e1"][:na] + r["x"][:na]) / (4 * math.pi), rtol=1e-12,
                               atol=1e-15 * r["emis"].max())


def _pos(sc, n):
    na = sc.n_atm
    if n >= na:
        c = n - na
        return np.array([(c % sc.nx + 0.5) * sc.hx, (c // sc.nx + 0.5) * sc.hy, 0.0])
    iz, rem = divmod(n, sc.nx * sc.ny)
    iy, ix = divmod(rem, sc.nx)
    return np.array([(ix + 0.5) * sc.hx, (iy + 0.5) * sc.hy, (iz + 0.5) * sc.hz])


def test_emission_directions_from_node_geometry():
    """E_i recomputed from the slot list with each in-edge's travel direction
    taken from the node positions (source -> receiver, nearest periodic image)
    rather than from the direction tables."""
    sc = scenes.make_random(6, 6, 4, seed=12, S=2, R=2, M=1024, vza=40.0, vaa=70.0)
    r = O.run(sc)
    v = view_vec(sc.vza, sc.vaa)
    s0 = sun_vec(sc.sza, sc.saa)
    Lx, Ly = sc.nx * sc.hx, sc.ny * sc.hy
    mus = sc.mu_s.reshape(sc.n_species, -1)
    tot = mus.sum(0)
    dirs = r["dirs"]
    rows = np.random.default_rng(0).choice(r["n_atm"], 25, replace=False)
    for i in rows:
        w = mus[:, i] / tot[i] if tot[i] > 0 else np.full(sc.n_species, 1 / sc.n_species)
        theta = lambda mu: sum(w[s] * hg(sc.g[s], mu) for s in range(sc.n_species))
        E = r["e1"][i] * theta(float(s0 @ v))
        m = np.nonzero(r["slot_row"] == i)[0]
        for e in m:
            j, k = r["slot_col"][e], r["slot_k"][e]
            if k == O.K_SELF:
                u = dirs[r["slot_dir"][e]] * np.array([sc.hx, sc.hy, sc.hz])
            else:
                u = _pos(sc, i) - _pos(sc, j)
                u[0] -= Lx * round(u[0] / Lx)
                u[1] -= Ly * round(u[1] / Ly)
            u = u / np.linalg.norm(u)
            E += theta(float(u @ v)) * (r["slot_valsun"][e] * r["e1"][j] + r["slot_val"][e] * r["x"][j])
        assert abs(E - r["emis"][i]) <= 1e-12 * abs(E)


def test_ground_hit_columns_brute_force():
    """Every chain that reaches the ground deposits on the column(s) that a
    dense exact walk of its ray meets at z = 0, split equally on ties."""
    sc = scenes.make_random(7, 6, 3, seed=13, S=1, R=2, M=512)
    r = O.run(sc, flags=O.NO_SOLVE)
    na = r["n_atm"]
    dirs = r["dirs"]
    m = r["slot_k"] == O.K_GROUND
    groups = {}
    for row, col, d, val in zip(r["slot_row"][m], r["slot_col"][m], r["slot_dir"][m], r["slot_dep"][m]):
        groups.setdefault((int(col), int(d)), []).append((int(row) - na, float(val)))
    assert groups
    for (j, d), hits in groups.items():
        u = [Fraction(int(c)) for c in dirs[d]]
        iz, rem = divmod(j, sc.nx * sc.ny)
        iy, ix = divmod(rem, sc.nx)
        P = [Fraction(ix) + Fraction(1, 2), Fraction(iy) + Fraction(1, 2), Fraction(iz) + Fraction(1, 2)]
        t = P[2] / -u[2]
        hx, hy = P[0] + t * u[0], P[1] + t * u[1]
        xs = [hx - 1, hx] if hx.denominator == 1 else [math.floor(hx)]
        ys = [hy - 1, hy] if hy.denominator == 1 else [math.floor(hy)]
        expect = sorted((int(y) % sc.ny) * sc.nx + int(x) % sc.nx for x in xs for y in ys)
        got = sorted(c for c, _ in hits)
        assert got == expect
        vals = [v for _, v in hits]
        assert max(vals) - min(vals) <= 1e-15 * max(vals)


@pytest.mark.parametrize("make", [
    lambda: scenes.make_random(7, 6, 5, seed=61, S=2, R=2, M=512),
    lambda: scenes.make_random(8, 7, 4, seed=62, S=3, R=1, M=512, sza=20.0, vza=55.0),
])
def test_p12_rowwise_edge_map_fixes_the_oracle_edge_solution(make):
    """The row-wise edge-form map (orc_aniso_rows, which builds each needed
    source's leaving power on the fly) reproduces the converged series of
    orc_aniso at every row: F(X) = X, and a change of X at one source moves
    F at its receivers only through that source's chains."""
    sc = make()
    r = O.run(sc, flags=O.ANISO)
    X = r["X"]
    rng = np.random.default_rng(5)
    rows = rng.choice(r["n_nodes"], 48, replace=False).astype(np.int32)
    F = O.aniso_rows(sc, X, rows)
    assert np.abs(F - X[rows]).max() <= 1e-12 * np.abs(X).max()
    # doubling X at one source changes F exactly at the rows its slots reach
    j = int(rows[0])
    X2 = X.copy()
    X2[j] *= 2.0
    reach = set(r["slot_row"][r["slot_col"] == j].tolist())
    F2 = O.aniso_rows(sc, X2, rows)
    moved = {int(i) for i, a, b in zip(rows, F, F2) if np.abs(a - b).max() > 1e-14 * np.abs(X).max()}
    assert moved and moved <= reach
