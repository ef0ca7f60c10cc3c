"""CPU tests of the C-ABI library's host logic (no GPU needed).

The library loads on a machine without a GPU; these tests call only its
host-only entry points: graph counts, the CSR structure of K and the
Fibonacci-partition quadrature, compared with the FP64 oracle (integer and
index work bit-exact).
"""
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_16037_gb300 import scenes
from paper_2503_16037_gb300 import tursca as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_16037_gb300 import build
    build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tursca.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tursca_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = T.lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_binding_constants_match_header_enums():
    """Every TURSCA_* enumerator of the header that the binding names (without
    the prefix) has the same value there."""
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "tursca.h")).read(), flags=re.S)
    pairs = re.findall(r"\bTURSCA_([A-Z0-9_]+)\s*=\s*(\d+)", src)
    assert len(pairs) >= 20
    seen = 0
    for name, value in pairs:
        if hasattr(T, name):
            assert getattr(T, name) == int(value), name
            seen += 1
    assert seen >= 10 and T.OPT_SINGLE_SCATTER == 6


def test_status_strings():
    for s in range(8):
        assert T.tursca_status_string(s)


def _structure(sc):
    row_ptr, col, dr, k = T.tursca_graph_structure(T.grid_desc(sc))
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    return row_ptr, rows, col, dr, k


SCENES = [
    lambda: scenes.make_plain(),
    lambda: scenes.make_random(5, 6, 4, seed=1, R=2, M=512),
    lambda: scenes.make_random(7, 5, 2, seed=2, R=2, M=512),    # nz = R
    lambda: scenes.make_random(5, 5, 1, seed=3, R=1, M=256),    # a single layer
    lambda: scenes.make_random(9, 8, 6, seed=4, R=1, M=512, h=(0.1, 0.07, 0.05)),
]


@pytest.mark.parametrize("maker", SCENES)
def test_csr_structure_matches_oracle(maker):
    sc = maker()
    r = O.run(sc, flags=O.NO_SOLVE)
    row_ptr, rows, col, dr, k = _structure(sc)
    assert np.all(dr >= 0) and np.all(k >= 0)
    lib_keys = np.stack([rows, col, dr.astype(np.int64), k.astype(np.int64)], 1)
    orc_keys = np.stack([r["slot_row"], r["slot_col"], r["slot_dir"], r["slot_k"]], 1)
    assert len(lib_keys) == len(orc_keys)
    a = lib_keys[np.lexsort(lib_keys.T[::-1])]
    b = orc_keys[np.lexsort(orc_keys.T[::-1])]
    assert np.array_equal(a, b)
    st = T.tursca_graph_info(T.grid_desc(sc))
    assert st.nnz_edges == r["n_slots"] and st.nnz == len(col)
    assert st.n_dirs == r["n_dirs"] and st.n_gdirs == r["n_gdirs"]


@pytest.mark.parametrize("maker", SCENES[:3])
def test_direction_order_and_quadrature_match_oracle(maker):
    sc = maker()
    r = O.run(sc, flags=O.NO_SOLVE)
    qi, ql = T.tursca_quadrature(T.grid_desc(sc))
    # the partition is an argmax taken in FP64 on both sides: counts are exact
    assert np.array_equal(qi, r["q_iso"])
    np.testing.assert_allclose(ql, r["q_lamb"], rtol=1e-15, atol=1e-17)


def test_plume_graph_counts():
    sc = scenes.make_plume()
    st = T.tursca_graph_info(T.grid_desc(sc))
    assert st.n_atm == 64 * 64 * 32 and st.n_nodes == 64 * 64 * 33
    assert st.n_dirs == 98 and st.n_up_dirs == 41 and st.n_gdirs == 49 and st.n_gmembers == 50
    # 124 in-stencil neighbours per voxel minus the vertical truncation:
    # per column 32 * 124 - (25 * 1 + 25 * 2) * 2 atmosphere-to-atmosphere edges
    row_ptr, rows, col, dr, k = _structure(sc)
    na = st.n_atm
    atm = (rows < na) & (col < na) & (k >= 1) & (k <= 2)
    assert atm.sum() == 4096 * (32 * 124 - 150) == 15638528
    assert ((col >= na) & (k >= 1)).sum() == 4096 * 50  # ground sources: 50 members per column
    # an interior voxel receives exactly its 124 stencil neighbours
    lens = np.diff(row_ptr)
    assert lens[16 * 4096] == 124 and st.max_row == lens.max()


@pytest.mark.parametrize("field,value", [("nx", 4), ("stencil_radius", 3), ("nz", 1), ("n_species", 5),
                                         ("precision", 7), ("fib_points", 10), ("hx", -1.0)])
def test_invalid_descriptor_rejected(field, value):
    sc = scenes.make_plume(nx=16, ny=16, nz=8)
    d = T.grid_desc(sc)
    setattr(d, field, value)
    with pytest.raises(T.TurscaError) as ei:
        T.tursca_graph_info(d)
    assert ei.value.status == T.E_INVALID


def test_null_handles():
    L = T.lib()
    assert L.tursca_build_graph(None) == T.E_INVALID
    assert L.tursca_scene_destroy(None) == T.OK
    assert L.tursca_solve(None, 1e-10, 10, None) == T.E_INVALID
