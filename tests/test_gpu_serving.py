"""Serving: requests of uneven grid sizes run concurrently on resident slots
(the tursca_server_* calls).  Every request's radiance must equal, bit for
bit, the radiance of the same request run alone through a Runner, whatever
else runs with it and however the memory budget makes the server evict and
rebuild slots."""
import numpy as np
import pytest

from paper_2503_16037_gb300 import scenes
from paper_2503_16037_gb300 import tursca as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(16, 16, 16), (24, 24, 16), (32, 32, 24)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2503_16037_gb300 import build
    build.build()
    torch.cuda.init()


def requests(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx, ny, nz = SHAPES[rng.integers(len(SHAPES))]
        out.append(scenes.make_plume(nx=nx, ny=ny, nz=nz, sza=float(rng.uniform(20.0, 75.0))))
    return out


def alone(sc, rtol=1e-10):
    rn = T.Runner(sc, T.FP32_REFINE)
    mu_a, mu_s = rn.fields("cuda")
    rad, _ = rn.run(mu_a, mu_s, rtol=rtol)
    torch.cuda.synchronize()
    r = rad.cpu().numpy().copy()
    rn.close()
    return r


def served(reqs, budget, workers):
    srv = T.Server(budget, workers)
    tickets = [srv.submit(sc, T.FP32_REFINE, 1e-10) for sc in reqs]
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    return outs, st


def test_mixed_requests_equal_alone():
    reqs = requests(24)
    ref = [alone(sc) for sc in reqs]
    outs, st = served(reqs, 8 << 30, 4)
    for (rad, info), r in zip(outs, ref):
        assert info["status"] == T.OK
        assert info["rel_resid64"] <= 1e-10
        assert np.array_equal(rad.numpy(), r)
    assert st["slots_built"] <= 4 * len(SHAPES)          # slots are reused, not rebuilt per request
    assert sum(info["slot_reused"] for _, info in outs) >= len(reqs) - st["slots_built"]
    assert st["peak_bytes"] <= st["budget_bytes"]


def test_tight_budget_evicts_and_stays_exact():
    reqs = requests(12, seed=1)
    ref = [alone(sc) for sc in reqs]
    # room for about one slot of the largest shape: requests wait, slots are evicted
    rn = T.Runner(reqs[0].replace(), T.FP32_REFINE)
    big = scenes.make_plume(nx=32, ny=32, nz=24)
    rb = T.Runner(big, T.FP32_REFINE)
    mu_a, mu_s = rb.fields("cuda")
    rb.run(mu_a, mu_s)
    one = T.lib().tursca_scene_device_bytes(rb.handle)
    rb.close()
    rn.close()
    outs, st = served(reqs, int(one * 1.6), 3)
    for (rad, info), r in zip(outs, ref):
        assert info["status"] == T.OK
        assert np.array_equal(rad.numpy(), r)
    assert st["evictions"] > 0
    assert st["peak_bytes"] <= st["budget_bytes"]


def test_request_that_cannot_fit_fails():
    srv = T.Server(1 << 20, 2)  # 1 MiB: no slot fits
    t = srv.submit(scenes.make_plume(nx=16, ny=16, nz=16), T.FP32_REFINE)
    with pytest.raises(T.TurscaError) as e:
        srv.wait(t)
    assert e.value.status == T.E_NOMEM
    srv.close()
