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


def served(reqs, budget, workers, batch_solves=False):
    srv = T.Server(budget, workers, batch_solves=batch_solves)
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


# Batched refinements (tursca_server_configure(TURSCA_SERVER_BATCH_SOLVES)):
# the Chebyshev refinements of concurrent requests run in one persistent
# kernel; each request keeps its own schedule and every group is computed by
# the code of the request's own pass, so results are bit for bit those of the
# request alone.

def test_batched_refinements_run_together_and_change_no_bit():
    reqs = requests(32, seed=3)
    ref = [alone(sc) for sc in reqs]
    outs_on, st_on = served(reqs, 8 << 30, 8, batch_solves=True)
    assert st_on["batches"] > 0 and st_on["max_batch"] >= 2
    assert st_on["batched_refinements"] > st_on["batches"]
    srv = T.Server(8 << 30, 8, batch_solves=False)
    tickets = [srv.submit(sc, T.FP32_REFINE, 1e-10) for sc in reqs]
    outs_off = [srv.wait(t) for t in tickets]
    st_off = srv.stats()
    srv.close()
    assert st_off["batches"] == 0
    for (a, ia), (b, ib), r in zip(outs_on, outs_off, ref):
        assert ia["status"] == T.OK and ib["status"] == T.OK and ia["rel_resid64"] <= 1e-10
        assert np.array_equal(a.numpy(), r) and np.array_equal(b.numpy(), r)
    print("batched: %d launches, %d refinements, at most %d in one"
          % (st_on["batches"], st_on["batched_refinements"], st_on["max_batch"]))


def test_served_mix_matches_the_oracle():
    """A small mixed batch of shapes and species against the FP64 oracle,
    1e-4 relative on every pixel."""
    from oracle import oracle as O
    reqs = [scenes.make_plume(nx=16, ny=16, nz=8, sza=35.0), scenes.make_random(13, 11, 7, seed=8, S=3, R=1, M=1024),
            scenes.make_plume(nx=20, ny=16, nz=10, sza=65.0), scenes.make_random(12, 11, 6, seed=10, S=2, R=2, M=1024)]
    outs, st = served(reqs * 3, 4 << 30, 6, batch_solves=True)
    for (rad, info), sc in zip(outs, reqs * 3):
        assert info["status"] == T.OK
        ref = O.run(sc)["rad"]
        err = (np.abs(rad.numpy().astype(np.float64) - ref) / np.abs(ref)).max()
        assert err < 1e-4, err


def test_barrier_that_completes_and_one_that_runs_out():
    s = torch.cuda.current_stream().cuda_stream
    assert T.tursca_selftest_barrier(8, True, s) == T.OK
    assert T.tursca_selftest_barrier(8, False, s) == T.E_TIMEOUT
    # the device still serves afterwards
    outs, _ = served(requests(4, seed=5), 2 << 30, 2, batch_solves=True)
    assert all(info["status"] == T.OK for _, info in outs)
