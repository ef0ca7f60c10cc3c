"""The bounded device wait of the pipelined passes gives up with
TURSCA_E_TIMEOUT instead of hanging, and the context stays usable.

The self-test entry point waits, with the passes' own wait helper, on an
mbarrier that gets its one expected arrival (control) or none (the wait runs
out after its bounded number of polls).  No fault is provoked: the kernel
returns normally either way.
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


def test_wait_that_completes_returns_ok():
    rc, sec = T.tursca_selftest_wait(True, torch.cuda.current_stream().cuda_stream)
    assert rc == T.OK
    print("completed wait: %.3f s" % sec)


def test_wait_that_runs_out_returns_timeout_and_context_stays_usable():
    rc, sec = T.tursca_selftest_wait(False, torch.cuda.current_stream().cuda_stream)
    print("unsatisfied wait gave up after %.3f s" % sec)
    assert rc == T.E_TIMEOUT
    # the device still runs the full path correctly afterwards
    sc = scenes.make_plume(nx=16, ny=16, nz=8)
    rn = T.Runner(sc, T.FP32_REFINE)
    mu_a, mu_s = rn.fields("cuda")
    rn.run(mu_a, mu_s, rtol=1e-10)
    torch.cuda.synchronize()
    rad = rn.rad.cpu().numpy().astype(np.float64)
    ref = O.run(sc)["rad"]
    assert (np.abs(rad - ref) / np.abs(ref)).max() < 1e-4
    rc2, _ = T.tursca_selftest_wait(True, torch.cuda.current_stream().cuda_stream)
    assert rc2 == T.OK
