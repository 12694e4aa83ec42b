"""Failure detection on the GPU without a fault: the library's grid-wide barrier waits a
bounded number of polls, then sets HW_ETIMEOUT and lets every CTA leave.  The test runs the
barrier self-test with one CTA that never arrives and a tiny wait bound (the wait must run
out), checks the status word, and then checks that the context still works (an H X product
against the oracle).  Nothing here traps, faults or hangs the GPU: every wait is bounded."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import basis as B
from oracle import hamiltonian as Hm
from oracle import potential as P
from paper_2210_12252_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hwmod():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2210_12252_gb300 import build
    build.build()
    from paper_2210_12252_gb300 import helicwave
    return helicwave


def test_barrier_completes_when_every_block_arrives(hwmod):
    ctx = hwmod.Context(0)
    assert hwmod.hw_selftest_barrier(ctx.h, 8, 1 << 20, -1) == hwmod.HW_OK
    ctx.close()


def test_barrier_wait_runs_out_and_context_stays_usable(hwmod):
    w = inputs.tiny()
    ctx = hwmod.Context(0)
    L = int(ctx.setup_basis(w.geom, w.etas)[0])
    ctx.build_potential(w.atoms)
    t0 = time.perf_counter()
    st = hwmod.hw_selftest_barrier(ctx.h, 4, 2000, 2)    # CTA 2 never arrives; ~0.2 ms bound
    assert st == hwmod.HW_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    # the same context keeps working after the timed-out kernel
    g = w.geom
    b = B.Basis(g.R, g.tau, g.alpha, g.Nr, g.Nth1, g.Nth2, g.ncyc, g.oversample)
    kp = B.KPoint(b, 0.0, 0.0, g.ecut)
    X = inputs.random_block(L, 3, 17)
    Y = ctx.apply_H(0, torch.from_numpy(np.ascontiguousarray(X.T)).cuda()).cpu().numpy().T
    Yref = Hm.apply_H(kp, P.gaussian_wells(b, w.atoms), X)
    assert np.abs(Y - Yref).max() < 1e-10 * np.abs(Yref).max()
    # and a barrier with every block present completes again
    assert hwmod.hw_selftest_barrier(ctx.h, 4, 1 << 20, -1) == hwmod.HW_OK
    ctx.close()


def test_barrier_selftest_rejects_bad_arguments(hwmod):
    ctx = hwmod.Context(0)
    for args in ((1, 100, -1), (4, 0, -1), (4, 100, 4), (4, 1 << 25, -1), (100000, 100, -1)):
        with pytest.raises(hwmod.HwError) as e:
            hwmod.hw_selftest_barrier(ctx.h, *args)
        assert e.value.status == hwmod.HW_EINVAL
    ctx.close()
