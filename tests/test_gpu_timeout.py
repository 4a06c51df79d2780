"""The timeout status: a bounded device wait that expires is reported, and the process recovers.

Every wait of the tensor-core kernels on an mbarrier is bounded and reports OMM_ERR_TIMEOUT instead
of trapping. With omm_opts.debug_expire_wait the first tensor-core GEMM of every line search waits
about 1 ms on a barrier that nothing arrives at, before it issues any copy or MMA, so no
asynchronous work is in flight when it gives up. The solve must return OMM_ERR_TIMEOUT promptly,
and a normal solve in the same process must then succeed.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precondition", [True, False])
def test_expired_wait_is_reported_and_the_process_recovers(precondition):
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300 import _native as N
    from paper_1312_1549_gb300.solver import OMMSolver
    from synth import configs
    from oracle import exact
    p = configs.si64_sz()
    t0 = time.perf_counter()
    with OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, precision="mixed",
                   precondition=precondition, debug_expire_wait=True) as s:
        _, _, _, info = s.solve(dev(p.C0), raise_on_error=False)
    assert info["status"] == 6, N.STATUS_NAMES.get(info["status"])  # OMM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    with OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, precision="mixed",
                   precondition=precondition) as s:
        _, E, _, info = s.solve(dev(p.C0))
    ex = exact.exact_minimum(p.H, p.S, p.n, want_matrices=False)
    assert info["status"] == 0 and abs(E - ex["E"]) / abs(ex["E"]) <= 1e-9
