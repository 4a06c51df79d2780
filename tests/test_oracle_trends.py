"""The convergence trends of Sec. 2.5.1 on the oracle (CPU): the tau and eta sweeps.

The paper reports line-search counts only in figures, so the checks are qualitative, on the Si
64-atom DZP-like cell (m = 832, n = 128) from its seeded start:
  * the kinetic preconditioner P = (S + T/tau)^-1 needs fewest line searches at an intermediate
    tau, fewer than the pure tensorial correction S^-1 (tau -> infinity), which needs fewer than
    no preconditioning;
  * raising eta above the lowest unoccupied level costs line searches, more the higher it goes;
  * every variant reaches the same minimum 2 sum eps_i.
The float64 GPU path takes the same steps (its iteration counts are compared with the oracle's
in the GPU tests), so these trends hold for it too.
"""
import math

import numpy as np
import pytest

from oracle import exact, omm


@pytest.fixture(scope="module")
def si64_dzp():
    from synth import configs
    p = configs.silicon(k=(2, 2, 2), basis="DZP", seed=0)
    return p, exact.exact_minimum(p.H, p.S, p.n, want_matrices=False)


def _run(p, eta, tau, precondition=True):
    r = omm.solve(p.H, p.S, p.T, eta, tau, p.C0, tol_grad=1e-9, max_iter=20000, precondition=precondition,
                  want_matrices=False)
    assert r["status"] == omm.STATUS_OK
    return r


def test_tau_sweep_has_an_interior_optimum(si64_dzp):
    p, ex = si64_dzp
    taus = [0.25, 1.0, 2.0, 5.0, 20.0, math.inf]
    runs = {tau: _run(p, p.eta, tau) for tau in taus}
    none = _run(p, p.eta, 1.0, precondition=False)
    for r in list(runs.values()) + [none]:
        assert abs(r["E"] - ex["E"]) / abs(ex["E"]) < 1e-12
    its = {tau: r["iters"] for tau, r in runs.items()}
    best = min(its, key=its.get)
    assert 0.25 < best < math.inf, its
    assert its[best] < its[math.inf] < none["iters"], (its, none["iters"])


def test_eta_above_the_gap_costs_line_searches(si64_dzp):
    p, ex = si64_dzp
    its = []
    for d in (0.05, 0.2, 0.5, 1.0, 1.5):
        r = _run(p, ex["lumo"] + d, p.tau)
        assert abs(r["E"] - ex["E"]) / abs(ex["E"]) < 1e-12
        its.append(r["iters"])
    assert all(b >= a for a, b in zip(its, its[1:])), its
    assert its[-1] > 1.5 * its[0], its
