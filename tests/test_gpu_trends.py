"""Convergence trends the paper reports (Sec. 2.5.1), checked qualitatively on the GPU path.

Line-search counts are not pinned by the paper (only its figures show them), so these tests check
the direction of the effects on the synthetic workloads, not numbers:
  * kinetic preconditioning cuts the line searches for a DZP-like basis;
  * raising eta well above the lowest unoccupied level costs line searches;
  * every variant still reaches the same minimum (2 sum eps_i).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def si64_dzp():
    from paper_1312_1549_gb300 import build
    build.build()
    from synth import configs
    from oracle import exact
    p = configs.silicon(k=(2, 2, 2), basis="DZP", seed=0)   # m = 832, n = 128
    return p, exact.exact_minimum(p.H, p.S, p.n, want_matrices=False)


def _iters(p, eta=None, tau=None, precondition=True):
    from paper_1312_1549_gb300.solver import OMMSolver
    eta = p.eta if eta is None else eta
    tau = p.tau if tau is None else tau
    with OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, eta, tau, precondition=precondition,
                   max_iter=20000) as s:
        _, E, _, info = s.solve(dev(p.C0))
    return info["iterations"], E


def test_kinetic_preconditioner_cuts_line_searches(si64_dzp):
    p, ex = si64_dzp
    it_p, E_p = _iters(p)                          # tau = 10 Ry
    it_s, E_s = _iters(p, tau=float("inf"))        # pure tensorial correction S^-1
    it_n, E_n = _iters(p, precondition=False)      # plain gradient
    for E in (E_p, E_s, E_n):
        assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-10
    assert it_p < it_n, (it_p, it_s, it_n)
    assert it_s < it_n, (it_p, it_s, it_n)


def test_eta_far_above_lumo_costs_line_searches(si64_dzp):
    p, ex = si64_dzp
    lumo = ex["lumo"]
    it_lo, E_lo = _iters(p, eta=lumo + 0.01)
    it_hi, E_hi = _iters(p, eta=lumo + 1.5)
    assert abs(E_lo - ex["E"]) / abs(ex["E"]) <= 1e-10
    assert abs(E_hi - ex["E"]) / abs(ex["E"]) <= 1e-10
    assert it_hi > it_lo, (it_lo, it_hi)
