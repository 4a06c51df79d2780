"""The search direction's precision (a reading of Sec. 2.4), checked on the oracle (CPU).

The mixed path forms the preconditioned gradient of the search direction as one bf16 product,
bf16(P) bf16(G), while the line search (Eqs. 13-16) and the gradient that decides convergence
(Eq. 12) keep full accuracy. The reading: P only steers the search, so a direction built from
the rounded operands reaches the same minimum in about as many line searches. Checked here on the
float64 oracle with its P G replaced by the rounded product (everything else unchanged), on the
Si 64-atom DZP-like cell (m = 832, n = 128) with the kinetic preconditioner and with S^-1; and
bf16(P) stays positive definite there.
"""
import numpy as np
import pytest

from oracle import exact, omm


def bf16(x):
    """float64 -> nearest bf16 (8 significant bits, ties to even), as float64."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


class RoundedP:
    """Stands in for P in the oracle's direction step: P @ G -> bf16(P) @ bf16(G)."""

    def __init__(self, P):
        self.P = bf16(P)

    def __matmul__(self, G):
        return self.P @ bf16(G)


@pytest.fixture(scope="module")
def si64_dzp():
    from synth import configs
    p = configs.silicon(k=(2, 2, 2), basis="DZP", seed=0)
    return p, exact.exact_minimum(p.H, p.S, p.n, want_matrices=False)


@pytest.mark.parametrize("tau", [5.0, float("inf")])
def test_rounded_direction_reaches_the_same_minimum(si64_dzp, tau, monkeypatch):
    p, ex = si64_dzp
    ref = omm.solve(p.H, p.S, p.T, p.eta, tau, p.C0, tol_grad=1e-9, want_matrices=False)
    exact_P = omm.preconditioner
    monkeypatch.setattr(omm, "preconditioner", lambda S, T, t: RoundedP(exact_P(S, T, t)))
    got = omm.solve(p.H, p.S, p.T, p.eta, tau, p.C0, tol_grad=1e-9, want_matrices=False)
    assert ref["status"] == got["status"] == omm.STATUS_OK
    assert abs(got["E"] - ex["E"]) <= 1e-10 * abs(ex["E"])
    assert abs(got["iters"] - ref["iters"]) <= max(2, ref["iters"] // 20), (got["iters"], ref["iters"])


@pytest.mark.parametrize("tau", [5.0, float("inf")])
def test_rounded_preconditioner_stays_positive_definite(si64_dzp, tau):
    p, _ = si64_dzp
    P = omm.preconditioner(p.S, p.T, tau)
    w = np.linalg.eigvalsh(P)
    wr = np.linalg.eigvalsh(bf16(P))
    assert wr[0] > 0.9 * w[0] > 0.0
