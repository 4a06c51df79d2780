"""GPU parity of the Cholesky flavour (reduction to standard form, Sec. 2.4) through the C ABI.

The library factors S = L L^T, minimises over H_r = L^-1 H L^-T with S = I and no
preconditioner, and returns C = L^-T C_r. Checked against the oracle's Cholesky flavour and
its plain definition of the minimum (the n lowest generalised eigenpairs), at sizes that span
several 64-wide tiles and a ragged tail (m = 207, 256, 416).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def S():
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300 import solver
    return solver


PROBLEMS = {
    "si64_sz": lambda c: c.si64_sz(),                                        # m = 256, n = 128
    "water9": lambda c: c.water(nmol=9, seed=1),                             # m = 207
    "si16_dzp": lambda c: c.silicon(k=(1, 2, 2), basis="DZP", seed=4),       # m = 416
}


@pytest.fixture(scope="module", params=sorted(PROBLEMS))
def case(request):
    from synth import configs
    from oracle import exact, omm
    p = PROBLEMS[request.param](configs)
    ref = omm.solve_cholesky(p.H, p.S, p.eta, p.C0, tol_grad=1e-9)
    ex = exact.exact_minimum(p.H, p.S, p.n)
    return p, ref, ex


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cholesky_solve_matches_oracle(S, case, precision):
    p, ref, ex = case
    with S.OMMSolver(dev(p.H), dev(p.S), None, p.n, p.eta, p.tau, precision=precision,
                     cholesky=True) as s:
        C, E, D, info = s.solve(dev(p.C0), want_D=True)
        dH, dS = s.backward()
    C, D, dH, dS = (t.cpu().numpy() for t in (C, D, dH, dS))
    assert info["status"] == 0 and info["gmax"] < 1e-9
    tol = 1e-10 if precision == "fp64" else 1e-9
    assert abs(E - ex["E"]) / abs(ex["E"]) <= tol
    assert abs(E - ref["E"]) / abs(ref["E"]) <= tol
    assert np.abs(D - ex["D"]).max() <= 1e-7
    assert np.abs(dH - D).max() == 0.0
    assert np.abs(dS + ex["EDM"]).max() <= 1e-7
    Cm = C.T                                   # back in the original basis: C^T S C = I
    assert np.abs(Cm.T @ p.S @ Cm - np.eye(p.n)).max() < 1e-8
    assert info["ms_transform"] > 0.0
    if precision == "fp64":
        # the oracle's reduced trajectory, up to rounding near the end
        assert abs(info["iterations"] - ref["iters"]) <= max(3, ref["iters"] // 10)


def test_cholesky_follows_s_inverse_preconditioning(S, case):
    """Sec. 2.4: the reduced minimisation takes the steps of the S^-1-preconditioned one."""
    p, ref, ex = case
    with S.OMMSolver(dev(p.H), dev(p.S), None, p.n, p.eta, p.tau, cholesky=True) as s:
        _, E1, _, i1 = s.solve(dev(p.C0))
    with S.OMMSolver(dev(p.H), dev(p.S), None, p.n, p.eta, math.inf) as s:   # P = S^-1
        _, E2, _, i2 = s.solve(dev(p.C0))
    assert i1["status"] == 0 and i2["status"] == 0
    assert abs(E1 - E2) / abs(E2) <= 1e-10
    assert abs(i1["iterations"] - i2["iterations"]) <= max(3, i2["iterations"] // 10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cholesky_warm_start_update_H(S, case, precision):
    """omm_update_H reduces the new H with the kept factor (SCF step, Sec. 2.5.2)."""
    p, ref, ex = case
    from oracle import exact
    rng = np.random.default_rng(3)
    H2 = p.H + np.diag(rng.normal(0.0, 0.01, size=p.m))
    with S.OMMSolver(dev(p.H), dev(p.S), None, p.n, p.eta, p.tau, precision=precision,
                     cholesky=True) as s:
        C, E, _, info0 = s.solve(dev(p.C0))
        s.update_H(dev(H2))
        C2, E2, D2, info1 = s.solve(C, want_D=True)
    ex2 = exact.exact_minimum(H2, p.S, p.n)
    assert info1["status"] == 0
    assert abs(E2 - ex2["E"]) / abs(ex2["E"]) <= (1e-10 if precision == "fp64" else 1e-9)
    assert np.abs(D2.cpu().numpy() - ex2["D"]).max() <= 1e-7
    assert info1["iterations"] < info0["iterations"]


def test_cholesky_rejects_indefinite_overlap(S):
    from synth import configs
    from paper_1312_1549_gb300 import _native as N
    p = configs.si64_sz()
    Sbad = p.S.copy()
    Sbad[100, 100] = -1.0
    for precision in ("fp64", "mixed"):
        with pytest.raises(N.OMMError) as e:
            S.OMMSolver(dev(p.H), dev(Sbad), None, p.n, p.eta, p.tau, precision=precision, cholesky=True)
        assert e.value.status == 2


def test_cholesky_batched_matches_exact(S):
    """A mixed batch in the Cholesky flavour: every instance reaches its own minimum."""
    from synth import configs
    from oracle import exact
    probs = [configs.silicon(k=(2, 2, 2), basis="SZ", seed=0),     # m = 256
             configs.water(nmol=9, seed=1),                       # m = 207
             configs.silicon(k=(1, 2, 2), basis="DZP", seed=4)]   # m = 416
    batch = S.OMMBatch([(dev(p.H), dev(p.S), None, p.n, p.eta, p.tau) for p in probs],
                       precision="mixed", cholesky=True)
    try:
        Cs, Es, infos = batch.solve([dev(p.C0) for p in probs])
    finally:
        batch.close()
    for p, C, E, info in zip(probs, Cs, Es, infos):
        ex = exact.exact_minimum(p.H, p.S, p.n)
        assert info["status"] == 0
        assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-9
        Cm = C.cpu().numpy().T
        assert np.abs(Cm.T @ p.S @ Cm - np.eye(p.n)).max() < 1e-8
