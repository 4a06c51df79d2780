"""Batched OMM (independent instances of uneven size in lockstep, one launch per phase)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def batch_problems():
    from paper_1312_1549_gb300 import build
    build.build()
    from synth import configs
    from oracle import exact
    probs = [configs.silicon(k=(2, 2, 2), basis="SZ", seed=0),     # m = 256
             configs.water(nmol=9, seed=1),                       # m = 207
             configs.silicon(k=(1, 1, 2), basis="DZP", seed=2),   # m = 208
             configs.water(nmol=14, seed=3),                      # m = 322
             configs.silicon(k=(1, 2, 2), basis="DZP", seed=4)]   # m = 416
    ex = [exact.exact_minimum(p.H, p.S, p.n) for p in probs]
    return probs, ex


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batched_solve_matches_exact(batch_problems, precision):
    from paper_1312_1549_gb300.solver import OMMBatch
    probs, ex = batch_problems
    with OMMBatch([(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau) for p in probs],
                  precision=precision) as b:
        Cs, E, infos = b.solve([dev(p.C0) for p in probs])
        for i, p in enumerate(probs):
            assert infos[i]["status"] == 0 and infos[i]["gmax"] < 1e-9, (i, infos[i])
            tol = 1e-10 if precision == "fp64" else 1e-9
            assert abs(E[i] - ex[i]["E"]) / abs(ex[i]["E"]) <= tol, (i, E[i], ex[i]["E"])
            Cm = Cs[i].cpu().numpy().T
            assert np.abs(Cm.T @ p.S @ Cm - np.eye(p.n)).max() < 1e-8
            dH, dS = b.backward(i)
            assert np.abs(dH.cpu().numpy() - ex[i]["D"]).max() <= 1e-7
            assert np.abs(dS.cpu().numpy() + ex[i]["EDM"]).max() <= 1e-7


def test_batched_matches_single_instance_solves(batch_problems):
    """Same instances one by one through omm_solve reach the same energies."""
    from paper_1312_1549_gb300.solver import OMMBatch, OMMSolver
    probs, ex = batch_problems
    with OMMBatch([(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau) for p in probs]) as b:
        _, E, _ = b.solve([dev(p.C0) for p in probs])
    for i, p in enumerate(probs):
        with OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, precision="mixed") as s:
            _, Ei, _, _ = s.solve(dev(p.C0))
        assert abs(E[i] - Ei) / abs(Ei) <= 1e-9
