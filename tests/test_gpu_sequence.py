"""SCF-like warm-start sequence: H_k = H_0 + k delta, each solve from the previous C (Sec. 2.5.2)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("native_certificate", [False, True])
def test_warm_started_sequence_matches_exact(native_certificate):
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300.solver import OMMSolver
    from synth import configs
    from oracle import exact
    p = configs.silicon(k=(4, 4, 4), basis="SZ", seed=0)   # m = 2048, n = 1024
    delta = configs.warm_start_delta(p, 1)
    iters = []
    with OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, precision="mixed",
                   native_certificate=native_certificate) as s:
        C = dev(p.C0)
        for k in range(4):
            Hk = p.H + np.diag(k * delta)
            if k > 0:
                s.update_H(dev(Hk))
            C, E, D, info = s.solve(C, want_D=True)
            dH, _ = s.backward(want_S=False)
            ex = exact.exact_minimum(Hk, p.S, p.n)
            assert info["status"] == 0 and info["gmax"] < 1e-9
            assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-9, (k, E, ex["E"])
            assert np.abs(D.cpu().numpy() - ex["D"]).max() <= 1e-7
            assert torch.equal(dH, D)
            iters.append(info["iterations"])
    assert max(iters[1:]) < iters[0], iters   # warm starts need fewer line searches
