"""Autograd through the OMM solve: dE/dH and dE/dS against central differences and the oracle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300.autograd import omm_energy
    from synth import si64_sz
    from oracle import exact
    p = si64_sz()
    return omm_energy, p, exact.exact_minimum(p.H, p.S, p.n)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autograd_matches_exact_gradients(setup, precision):
    omm_energy, p, ex = setup
    H = dev(p.H).requires_grad_(True)
    S = dev(p.S).requires_grad_(True)
    E, C = omm_energy(H, S, dev(p.T), dev(p.C0), p.n, p.eta, p.tau, precision=precision)
    E.backward()
    assert abs(E.item() - ex["E"]) / abs(ex["E"]) <= (1e-10 if precision == "fp64" else 1e-9)
    assert np.abs(H.grad.cpu().numpy() - ex["D"]).max() <= 1e-7
    assert np.abs(S.grad.cpu().numpy() + ex["EDM"]).max() <= 1e-7


def test_autograd_central_differences(setup):
    """<dE/dH, dH> and <dE/dS, dS> against [E(+h) - E(-h)] / 2h (h = 1e-5, warm-started solves).

    The random symmetric directions have unit Frobenius norm, so the h^2 truncation term of the
    central difference (about h^2 |dH|^3 / gap^2) stays far below the tolerance.
    """
    omm_energy, p, ex = setup
    H = dev(p.H).requires_grad_(True)
    S = dev(p.S).requires_grad_(True)
    T = dev(p.T)
    E, C = omm_energy(H, S, T, dev(p.C0), p.n, p.eta, p.tau, tol_grad=1e-11)
    E.backward()
    gH, gS = H.grad.detach(), S.grad.detach()
    rng = np.random.default_rng(11)
    h = 1e-5
    for k in range(4):
        dH = rng.normal(size=(p.m, p.m)); dH = 0.5 * (dH + dH.T); dH = dev(dH / np.linalg.norm(dH))
        dS = rng.normal(size=(p.m, p.m)); dS = (dS + dS.T) * (np.abs(p.S) > 0)
        dS = dev(dS / np.linalg.norm(dS))
        with torch.no_grad():
            Ep, _ = omm_energy(H + h * dH, S, T, C, p.n, p.eta, p.tau, tol_grad=1e-11)
            Em, _ = omm_energy(H - h * dH, S, T, C, p.n, p.eta, p.tau, tol_grad=1e-11)
            fd = (Ep.item() - Em.item()) / (2 * h)
            assert fd == pytest.approx(float((gH * dH).sum()), rel=1e-6, abs=5e-7)
            Ep, _ = omm_energy(H, S + h * dS, T, C, p.n, p.eta, p.tau, tol_grad=1e-11)
            Em, _ = omm_energy(H, S - h * dS, T, C, p.n, p.eta, p.tau, tol_grad=1e-11)
            fd = (Ep.item() - Em.item()) / (2 * h)
            assert fd == pytest.approx(float((gS * dS).sum()), rel=1e-6, abs=5e-7)
