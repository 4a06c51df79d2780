"""Pins for the oracle: brute force, closed forms, finite differences and invariants.

Each test checks the oracle against something other than itself, chosen so
that a dropped term, a wrong sign, a wrong index or a transposed operand in
the oracle fails at least one of them. CPU only.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import exact, jacobi, omm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_problem(m, n, seed, gap=0.3):
    """Random symmetric H, SPD S and SPD T with a generalised gap at n."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, m))
    S = np.eye(m) + 0.08 * (A + A.T) / math.sqrt(m)
    S = S @ S.T / np.max(np.abs(np.linalg.eigvalsh(S @ S.T)))  # SPD, eigenvalues in (0, 1]
    S = 0.5 * (S + S.T) + 0.2 * np.eye(m)
    B = rng.normal(size=(m, m))
    T = B @ B.T / m + 0.1 * np.eye(m)
    # H with eigenvalues chosen in the S-metric: H = S X diag(w) X^T S, X S-orthonormal
    L = np.linalg.cholesky(S)
    Q, _ = np.linalg.qr(rng.normal(size=(m, m)))
    X = np.linalg.solve(L.T, Q)                    # X^T S X = I
    w = np.sort(rng.uniform(-1.0, 1.0, size=m))
    w[n:] += gap
    H = S @ X @ np.diag(w) @ X.T @ S
    H = 0.5 * (H + H.T)
    eta = 0.5 * (w[n - 1] + w[n])
    C0 = rng.normal(0.0, 0.1, size=(n, m)) / math.sqrt(m)
    return H, S, T, eta, C0, w


# ---------------------------------------------------------------- brute force
def test_jacobi_closed_form_2x2():
    a, b, c = 0.7, -0.3, -1.1
    w, V = jacobi.jacobi_eigh(np.array([[a, b], [b, c]]))
    mean, rad = 0.5 * (a + c), math.sqrt(0.25 * (a - c) ** 2 + b * b)
    assert np.allclose(w, [mean - rad, mean + rad], atol=1e-15)
    assert np.allclose(V.T @ V, np.eye(2), atol=1e-14)


def test_jacobi_known_spectrum():
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.normal(size=(9, 9)))
    lam = np.array([-3.0, -1.0, -1.0, 0.0, 0.5, 2.0, 2.5, 4.0, 7.0])
    A = Q @ np.diag(lam) @ Q.T
    w, V = jacobi.jacobi_eigh(0.5 * (A + A.T))
    assert np.allclose(w, lam, atol=1e-12)
    assert np.allclose(A @ V, V * w[None, :], atol=1e-11)


def test_generalized_jacobi_matches_lapack():
    H, S, T, eta, C0, w = tiny_problem(14, 5, 1)
    wj, Xj = jacobi.generalized_eigh(H, S)
    assert np.allclose(wj, w, atol=1e-11)          # the spectrum H was built with
    import scipy.linalg
    assert np.allclose(wj, scipy.linalg.eigh(H, S, eigvals_only=True), atol=1e-11)
    assert np.allclose(Xj.T @ S @ Xj, np.eye(14), atol=1e-11)
    assert np.allclose(H @ Xj, S @ Xj * wj[None, :], atol=1e-10)


def test_exact_minimum_invariants():
    H, S, T, eta, C0, w = tiny_problem(16, 6, 2)
    ex = exact.exact_minimum(H, S, 6, method="jacobi")
    D = ex["D"]
    assert ex["E"] == pytest.approx(2.0 * w[:6].sum(), abs=1e-11)
    assert np.trace(D @ S) == pytest.approx(12.0, abs=1e-11)          # Tr(DS) = 2n
    assert np.allclose(0.5 * D @ S @ (0.5 * D), 0.5 * D, atol=1e-11)   # idempotent in the S metric
    # EDM = H-weighted density matrix: EDM = D S^-1 H-ish check through H X = S X eps
    assert np.allclose(ex["EDM"], 0.5 * (D @ H @ D), atol=1e-10)


# ---------------------------------------------------------------- the OMM reaches the exact minimum
@pytest.mark.parametrize("m,n,seed,precondition", [(12, 3, 10, True), (20, 7, 11, True),
                                                   (20, 7, 11, False), (24, 10, 12, True)])
def test_omm_reaches_brute_force(m, n, seed, precondition):
    H, S, T, eta, C0, w = tiny_problem(m, n, seed)
    r = omm.solve(H, S, T, eta, 1.3, C0, tol_grad=1e-11, max_iter=5000, precondition=precondition)
    assert r["status"] == omm.STATUS_OK
    ex = exact.exact_minimum(H, S, n, method="jacobi")
    assert r["E"] == pytest.approx(ex["E"], rel=1e-12, abs=1e-12)
    assert np.allclose(r["SW"], np.eye(n), atol=1e-9)
    assert np.allclose(r["D"], ex["D"], atol=1e-9)
    assert np.allclose(r["EDM"], ex["EDM"], atol=1e-9)
    assert np.trace(r["D"] @ S) == pytest.approx(2 * n, abs=1e-9)


def test_shift_correction_two_n_eta():
    """E does not depend on eta (above the HOMO) and E - E~ = 2 n eta (Eq. 10 read with spin 2)."""
    H, S, T, eta, C0, w = tiny_problem(18, 6, 21)
    n = 6
    r1 = omm.solve(H, S, T, eta, 2.0, C0, tol_grad=1e-11)
    r2 = omm.solve(H, S, T, eta + 0.07, 2.0, C0, tol_grad=1e-11)
    assert r1["E"] == pytest.approx(r2["E"], abs=1e-10)
    assert r1["E"] - r1["Etilde"] == pytest.approx(2 * n * eta, abs=1e-12)
    assert r1["E"] == pytest.approx(2.0 * w[:n].sum(), abs=1e-10)


def test_golden_diagonal_case():
    g = json.load(open(os.path.join(GOLDEN, "diagonal_case.json")))
    m, n = g["m"], g["n"]
    H = np.diag(g["H_diag"])
    S = np.eye(m)
    rng = np.random.default_rng(0)
    C0 = rng.normal(0.0, 0.3, size=(n, m))
    r = omm.solve(H, S, np.eye(m), g["eta"], g["tau"], C0, tol_grad=1e-12)
    assert r["E"] == pytest.approx(g["E"], abs=1e-12)
    assert np.allclose(r["D"], np.diag(g["D_diag"]), atol=1e-11)
    assert np.allclose(r["EDM"], np.diag(g["EDM_diag"]), atol=1e-11)


# ---------------------------------------------------------------- functional, gradient, quartic
def _random_state(m, n, seed):
    H, S, T, eta, C0, w = tiny_problem(m, n, seed)
    rng = np.random.default_rng(seed + 100)
    C = rng.normal(size=(m, n)) * 0.4
    Dl = rng.normal(size=(m, n)) * 0.3
    return omm.shift(H, S, eta), S, C, Dl


def test_functional_two_forms():
    Ht, S, C, _ = _random_state(11, 4, 5)
    HW, SW = C.T @ Ht @ C, C.T @ S @ C
    first = 2.0 * np.trace((np.eye(4) + (np.eye(4) - SW)) @ HW)   # Eq. 8, left form
    assert omm.functional(C, Ht, S) == pytest.approx(first, rel=1e-13)


def test_quartic_coefficients_match_direct_evaluation():
    Ht, S, C, Dl = _random_state(13, 5, 6)
    HC, SC, HW, SW = omm.subspace_operators(C, Ht, S)
    E = omm.functional_from_subspace(HW, SW)
    a = omm.quartic_coefficients(E, HW, SW, Dl.T @ HC, Dl.T @ SC, Dl.T @ Ht @ Dl, Dl.T @ S @ Dl)
    xs = np.array([-2.0, -1.0, -0.4, 0.3, 1.0, 1.7, 2.5])
    direct = np.array([omm.functional(C + x * Dl, Ht, S) for x in xs])
    poly = np.array([omm.quartic_value(a, x) for x in xs])
    assert np.allclose(poly, direct, rtol=1e-11, atol=1e-11)
    # and the coefficients are what five exact samples determine
    V = np.vander(xs[:5], 5, increasing=True)
    assert np.allclose(np.linalg.solve(V, direct[:5]), a, rtol=1e-8, atol=1e-9)


def test_alpha1_is_directional_derivative():
    Ht, S, C, Dl = _random_state(10, 3, 7)
    HC, SC, HW, SW = omm.subspace_operators(C, Ht, S)
    G = omm.gradient(HC, SC, HW, SW)
    a = omm.quartic_coefficients(0.0, HW, SW, Dl.T @ HC, Dl.T @ SC, Dl.T @ Ht @ Dl, Dl.T @ S @ Dl)
    assert a[1] == pytest.approx(float(np.vdot(G, Dl)), rel=1e-12)


def test_gradient_central_differences():
    Ht, S, C, _ = _random_state(9, 4, 8)
    HC, SC, HW, SW = omm.subspace_operators(C, Ht, S)
    G = omm.gradient(HC, SC, HW, SW)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 1), (8, 3), (5, 2)]:
        Cp = C.copy(); Cp[i, j] += h
        Cm = C.copy(); Cm[i, j] -= h
        fd = (omm.functional(Cp, Ht, S) - omm.functional(Cm, Ht, S)) / (2 * h)
        assert fd == pytest.approx(G[i, j], rel=1e-7, abs=1e-8)


# ---------------------------------------------------------------- line minimum
def _first_min_by_scan(a, xmax=50.0, npts=2_000_001):
    xs = np.linspace(0.0, xmax, npts)
    p = a[0] + xs * (a[1] + xs * (a[2] + xs * (a[3] + xs * a[4])))
    d = np.diff(p)
    k = np.nonzero(d >= 0)[0]
    return None if k.size == 0 else xs[k[0]]


@pytest.mark.parametrize("a", [
    [0.0, -1.0, 0.5, 0.0, 0.0],            # quadratic: x = 1
    [0.0, -2.0, 1.0, -0.3, 0.05],          # alpha4 > 0
    [1.0, -0.5, 3.0, -4.0, 1.2],           # two minima, the first one is taken
    [0.0, -1.0, 2.0, 0.5, -0.1],           # alpha4 < 0, local minimum exists
    [0.0, -1e-3, 1.0, 0.0, 1.0],
])
def test_line_minimum_matches_scan(a):
    a = np.array(a, float)
    x, st = omm.line_minimum(a)
    assert st == omm.STATUS_OK
    xs = _first_min_by_scan(a)
    assert x == pytest.approx(xs, abs=5e-5)
    d1 = a[1] + x * (2 * a[2] + x * (3 * a[3] + 4 * a[4] * x))
    assert abs(d1) < 1e-12 * (1 + abs(a).max())


def test_line_minimum_unbounded():
    x, st = omm.line_minimum(np.array([0.0, -1.0, -0.5, 0.1, -0.2]))
    assert st == omm.STATUS_UNBOUNDED and x == 0.0


# ---------------------------------------------------------------- preconditioner
def test_preconditioner_is_inverse():
    H, S, T, eta, C0, w = tiny_problem(15, 4, 30)
    for tau in (0.5, 5.0):
        P = omm.preconditioner(S, T, tau)
        assert np.allclose(P @ (S + T / tau), np.eye(15), atol=1e-12)
    assert np.allclose(omm.preconditioner(S, T, np.inf) @ S, np.eye(15), atol=1e-12)


# ---------------------------------------------------------------- backward (dE/dH, dE/dS)
def test_backward_central_differences():
    """<dE/dH, dH> and <dE/dS, dS> by central differences of warm-started re-solves."""
    H, S, T, eta, C0, w = tiny_problem(14, 4, 40)
    r = omm.solve(H, S, T, eta, 2.0, C0, tol_grad=1e-12)
    Cstar = r["C"].T.copy()
    rng = np.random.default_rng(41)
    h = 1e-5
    for _ in range(3):
        dH = rng.normal(size=H.shape); dH = 0.5 * (dH + dH.T)
        dS = rng.normal(size=S.shape); dS = 0.05 * (dS + dS.T)
        Ep = omm.solve(H + h * dH, S, T, eta, 2.0, Cstar, tol_grad=1e-12)["E"]
        Em = omm.solve(H - h * dH, S, T, eta, 2.0, Cstar, tol_grad=1e-12)["E"]
        assert (Ep - Em) / (2 * h) == pytest.approx(float(np.vdot(r["D"], dH)), rel=1e-7, abs=1e-8)
        Ep = omm.solve(H, S + h * dS, T, eta, 2.0, Cstar, tol_grad=1e-12)["E"]
        Em = omm.solve(H, S - h * dS, T, eta, 2.0, Cstar, tol_grad=1e-12)["E"]
        assert (Ep - Em) / (2 * h) == pytest.approx(-float(np.vdot(r["EDM"], dS)), rel=1e-7, abs=1e-8)


# ---------------------------------------------------------------- the Si64 workload
def test_si64_workload_reaches_lapack_minimum():
    from synth import si64_sz
    p = si64_sz()
    r = omm.solve(p.H, p.S, p.T, p.eta, p.tau, p.C0, tol_grad=1e-9)
    assert r["status"] == omm.STATUS_OK and r["gmax"] < 1e-9
    ex = exact.exact_minimum(p.H, p.S, p.n)
    assert abs(r["E"] - ex["E"]) / abs(ex["E"]) < 1e-12
    assert np.abs(r["D"] - ex["D"]).max() < 1e-7
    assert np.abs(r["SW"] - np.eye(p.n)).max() < 1e-8


# ---------------------------------------------------------------- the Cholesky flavour (Sec. 2.4)
@pytest.mark.parametrize("m,n,seed", [(12, 3, 10), (20, 7, 11), (24, 10, 12)])
def test_cholesky_flavour_reaches_brute_force(m, n, seed):
    """Reduced to standard form, the OMM still reaches 2 sum eps_i, D and EDM of H x = eps S x."""
    H, S, T, eta, C0, w = tiny_problem(m, n, seed)
    r = omm.solve_cholesky(H, S, eta, C0, tol_grad=1e-11, max_iter=5000)
    assert r["status"] == omm.STATUS_OK
    ex = exact.exact_minimum(H, S, n, method="jacobi")
    assert r["E"] == pytest.approx(ex["E"], rel=1e-12, abs=1e-12)
    C = r["C"]                                     # back in the original basis
    assert np.allclose(C.T @ S @ C, np.eye(n), atol=1e-9)
    assert np.allclose(r["D"], ex["D"], atol=1e-9)
    assert np.allclose(r["EDM"], ex["EDM"], atol=1e-9)
    assert np.allclose(C.T @ (H - eta * S) @ C, r["HW"], atol=1e-9)   # H_W is basis-invariant


@pytest.mark.parametrize("m,n,seed", [(20, 7, 11), (30, 9, 13)])
def test_cholesky_flavour_follows_s_inverse_preconditioning(m, n, seed):
    """Sec. 2.4: minimising the reduced problem follows the original one preconditioned by S^-1.

    Same start (C_r = L^T C0), so the line-search steps x, the PR coefficients and the energies
    agree iteration by iteration (up to rounding), and both stop after the same number of steps.
    """
    H, S, T, eta, C0, w = tiny_problem(m, n, seed)
    red, orig = [], []
    omm.solve_cholesky(H, S, eta, C0, tol_grad=1e-30, max_iter=12,
                       callback=lambda it, E, x, b: red.append((E, x, b)), want_matrices=False)
    omm.solve(H, S, None, eta, math.inf, C0, tol_grad=1e-30, max_iter=12, precondition=True,
              callback=lambda it, E, x, b: orig.append((E, x, b)), want_matrices=False)
    assert len(red) == len(orig) == 12
    for (Er, xr, br), (Eo, xo, bo) in zip(red, orig):
        assert Er == pytest.approx(Eo, rel=1e-10, abs=1e-12)
        assert xr == pytest.approx(xo, rel=1e-7)
        assert br == pytest.approx(bo, rel=1e-6, abs=1e-12)
    # and not the unpreconditioned trajectory
    plain = []
    omm.solve(H, S, None, eta, math.inf, C0, tol_grad=1e-30, max_iter=12, precondition=False,
              callback=lambda it, E, x, b: plain.append((E, x, b)), want_matrices=False)
    assert any(abs(a[1] - b[1]) > 1e-3 * abs(b[1]) for a, b in zip(plain, orig))


def test_cholesky_flavour_si64_workload():
    from synth import si64_sz
    p = si64_sz()
    r = omm.solve_cholesky(p.H, p.S, p.eta, p.C0, tol_grad=1e-9)
    assert r["status"] == omm.STATUS_OK and r["gmax"] < 1e-9
    ex = exact.exact_minimum(p.H, p.S, p.n)
    assert abs(r["E"] - ex["E"]) / abs(ex["E"]) < 1e-12
    assert np.abs(r["D"] - ex["D"]).max() < 1e-7


# ---------------------------------------------------------------- degenerate and extreme cases
def test_single_orbital_and_n_equals_m_minus_one():
    """n = 1 (E = 2 eps_1) and n = m - 1 (all but the highest state occupied) reach the brute force."""
    for (m, n, seed) in [(9, 1, 31), (9, 8, 32), (2, 1, 33)]:
        H, S, T, eta, C0, w = tiny_problem(m, n, seed)
        r = omm.solve(H, S, T, eta, 1.3, C0, tol_grad=1e-11, max_iter=5000)
        assert r["status"] == omm.STATUS_OK, (m, n)
        we, X = jacobi.generalized_eigh(H, S)
        assert r["E"] == pytest.approx(2.0 * float(np.sum(we[:n])), rel=1e-12, abs=1e-12)
        occ = X[:, :n]
        assert np.abs(r["D"] - 2.0 * occ @ occ.T).max() < 1e-9


def test_degenerate_occupied_levels():
    """Equal eigenvalues inside the occupied set: the orbitals are not unique, D and E are."""
    m, n = 14, 5
    rng = np.random.default_rng(40)
    S = np.eye(m) + 0.05 * np.diag(rng.uniform(size=m))
    L = np.linalg.cholesky(S)
    Q, _ = np.linalg.qr(rng.normal(size=(m, m)))
    X = np.linalg.solve(L.T, Q)
    w = np.sort(rng.uniform(0.0, 1.0, size=m)) + 0.5
    w[:3] = -0.7                                  # a threefold degenerate level in the occupied set
    w[3:5] = -0.2                                 # and a twofold one
    H = S @ X @ np.diag(w) @ X.T @ S
    H = 0.5 * (H + H.T)
    C0 = rng.normal(0.0, 0.1, size=(n, m))
    r = omm.solve(H, S, None, 0.1, 1.0, C0, tol_grad=1e-11, max_iter=5000, precondition=False)
    assert r["status"] == omm.STATUS_OK
    assert r["E"] == pytest.approx(2.0 * (3 * -0.7 + 2 * -0.2), rel=1e-12)
    occ = X[:, :n]
    assert np.abs(r["D"] - 2.0 * occ @ occ.T).max() < 1e-9


def test_start_at_the_minimum_takes_no_line_search():
    """From the converged C the gradient is already below the tolerance: zero line searches."""
    H, S, T, eta, C0, w = tiny_problem(16, 5, 41)
    r = omm.solve(H, S, T, eta, 1.3, C0, tol_grad=1e-11, max_iter=5000)
    r2 = omm.solve(H, S, T, eta, 1.3, r["C"], tol_grad=1e-10, C_is_mn=True)
    assert r2["iters"] == 0 and r2["status"] == omm.STATUS_OK
    assert r2["E"] == pytest.approx(r["E"], rel=1e-14)


def test_cholesky_flavour_trajectory_at_si64_dzp():
    """Sec. 2.4 at a workload's size (m = 832): 30 line searches of the reduced problem and of the
    S^-1-preconditioned original one give the same energies to rounding."""
    from synth import configs
    p = configs.silicon(k=(2, 2, 2), basis="DZP", seed=0)
    a = omm.solve_cholesky(p.H, p.S, p.eta, p.C0, tol_grad=1e-30, max_iter=30, want_matrices=False)
    b = omm.solve(p.H, p.S, None, p.eta, math.inf, p.C0, tol_grad=1e-30, max_iter=30, want_matrices=False)
    ea = np.array([h[0] for h in a["history"]])
    eb = np.array([h[0] for h in b["history"]])
    assert len(ea) == len(eb) == 31
    assert np.abs((ea - eb) / eb).max() < 1e-12
