"""Pins of the complex (Hermitian, k-point) oracle and of the k-point input generator.

The complex OMM is checked against things other than itself: the project's own Jacobi brute
force on the real form [[Re A, -Im A], [Im A, Re A]] (whose spectrum is the complex one twice),
the real oracle run on that real form (same steps, twice the energies), central differences of
the functional in Re C and Im C, direct evaluation of E~(C + x Delta) against the quartic, and
the real special case. The generator is pinned by the folding identity: the supercell's
Gamma-point spectrum is the union of the k-point spectra.
"""
import math

import numpy as np
import pytest

from oracle import exact, hermitian, omm


def hermitian_problem(m, n, seed, gap=0.3):
    """Random Hermitian H, Hermitian positive definite S and T, with a generalised gap at n."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    S = np.eye(m) + 0.05 * (A + A.conj().T) / math.sqrt(m)
    S = S @ S.conj().T
    S = 0.5 * (S + S.conj().T) / np.linalg.eigvalsh(S).max() + 0.2 * np.eye(m)
    B = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    T = B @ B.conj().T / m + 0.1 * np.eye(m)
    L = np.linalg.cholesky(S)
    Q, _ = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    X = np.linalg.solve(L.conj().T, Q)                 # X^H S X = I
    w = np.sort(rng.uniform(-1.0, 1.0, size=m))
    w[n:] += gap
    H = S @ X @ np.diag(w) @ X.conj().T @ S
    H = 0.5 * (H + H.conj().T)
    eta = 0.5 * (w[n - 1] + w[n])
    C0 = (rng.normal(0.0, 0.1, size=(n, m)) + 1j * rng.normal(0.0, 0.1, size=(n, m))) / math.sqrt(2 * m)
    return H, S, T, eta, C0, w


def embed_rows(C0):
    """Library-layout rows of the real form of C (m x n): [Re c_j, Im c_j] and [-Im c_j, Re c_j]."""
    return np.vstack([np.hstack([C0.real, C0.imag]), np.hstack([-C0.imag, C0.real])])


@pytest.mark.parametrize("m,n,seed,precondition", [(12, 3, 1, True), (20, 7, 2, True), (20, 7, 2, False)])
def test_hermitian_oracle_reaches_jacobi_brute_force(m, n, seed, precondition):
    H, S, T, eta, C0, w = hermitian_problem(m, n, seed)
    r = hermitian.solve(H, S, T, eta, 1.3, C0, tol_grad=1e-11, max_iter=5000, precondition=precondition)
    assert r["status"] == omm.STATUS_OK
    # brute force: the real form holds every eigenvalue twice, so E = sum of its 2n lowest
    we, _ = exact.eigenpairs(hermitian.embed(H), hermitian.embed(S), method="jacobi")
    assert r["E"] == pytest.approx(float(np.sum(we[:2 * n])), rel=1e-12, abs=1e-12)
    assert r["E"] == pytest.approx(2.0 * float(np.sum(w[:n])), rel=1e-12, abs=1e-12)
    ex = hermitian.exact_minimum(H, S, n)
    assert np.abs(r["D"] - ex["D"]).max() < 1e-9
    assert np.abs(r["EDM"] - ex["EDM"]).max() < 1e-9
    assert np.abs(r["SW"] - np.eye(n)).max() < 1e-9
    assert np.real(np.trace(r["D"] @ S)) == pytest.approx(2 * n, abs=1e-9)


def test_hermitian_oracle_follows_real_form_step_by_step():
    """The real form of the complex problem takes the same line-search steps, with twice the energy."""
    H, S, T, eta, C0, w = hermitian_problem(16, 5, 3)
    zc, zr = [], []
    hermitian.solve(H, S, T, eta, 1.3, C0, tol_grad=1e-30, max_iter=10,
                    callback=lambda it, E, x, b: zc.append((E, x, b)), want_matrices=False)
    omm.solve(hermitian.embed(H), hermitian.embed(S), hermitian.embed(T), eta, 1.3, embed_rows(C0),
              tol_grad=1e-30, max_iter=10, callback=lambda it, E, x, b: zr.append((E, x, b)),
              want_matrices=False)
    assert len(zc) == len(zr) == 10
    for (Ec, xc, bc), (Er, xr, br) in zip(zc, zr):
        assert Er == pytest.approx(2.0 * Ec, rel=1e-10, abs=1e-12)
        assert xr == pytest.approx(xc, rel=1e-8)
        assert br == pytest.approx(bc, rel=1e-7, abs=1e-12)


def test_hermitian_gradient_central_differences():
    """dE~ = Re Tr(G^H dC): G's real and imaginary parts are the derivatives in Re C and Im C."""
    H, S, T, eta, C0, w = hermitian_problem(10, 4, 4)
    Ht = H - eta * S
    C = C0.T.copy() * 5.0
    f = lambda C: hermitian.functional(C.conj().T @ Ht @ C, C.conj().T @ S @ C)
    G = hermitian.gradient(Ht @ C, S @ C, C.conj().T @ Ht @ C, C.conj().T @ S @ C)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 1), (9, 3)]:
        for unit, part in ((1.0, G.real), (1j, G.imag)):
            E = np.zeros_like(C)
            E[i, j] = unit * h
            fd = (f(C + E) - f(C - E)) / (2 * h)
            assert fd == pytest.approx(part[i, j], rel=1e-6, abs=1e-8)


def test_hermitian_quartic_matches_direct_evaluation():
    H, S, T, eta, C0, w = hermitian_problem(12, 4, 5)
    rng = np.random.default_rng(9)
    Ht = H - eta * S
    C = C0.T * 4.0
    Dl = (rng.normal(size=C.shape) + 1j * rng.normal(size=C.shape)) * 0.1
    h = lambda A: A.conj().T
    HW, SW = h(C) @ Ht @ C, h(C) @ S @ C
    a = hermitian.quartic_coefficients(hermitian.functional(HW, SW), HW, SW, h(Dl) @ Ht @ C, h(Dl) @ S @ C,
                                       h(Dl) @ Ht @ Dl, h(Dl) @ S @ Dl)
    for x in (-1.3, -0.2, 0.0, 0.4, 1.1, 2.5):
        Cx = C + x * Dl
        direct = hermitian.functional(h(Cx) @ Ht @ Cx, h(Cx) @ S @ Cx)
        assert omm.quartic_value(a, x) == pytest.approx(direct, rel=1e-11, abs=1e-11)


def test_hermitian_oracle_with_real_inputs_is_the_real_oracle():
    from tests.test_oracle_pins import tiny_problem
    H, S, T, eta, C0, w = tiny_problem(18, 6, 21)
    rc = hermitian.solve(H, S, T, eta, 2.0, C0.astype(complex), tol_grad=1e-11)
    rr = omm.solve(H, S, T, eta, 2.0, C0, tol_grad=1e-11)
    assert rc["iters"] == rr["iters"]
    assert rc["E"] == pytest.approx(rr["E"], rel=1e-13)
    assert np.abs(rc["D"].imag).max() == 0.0


# ---------------------------------------------------------------- the k-point generator
def test_kpoint_folding_matches_supercell_spectrum():
    """Bloch matrices of a 3 x 3 x 3 grid: Hermitian, complex, and their spectra together are the
    Gamma-point spectrum of the 27-cell supercell they were folded from."""
    import scipy.linalg
    from synth.kpoints import silicon_kpoints
    p = silicon_kpoints((3, 3, 3), keep_supercell=True)
    assert (p.m, p.n, len(p.H)) == (104, 16, 27)
    assert max(np.abs(h.imag).max() for h in p.H) > 1e-3
    w = np.sort(np.concatenate([scipy.linalg.eigh(h, s, eigvals_only=True) for h, s in zip(p.H, p.S)]))
    Hs, Ss = p.supercell
    ws = scipy.linalg.eigh(Hs, Ss, eigvals_only=True)
    assert np.abs(w - ws).max() < 1e-12
    # one eta inside the gap of the whole grid
    assert p.meta["homo"] < p.eta < p.meta["lumo"]


def test_kpoint_oracle_reaches_exact_minimum():
    from synth.kpoints import silicon_kpoints
    p = silicon_kpoints((3, 3, 3))
    for i in (1, 13):                                    # two complex k points
        r = hermitian.solve(p.H[i], p.S[i], p.T[i], p.eta, p.tau, p.C0[i], tol_grad=1e-9)
        ex = hermitian.exact_minimum(p.H[i], p.S[i], p.n)
        assert r["status"] == omm.STATUS_OK
        assert abs(r["E"] - ex["E"]) / abs(ex["E"]) < 1e-12
        assert np.abs(r["D"] - ex["D"]).max() < 1e-8


def test_bloch_sums_do_not_depend_on_the_supercell():
    """h(R) read from the 4x4x4 and from the 4x4x5 supercell give the same H(k), S(k) at
    Monkhorst-Pack points that neither supercell folds onto Gamma: no element mixes images."""
    from synth.kpoints import bloch_matrices, monkhorst_pack
    ks, _ = monkhorst_pack((9, 9, 9))
    pick = ks[[1, 40, 200]]
    H4, S4, _, _ = bloch_matrices(pick, sc=(4, 4, 4))
    H5, S5, _, _ = bloch_matrices(pick, sc=(4, 4, 5))
    for a, b in zip(H4 + S4, H5 + S5):
        assert np.abs(a - b).max() < 1e-13
    # time reversal: H(-k) = conj H(k)
    Hm, _, _, _ = bloch_matrices(-pick[:1])
    assert np.abs(Hm[0] - H4[0].conj()).max() < 1e-13


def test_monkhorst_pack_weights():
    from synth.kpoints import monkhorst_pack
    k, w = monkhorst_pack((9, 9, 9))
    assert len(k) == 365 and w.sum() == pytest.approx(1.0, abs=1e-14)
    k, w = monkhorst_pack((4, 4, 4), time_reversal=False)
    assert len(k) == 64 and np.all(w == 1.0 / 64)


def test_mp_grid_problems_are_well_posed():
    """Every problem of the 9 x 9 x 9 grid: Hermitian, S(k) positive definite, and the one eta lies
    above its n-th and below its (n+1)-th level (Sec. 2.2), so each OMM minimum is its band energy."""
    import scipy.linalg
    from synth.kpoints import silicon_mp_grid
    p = silicon_mp_grid((9, 9, 9))
    assert len(p.H) == 365 and sum(p.meta["weights"]) == pytest.approx(1.0, abs=1e-14)
    for h, s in zip(p.H, p.S):
        assert np.abs(h - h.conj().T).max() == 0.0 and np.abs(s - s.conj().T).max() == 0.0
        assert np.linalg.eigvalsh(s).min() > 1e-3
        e = scipy.linalg.eigh(h, s, eigvals_only=True, subset_by_index=[p.n - 1, p.n])
        assert e[0] < p.eta < e[1]


def test_neighbouring_k_point_start_saves_line_searches():
    """Sec. 3.3: solving the k points one after another, each from its neighbour's C, reuses
    information: fewer line searches than from the seeded start, the same minimum."""
    from synth.kpoints import silicon_mp_grid
    p = silicon_mp_grid((9, 9, 9))
    ks = np.array(p.k)
    path = sorted((i for i, k in enumerate(ks) if abs(k[1] - ks[0][1]) < 1e-12 and abs(k[2] - ks[0][2]) < 1e-12),
                  key=lambda i: ks[i][0])
    prev = None
    for i in path:
        cold = hermitian.solve(p.H[i], p.S[i], p.T[i], p.eta, p.tau, p.C0[i], tol_grad=1e-9, want_matrices=False)
        if prev is not None:
            warm = hermitian.solve(p.H[i], p.S[i], p.T[i], p.eta, p.tau, prev.T.copy(), tol_grad=1e-9,
                                   want_matrices=False)
            assert warm["iters"] < cold["iters"], (i, warm["iters"], cold["iters"])
            assert abs(warm["E"] - cold["E"]) <= 1e-12 * abs(cold["E"])
        prev = cold["C"]


# ---------------------------------------------------------------- graphene (the second k-point system)
@pytest.fixture(scope="module")
def graphene():
    from synth.kpoints import graphene_mp_grid
    return graphene_mp_grid((19, 19))


def test_graphene_grid_is_well_posed(graphene):
    """19 x 19 grid, k/-k merged: 181 Hermitian problems of m = 26, n = 4, S(k) positive definite,
    one eta inside every gap."""
    import scipy.linalg
    p = graphene
    assert (p.m, p.n, len(p.H)) == (26, 4, 181)
    assert sum(p.meta["weights"]) == pytest.approx(1.0, abs=1e-14)
    gaps = []
    for h, s in zip(p.H, p.S):
        assert np.abs(h - h.conj().T).max() == 0.0
        assert np.linalg.eigvalsh(s).min() > 1e-3
        e = scipy.linalg.eigh(h, s, eigvals_only=True, subset_by_index=[p.n - 1, p.n])
        assert e[0] < p.eta < e[1]
        gaps.append(e[1] - e[0])
    assert min(gaps) == pytest.approx(p.meta["min_gap"], rel=1e-12)


def test_graphene_bloch_sums_do_not_depend_on_the_supercell():
    from synth.kpoints import graphene_mp_grid
    p1 = graphene_mp_grid((5, 5), sc=(9, 6))
    p2 = graphene_mp_grid((5, 5), sc=(10, 7))
    for a, b in zip(p1.H + p1.S, p2.H + p2.S):
        assert np.abs(a - b).max() < 1e-13


def test_graphene_oracle_reaches_exact_minimum(graphene):
    p = graphene
    for i in (0, 90, int(np.argmin(p.meta["gaps"]))):              # incl. the smallest gap
        r = hermitian.solve(p.H[i], p.S[i], p.T[i], p.eta, p.tau, p.C0[i], tol_grad=1e-9)
        ex = hermitian.exact_minimum(p.H[i], p.S[i], p.n)
        assert r["status"] == omm.STATUS_OK
        assert abs(r["E"] - ex["E"]) / abs(ex["E"]) < 1e-12
        assert np.abs(r["D"] - ex["D"]).max() < 1e-8


def test_hermitian_backward_central_differences():
    """dE = Re Tr(D dH) - Re Tr(EDM dS) for Hermitian dH, dS (the convention of the complex
    dE/dH and dE/dS): central differences of re-solved energies."""
    H, S, T, eta, C0, w = hermitian_problem(14, 4, 7)
    r = hermitian.solve(H, S, T, eta, 1.3, C0, tol_grad=1e-12, max_iter=5000)
    Cstar = r["C"].T.copy()
    rng = np.random.default_rng(8)
    A = rng.normal(size=H.shape) + 1j * rng.normal(size=H.shape)
    dH = 0.5 * (A + A.conj().T)
    B = rng.normal(size=S.shape) + 1j * rng.normal(size=S.shape)
    dS = 0.05 * (B + B.conj().T)
    h = 1e-5
    Ep = hermitian.solve(H + h * dH, S, T, eta, 1.3, Cstar, tol_grad=1e-12)["E"]
    Em = hermitian.solve(H - h * dH, S, T, eta, 1.3, Cstar, tol_grad=1e-12)["E"]
    assert (Ep - Em) / (2 * h) == pytest.approx(float(np.real(np.trace(r["D"] @ dH))), rel=1e-7, abs=1e-8)
    Ep = hermitian.solve(H, S + h * dS, T, eta, 1.3, Cstar, tol_grad=1e-12)["E"]
    Em = hermitian.solve(H, S - h * dS, T, eta, 1.3, Cstar, tol_grad=1e-12)["E"]
    assert (Ep - Em) / (2 * h) == pytest.approx(-float(np.real(np.trace(r["EDM"] @ dS))), rel=1e-7, abs=1e-8)


def test_hermitian_cholesky_flavour():
    """Complex Cholesky flavour: the brute-force minimum, and the steps of the S^-1-preconditioned
    complex method (Sec. 2.4)."""
    H, S, T, eta, C0, w = hermitian_problem(18, 6, 9)
    r = hermitian.solve_cholesky(H, S, eta, C0, tol_grad=1e-11, max_iter=5000)
    assert r["status"] == omm.STATUS_OK
    assert r["E"] == pytest.approx(2.0 * float(np.sum(w[:6])), rel=1e-12, abs=1e-12)
    ex = hermitian.exact_minimum(H, S, 6)
    assert np.abs(r["D"] - ex["D"]).max() < 1e-9
    assert np.abs(r["EDM"] - ex["EDM"]).max() < 1e-9
    Cm = r["C"]
    assert np.abs(Cm.conj().T @ S @ Cm - np.eye(6)).max() < 1e-9
    red, orig = [], []
    hermitian.solve_cholesky(H, S, eta, C0, tol_grad=1e-30, max_iter=10,
                             callback=lambda it, E, x, b: red.append((E, x)), want_matrices=False)
    hermitian.solve(H, S, None, eta, math.inf, C0, tol_grad=1e-30, max_iter=10,
                    callback=lambda it, E, x, b: orig.append((E, x)), want_matrices=False)
    for (Er, xr), (Eo, xo) in zip(red, orig):
        assert Er == pytest.approx(Eo, rel=1e-10, abs=1e-12)
        assert xr == pytest.approx(xo, rel=1e-7)
