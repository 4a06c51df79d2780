"""GPU parity of the Hermitian (complex, k-point) entry points through the C ABI.

Bulk Si in its 8-atom cell (DZP-like: m = 104, n = 16) on a 3 x 3 x 3 k grid, as in the
paper's k-point tests (Sec. 3.3). Checked against the complex oracle and the plain definition
of the minimum (LAPACK eigenpairs of each H(k) x = eps S(k) x), and the grid as a whole
against the Gamma-point band energy of the 27-cell supercell it was folded from.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def zdev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


@pytest.fixture(scope="module")
def S():
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300 import solver
    return solver


@pytest.fixture(scope="module")
def grid():
    from synth.kpoints import silicon_kpoints
    return silicon_kpoints((3, 3, 3), keep_supercell=True)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ik", [1, 13, 0])            # two complex k points and Gamma
def test_hermitian_solve_matches_oracle(S, grid, precision, ik):
    from oracle import hermitian
    p = grid
    H, Sk, T, C0 = p.H[ik], p.S[ik], p.T[ik], p.C0[ik]
    ex = hermitian.exact_minimum(H, Sk, p.n)
    with S.OMMHermitian(zdev(H), zdev(Sk), zdev(T), p.n, p.eta, p.tau, precision=precision) as s:
        C, E, D, info = s.solve(zdev(C0), want_D=True)
        dH, dS = s.backward()
    C, D, dH, dS = (t.cpu().numpy() for t in (C, D, dH, dS))
    assert info["status"] == 0 and info["gmax"] < 1e-9
    tol = 1e-10 if precision == "fp64" else 1e-9
    assert abs(E - ex["E"]) / abs(ex["E"]) <= tol
    assert abs(info["E"] - E) <= 1e-12 * abs(E)
    assert np.abs(D - ex["D"]).max() <= 1e-7
    assert np.abs(dH - D).max() == 0.0
    assert np.abs(dS + ex["EDM"]).max() <= 1e-7
    Cm = C.T                                            # paper layout m x n
    assert np.abs(Cm.conj().T @ Sk @ Cm - np.eye(p.n)).max() < 1e-8
    if precision == "fp64":
        ref = hermitian.solve(H, Sk, T, p.eta, p.tau, C0, tol_grad=1e-9, want_matrices=False)
        assert abs(info["iterations"] - ref["iters"]) <= max(3, ref["iters"] // 10)


def test_hermitian_host_buffers_and_cholesky(S, grid):
    """numpy (host) complex buffers, and the Cholesky flavour of a complex problem."""
    from oracle import hermitian
    p = grid
    ex = hermitian.exact_minimum(p.H[5], p.S[5], p.n)
    with S.OMMHermitian(p.H[5], p.S[5], None, p.n, p.eta, p.tau, cholesky=True) as s:
        C, E, D, info = s.solve(p.C0[5].copy(), want_D=True)
    assert isinstance(C, np.ndarray) and C.dtype == np.complex128
    assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-10
    assert np.abs(D - ex["D"]).max() <= 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hermitian_batch_over_the_grid(S, grid, precision):
    """All 27 k points in one batch: each reaches its own minimum, and together the band energy
    of the supercell they were folded from (sum over k of E(k) = E of the 27-cell Gamma point)."""
    import scipy.linalg
    from oracle import hermitian
    p = grid
    probs = [(zdev(p.H[i]), zdev(p.S[i]), zdev(p.T[i]), p.n, p.eta, p.tau) for i in range(len(p.H))]
    with S.OMMHermitianBatch(probs, precision=precision) as b:
        Cs, Es, infos = b.solve([zdev(c) for c in p.C0])
        dH, dS = b.backward(7)
    for i, (E, info) in enumerate(zip(Es, infos)):
        ex = hermitian.exact_minimum(p.H[i], p.S[i], p.n)
        assert info["status"] == 0
        assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-9
    ex7 = hermitian.exact_minimum(p.H[7], p.S[7], p.n)
    assert np.abs(dH.cpu().numpy() - ex7["D"]).max() <= 1e-7
    Hs, Ss = p.supercell
    w = scipy.linalg.eigh(Hs, Ss, eigvals_only=True, subset_by_index=[0, p.n * len(p.H) - 1])
    assert abs(Es.sum() - 2.0 * w.sum()) / abs(2.0 * w.sum()) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hermitian_warm_start_update_H(S, grid, precision):
    from oracle import hermitian
    p = grid
    rng = np.random.default_rng(3)
    H2 = p.H[13] + np.diag(rng.normal(0.0, 0.01, size=p.m))
    with S.OMMHermitian(zdev(p.H[13]), zdev(p.S[13]), zdev(p.T[13]), p.n, p.eta, p.tau, precision=precision) as s:
        C, E, _, i0 = s.solve(zdev(p.C0[13]))
        s.update_H(zdev(H2))
        C2, E2, D2, i1 = s.solve(C, want_D=True)
    ex2 = hermitian.exact_minimum(H2, p.S[13], p.n)
    assert i1["status"] == 0
    assert abs(E2 - ex2["E"]) / abs(ex2["E"]) <= 1e-9
    assert np.abs(D2.cpu().numpy() - ex2["D"]).max() <= 1e-7
    assert i1["iterations"] < i0["iterations"]


def test_real_entry_points_reject_hermitian_context(S, grid):
    import ctypes as ct
    from paper_1312_1549_gb300 import _native as N
    p = grid
    with S.OMMHermitian(zdev(p.H[1]), zdev(p.S[1]), zdev(p.T[1]), p.n, p.eta, p.tau) as s:
        C0 = torch.zeros((2 * p.n, 2 * p.m), dtype=torch.float64, device="cuda")
        E = ct.c_double(0.0)
        rc = N.lib().omm_solve(s._h, ct.c_void_p(C0.data_ptr()), None, ct.byref(E), None, None)
        assert rc == 1
        assert N.lib().omm_backward(s._h, None, None) == 1


def test_neighbouring_k_point_start(S, grid):
    """Sec. 3.3: the converged C of one k point as the start of its neighbour: fewer line searches
    than from the seeded start, the neighbour's own minimum (float64 path)."""
    from oracle import hermitian
    p = grid
    a, b = 1, 2                                        # neighbours along the third axis of the grid
    with S.OMMHermitian(zdev(p.H[a]), zdev(p.S[a]), zdev(p.T[a]), p.n, p.eta, p.tau) as s:
        Ca, _, _, _ = s.solve(zdev(p.C0[a]))
    with S.OMMHermitian(zdev(p.H[b]), zdev(p.S[b]), zdev(p.T[b]), p.n, p.eta, p.tau) as s:
        _, E_cold, _, i_cold = s.solve(zdev(p.C0[b]))
        _, E_warm, _, i_warm = s.solve(Ca)
    ex = hermitian.exact_minimum(p.H[b], p.S[b], p.n)
    assert abs(E_warm - ex["E"]) / abs(ex["E"]) <= 1e-10
    assert i_warm["iterations"] < i_cold["iterations"], (i_warm["iterations"], i_cold["iterations"])
