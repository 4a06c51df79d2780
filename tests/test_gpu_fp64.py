"""GPU parity of the float64 path against the oracle (through the C ABI)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300 import solver
    return solver


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------- float64 GEMM
@pytest.mark.parametrize("tA,tB", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (64, 64, 16), (77, 130, 45), (200, 63, 257)])
def test_dgemm_matches_fp64_matmul(S, tA, tB, M, N, K):
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.normal(size=(K, M) if tA else (M, K))
    B = rng.normal(size=(N, K) if tB else (K, N))
    C0 = rng.normal(size=(M, N))
    ref = 1.5 * (A.T if tA else A) @ (B.T if tB else B) - 0.5 * C0
    C = dev(C0)
    S.dgemm(tA, tB, dev(A), dev(B), C, alpha=1.5, beta=-0.5)
    assert np.allclose(C.cpu().numpy(), ref, rtol=1e-13, atol=1e-12 * np.sqrt(K))


def test_dgemm_empty_k(S):
    C = dev(np.ones((5, 7)))
    A = dev(np.zeros((5, 1)))
    B = dev(np.zeros((1, 7)))
    import ctypes as ct
    from paper_1312_1549_gb300 import _native as N
    rc = N.lib().omm_kernel_dgemm(0, 0, 5, 7, 0, 1.0, ct.c_void_p(A.data_ptr()), 1,
                                  ct.c_void_p(B.data_ptr()), 7, 2.0, ct.c_void_p(C.data_ptr()), 7, None)
    assert rc == 0
    assert np.all(C.cpu().numpy() == 2.0)


# ---------------------------------------------------------------- Cholesky inverse
@pytest.mark.parametrize("m", [1, 5, 64, 65, 200, 333])
def test_spd_inverse(S, m):
    rng = np.random.default_rng(m)
    X = rng.normal(size=(m, m))
    A = X @ X.T / m + 0.5 * np.eye(m)
    P = S.spd_inverse(dev(A)).cpu().numpy()
    assert np.allclose(P, P.T, atol=0)
    assert np.allclose(P @ A, np.eye(m), atol=1e-11)


def test_spd_inverse_rejects_indefinite(S):
    A = np.eye(70)
    A[40, 40] = -1.0
    from paper_1312_1549_gb300 import _native as N
    with pytest.raises(N.OMMError) as e:
        S.spd_inverse(dev(A))
    assert e.value.status == 2


def test_preconditioner_of_si64(S):
    from synth import si64_sz
    from oracle import omm
    p = si64_sz()
    P_ref = omm.preconditioner(p.S, p.T, p.tau)
    P = S.spd_inverse(dev(p.S + p.T / p.tau)).cpu().numpy()
    assert np.abs(P - P_ref).max() < 1e-11 * np.abs(P_ref).max()


# ---------------------------------------------------------------- quartic and line minimum
def test_line_minimum_matches_oracle(S):
    from oracle import omm
    rng = np.random.default_rng(5)
    for _ in range(200):
        a = rng.normal(size=5)
        a[1] = -abs(a[1])
        x, rc = S.line_minimum(a)
        xo, so = omm.line_minimum(a)
        assert (rc == 0) == (so == omm.STATUS_OK)
        if rc == 0:
            assert x == pytest.approx(xo, rel=1e-10, abs=1e-14)


def test_quartic_coefficients_match_oracle(S):
    from oracle import omm
    rng = np.random.default_rng(8)
    m, n = 90, 37
    X = rng.normal(size=(m, m)); Ht = 0.5 * (X + X.T)
    Y = rng.normal(size=(m, m)); Sm = Y @ Y.T / m + np.eye(m)
    C = rng.normal(size=(m, n)); Dl = rng.normal(size=(m, n))
    HC, SC, HW, SW = omm.subspace_operators(C, Ht, Sm)
    E = omm.functional_from_subspace(HW, SW)
    H1, S1, H2, S2 = Dl.T @ HC, Dl.T @ SC, Dl.T @ Ht @ Dl, Dl.T @ Sm @ Dl
    ref = omm.quartic_coefficients(E, HW, SW, H1, S1, H2, S2)
    SWHW = np.hstack([SW, HW])
    Proj = np.hstack([H1, S1, H2, S2])
    a = S.quartic_coefficients(dev(SWHW), dev(Proj), E)
    assert np.allclose(a, ref, rtol=1e-12, atol=1e-10)


# ---------------------------------------------------------------- whole solve, Si64
@pytest.fixture(scope="module")
def si64():
    from synth import si64_sz
    from oracle import exact, omm
    p = si64_sz()
    ref = omm.solve(p.H, p.S, p.T, p.eta, p.tau, p.C0, tol_grad=1e-9)
    ex = exact.exact_minimum(p.H, p.S, p.n)
    return p, ref, ex


def _solve(S, p, **kw):
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, **kw) as s:
        C, E, D, info = s.solve(dev(p.C0), want_D=True)
        dH, dS = s.backward()
    return C.cpu().numpy(), E, D.cpu().numpy(), info, dH.cpu().numpy(), dS.cpu().numpy()


def test_fp64_solve_si64_matches_oracle(S, si64):
    p, ref, ex = si64
    C, E, D, info, dH, dS = _solve(S, p)
    assert info["status"] == 0 and info["gmax"] < 1e-9
    assert abs(E - ref["E"]) / abs(ref["E"]) <= 1e-10
    assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-10
    assert np.abs(D - ref["D"]).max() <= 1e-7
    assert np.abs(D - ex["D"]).max() <= 1e-7
    Cm = C.T
    SW = Cm.T @ p.S @ Cm
    assert np.abs(SW - np.eye(p.n)).max() < 1e-8
    assert np.trace(D @ p.S) == pytest.approx(2 * p.n, abs=1e-7)
    assert np.abs(dH - D).max() == 0.0
    assert np.abs(dS + ex["EDM"]).max() <= 1e-7


def test_fp64_solve_host_pointers(S, si64):
    """The same solve through host (numpy) buffers: copies in and out inside the library."""
    p, ref, ex = si64
    with S.OMMSolver(p.H, p.S, p.T, p.n, p.eta, p.tau) as s:
        C, E, D, info = s.solve(p.C0.copy(), want_D=True)
    assert isinstance(C, np.ndarray) and isinstance(D, np.ndarray)
    assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-10
    assert np.abs(D - ex["D"]).max() <= 1e-7


def test_fp64_solve_without_preconditioner(S, si64):
    p, ref, ex = si64
    C, E, D, info, dH, dS = _solve(S, p, precondition=False)
    assert info["status"] == 0
    assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-10


def test_fp64_energy_criterion(S, si64):
    """Eq. 18 (read with |.|) stops earlier than the gradient test."""
    p, ref, ex = si64
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, e_tol=1e-9, tol_grad=1e-14) as s:
        C, E, D, info = s.solve(dev(p.C0))
    assert info["status"] == 0
    assert abs(E - ex["E"]) / abs(ex["E"]) < 1e-8


def test_iteration_cap_reports_no_convergence(S, si64):
    p, ref, ex = si64
    from paper_1312_1549_gb300 import _native as N
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, max_iter=3) as s:
        with pytest.raises(N.OMMError) as e:
            s.solve(dev(p.C0))
        assert e.value.status == 4
        assert s.info["iterations"] == 3


def test_nonfinite_input_is_reported(S, si64):
    p, ref, ex = si64
    H = p.H.copy()
    H[3, 3] = np.nan
    from paper_1312_1549_gb300 import _native as N
    with S.OMMSolver(dev(H), dev(p.S), dev(p.T), p.n, p.eta, p.tau) as s:
        with pytest.raises(N.OMMError) as e:
            s.solve(dev(p.C0))
        assert e.value.status == 5


def test_not_spd_preconditioner_is_reported(S, si64):
    p, ref, ex = si64
    from paper_1312_1549_gb300 import _native as N
    with pytest.raises(N.OMMError) as e:
        S.OMMSolver(dev(p.H), dev(-p.S), dev(p.T), p.n, p.eta, p.tau)
    assert e.value.status == 2


def test_backward_before_solve_is_rejected(S, si64):
    p, ref, ex = si64
    from paper_1312_1549_gb300 import _native as N
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau) as s:
        with pytest.raises(N.OMMError) as e:
            s.backward()
        assert e.value.status == 9


def test_warm_start_update_H(S, si64):
    """omm_update_H + a solve from the previous C: one of the SCF-sequence steps (Sec. 2.5.2)."""
    p, ref, ex = si64
    from oracle import exact
    rng = np.random.default_rng(3)
    delta = np.diag(rng.normal(0.0, 0.01, size=p.m))
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau) as s:
        C, E, _, info0 = s.solve(dev(p.C0))
        s.update_H(dev(p.H + delta))
        C2, E2, D2, info1 = s.solve(C, want_D=True)
    ex2 = exact.exact_minimum(p.H + delta, p.S, p.n)
    assert abs(E2 - ex2["E"]) / abs(ex2["E"]) <= 1e-10
    assert np.abs(D2.cpu().numpy() - ex2["D"]).max() <= 1e-7
    assert info1["iterations"] < info0["iterations"]
