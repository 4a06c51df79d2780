"""Pins of the oracle's conjugate-gradient step (Sec. 2.3-2.4) through identities it must satisfy.

The Polak-Ribiere coefficient beta = <G_k, P(G_k - G_{k-1})> / <G_{k-1}, P G_{k-1}> is not
pinned by the fixed point (any beta reaches the same minimum). With exact line searches, which
the quartic minimum gives, it equals the Hestenes-Stiefel coefficient
<P G_k, G_k - G_{k-1}> / <Delta_{k-1}, G_k - G_{k-1}>: the denominators agree because
<G_k, Delta_{k-1}> = 0 (exact line search) and <G_{k-1}, Delta_{k-1}> = -<G_{k-1}, P G_{k-1}>
(the previous direction's own recurrence and exact line search). The test below rebuilds the
directions from the iterates alone, Delta_k = (C_{k+1} - C_k) / x_k, and checks that
identity, the exact-line-search orthogonality and the direction recurrence; a dropped term, a
wrong sign or a misplaced preconditioner in beta breaks the first.
"""
import math

import numpy as np
import pytest

from oracle import omm


def _problem(m, n, seed, gap=0.3):
    """Random symmetric H, SPD S and SPD T with a generalised gap at n (the pins' recipe)."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, m))
    S = np.eye(m) + 0.08 * (A + A.T) / math.sqrt(m)
    S = S @ S.T / np.max(np.abs(np.linalg.eigvalsh(S @ S.T)))
    S = 0.5 * (S + S.T) + 0.2 * np.eye(m)
    B = rng.normal(size=(m, m))
    T = B @ B.T / m + 0.1 * np.eye(m)
    L = np.linalg.cholesky(S)
    Q, _ = np.linalg.qr(rng.normal(size=(m, m)))
    X = np.linalg.solve(L.T, Q)
    w = np.sort(rng.uniform(-1.0, 1.0, size=m))
    w[n:] += gap
    H = S @ X @ np.diag(w) @ X.T @ S
    H = 0.5 * (H + H.T)
    eta = 0.5 * (w[n - 1] + w[n])
    C0 = rng.normal(0.0, 0.1, size=(n, m)) / math.sqrt(m)
    return H, S, T, eta, C0


def _iterate(H, S, T, eta, tau, C0, k, precondition):
    """C (m x n) after k line searches, and the (x, beta) of every line search."""
    steps = []
    r = omm.solve(H, S, T, eta, tau, C0, tol_grad=0.0, max_iter=k, precondition=precondition,
                  callback=lambda it, E, x, beta: steps.append((x, beta)), want_matrices=False)
    return r["C"], steps


@pytest.mark.parametrize("m,n,seed,precondition", [(24, 6, 21, True), (30, 9, 22, True), (24, 6, 23, False)])
def test_polak_ribiere_equals_hestenes_stiefel(m, n, seed, precondition):
    H, S, T, eta, C0 = _problem(m, n, seed)
    tau = 1.3
    K = 12
    Ht = omm.shift(H, S, eta)
    P = omm.preconditioner(S, T, tau) if precondition else np.eye(m)
    Cs = [_iterate(H, S, T, eta, tau, C0, k, precondition)[0] for k in range(K + 1)]
    _, steps = _iterate(H, S, T, eta, tau, C0, K, precondition)
    assert len(steps) == K

    def grad(C):
        HC, SC, HW, SW = omm.subspace_operators(C, Ht, S)
        return omm.gradient(HC, SC, HW, SW)

    Gs = [grad(C) for C in Cs]
    D = [(Cs[k + 1] - Cs[k]) / steps[k][0] for k in range(K)]
    checked = 0
    for k in range(K - 1):
        G0, G1 = Gs[k], Gs[k + 1]
        # exact line search along D[k]: the new gradient is orthogonal to it
        assert abs(np.vdot(G1, D[k])) <= 1e-8 * np.linalg.norm(G1) * np.linalg.norm(D[k])
        beta = steps[k + 1][1]
        if beta <= 0.0:
            continue
        # the next direction is -P G + beta D (no restart at these steps)
        assert np.allclose(D[k + 1], -P @ G1 + beta * D[k], rtol=0, atol=1e-7 * np.max(np.abs(D[k + 1])))
        dG = G1 - G0
        beta_hs = np.vdot(P @ G1, dG) / np.vdot(D[k], dG)
        assert beta == pytest.approx(beta_hs, rel=1e-6)
        checked += 1
    assert checked >= 5


def test_hestenes_stiefel_pin_catches_a_wrong_beta():
    """The same identity fails for the Fletcher-Reeves coefficient <G_k, P G_k> / <G_{k-1}, P G_{k-1}>
    computed on the oracle's own iterates: the pin separates the two formulas."""
    H, S, T, eta, C0 = _problem(24, 6, 21)
    tau = 1.3
    Ht = omm.shift(H, S, eta)
    P = omm.preconditioner(S, T, tau)
    Cs = [_iterate(H, S, T, eta, tau, C0, k, True)[0] for k in range(6)]
    _, steps = _iterate(H, S, T, eta, tau, C0, 5, True)

    def grad(C):
        HC, SC, HW, SW = omm.subspace_operators(C, Ht, S)
        return omm.gradient(HC, SC, HW, SW)

    G = [grad(C) for C in Cs]
    D = [(Cs[k + 1] - Cs[k]) / steps[k][0] for k in range(5)]
    far = 0
    for k in range(1, 4):
        dG = G[k + 1] - G[k]
        beta_hs = np.vdot(P @ G[k + 1], dG) / np.vdot(D[k], dG)
        beta_fr = np.vdot(G[k + 1], P @ G[k + 1]) / np.vdot(G[k], P @ G[k])
        far += abs(beta_fr - beta_hs) > 1e-3 * abs(beta_hs)
    assert far >= 2


def _hermitian_problem(m, n, seed, gap=0.3):
    """Random Hermitian H, Hermitian positive definite S and T with a generalised gap at n."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    S = np.eye(m) + 0.05 * (A + A.conj().T) / math.sqrt(m)
    S = S @ S.conj().T
    S = 0.5 * (S + S.conj().T) / np.linalg.eigvalsh(S).max() + 0.2 * np.eye(m)
    B = rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))
    T = B @ B.conj().T / m + 0.1 * np.eye(m)
    L = np.linalg.cholesky(S)
    Q, _ = np.linalg.qr(rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m)))
    X = np.linalg.solve(L.conj().T, Q)
    w = np.sort(rng.uniform(-1.0, 1.0, size=m))
    w[n:] += gap
    H = S @ X @ np.diag(w) @ X.conj().T @ S
    H = 0.5 * (H + H.conj().T)
    eta = 0.5 * (w[n - 1] + w[n])
    C0 = (rng.normal(0.0, 0.1, size=(n, m)) + 1j * rng.normal(0.0, 0.1, size=(n, m))) / math.sqrt(2 * m)
    return H, S, T, eta, C0


@pytest.mark.parametrize("m,n,seed", [(20, 5, 31), (24, 8, 32)])
def test_hermitian_polak_ribiere_equals_hestenes_stiefel(m, n, seed):
    """The same identity for complex C with the real inner product Re Tr(A^H B) (Secs. 2.1-2.3
    written with Hermitian conjugates), on the complex oracle's iterates."""
    from oracle import hermitian

    H, S, T, eta, C0 = _hermitian_problem(m, n, seed)
    tau = 1.3
    K = 10
    Ht = H - eta * S
    P = hermitian.preconditioner(S, T, tau)
    rdot = lambda A, B: float(np.real(np.vdot(A, B)))

    def run(k):
        steps = []
        r = hermitian.solve(H, S, T, eta, tau, C0, tol_grad=0.0, max_iter=k,
                            callback=lambda it, E, x, beta: steps.append((x, beta)), want_matrices=False)
        return r["C"], steps

    def grad(C):
        HC, SC = Ht @ C, S @ C
        return hermitian.gradient(HC, SC, C.conj().T @ HC, C.conj().T @ SC)

    Cs = [run(k)[0] for k in range(K + 1)]
    _, steps = run(K)
    Gs = [grad(C) for C in Cs]
    D = [(Cs[k + 1] - Cs[k]) / steps[k][0] for k in range(K)]
    checked = 0
    for k in range(K - 1):
        G0, G1 = Gs[k], Gs[k + 1]
        assert abs(rdot(G1, D[k])) <= 1e-8 * np.linalg.norm(G1) * np.linalg.norm(D[k])
        beta = steps[k + 1][1]
        if beta <= 0.0:
            continue
        assert np.allclose(D[k + 1], -P @ G1 + beta * D[k], rtol=0, atol=1e-7 * np.max(np.abs(D[k + 1])))
        dG = G1 - G0
        assert beta == pytest.approx(rdot(P @ G1, dG) / rdot(D[k], dG), rel=1e-6)
        checked += 1
    assert checked >= 4
