"""GPU parity of the tensor-core (tcgen05) contraction and of the mixed-precision solve."""
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


def bf16_round(x):
    """float64 -> nearest bf16 (8 significant bits, ties to even), rounded once."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


@pytest.mark.parametrize("tile_n", [256, 128])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (130, 257, 70), (256, 512, 1000), (1, 1, 1), (384, 96, 200)])
def test_gemm_tc_single_pass_is_exact_bf16_product(S, M, N, K, tile_n):
    """npass = 1: the product of the bf16-rounded operands up to FP32 accumulation (K * 2^-23)."""
    rng = np.random.default_rng(M + N + K)
    A = rng.normal(size=(M, K)); B = rng.normal(size=(N, K))
    C = dev(np.zeros((M, N)))
    S.gemm_tc(dev(A), dev(B), C, npass=1, tile_n=tile_n)
    ref = bf16_round(A) @ bf16_round(B).T
    scale = np.abs(bf16_round(A)) @ np.abs(bf16_round(B)).T
    assert np.all(np.abs(C.cpu().numpy() - ref) <= K * 2.0 ** -23 * scale + 1e-30)


@pytest.mark.parametrize("tile_n", [256, 128])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (130, 300, 72), (200, 512, 1000), (1024, 640, 256)])
def test_gemm_tc_kn_matches_the_k_major_product(S, M, N, K, tile_n):
    """B given K x N and read MN-major (the gradient product's layout): within the split error bound
    2^-14 |A||B| and the same bits as the K-major kernel on B^T (the same MMAs in the same order)."""
    rng = np.random.default_rng(3 * M + N + K)
    A = rng.normal(size=(M, K)); B = rng.normal(size=(K, N))
    C0 = rng.normal(size=(M, N))
    C = dev(C0)
    S.gemm_tc_kn(dev(A), dev(B), C, alpha=2.0, beta=-1.0, tile_n=tile_n)
    ref = 2.0 * A @ B - C0
    scale = 2.0 * np.abs(A) @ np.abs(B)
    got = C.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 2.0 ** -14 * scale + 1e-12)
    Ck = dev(C0)
    S.gemm_tc(dev(A), dev(np.ascontiguousarray(B.T)), Ck, alpha=2.0, beta=-1.0, npass=3, tile_n=tile_n)
    assert np.array_equal(got, Ck.cpu().numpy())


@pytest.mark.parametrize("tile_n", [256, 128])
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (200, 300, 100), (256, 512, 1024), (129, 700, 333)])
def test_gemm_tc_split_error_bound(S, M, N, K, tile_n):
    """npass = 3: error of the 3-term split product within 2^-14 |A||B|^T elementwise."""
    rng = np.random.default_rng(7 * M + N + K)
    A = rng.normal(size=(M, K)); B = rng.normal(size=(N, K))
    C0 = rng.normal(size=(M, N))
    C = dev(C0)
    S.gemm_tc(dev(A), dev(B), C, alpha=2.0, beta=-1.0, npass=3, tile_n=tile_n)
    ref = 2.0 * A @ B.T - C0
    scale = 2.0 * np.abs(A) @ np.abs(B).T
    err = np.abs(C.cpu().numpy() - ref)
    assert np.all(err <= 2.0 ** -14 * scale + 1e-12)
    # and far better than the single pass
    C1 = dev(np.zeros((M, N)))
    S.gemm_tc(dev(A), dev(B), C1, npass=1)
    e1 = np.abs(C1.cpu().numpy() - A @ B.T).max()
    assert err.max() < e1 / 50


@pytest.fixture(scope="module")
def si64():
    from synth import si64_sz
    from oracle import exact, omm
    p = si64_sz()
    ref = omm.solve(p.H, p.S, p.T, p.eta, p.tau, p.C0, tol_grad=1e-9)
    ex = exact.exact_minimum(p.H, p.S, p.n)
    return p, ref, ex


def test_mixed_solve_si64_matches_oracle(S, si64):
    p, ref, ex = si64
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, precision="mixed") as s:
        C, E, D, info = s.solve(dev(p.C0), want_D=True)
        dH, dS = s.backward()
    D = D.cpu().numpy()
    assert info["status"] == 0 and info["gmax"] < 1e-9
    assert info["gemm_flop_tc"] > 0
    assert abs(E - ref["E"]) / abs(ref["E"]) <= 1e-9
    assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-9
    assert np.abs(D - ex["D"]).max() <= 1e-7
    Cm = C.cpu().numpy().T
    assert np.abs(Cm.T @ p.S @ Cm - np.eye(p.n)).max() < 1e-8
    assert np.abs(dS.cpu().numpy() + ex["EDM"]).max() <= 1e-7


def test_mixed_solve_without_preconditioner(S, si64):
    p, ref, ex = si64
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, precision="mixed",
                     precondition=False) as s:
        C, E, D, info = s.solve(dev(p.C0), want_D=True)
    assert info["status"] == 0
    assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-9
    assert np.abs(D.cpu().numpy() - ex["D"]).max() <= 1e-7


# few output tiles: every chunk on its own CTA and a reduction; (1024, 4096, 2048): 128 tiles, chunks in
# order on one CTA per tile; (1024, 6144, 1000) and (2048, 5000, 333): at least a wave of 256-row tiles,
# chunks in order on SM pairs
@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (200, 300, 1000), (64, 1000, 6656), (130, 70, 16384),
                                   (1024, 4096, 2048), (1024, 6144, 1000), (2048, 5000, 333)])
def test_gemm_emu_is_float64_class(S, M, N, K):
    """10 fixed-point slices: error within 2^-44 of |alpha||A||B|^T + |beta C| elementwise."""
    rng = np.random.default_rng(M * N + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.normal(size=(M, 1)))   # rows of different scales
    B = rng.normal(size=(N, K))
    C0 = rng.normal(size=(M, N))
    C = dev(C0)
    S.gemm_emu(dev(A), dev(B), C, alpha=-4.0, beta=1.0, slices=10)
    ref = -4.0 * A @ B.T + C0
    scale = 4.0 * np.abs(A) @ np.abs(B).T + np.abs(C0)
    assert np.all(np.abs(C.cpu().numpy() - ref) <= 2.0 ** -44 * scale)


def test_gemm_emu_error_falls_with_slices(S):
    rng = np.random.default_rng(5)
    A = rng.normal(size=(128, 512)); B = rng.normal(size=(256, 512))
    ref = A @ B.T
    errs = []
    for s in (2, 4, 6, 8):
        C = dev(np.zeros((128, 256)))
        S.gemm_emu(dev(A), dev(B), C, slices=s)
        errs.append(np.abs(C.cpu().numpy() - ref).max())
    assert all(errs[i + 1] < errs[i] / 100 for i in range(3)), errs


def test_mixed_solve_with_native_certificate(S, si64):
    """A native float64 certificate and density matrix meet the same bars as the sliced ones."""
    p, ref, ex = si64
    with S.OMMSolver(dev(p.H), dev(p.S), dev(p.T), p.n, p.eta, p.tau, precision="mixed",
                     native_certificate=True) as s:
        C, E, D, info = s.solve(dev(p.C0), want_D=True)
    assert info["status"] == 0 and info["gmax"] < 1e-9
    assert abs(E - ex["E"]) / abs(ex["E"]) <= 1e-9
    assert np.abs(D.cpu().numpy() - ex["D"]).max() <= 1e-7


# ---------------------------------------------------------------- float64-class preconditioner inverse
# Every off-diagonal product of the recursive factorisation carries at most about 2^-44 of
# |A||B| (10 slices, see test_gemm_emu_is_float64_class); with condition numbers near 10 the
# residual P A - I stays within 1e-11, as for the native float64 path.
@pytest.mark.parametrize("m", [1, 5, 64, 65, 128, 200, 333, 1000, 2500])
def test_spd_inverse_sliced(S, m):
    rng = np.random.default_rng(m)
    X = rng.normal(size=(m, m))
    A = X @ X.T / m + 0.5 * np.eye(m)
    P = S.spd_inverse(dev(A), sliced=True).cpu().numpy()
    assert np.array_equal(P, P.T)
    assert np.abs(P @ A - np.eye(m)).max() <= 1e-11


def test_spd_inverse_sliced_rejects_indefinite(S):
    A = np.eye(200)
    A[150, 150] = -1.0
    from paper_1312_1549_gb300 import _native as N
    with pytest.raises(N.OMMError) as e:
        S.spd_inverse(dev(A), sliced=True)
    assert e.value.status == 2


def test_spd_inverse_sliced_preconditioner_matches_oracle(S):
    from synth import configs
    from oracle import omm
    p = configs.silicon(k=(2, 2, 2), basis="DZP", seed=0)   # m = 832
    P_ref = omm.preconditioner(p.S, p.T, p.tau)
    P = S.spd_inverse(dev(p.S + p.T / p.tau), sliced=True).cpu().numpy()
    assert np.abs(P - P_ref).max() <= 1e-11 * np.abs(P_ref).max()


# The preconditioner-grade inverses: float32 leaves and, for slices = 1 (the mixed solver's default),
# every product of the recursion in the 3-term bf16 split form (about 2^-16 of |A||B|), else that many
# 5-bit fixed-point slices (5 slices: about 2^-24 of each row-scaled operand). P reaches the line
# searches only through its bf16 rounding (2^-9 of each element, the single-pass P G); the residual
# bounds below (condition numbers near 10) keep P well inside that.
@pytest.mark.parametrize("m", [5, 65, 200, 1000, 2500])
@pytest.mark.parametrize("slices", [1, 5, 7])
def test_spd_inverse_precond(S, m, slices):
    rng = np.random.default_rng(m)
    X = rng.normal(size=(m, m))
    A = X @ X.T / m + 0.5 * np.eye(m)
    P = S.spd_inverse(dev(A), slices=slices).cpu().numpy()
    assert np.array_equal(P, P.T)
    assert np.abs(P @ A - np.eye(m)).max() <= (1e-3 if slices == 1 else 1e-5)
    assert np.linalg.eigvalsh(P).min() > 0.0


def test_spd_inverse_precond_rejects_bad_arguments(S):
    from paper_1312_1549_gb300 import _native as N
    A = np.eye(200)
    A[150, 150] = -1.0
    with pytest.raises(N.OMMError) as e:
        S.spd_inverse(dev(A), slices=5)
    assert e.value.status == 2
    with pytest.raises(N.OMMError) as e:
        S.spd_inverse(dev(np.eye(10)), slices=10)
    assert e.value.status == 1


# ---------------------------------------------------------------- block-sparse operator products
@pytest.mark.parametrize("tile_n", [256, 128])
@pytest.mark.parametrize("M,N,K", [(256, 1024, 640), (130, 700, 333), (1024, 2048, 1024)])
def test_gemm_tc_blocksparse_equals_dense(S, M, N, K, tile_n):
    """Skipping the all-zero 64-wide K blocks of B changes no bit of the result."""
    rng = np.random.default_rng(M + 3 * N + K + tile_n)
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(N, K))
    # zero a random pattern of (tile_n rows x 64 columns) blocks, and a whole block row
    for r0 in range(0, N, tile_n):
        for k0 in range(0, K, 64):
            if rng.uniform() < 0.6:
                B[r0:r0 + tile_n, k0:k0 + 64] = 0.0
    B[:min(tile_n, N), :] = 0.0
    C0 = rng.normal(size=(M, N))
    Cd, Cs = dev(C0), dev(C0)
    S.gemm_tc(dev(A), dev(B), Cd, alpha=-4.0, beta=1.0, npass=3, tile_n=tile_n)
    S.gemm_tc(dev(A), dev(B), Cs, alpha=-4.0, beta=1.0, npass=3, tile_n=tile_n, block_sparse=True)
    assert torch.equal(Cd, Cs)
    ref = -4.0 * A @ B.T + C0
    assert np.all(np.abs(Cs.cpu().numpy() - ref) <= 2.0 ** -14 * 4.0 * np.abs(A) @ np.abs(B).T + 1e-12)
