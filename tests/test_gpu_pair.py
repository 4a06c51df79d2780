"""GPU parity of the SM-pair (tcgen05 cta_group::2) form of the 3-term split contraction.

A cluster of two CTAs computes a 256-row output tile; each SM stages 128 rows of A and half of
B. The contraction is the same as the single-SM kernel's (the split form A_hi B_hi + A_hi B_lo +
A_lo B_hi over the same 64-wide K blocks in the same order), so the result is checked against the
float64 product within the split error bound 2^-14 |A||B| and against the single-SM kernel.
"""
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


SHAPES = [(256, 256, 64), (512, 384, 1000), (130, 257, 70), (1024, 1000, 333), (300, 700, 128), (1, 1, 1)]


@pytest.mark.parametrize("cp", [1, 2])
@pytest.mark.parametrize("tile_n", [128, 192, 256])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_pair_split_product(S, M, N, K, tile_n, cp):
    """cp = 2: two pairs per cluster sharing A by multicast (an odd number of column tiles leaves the
    second pair of the last cluster without columns)."""
    rng = np.random.default_rng(11 * M + N + K + tile_n)
    A = rng.normal(size=(M, K)); B = rng.normal(size=(N, K))
    C0 = rng.normal(size=(M, N))
    C = dev(C0)
    S.gemm_tc_pair(dev(A), dev(B), C, alpha=2.0, beta=-1.0, tile_n=tile_n, cluster_pairs=cp)
    got = C.cpu().numpy()
    ref = 2.0 * A @ B.T - C0
    scale = 2.0 * np.abs(A) @ np.abs(B).T
    assert np.all(np.abs(got - ref) <= 2.0 ** -14 * scale + 1e-12)
    # the single-SM kernel accumulates the same products over the same K blocks
    C1 = dev(C0)
    S.gemm_tc(dev(A), dev(B), C1, alpha=2.0, beta=-1.0, npass=3, tile_n=128)
    assert np.abs(got - C1.cpu().numpy()).max() <= 2.0 ** -20 * scale.max()


def bf16_round(x):
    """float64 -> nearest bf16 (8 significant bits, ties to even), rounded once."""
    m, e = np.frexp(x)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


@pytest.mark.parametrize("cp", [1, 2])
@pytest.mark.parametrize("tile_n", [128, 192, 256])
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (130, 257, 70), (1024, 1664, 1000), (1, 1, 1)])
def test_pair_single_pass_is_exact_bf16_product(S, M, N, K, tile_n, cp):
    """npass = 1 (the search direction's P G): the product of the bf16-rounded operands up to FP32
    accumulation (K 2^-23), and the single-SM kernel's value."""
    rng = np.random.default_rng(M + 5 * N + K + tile_n)
    A = rng.normal(size=(M, K)); B = rng.normal(size=(N, K))
    C = dev(np.zeros((M, N)))
    S.gemm_tc_pair(dev(A), dev(B), C, npass=1, tile_n=tile_n, cluster_pairs=cp)
    got = C.cpu().numpy()
    ref = bf16_round(A) @ bf16_round(B).T
    scale = np.abs(bf16_round(A)) @ np.abs(bf16_round(B)).T
    assert np.all(np.abs(got - ref) <= K * 2.0 ** -23 * scale + 1e-30)
    C1 = dev(np.zeros((M, N)))
    S.gemm_tc(dev(A), dev(B), C1, npass=1, tile_n=128)
    assert np.abs(got - C1.cpu().numpy()).max() <= 2.0 ** -20 * scale.max()


@pytest.mark.parametrize("cp", [1, 2])
@pytest.mark.parametrize("tile_n", [128, 256])
@pytest.mark.parametrize("M,N,K", [(256, 256, 64), (1024, 640, 256), (200, 300, 72), (512, 6656 // 4, 4096 // 4)])
def test_pair_mn_major_b(S, M, N, K, tile_n, cp):
    """B given K x N and read MN-major (the gradient product's layout)."""
    rng = np.random.default_rng(5 * M + N + K + tile_n)
    A = rng.normal(size=(M, K)); B = rng.normal(size=(K, N))
    C0 = rng.normal(size=(M, N))
    C = dev(C0)
    S.gemm_tc_pair(dev(A), dev(B), C, alpha=-4.0, beta=1.0, tile_n=tile_n, b_kn=True, cluster_pairs=cp)
    got = C.cpu().numpy()
    ref = -4.0 * A @ B + C0
    scale = 4.0 * np.abs(A) @ np.abs(B)
    assert np.all(np.abs(got - ref) <= 2.0 ** -14 * scale + 1e-12)
    C1 = dev(C0)
    S.gemm_tc_kn(dev(A), dev(B), C1, alpha=-4.0, beta=1.0, tile_n=128)
    assert np.abs(got - C1.cpu().numpy()).max() <= 2.0 ** -20 * scale.max()


@pytest.mark.parametrize("tile_n", [128, 192, 256])
@pytest.mark.parametrize("M,N,K", [(256, 1024, 640), (1024, 2048, 1024), (300, 700, 333)])
def test_pair_blocksparse_equals_dense(S, M, N, K, tile_n):
    """Skipping the all-zero 64-wide K blocks of B changes no bit of the SM-pair result."""
    rng = np.random.default_rng(M + 7 * N + K + tile_n)
    A = rng.normal(size=(M, K))
    B = rng.normal(size=(N, K))
    for r0 in range(0, N, 64):
        for k0 in range(0, K, 64):
            if rng.uniform() < 0.7:
                B[r0:r0 + 64, k0:k0 + 64] = 0.0
    B[:min(tile_n, N), :] = 0.0
    C0 = rng.normal(size=(M, N))
    Cd, Cs = dev(C0), dev(C0)
    S.gemm_tc_pair(dev(A), dev(B), Cd, alpha=-4.0, beta=1.0, tile_n=tile_n)
    S.gemm_tc_pair(dev(A), dev(B), Cs, alpha=-4.0, beta=1.0, tile_n=tile_n, block_sparse=True)
    assert torch.equal(Cd, Cs)
    ref = -4.0 * A @ B.T + C0
    assert np.all(np.abs(Cs.cpu().numpy() - ref) <= 2.0 ** -14 * 4.0 * np.abs(A) @ np.abs(B).T + 1e-12)


def test_pair_rejects_bad_arguments(S):
    from paper_1312_1549_gb300 import _native as N
    A = dev(np.ones((256, 64))); B = dev(np.ones((64, 64))); C = dev(np.zeros((256, 64)))
    for kw in ({"tile_n": 64}, {"tile_n": 192, "b_kn": True}, {"tile_n": 128, "b_kn": True, "block_sparse": True},
               {"npass": 2}, {"npass": 1, "b_kn": True}, {"cluster_pairs": 3},
               {"cluster_pairs": 2, "block_sparse": True}):
        with pytest.raises(N.OMMError) as e:
            S.gemm_tc_pair(A, B, C, **kw)
        assert e.value.status == 1
