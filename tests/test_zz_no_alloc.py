"""The allocation-free quartic-coefficient entry point agrees with the allocating one.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test. Callers that cannot allocate device
memory use omm_kernel_quartic_coefficients_noalloc, whose scratch is a static
device array (n <= 2048); it must give the same alpha_0..alpha_4 as
omm_kernel_quartic_coefficients on the same inputs, call after call.
"""
import ctypes as ct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, n)); SW = np.eye(n) + 0.01 * (X + X.T)
    Y = rng.normal(size=(n, n)); HW = 0.5 * (Y + Y.T)
    P = rng.normal(size=(n, 4 * n))
    P[:, 2 * n:3 * n] = 0.5 * (P[:, 2 * n:3 * n] + P[:, 2 * n:3 * n].T)
    P[:, 3 * n:] = 0.5 * (P[:, 3 * n:] + P[:, 3 * n:].T)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return dev(np.hstack([SW, HW])), dev(P), float(rng.normal())


def _noalloc(SWHW, Proj, E):
    from paper_1312_1549_gb300 import _native as N
    out = (ct.c_double * 5)()
    rc = N.lib().omm_kernel_quartic_coefficients_noalloc(SWHW.shape[0], ct.c_void_p(SWHW.data_ptr()),
                                                         ct.c_void_p(Proj.data_ptr()), E, out, None)
    return rc, np.array(list(out))


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300 import solver as S
    # n = 2048 fills the static array exactly; the smaller calls after it reuse what it left there
    for call, (n, seed) in enumerate([(2048, 4), (300, 1), (64, 2)]):
        SWHW, Proj, E = _inputs(n, seed)
        ref = S.quartic_coefficients(SWHW, Proj, E)
        rc, got = _noalloc(SWHW, Proj, E)
        assert rc == 0, f"call {call}"
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-10), (call, got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    SWHW, Proj, E = _inputs(8, 3)
    from paper_1312_1549_gb300 import _native as N
    for n in (2049, 4096):  # the first size past the limit, and one far past it
        out = (ct.c_double * 5)(*([7.0] * 5))
        rc = N.lib().omm_kernel_quartic_coefficients_noalloc(n, ct.c_void_p(SWHW.data_ptr()),
                                                             ct.c_void_p(Proj.data_ptr()), E, out, None)
        assert rc == 1
        assert list(out) == [7.0] * 5
        assert b"2048" in N.lib().omm_last_error()
