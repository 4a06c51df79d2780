"""Python binding of the OMM library: argument marshalling only.

Tensors are passed to the C ABI as raw pointers; every step of the solve runs
in the CUDA library. torch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as ct
import math

import numpy as np
import torch

from . import _native as N


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("expected a contiguous float64 tensor")
        return ct.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float64 array")
        return ct.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, torch.cuda.Stream):
        return ct.c_void_p(stream.cuda_stream)
    return ct.c_void_p(int(stream))


class OMMSolver:
    """One (H, S, T, eta, tau) problem: omm_create / omm_solve / omm_backward / omm_free.

    H, S, T: m x m float64 (torch CUDA/CPU tensors or numpy arrays).
    n: number of Wannier functions. precision: "fp64" or "mixed".
    cholesky=True: reduce to standard form by S = L L^T instead of preconditioning (the
    paper's Cholesky flavour, end of Sec. 2.4); T and tau are then ignored.
    debug_expire_wait=True (tests of the timeout status only): every mixed line search's first
    tensor-core GEMM lets a bounded wait expire, so solve() reports OMM_ERR_TIMEOUT.
    """

    def __init__(self, H, S, T, n, eta, tau, precision="fp64", stream=None, max_iter=0,
                 tol_grad=1e-9, e_tol=0.0, refine_ratio=0.0, precondition=True, check_every=0,
                 profile=False, native_certificate=False, cholesky=False, precond_slices=0,
                 debug_expire_wait=False):
        lib = N.lib()
        m = int(H.shape[0])
        self.m, self.n, self.eta, self.tau = m, int(n), float(eta), float(tau)
        self.stream = stream
        opts = N.OmmOpts(precision=N.PREC_MIXED if precision == "mixed" else N.PREC_FP64,
                         max_iter=int(max_iter), no_precondition=0 if precondition else 1,
                         check_every=int(check_every), tol_grad=float(tol_grad),
                         e_tol=float(e_tol), refine_ratio=float(refine_ratio),
                         profile=1 if profile else 0,
                         native_certificate=1 if native_certificate else 0,
                         cholesky=1 if cholesky else 0, precond_slices=int(precond_slices),
                         debug_expire_wait=1 if debug_expire_wait else 0)
        self._keep = (H, S, T)
        h = ct.c_void_p()
        tau_arg = math.inf if tau is None else float(tau)
        N.check(lib.omm_create(m, self.n, _ptr(H), _ptr(S), _ptr(T), self.eta, tau_arg,
                               ct.byref(opts), _stream_handle(stream), ct.byref(h)), "omm_create")
        self._keep = None
        self._h = h
        self.info = None

    def close(self):
        if getattr(self, "_h", None):
            N.lib().omm_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, C0, want_D=False, C_out=None, D_out=None, raise_on_error=True):
        """Minimise from C0 (n x m). Returns (C, E, D or None, info dict)."""
        like_cuda = isinstance(C0, torch.Tensor) and C0.is_cuda
        if C_out is None:
            if isinstance(C0, torch.Tensor):
                C_out = torch.empty_like(C0)
            else:
                C_out = np.empty_like(C0)
        if want_D and D_out is None:
            if like_cuda:
                D_out = torch.empty((self.m, self.m), dtype=torch.float64, device=C0.device)
            else:
                D_out = np.empty((self.m, self.m))
        E = ct.c_double(0.0)
        info = N.OmmInfo()
        rc = N.lib().omm_solve(self._h, _ptr(C0), _ptr(C_out), ct.byref(E),
                               _ptr(D_out) if want_D else None, ct.byref(info))
        self.info = info.as_dict()
        if raise_on_error:
            N.check(rc, "omm_solve")
        return C_out, E.value, (D_out if want_D else None), self.info

    def backward(self, dEdH=None, dEdS=None, device=None, want_H=True, want_S=True):
        """(dE/dH, dE/dS) = (D, -EDM) at the last converged solve (m x m)."""
        dev = device if device is not None else torch.device("cuda")
        if dEdH is None and want_H:
            dEdH = torch.empty((self.m, self.m), dtype=torch.float64, device=dev)
        if dEdS is None and want_S:
            dEdS = torch.empty((self.m, self.m), dtype=torch.float64, device=dev)
        N.check(N.lib().omm_backward(self._h, _ptr(dEdH), _ptr(dEdS)), "omm_backward")
        return dEdH, dEdS

    def update_H(self, H):
        N.check(N.lib().omm_update_H(self._h, _ptr(H)), "omm_update_H")


# ------------------------------------------------------------------ step-level entry points
def dgemm(transA, transB, A, B, C, alpha=1.0, beta=0.0, stream=None):
    M = C.shape[0]
    Ncols = C.shape[1]
    K = A.shape[0] if transA else A.shape[1]
    N.check(N.lib().omm_kernel_dgemm(int(transA), int(transB), M, Ncols, K, float(alpha), _ptr(A),
                                     A.stride(0), _ptr(B), B.stride(0), float(beta), _ptr(C),
                                     C.stride(0), _stream_handle(stream)), "omm_kernel_dgemm")
    return C


def spd_inverse(A, P=None, stream=None, sliced=False, slices=None):
    """P = A^-1 of an SPD matrix: float64 Cholesky, or (sliced=True) float64-class tensor-core products,
    or (slices=2..9) the preconditioner-grade sliced inverse with float32 diagonal blocks."""
    m = A.shape[0]
    if P is None:
        P = torch.empty_like(A)
    info = ct.c_int(0)
    if slices is not None:
        N.check(N.lib().omm_kernel_spd_inverse_precond(m, _ptr(A), _ptr(P), int(slices), ct.byref(info),
                                                       _stream_handle(stream)), "omm_kernel_spd_inverse_precond")
        return P
    fn = "omm_kernel_spd_inverse_sliced" if sliced else "omm_kernel_spd_inverse"
    N.check(getattr(N.lib(), fn)(m, _ptr(A), _ptr(P), ct.byref(info), _stream_handle(stream)), fn)
    return P


def line_minimum(alpha):
    a = (ct.c_double * 5)(*[float(v) for v in alpha])
    x = ct.c_double(0.0)
    rc = N.lib().omm_kernel_line_minimum(a, ct.byref(x))
    return x.value, rc


def quartic_coefficients(SWHW, Proj, E, stream=None):
    n = SWHW.shape[0]
    out = (ct.c_double * 5)()
    N.check(N.lib().omm_kernel_quartic_coefficients(n, _ptr(SWHW), _ptr(Proj), float(E), out,
                                                    _stream_handle(stream)),
            "omm_kernel_quartic_coefficients")
    return np.array(list(out))


def gemm_tc(A, B, C, alpha=1.0, beta=0.0, npass=3, stream=None, tile_n=None, block_sparse=False):
    """C = alpha A B^T + beta C on the BF16 tensor cores (split operands); tile_n 256 or 128;
    block_sparse skips the K blocks where B is zero."""
    M, K = A.shape
    Nn = B.shape[0]
    if block_sparse:
        N.check(N.lib().omm_kernel_gemm_tc_blocksparse(M, Nn, K, _ptr(A), _ptr(B), float(alpha), float(beta),
                                                       _ptr(C), int(npass), int(tile_n or 256),
                                                       _stream_handle(stream)), "omm_kernel_gemm_tc_blocksparse")
    elif tile_n is None:
        N.check(N.lib().omm_kernel_gemm_tc(M, Nn, K, _ptr(A), _ptr(B), float(alpha), float(beta), _ptr(C),
                                           int(npass), _stream_handle(stream)), "omm_kernel_gemm_tc")
    else:
        N.check(N.lib().omm_kernel_gemm_tc_tiled(M, Nn, K, _ptr(A), _ptr(B), float(alpha), float(beta), _ptr(C),
                                                 int(npass), int(tile_n), _stream_handle(stream)),
                "omm_kernel_gemm_tc_tiled")
    return C


def gemm_tc_kn(A, B, C, alpha=1.0, beta=0.0, tile_n=256, stream=None):
    """C = alpha A B + beta C on the BF16 tensor cores (split operands), B given K x N and read
    MN-major (the gradient product's operand layout)."""
    M, K = A.shape
    Nn = B.shape[1]
    N.check(N.lib().omm_kernel_gemm_tc_kn(M, Nn, K, _ptr(A), _ptr(B), float(alpha), float(beta), _ptr(C),
                                          int(tile_n), _stream_handle(stream)), "omm_kernel_gemm_tc_kn")
    return C


def gemm_tc_pair(A, B, C, alpha=1.0, beta=0.0, tile_n=256, b_kn=False, block_sparse=False, npass=3, cluster_pairs=1,
                 stream=None):
    """The tensor-core contraction on pairs of SMs (256-row tiles, tcgen05 cta_group::2): C = alpha A B^T
    + beta C (B N x K), or with b_kn C = alpha A B + beta C (B K x N, read MN-major); npass 3 (split
    form) or 1 (single bf16 pass); tile_n 128, 192 (K-major B only) or 256; block_sparse skips the K
    blocks where B is zero; cluster_pairs 2 runs two pairs per cluster that share A (dense B)."""
    M, K = A.shape
    Nn = B.shape[1] if b_kn else B.shape[0]
    N.check(N.lib().omm_kernel_gemm_tc_pair(M, Nn, K, _ptr(A), _ptr(B), float(alpha), float(beta), _ptr(C),
                                            int(npass), int(tile_n), int(bool(b_kn)), int(bool(block_sparse)),
                                            int(cluster_pairs), _stream_handle(stream)), "omm_kernel_gemm_tc_pair")
    return C


def gemm_emu(A, B, C, alpha=1.0, beta=0.0, slices=10, stream=None):
    """C = alpha A B^T + beta C, float64-class, on the BF16 tensor cores (fixed-point slices)."""
    M, K = A.shape
    Nn = B.shape[0]
    N.check(N.lib().omm_kernel_gemm_emu(M, Nn, K, _ptr(A), _ptr(B), float(alpha), float(beta), _ptr(C),
                                        int(slices), _stream_handle(stream)), "omm_kernel_gemm_emu")
    return C


def launch_count():
    """Kernels launched by the library in this process."""
    return int(N.lib().omm_launch_count())


class OMMBatch:
    """Independent problems solved together: omm_create_batched / omm_solve_batched.

    problems: list of (H, S, T, n, eta, tau). With precision="mixed" every phase of a
    line search is one launch over the batch (grouped tensor-core GEMMs, batched vector
    kernels) replayed from a CUDA graph; "fp64" solves the instances one by one.
    """

    def __init__(self, problems, precision="mixed", stream=None, max_iter=0, tol_grad=1e-9,
                 refine_ratio=0.0, precondition=True, check_every=0, profile=False,
                 native_certificate=False, cholesky=False, precond_slices=0):
        lib = N.lib()
        cnt = len(problems)
        self.count = cnt
        self.shapes = [(int(p[0].shape[0]), int(p[3])) for p in problems]
        opts = N.OmmOpts(precision=N.PREC_MIXED if precision == "mixed" else N.PREC_FP64,
                         max_iter=int(max_iter), no_precondition=0 if precondition else 1,
                         check_every=int(check_every), tol_grad=float(tol_grad), e_tol=0.0,
                         refine_ratio=float(refine_ratio), profile=1 if profile else 0,
                         native_certificate=1 if native_certificate else 0,
                         cholesky=1 if cholesky else 0, precond_slices=int(precond_slices))
        P = ct.c_void_p * cnt
        ms = (ct.c_int * cnt)(*[s[0] for s in self.shapes])
        ns = (ct.c_int * cnt)(*[s[1] for s in self.shapes])
        Hs = P(*[_ptr(p[0]) for p in problems])
        Ss = P(*[_ptr(p[1]) for p in problems])
        Ts = P(*[_ptr(p[2]) for p in problems])
        etas = (ct.c_double * cnt)(*[float(p[4]) for p in problems])
        taus = (ct.c_double * cnt)(*[float(p[5]) for p in problems])
        self.etas = [float(p[4]) for p in problems]
        h = ct.c_void_p()
        N.check(lib.omm_create_batched(cnt, ms, ns, Hs, Ss, Ts, etas, taus, ct.byref(opts),
                                       _stream_handle(stream), ct.byref(h)), "omm_create_batched")
        self._h = h
        self.infos = None

    def close(self):
        if getattr(self, "_h", None):
            N.lib().omm_free_batched(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, C0s, C_outs=None, raise_on_error=True):
        """Solve all instances from C0s (list of n_i x m_i). Returns (C list, E array, infos)."""
        cnt = self.count
        if C_outs is None:
            C_outs = [torch.empty_like(c) if isinstance(c, torch.Tensor) else np.empty_like(c) for c in C0s]
        P = ct.c_void_p * cnt
        E = (ct.c_double * cnt)()
        infos = (N.OmmInfo * cnt)()
        rc = N.lib().omm_solve_batched(self._h, P(*[_ptr(c) for c in C0s]), P(*[_ptr(c) for c in C_outs]),
                                       E, infos)
        self.infos = [infos[i].as_dict() for i in range(cnt)]
        if raise_on_error:
            N.check(rc, "omm_solve_batched")
        return C_outs, np.array(list(E)), self.infos

    def backward(self, i, device=None):
        """(dE/dH, dE/dS) of instance i after a converged batched solve."""
        m = self.shapes[i][0]
        dev = device if device is not None else torch.device("cuda")
        ctx = N.lib().omm_batch_instance(self._h, int(i))
        dH = torch.empty((m, m), dtype=torch.float64, device=dev)
        dS = torch.empty((m, m), dtype=torch.float64, device=dev)
        N.check(N.lib().omm_backward(ctx, _ptr(dH), _ptr(dS)), "omm_backward")
        return dH, dS


# ------------------------------------------------------------------ Hermitian (complex) problems
def _zptr(x):
    """Pointer to a contiguous complex128 tensor or array (interleaved real, imaginary)."""
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.complex128 or not x.is_contiguous():
            raise ValueError("expected a contiguous complex128 tensor")
        return ct.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if x.dtype != np.complex128 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous complex128 array")
        return ct.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _zlike(x, shape):
    if isinstance(x, torch.Tensor):
        return torch.empty(shape, dtype=torch.complex128, device=x.device)
    return np.empty(shape, dtype=np.complex128)


def _opts(precision, max_iter, tol_grad, e_tol, refine_ratio, precondition, check_every, profile,
          native_certificate, cholesky):
    return N.OmmOpts(precision=N.PREC_MIXED if precision == "mixed" else N.PREC_FP64,
                     max_iter=int(max_iter), no_precondition=0 if precondition else 1,
                     check_every=int(check_every), tol_grad=float(tol_grad), e_tol=float(e_tol),
                     refine_ratio=float(refine_ratio), profile=1 if profile else 0,
                     native_certificate=1 if native_certificate else 0, cholesky=1 if cholesky else 0)


class OMMHermitian:
    """One Hermitian (complex) problem: omm_create_hermitian / omm_solve_hermitian / ...

    H, S, T: m x m complex128 (torch or numpy); C0: n x m complex128. E is the complex problem's
    band energy; D and dE/dS = -EDM are m x m complex128.
    """

    def __init__(self, H, S, T, n, eta, tau, precision="fp64", stream=None, max_iter=0,
                 tol_grad=1e-9, e_tol=0.0, refine_ratio=0.0, precondition=True, check_every=0,
                 profile=False, native_certificate=False, cholesky=False):
        lib = N.lib()
        self.m, self.n, self.eta, self.tau = int(H.shape[0]), int(n), float(eta), float(tau)
        opts = _opts(precision, max_iter, tol_grad, e_tol, refine_ratio, precondition, check_every,
                     profile, native_certificate, cholesky)
        h = ct.c_void_p()
        N.check(lib.omm_create_hermitian(self.m, self.n, _zptr(H), _zptr(S), _zptr(T), self.eta,
                                         math.inf if tau is None else float(tau), ct.byref(opts),
                                         _stream_handle(stream), ct.byref(h)), "omm_create_hermitian")
        self._h = h
        self.info = None

    def close(self):
        if getattr(self, "_h", None):
            N.lib().omm_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, C0, want_D=False, C_out=None, D_out=None, raise_on_error=True):
        """Minimise from C0 (n x m complex). Returns (C, E, D or None, info dict)."""
        if C_out is None:
            C_out = _zlike(C0, (self.n, self.m))
        if want_D and D_out is None:
            D_out = _zlike(C0, (self.m, self.m))
        E = ct.c_double(0.0)
        info = N.OmmInfo()
        rc = N.lib().omm_solve_hermitian(self._h, _zptr(C0), _zptr(C_out), ct.byref(E),
                                         _zptr(D_out) if want_D else None, ct.byref(info))
        self.info = info.as_dict()
        if raise_on_error:
            N.check(rc, "omm_solve_hermitian")
        return C_out, E.value, (D_out if want_D else None), self.info

    def backward(self, device=None):
        """(dE/dH, dE/dS) = (D, -EDM) at the last converged solve (m x m complex)."""
        dev = device if device is not None else torch.device("cuda")
        dH = torch.empty((self.m, self.m), dtype=torch.complex128, device=dev)
        dS = torch.empty((self.m, self.m), dtype=torch.complex128, device=dev)
        N.check(N.lib().omm_backward_hermitian(self._h, _zptr(dH), _zptr(dS)), "omm_backward_hermitian")
        return dH, dS

    def update_H(self, H):
        N.check(N.lib().omm_update_H_hermitian(self._h, _zptr(H)), "omm_update_H_hermitian")


class OMMHermitianBatch:
    """Hermitian problems solved together (the points of a k grid): problems are
    (H, S, T, n, eta, tau) with complex128 matrices."""

    def __init__(self, problems, precision="mixed", stream=None, max_iter=0, tol_grad=1e-9,
                 refine_ratio=0.0, precondition=True, check_every=0, profile=False,
                 native_certificate=False, cholesky=False):
        cnt = len(problems)
        self.count = cnt
        self.shapes = [(int(p[0].shape[0]), int(p[3])) for p in problems]
        opts = _opts(precision, max_iter, tol_grad, 0.0, refine_ratio, precondition, check_every, profile,
                     native_certificate, cholesky)
        P = ct.c_void_p * cnt
        ms = (ct.c_int * cnt)(*[s[0] for s in self.shapes])
        ns = (ct.c_int * cnt)(*[s[1] for s in self.shapes])
        Ts = None if all(p[2] is None for p in problems) else P(*[_zptr(p[2]) for p in problems])
        etas = (ct.c_double * cnt)(*[float(p[4]) for p in problems])
        taus = (ct.c_double * cnt)(*[float(p[5]) for p in problems])
        h = ct.c_void_p()
        N.check(N.lib().omm_create_hermitian_batched(cnt, ms, ns, P(*[_zptr(p[0]) for p in problems]),
                                                     P(*[_zptr(p[1]) for p in problems]), Ts, etas, taus,
                                                     ct.byref(opts), _stream_handle(stream), ct.byref(h)),
                "omm_create_hermitian_batched")
        self._h = h
        self.infos = None

    def close(self):
        if getattr(self, "_h", None):
            N.lib().omm_free_batched(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, C0s, C_outs=None, raise_on_error=True):
        """Solve all instances from C0s (list of n_i x m_i complex). Returns (C list, E array, infos)."""
        cnt = self.count
        if C_outs is None:
            C_outs = [_zlike(c, c.shape) for c in C0s]
        P = ct.c_void_p * cnt
        E = (ct.c_double * cnt)()
        infos = (N.OmmInfo * cnt)()
        rc = N.lib().omm_solve_hermitian_batched(self._h, P(*[_zptr(c) for c in C0s]),
                                                 P(*[_zptr(c) for c in C_outs]), E, infos)
        self.infos = [infos[i].as_dict() for i in range(cnt)]
        if raise_on_error:
            N.check(rc, "omm_solve_hermitian_batched")
        return C_outs, np.array(list(E)), self.infos

    def backward(self, i, device=None):
        """(dE/dH, dE/dS) of instance i after a converged batched solve (m x m complex)."""
        m = self.shapes[i][0]
        dev = device if device is not None else torch.device("cuda")
        ctx = N.lib().omm_batch_instance(self._h, int(i))
        dH = torch.empty((m, m), dtype=torch.complex128, device=dev)
        dS = torch.empty((m, m), dtype=torch.complex128, device=dev)
        N.check(N.lib().omm_backward_hermitian(ctx, _zptr(dH), _zptr(dS)), "omm_backward_hermitian")
        return dH, dS
