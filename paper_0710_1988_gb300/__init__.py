"""Deflated BiCGStab for Wilson-Dirac systems on GB300: Python binding.

A thin ctypes layer over libwd.so (C ABI in include/wd.h).  It only
marshals arguments: every step of every solve runs in the library's CUDA
kernels.  Tensors are torch complex128 CUDA tensors (device pointers) or
complex128 numpy arrays (host pointers, staged by the library), laid out
as [nrhs][site][spin][colour] with site = x + Lx*(y + Ly*(z + Lz*t)).

Method: Abdel-Rehim, Morgan, Wilcox, "Deflated BiCGStab for linear
equations in QCD problems" (Lattice 2007): GMRES-DR(m,k) for the first
right-hand side (Sec. 1), then the left-right projection with U = gamma5 V
and BiCGStab for the others (Sec. 2).
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import WdError, WdStats, check, lib  # noqa: F401

__all__ = ["WilsonOperator", "Deflation", "WdError", "WdStats", "lib", "probe_fp64_peak",
           "tsgemm", "probe_bf16_mma_peak"]


def _ptr(a) -> int:
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(a.dtype) != "torch.complex128":
            raise TypeError(f"expected complex128, got {a.dtype}")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if a.dtype != np.complex128 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a C-contiguous complex128 array")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _numel(a) -> int:
    return a.numel() if hasattr(a, "numel") else a.size


def _stream(stream, *arrays) -> Optional[int]:
    if stream is not None:
        return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
    for a in arrays:
        if hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            return int(torch.cuda.current_stream(a.device).cuda_stream)
    return None


def probe_fp64_peak(iters: int = 1 << 15, reps: int = 3, stream=None):
    """Measured FP64 FMA throughput of the current device: (TFLOP/s, ms per
    launch) of the library's DFMA probe kernel, timed by CUDA events."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    check(lib().wd_probe_fp64_peak(int(iters), int(reps), ctypes.byref(tf), ctypes.byref(ms),
                                   _stream(stream)))
    return tf.value, ms.value


def tsgemm(V, kv: int, Y, ncol: int, OUT, IN=None, sign: float = 1.0,
           tensor_cores: bool = True, ldy: Optional[int] = None, stream=None):
    """OUT[c] = (IN[c] if IN is given else 0) + sign * sum_r V[r] Y[r, c] for
    complex128 CUDA tensors (V: kv vectors, Y: kv x ncol row-major, OUT and
    IN: ncol vectors), on the tensor cores or in FP64."""
    n = _numel(V) // kv
    check(lib().wd_tsgemm(_ptr(V), int(kv), _ptr(Y), int(ldy or ncol), int(ncol),
                          _ptr(IN) if IN is not None else None, _ptr(OUT),
                          1 if IN is not None else 0, float(sign), int(n),
                          1 if tensor_cores else 0, _stream(stream, V, OUT)))
    return OUT


def probe_bf16_mma_peak(iters: int = 8192, reps: int = 3, stream=None):
    """Measured BF16 tcgen05 MMA throughput of the current device: (TFLOP/s,
    ms per launch) of the library's tensor-core probe, timed by CUDA events."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    check(lib().wd_probe_bf16_mma_peak(int(iters), int(reps), ctypes.byref(tf),
                                       ctypes.byref(ms), _stream(stream)))
    return tf.value, ms.value


class WilsonOperator:
    """A = 1 - kappa*D + i*mu*gamma5 on a periodic lattice dims = (Lx, Ly, Lz, Lt)."""

    def __init__(self, dims: Sequence[int], links, kappa: float, mu: float = 0.0):
        self.dims = tuple(int(d) for d in dims)
        self.volume = int(np.prod(self.dims))
        self.n = 12 * self.volume
        if _numel(links) != 36 * self.volume:
            raise ValueError("links must hold V*4*3*3 complex numbers")
        self.kappa = float(kappa)
        self.mu = float(mu)
        lat = (ctypes.c_int * 4)(*self.dims)
        h = ctypes.c_void_p()
        check(lib().wd_create(lat, _ptr(links), self.kappa, self.mu, ctypes.byref(h)))
        self._h = h

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().wd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile(self, mask: int = 0x3F):
        """Start timing the kernel categories in mask (bit 0 FP64 dslash,
        1 streaming, 2 tall-skinny, 3 dense, 4 FP32/FP16 dslash, 5 the mixed
        solver's vector updates); mask = 0 stops.  Counters restart from zero."""
        check(lib().wd_profile_enable(self._h, int(mask)))

    def profile_read(self) -> dict:
        p = _lib.WdProfile()
        check(lib().wd_profile_read(self._h, ctypes.byref(p)))
        return p.as_dict()

    def set_params(self, kappa: float, mu: float = 0.0):
        self.kappa, self.mu = float(kappa), float(mu)
        check(lib().wd_set_params(self._h, self.kappa, self.mu))

    def set_operator(self, even_odd: bool):
        """Full operator (False) or the even-odd Schur complement on even-site
        half vectors (True); see wd_set_operator."""
        check(lib().wd_set_operator(self._h, 1 if even_odd else 0))
        self.even_odd = bool(even_odd)

    def eo_prepare(self, B, Bhat, stream=None):
        nrhs = _numel(B) // (12 * self.volume)
        check(lib().wd_eo_prepare(self._h, _ptr(B), _ptr(Bhat), nrhs, _stream(stream, B, Bhat)))
        return Bhat

    def eo_reconstruct(self, B, Xe, X, stream=None):
        nrhs = _numel(B) // (12 * self.volume)
        check(lib().wd_eo_reconstruct(self._h, _ptr(B), _ptr(Xe), _ptr(X), nrhs,
                                      _stream(stream, B, Xe, X)))
        return X

    @property
    def op_n(self) -> int:
        return self.n // 2 if getattr(self, "even_odd", False) else self.n

    def _nrhs(self, a) -> int:
        n = _numel(a)
        if n % self.op_n:
            raise ValueError("vector length is not a multiple of the operator's vector length")
        return n // self.op_n

    # -- operator
    def apply(self, x, out, dagger: bool = False, stream=None):
        """out = A x (or A^dagger x); x, out CUDA complex128, nrhs*12V elements."""
        nrhs = self._nrhs(x)
        if _numel(out) != _numel(x):
            raise ValueError("out must match x")
        check(lib().wd_apply(self._h, _ptr(x), _ptr(out), nrhs, 1 if dagger else 0,
                             _stream(stream, x, out)))
        return out

    # -- solvers
    def gmresdr(self, b, x, m: int, k: int, tol: float = 1e-10, max_mv: int = 100000,
                V_out=None, stream=None):
        """GMRES-DR(m,k): x (initial guess in, solution out).  Returns
        (status, stats, Hbar (k+1,k) numpy, theta (k,) numpy); V_out, if given,
        a CUDA tensor of k*12V elements, receives the deflation basis."""
        st = WdStats()
        hbar = np.zeros((k + 1, max(k, 1)), dtype=np.complex128)
        theta = np.zeros(max(k, 1), dtype=np.complex128)
        rc = lib().gmresdr_solve(
            self._h, _ptr(b), _ptr(x), int(m), int(k), float(tol), int(max_mv),
            _ptr(V_out) if V_out is not None else None,
            hbar.ctypes.data if k > 0 else None, theta.ctypes.data if k > 0 else None,
            ctypes.byref(st), _stream(stream, b, x))
        check(rc, allow=(_lib.WD_OK, _lib.WD_NOT_CONVERGED))
        return rc, st.as_dict(), hbar[:, :k], theta[:k]

    def set_contraction(self, tensor_cores: bool = True):
        """Wide V*Y products (GMRES-DR restart, projection updates) on the
        tensor cores (exact-split emulation, default) or in FP64 FMAs."""
        check(lib().wd_set_contraction(self._h, 1 if tensor_cores else 0))

    def set_eigen_estimates(self, fp32: bool = True):
        """GMRES-DR restart: harmonic Ritz pairs from FP32 estimates refined
        in FP64 (default) or from the FP64 QR iteration alone."""
        check(lib().wd_set_eigen_estimates(self._h, 1 if fp32 else 0))

    def gmresdr_history(self):
        """Least-squares residual / ||r0|| at the end of each cycle of the last
        gmresdr call on this operator (numpy float64 array)."""
        c = lib().gmresdr_history(self._h, None, 0)
        if c < 0:
            check(-c)
        out = np.zeros(max(c, 1), dtype=np.float64)
        lib().gmresdr_history(self._h, out.ctypes.data, c)
        return out[:c]

    def deflation(self, V, k: int, U=None, stream=None) -> "Deflation":
        return Deflation(self, V, k, U, stream)

    def dbicgstab(self, B, X, deflation: Optional["Deflation"] = None, tol: float = 1e-10,
                  max_iter: int = 100000, stream=None):
        """D-BiCGStab(k) for every right-hand side in B at once (deflation=None:
        plain BiCGStab).  X holds the initial guesses and receives the solutions.
        Returns (status, [stats per right-hand side])."""
        nrhs = self._nrhs(B)
        sts = (WdStats * nrhs)()
        rc = lib().dbicgstab_solve_deflated(
            self._h, deflation._d if deflation is not None else None, _ptr(B), _ptr(X),
            nrhs, float(tol), int(max_iter), sts, _stream(stream, B, X))
        check(rc, allow=(_lib.WD_OK, _lib.WD_NOT_CONVERGED, _lib.WD_BREAKDOWN))
        return rc, [s.as_dict() for s in sts]

    def dbicgstab_mixed(self, B, X, deflation: Optional["Deflation"] = None,
                        tol: float = 1e-10, max_iter: int = 100000, reliable_every: int = 50,
                        stream=None):
        """As dbicgstab, with the iteration in FP32 and FP64 reliable updates."""
        nrhs = self._nrhs(B)
        sts = (WdStats * nrhs)()
        rc = lib().dbicgstab_solve_mixed(
            self._h, deflation._d if deflation is not None else None, _ptr(B), _ptr(X),
            nrhs, float(tol), int(max_iter), int(reliable_every), sts, _stream(stream, B, X))
        check(rc, allow=(_lib.WD_OK, _lib.WD_NOT_CONVERGED, _lib.WD_BREAKDOWN))
        return rc, [s.as_dict() for s in sts]

    def adjoint_solve(self, G, LAM, deflation: Optional["Deflation"] = None,
                      tol: float = 1e-10, max_iter: int = 100000, mixed: bool = False,
                      reliable_every: int = 50, stream=None):
        """LAM = A^{-dagger} G (gamma5 A(-mu)^{-1} gamma5 G) for every column of G;
        mixed = True solves with the mixed-precision solver."""
        nrhs = self._nrhs(G)
        sts = (WdStats * nrhs)()
        d = deflation._d if deflation is not None else None
        if mixed:
            rc = lib().dbicgstab_solve_adjoint_mixed(
                self._h, d, _ptr(G), _ptr(LAM), nrhs, float(tol), int(max_iter),
                int(reliable_every), sts, _stream(stream, G, LAM))
        else:
            rc = lib().dbicgstab_solve_adjoint(
                self._h, d, _ptr(G), _ptr(LAM), nrhs, float(tol), int(max_iter), sts,
                _stream(stream, G, LAM))
        check(rc, allow=(_lib.WD_OK, _lib.WD_NOT_CONVERGED, _lib.WD_BREAKDOWN))
        return rc, [s.as_dict() for s in sts]

    def gradients(self, lam, x, force=None, want_dkappa: bool = True, stream=None):
        """Link force (into `force`, V*4*8 float64 CUDA tensor) and dL/dkappa for
        dL = Re(g^dagger dx), lam = A^{-dagger} g.  Returns dL/dkappa or None."""
        dk = ctypes.c_double(0.0)
        if force is not None and (str(force.dtype) != "torch.float64" or not force.is_contiguous()):
            raise TypeError("force must be a contiguous float64 tensor")
        check(lib().wd_gradients(self._h, _ptr(lam), _ptr(x),
                                 force.data_ptr() if force is not None else None,
                                 ctypes.byref(dk) if want_dkappa else None,
                                 _stream(stream, lam, x)))
        return dk.value if want_dkappa else None

    def multishift(self, B, X, mus: Sequence[float], tol: float = 1e-10, max_iter: int = 100000,
                   project: bool = True, mixed: bool = False, stream=None):
        """Sec. 4: A(mu_i) X[i] = B for the shifts in the given order, each
        projected over the earlier solutions.  X holds len(mus)*nrhs*12V
        complex128 ([shift][rhs][...]); full-lattice vectors also in even-odd
        mode, where each shift is solved through its Schur system.  Returns
        (status, stats [shift][rhs])."""
        # full-lattice vectors in both modes (even-odd: solved through A_hat)
        if _numel(B) % self.n:
            raise ValueError("B must hold whole full-lattice vectors")
        nrhs = _numel(B) // self.n
        ns = len(mus)
        if _numel(X) != ns * _numel(B):
            raise ValueError("X must hold len(mus) * nrhs vectors")
        sts = (WdStats * (ns * nrhs))()
        arr = (ctypes.c_double * ns)(*[float(m) for m in mus])
        rc = lib().tm_multishift_solve(self._h, _ptr(B), _ptr(X), nrhs, arr, ns, float(tol),
                                       int(max_iter), 1 if project else 0, 1 if mixed else 0,
                                       sts, _stream(stream, B, X))
        check(rc, allow=(_lib.WD_OK, _lib.WD_NOT_CONVERGED, _lib.WD_BREAKDOWN))
        out = [s.as_dict() for s in sts]
        return rc, [out[i * nrhs:(i + 1) * nrhs] for i in range(ns)]

    def autotune_f32(self, nrhs: int, stream=None):
        """Time every FP32 launch shape for nrhs right-hand sides; returns
        (R, threads per block, ms) of the fastest, now used by this handle."""
        R, T, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        check(lib().wd_autotune_f32(self._h, int(nrhs), ctypes.byref(R), ctypes.byref(T),
                                    ctypes.byref(ms), _stream(stream)))
        return R.value, T.value, ms.value

    def set_f32_shape(self, nrhs: int, R: int, threads: int):
        check(lib().wd_set_f32_shape(self._h, int(nrhs), int(R), int(threads)))

    def apply_f32(self, x, out, dagger: bool = False, stream=None):
        """out = A x with the FP32 kernel (FP64 vectors rounded on entry)."""
        nrhs = self._nrhs(x)
        check(lib().wd_apply_f32(self._h, _ptr(x), _ptr(out), nrhs, 1 if dagger else 0,
                                 _stream(stream, x, out)))
        return out

    def apply_f16(self, x, out, dagger: bool = False, stream=None):
        """out = A x with the FP16-storage kernel (FP64 vectors rounded to
        half with a per-site norm on entry, FP32 arithmetic)."""
        nrhs = self._nrhs(x)
        check(lib().wd_apply_f16(self._h, _ptr(x), _ptr(out), nrhs, 1 if dagger else 0,
                                 _stream(stream, x, out)))
        return out

    def autotune_f16(self, nrhs: int, stream=None):
        """As autotune_f32, for the FP16-storage kernel."""
        R, T, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        check(lib().wd_autotune_f16(self._h, int(nrhs), ctypes.byref(R), ctypes.byref(T),
                                    ctypes.byref(ms), _stream(stream)))
        return R.value, T.value, ms.value

    def set_f16_shape(self, nrhs: int, R: int, threads: int):
        check(lib().wd_set_f16_shape(self._h, int(nrhs), int(R), int(threads)))

    def set_mixed_restart(self, delta: float, max_inner: int = 300):
        """Mixed solver strategy: delta = 0 reliable updates (default); delta
        in (0, 1) restarted refinement, each low-precision pass reducing the
        residual by delta (at most max_inner iterations)."""
        check(lib().wd_set_mixed_restart(self._h, float(delta), int(max_inner)))

    def set_mixed_storage(self, bits: int):
        """Storage of the mixed solver's Krylov vectors: 32 (default) or 16."""
        check(lib().wd_set_mixed_storage(self._h, int(bits)))

    def dbicgstab_oneshot(self, B, X, V=None, k: int = 0, U=None, tol: float = 1e-10,
                          max_iter: int = 100000, stream=None):
        nrhs = self._nrhs(B)
        sts = (WdStats * nrhs)()
        rc = lib().dbicgstab_solve(
            self._h, _ptr(B), _ptr(X), nrhs, _ptr(V) if V is not None else None,
            _ptr(U) if U is not None else None, int(k), float(tol), int(max_iter), sts,
            _stream(stream, B, X))
        check(rc, allow=(_lib.WD_OK, _lib.WD_NOT_CONVERGED, _lib.WD_BREAKDOWN))
        return rc, [s.as_dict() for s in sts]


class Deflation:
    """The Sec. 2 deflation space: V, U (default gamma5 V), W = A V, LU(U^dagger A V)."""

    def __init__(self, op: WilsonOperator, V, k: int, U=None, stream=None):
        self.op = op
        self.k = int(k)
        d = ctypes.c_void_p()
        check(lib().wd_deflation_create(op._h, _ptr(V), _ptr(U) if U is not None else None,
                                        self.k, ctypes.byref(d), _stream(stream, V)))
        self._d = d

    def close(self):
        if getattr(self, "_d", None) is not None and self._d.value:
            lib().wd_deflation_destroy(self._d)
            self._d = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
