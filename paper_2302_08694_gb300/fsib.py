"""Thin Python binding of libfsib.so (the C ABI declared in include/fsib.h).

Argument marshalling only: every step of the FSIB path runs in the library's
CUDA kernels. Arrays may be torch tensors (CUDA or CPU) or NumPy arrays; CPU
arrays go through the library's host staging path. The library must be built
(paper_2302_08694_gb300.build); there is no CPU fallback.

Low-level functions carry the C names (fsib_create, fsib_spread, ...); the
Problem class wraps one handle.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FSIB_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT",
          -6: "EUNSUPPORTED", -7: "ESTATE"}
FSIB_FP64, FSIB_MIXED = 0, 1

EXPORTS = ["fsib_create", "fsib_destroy", "fsib_set_stream", "fsib_set_option", "fsib_get_info",
           "fsib_set_force_curve", "fsib_set_force_mesh", "fsib_force", "fsib_spread", "fsib_interp",
           "fsib_fluid_step", "fsib_step", "fsib_invariants", "fsib_last_error", "fsib_version",
           "fsib_profile_enable", "fsib_profile_reset", "fsib_profile_count", "fsib_profile_entry",
           "fsib_measure_peak", "fsib_spread_static", "fsib_static_last_error", "fsib_autotune",
           "fsib_batch_create", "fsib_batch_member", "fsib_batch_set_stream", "fsib_batch_autotune",
           "fsib_batch_step", "fsib_batch_info", "fsib_batch_last_error", "fsib_batch_destroy",
           "fsib_interp_grad", "fsib_step_adjoint", "fsib_set_force_target", "fsib_set_body_force",
           "fsib_band_flux", "fsib_set_force_tension", "fsib_pressure", "fsib_batch_set_option"]

_lib = None


class FsibError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fsib error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def load(path: str | None = None):
    """Load libfsib.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_2302_08694_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, ip, dp, d_, i_ = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), \
        ctypes.c_double, ctypes.c_int
    sig = {
        "fsib_create": ([ctypes.POINTER(vp), i_, i_, i_, d_, d_, d_, d_], i_),
        "fsib_destroy": ([vp], i_),
        "fsib_set_stream": ([vp, vp], i_),
        "fsib_set_option": ([vp, ctypes.c_char_p, d_], i_),
        "fsib_get_info": ([vp, ctypes.c_char_p, dp], i_),
        "fsib_set_force_curve": ([vp, d_], i_),
        "fsib_set_force_mesh": ([vp, vp, i_, vp, d_], i_),
        "fsib_force": ([vp, vp, vp], i_),
        "fsib_spread": ([vp, vp, vp, vp, vp], i_),
        "fsib_interp": ([vp, vp, vp, vp], i_),
        "fsib_fluid_step": ([vp, vp, vp, vp], i_),
        "fsib_step": ([vp, vp, vp, vp, i_], i_),
        "fsib_invariants": ([vp, vp, vp, dp], i_),
        "fsib_last_error": ([vp], ctypes.c_char_p),
        "fsib_version": ([], ctypes.c_char_p),
        "fsib_profile_enable": ([vp, i_], i_),
        "fsib_profile_reset": ([vp], i_),
        "fsib_profile_count": ([vp], i_),
        "fsib_profile_entry": ([vp, i_, ctypes.c_char_p, i_, dp, ip, dp, dp], i_),
        "fsib_measure_peak": ([i_, dp], i_),
        "fsib_spread_static": ([i_, i_, i_, d_, i_, vp, vp, vp, vp, vp], i_),
        "fsib_static_last_error": ([], ctypes.c_char_p),
        "fsib_autotune": ([vp, vp, vp, vp], i_),
        "fsib_batch_create": ([ctypes.POINTER(vp), i_, vp, vp, vp, vp, vp, vp, vp, i_], i_),
        "fsib_batch_member": ([vp, i_, ctypes.POINTER(vp)], i_),
        "fsib_batch_set_stream": ([vp, vp], i_),
        "fsib_batch_autotune": ([vp, vp, vp, vp], i_),
        "fsib_batch_step": ([vp, vp, vp, vp, i_], i_),
        "fsib_batch_info": ([vp, ctypes.c_char_p, dp], i_),
        "fsib_batch_last_error": ([vp], ctypes.c_char_p),
        "fsib_batch_destroy": ([vp], i_),
        "fsib_interp_grad": ([vp, vp, vp, vp], i_),
        "fsib_step_adjoint": ([vp, vp, i_, i_, vp, vp, vp], i_),
        "fsib_set_force_target": ([vp, vp, d_, d_], i_),
        "fsib_set_body_force": ([vp, dp], i_),
        "fsib_band_flux": ([vp, vp, i_, i_, d_, d_, dp], i_),
        "fsib_set_force_tension": ([vp, vp, i_, d_], i_),
        "fsib_pressure": ([vp, vp, vp, vp], i_),
        "fsib_batch_set_option": ([vp, ctypes.c_char_p, d_], i_),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(a):
    """Raw address of a torch tensor or NumPy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check(lib, h, rc):
    if rc != FSIB_OK:
        msg = lib.fsib_last_error(h)
        raise FsibError(rc, msg.decode() if msg else "")


class Problem:
    """One FSIB problem: periodic unit box, N modes per axis, M boundary points."""

    def __init__(self, N, d, M, mu, rho, dt, tol, precision="fp64", sigma=None, width=None, bin=None,
                 graph=True):
        self.lib = load()
        self.N, self.d, self.M = int(N), int(d), int(M)
        self.mu, self.rho, self.dt, self.tol = float(mu), float(rho), float(dt), float(tol)
        h = ctypes.c_void_p()
        rc = self.lib.fsib_create(ctypes.byref(h), self.N, self.d, self.M, self.mu, self.rho, self.dt,
                                  self.tol)
        if rc != FSIB_OK:
            raise FsibError(rc, self.lib.fsib_last_error(None).decode())
        self.h = h
        if precision not in ("fp64", "mixed"):
            raise ValueError("precision must be 'fp64' or 'mixed'")
        self.precision = precision
        if sigma is not None:
            self.set_option("sigma", sigma)
        if width is not None:
            self.set_option("width", width)
        if bin is not None:
            self.set_option("bin", bin)
        if precision == "mixed":
            self.set_option("precision", 1)
        if not graph:
            self.set_option("graph", 0)

    # -- helpers -------------------------------------------------------------------------------
    @property
    def spec_shape(self):
        return (self.d,) + (self.N,) * (self.d - 1) + (self.N // 2,)

    @property
    def spec_dtype(self):
        import torch
        return torch.complex128 if self.precision == "fp64" else torch.complex64

    def _stream(self):
        import torch
        if torch.cuda.is_available():
            self.lib.fsib_set_stream(self.h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    def _call(self, name, *args):
        self._stream()
        _check(self.lib, self.h, getattr(self.lib, name)(self.h, *args))

    def close(self):
        if getattr(self, "h", None):
            self.lib.fsib_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI wrappers ------------------------------------------------------------------------
    def set_option(self, key, value):
        self._call("fsib_set_option", key.encode(), float(value))

    def info(self, key):
        v = ctypes.c_double()
        self._call("fsib_get_info", key.encode(), ctypes.byref(v))
        return v.value

    def set_force_curve(self, K):
        self._call("fsib_set_force_curve", float(K))

    def set_force_mesh(self, tri, Xref, sigma):
        tri = np.ascontiguousarray(tri, dtype=np.int32) if isinstance(tri, np.ndarray) else tri
        self._call("fsib_set_force_mesh", _ptr(tri), int(tri.shape[0]), _ptr(Xref), float(sigma))

    def set_force_tension(self, tri, gamma):
        """Surface tension gamma S on the triangulated surface tri ([ntri][3] int32, ccw from outside)."""
        tri = np.ascontiguousarray(tri, dtype=np.int32) if isinstance(tri, np.ndarray) else tri
        self._call("fsib_set_force_tension", _ptr(tri), int(tri.shape[0]), float(gamma))

    def set_force_target(self, Xtarget, K, omega):
        """Target-point springs c = omega K (X~ - X); Xtarget [d][M] float64 (host or device)."""
        if isinstance(Xtarget, np.ndarray):
            Xtarget = np.ascontiguousarray(Xtarget, dtype=np.float64)
        self._call("fsib_set_force_target", _ptr(Xtarget), float(K), float(omega))

    def set_body_force(self, f):
        """Uniform body force density (d values), added to f-hat(0) in the Navier-Stokes update."""
        vals = [float(v) for v in f] + [0.0, 0.0, 0.0]
        arr = (ctypes.c_double * 3)(*vals[:3])
        self._call("fsib_set_body_force", arr)

    def pressure(self, fhat, uhat=None, out=None):
        """p-hat = -i k.(f-hat - rho s-hat(u-hat))/|k|^2 (one half-spectrum component)."""
        if out is None:
            import torch
            dev = fhat.device if hasattr(fhat, "device") else "cpu"
            out = torch.zeros(self.spec_shape[1:], dtype=self.spec_dtype, device=dev)
        self._call("fsib_pressure", _ptr(fhat), _ptr(uhat), _ptr(out))
        return out

    def pressure_at(self, phat, Y):
        """Pressure at the points Y ([d][n] float64) by the type-2 transform of phat."""
        n = Y.shape[1]
        probe = Problem(self.N, self.d, n, self.mu, self.rho if self.rho > 0 else 0.0, self.dt, self.tol,
                        precision=self.precision)
        spec = probe.new_spec(device=phat.device)
        spec[0] = phat
        U = probe.interp(spec, Y)
        probe.close()
        return U[0]

    def band_flux(self, uhat, comp, axis, y0, y1):
        """Flux of u_comp averaged over the other axes through y0 <= x_axis <= y1."""
        v = ctypes.c_double()
        self._call("fsib_band_flux", _ptr(uhat), int(comp), int(axis), float(y0), float(y1), ctypes.byref(v))
        return v.value

    def new_spec(self, device="cuda"):
        import torch
        return torch.zeros(self.spec_shape, dtype=self.spec_dtype, device=device)

    def force(self, X, out=None):
        import torch
        if out is None:
            out = torch.empty_like(X) if hasattr(X, "data_ptr") else np.empty_like(X)
        self._call("fsib_force", _ptr(X), _ptr(out))
        return out

    def spread(self, X, F, omega=None, out=None):
        if out is None:
            out = self.new_spec(device=X.device if hasattr(X, "device") else "cpu")
        self._call("fsib_spread", _ptr(X), _ptr(F), _ptr(omega), _ptr(out))
        return out

    def interp(self, uhat, X, out=None):
        import torch
        if out is None:
            out = torch.empty_like(X) if hasattr(X, "data_ptr") else np.empty_like(X)
        self._call("fsib_interp", _ptr(uhat), _ptr(X), _ptr(out))
        return out

    def fluid_step(self, fhat, uhat, uhat_half=None):
        self._call("fsib_fluid_step", _ptr(fhat), _ptr(uhat), _ptr(uhat_half))
        return uhat

    def step(self, X, uhat=None, U=None, nsteps=1):
        self._call("fsib_step", _ptr(X), _ptr(uhat), _ptr(U), int(nsteps))
        return X

    def invariants(self, X, uhat=None):
        out = (ctypes.c_double * 6)()
        self._call("fsib_invariants", _ptr(X), _ptr(uhat), out)
        keys = ("volume", "Ep", "Ek", "u0", "max_div", "dissipation")
        return dict(zip(keys, list(out)))


    def interp_grad(self, uhat, X, out=None):
        """G[b, a, j] = d u_a / d x_b at X_j."""
        import torch
        if out is None:
            shape = (self.d, self.d, self.M)
            out = torch.empty(shape, dtype=torch.float64, device=X.device) if hasattr(X, "device") \
                else np.empty(shape)
        self._call("fsib_interp_grad", _ptr(uhat), _ptr(X), _ptr(out))
        return out

    def step_adjoint(self, X0, K, ckpt_every, dLdXK, dLdX0=None):
        """(dL/dX0, dL/dsigma) of K quasi-static Stokes steps from X0."""
        import torch
        if dLdX0 is None:
            dLdX0 = torch.empty_like(X0) if hasattr(X0, "data_ptr") else np.empty_like(X0)
        gs = torch.zeros(1, dtype=torch.float64, device=X0.device) if hasattr(X0, "device") else np.zeros(1)
        self._call("fsib_step_adjoint", _ptr(X0), int(K), int(ckpt_every), _ptr(dLdXK), _ptr(dLdX0), _ptr(gs))
        return dLdX0, gs

    def autotune(self, X, uhat=None, U=None):
        """fsib_autotune: pick launch shapes by timing steps on copies of (X, uhat, U)."""
        self._call("fsib_autotune", _ptr(X), _ptr(uhat), _ptr(U))
        return {k: int(self.info(k)) for k in ("fft_tile", "fft_rows", "spread_slice")}

    # -- profiling ------------------------------------------------------------------------------
    def profile(self, on=True):
        self._call("fsib_profile_enable", 1 if on else 0)

    def profile_reset(self):
        self._call("fsib_profile_reset")

    def profile_entries(self):
        """List of dicts: name, total_ms, launches, bytes (per launch), flops (per launch)."""
        n = self.lib.fsib_profile_count(self.h)
        out = []
        for i in range(n):
            name = ctypes.create_string_buffer(64)
            t, b, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            k = ctypes.c_int()
            _check(self.lib, self.h, self.lib.fsib_profile_entry(self.h, i, name, 64, ctypes.byref(t),
                                                                 ctypes.byref(k), ctypes.byref(b),
                                                                 ctypes.byref(f)))
            out.append({"name": name.value.decode(), "total_ms": t.value, "launches": k.value,
                        "bytes": b.value, "flops": f.value})
        return out


def measure_peak(kind):
    """Measured FMA throughput of the current device in GFLOP/s: kind 0 = FP64, 1 = FP32."""
    lib = load()
    v = ctypes.c_double()
    rc = lib.fsib_measure_peak(int(kind), ctypes.byref(v))
    if rc != FSIB_OK:
        raise FsibError(rc, "peak measurement failed")
    return v.value


class Member(Problem):
    """A problem owned by a Batch (not destroyed on its own)."""

    def __init__(self, lib, h, N, d, M, mu, rho, dt, tol, precision):
        self.lib, self.h = lib, h
        self.N, self.d, self.M = N, d, M
        self.mu, self.rho, self.dt, self.tol = mu, rho, dt, tol
        self.precision = precision

    def close(self):
        self.h = None


class Batch:
    """fsib_batch_*: independent problems advanced by one CUDA graph launch per step."""

    def __init__(self, N, d, M, mu, rho, dt, tol, precision="mixed"):
        self.lib = load()
        n = len(N)
        I = ctypes.c_int * n
        D = ctypes.c_double * n
        self._args = (I(*N), I(*d), I(*M), D(*mu), D(*rho), D(*dt), D(*tol))
        b = ctypes.c_void_p()
        rc = self.lib.fsib_batch_create(ctypes.byref(b), n, *[ctypes.cast(a, ctypes.c_void_p) for a in self._args],
                                        FSIB_MIXED if precision == "mixed" else FSIB_FP64)
        if rc != FSIB_OK:
            raise FsibError(rc, self.lib.fsib_batch_last_error(None).decode())
        self.b = b
        self.members = []
        for i in range(n):
            h = ctypes.c_void_p()
            _check(self.lib, None, self.lib.fsib_batch_member(b, i, ctypes.byref(h)))
            self.members.append(Member(self.lib, h, N[i], d[i], M[i], mu[i], rho[i], dt[i], tol[i], precision))

    def _ptrs(self, arrs):
        if arrs is None:
            return None
        P = ctypes.c_void_p * len(arrs)
        return P(*[_ptr(a) for a in arrs])

    def _bcall(self, name, *args):
        import torch
        if torch.cuda.is_available():
            self.lib.fsib_batch_set_stream(self.b, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        rc = getattr(self.lib, name)(self.b, *args)
        if rc != FSIB_OK:
            raise FsibError(rc, self.lib.fsib_batch_last_error(self.b).decode())

    def step(self, X, uhat, U, nsteps=1):
        self._bcall("fsib_batch_step", self._ptrs(X), self._ptrs(uhat), self._ptrs(U), int(nsteps))

    def autotune(self, X, uhat, U):
        self._bcall("fsib_batch_autotune", self._ptrs(X), self._ptrs(uhat), self._ptrs(U))

    def set_option(self, key, value):
        self._bcall("fsib_batch_set_option", key.encode(), float(value))

    def info(self, key):
        v = ctypes.c_double()
        self._bcall("fsib_batch_info", key.encode(), ctypes.byref(v))
        return v.value

    def close(self):
        if getattr(self, "b", None):
            for m in self.members:
                m.close()
            self.lib.fsib_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rollout_function():
    import torch

    class StokesRollout(torch.autograd.Function):
        """X^K = (K quasi-static Stokes steps)(X^0; sigma) with a hand-written adjoint.

        forward: sets the mesh (or curve) force with stiffness sigma and runs fsib_step K
        times; backward: fsib_step_adjoint with checkpoints every ckpt_every steps."""

        @staticmethod
        def forward(ctx, X0, sigma, pb, K, ckpt_every, tri=None, Xref=None):
            s = float(sigma.detach().cpu().item())
            if tri is not None:
                pb.set_force_mesh(tri, Xref, s)
            else:
                pb.set_force_curve(s)
            X = X0.detach().clone().contiguous()
            pb.step(X, nsteps=int(K))
            ctx.pb, ctx.K, ctx.ck = pb, int(K), int(ckpt_every)
            ctx.sig_dev, ctx.sig_dtype = sigma.device, sigma.dtype
            ctx.save_for_backward(X0.detach().clone())
            return X

        @staticmethod
        def backward(ctx, gX):
            (X0,) = ctx.saved_tensors
            g0, gs = ctx.pb.step_adjoint(X0, ctx.K, ctx.ck, gX.detach().contiguous())
            return g0, gs.reshape(()).to(device=ctx.sig_dev, dtype=ctx.sig_dtype), None, None, None, None, None

    return StokesRollout


def stokes_rollout(X0, sigma, pb, K, ckpt_every, tri=None, Xref=None):
    """Differentiable K-step quasi-static Stokes rollout (torch.autograd.Function)."""
    return _rollout_function().apply(X0, sigma, pb, K, ckpt_every, tri, Xref)


def spread_static(N, d, M, tol, precision, X, F, omega, fhat, stream=None):
    """fsib_spread_static: the type-1 spread with no device allocation (device arrays only)."""
    lib = load()
    rc = lib.fsib_spread_static(int(N), int(d), int(M), float(tol), FSIB_MIXED if precision == "mixed" else FSIB_FP64,
                                _ptr(X), _ptr(F), _ptr(omega), _ptr(fhat), stream)
    if rc != FSIB_OK:
        raise FsibError(rc, lib.fsib_static_last_error().decode())
    return fhat


def version():
    return load().fsib_version().decode()
