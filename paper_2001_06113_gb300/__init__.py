"""GB300-native (sm_103a) solver for the time-dependent Schroedinger equation
by the Volterra / spectral-recurrence method of Kaye, Barnett & Greengard
(arXiv:2001.06113).

Every step of the method runs in the CUDA kernels of ``libtdse_gb300.so``
(C ABI in ``include/tdse.h``); this package only marshals arguments:
PyTorch provides the device workspace and the stream.  There is no CPU
fallback: if the library is not built, using it raises ImportError.
"""
from __future__ import annotations

import ctypes
from typing import Callable, Optional, Sequence

import numpy as np

from . import _native
from ._native import DEVICE, FP64, FREE, HOST, MIXED, PERIODIC, TdseError

__all__ = ["Problem", "Batch", "TdseError", "adams_weights", "free_choose_H", "FP64", "MIXED", "PERIODIC", "FREE"]


def _check(status: int, ctx=None):
    if status != _native.TDSE_OK:
        msg = ""
        if ctx is not None:
            raw = _native.lib().tdse_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise TdseError(status, msg)


def adams_weights(order: int) -> np.ndarray:
    """The library's implicit Adams weights mu_0..mu_{order-1} (Sec. 2.2)."""
    out = np.zeros(order, dtype=np.float64)
    _check(_native.lib().tdse_adams_weights(order, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def free_choose_H(eps: float, vnorm: float, phimax: float, dim: int, precision: str = "fp64") -> float:
    """Contour offset H of Remark Hchoice (library formula), with the machine
    epsilon of the precision the contour sums run in ("fp64" or "mixed")."""
    out = ctypes.c_double()
    prec = {"fp64": FP64, "mixed": MIXED}[precision]
    _check(_native.lib().tdse_free_choose_H_prec(float(eps), float(vnorm), float(phimax), int(dim), prec,
                                                 ctypes.byref(out)))
    return out.value


def _config(shape, dt, nsteps, order, batch, precision, startup_steps, bc, nu, H, alpert_p, gauss_q, n_r,
            potential="separable", c_transform="auto", layout_1d="auto"):
    cfg = _native.TdseConfig()
    cfg.c_transform = {"auto": 0, "direct": 1, "chebyshev": 2}[c_transform]
    cfg.layout_1d = {"auto": 0, "cta": 1, "passes": 2}[layout_1d]
    cfg.potential = {"separable": _native.TDSE_V_SEPARABLE, "table": _native.TDSE_V_TABLE,
                     "shared_table": _native.TDSE_V_TABLE_SHARED}[potential]
    cfg.dim = len(shape)
    cfg.bc = {"periodic": PERIODIC, "free": FREE}[bc]
    if bc == "free":
        nus = list(nu) if nu is not None else [8 * s for s in shape]
        cfg.nu[0] = int(nus[0])
        cfg.nu[1] = int(nus[1]) if len(nus) > 1 else 0
        cfg.nu_z = int(nus[2]) if len(nus) > 2 else 0
        cfg.alpert_p = int(alpert_p)
        cfg.gauss_q = int(gauss_q)
        cfg.n_r = int(n_r)
        cfg.H = float(H)
    cfg.n[0] = shape[0]
    cfg.n[1] = shape[1] if len(shape) > 1 else 1
    cfg.n_z = shape[2] if len(shape) > 2 else 1
    cfg.batch = int(batch)
    cfg.dt = float(dt)
    cfg.nsteps = int(nsteps)
    cfg.order = int(order)
    cfg.startup_steps = int(startup_steps)
    cfg.precision = {"fp64": FP64, "mixed": MIXED}[precision]
    return cfg


def _stream_handle(stream) -> Optional[int]:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _as_buffer(x, dtype):
    """(pointer, where, keepalive) for a host numpy array or a torch tensor."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        tdt = torch.complex128 if dtype == np.complex128 else torch.float64
        t = x.detach()
        if t.dtype != tdt:
            t = t.to(tdt)
        t = t.contiguous()
        return ctypes.c_void_p(t.data_ptr()), (DEVICE if t.is_cuda else HOST), t
    a = np.ascontiguousarray(np.asarray(x, dtype=dtype))
    return ctypes.c_void_p(a.ctypes.data), HOST, a


class Problem:
    """A batch of TDSE instances sharing grid, dt, step count and order.

    Parameters mirror ``tdse_config``: ``shape`` (n,), (n0, n1) or (n0, n1, n2); ``dt``;
    ``nsteps`` (steps the tables cover); ``order`` (Adams order, even <= 8);
    ``batch``; ``precision`` ("fp64" or "mixed"); ``startup_steps`` (-1 =
    order-1); ``bc`` ("periodic" or "free").  Free space also takes ``nu``
    (FFT length per dimension), ``H`` (contour offset), ``alpert_p``,
    ``gauss_q`` and ``n_r``.  ``layout_1d`` (1D periodic): "cta" (one CTA per
    instance), "passes" (the four-step form through the 2D pass kernels) or
    "auto" (one CTA where built).  ``potential``: "separable" (V = f(t) V0(x),
    ``set_potential``), "table" (general V(x, t) per instance, given at
    ``potential_times()``, ``set_potential_table`` / ``set_potential_fn``) or
    "shared_table" (one such table for every instance, instance = -1).
    The device workspace is a torch uint8 tensor owned here.
    """

    def __init__(self, shape: Sequence[int], dt: float, nsteps: int, order: int = 8, batch: int = 1,
                 precision: str = "fp64", startup_steps: int = -1, device=None, stream=None, bc: str = "periodic",
                 nu: Optional[Sequence[int]] = None, H: float = 0.0, alpert_p: int = 8, gauss_q: int = 10,
                 n_r: int = 1, potential: str = "separable", c_transform: str = "auto", layout_1d: str = "auto"):
        import torch
        self._lib = _native.lib()
        self.shape = tuple(int(s) for s in shape)
        self.batch = int(batch)
        self.dt = float(dt)
        self.nsteps = int(nsteps)
        self.bc = bc
        self.precision = precision
        self.potential = potential
        cfg = _config(self.shape, dt, nsteps, order, batch, precision, startup_steps, bc, nu, H, alpert_p, gauss_q,
                      n_r, potential, c_transform, layout_1d)
        self._ctx = ctypes.c_void_p()
        _check(self._lib.tdse_create(ctypes.byref(cfg), ctypes.byref(self._ctx)))
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.workspace_bytes = int(self._lib.tdse_workspace_bytes(self._ctx))
        self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        aligned = (base + 255) & ~255
        self._stream = stream
        _check(self._lib.tdse_bind_workspace(self._ctx, ctypes.c_void_p(aligned), self.workspace_bytes,
                                             _stream_handle(stream)), self._ctx)
        self._callbacks = []

    @staticmethod
    def workspace_bytes_for(shape: Sequence[int], dt: float, nsteps: int, order: int = 8, batch: int = 1,
                            precision: str = "fp64", startup_steps: int = -1, bc: str = "periodic",
                            nu: Optional[Sequence[int]] = None, H: float = 0.0, alpert_p: int = 8, gauss_q: int = 10,
                            n_r: int = 1, potential: str = "separable", c_transform: str = "auto",
                            layout_1d: str = "auto") -> int:
        """Device workspace a Problem of this configuration needs (host-only query)."""
        lib = _native.lib()
        cfg = _config(tuple(int(s) for s in shape), dt, nsteps, order, batch, precision, startup_steps, bc, nu, H,
                      alpert_p, gauss_q, n_r, potential, c_transform, layout_1d)
        ctx = ctypes.c_void_p()
        _check(lib.tdse_create(ctypes.byref(cfg), ctypes.byref(ctx)))
        n = int(lib.tdse_workspace_bytes(ctx))
        lib.tdse_destroy(ctx)
        return n + 256

    @property
    def npoints(self) -> int:
        return int(np.prod(self.shape))

    def set_potential(self, V0, time_factor=None, instance: int = -1):
        """V(x,t) = f(t) V0(x); time_factor = f(m dt/8), m = 0..8*nsteps (host array) or None."""
        pv, where, keep = _as_buffer(V0, np.float64)
        tf_ptr = None
        if time_factor is not None:
            tf = np.ascontiguousarray(np.asarray(time_factor, dtype=np.float64))
            if tf.size != 8 * self.nsteps + 1:
                raise ValueError("time_factor must have 8*nsteps+1 samples")
            tf_ptr = ctypes.c_void_p(tf.ctypes.data)
        _check(self._lib.tdse_set_potential(self._ctx, instance, pv, tf_ptr, where, _stream_handle(self._stream)),
               self._ctx)
        del keep

    def potential_times(self) -> np.ndarray:
        """Times at which a potential-table Problem evaluates V (every dt/8 of
        the start-up steps, then every step)."""
        n = int(self._lib.tdse_potential_times(self._ctx, None))
        if n < 0:
            raise TdseError(_native.TDSE_ESTATE, "not a potential-table Problem")
        t = np.empty(n, dtype=np.float64)
        self._lib.tdse_potential_times(self._ctx, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return t

    def set_potential_table(self, V, instance: int = -1):
        """V(x, t_r) for every t_r of potential_times(): array [R] + shape
        (numpy or torch, host or cuda)."""
        pv, where, keep = _as_buffer(V, np.float64)
        _check(self._lib.tdse_set_potential_table(self._ctx, instance, pv, where, _stream_handle(self._stream)),
               self._ctx)
        del keep

    def set_potential_fn(self, Vt: Callable, instance: int = -1):
        """V from a callable t -> V(x, t) on the grid, sampled at potential_times()."""
        t = self.potential_times()
        self.set_potential_table(np.stack([np.asarray(Vt(float(tt)), dtype=np.float64) for tt in t]), instance)

    def set_pulse(self, A0: float, omega: float, T_pulse: float, direction, instance: int = -1):
        d = (ctypes.c_double * 3)(*(list(direction) + [0.0, 0.0, 0.0])[:3])
        _check(self._lib.tdse_set_pulse(self._ctx, instance, A0, omega, T_pulse, d, _stream_handle(self._stream)),
               self._ctx)

    def set_vector_potential(self, A: Optional[Callable], instance: int = -1):
        """A(t) -> sequence of len(shape) floats, or None for A = 0."""
        dim = len(self.shape)
        if A is None:
            cb = _native.FIELD_FN()
        else:
            def _cb(t, out, user):
                v = A(t)
                for i in range(dim):
                    out[i] = float(v[i])
            cb = _native.FIELD_FN(_cb)
        self._callbacks.append(cb)
        _check(self._lib.tdse_set_vector_potential(self._ctx, instance, cb, None, _stream_handle(self._stream)),
               self._ctx)

    def set_initial(self, u0, instance: int = -1):
        pu, where, keep = _as_buffer(u0, np.complex128)
        _check(self._lib.tdse_set_initial(self._ctx, instance, pu, where, _stream_handle(self._stream)), self._ctx)
        del keep

    def set_initial_batch(self, u0):
        """u0 of every instance at once: array [batch] + shape (numpy or torch,
        host or cuda, complex128), one copy."""
        pu, where, keep = _as_buffer(u0, np.complex128)
        _check(self._lib.tdse_set_initial_batch(self._ctx, pu, where, _stream_handle(self._stream)), self._ctx)
        del keep

    def step(self, n: int = 1):
        _check(self._lib.tdse_step(self._ctx, int(n), _stream_handle(self._stream)), self._ctx)

    def solve_to(self, T: float):
        _check(self._lib.tdse_solve_to(self._ctx, float(T), _stream_handle(self._stream)), self._ctx)

    def read_u(self, instance: int = -1, out=None):
        """u on the grid: numpy complex128 (host) by default, or into `out`
        (numpy array or torch tensor, host or cuda, complex128)."""
        nb = self.batch if instance == -1 else 1
        shape = ((nb,) if instance == -1 else ()) + self.shape
        if out is None:
            out = np.empty(shape, dtype=np.complex128)
        try:
            import torch
            is_t = isinstance(out, torch.Tensor)
        except ImportError:  # pragma: no cover
            is_t = False
        if is_t:
            ptr, where = ctypes.c_void_p(out.data_ptr()), (DEVICE if out.is_cuda else HOST)
        else:
            ptr, where = ctypes.c_void_p(out.ctypes.data), HOST
        _check(self._lib.tdse_read_u(self._ctx, instance, ptr, where, _stream_handle(self._stream)), self._ctx)
        return out

    def read_modes(self, instance: int = -1) -> np.ndarray:
        """The FP64 mode state u^ (periodic: FFT order; free space: node order
        of ``free_rule``) as numpy complex128, [batch][...] for instance -1."""
        shape = self.mode_shape
        out = np.empty(((self.batch,) if instance == -1 else ()) + shape, dtype=np.complex128)
        _check(self._lib.tdse_read_modes(self._ctx, instance, ctypes.c_void_p(out.ctypes.data), HOST,
                                         _stream_handle(self._stream)), self._ctx)
        return out

    @property
    def mode_shape(self):
        if self.bc != "free":
            return self.shape
        return tuple(self.free_rule(a)[0].size for a in range(len(self.shape)))

    def cheb_terms(self, axis: int) -> int:
        """Free space: Chebyshev terms N_T of the C-type transforms of `axis`
        (0: direct sums)."""
        return int(self._lib.tdse_free_cheb_terms(self._ctx, axis))

    def free_rule(self, axis: int):
        """(zeta, w): nodes and weights of the contour rule of `axis` (free space)."""
        n = ctypes.c_int()
        _check(self._lib.tdse_free_rule(self._ctx, axis, ctypes.byref(n), None, None), self._ctx)
        z = np.empty(n.value, dtype=np.complex128)
        w = np.empty(n.value, dtype=np.complex128)
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self._lib.tdse_free_rule(self._ctx, axis, ctypes.byref(n), z.ctypes.data_as(dp), w.ctypes.data_as(dp)),
               self._ctx)
        return z, w

    def set_residual_check(self, every: int, tol: float = 1e-6):
        """FP64 residual check of the mixed implicit step after every `every`-th
        Adams step, with an FP64 redo where the residual exceeds `tol`."""
        _check(self._lib.tdse_set_residual_check(self._ctx, int(every), float(tol)), self._ctx)

    def residual_report(self):
        """(rho per instance of the last check, FP64 redos per instance, checks run)."""
        rho = np.zeros(self.batch, dtype=np.float64)
        corr = np.zeros(self.batch, dtype=np.int32)
        n = ctypes.c_int()
        _check(self._lib.tdse_residual_report(self._ctx, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              corr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.byref(n),
                                              _stream_handle(self._stream)), self._ctx)
        return rho, corr, n.value

    def save(self) -> bytes:
        """Checkpoint of the whole solve state (workspace and step counters)."""
        n = ctypes.c_size_t()
        _check(self._lib.tdse_save(self._ctx, None, ctypes.byref(n), _stream_handle(self._stream)), self._ctx)
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.tdse_save(self._ctx, buf, ctypes.byref(n), _stream_handle(self._stream)), self._ctx)
        return buf.raw[:n.value]

    def load(self, blob: bytes):
        """Resume from `save()` output of a Problem with the same configuration."""
        _check(self._lib.tdse_load(self._ctx, blob, len(blob), _stream_handle(self._stream)), self._ctx)

    def check_finite(self):
        _check(self._lib.tdse_check_finite(self._ctx, _stream_handle(self._stream)), self._ctx)

    def set_step_path(self, path: str):
        """Kernels of the 2D mixed Adams steps: "auto" (default), "passes" (row
        and column pass kernels) or "cluster" (512^2: one cluster of 16 CTAs per
        instance, intermediates in shared memory).  Same results either way."""
        code = {"auto": _native.PATH_AUTO, "passes": _native.PATH_PASSES, "cluster": _native.PATH_CLUSTER}[path]
        _check(self._lib.tdse_set_step_path(self._ctx, code), self._ctx)

    @property
    def step_path(self) -> str:
        """The kernels the next 2D mixed Adams steps use: "passes" or "cluster"."""
        return {_native.PATH_PASSES: "passes", _native.PATH_CLUSTER: "cluster"}.get(
            int(self._lib.tdse_step_path(self._ctx)), "passes")

    def set_step_groups(self, groups: int):
        """2D pass kernels: step chains of `groups` groups of instances on
        parallel streams (same results; default 4)."""
        _check(self._lib.tdse_set_step_groups(self._ctx, int(groups)), self._ctx)

    def set_shape_1d(self, shape: int):
        """1D mixed contexts: launch shape of the step kernel (0: n/8 threads per
        instance, at most 512 below n = 16384; 1: 1024 threads for n = 8192, half
        the default for the other n >= 512).  Same results."""
        _check(self._lib.tdse_set_shape_1d(self._ctx, int(shape)), self._ctx)

    @property
    def shape_1d(self) -> int:
        return int(self._lib.tdse_shape_1d(self._ctx))

    def describe_steps(self) -> dict:
        """Launch shape of the 2D mixed Adams steps (path, clusters, ...)."""
        import json
        buf = ctypes.create_string_buffer(512)
        _check(self._lib.tdse_describe_steps(self._ctx, buf, 512), self._ctx)
        return json.loads(buf.value.decode())

    @property
    def step_index(self) -> int:
        return int(self._lib.tdse_step_index(self._ctx))

    @property
    def time(self) -> float:
        return float(self._lib.tdse_time(self._ctx))

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.tdse_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Uneven batch of 1D periodic mixed-precision Problems stepped together
    (``tdse_batch_*``): the Adams phase as one persistent launch per step for
    all members ("fused") or each member's own kernel on its own stream
    ("streams"; chosen by ``tune``), the whole step sequence of a call
    captured into a CUDA graph and replayed.  The members stay owned by the
    caller and must outlive the batch."""

    def __init__(self, members: Sequence[Problem], stream=None):
        self._lib = _native.lib()
        self.members = list(members)
        self._stream = stream if stream is not None else self.members[0]._stream
        arr = (ctypes.c_void_p * len(self.members))(*[m._ctx.value for m in self.members])
        self._b = ctypes.c_void_p()
        st = self._lib.tdse_batch_create(arr, len(self.members), ctypes.byref(self._b))
        if st != _native.TDSE_OK:
            raise TdseError(st, "tdse_batch_create")

    def _check(self, st):
        if st != _native.TDSE_OK:
            raw = self._lib.tdse_batch_last_error(self._b)
            raise TdseError(st, raw.decode() if raw else "")

    def set_mode(self, mode: str):
        """Adams phase as one fused launch per step ("fused") or each member's
        own kernel on its own stream ("streams"); same results."""
        self._check(self._lib.tdse_batch_set_mode(self._b, {"fused": 0, "streams": 1}[mode]))

    def tune(self, trial_steps: int = 5):
        """Autotune the launch shape and the mode; afterwards every member needs set_initial."""
        self._check(self._lib.tdse_batch_tune(self._b, int(trial_steps), _stream_handle(self._stream)))

    def step(self, n: int, stream=None):
        """Advance all members n steps on the batch's stream (or `stream`).  On a
        side stream the launch sequence is captured into a CUDA graph the first
        time and replayed afterwards; on the legacy default stream it is launched
        directly."""
        s = self._stream if stream is None else stream
        self._check(self._lib.tdse_batch_step(self._b, int(n), _stream_handle(s)))

    def describe(self) -> dict:
        import json
        buf = ctypes.create_string_buffer(8192)
        self._check(self._lib.tdse_batch_describe(self._b, buf, len(buf)))
        return json.loads(buf.value.decode())

    def close(self):
        if getattr(self, "_b", None):
            self._lib.tdse_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
