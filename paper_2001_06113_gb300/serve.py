"""Request loop for many TDSE solves on one GPU (continuous admission).

Solve requests arrive over time (each with its own grid, V, A, u0, dt and
step count).  The loop

  * admits a waiting request as soon as its device workspace fits the HBM
    budget (and an active-solve slot is free), in arrival order;
  * keeps every admitted solve's state -- mode state and the (Vu)^ history
    ring -- resident in its own workspace until the solve ends;
  * enqueues the whole solve on the request's own CUDA stream at admission,
    so that the kernels of all admitted solves overlap on the device;
  * polls completion events, reads each finished result back, frees its
    workspace (which admits the next requests) and records its
    time-to-solution;
  * reports p50 / p99 time-to-solution and the aggregate point-steps/s.

Failures stay with their request: a request whose set-up or start fails (e.g.
no device memory), whose result is not finite, or which is cancelled
(`cancel_after` seconds after its arrival) gets `error` set, its workspace
released once nothing of it is left on the device, and the loop goes on with
the others.  Kernels already enqueued cannot be stopped: a cancelled active
solve runs to its end, and its result is dropped.

Every step runs in the library's kernels through `Problem`; this module is
host-side scheduling only.  The device operations are behind a small backend
interface so that the scheduling logic is testable without a GPU.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

# 1D requests of at least this many points run in the four-step layout: one
# instance of n = 16384 in one CTA holds a single SM for each step, the
# four-step passes spread it over 2 n0 / 8 CTAs (the layout beyond 16384
# anyway).
FOUR_STEP_FROM = 16384


@dataclasses.dataclass

class Request:
    """One solve: `inst` carries grid shape, V0 and its time factor, the pulse,
    u0, dt and the step count; `bc`/`precision` and the free-space contour
    parameters (`free`: nu, H, gauss_q, n_r) select the solver."""

    rid: int
    arrival: float
    inst: object
    bc: str = "periodic"
    precision: str = "mixed"
    free: Optional[dict] = None
    # filled in by the server
    cancel_after: Optional[float] = None   # seconds after arrival
    admitted: Optional[float] = None
    finished: Optional[float] = None
    result: Optional[np.ndarray] = None
    error: Optional[str] = None

    @property
    def points(self) -> int:
        return int(np.prod(self.inst.shape))

    @property
    def nsteps(self) -> int:
        return int(self.inst.nsteps)

    @property
    def latency(self) -> Optional[float]:
        return None if self.finished is None else self.finished - self.arrival


class Backend:
    """Device operations the server needs (one handle per admitted request)."""

    def prepare(self, req: Request):                 # host-only context; returns handle
        raise NotImplementedError

    def workspace_bytes(self, handle) -> int:
        raise NotImplementedError

    def start(self, handle):                         # allocate, upload inputs, enqueue the solve
        raise NotImplementedError

    def done(self, handle) -> bool:
        raise NotImplementedError

    def finish(self, handle) -> np.ndarray:          # read the result, release the workspace
        raise NotImplementedError

    def release(self, handle):                       # drop a started solve (after done) or a failed start
        pass


class TorchBackend(Backend):
    """Problem contexts with torch-allocated workspaces, one CUDA stream each."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = device

    def prepare(self, req: Request):
        from . import Problem
        it = req.inst
        kw = {}
        if req.bc == "free":
            kw = dict(bc="free", nu=req.free["nu"], H=req.free["H"], gauss_q=req.free.get("gauss_q", 10),
                      n_r=req.free.get("n_r", 1))
        elif len(it.shape) == 1 and it.shape[0] >= FOUR_STEP_FROM:
            kw = dict(layout_1d="passes")
        # sized on the host before any device memory is taken
        return {"req": req, "stream": None, "kw": kw, "prob": None, "event": None,
                "bytes": Problem.workspace_bytes_for(it.shape, it.dt, it.nsteps, precision=req.precision, **kw)}

    def workspace_bytes(self, handle) -> int:
        return int(handle["bytes"])

    def start(self, handle):
        from . import Problem
        req = handle["req"]
        stream = handle["stream"] = self.torch.cuda.Stream(device=self.device)
        it = req.inst
        prob = Problem(it.shape, it.dt, it.nsteps, precision=req.precision, stream=stream, device=self.device,
                       **handle["kw"])
        prob.set_potential(it.V0, it.vfac_table())
        if it.pulse is not None:
            p = it.pulse
            prob.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
        prob.set_initial(it.u0)
        prob.step(it.nsteps)
        ev = self.torch.cuda.Event()
        ev.record(stream)
        handle["prob"], handle["event"] = prob, ev

    def done(self, handle) -> bool:
        return handle["event"] is not None and handle["event"].query()

    def finish(self, handle) -> np.ndarray:
        prob = handle["prob"]
        try:
            prob.check_finite()
            return prob.read_u(0)
        finally:
            self.release(handle)

    def release(self, handle):
        prob = handle.get("prob")
        if prob is not None:
            prob.close()
            handle["prob"] = None


class Server:
    """Admission by HBM budget, overlapped solves, time-to-solution statistics.

    `clock` gives seconds (wall clock by default); request arrivals are in
    seconds from the start of `run`.
    """

    def __init__(self, backend: Backend, hbm_budget: int, max_active: int = 64,
                 clock: Callable[[], float] = time.perf_counter, idle_sleep: float = 2e-4):
        self.backend = backend
        self.hbm_budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.clock = clock
        self.idle_sleep = idle_sleep
        self.peak_bytes = 0
        self.peak_active = 0

    def run(self, requests: Sequence[Request]) -> Dict:
        waiting = sorted(requests, key=lambda r: (r.arrival, r.rid))
        handles = {}
        for r in waiting:
            try:
                handles[r.rid] = self.backend.prepare(r)
            except Exception as e:                   # invalid request: reported, not served
                r.error = f"prepare: {e}"
                continue
            if self.backend.workspace_bytes(handles[r.rid]) > self.hbm_budget:
                raise ValueError(f"request {r.rid} needs more than the HBM budget")
        waiting = [r for r in waiting if r.error is None]
        active: List[Request] = []
        used = 0
        t0 = self.clock()
        qi = 0

        def cancelled(r, now):
            return r.cancel_after is not None and now >= r.arrival + r.cancel_after

        while qi < len(waiting) or active:
            now = self.clock() - t0
            progressed = False
            # completions first: they free memory for admissions
            for r in list(active):
                h = handles[r.rid]
                try:
                    finished = self.backend.done(h)
                except Exception as e:
                    r.error, finished = f"done: {e}", True
                if not finished:
                    if cancelled(r, now) and r.error is None:
                        r.error = "cancelled"            # dropped once its enqueued work ends
                    continue
                if r.error is None:
                    try:
                        r.result = self.backend.finish(h)
                    except Exception as e:
                        r.error = f"finish: {e}"
                else:
                    self.backend.release(h)
                r.finished = self.clock() - t0
                used -= self.backend.workspace_bytes(h)
                active.remove(r)
                progressed = True
            # admissions in arrival order (head-of-line: a large request waits for memory)
            while qi < len(waiting) and len(active) < self.max_active:
                r = waiting[qi]
                if r.arrival > now:
                    break
                if cancelled(r, now):                    # cancelled while waiting
                    r.error = "cancelled"
                    r.finished = now
                    qi += 1
                    progressed = True
                    continue
                need = self.backend.workspace_bytes(handles[r.rid])
                if used + need > self.hbm_budget:
                    break
                r.admitted = self.clock() - t0
                qi += 1
                progressed = True
                try:
                    self.backend.start(handles[r.rid])
                except Exception as e:                   # e.g. no device memory: this request fails
                    r.error = f"start: {e}"
                    self.backend.release(handles[r.rid])
                    r.finished = self.clock() - t0
                    continue
                used += need
                active.append(r)
                self.peak_bytes = max(self.peak_bytes, used)
                self.peak_active = max(self.peak_active, len(active))
            if not progressed:
                if self.idle_sleep:
                    time.sleep(self.idle_sleep)
        makespan = self.clock() - t0
        return self.stats(requests, makespan)

    def stats(self, requests: Sequence[Request], makespan: float) -> Dict:
        ok = [r for r in requests if r.error is None]
        lat = np.array([r.latency for r in ok] or [np.nan], dtype=np.float64)
        work = float(sum(r.points * r.nsteps for r in ok))
        return {"requests": len(requests), "completed": len(ok),
                "failed": sum(1 for r in requests if r.error is not None and r.error != "cancelled"),
                "cancelled": sum(1 for r in requests if r.error == "cancelled"), "makespan_s": makespan,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(lat.mean()), "point_steps": work,
                "point_steps_per_s": work / makespan if makespan > 0 else None,
                "peak_bytes": self.peak_bytes, "peak_active": self.peak_active}



def free_contour_params(inst, eps: float = 1e-10, R: int = 8, gauss_q: int = 10, n_r: int = 1,
                        precision: str = "fp64") -> dict:
    """Contour parameters of a free-space request: nu = R n per axis and H of
    Remark Hchoice from ||V||_2 on the grid and max |phi| (phi integrated from
    the sampled pulse by the trapezoid rule on 4001 points), with the machine
    epsilon of `precision` ("mixed": FP32 contour sums)."""
    from . import free_choose_H
    d = len(inst.shape)
    vnorm = float(np.sqrt(np.sum(inst.V0 ** 2) * (2.0 / inst.shape[0]) ** d))
    vnorm *= float(np.max(np.abs(inst.vfac_table())))
    phimax = 0.0
    if inst.pulse is not None:
        t = np.linspace(0.0, inst.nsteps * inst.dt, 4001)
        A = inst.pulse.A(t)
        phi = np.cumsum(0.5 * (A[1:] + A[:-1]) * (t[1] - t[0]), axis=0)
        phimax = float(np.max(np.abs(phi)))
    return {"nu": [R * n for n in inst.shape], "H": free_choose_H(eps, vnorm, phimax, d, precision=precision),
            "gauss_q": gauss_q, "n_r": n_r}


FREE_EPS = {"fp64": 1e-10, "mixed": 1e-4}


def requests_from_trace(trace, free_eps: Optional[float] = None, free_precision: str = "fp64", free_R: int = 8):
    """Requests of a synth.serve_requests trace: periodic classes in mixed
    precision, free space in `free_precision` ("fp64", or "mixed" = FP32
    transforms) on the contour chosen for free_eps (default 1e-10 in FP64,
    1e-4 with FP32 sums) with nu = free_R n per axis."""
    eps = FREE_EPS[free_precision] if free_eps is None else free_eps
    out = []
    for i, (t, kind, inst) in enumerate(trace):
        if kind == "free":
            out.append(Request(i, t, inst, bc="free", precision=free_precision,
                               free=free_contour_params(inst, eps, R=free_R, precision=free_precision)))
        else:
            out.append(Request(i, t, inst, precision="mixed"))
    return out
