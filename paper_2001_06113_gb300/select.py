"""Accuracy-adaptive choice of the free-space discretisation: trading digits
for speed (Sec. 7, Example 4).

For a target precision eps the contour offset H follows Remark Hchoice with
the machine epsilon of the arithmetic that evaluates the contour sums; a
larger eps gives a larger H, a less oscillatory spectral Green's function
along Gamma and so allows a coarser equispaced spacing h = pi n / nu (a
shorter FFT length nu = R n) and, above the FP32 rounding floor, FP32
transforms.  The paper picks h by hand per eps; here the choice is measured:

* candidates (precision, R): "mixed" (FP32 transforms) where H > 0 for
  eps_m = 2^-23, and "fp64"; R in (4, 8, 16) with nu <= 4096;
* each candidate runs the problem for `probe_steps` steps on the device
  (its start-up, then timed Adams steps) and is compared on the grid with a
  reference run (FP64, the largest R, H for a precision 1e-3 of the target
  and at most 1e-11);
* the cheapest candidate by measured time per step whose probe error is at
  most `safety * eps` is chosen (the reference itself if none is).

The probe error measures what H, h and the transform precision control (the
contour quadrature and its rounding, per step and accumulated over the
probe); the time-stepping error of the caller's dt is the same for every
candidate and is not part of the choice.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import Problem, TdseError, free_choose_H



@dataclasses.dataclass
class Candidate:
    precision: str
    R: int
    nu: List[int]
    H: float
    err: Optional[float] = None          # probe error against the reference (rel. L2 on the grid)
    ms_per_step: Optional[float] = None


def _vnorm_phimax(inst) -> tuple:
    """||V||_{2,inf} on the grid over the time samples and max |phi| (phi from
    the sampled A by the trapezoid rule on 4001 points), as Remark Hchoice."""
    d = inst.dim
    cell = (2.0 / inst.shape[0]) ** d
    ts = np.linspace(0.0, inst.nsteps * inst.dt, 9)
    vnorm = max(math.sqrt(float(np.sum(inst.V_at(float(t)) ** 2)) * cell) for t in ts)
    phimax = 0.0
    if inst.pulse is not None:
        t = np.linspace(0.0, inst.nsteps * inst.dt, 4001)
        A = inst.pulse.A(t)
        phi = np.cumsum(0.5 * (A[1:] + A[:-1]) * (t[1] - t[0]), axis=0)
        phimax = float(np.max(np.abs(phi)))
    return vnorm, phimax


def candidates(inst, eps: float, R_values: Sequence[int] = (4, 8, 16), allow_mixed: bool = True) -> List[Candidate]:
    """Admissible (precision, R) for `inst` at target eps, with their H."""
    vnorm, phimax = _vnorm_phimax(inst)
    out = []
    for prec in (("mixed", "fp64") if allow_mixed else ("fp64",)):
        try:
            H = free_choose_H(eps, vnorm, phimax, inst.dim, precision=prec)
        except TdseError:          # eps below this precision's floor: H would not be positive
            continue
        for R in R_values:
            nu = [R * n for n in inst.shape]
            if max(nu) <= 4096:
                out.append(Candidate(prec, R, nu, H))
    return out


def choose(cands: Sequence[Candidate], eps: float, safety: float = 0.1) -> Optional[Candidate]:
    """The fastest candidate whose probe error is within safety * eps."""
    ok = [c for c in cands if c.err is not None and c.ms_per_step is not None and c.err <= safety * eps]
    return min(ok, key=lambda c: c.ms_per_step) if ok else None


def _probe(inst, n: int, precision: str, nu, H: float, gauss_q: int, n_r: int, startup: int):
    import torch
    table = inst.Vt is not None
    pr = Problem(inst.shape, inst.dt, inst.nsteps, precision=precision, bc="free", nu=nu, H=H, gauss_q=gauss_q,
                 n_r=n_r, potential="table" if table else "separable")
    if table:
        pr.set_potential_fn(inst.V_at)
    else:
        pr.set_potential(inst.V0, inst.vfac_table())
    if inst.pulse is not None:
        p = inst.pulse
        pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
    pr.set_initial(inst.u0)
    pr.step(startup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pr.step(n - startup)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (n - startup)
    u = pr.read_u(0)
    pr.close()
    return u, ms


def select_free(inst, eps: float, probe_steps: int = 24, safety: float = 0.1, R_values: Sequence[int] = (4, 8, 16),
                allow_mixed: bool = True, gauss_q: int = 10, n_r: int = 1) -> Dict:
    """Choose (precision, nu, H) for a free-space instance at target eps.
    Returns {"choice": Candidate, "reference": Candidate, "candidates": [...]}."""
    startup = 7
    if probe_steps <= startup or probe_steps > inst.nsteps:
        raise ValueError("probe_steps must exceed the start-up and fit the instance's nsteps")
    Rmax = max(R for R in R_values if max(R * n for n in inst.shape) <= 4096)
    eps_ref = min(1e-3 * eps, 1e-11)
    vnorm, phimax = _vnorm_phimax(inst)
    ref = Candidate("fp64", Rmax, [Rmax * n for n in inst.shape],
                    free_choose_H(eps_ref, vnorm, phimax, inst.dim, precision="fp64"), err=0.0)
    u_ref, ref.ms_per_step = _probe(inst, probe_steps, "fp64", ref.nu, ref.H, gauss_q, n_r, startup)
    cands = candidates(inst, eps, R_values, allow_mixed)
    for c in cands:
        u, c.ms_per_step = _probe(inst, probe_steps, c.precision, c.nu, c.H, gauss_q, n_r, startup)
        c.err = float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))
    pick = choose(cands, eps, safety)
    return {"choice": pick if pick is not None else ref, "reference": ref, "candidates": cands}
