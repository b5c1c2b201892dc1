"""GPU parity of the 3D free-space path against the FP64 oracle, through the
C ABI.

In 3D the contour modes are the tensor product of three one-axis rules and
both transforms are tensor products of the one-axis transforms (Sec. 4.3:
the construction of the 1D and 2D cases carried to a third axis); the step
is eq. uadamsk with zeta for k as in 1D and 2D.  The oracle
(oracle/freespace.py at d = 3) is pinned on the CPU by the outer product of
three 1D closed-form solves.  Both sides march the same seeded problem
(uneven axes, so that a mix-up of two axes shows) with the same contour
parameters; the bounds are those of the 1D and 2D tests: 1e-12 for FP64 on
the grid and on the contour, 2e-6 for the FP32-transform variant.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fields, gamma
from oracle.freespace import FreeSpaceOracle

pytestmark = pytest.mark.gpu

MIXED_TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def _instance(shape, n, seed=5, dt=1e-3, A0=40.0, omega=150.0):
    return synth.free_bump_gaussians(shape, seed=seed, dt=dt, nsteps=n, A0=A0, omega=omega,
                                     direction=(1.0, -0.5, 0.3),
                                     vfac=lambda t: 1.0 + 0.3 * np.sin(40.0 * np.asarray(t, dtype=np.float64)))


def _H(inst, eps, eps_m=gamma.EPS_M):
    phi = fields.phi_callable(inst.pulse, 3)
    phimax = max(float(np.max(np.abs(phi(t)))) for t in np.linspace(0.0, inst.t_max, 401))
    cell = np.prod([2.0 / m for m in inst.shape])
    vnorm = math.sqrt(float(np.sum(inst.V0 ** 2)) * cell) * float(np.max(np.abs(inst.vfac_table())))
    return gamma.choose_H(eps, vnorm, phimax, 3, eps_m=eps_m)


def _problem(insts, nu, H, q, n_r, order, startup, precision):
    from paper_2001_06113_gb300 import Problem
    it0 = insts[0]
    pr = Problem(it0.shape, it0.dt, it0.nsteps, order=order, startup_steps=startup, batch=len(insts), bc="free",
                 nu=nu, H=H, gauss_q=q, n_r=n_r, precision=precision)
    for b, inst in enumerate(insts):
        pr.set_potential(inst.V0, inst.vfac_table(), instance=b)
        pr.set_pulse(inst.pulse.A0, inst.pulse.omega, inst.pulse.T_pulse, inst.pulse.direction, instance=b)
        pr.set_initial(inst.u0, instance=b)
    return pr


def _oracle(inst, nu, H, n, q, n_r, order, startup, keep=None):
    rules = [gamma.GammaRule.for_nu(M, v, H, q=q, n_r=n_r) for M, v in zip(inst.shape, nu)]
    orc = FreeSpaceOracle(rules, inst.dt, inst.V0, inst.vfac, fields.phi_callable(inst.pulse, 3), order=order,
                          n_startup=startup)
    out = orc.solve(inst.u0, n, keep=keep)
    return out, orc.last_uhat


CASES = [
    # shape, nu, q, n_r, order, startup (None = order - 1), steps
    ((32, 64, 32), (128, 256, 128), 10, 1, 4, 3, 7),     # uneven axes, a few Adams steps past the start-up
    ((32, 32, 32), (128, 128, 256), 8, 1, 8, None, 9),   # the 8th-order scheme with its 7-step start-up
]


@pytest.mark.parametrize("shape,nu,q,n_r,order,startup,n", CASES)
def test_free_3d_matches_oracle(shape, nu, q, n_r, order, startup, n):
    import torch
    inst = _instance(shape, n + 2)
    H = _H(inst, 1e-10)
    pr = _problem([inst], nu, H, q, n_r, order, -1 if startup is None else startup, "fp64")
    pr.step(n)
    torch.cuda.synchronize()
    u, uh = pr.read_u(0), pr.read_modes(0)
    pr.close()
    uo, uho = _oracle(inst, nu, H, n, q, n_r, order, startup)
    e_u, e_h = rel(u, uo), rel(uh, uho)
    print(shape, "3D free space FP64 vs oracle", e_u, e_h)
    assert e_u < 1e-12 and e_h < 1e-12, (e_u, e_h)


def test_free_3d_read_out_inside_the_start_up_and_batch():
    """Read-outs after steps 2 and 5 of an 8-step run (inside and after the
    start-up of the 4th-order scheme), on instance 1 of a batch of two with
    different u0, V and A."""
    import torch
    shape, nu, q, n_r, order, startup = (32, 32, 32), (128, 128, 128), 10, 1, 4, 3
    insts = [_instance(shape, 10, seed=5 + 3 * i, A0=20.0 + 30.0 * i) for i in range(2)]
    H = min(_H(it, 1e-10) for it in insts)
    pr = _problem(insts, nu, H, q, n_r, order, startup, "fp64")
    got = {}
    for k, n in ((2, 2), (3, 5)):
        pr.step(k)
        torch.cuda.synchronize()
        got[n] = pr.read_u(1)
    pr.close()
    (_, kept), _ = _oracle(insts[1], nu, H, 5, q, n_r, order, startup, keep={2, 5})
    for n in (2, 5):
        e = rel(got[n], kept[n])
        print("3D free space, instance 1, step", n, e)
        assert e < 1e-12, (n, e)


def test_free_3d_mixed_matches_oracle():
    """FP32 transforms (H for FP32 contour sums) against the FP64 oracle on
    the same contour."""
    import torch
    shape, nu, q, n_r, order, n = (32, 64, 32), (128, 256, 128), 10, 1, 4, 7
    inst = _instance(shape, n + 2)
    H = _H(inst, 1e-4, eps_m=2.0 ** -23)
    pr = _problem([inst], nu, H, q, n_r, order, 3, "mixed")
    pr.step(n)
    torch.cuda.synchronize()
    u, uh = pr.read_u(0), pr.read_modes(0)
    pr.close()
    uo, uho = _oracle(inst, nu, H, n, q, n_r, order, 3)
    e_u, e_h = rel(u, uo), rel(uh, uho)
    print("3D free space mixed vs FP64 oracle", e_u, e_h)
    assert e_u < MIXED_TOL and e_h < MIXED_TOL, (e_u, e_h)


def test_free_3d_mixed_residual_check():
    """The FP64 residual check of the FP32-transform step runs in 3D (its
    re-evaluation goes through the FP64 3D passes); with tol = 0 every checked
    step is redone in FP64 and the result stays within the mixed bound."""
    import torch
    shape, nu, q, n_r, order, n = (32, 32, 32), (128, 128, 128), 10, 1, 4, 8
    inst = _instance(shape, n + 2, seed=9)
    H = _H(inst, 1e-4, eps_m=2.0 ** -23)
    pr = _problem([inst], nu, H, q, n_r, order, 3, "mixed")
    pr.set_residual_check(1, 0.0)
    pr.step(n)
    torch.cuda.synchronize()
    rho, corr, checks = pr.residual_report()
    u = pr.read_u(0)
    pr.close()
    assert checks == n - 3 and corr[0] == checks, (checks, corr)
    assert np.isfinite(rho[0]) and 0.0 < rho[0] < 1e-5, rho
    uo, _ = _oracle(inst, nu, H, n, q, n_r, order, 3)
    e = rel(u, uo)
    print("3D free space mixed with FP64 redo vs oracle", e, "rho", rho[0])
    assert e < MIXED_TOL, e
