"""General V(x, t) (potential tables, TDSE_V_TABLE) on the GPU through the
C ABI: the moving wells of Example 1 and drifting 2D / free-space wells
against the FP64 oracle with the same V(x, t); a table holding f(t) V0(x)
against the separable path (same bits); the Galilean closed form of the
moving well; tables in uneven batches and under the FP64 residual check.

Tolerances as for the separable potentials: FP64 1e-12 (periodic and free
space, relative L2), mixed 2e-6.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fields, gamma
from oracle.freespace import FreeSpaceOracle
from oracle.periodic import PeriodicOracle, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL, MIXED_TOL = 1e-12, 2e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _load(pr, insts, table):
    for b, it in enumerate(insts):
        if table:
            pr.set_potential_fn(it.V_at, instance=b)
        else:
            pr.set_potential(it.V0, it.vfac_table(), instance=b)
        if it.pulse is not None:
            p = it.pulse
            pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction, instance=b)
        pr.set_initial(it.u0, instance=b)


def gpu(inst, n, precision="fp64", table=True, batch_of=None, stream=None, **free):
    from paper_2001_06113_gb300 import Problem
    insts = batch_of or [inst]
    kw = dict(bc="free", **free) if free else {}
    pr = Problem(inst.shape, inst.dt, inst.nsteps, precision=precision, batch=len(insts), stream=stream,
                 potential="table" if table else "separable", **kw)
    _load(pr, insts, table)
    pr.step(n)
    return pr


def periodic_oracle(inst, n):
    orc = PeriodicOracle(inst.shape, inst.dt, inst.Vt or inst.V0, inst.vfac,
                         fields.phi_callable(inst.pulse, inst.dim))
    return orc.solve(inst.u0, n)


# ------------------------------------------------------------ periodic
@pytest.mark.parametrize("c", [15.0, 45.0])
def test_moving_well_1d_matches_oracle(c):
    """Example 1's well (V0 = 300, beta = 0.2) moving at speed c, M = 128."""
    inst = synth.moving_well_1d(c=c, M=128, nsteps=40, T=40 * 2e-3)
    n = 24
    uo = periodic_oracle(inst, n)
    assert rel_l2(gpu(inst, n).read_u(0), uo) < FP64_TOL
    assert rel_l2(gpu(inst, n, "mixed").read_u(0), uo) < MIXED_TOL


def test_moving_wells_2d_matches_oracle():
    inst = synth.moving_wells_2d(M=64, nsteps=16)
    n = 12
    uo = periodic_oracle(inst, n)
    assert rel_l2(gpu(inst, n).read_u(0), uo) < FP64_TOL
    assert rel_l2(gpu(inst, n, "mixed").read_u(0), uo) < MIXED_TOL


def test_galilean_closed_form_on_gpu():
    """The moving ground state carried exactly by the well (c / 2 integer):
    8th order in dt down to the spatial floor, as the oracle."""
    V0, beta, M, c, T = 50.0, 0.4, 64, 4.0, 0.2
    E, k, coef = synth.well_ground_state_coeffs(V0, beta)
    x = synth.periodic_grid(M)
    ref = (np.exp(1j * np.outer(x - c * T, k)) @ coef) * np.exp(-1j * E * T) * np.exp(1j * (c * x / 2 - c * c * T / 4))
    errs = []
    for n in (100, 200, 400):
        inst = synth.moving_well_1d(c=c, M=M, nsteps=n, T=T, V0=V0, beta=beta, u_shift=c / 2)
        errs.append(rel_l2(gpu(inst, n).read_u(0), ref))
    assert errs[1] < 1e-9 and errs[2] < 1e-10 and errs[0] / errs[1] > 100.0, errs


def test_galilean_closed_form_2d_on_gpu():
    """Two wells moving along x and y carry their boosted ground-state product
    (2D closed form): 8th order as on the oracle (3.8e-7, 1.6e-9)."""
    (V1, b1), (V2, b2), c, T, M = (40.0, 0.45), (60.0, 0.5), (4.0, -2.0), 0.2, 64
    E1, k1, c1 = synth.well_ground_state_coeffs(V1, b1)
    E2, k2, c2 = synth.well_ground_state_coeffs(V2, b2)
    x = synth.periodic_grid(M)
    X, Y = np.meshgrid(x, x, indexing="ij")
    ref = (np.outer(np.exp(1j * np.outer(x - c[0] * T, k1)) @ c1, np.exp(1j * np.outer(x - c[1] * T, k2)) @ c2)
           * np.exp(-1j * (E1 + E2) * T) * np.exp(1j * (0.5 * (c[0] * X + c[1] * Y) - 0.25 * (c[0] ** 2 + c[1] ** 2) * T)))
    errs = []
    for n in (100, 200):
        inst = synth.moving_separable_wells_2d(M=M, nsteps=n, T=T)
        errs.append(rel_l2(gpu(inst, n).read_u(0), ref))
    assert errs[1] < 1e-8 and errs[0] / errs[1] > 100.0, errs


@pytest.mark.parametrize("shape,precision", [((256,), "fp64"), ((64, 64), "fp64"), ((256,), "mixed"),
                                             ((64, 64), "mixed"), ((16384,), "mixed")])
def test_table_of_separable_potential_equals_separable_path(shape, precision):
    """A table whose rows are f(t_r) V0 gives the separable path's bits
    (FP64: f V0 rounds the same on host and device; mixed: f = 1)."""
    if len(shape) == 2:
        inst = synth.periodic_2d_wells(seed=5, M=shape[0], dt=1e-3, nsteps=20)
    else:
        inst = synth.periodic_1d_batch_member(3, dt=1e-3, nsteps=20, sizes=shape)
    from paper_2001_06113_gb300 import Problem
    if precision == "fp64":
        inst.vfac = lambda t: 1.0 + 0.4 * np.sin(30.0 * np.asarray(t, dtype=np.float64))
    pr = Problem(inst.shape, inst.dt, inst.nsteps, precision=precision, potential="table")
    f = inst.vfac_table()                                    # the separable path's samples f(m dt / 8)
    m = np.rint(pr.potential_times() * 8.0 / inst.dt).astype(int)
    pr.set_potential_table(f[m].reshape((-1,) + (1,) * inst.dim) * inst.V0[None])
    if inst.pulse is not None:
        p = inst.pulse
        pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
    pr.set_initial(inst.u0)
    pr.step(15)
    b = gpu(inst, 15, precision, table=False).read_u(0)
    assert np.array_equal(pr.read_u(0), b)


def test_table_batch_and_residual_check():
    """Moving wells in an uneven fused batch equal solo runs bit for bit; the
    FP64 residual check reads the table row of the checked step."""
    import torch
    from paper_2001_06113_gb300 import Batch, Problem
    insts = {N: [synth.moving_well_1d(c=15.0 + 10 * i, M=N, nsteps=30, T=30 * 1e-3, V0=100.0, beta=0.3)
                 for i in range(k)] for N, k in ((256, 3), (1024, 2))}
    stream = torch.cuda.Stream()
    probs = []
    for N, its in insts.items():
        pr = Problem((N,), 1e-3, 30, batch=len(its), precision="mixed", stream=stream, potential="table")
        _load(pr, its, True)
        probs.append(pr)
    Batch(probs, stream=stream).step(20)
    stream.synchronize()
    for pr, its in zip(probs, insts.values()):
        ub = pr.read_u()
        for b, it in enumerate(its):
            assert np.array_equal(gpu(it, 20, "mixed").read_u(0), ub[b])
    it = insts[256][0]
    pr = Problem((256,), 1e-3, 30, precision="mixed", potential="table")
    pr.set_residual_check(5, 1e-6)
    _load(pr, [it], True)
    pr.step(20)
    rho, corr, checks = pr.residual_report()
    assert checks >= 2 and float(np.max(rho)) < 1e-7 and int(np.sum(corr)) == 0
    assert np.array_equal(pr.read_u(0), gpu(it, 20, "mixed").read_u(0))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shared_table_equals_per_instance_tables(precision):
    """One table read by every instance (different u0 and pulses) gives the
    bits of per-instance copies of it."""
    from paper_2001_06113_gb300 import Problem, TdseError
    base = synth.moving_well_1d(c=30.0, M=256, nsteps=24, T=24 * 2e-3)
    insts = []
    for i, k0 in enumerate((0, 3, -5)):
        it = synth.moving_well_1d(c=30.0, M=256, nsteps=24, T=24 * 2e-3, u_shift=k0)
        if i == 2:
            it.pulse = synth.Pulse(2.0, 10.0, it.t_max, (1.0,))
        insts.append(it)
    shared = Problem((256,), base.dt, 24, batch=3, precision=precision, potential="shared_table")
    with pytest.raises(TdseError):
        shared.set_potential_fn(base.V_at, instance=1)
    shared.set_potential_fn(base.V_at)
    for b, it in enumerate(insts):
        if it.pulse is not None:
            shared.set_pulse(it.pulse.A0, it.pulse.omega, it.pulse.T_pulse, it.pulse.direction, instance=b)
        shared.set_initial(it.u0, instance=b)
    shared.step(20)
    per = gpu(base, 20, precision, batch_of=insts)
    assert np.array_equal(shared.read_u(), per.read_u())
    assert shared.workspace_bytes < per.workspace_bytes


def test_table_validation():
    from paper_2001_06113_gb300 import Problem, TdseError
    inst = synth.moving_well_1d(M=64, nsteps=10, T=0.01)
    sep = Problem((64,), inst.dt, 10)
    with pytest.raises(TdseError):
        sep.set_potential_table(np.zeros((5, 64)))
    tab = Problem((64,), inst.dt, 10, potential="table")
    with pytest.raises(TdseError):
        tab.set_potential(inst.V0)
    with pytest.raises(TdseError):
        tab.step(1)                                   # no V yet
    assert tab.potential_times().size == 8 * 7 + 1 + 3


# ------------------------------------------------------------ free space
def test_free_galilean_closed_form_on_gpu():
    """The deep well moving in free space carries its boosted ground state
    (closed form, any c): the GPU contour scheme converges at 8th order to it
    as the oracle does (oracle: 5.6e-7, 2.4e-9 at 400, 800 steps)."""
    from paper_2001_06113_gb300 import Problem
    M, V0, beta, x0, c, T = 256, 3000.0, 0.06, -0.1, 1.0, 0.02
    E, k, coef = synth.well_ground_state_coeffs(V0, beta, 320)
    x = synth.free_grid(M)
    ref = (np.exp(1j * np.outer(x - x0 - c * T, k)) @ coef) * np.exp(-1j * E * T) * np.exp(1j * (c * x / 2 - c * c * T / 4))
    H = gamma.choose_H(1e-12, V0 * math.sqrt(beta * math.sqrt(math.pi)), 0.0, 1)
    errs = []
    for n in (400, 800):
        inst = synth.free_moving_well(M=M, V0=V0, beta=beta, x0=x0, c=c, T=T, nsteps=n)
        pr = Problem((M,), inst.dt, n, bc="free", nu=(2048,), H=H, gauss_q=16, n_r=2, potential="table")
        pr.set_potential_fn(inst.V_at)
        pr.set_initial(inst.u0)
        pr.step(n)
        errs.append(rel_l2(pr.read_u(0), ref))
    assert errs[1] < 1e-8 and errs[0] / errs[1] > 100.0, errs



@pytest.mark.parametrize("shape,nu,precision,tol", [((64,), (512,), "fp64", FP64_TOL),
                                                     ((32, 32), (256, 256), "fp64", FP64_TOL),
                                                     ((64,), (512,), "mixed", MIXED_TOL)])
def test_free_moving_wells_match_oracle(shape, nu, precision, tol):
    inst = synth.free_moving_wells(shape, nsteps=14)
    n = 12
    phi = fields.phi_callable(inst.pulse, inst.dim)
    phimax = max(float(np.max(np.abs(phi(t)))) for t in np.linspace(0.0, inst.t_max, 201))
    vnorm = max(math.sqrt(float(np.sum(inst.V_at(t) ** 2)) * (2.0 / shape[0]) ** inst.dim)
                for t in np.linspace(0.0, inst.t_max, 5))
    eps = 1e-10 if precision == "fp64" else 1e-4
    H = gamma.choose_H(eps, vnorm, phimax, inst.dim, eps_m=gamma.EPS_M if precision == "fp64" else 2.0 ** -23)
    pr = gpu(inst, n, precision, nu=nu, H=H, gauss_q=10, n_r=1)
    rules = [gamma.GammaRule.for_nu(M, v, H, q=10, n_r=1) for M, v in zip(shape, nu)]
    orc = FreeSpaceOracle(rules, inst.dt, inst.Vt, None, phi)
    uo = orc.solve(inst.u0, n)
    assert rel_l2(pr.read_u(0), uo) < tol
