"""GPU parity of the free-space path (Sec. 3-4, Remark highorderfs) against
the FP64 oracle, through the C ABI.

Both sides march the same seeded problem with the same contour parameters
(H, nu, p, q, n_r).  The worst-case bound on the difference is eps, the
precision H was chosen for (Remark Hchoice): the transform pair amplifies
rounding by e^{2 d H (1 + phi_max)} (1 + ||V||), which H makes equal to
eps / eps_m, and the two sides round differently (FFT-based versus direct
sums).  The observed differences are 2e-15..3e-14 in relative L2, so the
tests hold both u on the grid and the mode state u^ on the contour to
1e-12, the FP64 bar of the periodic path.

The FP32-transform variant (precision "mixed": transforms, ring and
history sum in FP32, mode state and update in FP64) takes H from the same
remark with eps_m = 2^-23.  Against the FP64 oracle on the same contour the
bound is again that eps; the observed differences are 1.5e-7..2.4e-7 on the
grid and 4e-8..9e-8 on the contour (a few FP32 unit roundoffs, 2^-24 =
6e-8), independent of eps in 1e-5..1e-3, so these tests hold 2e-6 on both,
the mixed bar of the periodic path.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fields, gamma
from oracle.freespace import FreeSpaceOracle

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def _instance(shape, n, seed=11, dt=1e-3, A0=50.0, omega=200.0):
    d = len(shape)
    return synth.free_bump_gaussians(shape, seed=seed, dt=dt, nsteps=n, A0=A0, omega=omega,
                                     direction=(1.0, -0.5)[:d],
                                     vfac=lambda t: 1.0 + 0.3 * np.sin(40.0 * np.asarray(t, dtype=np.float64)))


MIXED_TOL = 2e-6
EPS_M32 = 2.0 ** -23


def _H(inst, eps, eps_m=gamma.EPS_M):
    phi = fields.phi_callable(inst.pulse, inst.dim)
    phimax = max(float(np.max(np.abs(phi(t)))) for t in np.linspace(0.0, inst.t_max, 401))
    vnorm = math.sqrt(float(np.sum(inst.V0 ** 2)) * (2.0 / inst.shape[0]) ** inst.dim)
    vnorm *= float(np.max(np.abs(inst.vfac_table())))
    return gamma.choose_H(eps, vnorm, phimax, inst.dim, eps_m=eps_m)


def _gpu(inst, nu, H, n, q=10, n_r=1, p=8, order=8, startup=-1, precision="fp64"):
    import torch
    from paper_2001_06113_gb300 import Problem
    pr = Problem(inst.shape, inst.dt, inst.nsteps, order=order, startup_steps=startup, bc="free", nu=nu, H=H,
                 gauss_q=q, n_r=n_r, alpert_p=p, precision=precision)
    pr.set_potential(inst.V0, inst.vfac_table())
    if inst.pulse is not None:
        pr.set_pulse(inst.pulse.A0, inst.pulse.omega, inst.pulse.T_pulse, inst.pulse.direction)
    pr.set_initial(inst.u0)
    pr.step(n)
    torch.cuda.synchronize()
    return pr.read_u(0), pr.read_modes(0), pr


def _oracle(inst, nu, H, n, q=10, n_r=1, p=8, order=8, startup=None):
    rules = [gamma.GammaRule.for_nu(M, v, H, p=p, q=q, n_r=n_r) for M, v in zip(inst.shape, nu)]
    phi = fields.phi_callable(inst.pulse, inst.dim)
    orc = FreeSpaceOracle(rules, inst.dt, inst.V0, inst.vfac, phi, order=order, n_startup=startup)
    u = orc.solve(inst.u0, n)
    return u, orc.last_uhat


CASES_1D = [
    # shape, nu, q, n_r, p, order, steps, eps
    ((64,), (512,), 10, 1, 8, 8, 12, 1e-10),
    ((32,), (512,), 8, 0, 4, 4, 9, 1e-10),
    ((128,), (512,), 12, 2, 8, 6, 10, 1e-11),
    ((256,), (1024,), 10, 1, 8, 8, 9, 1e-10),
    ((512,), (2048,), 10, 1, 8, 8, 9, 1e-10),
]


@pytest.mark.parametrize("shape,nu,q,n_r,p,order,n,eps", CASES_1D)
def test_free_1d_matches_oracle(shape, nu, q, n_r, p, order, n, eps):
    inst = _instance(shape, n + 2)
    H = _H(inst, eps)
    u, uh, _ = _gpu(inst, nu, H, n, q, n_r, p, order)
    uo, uho = _oracle(inst, nu, H, n, q, n_r, p, order)
    assert rel(u, uo) < 1e-12 and rel(uh, uho) < 1e-12, (rel(u, uo), rel(uh, uho))


CASES_2D = [
    ((64, 32), (512, 256), 10, 1, 8, 8, 10, 1e-10),
    ((32, 64), (256, 1024), 8, 2, 8, 8, 9, 1e-10),
    ((32, 32), (128, 512), 6, 0, 4, 4, 7, 1e-9),
]


@pytest.mark.parametrize("shape,nu,q,n_r,p,order,n,eps", CASES_2D)
def test_free_2d_matches_oracle(shape, nu, q, n_r, p, order, n, eps):
    inst = _instance(shape, n + 2)
    H = _H(inst, eps)
    u, uh, _ = _gpu(inst, nu, H, n, q, n_r, p, order)
    uo, uho = _oracle(inst, nu, H, n, q, n_r, p, order)
    assert rel(u, uo) < 1e-12 and rel(uh, uho) < 1e-12, (rel(u, uo), rel(uh, uho))


def test_free_2d_full_size_matches_oracle():
    """The 256^2 free-space workload (nu = 2048, q = 10, n_r = 1, eps = 1e-10)
    through the start-up and the first Adams step, in the launch sequence the
    benchmark times."""
    inst = synth.free_bump_gaussians((256, 256), seed=3, dt=5e-4, nsteps=2000, T_pulse=1.0)
    n = 8
    H = _H(inst, 1e-10)
    u, uh, _ = _gpu(inst, (2048, 2048), H, n)
    uo, uho = _oracle(inst, (2048, 2048), H, n)
    assert rel(u, uo) < 1e-12 and rel(uh, uho) < 1e-12, (rel(u, uo), rel(uh, uho))


def _wavepacket(x, t, sigma, phi=0.0):
    a = sigma ** 2 + 2j * t
    return (math.pi * sigma ** 2) ** -0.25 * sigma / np.sqrt(a) * np.exp(-(x + phi) ** 2 / (2 * a))


@pytest.mark.parametrize("A0", [0.0, 3.0])
def test_free_wavepacket_1d_closed_form(A0):
    """V = 0: the scheme has no time error (Sec. 7 Example 2); the GPU solution
    matches the closed form to the quadrature accuracy at every step."""
    M, sigma, dt, n = 64, 0.1, 0.01, 10
    pulse = synth.Pulse(A0, 20.0, 0.1, (1.0,)) if A0 else None
    phi = fields.phi_callable(pulse, 1)
    phimax = max(abs(phi(t)[0]) for t in np.linspace(0, 0.1, 101))
    H = gamma.choose_H(1e-12, 0.0, phimax, 1)
    x = synth.free_grid(M)
    from paper_2001_06113_gb300 import Problem
    pr = Problem((M,), dt, n, bc="free", nu=(512,), H=H, gauss_q=16, n_r=2)
    pr.set_potential(np.zeros(M))
    if pulse:
        pr.set_pulse(A0, 20.0, 0.1, (1.0,))
    pr.set_initial(_wavepacket(x, 0.0, sigma))
    for k in range(1, n + 1):
        pr.step(1)
        u = pr.read_u(0)
        ref = _wavepacket(x, k * dt, sigma, phi(k * dt)[0])
        err = math.sqrt(np.sum(np.abs(u - ref) ** 2) * 2 / M)
        assert err < 1e-12, (k, err)


def test_free_wavepacket_2d_closed_form():
    """2D, A = (A1, A2): u = u_1(x, t) u_2(y, t)."""
    M, dt, n = (64, 64), 0.01, 6
    s1, s2 = 0.1, 0.12
    pulse = synth.Pulse(2.0, 20.0, 0.06, (1.0, -0.5))
    phi = fields.phi_callable(pulse, 2)
    H = gamma.choose_H(1e-12, 0.0, 0.1, 2)
    x = synth.free_grid(M[0])
    y = synth.free_grid(M[1])
    u0 = np.outer(_wavepacket(x, 0.0, s1), _wavepacket(y, 0.0, s2))
    from paper_2001_06113_gb300 import Problem
    pr = Problem(M, dt, n, bc="free", nu=(512, 512), H=H, gauss_q=16, n_r=2)
    pr.set_potential(np.zeros(M))
    pr.set_pulse(2.0, 20.0, 0.06, (1.0, -0.5))
    pr.set_initial(u0)
    pr.step(n)
    u = pr.read_u(0)
    T = n * dt
    ph = phi(T)
    ref = np.outer(_wavepacket(x, T, s1, ph[0]), _wavepacket(y, T, s2, ph[1]))
    assert rel(u, ref) < 1e-11


def test_free_batch_members_equal_solo_runs():
    """Instances in one batch (different u0, V, A) give bit-identical results
    to the same instances run alone."""
    import torch
    from paper_2001_06113_gb300 import Problem
    shape, nu, n = (64, 32), (512, 256), 9
    insts = [_instance(shape, n + 2, seed=20 + i, A0=20.0 * i) for i in range(3)]
    H = 2.5

    def setup(pr, i, inst):
        pr.set_potential(inst.V0, inst.vfac_table(), instance=i)
        if inst.pulse is not None:
            pr.set_pulse(inst.pulse.A0, inst.pulse.omega, inst.pulse.T_pulse, inst.pulse.direction, instance=i)
        pr.set_initial(inst.u0, instance=i)

    pb = Problem(shape, insts[0].dt, n + 2, batch=3, bc="free", nu=nu, H=H)
    for i, inst in enumerate(insts):
        setup(pb, i, inst)
    pb.step(n)
    torch.cuda.synchronize()
    ub = pb.read_u()
    mb = pb.read_modes()
    for i, inst in enumerate(insts):
        ps = Problem(shape, inst.dt, n + 2, bc="free", nu=nu, H=H)
        setup(ps, 0, inst)
        ps.step(n)
        assert np.array_equal(ps.read_u(0), ub[i])
        assert np.array_equal(ps.read_modes(0), mb[i])


def test_free_read_u_before_and_across_calls():
    """u0 is readable before stepping; k calls of step(1) equal one step(k)."""
    from paper_2001_06113_gb300 import Problem, TdseError
    inst = _instance((32, 32), 12)
    H = 2.0
    pr = Problem((32, 32), inst.dt, 12, bc="free", nu=(256, 256), H=H)
    pr.set_potential(inst.V0, inst.vfac_table())
    pr.set_pulse(inst.pulse.A0, inst.pulse.omega, inst.pulse.T_pulse, inst.pulse.direction)
    pr.set_initial(inst.u0)
    assert np.array_equal(pr.read_u(0), inst.u0)
    with pytest.raises(TdseError):
        pr.read_modes(0)
    for _ in range(10):
        pr.step(1)
    pr.check_finite()
    q = Problem((32, 32), inst.dt, 12, bc="free", nu=(256, 256), H=H)
    q.set_potential(inst.V0, inst.vfac_table())
    q.set_pulse(inst.pulse.A0, inst.pulse.omega, inst.pulse.T_pulse, inst.pulse.direction)
    q.set_initial(inst.u0)
    q.solve_to(10 * inst.dt)
    assert q.step_index == 10
    assert np.array_equal(pr.read_u(0), q.read_u(0))
    assert np.array_equal(pr.read_modes(0), q.read_modes(0))


# ------------------------------------------------------------ FP32 transforms
MIXED_CASES = [
    # shape, nu, q, n_r, p, order, steps, eps (H for FP32 sums)
    ((64,), (512,), 10, 1, 8, 8, 12, 1e-4),
    ((256,), (1024,), 10, 1, 8, 8, 30, 1e-5),
    ((128,), (512,), 8, 0, 4, 6, 10, 1e-3),
    ((64, 64), (512, 512), 10, 1, 8, 8, 12, 1e-4),
    ((32, 64), (256, 1024), 8, 2, 8, 8, 9, 1e-4),
]


@pytest.mark.parametrize("shape,nu,q,n_r,p,order,n,eps", MIXED_CASES)
def test_free_mixed_matches_oracle(shape, nu, q, n_r, p, order, n, eps):
    """FP32 transforms and history, FP64 state: u and u^ within the mixed
    bar of the FP64 oracle on the same contour (H for eps_m = 2^-23)."""
    inst = _instance(shape, n + 2)
    H = _H(inst, eps, EPS_M32)
    u, uh, pr = _gpu(inst, nu, H, n, q, n_r, p, order, precision="mixed")
    pr.check_finite()
    uo, uho = _oracle(inst, nu, H, n, q, n_r, p, order)
    assert rel(u, uo) < MIXED_TOL and rel(uh, uho) < MIXED_TOL, (rel(u, uo), rel(uh, uho))


def test_free_mixed_full_size_against_fp64_path():
    """The 256^2 workload (nu = 2048) in the FP32-transform variant against
    the FP64 path (oracle-checked above) on the same contour, through the
    start-up and 32 Adams steps."""
    inst = synth.free_bump_gaussians((256, 256), seed=3, dt=5e-4, nsteps=2000, T_pulse=1.0)
    n = 40
    H = _H(inst, 1e-4, EPS_M32)
    um, mm, _ = _gpu(inst, (2048, 2048), H, n, precision="mixed")
    ud, md, _ = _gpu(inst, (2048, 2048), H, n)
    assert rel(um, ud) < MIXED_TOL and rel(mm, md) < MIXED_TOL, (rel(um, ud), rel(mm, md))


def test_free_mixed_wavepacket_closed_form():
    """V = 0 with a pulse: no time error, so the mixed variant matches the
    closed form to its rounding level on the FP32 contour."""
    M, sigma, dt, n = 128, 0.1, 0.01, 10
    pulse = synth.Pulse(3.0, 20.0, 0.1, (1.0,))
    phi = fields.phi_callable(pulse, 1)
    phimax = max(abs(phi(t)[0]) for t in np.linspace(0, 0.1, 101))
    H = gamma.choose_H(1e-4, 0.0, phimax, 1, eps_m=EPS_M32)
    x = synth.free_grid(M)
    from paper_2001_06113_gb300 import Problem
    pr = Problem((M,), dt, n, bc="free", nu=(1024,), H=H, gauss_q=16, n_r=2, precision="mixed")
    pr.set_potential(np.zeros(M))
    pr.set_pulse(3.0, 20.0, 0.1, (1.0,))
    pr.set_initial(_wavepacket(x, 0.0, sigma))
    pr.step(n)
    ref = _wavepacket(x, n * dt, sigma, phi(n * dt)[0])
    assert rel(pr.read_u(0), ref) < MIXED_TOL


def test_free_mixed_batch_and_checkpoint():
    """Batched instances equal solo runs bit for bit; a checkpoint taken
    mid-run restores the exact continuation."""
    import torch
    from paper_2001_06113_gb300 import Problem
    shape, nu, n = (64, 32), (512, 256), 12
    insts = [_instance(shape, n + 2, seed=40 + i, A0=20.0 * (i + 1)) for i in range(2)]
    H = 1.2

    def make(B):
        return Problem(shape, insts[0].dt, n + 2, batch=B, bc="free", nu=nu, H=H, precision="mixed")

    def setup(pr, i, inst):
        pr.set_potential(inst.V0, inst.vfac_table(), instance=i)
        pr.set_pulse(inst.pulse.A0, inst.pulse.omega, inst.pulse.T_pulse, inst.pulse.direction, instance=i)
        pr.set_initial(inst.u0, instance=i)

    pb = make(2)
    for i, inst in enumerate(insts):
        setup(pb, i, inst)
    pb.step(5)
    blob = pb.save()
    pb.step(n - 5)
    torch.cuda.synchronize()
    ub = pb.read_u()
    for i, inst in enumerate(insts):
        ps = make(1)
        setup(ps, 0, inst)
        ps.step(n)
        assert np.array_equal(ps.read_u(0), ub[i])
    pc = make(2)
    for i, inst in enumerate(insts):
        setup(pc, i, inst)
    pc.load(blob)
    assert pc.step_index == 5
    pc.step(n - 5)
    assert np.array_equal(pc.read_u(), ub)


@pytest.mark.parametrize("shape,nu", [((64,), (512,)), ((32, 32), (256, 256))])
def test_free_mixed_residual_check(shape, nu):
    """FP64 residual of the FP32-transform step: small and reported; with no
    redo the results keep their bits; a redo of every checked step (tol = 0)
    stays within the mixed bar of the FP64 oracle."""
    n = 14
    inst = _instance(shape, n + 2)
    H = _H(inst, 1e-4, EPS_M32)

    def run(every, tol):
        from paper_2001_06113_gb300 import Problem
        pr = Problem(inst.shape, inst.dt, inst.nsteps, bc="free", nu=nu, H=H, gauss_q=10, n_r=1, precision="mixed")
        if every:
            pr.set_residual_check(every, tol)
        pr.set_potential(inst.V0, inst.vfac_table())
        pr.set_pulse(inst.pulse.A0, inst.pulse.omega, inst.pulse.T_pulse, inst.pulse.direction)
        pr.set_initial(inst.u0)
        pr.step(n)
        out = (pr.read_u(0), pr.read_modes(0), pr.residual_report())
        pr.close()
        return out

    u0, m0, _ = run(0, 0.0)
    u1, m1, (rho, corr, checks) = run(3, 1e-3)
    assert checks == 2 and int(np.sum(corr)) == 0           # steps 9 and 12 (Adams steps 8..14)
    assert 0.0 < float(np.max(rho)) < 1e-6
    assert np.array_equal(u0, u1) and np.array_equal(m0, m1)
    u2, m2, (rho2, corr2, checks2) = run(3, 0.0)
    assert checks2 == 2 and int(np.min(corr2)) == 2
    uo, uho = _oracle(inst, nu, H, n)
    assert rel(u2, uo) < MIXED_TOL and rel(m2, uho) < MIXED_TOL, (rel(u2, uo), rel(m2, uho))
