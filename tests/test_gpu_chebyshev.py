"""Free-space steps with the C-type transforms through Chebyshev
interpolants (Sec. 4.1, eqs. expintrpm / expintrpp) against the FP64 oracle,
which evaluates them as direct sums (eq. fhatCsum).

With dyadic refinement n_r = 3, 4 the Gauss block has N^C = 60, 80 modes and
the interpolant N_T = 20 terms (the library picks it so that it reproduces
e^{-+i zeta x} to FP64 rounding at the C nodes), so TDSE_CT_AUTO takes the
interpolant.  Tolerances as for the other free-space tests: FP64 1e-12 on
the grid and on the contour, FP32 transforms 2e-6.
"""
import math

import numpy as np
import pytest

import synth
from oracle import fields, gamma
from oracle.freespace import FreeSpaceOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def rel(a, b):
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def _instance(shape, n, seed=11, dt=1e-3):
    d = len(shape)
    return synth.free_bump_gaussians(shape, seed=seed, dt=dt, nsteps=n, A0=50.0, omega=200.0,
                                     direction=(1.0, -0.5)[:d])


def _H(inst, eps, eps_m=gamma.EPS_M):
    phi = fields.phi_callable(inst.pulse, inst.dim)
    phimax = max(float(np.max(np.abs(phi(t)))) for t in np.linspace(0.0, inst.t_max, 401))
    vnorm = math.sqrt(float(np.sum(inst.V0 ** 2)) * (2.0 / inst.shape[0]) ** inst.dim)
    return gamma.choose_H(eps, vnorm, phimax, inst.dim, eps_m=eps_m)


def _gpu(inst, nu, H, n, n_r, c_transform, precision="fp64"):
    from paper_2001_06113_gb300 import Problem
    pr = Problem(inst.shape, inst.dt, inst.nsteps, bc="free", nu=nu, H=H, gauss_q=10, n_r=n_r,
                 precision=precision, c_transform=c_transform)
    nts = [pr.cheb_terms(a) for a in range(inst.dim)]
    pr.set_potential(inst.V0)
    p = inst.pulse
    pr.set_pulse(p.A0, p.omega, p.T_pulse, p.direction)
    pr.set_initial(inst.u0)
    pr.step(n)
    u, uh = pr.read_u(0), pr.read_modes(0)
    pr.close()
    return u, uh, nts


def _oracle(inst, nu, H, n, n_r):
    rules = [gamma.GammaRule.for_nu(M, v, H, q=10, n_r=n_r) for M, v in zip(inst.shape, nu)]
    orc = FreeSpaceOracle(rules, inst.dt, inst.V0, inst.vfac, fields.phi_callable(inst.pulse, inst.dim))
    u = orc.solve(inst.u0, n)
    return u, orc.last_uhat


@pytest.mark.parametrize("shape,nu,n_r", [((128,), (512,), 3), ((256,), (1024,), 4), ((64, 32), (256, 256), 3)])
def test_chebyshev_ctype_matches_oracle(shape, nu, n_r):
    inst = _instance(shape, 12)
    H = _H(inst, 1e-10)
    u, uh, nts = _gpu(inst, nu, H, 12, n_r, "auto")
    assert all(0 < t < 10 * 2 * n_r for t in nts), nts          # the interpolant was chosen (N_T < N^C)
    uo, uho = _oracle(inst, nu, H, 12, n_r)
    e_u, e_h = rel(u, uo), rel(uh.reshape(uho.shape), uho)
    print(shape, n_r, "N_T", nts, "u", e_u, "u^", e_h)
    assert e_u <= 1e-12 and e_h <= 1e-12, (e_u, e_h)


def test_chebyshev_equals_direct_on_the_gpu():
    inst = _instance((128,), 10, seed=5)
    H = _H(inst, 1e-10)
    u_c, uh_c, nt_c = _gpu(inst, (512,), H, 10, 4, "chebyshev")
    u_d, uh_d, nt_d = _gpu(inst, (512,), H, 10, 4, "direct")
    assert nt_c[0] > 0 and nt_d[0] == 0
    assert rel(u_c, u_d) <= 1e-12 and rel(uh_c, uh_d) <= 1e-12


def test_chebyshev_fp32_transforms():
    inst = _instance((128,), 12, seed=9)
    H = _H(inst, 1e-4, eps_m=2.0 ** -23)
    u, uh, nts = _gpu(inst, (512,), H, 12, 3, "chebyshev", precision="mixed")
    uo, uho = _oracle(inst, (512,), H, 12, 3)
    e = rel(u, uo)
    print("FP32 transforms with the interpolant", nts, e)
    assert nts[0] > 0 and e <= 2e-6, e
