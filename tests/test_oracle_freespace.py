"""Pins for the free-space oracle (Sec. 3-4): Alpert corrections from their
defining moment conditions, the contour rule against closed-form integrals,
the transform pair, the Gaussian wavepacket closed form with and without a
vector potential (1D and 2D), and a cross-check against the pinned periodic
oracle for a problem whose solution stays inside the box.  No GPU."""
import math

import numpy as np
import pytest
from scipy.special import erf

import synth
from oracle import fields, freespace, gamma
from oracle.periodic import PeriodicOracle


def wavepacket(x, t, sigma, phi=0.0):
    """Solution of i u_t = -u_xx with u(x,0) = (pi sigma^2)^(-1/4) exp(-x^2/(2 sigma^2)),
    shifted by phi(t) for the advected equation (Green's function eq. gfun).
    Derived directly (the printed prefactor is garbled: reading C6)."""
    a = sigma ** 2 + 2j * t
    return (math.pi * sigma ** 2) ** -0.25 * sigma / np.sqrt(a) * np.exp(-(x + phi) ** 2 / (2 * a))


# ------------------------------------------------------------------ Alpert
def test_alpert_p1_by_hand():
    """p = 1, kappa = 1: w = 1/2, x = 1/6 from the two moment conditions."""
    x, w = gamma.alpert_rule(1, 1)
    assert abs(x[0] - 1.0 / 6.0) < 1e-15 and abs(w[0] - 0.5) < 1e-15


@pytest.mark.parametrize("p,kappa", [(2, 2), (4, 4), (8, 7)])
def test_alpert_moments_and_shape(p, kappa):
    x, w = gamma.alpert_rule(p, kappa)
    assert gamma.alpert_residuals(p, kappa) < 1e-13
    assert all(0.0 < xi < kappa for xi in x)
    assert all(wi > 0 for wi in w)


@pytest.mark.parametrize("p,kappa,hs,rate_min", [(4, 4, (0.4, 0.2), 7.0), (8, 7, (1.0, 0.5), 14.0)])
def test_alpert_order(p, kappa, hs, rate_min):
    """int_0^inf e^{-x}(2 + sin 3x) dx = 2 + 3/10 with the corrected one-sided
    trapezoid rule: error O(h^{2p})."""
    x, w = gamma.alpert_rule(p, kappa)
    exact = 2.0 + 3.0 / 10.0
    f = lambda s: np.exp(-s) * (2.0 + np.sin(3.0 * s))
    errs = []
    for h in hs:
        reg = h * np.sum(f(h * (kappa + np.arange(int(60 / h)))))
        cor = h * np.sum(np.array(w) * f(h * np.array(x)))
        errs.append(abs(reg + cor - exact))
    assert errs[1] > 0
    rate = math.log2(errs[0] / errs[1])
    assert rate > rate_min, (errs, rate)


# ------------------------------------------------------------------ Gamma rule
def test_clustered_panels_integrate_polynomials():
    """Gamma_2 rule is exact for zeta^m, m < 2q: int = zeta^{m+1}/(m+1) between
    (1-i)(-H) and (1-i)H."""
    r = gamma.GammaRule(32, 3.0, 40, q=6, n_r=3)
    z, w = r.blocks["C"]
    a, b = (1 - 1j) * (-3.0), (1 - 1j) * 3.0
    for m in range(12):
        exact = (b ** (m + 1) - a ** (m + 1)) / (m + 1)
        scale = abs(b) ** (m + 1) / (m + 1)
        assert abs(np.sum(w * z ** m) - exact) < 1e-13 * scale, m


@pytest.mark.parametrize("a", [0.02, 0.005])
def test_whole_contour_gaussian(a):
    """int_Gamma e^{-a zeta^2} d zeta = sqrt(pi / a) (the contour deforms to the
    real line); slowly decaying a puts weight on all five node blocks."""
    r = gamma.GammaRule.for_nu(64, 512, 2.5, p=8, q=16, n_r=2)
    assert r.K * r.K * a > 40          # truncation negligible
    val = np.sum(r.w * np.exp(-a * r.zeta ** 2))
    assert abs(val - math.sqrt(math.pi / a)) < 1e-12 * math.sqrt(math.pi / a)


def test_transform_round_trip():
    """(1/2pi) int_Gamma e^{i zeta x} f^(zeta) d zeta = f(x) on [-1,1] for f
    compactly supported (Lemma uentire): pins 2/M and w/2pi (reading C5)."""
    M = 64
    r = gamma.GammaRule.for_nu(M, 512, gamma.choose_H(1e-13, 0.0, 0.0, 1), q=16, n_r=2)
    orc = freespace.FreeSpaceOracle([r], 0.1, np.zeros(M), lambda t: 1.0, lambda t: np.zeros(1))
    x = freespace.free_grid(M)
    f = wavepacket(x, 0.0, 0.12) * np.exp(2j * x)
    assert np.max(np.abs(orc.inv(orc.fwd(f)) - f)) < 1e-13


# ------------------------------------------------------------------ wavepacket
@pytest.mark.parametrize("A0", [0.0, 3.0])
def test_wavepacket_1d(A0):
    """V = 0: no time error (Example 2); quadrature/truncation error only."""
    M, sigma, dt, n = 64, 0.1, 0.01, 10
    pulse = synth.Pulse(A0, 20.0, 0.1, (1.0,)) if A0 else None
    phi = fields.phi_callable(pulse, 1)
    phimax = max(abs(phi(t)[0]) for t in np.linspace(0, 0.1, 101))
    r = gamma.GammaRule.for_nu(M, 512, gamma.choose_H(1e-12, 0.0, phimax, 1), q=16, n_r=2)
    orc = freespace.FreeSpaceOracle([r], dt, np.zeros(M), lambda t: 1.0, phi)
    x = freespace.free_grid(M)
    _, kept = orc.solve(wavepacket(x, 0.0, sigma), n, keep=set(range(1, n + 1)))
    err = max(np.sqrt(np.sum(np.abs(kept[k] - wavepacket(x, k * dt, sigma, phi(k * dt)[0])) ** 2) * 2 / M)
              for k in kept)
    assert err < 1e-12, err


def test_wavepacket_2d_product_with_field():
    """2D, A = (A1, A2): u = u_1(x,t) u_2(y,t) (tensor-product contour rule)."""
    M, dt, n = (64, 48), 0.01, 6
    pulse = synth.Pulse(2.0, 20.0, 0.06, (1.0, -0.5))
    phi = fields.phi_callable(pulse, 2)
    rules = [gamma.GammaRule.for_nu(m, 512, gamma.choose_H(1e-12, 0.0, 0.1, 2), q=16, n_r=2) for m in M]
    orc = freespace.FreeSpaceOracle(rules, dt, np.zeros(M), lambda t: 1.0, phi)
    x, y = freespace.free_grid(M[0]), freespace.free_grid(M[1])
    s1, s2 = 0.1, 0.12              # numerically supported in [-1,1] (e^{-35} at the edge)
    u0 = np.outer(wavepacket(x, 0.0, s1), wavepacket(y, 0.0, s2))
    u = orc.solve(u0, n)
    T = n * dt
    ph = phi(T)
    ref = np.outer(wavepacket(x, T, s1, ph[0]), wavepacket(y, T, s2, ph[1]))
    assert np.sqrt(np.sum(np.abs(u - ref) ** 2) / np.sum(np.abs(ref) ** 2)) < 1e-11


def test_3d_tensor_product_of_1d_solves():
    """d = 3, V = 0, pulse along (1, -0.5, 0.3): modes, phases and transforms
    are tensor products, so the 3D solve equals the outer product of three 1D
    solves (each pinned by the 1D wavepacket closed form) to rounding; uneven
    M per axis catches any mix-up of the axes."""
    M, dt, n = (16, 20, 16), 0.005, 9
    dirn = (1.0, -0.5, 0.3)
    rules = [gamma.GammaRule.for_nu(m, 4 * m, 1.5, q=10, n_r=1) for m in M]
    g = [freespace.free_grid(m) for m in M]
    f = [wavepacket(gg, 0.0, ss) * np.exp(1j * k * gg) for gg, ss, k in zip(g, (0.16, 0.14, 0.15), (2.0, -1.0, 0.5))]
    phi3 = fields.phi_callable(synth.Pulse(2.0, 20.0, 0.05, dirn), 3)
    u3 = freespace.FreeSpaceOracle(rules, dt, np.zeros(M), lambda t: 1.0, phi3).solve(np.einsum("i,j,k->ijk", *f), n)
    parts = [freespace.FreeSpaceOracle([rules[a]], dt, np.zeros(M[a]), lambda t: 1.0,
                                       fields.phi_callable(synth.Pulse(2.0 * dirn[a], 20.0, 0.05, (1.0,)), 1)).solve(f[a], n)
             for a in range(3)]
    ref = np.einsum("i,j,k->ijk", *parts)
    assert np.sqrt(np.sum(np.abs(u3 - ref) ** 2) / np.sum(np.abs(ref) ** 2)) < 1e-13


# ------------------------------------------------------- against the periodic oracle
def test_matches_periodic_solution_inside_box():
    """V != 0 and A != 0: while the solution stays far from the box edges the
    free-space and periodic schemes solve the same PDE; compare on [-1,1]
    (the periodic solution evaluated there by its Fourier series)."""
    M, dt, n = 64, 2e-3, 25
    sigma, k0 = 0.15, 4.0
    window = lambda z: np.where(np.abs(z) < 0.9, np.exp(1.0 - 1.0 / np.maximum(1e-300, 1.0 - (z / 0.9) ** 2)), 0.0)
    Vf = lambda z: -12.0 * np.exp(-z ** 2 / (2 * 0.2 ** 2)) * window(z)
    u0f = lambda z: wavepacket(z, 0.0, sigma) * np.exp(1j * k0 * z)
    vfac = lambda t: 1.0 + 0.4 * np.sin(8.0 * t)
    pulse = synth.Pulse(2.0, 15.0, n * dt, (1.0,))
    phi = fields.phi_callable(pulse, 1)
    x = freespace.free_grid(M)
    r = gamma.GammaRule.for_nu(M, 512, gamma.choose_H(1e-12, 12.0 * math.sqrt(0.5), 0.05, 1), q=16, n_r=2)
    u_free = freespace.FreeSpaceOracle([r], dt, Vf(x), vfac, phi).solve(u0f(x), n)
    Mp = 512
    xp = -math.pi + 2 * math.pi * np.arange(Mp) / Mp
    up = PeriodicOracle((Mp,), dt, Vf(xp), vfac, phi).solve(u0f(xp), n)
    coef = np.fft.fft(up) / Mp
    k = np.fft.fftfreq(Mp, 1.0 / Mp)
    u_per = np.exp(1j * np.outer(x + math.pi, k)) @ coef
    assert np.sqrt(np.sum(np.abs(u_free - u_per) ** 2) / np.sum(np.abs(u_per) ** 2)) < 1e-9


# ------------------------------------------------------- planted mistakes
@pytest.mark.parametrize("mistake", ["no_1mi", "gamma1_sign", "no_2overM"])
def test_planted_mistakes_fail(monkeypatch, mistake):
    if mistake == "no_1mi":
        orig = gamma.GammaRule.__init__

        def bad(self, *a, **k):
            orig(self, *a, **k)
            z, w = self.blocks["C"]
            nc = z.size
            i0 = self.NE + self.p
            self.w = self.w.copy()
            self.w[i0:i0 + nc] = self.w[i0:i0 + nc] / (1 - 1j)
        monkeypatch.setattr(gamma.GammaRule, "__init__", bad)
    elif mistake == "gamma1_sign":
        orig = gamma.GammaRule.__init__

        def bad(self, *a, **k):
            orig(self, *a, **k)
            self.zeta = self.zeta.copy()
            self.zeta[:self.NE] = np.conj(self.zeta[:self.NE])
        monkeypatch.setattr(gamma.GammaRule, "__init__", bad)
    elif mistake == "no_2overM":
        orig = freespace.FreeSpaceOracle.__init__

        def bad(self, *a, **k):
            orig(self, *a, **k)
            self.F = [F * (F.shape[1] / 2.0) for F in self.F]
        monkeypatch.setattr(freespace.FreeSpaceOracle, "__init__", bad)
    failed = False
    for fn in (lambda: test_whole_contour_gaussian(0.005), test_transform_round_trip):
        try:
            fn()
        except AssertionError:
            failed = True
    assert failed


# ------------------------------------------------ general V(x, t): moving well
def _free_galilean_errors(steps, M=256, nu=2048, V0=3000.0, beta=0.06, x0=-0.1, c=1.0, T=0.02):
    """Galilean invariance in free space: the ground state w0 of a static well
    carried by the well moving at speed c is u(x, t) = w0(x - x0 - c t)
    e^{-i E t} e^{i (c x / 2 - c^2 t / 4)} (any c).  A closed form for a
    non-separable V(x, t) on the contour scheme."""
    from oracle.periodic import rel_l2
    E, k, coef = synth.well_ground_state_coeffs(V0, beta, 320)
    x = synth.free_grid(M)
    ref = (np.exp(1j * np.outer(x - x0 - c * T, k)) @ coef) * np.exp(-1j * E * T) * np.exp(1j * (c * x / 2 - c * c * T / 4))
    vnorm = V0 * math.sqrt(beta * math.sqrt(math.pi))
    rule = gamma.GammaRule.for_nu(M, nu, gamma.choose_H(1e-12, vnorm, 0.0, 1), q=16, n_r=2)
    out = []
    for n in steps:
        inst = synth.free_moving_well(M=M, V0=V0, beta=beta, x0=x0, c=c, T=T, nsteps=n)
        orc = freespace.FreeSpaceOracle([rule], inst.dt, inst.Vt, None, fields.phi_callable(None, 1))
        out.append(rel_l2(orc.solve(inst.u0, n), ref))
    return out


def test_free_moving_well_galilean_closed_form():
    """8th order in dt (measured 5.6e-7, 2.4e-9 at 400, 800 steps)."""
    e400, e800 = _free_galilean_errors((400, 800))
    assert e800 < 1e-8 and e400 / e800 > 100.0


def test_free_moving_well_pin_catches_lagged_potential(monkeypatch):
    """Planted mistake: the implicit solve takes V one step late."""
    orig = freespace.FreeSpaceOracle.V

    def lagged(self, t):
        return orig(self, t - self.dt) if t > 8 * self.dt else orig(self, t)
    monkeypatch.setattr(freespace.FreeSpaceOracle, "V", lagged)
    e400, e800 = _free_galilean_errors((400, 800))
    assert not (e800 < 1e-8 and e400 / e800 > 100.0)


# ---------------------------------------------- Chebyshev form of the C-type transforms
@pytest.mark.parametrize("H,n_r", [(2.0, 3), (1.2, 4), (3.0, 2)])
def test_ctype_chebyshev_equals_direct_sums(H, n_r):
    """Sec. 4.1: the interpolants of e^{-+(1+i) tau x} reproduce the direct
    C-type sums (eq. fhatCsum and its inverse) to rounding once N_T is large
    enough, and are far off with too few terms (the degree matters)."""
    from oracle.freespace import ctype_chebyshev, free_grid
    rule = gamma.GammaRule.for_nu(64, 512, H, q=10, n_r=n_r)
    x = free_grid(64)
    zc, wc = rule.blocks["C"]
    rng = np.random.default_rng(7)
    f = rng.normal(size=64) + 1j * rng.normal(size=64)
    fh = rng.normal(size=zc.size) + 1j * rng.normal(size=zc.size)
    direct_f = (2.0 / 64) * np.exp(-1j * np.outer(zc, x)) @ f
    direct_i = (np.exp(1j * np.outer(x, zc)) * (wc[None, :] / (2.0 * math.pi))) @ fh
    fwd, inv = ctype_chebyshev(rule, 28)
    assert np.max(np.abs(fwd(f) - direct_f)) <= 1e-13 * np.max(np.abs(direct_f))
    assert np.max(np.abs(inv(fh) - direct_i)) <= 1e-13 * np.max(np.abs(direct_i))
    fwd6, _ = ctype_chebyshev(rule, 6)
    assert np.max(np.abs(fwd6(f) - direct_f)) > 1e-7 * np.max(np.abs(direct_f))


def test_ctype_chebyshev_is_exact_for_low_degree_interpolation_nodes():
    """With tau restricted to the interpolation points themselves the
    interpolant is exact for any N_T (a plain property of interpolation)."""
    from oracle.freespace import ctype_chebyshev
    rule = gamma.GammaRule.for_nu(32, 256, 1.5, q=10, n_r=1)
    NT = 10
    theta = math.pi * (np.arange(NT) + 0.5) / NT
    rule.tau_c = 1.5 * np.cos(theta)                       # evaluate at the Chebyshev points
    rule.blocks["C"] = ((1 - 1j) * rule.tau_c, np.ones(NT, dtype=np.complex128))
    fwd, _ = ctype_chebyshev(rule, NT)
    from oracle.freespace import free_grid
    x = free_grid(32)
    f = np.cos(3.0 * x) + 1j * x
    direct = (2.0 / 32) * np.exp(-1j * np.outer((1 - 1j) * rule.tau_c, x)) @ f
    assert np.max(np.abs(fwd(f) - direct)) <= 1e-13 * np.max(np.abs(direct))

