"""Pins of the oracle's optics against closed forms and independent formulas.

Each check would fail for a plausible slip in the oracle: a swapped r_s/r_p,
a sign error in the complex root, a dropped (1 - rho)^2 factor or a wrong
power of tau in the slab sum, a wrong k = alpha lambda / 4 pi conversion.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_normal_incidence_closed_form(oracle_mod):
    """Eq. 1 at normal incidence: R = ((n-1)^2 + k^2) / ((n+1)^2 + k^2)."""
    rng = np.random.default_rng(1)
    for n, k in zip(rng.uniform(0.2, 3.0, 50), rng.uniform(0.0, 8.0, 50)):
        want = ((n - 1) ** 2 + k * k) / ((n + 1) ** 2 + k * k)
        rs, rp = oracle_mod.fresnel(1.0, n, k)
        assert abs(rs - want) < 1e-12 and abs(rp - want) < 1e-12
        assert abs(oracle_mod.conductor(1.0, n, k) - want) < 1e-12


def test_dielectric_trig_form_and_brewster(oracle_mod):
    """k = 0: Fresnel's sine/tangent forms with Snell's law, and r_p = 0 at Brewster."""
    rng = np.random.default_rng(2)
    for n, th in zip(rng.uniform(1.05, 2.5, 40), rng.uniform(0.01, 1.5, 40)):
        tt = math.asin(math.sin(th) / n)
        want_s = (math.sin(th - tt) / math.sin(th + tt)) ** 2
        want_p = (math.tan(th - tt) / math.tan(th + tt)) ** 2
        rs, rp = oracle_mod.fresnel(math.cos(th), n, 0.0)
        assert abs(rs - want_s) < 1e-12 and abs(rp - want_p) < 1e-12
        thb = math.atan(n)
        rs, rp = oracle_mod.fresnel(math.cos(thb), n, 0.0)
        assert rp < 1e-24
        assert abs(rs - ((n * n - 1) / (n * n + 1)) ** 2) < 1e-12


def test_conductor_real_form(oracle_mod):
    """Complex index against the real-arithmetic conductor formula (a^2 + b^2 form)."""
    rng = np.random.default_rng(3)
    for n, k, th in zip(rng.uniform(0.2, 3.0, 60), rng.uniform(1.0, 8.0, 60), rng.uniform(0.0, 1.55, 60)):
        s2 = math.sin(th) ** 2
        c = math.cos(th)
        t0 = n * n - k * k - s2
        a2b2 = math.sqrt(t0 * t0 + 4 * n * n * k * k)
        a = math.sqrt(0.5 * (a2b2 + t0))
        rs = (a2b2 - 2 * a * c + c * c) / (a2b2 + 2 * a * c + c * c)
        st = math.sin(th) * math.tan(th)
        rp = rs * (a2b2 - 2 * a * st + st * st) / (a2b2 + 2 * a * st + st * st)
        want = 0.5 * (rs + rp)
        assert abs(oracle_mod.conductor(c, n, k) - want) < 1e-11


def test_grazing_and_zero_cos(oracle_mod):
    assert abs(oracle_mod.conductor(1e-9, 1.5, 3.0) - 1.0) < 1e-6
    R, T = oracle_mod.slab(0.0, 500.0, 1.5, 100.0, 0.004)
    assert R == 1.0 and T == 0.0


def test_lossless_slab_identities(oracle_mod):
    """k = 0, alpha = 0: R + T = 1 and T(0 deg) = 2n / (n^2 + 1)."""
    rng = np.random.default_rng(4)
    for n in rng.uniform(1.01, 2.5, 30):
        R, T = oracle_mod.slab(1.0, 550.0, n, 0.0, 0.004)
        assert abs(T - 2 * n / (n * n + 1)) < 1e-12
        for c in rng.uniform(0.0, 1.0, 10):
            R, T = oracle_mod.slab(c, 550.0, n, 0.0, 0.004)
            assert abs(R + T - 1.0) < 1e-12


def _tau(c, n, alpha, d):
    ct = math.sqrt(1.0 - (1.0 - c * c) / (n * n))
    return math.exp(-alpha * d / ct)


def test_slab_equals_explicit_multiple_reflection_series(oracle_mod):
    """Closed form == sum over internal bounces, beam by beam, per polarisation."""
    rng = np.random.default_rng(5)
    for _ in range(40):
        c = rng.uniform(0.05, 1.0)
        lam = rng.uniform(380, 780)
        n = rng.uniform(1.3, 1.9)
        alpha = rng.uniform(0.0, 600.0)
        d = rng.uniform(0.002, 0.01)
        k = alpha * lam * 1e-9 / (4 * math.pi)
        rhos = oracle_mod.fresnel(c, n, k)
        tau = _tau(c, n, alpha, d)
        R_want = T_want = 0.0
        for rho in rhos:
            r_sum = rho
            t_sum = 0.0
            beam = (1 - rho) * tau          # after entering and crossing once
            for _bounce in range(400):
                t_sum += beam * (1 - rho)   # leaves through the back face
                beam *= rho * tau           # reflected at the back, crosses again
                r_sum += beam * (1 - rho)   # leaves through the front face
                beam *= rho * tau
            R_want += 0.5 * r_sum
            T_want += 0.5 * t_sum
        R, T = oracle_mod.slab(c, lam, n, alpha, d)
        assert abs(R - R_want) < 1e-12 and abs(T - T_want) < 1e-12
        assert R + T <= 1.0 + 1e-12


def test_slab_monte_carlo_bounce_simulation(oracle_mod):
    """FP64 Monte Carlo of photons bouncing inside the slab agrees within 4 sigma."""
    rng = np.random.default_rng(6)
    for c, alpha in ((0.9, 120.0), (0.3, 400.0), (0.7, 0.0)):
        lam, n, d = 520.0, 1.52, 0.004
        k = alpha * lam * 1e-9 / (4 * math.pi)
        rs, rp = oracle_mod.fresnel(c, n, k)
        tau = _tau(c, n, alpha, d)
        N = 400_000
        refl = np.zeros(N, bool)
        trans = np.zeros(N, bool)
        pol = rng.uniform(size=N) < 0.5
        rho = np.where(pol, rs, rp)
        alive = rng.uniform(size=N) >= rho      # enters the slab
        refl |= ~alive
        side_back = np.ones(N, bool)            # travelling toward the back face
        for _ in range(60):
            survive = rng.uniform(size=N) < tau
            alive &= survive
            out = alive & (rng.uniform(size=N) >= rho)
            trans |= out & side_back
            refl |= out & ~side_back
            alive &= ~out
            side_back = ~side_back
        R, T = oracle_mod.slab(c, lam, n, alpha, d)
        for est, want in ((refl.mean(), R), (trans.mean(), T)):
            sig = math.sqrt(max(want * (1 - want), 1e-12) / N)
            assert abs(est - want) < 4 * sig + 1e-9


def test_absorption_energy_balance(oracle_mod):
    """R + T + A = 1 with A >= 0, and more absorption transmits less."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        c, lam, n = rng.uniform(0.01, 1), rng.uniform(380, 780), rng.uniform(1.3, 1.9)
        R1, T1 = oracle_mod.slab(c, lam, n, 50.0, 0.004)
        R2, T2 = oracle_mod.slab(c, lam, n, 500.0, 0.004)
        assert 0.0 <= R1 + T1 <= 1.0 + 1e-12
        assert T2 < T1


def test_branch_proxy(oracle_mod):
    """Proxy = clamp(mean over bins of the lossless slab reflectance, 0.05, 0.95), in float."""
    n = np.full(8, 1.5, np.float32)
    rho = ((1.5 - 1) / 2.5) ** 2
    assert abs(oracle_mod.branch_proxy(1.0, n) - 2 * rho / (1 + rho)) < 1e-6
    assert oracle_mod.branch_proxy(1.0, np.ones(4, np.float32)) == np.float32(0.05)
    assert oracle_mod.branch_proxy(1e-4, n) == np.float32(0.95)
    rng = np.random.default_rng(8)
    for _ in range(20):
        nc = rng.uniform(1.3, 1.8, 41).astype(np.float32)
        c = float(np.float32(rng.uniform(0.05, 1.0)))
        want = 0.0
        for ni in nc.astype(np.float64):
            rs, rp = oracle_mod.fresnel(c, ni, 0.0)
            want += 0.5 * (2 * rs / (1 + rs) + 2 * rp / (1 + rp))
        want = min(max(want / 41, 0.05), 0.95)
        assert abs(oracle_mod.branch_proxy(c, nc) - want) < 2e-6
