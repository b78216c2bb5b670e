"""Pins of the oracle's coated slab (glass with the same thin-film stack on
both faces, e.g. an electrochromic device), against thin-film closed forms
that do not use the characteristic-matrix code:

* a zero-thickness film, or a half-wave film at normal incidence, leaves the
  bare interface: R = ((1 - n)/(1 + n))^2 (absentee layer);
* a lossless quarter-wave film at normal incidence: R = ((n_s - n_1^2)/(n_s + n_1^2))^2;
* one absorbing film at oblique incidence equals the Airy sum
  r = (r01 + r12 e^{2i beta}) / (1 + r01 r12 e^{2i beta}), both polarisations;
* reciprocity: the face transmits the same from air and from the glass;
* energy: lossless films on a clear slab give R + T = 1; absorption is >= 0 and
  grows with the coloration state;
* no films: the bare slab; a lossless AR-coated clear slab at normal incidence
  transmits (1 - R_a)/(1 + R_a).
"""
import numpy as np


def _airy(c, lam, n_sub, n1, k1, t_nm, pol):
    s2 = 1 - c * c
    N1 = complex(n1, k1)
    c1 = np.sqrt(1 - s2 / N1 ** 2 + 0j)
    if (N1 * c1).imag < 0:
        c1 = -c1
    cs = np.sqrt(1 - s2 / n_sub ** 2)
    if pol == 0:
        r01 = (c - N1 * c1) / (c + N1 * c1)
        r12 = (N1 * c1 - n_sub * cs) / (N1 * c1 + n_sub * cs)
    else:
        r01 = (N1 * c - c1) / (N1 * c + c1)
        r12 = (n_sub * c1 - N1 * cs) / (n_sub * c1 + N1 * cs)
    e = np.exp(2j * (2 * np.pi * N1 * t_nm * c1 / lam))
    r = (r01 + r12 * e) / (1 + r01 * r12 * e)
    return abs(r) ** 2


def test_absentee_and_zero_thickness(oracle_mod):
    for n_sub in (1.45, 1.52):
        bare = ((1 - n_sub) / (1 + n_sub)) ** 2
        for layers in ([(2.1, 0.0, 0.0)], [(2.1, 0.0, 550.0 / (2 * 2.1))], [(1.9, 0.0, 550.0 / 1.9)]):
            Ra, Ta, Rg, Tg = oracle_mod.coated_face(1.0, 550.0, n_sub, layers, 0)
            assert abs(Ra - bare) <= 1e-12 and abs(Rg - bare) <= 1e-12
            assert abs(Ra + Ta - 1) <= 1e-12
    # oblique, zero thickness == bare Fresnel (real index)
    for c in (0.9, 0.5, 0.2):
        Rs, Rp = oracle_mod.fresnel(c, 1.52, 0.0)
        for pol, want in ((0, Rs), (1, Rp)):
            Ra, _, _, _ = oracle_mod.coated_face(c, 600.0, 1.52, [(2.0, 0.05, 0.0)], pol)
            assert abs(Ra - want) <= 1e-12


def test_quarter_wave_film(oracle_mod):
    for n1, n_sub in ((1.38, 1.52), (1.23, 1.52), (2.0, 1.45)):
        t = 550.0 / (4 * n1)
        want = ((n_sub - n1 * n1) / (n_sub + n1 * n1)) ** 2
        for pol in (0, 1):
            Ra, Ta, Rg, Tg = oracle_mod.coated_face(1.0, 550.0, n_sub, [(n1, 0.0, t)], pol)
            assert abs(Ra - want) <= 1e-12
            assert abs(Ra + Ta - 1) <= 1e-12


def test_single_film_equals_airy(oracle_mod):
    rng = np.random.default_rng(4)
    for _ in range(40):
        c, lam = rng.uniform(0.05, 1), rng.uniform(380, 780)
        n1, k1, t = rng.uniform(1.3, 2.6), rng.uniform(0, 0.3), rng.uniform(5, 800)
        n_sub = rng.uniform(1.4, 1.7)
        for pol in (0, 1):
            Ra, _, _, _ = oracle_mod.coated_face(c, lam, n_sub, [(n1, k1, t)], pol)
            assert abs(Ra - _airy(c, lam, n_sub, n1, k1, t, pol)) <= 1e-12


def test_reciprocity_and_energy(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(30):
        J = int(rng.integers(1, 5))
        layers = [(rng.uniform(1.3, 2.5), rng.uniform(0, 0.2), rng.uniform(10, 500)) for _ in range(J)]
        c, lam, n_sub = rng.uniform(0.05, 1), rng.uniform(380, 780), rng.uniform(1.4, 1.7)
        for pol in (0, 1):
            Ra, Ta, Rg, Tg = oracle_mod.coated_face(c, lam, n_sub, layers, pol)
            assert abs(Ta - Tg) <= 1e-12 * max(1.0, Ta)
            assert Ra + Ta <= 1 + 1e-12 and Rg + Tg <= 1 + 1e-12
        lossless = [(n, 0.0, t) for n, _, t in layers]
        R, T = oracle_mod.coated_slab(c, lam, n_sub, 0.0, 0.004, lossless)
        assert abs(R + T - 1) <= 1e-12
        R, T = oracle_mod.coated_slab(c, lam, n_sub, 30.0, 0.004, layers)
        assert R >= 0 and T >= 0 and R + T <= 1
    # absorption grows with the coloration state of an absorbing film
    A = []
    for s in (0.0, 0.25, 0.5, 1.0):
        R, T = oracle_mod.coated_slab(0.8, 650.0, 1.52, 10.0, 0.004, [(1.9, 0.002, 250.0), (2.1, 0.01 + 0.3 * s, 400.0)])
        A.append(1 - R - T)
    assert all(b > a for a, b in zip(A, A[1:]))


def test_no_films_and_ar_coated_slab(oracle_mod):
    for c in (1.0, 0.7, 0.3):
        for alpha in (0.0, 120.0):
            assert oracle_mod.coated_slab(c, 500.0, 1.52, alpha, 0.006, []) == oracle_mod.slab(c, 500.0, 1.52, alpha, 0.006)
    n1 = 1.23
    Ra = ((1.52 - n1 * n1) / (1.52 + n1 * n1)) ** 2
    R, T = oracle_mod.coated_slab(1.0, 550.0, 1.52, 0.0, 0.004, [(n1, 0.0, 550.0 / (4 * n1))])
    assert abs(T - (1 - Ra) / (1 + Ra)) <= 1e-12
