"""Pins of the oracle's RGB -> spectrum conversion (Cohen and Kappauf's
matrix R, the Matrice-R theory the paper applies to materials known only by
their RGB appearance):

* R is symmetric, idempotent and of rank 3 (an orthogonal projector), and it
  leaves the colour-matching basis itself unchanged;
* every spectrum splits into R N plus a metameric black N - R N whose XYZ is
  exactly zero, the two parts orthogonal;
* spectra from RGB values return the same RGB (the paper's round trip), and
  clamping to physical reflectances is what costs accuracy, not the method;
* a spectrum that already lies in the stimulus space is its own fundamental.
"""
import numpy as np

from paper_1912_06474_gb300 import scenes


def _basis(L=41):
    lam = scenes.wavelengths(L)
    return lam, scenes.trapezoid_weights(lam), scenes.cmf_xyz(lam)


def test_projector_properties(oracle_mod):
    for L in (16, 41, 81):
        _, w, cmf = _basis(L)
        A = oracle_mod.color_basis(w, cmf)
        R = oracle_mod.matrice_r(A)
        assert np.allclose(R, R.T, atol=1e-12)
        assert np.allclose(R @ R, R, atol=1e-12)
        assert abs(np.trace(R) - 3.0) <= 1e-10
        assert np.allclose(R @ A, A, atol=1e-12)


def test_fundamental_plus_metameric_black(oracle_mod):
    _, w, cmf = _basis(41)
    A = oracle_mod.color_basis(w, cmf)
    R = oracle_mod.matrice_r(A)
    rng = np.random.default_rng(0)
    for _ in range(20):
        N = rng.uniform(0, 1, 41)
        F = R @ N
        B = N - F
        assert np.allclose(A.T @ B, 0.0, atol=1e-12)          # metameric black: X = Y = Z = 0
        assert np.allclose(A.T @ F, A.T @ N, atol=1e-12)      # same colour stimulus
        assert abs(F @ B) <= 1e-10 * (N @ N)                   # orthogonal parts
        assert np.allclose(oracle_mod.fundamental_from_xyz(A.T @ N, A), F, atol=1e-12)


def test_rgb_round_trip(oracle_mod):
    _, w, cmf = _basis(41)
    rng = np.random.default_rng(1)
    rgb = rng.uniform(0.05, 0.95, (200, 3))
    spec = oracle_mod.rgb_to_spectrum(rgb, w, cmf)
    assert np.allclose(oracle_mod.spectrum_to_rgb(spec, w, cmf), rgb, atol=1e-12)
    # in-space spectrum is its own fundamental
    A = oracle_mod.color_basis(w, cmf)
    assert np.allclose(oracle_mod.rgb_to_spectrum(rgb[:1], w, cmf, clamp=False)[0],
                       oracle_mod.matrice_r(A) @ spec[0], atol=1e-12)
    # clamping to [0, 1] keeps physical reflectances; the round trip then holds
    # only where nothing was clamped
    cl = oracle_mod.rgb_to_spectrum(rgb, w, cmf, clamp=True)
    same = np.all((spec >= 0) & (spec <= 1), axis=1)
    back = oracle_mod.spectrum_to_rgb(cl, w, cmf)
    assert np.allclose(back[same], rgb[same], atol=1e-12)
