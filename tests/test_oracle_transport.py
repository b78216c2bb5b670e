"""Pins of the oracle's estimator (render.c) against closed forms.

* white furnace: every sample equals Le * sum_{j<D} rho0^j exactly (P-c);
* an emitter seen directly returns its radiance;
* a glass pane at normal incidence: each sample is 0 (reflect into black) or
  T Le / (1 - P_r) (transmit, the pane's own faces skipped);
* a metal mirror at 45 degrees returns F(cos) Le;
* next-event estimation and BSDF-only sampling agree in expectation (P-h);
* direct light from a parallel rectangle matches the analytic form factor.
"""
import math

import numpy as np
import pytest

from paper_1912_06474_gb300 import scenes


def _xyz_of(scene, spectrum):
    w = scene.quad_w.astype(np.float64)
    cmf = scene.cmf.astype(np.float64)
    return (w[:, None] * np.asarray(spectrum, np.float64)[:, None] * cmf).sum(0)


def _scene(L, mats, meshes, cam):
    lam = scenes.wavelengths(L)
    mb = scenes._MeshBuilder()
    for (V, F), m in meshes:
        mb.add(V, F, m)
    V, F, M, O = mb.arrays()
    return scenes.Scene(lam, scenes.trapezoid_weights(lam), scenes.cmf_xyz(lam), mats, V, F, M, O, cam)


@pytest.mark.parametrize("D", [1, 3, 6])
def test_white_furnace_exact(oracle_mod, D):
    rho0, Le0 = 0.6, 0.7
    sc = scenes.furnace_box(L=8, rho0=rho0, Le0=Le0)
    spec = scenes.RenderSpec(8, 8, 4, D, seed=3, camera=sc.camera, nee=False)
    res = oracle_mod.Oracle(sc).render_pixels(spec, per_sample=True)
    Le0, rho0 = float(np.float32(Le0)), float(np.float32(rho0))   # the inputs are float32
    want = Le0 * sum(rho0 ** j for j in range(D)) * _xyz_of(sc, np.ones(sc.L))
    assert np.allclose(res["sample_xyz"], want, rtol=1e-12, atol=0)
    assert res["segments"] == (8 * 8 * 4 * D, 0)


def test_emitter_seen_directly(oracle_mod):
    L = 8
    Le = np.linspace(0.5, 2.0, L).astype(np.float32)
    mats = [scenes.Material(scenes.LAMBERT, rho=np.zeros(L, np.float32)),
            scenes.Material(scenes.EMITTER, Le=Le)]
    light = scenes.quad_mesh((3, -1, -1), (3, -1, 1), (3, 1, 1), (3, 1, -1))   # faces -x
    box = scenes.box_mesh((-5, -5, -5), (5, 5, 5), inward=True)
    sc = _scene(L, mats, [(light, 1), (box, 0)], scenes.Camera((0, 0, 0), (1, 0, 0), vfov_deg=90))
    spec = scenes.RenderSpec(16, 16, 2, 3, camera=sc.camera)
    res = oracle_mod.Oracle(sc).render_pixels(spec, per_sample=True)
    on_light = res["first_prim"] < 2
    assert on_light.sum() > 20 and (~on_light).sum() > 20
    assert np.allclose(res["sample_xyz"][on_light], _xyz_of(sc, Le), rtol=1e-12)
    assert np.all(res["sample_xyz"][~on_light] == 0.0)


def test_glass_pane_normal_incidence(oracle_mod):
    L = 8
    lam = scenes.wavelengths(L)
    Le = np.linspace(1.0, 3.0, L).astype(np.float32)
    n = scenes.cauchy_index(lam)
    a_clear = np.linspace(5.0, 20.0, L).astype(np.float32)
    dalpha = np.linspace(300.0, 50.0, L).astype(np.float32)
    s, thick = 0.4, 0.004
    mats = [scenes.Material(scenes.LAMBERT, rho=np.zeros(L, np.float32)),
            scenes.Material(scenes.EMITTER, Le=Le),
            scenes.Material(scenes.GLASS, n=n, alpha_clear=a_clear, dalpha=dalpha,
                            thickness_m=thick, s_default=s)]
    pane = scenes.box_mesh((2.0, -1, -1), (2.004, 1, 1))
    light = scenes.quad_mesh((3, -2, -2), (3, -2, 2), (3, 2, 2), (3, 2, -2))
    box = scenes.box_mesh((-5, -5, -5), (5, 5, 5), inward=True)
    cam = scenes.Camera((0, 0, 0), (1, 0, 0), ortho_height=0.5)
    sc = _scene(L, mats, [(pane, 2), (light, 1), (box, 0)], cam)
    orc = oracle_mod.Oracle(sc)
    spec = scenes.RenderSpec(8, 8, 64, 2, seed=5, camera=cam)
    res = orc.render_pixels(spec, per_sample=True)
    pr = float(oracle_mod.branch_proxy(1.0, n))
    s64, th64 = float(np.float32(s)), float(np.float32(thick))     # the inputs are float32
    T = np.array([oracle_mod.slab(1.0, float(lam[i]), float(n[i]),
                                  float(a_clear[i]) + s64 * float(dalpha[i]), th64)[1]
                  for i in range(L)])
    want = _xyz_of(sc, T * Le / (1.0 - pr))
    smp = res["sample_xyz"].reshape(-1, 3)
    through = np.all(np.isclose(smp, want, rtol=1e-12, atol=0), axis=1)
    zero = np.all(smp == 0.0, axis=1)
    assert np.all(through | zero)
    N = smp.shape[0]
    assert abs(zero.mean() - pr) < 4 * math.sqrt(pr * (1 - pr) / N) + 1.0 / N
    # at D = 1 the glass vertex is the last one: nothing is seen
    res1 = orc.render_pixels(scenes.RenderSpec(8, 8, 4, 1, camera=cam), per_sample=True)
    assert np.all(res1["sample_xyz"] == 0.0)


def test_metal_mirror_45_degrees(oracle_mod):
    L = 8
    Le = np.linspace(2.0, 1.0, L).astype(np.float32)
    nm = np.linspace(0.3, 2.5, L).astype(np.float32)
    km = np.linspace(6.0, 2.0, L).astype(np.float32)
    mats = [scenes.Material(scenes.LAMBERT, rho=np.zeros(L, np.float32)),
            scenes.Material(scenes.EMITTER, Le=Le),
            scenes.Material(scenes.CONDUCTOR, n=nm, k=km)]
    # mirror plane through x = 2 tilted 45 degrees about z, sending +x rays to +y
    mirror = scenes.quad_mesh((1, -1, -1), (3, 1, -1), (3, 1, 1), (1, -1, 1))
    light = scenes.quad_mesh((0, 3, -3), (4, 3, -3), (4, 3, 3), (0, 3, 3))   # faces -y
    box = scenes.box_mesh((-5, -5, -5), (5, 5, 5), inward=True)
    cam = scenes.Camera((-1, 0, 0), (0, 0, 0), ortho_height=0.4)
    sc = _scene(L, mats, [(mirror, 2), (light, 1), (box, 0)], cam)
    res = oracle_mod.Oracle(sc).render_pixels(scenes.RenderSpec(8, 8, 4, 2, camera=cam),
                                              per_sample=True)
    c = math.cos(math.pi / 4)
    F = np.array([oracle_mod.conductor(c, nm[i], km[i]) for i in range(L)])
    assert np.allclose(res["sample_xyz"].reshape(-1, 3), _xyz_of(sc, F * Le), rtol=1e-9)


def _lit_floor(L=8, rho_val=None, light_half=(0.5, 0.7), h=2.0):
    lam = scenes.wavelengths(L)
    rho = np.linspace(0.3, 0.8, L).astype(np.float32) if rho_val is None else rho_val
    Le = np.linspace(1.0, 2.0, L).astype(np.float32)
    mats = [scenes.Material(scenes.LAMBERT, rho=rho), scenes.Material(scenes.EMITTER, Le=Le),
            scenes.Material(scenes.LAMBERT, rho=np.zeros(L, np.float32))]
    ax, ay = light_half
    floor = scenes.quad_mesh((-4, -4, 0), (4, -4, 0), (4, 4, 0), (-4, 4, 0))
    light = scenes.quad_mesh((-ax, -ay, h), (-ax, ay, h), (ax, ay, h), (ax, -ay, h))  # faces -z
    box = scenes.box_mesh((-4.5, -4.5, -0.5), (4.5, 4.5, 4.0), inward=True)
    return lam, rho, Le, mats, [(floor, 0), (light, 1), (box, 2)]


def test_direct_light_form_factor(oracle_mod):
    """NEE at a floor point under a parallel rectangle: L = rho * Le * F_rect."""
    ax, ay, h = 0.5, 0.7, 2.0
    lam, rho, Le, mats, meshes = _lit_floor(light_half=(ax, ay), h=h)
    cam = scenes.Camera((0, 0, 1.0), (0, 0, 0), up=(0, 1, 0), ortho_height=1e-4)
    sc = _scene(8, mats, meshes, cam)
    spec = scenes.RenderSpec(1, 1, 40000, 1, seed=9, camera=cam)
    res = oracle_mod.Oracle(sc).render_pixels(spec, per_sample=True)

    def f_corner(x, y):
        X, Y = x / h, y / h
        return (X / math.sqrt(1 + X * X) * math.atan(Y / math.sqrt(1 + X * X))
                + Y / math.sqrt(1 + Y * Y) * math.atan(X / math.sqrt(1 + Y * Y))) / (2 * math.pi)
    F = 4 * f_corner(ax, ay)
    want = _xyz_of(sc, rho.astype(np.float64) * Le * F)
    smp = res["sample_xyz"].reshape(-1, 3)
    sig = smp.std(0) / math.sqrt(smp.shape[0])
    assert np.all(np.abs(smp.mean(0) - want) < 4 * sig)
    assert np.all(sig < 0.01 * want)


def test_nee_matches_bsdf_sampling(oracle_mod):
    """Direct light by next-event estimation == by BSDF sampling (P-h)."""
    lam, rho, Le, mats, meshes = _lit_floor(light_half=(0.8, 0.8), h=1.5)
    cam = scenes.Camera((0, -1.0, 1.0), (0, 0.5, 0), up=(0, 0, 1), vfov_deg=50)
    sc = _scene(8, mats, meshes, cam)
    orc = oracle_mod.Oracle(sc)
    a = orc.render_pixels(scenes.RenderSpec(6, 6, 3000, 2, seed=1, camera=cam, nee=True),
                          per_sample=True)["sample_xyz"]
    b = orc.render_pixels(scenes.RenderSpec(6, 6, 3000, 2, seed=2, camera=cam, nee=False),
                          per_sample=True)["sample_xyz"]
    ma, mb = a.mean(1), b.mean(1)
    sa, sb = a.std(1) / math.sqrt(a.shape[1]), b.std(1) / math.sqrt(b.shape[1])
    z = np.abs(ma - mb) / np.sqrt(sa ** 2 + sb ** 2 + 1e-30)
    assert np.all(z[..., 1] < 4.5), z[..., 1].max()
    assert ma[..., 1].mean() > 0
