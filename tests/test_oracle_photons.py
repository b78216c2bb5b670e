"""Pins of the oracle's photon mapping (Sec. 4, global illumination by photon
mapping), in the closed white furnace (every surface Lambertian with
reflectance rho0 and emitting Le0; no photon can escape):

* every photon deposits once per hit from its second hit on (its first
  deposit follows a diffuse bounce), so N (D - 2) photons are stored, and the
  stored power at hit b sums to the emitted power pi Le0 A times rho0^(b-1):
  in total pi Le0 A sum_{b=2}^{D-1} rho0^(b-1), exactly;
* photons only reach a surface straight from the light when D = 2: nothing
  is stored (that light is next-event light);
* away from the box's edges (where the gather disc leaves the face), the
  photon-mapped image equals the furnace's closed form Le0 sum_{j<D} rho0^j
  (emission + next-event + photons) within the estimate's noise.
"""
import numpy as np

from paper_1912_06474_gb300 import scenes


def _furnace(D, rho0=0.6, Le0=0.7):
    sc = scenes.furnace_box(L=8, rho0=rho0, Le0=Le0)
    spec = scenes.RenderSpec(32, 32, 2, D, seed=1, camera=sc.camera, nee=True)
    return sc, spec, float(np.float32(rho0)), float(np.float32(Le0))


def test_stored_power_in_the_furnace(oracle_mod):
    D, N = 5, 50000
    sc, spec, rho0, Le0 = _furnace(D)
    pm = oracle_mod.Oracle(sc).photon_map(spec, N, 0.1)
    pos, dirs, pw = pm.photons()
    assert len(pos) == N * (D - 2)
    V = sc.V.astype(np.float64)[sc.F.astype(np.int64)]
    area = 0.5 * np.linalg.norm(np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0]), axis=1).sum()
    want = np.pi * Le0 * area * sum(rho0 ** (b - 1) for b in range(2, D))
    assert np.allclose(pw.sum(0), want, rtol=1e-12)
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1.0, atol=1e-12)


def test_no_photon_without_a_direction_change(oracle_mod):
    sc, spec, _, _ = _furnace(2)
    pm = oracle_mod.Oracle(sc).photon_map(spec, 10000, 0.1)
    assert len(pm.photons()[0]) == 0


def test_furnace_radiance_away_from_edges(oracle_mod):
    D = 5
    sc, spec, rho0, Le0 = _furnace(D)
    orc = oracle_mod.Oracle(sc)
    pm = orc.photon_map(spec, 200000, 0.1)
    img = orc.render_pixels(spec, photon_map=pm)["xyz"].reshape(32, 32, 3)
    want = Le0 * sum(rho0 ** j for j in range(D)) * (sc.quad_w.astype(np.float64)[:, None]
                                                     * sc.cmf.astype(np.float64)).sum(0)
    centre = img[8:24, 8:24].mean((0, 1))
    assert np.all(np.abs(centre / want - 1) < 0.01), centre / want


def test_empty_map_leaves_emission_and_direct_light(oracle_mod):
    """No photons: the path still stops at its first diffuse vertex, so the
    furnace shows emission plus one bounce of next-event light, Le0 (1 + rho0)
    (the closed box irradiates every point with pi Le0)."""
    sc, _, rho0, Le0 = _furnace(5)
    spec = scenes.RenderSpec(32, 32, 16, 5, seed=2, camera=sc.camera, nee=True)
    orc = oracle_mod.Oracle(sc)
    pm = orc.photon_map(spec, 0, 0.1)
    assert len(pm.photons()[0]) == 0
    img = orc.render_pixels(spec, photon_map=pm)["xyz"].reshape(32, 32, 3)
    want = Le0 * (1 + rho0) * (sc.quad_w.astype(np.float64)[:, None] * sc.cmf.astype(np.float64)).sum(0)
    mean = img.mean((0, 1))
    assert np.all(np.abs(mean / want - 1) < 0.01), mean / want


def test_global_and_caustic_maps_split_the_same_photons(oracle_mod):
    """Global and caustic maps hold the same stored photons as the single map
    (a photon is caustic when only reflections, no diffuse bounce, turned it):
    counts and power add up, and with equal radii the two-map render equals the
    one-map render. The closed furnace has no specular surface, so no caustics."""
    sc = scenes.tiny_room(L=16)
    spec = scenes.RenderSpec(24, 16, 2, 5, seed=4, camera=sc.camera, nee=True)
    orc = oracle_mod.Oracle(sc)
    n, r = 40000, 0.2
    pa, pg, pc = (orc.photon_map(spec, n, r, kind=k) for k in ("all", "global", "caustic"))
    (xa, _, wa), (xg, _, wg), (xc, _, wc) = pa.photons(), pg.photons(), pc.photons()
    assert len(xc) > 0 and len(xg) > 0
    assert len(xa) == len(xg) + len(xc)
    assert np.allclose(wa.sum(0), wg.sum(0) + wc.sum(0), rtol=1e-12)
    img_a = orc.render_pixels(spec, photon_map=pa)["xyz"]
    img_s = orc.render_pixels(spec, photon_map=pg, caustic_map=pc)["xyz"]
    assert np.allclose(img_a, img_s, rtol=1e-12, atol=1e-15)
    # a smaller caustic radius changes the estimate only through the caustic photons
    pc_small = orc.photon_map(spec, n, 0.05, kind="caustic")
    img_c = orc.render_pixels(spec, photon_map=pg, caustic_map=pc_small)["xyz"]
    img_g = orc.render_pixels(spec, photon_map=pg)["xyz"]
    assert not np.allclose(img_c, img_s) and np.all(img_c >= img_g - 1e-15)
    fsc, fspec, _, _ = _furnace(5)
    assert len(oracle_mod.Oracle(fsc).photon_map(fspec, 20000, 0.1, kind="caustic").photons()[0]) == 0
