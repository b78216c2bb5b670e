"""Pins of the oracle's geometry, sampling and random stream.

Independent formulations: plane intersection with area-ratio barycentrics for
Moller-Trumbore, brute force for the BVH, moments of the cosine law for the
direction sampler, the pinhole geometry for the camera, and for the
counter-based stream the published known-answer vectors of Philox4x32-10 plus
statistics.
"""
import math

import numpy as np
import pytest

from paper_1912_06474_gb300 import scenes


def test_philox_known_answers(oracle_mod):
    """Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) against the known-answer
    vectors published with the generator's reference implementation (Random123):
    counter and key all zeros, all ones, and the digits of pi."""
    cases = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for ctr, key, want in cases:
        assert tuple(int(x) for x in oracle_mod.philox4x32_10(list(ctr), list(key))) == want


def test_philox_statistics(oracle_mod):
    """Uniforms of distinct counters: mean, variance, chi^2 over 64 bins, avalanche."""
    n = 1 << 14
    u = np.empty(4 * n)
    words = np.empty((n, 4), np.uint32)
    for i in range(n):
        x = oracle_mod.philox4x32_10([i, 7, 3, 0x10001], [0, 0])
        words[i] = x
    u = (words.astype(np.float64).ravel() / 256.0).astype(np.int64) * 2.0 ** -24
    N = u.size
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / N)
    assert abs(u.var() - 1 / 12) < 4 * math.sqrt(1 / 180 / N)
    hist = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = ((hist - N / 64) ** 2 / (N / 64)).sum()
    assert chi2 < 63 + 6 * math.sqrt(2 * 63)
    assert len({tuple(w) for w in words.tolist()}) == n
    flips = []
    base = oracle_mod.philox4x32_10([12345, 1, 2, 3], [99, 5])
    for bit in range(128):
        ctr = [12345, 1, 2, 3]
        ctr[bit // 32] ^= 1 << (bit % 32)
        x = oracle_mod.philox4x32_10(ctr, [99, 5])
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(x, base)))
    assert abs(np.mean(flips) - 64) < 4 * math.sqrt(32 / 128)
    assert oracle_mod.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24 and oracle_mod.u01(255) == 0.0
    # the key matters
    assert not np.array_equal(oracle_mod.philox4x32_10([1, 2, 3, 4], [0, 0]),
                              oracle_mod.philox4x32_10([1, 2, 3, 4], [0, 1]))


@pytest.mark.parametrize("ns", [(0, 0, 1), (0, 0, -1), (1, 0, 0), (0.3, -0.5, -0.81),
                                (1e-7, 0, -1)])
def test_cosine_sampling_moments(oracle_mod, ns):
    """Directions lie in the hemisphere, are unit, and have E[cos]=2/3, E[cos^2]=1/2."""
    ns = np.asarray(ns, float)
    ns /= np.linalg.norm(ns)
    rng = np.random.default_rng(11)
    N = 20000
    cs = np.empty(N)
    for i in range(N):
        d = oracle_mod.cosine_dir(ns, rng.uniform(), rng.uniform())
        assert abs(np.linalg.norm(d) - 1) < 1e-12
        cs[i] = d @ ns
    assert cs.min() >= -1e-12
    sig1 = math.sqrt((0.5 - 4 / 9) / N)
    sig2 = math.sqrt((1 / 3 - 1 / 4) / N)
    assert abs(cs.mean() - 2 / 3) < 4 * sig1
    assert abs((cs ** 2).mean() - 0.5) < 4 * sig2


def test_camera_pinhole_geometry(oracle_mod):
    s = scenes.tiny_room()
    spec = scenes.RenderSpec(64, 48, 1, 1, camera=s.camera)
    orc = oracle_mod.Oracle(s)
    o, d = orc.camera_ray(spec, 32.0, 24.0)
    f = np.subtract(s.camera.look, s.camera.pos)
    f /= np.linalg.norm(f)
    assert np.allclose(o, s.camera.pos) and np.allclose(d, f, atol=1e-15)
    _, d = orc.camera_ray(spec, 32.0, 0.0)      # top edge: half the vertical field
    assert abs(math.degrees(math.acos(d @ f)) - 30.0) < 1e-9 and d[2] > 0
    _, d = orc.camera_ray(spec, 64.0, 24.0)     # right edge: aspect-scaled tangent
    assert abs(math.tan(math.acos(d @ f)) - math.tan(math.radians(30)) * 64 / 48) < 1e-12


def _plane_area_bary(v0, v1, v2, o, d):
    """Plane hit t and barycentrics from signed sub-triangle areas."""
    n = np.cross(v1 - v0, v2 - v0)
    t = ((v0 - o) @ n) / (d @ n)
    p = o + t * d
    A = n @ n
    b1 = (np.cross(p - v0, v2 - v0) @ n) / A
    b2 = (np.cross(v1 - v0, p - v0) @ n) / A
    return t, 1 - b1 - b2, b1, b2


def test_moller_trumbore_against_plane_intersection(oracle_mod):
    """The oracle's hit t and barycentrics equal plane intersection + area ratios."""
    sc = scenes.random_soup(1, seed=3)
    orc = oracle_mod.Oracle(sc)
    v = sc.V.astype(np.float64)
    rng = np.random.default_rng(12)
    hits = 0
    for _ in range(3000):
        o = rng.uniform(-1.0, 2.0, 3)
        target = v.mean(0) + rng.normal(0, 0.2, 3)
        d = target - o
        d /= np.linalg.norm(d)
        prim, t, b = orc.closest_hit(o, d, brute_force=True)
        t2, *bb = _plane_area_bary(v[0], v[1], v[2], o, d)
        inside = min(bb) >= 0 and t2 > 0
        if abs(min(bb)) < 1e-9:
            continue
        assert (prim == 0) == inside
        if inside:
            hits += 1
            assert abs(t - t2) < 1e-9 * max(1, t2)
            assert np.allclose(b, bb, atol=1e-9)
    assert hits > 100


def test_bvh_equals_brute_force(oracle_mod):
    """Closest hits through the median-split BVH equal brute force (P-e)."""
    rng = np.random.default_rng(13)
    for seed, ntri in ((1, 50), (2, 400), (3, 1000)):
        sc = scenes.random_soup(ntri, seed=seed)
        orc = oracle_mod.Oracle(sc)
        for _ in range(1500):
            o = rng.uniform(-0.5, 1.5, 3)
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            pb, tb, _ = orc.closest_hit(o, d, brute_force=True)
            pv, tv, _ = orc.closest_hit(o, d, brute_force=False)
            assert pb == pv and (pb < 0 or tb == tv)


def _glass_slabs_scene(n_slabs, with_blocker=False):
    lam = scenes.wavelengths(4)
    mats = [scenes.Material(scenes.LAMBERT, rho=np.full(4, 0.5, np.float32)),
            scenes.Material(scenes.GLASS, n=np.full(4, 1.5, np.float32),
                            alpha_clear=np.zeros(4, np.float32), dalpha=np.zeros(4, np.float32),
                            thickness_m=0.01, s_default=0.0)]
    mb = scenes._MeshBuilder()
    for i in range(n_slabs):
        x = 1.0 + i
        mb.add(*scenes.box_mesh((x, -1, -1), (x + 0.01, 1, 1)), 1)
    if with_blocker:
        mb.add(*scenes.quad_mesh((0.5, -1, -1), (0.5, 1, -1), (0.5, 1, 1), (0.5, -1, 1)), 0)
    V, F, M, O = mb.arrays()
    return scenes.Scene(lam, scenes.trapezoid_weights(lam), scenes.cmf_xyz(lam), mats, V, F, M, O,
                        scenes.Camera((0, 0, 0), (1, 0, 0)))


@pytest.mark.parametrize("brute", [True, False])
def test_shadow_glass_crossings(oracle_mod, brute):
    """Each slab crossed counts once, at its entering face; opaque occludes;
    a fifth distinct slab occludes."""
    d = np.array([1.0, 0.2, 0.1])
    d /= np.linalg.norm(d)
    for n_slabs in (1, 2, 4):
        orc = oracle_mod.Oracle(_glass_slabs_scene(n_slabs))
        occ, cr = orc.shadow([0, 0, 0], d, 20.0, brute_force=brute)
        assert not occ and len(cr) == n_slabs
        assert sorted(o for o, _ in cr) == list(range(n_slabs))
        assert all(abs(c - d[0]) < 1e-12 for _, c in cr)
        occ, cr = orc.shadow([0, 0, 0], d, 0.5, brute_force=brute)   # stops short of every slab
        assert not occ and cr == []
    orc = oracle_mod.Oracle(_glass_slabs_scene(5))
    assert orc.shadow([0, 0, 0], d, 20.0, brute_force=brute)[0]
    orc = oracle_mod.Oracle(_glass_slabs_scene(1, with_blocker=True))
    assert orc.shadow([0, 0, 0], d, 20.0, brute_force=brute)[0]
    # travelling the other way the entering faces are the +x faces
    orc = oracle_mod.Oracle(_glass_slabs_scene(2))
    occ, cr = orc.shadow([5, 0, 0], -d, 20.0, brute_force=brute)
    assert not occ and len(cr) == 2


def test_watertight_equals_moller_trumbore_away_from_edges(oracle_mod):
    """The FP64 watertight test (Woop, Benthin, Wald 2013) agrees with the
    Moller-Trumbore test the oracle renders with wherever the ray is clearly
    inside or clearly outside the triangle: the same hit decision, and the
    same distance to 1e-12."""
    rng = np.random.default_rng(31)
    agree = hits = 0
    for _ in range(20000):
        tri = rng.uniform(-1, 1, (3, 3))
        o = rng.uniform(-2, 2, 3)
        d = tri.mean(0) + rng.normal(0, 0.6, 3) - o
        d /= np.linalg.norm(d)
        mh, mt, (u, w) = oracle_mod.moller_trumbore(tri, o, d)
        if not np.isfinite(mt) or min(abs(u), abs(w), abs(1 - u - w)) < 1e-9:
            continue
        wh, wt = oracle_mod.watertight(tri, o, d)
        assert wh == mh, (tri, o, d)
        if wh:
            hits += 1
            assert abs(wt - mt) <= 1e-12 * max(1.0, abs(mt))
        agree += 1
    assert agree > 19000 and hits > 2000


def _icosphere(levels):
    """Closed triangle mesh of the unit sphere with shared vertices."""
    t = (1 + 5 ** 0.5) / 2
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
         (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11),
         (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(levels):
        mid = {}

        def m(a, b):
            k = (min(a, b), max(a, b))
            if k not in mid:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                mid[k] = len(V) - 1
            return mid[k]
        F = [f for a, b, c in F for f in ((a, m(a, b), m(c, a)), (b, m(b, c), m(a, b)), (c, m(c, a), m(b, c)),
                                            (m(a, b), m(b, c), m(c, a)))]
    return np.array(V), np.array(F)


def test_watertight_closed_mesh_has_no_cracks(oracle_mod):
    """Rays from inside a closed mesh aimed exactly at its vertices, at points
    on its edges and at random points never miss every triangle with the
    watertight test: a shared edge or vertex belongs to at least one of the
    triangles around it."""
    V, F = _icosphere(2)
    rng = np.random.default_rng(5)
    E = {tuple(sorted((f[i], f[(i + 1) % 3]))) for f in F for i in range(3)}
    targets = [V[i] for i in range(len(V))]
    for a, b in sorted(E):
        for s in (0.5, rng.uniform(0.01, 0.99)):
            targets.append(V[a] + s * (V[b] - V[a]))
    targets += list(rng.normal(0, 1, (200, 3)))
    mt_missed = 0
    for origin in (np.zeros(3), np.array([0.1, -0.2, 0.15]), np.array([1e-3, 3e-3, -2e-3])):
        for x in targets:
            d = x - origin
            d /= np.linalg.norm(d)
            n_wt = sum(oracle_mod.watertight(V[f], origin, d)[1] > 0 for f in F)
            assert n_wt >= 1, (origin, x)
            n_mt = sum(oracle_mod.moller_trumbore(V[f], origin, d)[0] and
                       oracle_mod.moller_trumbore(V[f], origin, d)[1] > 0 for f in F)
            mt_missed += n_mt == 0
    print(f"rays through vertices and edges that Moller-Trumbore lets through: {mt_missed}")


def test_watertight_exact_shared_edge(oracle_mod):
    """A unit square split along its diagonal into two triangles, rays along
    +z and -z through points of the diagonal (and through the shared corners):
    the edge functions vanish exactly there, and the watertight test must
    count the point as inside both triangles (a boundary point belongs to
    the triangle), so the ray is never lost between them."""
    t1 = np.array([[0, 0, 1], [1, 0, 1], [1, 1, 1]], float)
    t2 = np.array([[0, 0, 1], [1, 1, 1], [0, 1, 1]], float)
    for k in range(0, 9):
        p = k / 8.0
        for dz in (1.0, -1.0):
            o = np.array([p, p, 1.0 - 2.0 * dz])
            d = np.array([0.0, 0.0, dz])
            h1, ta = oracle_mod.watertight(t1, o, d)
            h2, tb = oracle_mod.watertight(t2, o, d)
            assert h1 and h2, (p, dz)
            assert ta == tb == 2.0
