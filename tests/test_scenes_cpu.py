"""The seeded synthetic inputs have the sizes and structure the workloads name
(they stand in for the paper's hotel room, which is not available): triangle
counts, material kinds and value ranges, glass states, camera placement and
the batched-render distributions. No rendering arithmetic here."""
import numpy as np
import pytest

from paper_1912_06474_gb300 import scenes

GLASS, CONDUCTOR = scenes.GLASS, scenes.CONDUCTOR


def _kinds(sc):
    return np.array([m.kind for m in sc.materials])


def _closed_mesh_ok(sc):
    assert sc.V.dtype == np.float32 and sc.F.dtype == np.uint32
    assert sc.F.max() < len(sc.V)
    assert len(sc.mat_id) == len(sc.F) == len(sc.obj_id)
    assert sc.mat_id.max() < len(sc.materials)
    e1 = sc.V[sc.F[:, 1]] - sc.V[sc.F[:, 0]]
    e2 = sc.V[sc.F[:, 2]] - sc.V[sc.F[:, 0]]
    area = 0.5 * np.linalg.norm(np.cross(e1.astype(np.float64), e2.astype(np.float64)), axis=1)
    assert np.all(area > 0), "degenerate triangles"


def test_spectral_grid():
    for L, step in [(41, 10.0), (81, 5.0)]:
        lam = scenes.wavelengths(L)
        assert lam[0] == 380.0 and lam[-1] == 780.0 and np.allclose(np.diff(lam), step)
        w = scenes.trapezoid_weights(lam)
        assert np.isclose(w.sum(), 400.0) and np.isclose(w[0], step / 2) and np.isclose(w[1], step)
    n = scenes.cauchy_index(np.array([500.0]))
    assert np.isclose(n[0], 1.52 + 0.004 / 0.25)


def test_tiny_room_layout():
    sc = scenes.tiny_room(L=16)
    _closed_mesh_ok(sc)
    assert sc.n_tris == 38
    g = sc.glass_materials()
    assert len(g) == 1
    pane = sc.materials[g[0]]
    assert pane.thickness_m == pytest.approx(0.004)
    tri = np.isin(sc.mat_id, g)
    v = sc.V[sc.F[tri].reshape(-1)]
    assert v[:, 0].min() == pytest.approx(2.0) and v[:, 0].max() == pytest.approx(2.004)
    assert tuple(sc.camera.pos) == (0.5, 2.0, 1.5)


def test_hotel_room_structure():
    sc = scenes.hotel_room(L=41, seed=0)
    _closed_mesh_ok(sc)
    assert sc.n_tris == 200522
    kinds = _kinds(sc)
    # two photochromic panes at s = 0.5 and 20 metal spheres
    g = sc.glass_materials()
    assert len(np.unique(sc.obj_id[np.isin(sc.mat_id, g)])) == 2
    assert all(sc.materials[m].s_default == pytest.approx(0.5) for m in g)
    metal_objs = np.unique(sc.obj_id[np.isin(sc.mat_id, np.flatnonzero(kinds == CONDUCTOR))])
    assert len(metal_objs) == 20
    for m in sc.materials:
        if m.kind == CONDUCTOR:
            assert 0.2 <= m.n.min() and m.n.max() <= 3.0 and 1.0 <= m.k.min() and m.k.max() <= 8.0
        if m.rho is not None:
            assert 0.05 <= m.rho.min() and m.rho.max() <= 0.9
        if m.kind == GLASS:
            assert m.alpha_clear.min() >= 0 and m.dalpha.min() >= 0
    # a 6 x 4 x 3 m room; a few spheres cross a wall, floor or ceiling (their outer
    # part is out of the rays' reach): 98.6% of the vertices lie in the room box
    room = np.array([6.0, 4.0, 3.0], np.float32)
    inside = np.all((sc.V >= -1e-6) & (sc.V <= room + 1e-6), axis=1)
    assert inside.mean() > 0.98
    walls = sc.V[sc.F[np.isin(sc.obj_id, [0, 1])].reshape(-1)]   # floor, then walls and ceiling
    assert np.allclose(walls.min(0), 0.0) and np.allclose(walls.max(0), room)


def test_batched_render_distribution():
    sc = scenes.tiny_room(L=41)
    specs = scenes.batched_renders(sc, 64, seed=0)
    assert len(specs) == 64
    assert {s.width for s in specs} <= {128, 256, 512, 1024} and all(s.width == s.height for s in specs)
    assert {s.spp for s in specs} <= {4, 16, 64}
    states = [v for s in specs for v in s.glass_s.values()]
    assert min(states) >= 0.0 and max(states) <= 1.0
    assert len({s.render_id for s in specs}) == 64
    assert specs == scenes.batched_renders(sc, 64, seed=0)   # seeded


def test_furnace_and_pixel_subsets():
    sc = scenes.furnace_box(L=8)
    _closed_mesh_ok(sc)
    assert all(m.kind == scenes.DIFFUSE_EMITTER for m in sc.materials)
    p = scenes.pixel_subset(64, 48, 500, seed=3)
    assert len(p) == 500 and len(np.unique(p)) == 500 and p.min() >= 0 and p.max() < 64 * 48
    assert np.all(np.diff(p) > 0) and np.array_equal(p, scenes.pixel_subset(64, 48, 500, seed=3))
