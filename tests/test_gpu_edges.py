"""Edge cases of the GPU path, each against the FP64 oracle or a closed form:

* the largest subdomain grid (2048 cells) and a grid finer along one axis;
* an orthographic camera whose rays run exactly along the x axis (zero
  direction components: the grid entry and exit skip those axes);
* a single-pixel, single-sample render and a 2-bin spectrum;
* the deepest path (64 vertices) in the white furnace, against its closed form;
* a scene without any light (every pixel exactly black);
* a camera outside the scene box (rays enter the grid from outside).
"""
import dataclasses

import numpy as np
import pytest

from paper_1912_06474_gb300 import scenes
from tests.helpers import rel_rmse

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module")
def sddm():
    from paper_1912_06474_gb300 import sddm as m
    return m


@pytest.fixture(scope="module")
def room():
    return scenes.tiny_room(L=16, seed=0)


def _check(sddm, oracle_mod, sc, spec, grids, tol=1e-3):
    ref = oracle_mod.Oracle(sc).render_pixels(spec, brute_force=True)["xyz"]
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    out = {}
    for method, grid in grids:
        ctx.build(grid=grid)
        imgs, st = ctx.render([spec], method=method)
        e = rel_rmse(imgs[0].cpu().numpy().reshape(-1, 3), ref) if np.linalg.norm(ref) > 0 else \
            float(np.abs(imgs[0].cpu().numpy()).max())
        out[(method, grid)] = e
        assert e <= tol, (method, grid, e)
    ctx.close()
    return out


def test_largest_grid_and_skewed_grids(sddm, oracle_mod, room):
    spec = scenes.RenderSpec(48, 36, 2, 4, seed=5, camera=room.camera)
    print(_check(sddm, oracle_mod, room, spec,
                 [("ddm", (16, 16, 8)), ("ddm", (64, 1, 1)), ("ddm", (1, 32, 2)), ("megakernel", (1, 1, 1))]))


def test_axis_aligned_orthographic_rays(sddm, oracle_mod, room):
    cam = scenes.Camera(pos=(0.3, 2.0, 1.5), look=(1.3, 2.0, 1.5), up=(0.0, 0.0, 1.0), ortho_height=2.5)
    spec = scenes.RenderSpec(40, 40, 1, 4, seed=6, camera=cam)
    print(_check(sddm, oracle_mod, room, spec, [("ddm", (4, 4, 2)), ("ddm", (1, 1, 1)), ("megakernel", (1, 1, 1))]))


def test_single_pixel_and_two_bins(sddm, oracle_mod):
    sc = scenes.tiny_room(L=2, seed=2)   # the generator needs two bins at least
    for W, H, spp in ((1, 1, 1), (3, 1, 5), (1, 7, 2)):
        spec = scenes.RenderSpec(W, H, spp, 5, seed=7, camera=sc.camera)
        _check(sddm, oracle_mod, sc, spec, [("ddm", (2, 2, 2)), ("megakernel", (1, 1, 1))])


@pytest.mark.parametrize("method,grid", [("megakernel", (1, 1, 1)), ("ddm", (2, 2, 1))])
def test_deepest_paths_white_furnace(sddm, method, grid):
    rho0, Le0, D = 0.9, 0.5, 64
    sc = scenes.furnace_box(L=8, rho0=rho0, Le0=Le0)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    ctx.build(grid=grid)
    spec = scenes.RenderSpec(8, 8, 2, D, seed=1, camera=sc.camera, nee=False)
    imgs, st = ctx.render([spec], method=method)
    Le0, rho0 = float(np.float32(Le0)), float(np.float32(rho0))
    want = Le0 * sum(rho0 ** j for j in range(D)) * (sc.quad_w.astype(np.float64)[:, None]
                                                     * sc.cmf.astype(np.float64)).sum(0)
    got = imgs[0].cpu().numpy().reshape(-1, 3)
    assert np.allclose(got, want, rtol=2e-5), (got[0], want)
    assert st["segments_ext"] == 8 * 8 * 2 * D
    ctx.close()


def test_scene_without_lights(sddm, oracle_mod, room):
    mats = [dataclasses.replace(m, kind=scenes.LAMBERT, rho=np.full(room.L, 0.5, np.float32), Le=None)
            if m.kind in (scenes.EMITTER, scenes.DIFFUSE_EMITTER) else m for m in room.materials]
    dark = dataclasses.replace(room, materials=mats)
    spec = scenes.RenderSpec(24, 24, 2, 4, seed=8, camera=room.camera)
    ctx = sddm.Context(0)
    ctx.set_scene(dark)
    for method, grid in (("ddm", (2, 2, 2)), ("megakernel", (1, 1, 1))):
        ctx.build(grid=grid)
        imgs, st = ctx.render([spec], method=method)
        assert float(imgs[0].abs().max()) == 0.0
        assert st["segments_shadow"] == 0
    ctx.close()
    ref = oracle_mod.Oracle(dark).render_pixels(spec)["xyz"]
    assert np.abs(ref).max() == 0.0


def test_camera_outside_the_scene_box(sddm, oracle_mod):
    """A triangle soup with a fifth of its triangles emitting, seen from outside
    its bounding box: every camera ray enters the subdomain grid from outside."""
    sc = scenes.random_soup(400, seed=3)
    rng = np.random.default_rng(3)
    mats = [sc.materials[0], scenes.Material(scenes.EMITTER, Le=np.full(sc.L, 2.0, np.float32), name="glow")]
    mat_id = (rng.uniform(0, 1, sc.n_tris) < 0.2).astype(np.uint32)
    cam = scenes.Camera(pos=(-2.5, 0.3, 0.2), look=(0.5, 0.5, 0.5), up=(0.0, 0.0, 1.0), vfov_deg=40.0)
    sc = dataclasses.replace(sc, materials=mats, mat_id=mat_id, camera=cam)
    spec = scenes.RenderSpec(32, 32, 2, 3, seed=9, camera=cam)
    print(_check(sddm, oracle_mod, sc, spec, [("ddm", (4, 4, 4)), ("megakernel", (1, 1, 1))]))
