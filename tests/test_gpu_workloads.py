"""Full-size workloads on the GPU, checked on seeded pixel subsets the FP64
oracle computes pixel by pixel (the counter-based random stream makes any
subset exact).

* hotel room, 512 x 512 x 16 spp, depth 5, 41 bins: the configuration the
  benchmark times (DDM 4x4x2), the megakernel, and DDM with the surrogate;
* 64 batched renders of the tiny room (resolution ~ U{128..1024}^2,
  spp ~ U{4,16,64}, s ~ U[0,1]) in one call, after the autotuner;
* the tiny room at 1024 x 1024 x 64 spp with the surrogate and the exact slab.
Acceptance: relative RMSE over the subset <= 1e-3.
"""
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
def hotel():
    return scenes.hotel_room(L=41, seed=0)


@pytest.fixture(scope="module")
def hotel_ref(oracle_mod, hotel):
    spec = scenes.hotel_room_render(hotel, 512, 512, 16, 5, seed=0)
    pix = scenes.pixel_subset(512, 512, 2048, seed=1)
    ref = oracle_mod.Oracle(hotel).render_pixels(spec, pix)
    return spec, pix, ref["xyz"]


@pytest.mark.parametrize("method,grid,bsdf", [("ddm", (4, 4, 2), "exact"), ("megakernel", (1, 1, 1), "exact"),
                                              ("ddm", (4, 4, 2), "mlp")])
def test_hotel_room_full_size(sddm, hotel, hotel_ref, method, grid, bsdf):
    spec, pix, ref = hotel_ref
    ctx = sddm.Context(0)
    ctx.set_scene(hotel)
    ctx.build(grid=grid)
    if bsdf == "mlp":
        ctx.mlp_train(hotel.glass_materials()[0], seed=7)
    imgs, st = ctx.render([spec], method=method, bsdf=bsdf)
    got = imgs[0].cpu().numpy().reshape(-1, 3)[pix]
    e = rel_rmse(got, ref)
    print(f"hotel {method} {bsdf}: rel-RMSE on {len(pix)} px = {e:.2e}, segments "
          f"{st['segments_ext'] + st['segments_shadow']}, fallbacks {st['mlp_fallbacks']}")
    assert e <= 1e-3
    ctx.close()


def test_batched_64_renders_autotuned(oracle_mod, sddm):
    sc = scenes.tiny_room(L=41, seed=0)
    specs = scenes.batched_renders(sc, 64, seed=0, max_depth=5)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    best = ctx.autotune(specs, method="ddm")
    print("autotuned:", best)
    assert tuple(best["grid"]) in {(1, 1, 1), (2, 2, 2), (4, 4, 2), (8, 4, 4)}
    imgs, st = ctx.render(specs, method="ddm")
    print(f"64 renders: {st['paths']} paths, {st['segments_ext'] + st['segments_shadow']} segments, "
          f"{st['gpu_ms']:.1f} ms")
    orc = oracle_mod.Oracle(sc)
    errs = []
    for r in range(0, 64, 4):
        sp = specs[r]
        pix = scenes.pixel_subset(sp.width, sp.height, 256, seed=r)
        ref = orc.render_pixels(sp, pix)["xyz"]
        got = imgs[r].cpu().numpy().reshape(-1, 3)[pix]
        errs.append(rel_rmse(got, ref))
    print("per-render rel-RMSE max", max(errs))
    assert max(errs) <= 1e-3
    ctx.close()


def test_tiny_room_1024_64spp_surrogate_vs_exact(oracle_mod, sddm):
    sc = scenes.tiny_room(L=41, seed=0)
    spec = scenes.RenderSpec(1024, 1024, 64, 5, seed=0, camera=sc.camera)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    ctx.build(grid=(2, 2, 2))
    rep = ctx.mlp_train(sc.glass_materials()[0], seed=7)
    pix = scenes.pixel_subset(1024, 1024, 1024, seed=2)
    # pixels looking through the pane are where the glass model matters
    centre = np.array([(512 + dy) * 1024 + 512 + dx for dy in range(-64, 64, 8) for dx in range(-64, 64, 8)])
    pix = np.unique(np.concatenate([pix, centre]))
    ref = oracle_mod.Oracle(sc).render_pixels(spec, pix)["xyz"]
    out = {}
    for bsdf in ("exact", "mlp"):
        imgs, st = ctx.render([spec], method="ddm", bsdf=bsdf)
        got = imgs[0].cpu().numpy().reshape(-1, 3)[pix]
        out[bsdf] = (rel_rmse(got, ref), st["gpu_ms"], st["segments_ext"] + st["segments_shadow"],
                     st["mlp_fallbacks"])
    print("surrogate training", rep)
    print("1024^2 x 64 spp: exact rel-RMSE %.2e %.1f ms %d seg; surrogate rel-RMSE %.2e %.1f ms %d seg, "
          "%d fallback batches" % (*out["exact"][:3], *out["mlp"]))
    assert out["exact"][0] <= 1e-3 and out["mlp"][0] <= 1e-3
    ctx.close()
