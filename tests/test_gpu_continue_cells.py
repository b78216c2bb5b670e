"""A ray that leaves its subdomain without a hit is either handed to the
neighbour's queue for the next wave (Sec. 5's interface exchange) or carried
on by the same lane into the neighbour's BVH within the wave. The two
schedules trace each ray through the same subdomains with the same hit
windows, so images, segment and crossing counts are identical; the
throughput of both is printed."""
import pytest

from paper_1912_06474_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.mark.parametrize("which,grid", [("tiny", (2, 2, 2)), ("hotel", (4, 4, 2))])
def test_continue_across_cells_matches_queue_handoff(which, grid):
    from paper_1912_06474_gb300 import sddm
    if which == "tiny":
        sc = scenes.tiny_room(L=16)
        spec = scenes.RenderSpec(96, 64, 4, 5, seed=2, camera=sc.camera)
    else:
        sc = scenes.hotel_room(L=41, seed=0)
        spec = scenes.hotel_room_render(sc, 256, 256, 8, 5, seed=0)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    out, st, rate = {}, {}, {}
    for cont in (False, True):
        ctx.build(grid=grid, continue_cells=cont)
        ctx.render([spec], method="ddm")
        imgs, s = ctx.render([spec], method="ddm")
        out[cont], st[cont] = imgs[0].clone(), s
        rate[cont] = (s["segments_ext"] + s["segments_shadow"]) / (s["gpu_ms"] * 1e3)
    print(f"{which} {grid}: queue hand-off {rate[False]:.0f} Mseg/s, lane continues {rate[True]:.0f} Mseg/s")
    assert torch.equal(out[False], out[True])
    for k in ("segments_ext", "segments_shadow", "crossings", "glass_queries"):
        assert st[False][k] == st[True][k], k
    with pytest.raises(sddm.SddmError):
        ctx.build(grid=grid, continue_cells=True, cell_cache_bytes=1 << 30)
    ctx.close()
