"""A ray that leaves its subdomain without a hit is either handed to the
neighbour's queue for the next wave (Sec. 5's interface exchange) or carried
on by the same lane into the neighbour's BVH within the wave; the mixed
schedule hands rays over for the first waves of a bounce and then carries
the rest. All schedules trace each ray through the same subdomains with the
same hit windows, so images, segment and crossing counts are identical; the
throughput of each is printed."""
import pytest

from paper_1912_06474_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]

SCHEDULES = {"queue hand-off": {}, "lane continues": dict(continue_cells=True),
             "1 queue wave, then the lane": dict(handoff_waves=1),
             "2 queue waves, then the lane": dict(handoff_waves=2)}


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
    for name, opts in SCHEDULES.items():
        ctx.build(grid=grid, **opts)
        ctx.render([spec], method="ddm")
        imgs, s = ctx.render([spec], method="ddm")
        out[name], st[name] = imgs[0].clone(), s
        rate[name] = (s["segments_ext"] + s["segments_shadow"]) / (s["gpu_ms"] * 1e3)
    print(f"{which} {grid}: " + ", ".join(f"{k} {v:.0f} Mseg/s" for k, v in rate.items()))
    ref = "queue hand-off"
    for name in SCHEDULES:
        assert torch.equal(out[ref], out[name]), name
        for k in ("segments_ext", "segments_shadow", "crossings", "glass_queries"):
            assert st[ref][k] == st[name][k], (name, k)
    with pytest.raises(sddm.SddmError):
        ctx.build(grid=grid, continue_cells=True, cell_cache_bytes=1 << 30)
    with pytest.raises(sddm.SddmError):
        ctx.build(grid=grid, handoff_waves=2, cell_cache_bytes=1 << 30)
    with pytest.raises(sddm.SddmError):
        ctx.build(grid=grid, handoff_waves=2, continue_cells=True)
    ctx.close()


def test_carried_crossings_are_counted():
    """The counting trace kernel splits interface crossings into hand-offs
    through a neighbour's queue and crossings the tracing thread carries on
    itself: none carried with the queue in every wave, all of them with the
    lane carrying rays from the first wave, some with one queue wave."""
    from paper_1912_06474_gb300 import sddm
    sc = scenes.hotel_room(L=41, seed=0)
    spec = scenes.hotel_room_render(sc, 128, 128, 4, 5, seed=0)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    ctx.set_profiling(count_traversal=True)
    got = {}
    for name, opts in (("queue", {}), ("lane", dict(continue_cells=True)), ("mixed", dict(handoff_waves=1))):
        ctx.build(grid=(4, 4, 2), **opts)
        _, s = ctx.render([spec], method="ddm")
        got[name] = (s["crossings"], s["ray_continues"])
    ctx.close()
    crossings = got["queue"][0]
    assert crossings > 0 and all(c == crossings for c, _ in got.values())
    assert got["queue"][1] == 0
    assert got["lane"][1] == crossings
    assert 0 < got["mixed"][1] < crossings
    print("crossings", crossings, "carried by the thread with one queue wave:", got["mixed"][1])
