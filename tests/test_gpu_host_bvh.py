"""Subdomain BVHs kept in host memory and read by the trace kernel over the
coherent host link (the option for scenes whose subdomains exceed HBM): the
images are bit-identical to the HBM-resident build, and the cost of reading
nodes and triangles from host memory is printed for the hotel room (BVH set in
L2) and the 5 M-triangle facade (BVH set larger than L2)."""
import pytest

from paper_1912_06474_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.mark.parametrize("which", ["hotel", "facade"])
def test_host_resident_subdomain_bvhs(which):
    from paper_1912_06474_gb300 import sddm
    if which == "hotel":
        sc = scenes.hotel_room(L=41, seed=0)
        spec = scenes.hotel_room_render(sc, 256, 256, 8, 5, seed=0)
        grid = (4, 4, 2)
    else:
        sc = scenes.facade_room(L=81, seed=0)
        spec = scenes.facade_renders(sc, n_renders=1, width=960, height=540, spp=2, max_depth=8)[0]
        grid = (8, 8, 4)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    out, rate = {}, {}
    for host in (False, True):
        ctx.build(grid=grid, bvh_in_host_memory=host)
        ctx.render([spec], method="ddm")
        imgs, st = ctx.render([spec], method="ddm")
        out[host] = imgs[0].clone()
        rate[host] = (st["segments_ext"] + st["segments_shadow"]) / (st["gpu_ms"] * 1e3)
    print(f"{which}: subdomain BVHs in HBM {rate[False]:.0f} Mseg/s, in host memory {rate[True]:.0f} Mseg/s")
    assert torch.equal(out[False], out[True])
    ctx.close()
