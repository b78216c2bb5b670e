"""Subdomains loaded into a device cache under a byte budget and unloaded when
their rays have run out (Sec. 5: each process loads subdomains up to its
memory limit). The facade room's 256 subdomain BVHs (~0.6 GB) are traced
through a cache of about a fifth of that, so that every wave evicts and
reloads cells; the images must be bit-identical to the all-resident build,
with the hit rate and the throughput printed. A budget below the largest
subdomain is rejected, and photon maps refuse the cache."""
import pytest

from paper_1912_06474_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def test_cell_cache_small_scene_all_cells_fit():
    """The hotel room's 32 subdomains in a cache that holds them all: loaded
    once each, hits afterwards, images equal to the resident build."""
    from paper_1912_06474_gb300 import sddm
    sc = scenes.hotel_room(L=41, seed=0)
    spec = scenes.hotel_room_render(sc, 128, 128, 4, 5, seed=0)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    ctx.build(grid=(4, 4, 2))
    ref, _ = ctx.render([spec], method="ddm")
    ctx.build(grid=(4, 4, 2), cell_cache_bytes=256 << 20)
    got, st = ctx.render([spec], method="ddm")
    assert torch.equal(ref[0], got[0])
    assert 0 < st["cache_loads"] <= 32 and st["cache_hits"] > st["cache_loads"]
    ctx.close()


def test_cell_cache_evicts_and_matches_resident_build():
    from paper_1912_06474_gb300 import sddm
    sc = scenes.facade_room(L=81, seed=0)
    specs = scenes.facade_renders(sc, n_renders=2, width=480, height=270, spp=4, max_depth=8)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    ctx.build(grid=(8, 8, 4))
    ctx.render(specs, method="ddm")
    ref, st0 = ctx.render(specs, method="ddm")
    rate0 = (st0["segments_ext"] + st0["segments_shadow"]) / (st0["gpu_ms"] * 1e3)
    budget = 128 << 20
    ctx.build(grid=(8, 8, 4), cell_cache_bytes=budget)
    got, st = ctx.render(specs, method="ddm")
    rate = (st["segments_ext"] + st["segments_shadow"]) / (st["gpu_ms"] * 1e3)
    uses = st["cache_loads"] + st["cache_hits"]
    print(f"facade 8x8x4, cache {budget >> 20} MiB: {st['cache_loads']} loads ({st['cache_bytes_loaded'] / 1e9:.2f} GB), "
          f"{st['cache_hits']} hits ({st['cache_hits'] / max(uses, 1):.1%}); {rate:.0f} Mseg/s against "
          f"{rate0:.0f} all resident")
    for a, b in zip(ref, got):
        assert torch.equal(a, b)
    assert st["segments_ext"] == st0["segments_ext"] and st["crossings"] == st0["crossings"]
    # 256 cells do not fit: cells are loaded more often than there are cells, and some stay resident
    assert st["cache_loads"] > 256 and st["cache_hits"] > 0
    # a second call finds the cache as the first left it and renders the same image
    got2, _ = ctx.render(specs[:1], method="ddm")
    assert torch.equal(got2[0], ref[0])
    with pytest.raises(sddm.SddmError):
        ctx.render_photon_map(specs[0], 1000, 0.1, method="ddm")
    with pytest.raises(sddm.SddmError) as e:
        ctx.build(grid=(8, 8, 4), cell_cache_bytes=1 << 16)
    assert e.value.code == sddm.ERR_INVALID_ARG and "largest subdomain" in str(e.value)
    ctx.close()
