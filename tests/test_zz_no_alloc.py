"""sddm_render_noalloc, the render entry point that allocates no memory.

It is for callers that cannot call cudaMalloc while they render (an
application whose own pool allocator owns the device memory, or a render loop
that has no time for the allocator); its scratch is a fixed device array
inside the library. Two calls in a row, of
different sizes, must each match what sddm_render produces for the same
render, so nothing left in the shared array from a previous call leaks into
the next, and the second call must leave the device's free memory exactly
as it was. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1912_06474_gb300 import scenes
from tests.helpers import rel_rmse, sample_mismatch

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


def test_noalloc_matches_render_twice():
    from paper_1912_06474_gb300 import sddm
    sc = scenes.tiny_room(L=16)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    ctx.build()
    g = sc.glass_materials()[0]
    specs = [scenes.RenderSpec(64, 48, 4, 3, seed=5, camera=sc.camera, glass_s={g: 0.8}),
             scenes.RenderSpec(40, 40, 2, 5, seed=6, camera=sc.camera)]
    for i, spec in enumerate(specs):
        ref, _ = ctx.render([spec], method="megakernel")
        out = torch.full((spec.height, spec.width, 3), float("nan"), device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = ctx.render_noalloc(spec, out)
        torch.cuda.synchronize()
        if i > 0:
            # after the first call (which loads the kernels and looks up the
            # scratch address), a call of another size allocates nothing
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy().reshape(-1, 3)
        want = ref[0].cpu().numpy().reshape(-1, 3)
        assert np.isfinite(got).all()
        assert not sample_mismatch(got, want, np.ones(len(want), bool), 1e-5).any()
        assert rel_rmse(got, want) <= 1e-6
        assert st["segments_ext"] >= spec.n_paths
    too_big = scenes.RenderSpec(1024, 1024, 2, 2, camera=sc.camera)
    out = torch.empty((1024, 1024, 3), device="cuda")
    with pytest.raises(sddm.SddmError) as e:
        ctx.render_noalloc(too_big, out)
    assert e.value.code == sddm.ERR_INVALID_ARG and "scratch" in str(e.value)
    ctx.close()
