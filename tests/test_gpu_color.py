"""RGB -> spectrum on the GPU (Matrice-R fundamental) against the FP64
oracle, and the paper's accuracy check: spectra computed from representative
RGB values convert back to the same RGB."""
import numpy as np
import pytest

from paper_1912_06474_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.mark.parametrize("L", [16, 41, 81])
def test_rgb_to_spectrum_matches_oracle(oracle_mod, L):
    from paper_1912_06474_gb300 import sddm
    sc = scenes.tiny_room(L=L, seed=0)
    ctx = sddm.Context(0)
    ctx.set_scene(sc)
    rng = np.random.default_rng(L)
    rgb = rng.uniform(0.02, 0.98, (5000, 3)).astype(np.float32)
    for clamp in (False, True):
        got = ctx.rgb_to_spectrum(rgb, clamp=clamp).astype(np.float64)
        want = oracle_mod.rgb_to_spectrum(rgb.astype(np.float64), sc.quad_w, sc.cmf, clamp=clamp)
        err = np.abs(got - want).max()
        assert err <= 2e-6 * max(1.0, np.abs(want).max()), err
        back = oracle_mod.spectrum_to_rgb(got, sc.quad_w, sc.cmf)
        if not clamp:
            assert np.abs(back - rgb).max() <= 1e-5
        else:
            free = oracle_mod.rgb_to_spectrum(rgb.astype(np.float64), sc.quad_w, sc.cmf, clamp=False)
            ok = np.all((free >= 0) & (free <= 1), axis=1)
            assert np.abs(back[ok] - rgb[ok]).max() <= 1e-5
            print(f"L={L}: {ok.mean():.1%} of the RGB values have a physical fundamental")
    ctx.close()
