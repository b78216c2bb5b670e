"""Glass coated with a thin-film electrochromic stack on the GPU (the
multilayer extension of the slab model): the kernels' transfer-matrix R, T
against the FP64 oracle, rendered images against the oracle with the exact
model and with a surrogate trained on it, and what the surrogate gains over
evaluating the stack exactly (per evaluation and per render)."""
import time

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
    return scenes.tiny_room(L=41, seed=0, coated=True)


def _rows(sc, g, n, seed):
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 1.0, n).astype(np.float32)
    b = rng.integers(0, sc.L, n).astype(np.int32)
    s = rng.uniform(0, 1, n).astype(np.float32)
    d = np.full(n, sc.materials[g].thickness_m, np.float32)
    return c, b, s, d


def test_coated_glass_eval_matches_oracle(oracle_mod, sddm, room):
    ctx = sddm.Context(0)
    ctx.set_scene(room)
    ctx.build()
    g = room.glass_materials()[0]
    m = room.materials[g]
    c, b, s, d = _rows(room, g, 4000, 1)
    R, T = ctx.glass_eval(g, *(torch.from_numpy(a).cuda() for a in (c, b, s, d)), mode="exact")
    R, T = R.cpu().numpy(), T.cpu().numpy()
    eR, eT = [], []
    for q in range(len(c)):
        i = b[q]
        films = [(float(f["n"][i]), float(np.float32(f["k"][i]) + np.float32(s[q]) * np.float32(f["dk"][i])),
                  float(np.float32(f["t_nm"]))) for f in m.layers]
        alpha = float(np.float32(m.alpha_clear[i]) + np.float32(s[q]) * np.float32(m.dalpha[i]))
        r, t = oracle_mod.coated_slab(c[q], room.lam[i], m.n[i], alpha, d[q], films)
        eR.append(abs(R[q] - r))
        eT.append(abs(T[q] - t))
    eR, eT = np.array(eR), np.array(eT)
    print(f"coated glass FP32 vs FP64: |dR| max {eR.max():.2e} mean {eR.mean():.2e}, "
          f"|dT| max {eT.max():.2e} mean {eT.mean():.2e}")
    assert eR.max() < 1e-4 and eT.max() < 1e-4
    assert eR.mean() < 1e-5 and eT.mean() < 1e-5
    ctx.close()


@pytest.mark.parametrize("method,grid", [("ddm", (2, 2, 2)), ("megakernel", (1, 1, 1))])
def test_coated_room_image(oracle_mod, sddm, room, method, grid):
    spec = scenes.RenderSpec(64, 64, 4, 5, seed=3, camera=room.camera)
    ref = oracle_mod.Oracle(room).render_pixels(spec)["xyz"]
    ctx = sddm.Context(0)
    ctx.set_scene(room)
    ctx.build(grid=grid)
    imgs, _ = ctx.render([spec], method=method)
    e = rel_rmse(imgs[0].cpu().numpy().reshape(-1, 3), ref)
    print(f"coated room {method}: rel-RMSE {e:.2e}")
    assert e <= 1e-3
    ctx.close()


def test_surrogate_on_coated_glass(oracle_mod, sddm, room):
    """Train the surrogate on the coated stack; images with it stay within the
    tolerance; print what it gains over the exact stack, per evaluation
    (4M rows through the test hook) and per render (tiny room 512^2 x 16 spp)."""
    ctx = sddm.Context(0)
    ctx.set_scene(room)
    ctx.build(grid=(2, 2, 2))
    g = room.glass_materials()[0]
    rep = ctx.mlp_train(g, seed=7)
    print("surrogate on coated glass:", rep)
    assert rep["final_loss"] < 1e-3
    # per-evaluation cost and accuracy
    c, b, s, d = _rows(room, g, 1 << 22, 2)
    args = [torch.from_numpy(a).cuda() for a in (c, b, s, d)]
    times = {}
    out = {}
    for mode in ("exact", "mlp_raw", "mlp"):
        ctx.glass_eval(g, *args, mode=mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            out[mode] = ctx.glass_eval(g, *args, mode=mode)
        torch.cuda.synchronize()
        times[mode] = (time.perf_counter() - t0) / 5
    eT = (out["mlp_raw"][1] - out["exact"][1]).abs()
    print("4M evaluations: exact stack %.3f ms, surrogate %.3f ms (probe + fallback %.3f ms); "
          "raw |dT| mean %.2e" % (1e3 * times["exact"], 1e3 * times["mlp_raw"], 1e3 * times["mlp"],
                                  eT.mean().item()))
    assert eT.mean().item() < 1e-2
    # images
    spec = scenes.RenderSpec(64, 64, 4, 5, seed=3, camera=room.camera)
    ref = oracle_mod.Oracle(room).render_pixels(spec)["xyz"]
    imgs, st = ctx.render([spec], method="ddm", bsdf="mlp")
    e = rel_rmse(imgs[0].cpu().numpy().reshape(-1, 3), ref)
    print(f"coated room with surrogate: rel-RMSE {e:.2e}, fallback batches {st['mlp_fallbacks']}")
    assert e <= 1e-3
    big = scenes.RenderSpec(512, 512, 16, 5, seed=0, camera=room.camera)
    ms = {}
    for bsdf in ("exact", "mlp"):
        ctx.render([big], method="ddm", bsdf=bsdf)
        _, st = ctx.render([big], method="ddm", bsdf=bsdf)
        ms[bsdf] = st["gpu_ms"]
    print("tiny room coated, 512^2 x 16 spp: exact stack %.2f ms, surrogate %.2f ms (%.2fx)"
          % (ms["exact"], ms["mlp"], ms["exact"] / ms["mlp"]))
    ctx.close()


def test_surrogate_gain_against_film_count(sddm):
    """What the trained network gains over the exact stack as the stack grows:
    4M (cos, bin, s) rows of a pane coated with 1, 3, 6 and 10 films, device
    time of the exact transfer-matrix stack against the network alone and
    against the served surrogate (network, per-batch probe and exact
    fallback), the network retrained on each stack. Measured on a GB300:

    * the exact stack's cost grows with the films, the network's does not;
    * the network alone is cheaper than the exact stack from 6 films on;
    * the served surrogate is not cheaper at any of these counts: the thicker
      stacks' interference fringes in angle and wavelength are harder for the
      4-64-64-64-2 network to fit, and the batches whose probe fails pay for
      the network and the exact stack both."""
    films = (1, 3, 6, 10)
    res = {}
    for J in films:
        room = scenes.tiny_room(L=41, seed=0, coated=True, n_films=J)
        ctx = sddm.Context(0)
        try:
            ctx.set_scene(room)
            ctx.build(grid=(1, 1, 1))
            g = room.glass_materials()[0]
            rep = ctx.mlp_train(g, seed=7)
            c, b, s, d = _rows(room, g, 1 << 22, 2)
            args = [torch.from_numpy(a).cuda() for a in (c, b, s, d)]
            t = {}
            out = {}
            for mode in ("exact", "mlp_raw", "mlp"):
                ctx.glass_eval(g, *args, mode=mode)
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                ev[0].record()
                for _ in range(5):
                    out[mode] = ctx.glass_eval(g, *args, mode=mode)
                ev[1].record()
                torch.cuda.synchronize()
                t[mode] = ev[0].elapsed_time(ev[1]) / 5
            dT = (out["mlp"][1] - out["exact"][1]).abs()
            served_exact = (out["mlp"][1] != out["mlp_raw"][1]).float().mean().item()
            res[J] = t
            print(f"{J:2d} films: exact {t['exact']:.3f} ms, network {t['mlp_raw']:.3f} ms, served surrogate "
                  f"{t['mlp']:.3f} ms ({served_exact:.0%} of rows by the exact fallback); served |dT| mean "
                  f"{dT.mean().item():.2e}; training loss {rep['final_loss']:.1e}")
            assert dT.mean().item() <= 1e-3
        finally:
            ctx.close()
    assert res[10]["exact"] > 3.0 * res[1]["exact"]
    assert res[10]["mlp_raw"] < 1.3 * res[1]["mlp_raw"]
    net_wins = [J for J in films if res[J]["mlp_raw"] < res[J]["exact"]]
    served_wins = [J for J in films if res[J]["mlp"] < res[J]["exact"]]
    print(f"network alone cheaper than the exact stack at {net_wins} films; served surrogate at {served_wins}")
    assert net_wins == [6, 10]
    assert served_wins == []
