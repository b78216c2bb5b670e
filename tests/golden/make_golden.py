"""Write the stored expected values under tests/golden/ from the FP64 oracle
(the only source of stored values besides the paper, which prints no worked
example). Run from the repository root:  python tests/golden/make_golden.py

* c1_tiny_room_64x64_1spp_d2_L16.txt -- the tiny-room workload (38 triangles,
  4 mm pane at s = 0.5, 64 x 64 px, 1 spp, depth 2, 16 bins, Philox seed 0,
  scene seed 0): XYZ of every 8th pixel, with the oracle's decision margin and
  minimum NEE cosine of each pixel's sample.
* slab_rt.txt -- exact absorbing-slab R, T (the slab model of Sec. 6's glass)
  at a grid of (cos, n, k from alpha, thickness), on the oracle's formula.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1912_06474_gb300 import scenes  # noqa: E402


def c1_rows():
    sc = scenes.tiny_room(L=16, seed=0)
    spec = scenes.RenderSpec(64, 64, 1, 2, seed=0, camera=sc.camera)
    pix = np.arange(0, 64 * 64, 8, dtype=np.int64)
    r = oracle.Oracle(sc).render_pixels(spec, pix, per_sample=True, brute_force=True)
    return pix, r["xyz"], r["margin"][:, 0], r["cos_min"][:, 0]


def slab_rows():
    rows = []
    for c in (1.0, 0.8, 0.5, 0.2, 0.05):
        for n in (1.45, 1.52, 1.7):
            for alpha in (0.0, 50.0, 400.0):
                for d in (0.002, 0.004, 0.010):
                    lam = 550.0
                    R, T = oracle.slab(c, lam, n, alpha, d)
                    rows.append((c, lam, n, alpha, d, R, T))
    return rows


def main():
    pix, xyz, margin, cmin = c1_rows()
    with open(os.path.join(HERE, "c1_tiny_room_64x64_1spp_d2_L16.txt"), "w") as f:
        f.write("# tiny room, 64x64 px, 1 spp, depth 2, 16 bins, Philox seed 0, scene seed 0 (FP64 oracle, brute force)\n")
        f.write("# pixel X Y Z margin cos_min\n")
        for p, v, m, cm in zip(pix, xyz, margin, cmin):
            f.write(f"{p} {v[0]:.17g} {v[1]:.17g} {v[2]:.17g} {m:.6g} {cm:.6g}\n")
    with open(os.path.join(HERE, "slab_rt.txt"), "w") as f:
        f.write("# exact absorbing slab (FP64 oracle): cos lambda_nm n alpha_per_m thickness_m R T\n")
        for row in slab_rows():
            f.write(" ".join(f"{x:.17g}" for x in row) + "\n")


if __name__ == "__main__":
    main()
