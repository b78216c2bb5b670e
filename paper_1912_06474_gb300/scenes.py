"""Seeded synthetic scenes: the input data for the spectral DDM path tracer.

This module produces INPUTS only: wavelength bins, quadrature weights, colour
matching functions, material curves (reflectance, complex index n + ik of
metals, Cauchy index and absorption curves of glass, emission spectra),
triangle meshes, cameras and render descriptions. It contains none of the
method's arithmetic (no Fresnel, no slab model, no intersection, no transport)
and imports nothing else from this package, so the CUDA path and the FP64
oracle can both be fed from it without sharing any of the computation.

Scenes stand in for the paper's hotel room (Sec. 6), whose geometry, measured
BK7 data and spectra are not available:

* ``tiny_room``      -- 5x4x3 m box room, one freestanding 4 mm pane, one cube,
                        one 1x1 m ceiling light (38 triangles).
* ``hotel_room``     -- 6x4x3 m room, 40 boxes, 100 tessellated spheres
                        (2000 triangles each, 20 of them metallic), two
                        photochromic window panes lit from behind (~200.5k tris).
* ``facade_room``    -- 12x8x3 m room with seeded furniture meshes up to a
                        target triangle count and 8 electrochromic panes.
* ``furnace_box``    -- closed box whose every face is emissive + Lambertian.

All curves are drawn with ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

LAMBDA_MIN_NM = 380.0
LAMBDA_MAX_NM = 780.0

# Material kinds (same integer codes on every consumer of these inputs).
LAMBERT = 0
CONDUCTOR = 1
GLASS = 2
EMITTER = 3           # one-sided emitter, black to reflection
DIFFUSE_EMITTER = 4   # one-sided emitter that is also Lambertian


# --------------------------------------------------------------------------
# Spectral inputs
# --------------------------------------------------------------------------
def wavelengths(L: int) -> np.ndarray:
    """L bins evenly spaced over [380, 780] nm (10 nm for L=41, 5 nm for L=81)."""
    if L < 2:
        raise ValueError("need at least two wavelength bins")
    return np.linspace(LAMBDA_MIN_NM, LAMBDA_MAX_NM, L).astype(np.float32)


def trapezoid_weights(lam: np.ndarray) -> np.ndarray:
    """Trapezoidal quadrature weights (nm) for an increasing wavelength grid."""
    lam = np.asarray(lam, dtype=np.float64)
    w = np.zeros_like(lam)
    d = np.diff(lam)
    w[:-1] += 0.5 * d
    w[1:] += 0.5 * d
    return w.astype(np.float32)


def _lobe(lam, mu, s_lo, s_hi):
    s = np.where(lam < mu, s_lo, s_hi)
    t = (lam - mu) / s
    return np.exp(-0.5 * t * t)


def cmf_xyz(lam: np.ndarray) -> np.ndarray:
    """CIE 1931 2-degree colour matching functions, [L][3].

    The CIE tables are not available offline; this is the analytic multi-lobe
    piecewise-Gaussian fit published by Wyman, Sloan and Shirley (JCGT 2(2),
    2013), evaluated at the bin centres. It is an input table: both the CUDA
    path and the oracle receive the same float32 values.
    """
    lam = np.asarray(lam, dtype=np.float64)
    x = (1.056 * _lobe(lam, 599.8, 37.9, 31.0) + 0.362 * _lobe(lam, 442.0, 16.0, 26.7)
         - 0.065 * _lobe(lam, 501.1, 20.4, 26.2))
    y = 0.821 * _lobe(lam, 568.8, 46.9, 40.5) + 0.286 * _lobe(lam, 530.9, 16.3, 31.1)
    z = 1.217 * _lobe(lam, 437.0, 11.8, 36.0) + 0.681 * _lobe(lam, 459.0, 26.0, 13.8)
    return np.stack([x, y, z], axis=1).astype(np.float32)


def planck_normalised(lam: np.ndarray, temperature_k: float = 5800.0,
                      scale: float = 1.0) -> np.ndarray:
    """Black-body radiance at ``temperature_k``, peak over 380-780 nm equal to ``scale``."""
    h, c, kb = 6.62607015e-34, 2.99792458e8, 1.380649e-23

    def B(l_nm):
        l = np.asarray(l_nm, dtype=np.float64) * 1e-9
        return 1.0 / (l ** 5 * (np.exp(h * c / (l * kb * temperature_k)) - 1.0))

    peak_nm = np.clip(2.897771955e-3 / temperature_k * 1e9, LAMBDA_MIN_NM, LAMBDA_MAX_NM)
    dense = np.linspace(LAMBDA_MIN_NM, LAMBDA_MAX_NM, 4001)
    peak = max(B(peak_nm), B(dense).max())
    return (scale * B(lam) / peak).astype(np.float32)


def cauchy_index(lam: np.ndarray, a: float = 1.52, b_um2: float = 0.004) -> np.ndarray:
    """Cauchy dispersion n = a + b / lambda^2 with lambda in micrometres."""
    l_um = np.asarray(lam, dtype=np.float64) * 1e-3
    return (a + b_um2 / (l_um * l_um)).astype(np.float32)


_DENSE = np.linspace(LAMBDA_MIN_NM, LAMBDA_MAX_NM, 401)


def _gauss_sum(rng, n_lobes, amp_lo, amp_hi, mu_lo=380.0, mu_hi=780.0, sig_lo=20.0, sig_hi=100.0):
    amps = rng.uniform(amp_lo, amp_hi, n_lobes)
    mus = rng.uniform(mu_lo, mu_hi, n_lobes)
    sigs = rng.uniform(sig_lo, sig_hi, n_lobes)

    def f(lam):
        lam = np.asarray(lam, dtype=np.float64)[..., None]
        return (amps * np.exp(-0.5 * ((lam - mus) / sigs) ** 2)).sum(-1)
    return f


def smooth_curve(rng, lam, lo, hi, n_lobes=3):
    """Seeded smooth curve inside [lo, hi]: a Gaussian sum mapped affinely.

    The map sends the dense-grid minimum and maximum of the sum to two seeded
    levels lo <= a < b <= hi, so every curve is smooth, bounded and varied.
    """
    f = _gauss_sum(rng, n_lobes, 0.2, 1.0)
    g = f(_DENSE)
    gmin, gmax = float(g.min()), float(g.max())
    a = rng.uniform(0.0, 0.6)
    b = rng.uniform(a + 0.25, 1.0)
    t = (f(lam) - gmin) / max(gmax - gmin, 1e-12)
    return (lo + (hi - lo) * (a + (b - a) * np.clip(t, 0.0, 1.0))).astype(np.float32)


def absorption_curve(rng, lam, amp_lo, amp_hi, n_lobes=3):
    """Absorption coefficient alpha(lambda) in 1/m: a sum of seeded Gaussians."""
    f = _gauss_sum(rng, n_lobes, amp_lo, amp_hi)
    return np.maximum(f(lam), 0.0).astype(np.float32)


# --------------------------------------------------------------------------
# Materials, camera, scene containers
# --------------------------------------------------------------------------
@dataclass
class Material:
    kind: int
    rho: Optional[np.ndarray] = None          # Lambertian reflectance [L]
    n: Optional[np.ndarray] = None            # real index [L] (conductor, glass)
    k: Optional[np.ndarray] = None            # extinction [L] (conductor)
    alpha_clear: Optional[np.ndarray] = None  # glass absorption, clear state [1/m]
    dalpha: Optional[np.ndarray] = None       # glass absorption increment at s=1 [1/m]
    thickness_m: float = 0.0
    s_default: float = 0.0
    Le: Optional[np.ndarray] = None           # emitted radiance [L]
    name: str = ""
    # glass coated on both faces with thin films (up to 10 per face), outermost
    # first: each a dict n [L], k [L] (extinction at s = 0), dk [L] (added at
    # s = 1), t_nm (thickness, nm)
    layers: Optional[list] = None


@dataclass
class Camera:
    pos: Sequence[float]
    look: Sequence[float]
    up: Sequence[float] = (0.0, 0.0, 1.0)
    vfov_deg: float = 60.0
    ortho_height: float = 0.0   # > 0 selects an orthographic camera of this height (m)


@dataclass
class RenderSpec:
    width: int
    height: int
    spp: int
    max_depth: int
    seed: int = 0
    render_id: int = 0
    camera: Optional[Camera] = None
    glass_s: Optional[dict] = None   # material index -> coloration state s
    nee: bool = True
    bsdf: str = "exact"              # "exact" | "mlp"

    @property
    def n_paths(self) -> int:
        return self.width * self.height * self.spp


@dataclass
class Scene:
    lam: np.ndarray
    quad_w: np.ndarray
    cmf: np.ndarray
    materials: List[Material]
    V: np.ndarray                    # [nv, 3] float32, metres
    F: np.ndarray                    # [nt, 3] uint32
    mat_id: np.ndarray               # [nt] uint32
    obj_id: np.ndarray               # [nt] uint32
    camera: Camera
    name: str = ""

    @property
    def L(self) -> int:
        return int(self.lam.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.F.shape[0])

    def glass_materials(self) -> List[int]:
        return [i for i, m in enumerate(self.materials) if m.kind == GLASS]


class _MeshBuilder:
    def __init__(self):
        self.V: List[np.ndarray] = []
        self.F: List[np.ndarray] = []
        self.M: List[np.ndarray] = []
        self.O: List[np.ndarray] = []
        self.nv = 0
        self.n_obj = 0

    def add(self, V, F, mat):
        V = np.asarray(V, dtype=np.float64)
        F = np.asarray(F, dtype=np.int64)
        self.V.append(V)
        self.F.append(F + self.nv)
        self.M.append(np.full(len(F), mat, dtype=np.uint32))
        self.O.append(np.full(len(F), self.n_obj, dtype=np.uint32))
        self.nv += len(V)
        self.n_obj += 1
        return self.n_obj - 1

    def arrays(self):
        return (np.concatenate(self.V).astype(np.float32),
                np.concatenate(self.F).astype(np.uint32),
                np.concatenate(self.M), np.concatenate(self.O))


# --------------------------------------------------------------------------
# Geometry primitives (outward counter-clockwise winding)
# --------------------------------------------------------------------------
def box_mesh(lo, hi, inward=False):
    """Axis-aligned box, 12 triangles, CCW seen from outside (or inside if ``inward``)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    V = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float64)
    F = np.array([[0, 2, 1], [0, 3, 2],      # z = z0, normal -z
                  [4, 5, 6], [4, 6, 7],      # z = z1, normal +z
                  [0, 1, 5], [0, 5, 4],      # y = y0, normal -y
                  [3, 7, 6], [3, 6, 2],      # y = y1, normal +y
                  [0, 4, 7], [0, 7, 3],      # x = x0, normal -x
                  [1, 2, 6], [1, 6, 5]],     # x = x1, normal +x
                 dtype=np.int64)
    if inward:
        F = F[:, ::-1].copy()
    return V, F


def quad_mesh(p0, p1, p2, p3):
    """Planar quad p0,p1,p2,p3 (CCW about its front normal), 2 triangles."""
    V = np.array([p0, p1, p2, p3], dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int64)
    return V, F


def uv_sphere(center, radius, n_lat, n_lon):
    """UV sphere with 2*n_lon*(n_lat-1) triangles, outward CCW."""
    cx, cy, cz = center
    th = math.pi * np.arange(1, n_lat) / n_lat
    ph = 2.0 * math.pi * np.arange(n_lon) / n_lon
    st, ct = np.sin(th)[:, None], np.cos(th)[:, None]
    ring = np.stack([cx + radius * st * np.cos(ph)[None, :], cy + radius * st * np.sin(ph)[None, :],
                     np.broadcast_to(cz + radius * ct, (n_lat - 1, n_lon))], -1).reshape(-1, 3)
    V = np.concatenate([[[cx, cy, cz + radius]], ring, [[cx, cy, cz - radius]]]).astype(np.float64)
    south = len(V) - 1
    j = np.arange(n_lon)
    jn = (j + 1) % n_lon

    def idx(i, jj):
        return 1 + (i - 1) * n_lon + jj
    top = np.stack([np.zeros(n_lon, np.int64), idx(1, j), idx(1, jn)], 1)
    i = np.arange(1, n_lat - 1)[:, None]
    a, b, c, d = idx(i, j[None]), idx(i, jn[None]), idx(i + 1, j[None]), idx(i + 1, jn[None])
    mid = np.stack([np.stack([a, c, d], -1), np.stack([a, d, b], -1)], 2).reshape(-1, 3)
    bot = np.stack([np.full(n_lon, south, np.int64), idx(n_lat - 1, jn), idx(n_lat - 1, j)], 1)
    return V, np.concatenate([top, mid, bot]).astype(np.int64)


def extrusion_mesh(rng, center, radius, height, n_sides, n_rings):
    """Seeded irregular prism (star-shaped polygon extruded along z), closed."""
    cx, cy, z0 = center
    ang = np.sort(rng.uniform(0, 2 * math.pi, n_sides))
    rad = radius * rng.uniform(0.5, 1.0, n_sides)
    rx, ry = cx + rad * np.cos(ang), cy + rad * np.sin(ang)
    z = z0 + height * np.arange(n_rings + 1) / n_rings
    V = np.stack([np.broadcast_to(rx, (n_rings + 1, n_sides)), np.broadcast_to(ry, (n_rings + 1, n_sides)),
                  np.broadcast_to(z[:, None], (n_rings + 1, n_sides))], -1).reshape(-1, 3)
    bot, top = len(V), len(V) + 1
    V = np.concatenate([V, [[cx, cy, z0], [cx, cy, z0 + height]]]).astype(np.float64)
    k = np.arange(n_sides)
    kn = (k + 1) % n_sides
    r = np.arange(n_rings)[:, None]
    a, b = r * n_sides + k[None], r * n_sides + kn[None]
    c, d = a + n_sides, b + n_sides
    side = np.stack([np.stack([a, b, d], -1), np.stack([a, d, c], -1)], 2).reshape(-1, 3)
    caps = np.concatenate([np.stack([np.full(n_sides, bot), kn, k], 1),
                           np.stack([np.full(n_sides, top), n_rings * n_sides + k, n_rings * n_sides + kn], 1)])
    return V, np.concatenate([side, caps]).astype(np.int64)


def _spectral_base(L):
    lam = wavelengths(L)
    return lam, trapezoid_weights(lam), cmf_xyz(lam)


def _glass(rng, lam, thickness_m, s, name):
    return Material(GLASS, n=cauchy_index(lam),
                    alpha_clear=absorption_curve(rng, lam, 0.0, 20.0),
                    dalpha=absorption_curve(rng, lam, 50.0, 600.0),
                    thickness_m=thickness_m, s_default=s, name=name)


def electrochromic_glass(rng, lam, thickness_m=0.006, s=0.5, name="electrochromic", n_films=3) -> Material:
    """Clear glass substrate coated on both faces with an electrochromic stack
    of n_films films, outermost first, alternating transparent conductor
    (~150 nm, n ~ 1.9) and electrochromic film (~350 nm, n ~ 2.1, extinction
    rising with the coloration state s mostly toward the red); the default 3
    films are conductor, electrochromic film, conductor, and a single film is
    the electrochromic one. Seeded smooth curves; the substrate's own
    absorption does not depend on s."""
    lam = np.asarray(lam, np.float64)
    x = (lam - 380.0) / 400.0
    tco_n = (1.95 - 0.15 * x + rng.uniform(-0.03, 0.03)).astype(np.float32)
    tco_k = (0.004 + 0.006 * x).astype(np.float32)
    ec_n = (2.15 - 0.12 * x + rng.uniform(-0.03, 0.03)).astype(np.float32)
    ec_k = np.full_like(x, 0.002, dtype=np.float64).astype(np.float32)
    mu, sig = rng.uniform(650.0, 780.0), rng.uniform(120.0, 200.0)
    ec_dk = (rng.uniform(0.08, 0.15) * np.exp(-0.5 * ((lam - mu) / sig) ** 2)).astype(np.float32)
    zero = np.zeros_like(x, dtype=np.float32)
    layers = []
    for j in range(n_films):
        if n_films > 1 and j % 2 == 0:
            layers.append(dict(n=tco_n, k=tco_k, dk=zero, t_nm=float(rng.uniform(130, 170))))
        else:
            layers.append(dict(n=ec_n, k=ec_k, dk=ec_dk, t_nm=float(rng.uniform(300, 400))))
    return Material(GLASS, n=cauchy_index(lam), alpha_clear=absorption_curve(rng, lam, 0.0, 5.0),
                    dalpha=np.zeros(len(lam), np.float32), thickness_m=thickness_m, s_default=s, name=name,
                    layers=layers)


def _metal(rng, lam, name):
    return Material(CONDUCTOR, n=smooth_curve(rng, lam, 0.2, 3.0),
                    k=smooth_curve(rng, lam, 1.0, 8.0), name=name)


# --------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------
def tiny_room(L: int = 16, seed: int = 0, s: float = 0.5, light_scale: float = 10.0,
              with_pane: bool = True, pane_override: Optional[Material] = None, coated: bool = False,
              n_films: int = 3) -> Scene:
    """5x4x3 m room, freestanding 1x1 m pane 4 mm thick, 0.8 m cube, ceiling light.

    36 triangles of geometry plus the 2-triangle light quad. z is up, the
    camera sits at (0.5, 2, 1.5) looking along +x with a 60 degree field.
    """
    rng = np.random.default_rng(seed)
    lam, w, cmf = _spectral_base(L)
    mats = [
        Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name="walls"),
        Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name="floor"),
        Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name="cube"),
        pane_override if pane_override is not None else (
            electrochromic_glass(np.random.default_rng(seed + 77), lam, 0.004, s, "pane", n_films) if coated
            else _glass(rng, lam, 0.004, s, "pane")),
        Material(EMITTER, Le=planck_normalised(lam, 5800.0, light_scale), name="light"),
    ]
    mb = _MeshBuilder()
    V, F = box_mesh((0, 0, 0), (5, 4, 3), inward=True)
    floor = np.array([0, 1])            # z = 0 faces
    mb.add(V, F[floor], 1)
    mb.add(V, np.delete(F, floor, axis=0), 0)
    if with_pane:
        mb.add(*box_mesh((2.0, 1.5, 1.0), (2.004, 2.5, 2.0)), 3)
    mb.add(*box_mesh((3.5, 0.5, 0.0), (4.3, 1.3, 0.8)), 2)
    # light at z = 2.99 facing -z: CCW seen from below
    mb.add(*quad_mesh((2, 1.5, 2.99), (2, 2.5, 2.99), (3, 2.5, 2.99), (3, 1.5, 2.99)), 4)
    Vv, Ff, M, O = mb.arrays()
    cam = Camera(pos=(0.5, 2.0, 1.5), look=(1.5, 2.0, 1.5), up=(0, 0, 1), vfov_deg=60.0)
    return Scene(lam, w, cmf, mats, Vv, Ff, M, O, cam, name="tiny_room")


def hotel_room(L: int = 41, seed: int = 0, s: float = 0.5, n_boxes: int = 40,
               n_spheres: int = 100, n_metal: int = 20, sphere_lat: int = 21,
               sphere_lon: int = 50, light_scale: float = 10.0) -> Scene:
    """6x4x3 m room with 40 boxes, 100 spheres of 2000 triangles (20 metallic),
    two photochromic window panes, each lit by a 'sun' quad behind it, and a
    1x1 m ceiling lamp."""
    rng = np.random.default_rng(seed)
    lam, w, cmf = _spectral_base(L)
    mats: List[Material] = [
        Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name="walls"),
        Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name="floor"),
    ]
    diffuse_ids = []
    for i in range(6):
        mats.append(Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name=f"diffuse{i}"))
        diffuse_ids.append(len(mats) - 1)
    metal_ids = []
    for i in range(4):
        mats.append(_metal(rng, lam, f"metal{i}"))
        metal_ids.append(len(mats) - 1)
    glass_id = len(mats)
    mats.append(_glass(rng, lam, 0.004, s, "photochromic"))
    light_id = len(mats)
    mats.append(Material(EMITTER, Le=planck_normalised(lam, 5800.0, light_scale), name="sun"))
    lamp_id = len(mats)
    mats.append(Material(EMITTER, Le=planck_normalised(lam, 3000.0, 0.5 * light_scale), name="lamp"))

    mb = _MeshBuilder()
    V, F = box_mesh((0, 0, 0), (6, 4, 3), inward=True)
    mb.add(V, F[[0, 1]], 1)
    mb.add(V, np.delete(F, [0, 1], axis=0), 0)
    # two windows on the x = 6 wall: pane 5 cm inside, sun quad just in front of the wall
    for yc in (1.0, 3.0):
        mb.add(*box_mesh((5.9, yc - 0.6, 0.9), (5.904, yc + 0.6, 2.3)), glass_id)
        mb.add(*quad_mesh((5.99, yc - 0.58, 0.92), (5.99, yc - 0.58, 2.28),
                          (5.99, yc + 0.58, 2.28), (5.99, yc + 0.58, 0.92)), light_id)
    # ceiling lamp, facing -z
    mb.add(*quad_mesh((2.5, 1.5, 2.99), (2.5, 2.5, 2.99), (3.5, 2.5, 2.99), (3.5, 1.5, 2.99)),
           lamp_id)
    for i in range(n_boxes):
        sx, sy, sz = rng.uniform(0.1, 0.7, 3)
        x = rng.uniform(1.2, 5.5 - sx)   # keep clear of the camera at x < 1.2
        y = rng.uniform(0.1, 3.9 - sy)
        z = rng.uniform(0.0, 1.2)
        mb.add(*box_mesh((x, y, z), (x + sx, y + sy, z + sz)),
               diffuse_ids[int(rng.integers(len(diffuse_ids)))])
    for i in range(n_spheres):
        r = rng.uniform(0.1, 0.6)
        c = (rng.uniform(1.2 + r, 5.5 - r * 0.5), rng.uniform(r * 0.5 + 0.1, 3.9 - r * 0.5),
             rng.uniform(r * 0.5, 2.8 - r * 0.5))
        mat = metal_ids[i % len(metal_ids)] if i < n_metal else \
            diffuse_ids[int(rng.integers(len(diffuse_ids)))]
        mb.add(*uv_sphere(c, r, sphere_lat, sphere_lon), mat)
    Vv, Ff, M, O = mb.arrays()
    cam = Camera(pos=(0.3, 2.0, 1.6), look=(5.0, 2.0, 1.3), up=(0, 0, 1), vfov_deg=70.0)
    return Scene(lam, w, cmf, mats, Vv, Ff, M, O, cam, name="hotel_room")


def facade_room(L: int = 81, seed: int = 0, target_tris: int = 5_000_000,
                n_panes: int = 8, light_scale: float = 10.0) -> Scene:
    """12x8x3 m room, seeded furniture meshes (5k-50k triangles each) up to
    ``target_tris`` triangles, 8 electrochromic panes on the x = 12 facade,
    each with its own coloration state s ~ U[0, 1] and its own sun quad, and
    four ceiling lamps."""
    rng = np.random.default_rng(seed)
    lam, w, cmf = _spectral_base(L)
    mats: List[Material] = [
        Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name="walls"),
        Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name="floor"),
    ]
    diffuse_ids, metal_ids = [], []
    for i in range(8):
        mats.append(Material(LAMBERT, rho=smooth_curve(rng, lam, 0.05, 0.9), name=f"diffuse{i}"))
        diffuse_ids.append(len(mats) - 1)
    for i in range(4):
        mats.append(_metal(rng, lam, f"metal{i}"))
        metal_ids.append(len(mats) - 1)
    base_glass = _glass(rng, lam, 0.006, 0.5, "electrochromic")
    glass_ids = []
    for i in range(n_panes):
        g = Material(GLASS, n=base_glass.n, alpha_clear=base_glass.alpha_clear,
                     dalpha=base_glass.dalpha, thickness_m=base_glass.thickness_m,
                     s_default=float(rng.uniform(0.0, 1.0)), name=f"pane{i}")
        mats.append(g)
        glass_ids.append(len(mats) - 1)
    light_id = len(mats)
    mats.append(Material(EMITTER, Le=planck_normalised(lam, 5800.0, light_scale), name="sun"))
    lamp_id = len(mats)
    mats.append(Material(EMITTER, Le=planck_normalised(lam, 3000.0, 0.5 * light_scale), name="lamp"))

    mb = _MeshBuilder()
    V, F = box_mesh((0, 0, 0), (12, 8, 3), inward=True)
    mb.add(V, F[[0, 1]], 1)
    mb.add(V, np.delete(F, [0, 1], axis=0), 0)
    for i in range(n_panes):
        yc = 0.5 + (i + 0.5) * 7.0 / n_panes
        hw = 0.38
        mb.add(*box_mesh((11.9, yc - hw, 0.8), (11.906, yc + hw, 2.4)), glass_ids[i])
        mb.add(*quad_mesh((11.99, yc - hw + 0.05, 0.9), (11.99, yc - hw + 0.05, 2.3),
                          (11.99, yc + hw - 0.05, 2.3), (11.99, yc + hw - 0.05, 0.9)), light_id)
    # four ceiling lamps
    for lx in (4.0, 8.0):
        for ly in (2.5, 5.5):
            mb.add(*quad_mesh((lx - 0.4, ly - 0.4, 2.99), (lx - 0.4, ly + 0.4, 2.99), (lx + 0.4, ly + 0.4, 2.99),
                              (lx + 0.4, ly - 0.4, 2.99)), lamp_id)
    # furniture: finely tessellated objects, knee to chest height, x >= 3 m (the cameras stand nearer)
    n_now = sum(len(f) for f in mb.F)
    while n_now < target_tris:
        budget = int(rng.integers(5_000, 50_001))
        budget = min(budget, max(target_tris - n_now, 12))
        kind = int(rng.integers(3))
        cx, cy = rng.uniform(3.0, 10.5), rng.uniform(0.8, 7.2)
        if kind == 0 or budget < 200:        # cluster of small boxes
            nb = max(1, budget // 12)
            for _ in range(nb):
                s3 = rng.uniform(0.02, 0.15, 3)
                p = (cx + rng.uniform(-0.4, 0.4), cy + rng.uniform(-0.4, 0.4), rng.uniform(0, 1.0))
                mb.add(*box_mesh(p, (p[0] + s3[0], p[1] + s3[1], p[2] + s3[2])),
                       diffuse_ids[int(rng.integers(len(diffuse_ids)))])
            n_now += nb * 12
        elif kind == 1:                      # sphere
            n_lon = max(8, int(math.sqrt(budget / 2.0) * 1.4))
            n_lat = max(4, budget // (2 * n_lon) + 1)
            r = rng.uniform(0.1, 0.35)
            mat = metal_ids[int(rng.integers(len(metal_ids)))] if rng.uniform() < 0.3 else \
                diffuse_ids[int(rng.integers(len(diffuse_ids)))]
            V_, F_ = uv_sphere((cx, cy, rng.uniform(r, 1.2)), r, n_lat, n_lon)
            mb.add(V_, F_, mat)
            n_now += len(F_)
        else:                                # extrusion
            n_sides = int(rng.integers(12, 64))
            n_rings = max(1, budget // (2 * n_sides))
            V_, F_ = extrusion_mesh(rng, (cx, cy, 0.0), rng.uniform(0.1, 0.4), rng.uniform(0.3, 1.4),
                                    n_sides, n_rings)
            mb.add(V_, F_, diffuse_ids[int(rng.integers(len(diffuse_ids)))])
            n_now += len(F_)
    Vv, Ff, M, O = mb.arrays()
    cam = Camera(pos=(0.4, 4.0, 1.6), look=(11.0, 4.0, 1.4), up=(0, 0, 1), vfov_deg=75.0)
    return Scene(lam, w, cmf, mats, Vv, Ff, M, O, cam, name="facade_room")


def furnace_box(L: int = 8, rho0: float = 0.6, Le0: float = 0.7, size=(2.0, 3.0, 1.5)) -> Scene:
    """Closed box whose every face is a one-sided (inward) diffuse emitter with
    constant reflectance rho0 and constant radiance Le0."""
    lam, w, cmf = _spectral_base(L)
    mats = [Material(DIFFUSE_EMITTER, rho=np.full(L, rho0, np.float32),
                     Le=np.full(L, Le0, np.float32), name="furnace")]
    mb = _MeshBuilder()
    mb.add(*box_mesh((0, 0, 0), size, inward=True), 0)
    Vv, Ff, M, O = mb.arrays()
    cam = Camera(pos=(size[0] * 0.3, size[1] * 0.4, size[2] * 0.5),
                 look=(size[0], size[1] * 0.6, size[2] * 0.4), vfov_deg=80.0)
    return Scene(lam, w, cmf, mats, Vv, Ff, M, O, cam, name="furnace")


def random_soup(n_tris: int, seed: int = 0, extent: float = 1.0, size: float = 0.15,
                L: int = 4) -> Scene:
    """Random triangle soup in a cube (for intersection / BVH cross-checks)."""
    rng = np.random.default_rng(seed)
    lam, w, cmf = _spectral_base(L)
    c = rng.uniform(0, extent, (n_tris, 1, 3))
    V = (c + rng.normal(0, size, (n_tris, 3, 3))).reshape(-1, 3).astype(np.float32)
    F = np.arange(3 * n_tris, dtype=np.uint32).reshape(-1, 3)
    mats = [Material(LAMBERT, rho=np.full(L, 0.5, np.float32))]
    cam = Camera(pos=(-1, 0.5, 0.5), look=(0.5, 0.5, 0.5))
    return Scene(lam, w, cmf, mats, V, F, np.zeros(n_tris, np.uint32),
                 np.arange(n_tris, dtype=np.uint32), cam, name="soup")


# --------------------------------------------------------------------------
# Render descriptions of the five workloads
# --------------------------------------------------------------------------
def tiny_room_render(scene: Scene, width=64, height=64, spp=1, max_depth=2, seed=0) -> RenderSpec:
    return RenderSpec(width, height, spp, max_depth, seed=seed, camera=scene.camera)


def hotel_room_render(scene: Scene, width=512, height=512, spp=16, max_depth=5, seed=0) -> RenderSpec:
    return RenderSpec(width, height, spp, max_depth, seed=seed, camera=scene.camera)


def batched_renders(scene: Scene, n_renders=64, seed=0, max_depth=5):
    """64 renders of the tiny room with resolution ~U{128,256,512,1024}^2,
    spp ~ U{4,16,64} and coloration state s ~ U[0,1], drawn with ``seed``."""
    rng = np.random.default_rng(seed)
    res = rng.choice([128, 256, 512, 1024], size=n_renders)
    spp = rng.choice([4, 16, 64], size=n_renders)
    s = rng.uniform(0.0, 1.0, size=n_renders)
    glass = scene.glass_materials()
    out = []
    for r in range(n_renders):
        out.append(RenderSpec(int(res[r]), int(res[r]), int(spp[r]), max_depth, seed=seed,
                              render_id=r, camera=scene.camera,
                              glass_s={g: float(s[r]) for g in glass}))
    return out


def facade_renders(scene: Scene, n_renders=16, width=1920, height=1080, spp=64, max_depth=8, seed=0):
    """16 renders of the facade room from seeded camera positions."""
    rng = np.random.default_rng(seed + 1)
    out = []
    for r in range(n_renders):
        pos = (rng.uniform(0.4, 2.5), rng.uniform(1.0, 7.0), rng.uniform(1.2, 2.0))
        look = (11.0, rng.uniform(2.0, 6.0), rng.uniform(1.0, 1.8))
        out.append(RenderSpec(width, height, spp, max_depth, seed=seed, render_id=r,
                              camera=Camera(pos=pos, look=look, vfov_deg=75.0)))
    return out


def pixel_subset(width: int, height: int, n: int, seed: int = 0) -> np.ndarray:
    """Seeded subset of ``n`` distinct linear pixel indices (sorted)."""
    n = min(n, width * height)
    rng = np.random.default_rng(seed + 12345)
    return np.sort(rng.choice(width * height, size=n, replace=False)).astype(np.int64)
