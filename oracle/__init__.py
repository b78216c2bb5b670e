"""FP64 CPU oracle of the spectral DDM path tracer -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It is plain C (``*.c`` beside this file,
compiled with gcc, ``-ffp-contract=off``) driven through ctypes, and it shares
no code with the CUDA path: the two meet only in the seeded scene arrays.

What each C function follows in the paper (arXiv:1912.06474):
  optics.c  -- Eq. 1 complex index, Fresnel for metals (Sec. 2) and the glass
               slab from the Fresnel equations (Sec. 6) with multiple reflections.
  geom.c    -- ray/object interactions (Sec. 4-5): Moller-Trumbore, closest
               hit, shadow query through glass; brute force or median-split BVH.
  render.c  -- Eq. 2 by path tracing with Eq. 3's light sum as next-event
               estimation (Sec. 3-4); spectral XYZ output.
  philox.c  -- the counter-based random stream both sides draw from.

The random stream is pinned by Philox4x32-10's published known-answer vectors and statistically.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["philox.c", "optics.c", "geom.c", "render.c", "mlp.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "libsddm_oracle.so")
_lock = threading.Lock()
_lib = None

# coating films per glass face (ORC_MAX_FILMS in oracle_internal.h)
MAX_FILMS = 10
# material kinds: same integer codes as the scene inputs
LAMBERT, CONDUCTOR, GLASS, EMITTER, DIFFUSE_EMITTER = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libsddm_oracle.so`` with gcc."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdrs = [os.path.join(_HERE, h) for h in ("sddm_oracle.h", "oracle_internal.h")]
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs + hdrs):
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unused-function", "-o", tmp] + srcs + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _SceneDesc(C.Structure):
    _fields_ = [("L", C.c_int), ("lam_nm", C.c_void_p), ("quad_w", C.c_void_p), ("cmf", C.c_void_p),
                ("n_mat", C.c_int), ("mat_kind", C.c_void_p), ("mat_a", C.c_void_p),
                ("mat_b", C.c_void_p), ("mat_c", C.c_void_p), ("mat_thick", C.c_void_p),
                ("mat_s", C.c_void_p), ("nv", C.c_int), ("V", C.c_void_p), ("nt", C.c_int),
                ("F", C.c_void_p), ("mat_id", C.c_void_p), ("obj_id", C.c_void_p),
                ("mat_nlayers", C.c_void_p), ("layer_n", C.c_void_p), ("layer_k", C.c_void_p),
                ("layer_dk", C.c_void_p), ("layer_t", C.c_void_p)]


class _RenderDesc(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("spp", C.c_int), ("max_depth", C.c_int),
                ("seed", C.c_uint32), ("render_id", C.c_uint32), ("nee", C.c_int),
                ("cam_pos", C.c_double * 3), ("cam_look", C.c_double * 3), ("cam_up", C.c_double * 3),
                ("vfov_deg", C.c_double), ("ortho_height", C.c_double), ("s_override", C.c_void_p),
                ("brute_force", C.c_int), ("photon_map", C.c_void_p), ("caustic_map", C.c_void_p)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        lib.orc_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(_SceneDesc)]
        lib.orc_create.restype = C.c_int
        lib.orc_destroy.argtypes = [P]
        lib.orc_render_pixels.argtypes = [P, C.POINTER(_RenderDesc), C.c_int64, P, P, P, P, P, P,
                                          C.c_int, P]
        lib.orc_render_pixels.restype = C.c_int
        lib.orc_philox4x32_10.argtypes = [P, P, P]
        lib.orc_u01.argtypes = [C.c_uint32]
        lib.orc_u01.restype = C.c_double
        lib.orc_fresnel.argtypes = [C.c_double, C.c_double, C.c_double, P, P]
        lib.orc_slab.argtypes = [C.c_double] * 5 + [P, P]
        lib.orc_photon_map_build.argtypes = [P, P, C.c_int64, C.c_double, C.c_int]
        lib.orc_photon_map_build.restype = C.c_void_p
        lib.orc_photon_map_build_kind.argtypes = [P, P, C.c_int64, C.c_double, C.c_int, C.c_int]
        lib.orc_photon_map_build_kind.restype = C.c_void_p
        lib.orc_photon_map_free.argtypes = [P]
        lib.orc_photon_map_get.argtypes = [P, P, P, P]
        lib.orc_photon_map_get.restype = C.c_int64
        lib.orc_coated_face.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, P, P, P, C.c_int, P, P, P, P]
        lib.orc_coated_slab.argtypes = [C.c_double] * 5 + [C.c_int, P, P, P, P, P]
        lib.orc_conductor.argtypes = [C.c_double] * 3
        lib.orc_conductor.restype = C.c_double
        lib.orc_branch_proxy.argtypes = [C.c_float, C.c_int, P]
        lib.orc_branch_proxy.restype = C.c_float
        lib.orc_cosine_dir.argtypes = [P, C.c_double, C.c_double, P]
        lib.orc_camera_ray.argtypes = [C.POINTER(_RenderDesc), C.c_double, C.c_double, P, P]
        lib.orc_closest_hit.argtypes = [P, P, P, C.c_int, P, P]
        lib.orc_closest_hit.restype = C.c_int
        lib.orc_shadow.argtypes = [P, P, P, C.c_double, C.c_int, C.c_int, P, P, P]
        lib.orc_shadow.restype = C.c_int
        lib.orc_watertight.argtypes = [P, P, P, C.POINTER(C.c_double)]
        lib.orc_watertight.restype = C.c_int
        lib.orc_plane.argtypes = [P, P, P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.orc_plane.restype = C.c_int
        lib.orc_num_lights.argtypes = [P]
        lib.orc_num_lights.restype = C.c_int
        lib.orc_mlp_n_params.restype = C.c_int
        lib.orc_mlp_features.argtypes = [C.c_double] * 6 + [P]
        lib.orc_mlp_forward.argtypes = [P, P, P]
        lib.orc_mlp_rt.argtypes = [P, P, P]
        lib.orc_mlp_forward_d.argtypes = [P, P, P]
        lib.orc_mlp_loss_grad.argtypes = [P, C.c_int, P, P, P]
        lib.orc_mlp_loss_grad.restype = C.c_double
        lib.orc_mlp_loss_grad_d.argtypes = [P, C.c_int, P, P, P]
        lib.orc_mlp_loss_grad_d.restype = C.c_double
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------ primitives ---
def philox4x32_10(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(x: int) -> float:
    return _load().orc_u01(int(x) & 0xFFFFFFFF)


def fresnel(c, n, k):
    lib = _load()
    rs, rp = C.c_double(), C.c_double()
    lib.orc_fresnel(float(c), float(n), float(k), C.byref(rs), C.byref(rp))
    return rs.value, rp.value


def slab(c, lam_nm, n, alpha_per_m, thick_m):
    lib = _load()
    R, T = C.c_double(), C.c_double()
    lib.orc_slab(float(c), float(lam_nm), float(n), float(alpha_per_m), float(thick_m),
                 C.byref(R), C.byref(T))
    return R.value, T.value


def _films(layers):
    nf = np.ascontiguousarray([f[0] for f in layers], np.float64)
    kf = np.ascontiguousarray([f[1] for f in layers], np.float64)
    tf = np.ascontiguousarray([f[2] for f in layers], np.float64)
    return nf, kf, tf


def coated_face(c, lam_nm, n_sub, layers, pol):
    """One coated face: (R, T) seen from air and (R, T) seen from the glass,
    for films [(n, k, t_nm), ...] outermost first; pol 0 = s, 1 = p."""
    lib = _load()
    nf, kf, tf = _films(layers) if layers else (np.zeros(1), np.zeros(1), np.zeros(1))
    out = [C.c_double() for _ in range(4)]
    lib.orc_coated_face(float(c), float(lam_nm), float(n_sub), len(layers), _ptr(nf), _ptr(kf), _ptr(tf),
                        int(pol), *[C.byref(o) for o in out])
    return tuple(o.value for o in out)


def coated_slab(c, lam_nm, n_sub, alpha_per_m, thick_m, layers):
    """Slab coated on both faces with films [(n, k, t_nm), ...]: (R, T)."""
    lib = _load()
    nf, kf, tf = _films(layers) if layers else (np.zeros(1), np.zeros(1), np.zeros(1))
    R, T = C.c_double(), C.c_double()
    lib.orc_coated_slab(float(c), float(lam_nm), float(n_sub), float(alpha_per_m), float(thick_m), len(layers),
                        _ptr(nf), _ptr(kf), _ptr(tf), C.byref(R), C.byref(T))
    return R.value, T.value


def conductor(c, n, k):
    return _load().orc_conductor(float(c), float(n), float(k))


def branch_proxy(c, n_curve):
    n = np.ascontiguousarray(n_curve, dtype=np.float32)
    return _load().orc_branch_proxy(float(c), int(n.shape[0]), _ptr(n))


def cosine_dir(ns, u0, u1):
    n = np.ascontiguousarray(ns, dtype=np.float64)
    out = np.zeros(3)
    _load().orc_cosine_dir(_ptr(n), float(u0), float(u1), _ptr(out))
    return out


# ------------------------------------------------------------------- MLP ---
MLP_PARAMS = 8770


def watertight(tri, o, d):
    """Watertight ray/triangle test (FP64): (hit, t) for the line of ray
    (o, d) against triangle tri[3][3]; t may be negative."""
    v = np.ascontiguousarray(tri, np.float64).reshape(9)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    t = C.c_double()
    hit = _load().orc_watertight(_ptr(v), _ptr(o), _ptr(d), C.byref(t))
    return bool(hit), (t.value if hit else np.inf)


def moller_trumbore(tri, o, d):
    """The renderer's Moller-Trumbore test (FP64): (hit, t, (u, w)) with hit
    when the line meets the triangle (u, w >= 0, u + w <= 1)."""
    v = np.ascontiguousarray(tri, np.float64).reshape(9)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    t, u, w = C.c_double(), C.c_double(), C.c_double()
    if not _load().orc_plane(_ptr(v), _ptr(o), _ptr(d), C.byref(t), C.byref(u), C.byref(w)):
        return False, np.inf, (np.nan, np.nan)
    hit = u.value >= 0 and w.value >= 0 and u.value + w.value <= 1
    return hit, t.value, (u.value, w.value)


def mlp_features(c, lam_nm, s, d, alpha, film_absorbance=0.0):
    """Network inputs of one row: cos, wavelength (nm), coloration state,
    thickness (m), the absorption coefficient alpha(lambda, s) (1/m) and the
    coating films' normal-incidence absorbance sum 4 pi k t / lambda."""
    x = np.zeros(4)
    _load().orc_mlp_features(float(c), float(lam_nm), float(s), float(d), float(alpha), float(film_absorbance),
                             _ptr(x))
    return x


def mlp_rt(params, X):
    """Served (R, T) of the surrogate for rows X [n,4]: exp(y) - 1e-3, clamped at 0."""
    lib = _load()
    X = np.ascontiguousarray(np.atleast_2d(X), np.float64)
    p = np.ascontiguousarray(params, np.float32)
    out = np.zeros((X.shape[0], 2))
    for i in range(X.shape[0]):
        lib.orc_mlp_rt(_ptr(p), _ptr(X[i]), _ptr(out[i]))
    return out


def mlp_forward(params, X):
    """FP64 forward of the surrogate for rows X [n,4]; params float32 (or float64) [8770]."""
    lib = _load()
    X = np.ascontiguousarray(np.atleast_2d(X), np.float64)
    p = np.ascontiguousarray(params)
    out = np.zeros((X.shape[0], 2))
    fn = lib.orc_mlp_forward_d if p.dtype == np.float64 else lib.orc_mlp_forward
    if p.dtype != np.float64:
        p = np.ascontiguousarray(p, np.float32)
    for i in range(X.shape[0]):
        fn(_ptr(p), _ptr(X[i]), out[i:].ctypes.data_as(C.c_void_p))
    return out


def mlp_loss_grad(params, X, Y):
    """FP64 loss (mean squared error over rows and both outputs) and its gradient."""
    lib = _load()
    X = np.ascontiguousarray(X, np.float64)
    Y = np.ascontiguousarray(Y, np.float64)
    p = np.ascontiguousarray(params)
    g = np.zeros(MLP_PARAMS)
    if p.dtype == np.float64:
        loss = lib.orc_mlp_loss_grad_d(_ptr(p), int(X.shape[0]), _ptr(X), _ptr(Y), _ptr(g))
    else:
        p = np.ascontiguousarray(p, np.float32)
        loss = lib.orc_mlp_loss_grad(_ptr(p), int(X.shape[0]), _ptr(X), _ptr(Y), _ptr(g))
    return loss, g


# ----------------------------------------------------------------- scene ---
def _material_arrays(scene):
    L = scene.L
    M = len(scene.materials)
    kind = np.zeros(M, np.int32)
    a = np.zeros((M, L), np.float32)
    b = np.zeros((M, L), np.float32)
    c = np.zeros((M, L), np.float32)
    thick = np.zeros(M, np.float32)
    s = np.zeros(M, np.float32)
    for i, m in enumerate(scene.materials):
        kind[i] = m.kind
        if m.kind == LAMBERT:
            a[i] = m.rho
        elif m.kind == CONDUCTOR:
            a[i], b[i] = m.n, m.k
        elif m.kind == GLASS:
            a[i], b[i], c[i] = m.n, m.alpha_clear, m.dalpha
            thick[i], s[i] = m.thickness_m, m.s_default
        elif m.kind == EMITTER:
            a[i] = m.Le
        elif m.kind == DIFFUSE_EMITTER:
            a[i], b[i] = m.Le, m.rho
        else:
            raise ValueError(f"unknown material kind {m.kind}")
    return kind, a, b, c, thick, s


def _layer_arrays(scene):
    L, M = scene.L, len(scene.materials)
    nl = np.zeros(M, np.int32)
    ln = np.zeros((M, MAX_FILMS, L), np.float32)
    lk = np.zeros((M, MAX_FILMS, L), np.float32)
    ldk = np.zeros((M, MAX_FILMS, L), np.float32)
    lt = np.zeros((M, MAX_FILMS), np.float32)
    for i, m in enumerate(scene.materials):
        if m.kind == GLASS and m.layers:
            if len(m.layers) > MAX_FILMS:
                raise ValueError(f"at most {MAX_FILMS} films per face")
            nl[i] = len(m.layers)
            for j, f in enumerate(m.layers):
                ln[i, j], lk[i, j], ldk[i, j], lt[i, j] = f["n"], f["k"], f["dk"], f["t_nm"]
    return nl, ln, lk, ldk, lt


class _PhotonMap:
    """Owned oracle photon map (freed with the object)."""

    def __init__(self, lib, h, L):
        self.lib, self.h, self.L = lib, C.c_void_p(h), L

    def photons(self):
        n = self.lib.orc_photon_map_get(self.h, None, None, None)
        pos, dirs, pw = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, self.L))
        self.lib.orc_photon_map_get(self.h, _ptr(pos), _ptr(dirs), _ptr(pw))
        return pos, dirs, pw

    def __del__(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.orc_photon_map_free(self.h)
            self.h = None


class Oracle:
    """FP64 oracle bound to one scene (inputs copied on construction)."""

    def __init__(self, scene):
        self.lib = _load()
        self.scene = scene
        kind, a, b, c, thick, s = _material_arrays(scene)
        nl, ln, lk, ldk, lt = _layer_arrays(scene)
        keep = dict(nl=nl, ln=ln, lk=lk, ldk=ldk, lt=lt, lam=np.ascontiguousarray(scene.lam, np.float32),
                    w=np.ascontiguousarray(scene.quad_w, np.float32),
                    cmf=np.ascontiguousarray(scene.cmf, np.float32),
                    kind=kind, a=a, b=b, c=c, thick=thick, s=s,
                    V=np.ascontiguousarray(scene.V, np.float32),
                    F=np.ascontiguousarray(scene.F, np.uint32),
                    M=np.ascontiguousarray(scene.mat_id, np.uint32),
                    O=np.ascontiguousarray(scene.obj_id, np.uint32))
        d = _SceneDesc(scene.L, _ptr(keep["lam"]), _ptr(keep["w"]), _ptr(keep["cmf"]),
                       len(scene.materials), _ptr(kind), _ptr(a), _ptr(b), _ptr(c), _ptr(thick),
                       _ptr(s), int(keep["V"].shape[0]), _ptr(keep["V"]), int(keep["F"].shape[0]),
                       _ptr(keep["F"]), _ptr(keep["M"]), _ptr(keep["O"]), _ptr(nl), _ptr(ln), _ptr(lk),
                       _ptr(ldk), _ptr(lt))
        h = C.c_void_p()
        rc = self.lib.orc_create(C.byref(h), C.byref(d))
        if rc != 0:
            raise RuntimeError(f"orc_create failed ({rc})")
        self._h = h
        self._keep = keep

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.orc_destroy(h)
            self._h = None

    @property
    def n_lights(self):
        return self.lib.orc_num_lights(self._h)

    def _render_desc(self, spec, brute_force=False):
        cam = spec.camera if spec.camera is not None else self.scene.camera
        s_ov = np.full(len(self.scene.materials), -1.0, np.float32)
        for m, val in (spec.glass_s or {}).items():
            s_ov[int(m)] = float(val)
        r = _RenderDesc()
        r.width, r.height, r.spp, r.max_depth = spec.width, spec.height, spec.spp, spec.max_depth
        r.seed, r.render_id = spec.seed & 0xFFFFFFFF, spec.render_id & 0xFFFFFFFF
        r.nee = 1 if spec.nee else 0
        f32 = lambda v: float(np.float32(v))   # the camera reaches the CUDA path as float32
        for i in range(3):
            r.cam_pos[i], r.cam_look[i], r.cam_up[i] = f32(cam.pos[i]), f32(cam.look[i]), f32(cam.up[i])
        r.vfov_deg, r.ortho_height = f32(cam.vfov_deg), f32(cam.ortho_height)
        r.s_override = _ptr(s_ov)
        r.brute_force = 1 if brute_force else 0
        return r, s_ov

    def camera_ray(self, spec, px, py):
        r, _keep = self._render_desc(spec)
        o, d = np.zeros(3), np.zeros(3)
        self.lib.orc_camera_ray(C.byref(r), float(px), float(py), _ptr(o), _ptr(d))
        return o, d

    def photon_map(self, spec, n_photons, radius, n_threads=0, kind="all"):
        """Photon map of this scene for the render ``spec`` (its seed, render id,
        depth and coloration states): a handle for render_pixels. ``kind``:
        "all" stored photons, or only the "global" or the "caustic" ones."""
        r, keep = self._render_desc(spec, False)
        h = self.lib.orc_photon_map_build_kind(self._h, C.byref(r), int(n_photons), float(radius),
                                               {"all": 0, "global": 1, "caustic": 2}[kind], int(n_threads))
        if not h:
            raise RuntimeError("orc_photon_map_build failed")
        return _PhotonMap(self.lib, h, self.scene.L)

    def render_pixels(self, spec, pix=None, n_threads=0, per_sample=False, brute_force=False, photon_map=None,
                      caustic_map=None):
        """Render the listed pixels (all if None). Returns a dict with ``xyz``
        [n,3]; with ``per_sample`` also ``sample_xyz`` [n,spp,3], ``first_prim``
        [n,spp], ``margin`` [n,spp] and ``cos_min`` [n,spp]; ``segments`` = (extension, shadow)."""
        if pix is None:
            pix = np.arange(spec.width * spec.height, dtype=np.int64)
        pix = np.ascontiguousarray(pix, dtype=np.int64)
        n = int(pix.shape[0])
        r, s_keep = self._render_desc(spec, brute_force)
        if photon_map is not None:
            r.photon_map = photon_map.h
            if caustic_map is not None:
                r.caustic_map = caustic_map.h
        xyz = np.zeros((n, 3), np.float64)
        sx = fp = mg = cm = None
        if per_sample:
            sx = np.zeros((n, spec.spp, 3), np.float64)
            fp = np.zeros((n, spec.spp), np.int32)
            mg = np.zeros((n, spec.spp), np.float64)
            cm = np.zeros((n, spec.spp), np.float64)
        seg = np.zeros(2, np.int64)
        rc = self.lib.orc_render_pixels(self._h, C.byref(r), n, _ptr(pix), _ptr(xyz), _ptr(sx),
                                        _ptr(fp), _ptr(mg), _ptr(cm), int(n_threads), _ptr(seg))
        if rc != 0:
            raise RuntimeError(f"orc_render_pixels failed ({rc})")
        out = dict(xyz=xyz, segments=(int(seg[0]), int(seg[1])), pix=pix)
        if per_sample:
            out.update(sample_xyz=sx, first_prim=fp, margin=mg, cos_min=cm)
        return out

    def render_image(self, spec, n_threads=0):
        res = self.render_pixels(spec, None, n_threads)
        return res["xyz"].reshape(spec.height, spec.width, 3)

    def closest_hit(self, o, d, brute_force=False):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t = C.c_double()
        b = np.zeros(3)
        prim = self.lib.orc_closest_hit(self._h, _ptr(o), _ptr(d), 1 if brute_force else 0,
                                        C.byref(t), _ptr(b))
        return prim, (t.value if prim >= 0 else np.inf), b

    def shadow(self, o, d, tmax, excl_prim=-1, brute_force=False):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        ncr = C.c_int()
        cobj = np.zeros(4, np.int32)
        ccos = np.zeros(4)
        occ = self.lib.orc_shadow(self._h, _ptr(o), _ptr(d), float(tmax), int(excl_prim),
                                  1 if brute_force else 0, C.byref(ncr), _ptr(cobj), _ptr(ccos))
        return bool(occ), list(zip(cobj[:ncr.value].tolist(), ccos[:ncr.value].tolist()))


# --------------------------------------------------------------------------
# RGB -> spectrum by Cohen and Kappauf's matrix R (Sec. 3 of the paper: every
# spectrum splits into a fundamental, which carries its colour stimulus, and a
# metameric black, which has X = Y = Z = 0; the fundamental of a stimulus
# follows from one matrix equation). FP64, numpy.
# --------------------------------------------------------------------------
# Linear sRGB primaries with the D65 white, RGB -> XYZ (IEC 61966-2-1).
SRGB_TO_XYZ = np.array([[0.4124, 0.3576, 0.1805],
                        [0.2126, 0.7152, 0.0722],
                        [0.0193, 0.1192, 0.9505]])


def color_basis(quad_w, cmf):
    """A [L,3]: the XYZ of a reflectance spectrum rho under an equal-energy
    illuminant is A^T rho, with A = w_i cmf(lambda_i) / sum_i w_i ybar_i
    (so that rho = 1 has Y = 1)."""
    W = np.asarray(quad_w, np.float64)[:, None] * np.asarray(cmf, np.float64)
    return W / W[:, 1].sum()


def matrice_r(A):
    """Cohen's matrix R = A (A^T A)^-1 A^T, the orthogonal projector onto the
    colour-stimulus space: R N is the fundamental of spectrum N."""
    return A @ np.linalg.solve(A.T @ A, A.T)


def fundamental_from_xyz(xyz, A):
    """The fundamental spectrum with tristimulus xyz: A (A^T A)^-1 xyz."""
    return A @ np.linalg.solve(A.T @ A, np.asarray(xyz, np.float64).T)


def rgb_to_spectrum(rgb, quad_w, cmf, rgb_to_xyz=None, clamp=False):
    """Spectra [n,L] of RGB values [n,3]: XYZ = M rgb, then the fundamental;
    with clamp, limited to [0, 1] afterwards."""
    A = color_basis(quad_w, cmf)
    M = SRGB_TO_XYZ if rgb_to_xyz is None else np.asarray(rgb_to_xyz, np.float64)
    xyz = np.atleast_2d(np.asarray(rgb, np.float64)) @ M.T
    s = fundamental_from_xyz(xyz, A).T
    return np.clip(s, 0.0, 1.0) if clamp else s


def spectrum_to_rgb(spec, quad_w, cmf, rgb_to_xyz=None):
    A = color_basis(quad_w, cmf)
    M = SRGB_TO_XYZ if rgb_to_xyz is None else np.asarray(rgb_to_xyz, np.float64)
    xyz = np.atleast_2d(np.asarray(spec, np.float64)) @ A
    return np.linalg.solve(M, xyz.T).T
