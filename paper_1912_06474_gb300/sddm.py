"""Thin Python binding of libsddm.so (include/sddm.h), argument marshalling only.

Every step of rendering runs in the library's CUDA kernels; this module turns
scene inputs (see ``scenes``) into the C ABI calls and uses PyTorch only to
hold device buffers and to pass the current CUDA stream. There is no CPU
fallback: if the library is missing or cannot load, importing raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsddm.so")

OK = 0
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_QUEUE_OVERFLOW = -1, -2, -3, -4
ERR_TIMEOUT, ERR_NOT_BUILT, ERR_MLP_UNTRAINED, ERR_DEVICE_CHECK = -5, -6, -7, -8
BSDF_EXACT, BSDF_MLP, BSDF_MLP_RAW = 0, 1, 2
MLP_PARAMS = 8770
METHOD_MEGAKERNEL, METHOD_DDM = 0, 1
METHODS = {"megakernel": METHOD_MEGAKERNEL, "ddm": METHOD_DDM}
BSDFS = {"exact": BSDF_EXACT, "mlp": BSDF_MLP, "mlp_raw": BSDF_MLP_RAW}

EXPORTED = ["sddm_create", "sddm_destroy", "sddm_last_error", "sddm_version", "sddm_set_spectrum",
            "sddm_add_lambertian", "sddm_add_conductor", "sddm_add_glass_slab", "sddm_add_coated_glass",
            "sddm_rgb_to_spectrum", "sddm_render_photon_map",
            "sddm_render_progressive_photon_map",
            "sddm_add_emitter",
            "sddm_add_diffuse_emitter", "sddm_set_mesh", "sddm_build", "sddm_render", "sddm_render_host",
            "sddm_autotune", "sddm_glass_eval", "sddm_philox", "sddm_set_profiling",
            "sddm_render_noalloc", "sddm_mlp_train", "sddm_mlp_get_weights", "sddm_mlp_set_weights",
            "sddm_mlp_save", "sddm_mlp_load", "sddm_mlp_grad"]


class SddmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sddm error {code}: {msg}")
        self.code = code


class BuildOpts(C.Structure):
    _fields_ = [("grid", C.c_int * 3), ("leaf_size", C.c_int), ("sah_bins", C.c_int),
                ("queue_capacity", C.c_int64), ("blocks_per_sm", C.c_int), ("paths_in_flight", C.c_int64),
                ("bvh_in_host_memory", C.c_int), ("cell_cache_bytes", C.c_int64), ("continue_cells", C.c_int),
                ("handoff_waves", C.c_int)]


class MlpTrainOpts(C.Structure):
    _fields_ = [("samples", C.c_int64), ("steps", C.c_int), ("batch", C.c_int), ("lr", C.c_float),
                ("seed", C.c_uint32), ("thick_min", C.c_float), ("thick_max", C.c_float), ("resume", C.c_int)]


class MlpReport(C.Structure):
    _fields_ = [("final_loss", C.c_double), ("max_abs_err_R", C.c_double), ("max_abs_err_T", C.c_double),
                ("train_ms", C.c_double), ("tflops", C.c_double), ("steps", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("ortho_height", C.c_float)]


class RenderDesc(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("spp", C.c_int), ("max_depth", C.c_int),
                ("seed", C.c_uint32), ("render_id", C.c_uint32), ("nee", C.c_int), ("bsdf_mode", C.c_int),
                ("method", C.c_int), ("camera", Camera), ("glass_s", C.c_void_p), ("xyz_out", C.c_void_p),
                ("aov_sample_xyz", C.c_void_p), ("aov_first_prim", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("paths", C.c_int64), ("segments_ext", C.c_int64), ("segments_shadow", C.c_int64),
                ("crossings", C.c_int64), ("glass_queries", C.c_int64), ("mlp_fallbacks", C.c_int64),
                ("gpu_ms", C.c_double), ("kernel_launches", C.c_int64), ("trace_ms", C.c_double),
                ("trace_launches", C.c_int64), ("node_visits", C.c_int64), ("tri_tests", C.c_int64),
                ("ray_visits", C.c_int64), ("mlp_batches", C.c_int64), ("cache_loads", C.c_int64),
                ("cache_hits", C.c_int64), ("cache_bytes_loaded", C.c_int64), ("mlp_ms", C.c_double),
                ("mlp_rows", C.c_int64), ("ray_continues", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PhotonStats(C.Structure):
    _fields_ = [("photons", C.c_int64), ("photon_segments", C.c_int64), ("stored", C.c_int64),
                ("grid_cells", C.c_int64), ("photon_ms", C.c_double), ("kernel_launches", C.c_int64),
                ("stored_caustic", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P, I = C.c_void_p, C.c_int
    sig = {
        "sddm_create": ([C.POINTER(C.c_void_p), I, P], I),
        "sddm_destroy": ([P], I),
        "sddm_last_error": ([], C.c_char_p),
        "sddm_version": ([], C.c_char_p),
        "sddm_set_spectrum": ([P, I, P, P, P], I),
        "sddm_add_lambertian": ([P, P, P], I),
        "sddm_add_conductor": ([P, P, P, P], I),
        "sddm_add_glass_slab": ([P, P, P, P, C.c_float, C.c_float, P], I),
        "sddm_add_coated_glass": ([P, P, P, P, C.c_float, C.c_float, C.c_int, P, P, P, P, P], I),
        "sddm_rgb_to_spectrum": ([P, C.c_int, P, P, P, C.c_int], I),
        "sddm_add_emitter": ([P, P, P], I),
        "sddm_add_diffuse_emitter": ([P, P, P, P], I),
        "sddm_set_mesh": ([P, P, I, P, I, P, P], I),
        "sddm_build": ([P, C.POINTER(BuildOpts)], I),
        "sddm_render": ([P, C.POINTER(RenderDesc), I, C.POINTER(Stats)], I),
        "sddm_render_host": ([P, C.POINTER(RenderDesc), I, C.POINTER(Stats)], I),
        "sddm_autotune": ([P, C.POINTER(RenderDesc), I, C.POINTER(BuildOpts)], I),
        "sddm_glass_eval": ([P, C.c_uint32, I, P, P, P, P, P, P, I], I),
        "sddm_philox": ([P, I, P, C.c_uint32, C.c_uint32, P], I),
        "sddm_set_profiling": ([P, I], I),
        "sddm_render_noalloc": ([P, C.POINTER(RenderDesc), C.POINTER(Stats)], I),
        "sddm_render_photon_map": ([P, C.POINTER(RenderDesc), C.c_int64, C.c_float, C.c_float, C.POINTER(Stats),
                                    C.POINTER(PhotonStats)], I),
        "sddm_render_progressive_photon_map": ([P, C.POINTER(RenderDesc), I, C.c_int64, C.c_float, C.c_float,
                                                C.c_float, C.POINTER(Stats), C.POINTER(PhotonStats)], I),
        "sddm_mlp_train": ([P, C.c_uint32, C.POINTER(MlpTrainOpts), C.POINTER(MlpReport)], I),
        "sddm_mlp_get_weights": ([P, C.c_uint32, P], I),
        "sddm_mlp_set_weights": ([P, C.c_uint32, P, C.c_float, C.c_float], I),
        "sddm_mlp_save": ([P, C.c_uint32, C.c_char_p], I),
        "sddm_mlp_load": ([P, C.c_uint32, C.c_char_p], I),
        "sddm_mlp_grad": ([P, I, P, P, P, P, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def version() -> str:
    return lib.sddm_version().decode()


def _check(rc):
    if rc != OK:
        raise SddmError(rc, lib.sddm_last_error().decode(errors="replace"))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Context:
    """One libsddm context bound to a CUDA device and stream, holding a scene."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        self._torch_stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        _check(lib.sddm_create(C.byref(h), int(device), _stream_handle(self._torch_stream)))
        self._h = h
        self.scene = None
        self.n_mat = 0
        self.last_stats = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.sddm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # -- scene --------------------------------------------------------------
    def set_scene(self, scene):
        """sddm_set_spectrum + sddm_add_* (in material order) + sddm_set_mesh."""
        from . import scenes as S
        h = self._h
        lam, w, cmf = _f32(scene.lam), _f32(scene.quad_w), _f32(scene.cmf)
        _check(lib.sddm_set_spectrum(h, scene.L, _ptr(lam), _ptr(w), _ptr(cmf)))
        mid = C.c_uint32()
        for i, m in enumerate(scene.materials):
            if m.kind == S.LAMBERT:
                _check(lib.sddm_add_lambertian(h, _ptr(_f32(m.rho)), C.byref(mid)))
            elif m.kind == S.CONDUCTOR:
                _check(lib.sddm_add_conductor(h, _ptr(_f32(m.n)), _ptr(_f32(m.k)), C.byref(mid)))
            elif m.kind == S.GLASS and m.layers:
                fn = _f32(np.stack([f["n"] for f in m.layers]))
                fk = _f32(np.stack([f["k"] for f in m.layers]))
                fd = _f32(np.stack([f["dk"] for f in m.layers]))
                ft = _f32([f["t_nm"] for f in m.layers])
                _check(lib.sddm_add_coated_glass(h, _ptr(_f32(m.n)), _ptr(_f32(m.alpha_clear)),
                                                 _ptr(_f32(m.dalpha)), float(m.thickness_m), float(m.s_default),
                                                 len(m.layers), _ptr(fn), _ptr(fk), _ptr(fd), _ptr(ft),
                                                 C.byref(mid)))
            elif m.kind == S.GLASS:
                _check(lib.sddm_add_glass_slab(h, _ptr(_f32(m.n)), _ptr(_f32(m.alpha_clear)),
                                               _ptr(_f32(m.dalpha)), float(m.thickness_m),
                                               float(m.s_default), C.byref(mid)))
            elif m.kind == S.EMITTER:
                _check(lib.sddm_add_emitter(h, _ptr(_f32(m.Le)), C.byref(mid)))
            elif m.kind == S.DIFFUSE_EMITTER:
                _check(lib.sddm_add_diffuse_emitter(h, _ptr(_f32(m.rho)), _ptr(_f32(m.Le)), C.byref(mid)))
            else:
                raise ValueError(f"material {i}: unknown kind {m.kind}")
            assert mid.value == i
        V = _f32(scene.V)
        F = np.ascontiguousarray(scene.F, np.uint32)
        M = np.ascontiguousarray(scene.mat_id, np.uint32)
        O = np.ascontiguousarray(scene.obj_id, np.uint32)
        _check(lib.sddm_set_mesh(h, _ptr(V), int(V.shape[0]), _ptr(F), int(F.shape[0]), _ptr(M), _ptr(O)))
        self.scene = scene
        self.n_mat = len(scene.materials)

    def build(self, grid=(1, 1, 1), leaf_size=4, sah_bins=16, queue_capacity=0, blocks_per_sm=0,
              paths_in_flight=0, bvh_in_host_memory=False, cell_cache_bytes=0, continue_cells=False,
              handoff_waves=0):
        o = BuildOpts((C.c_int * 3)(*grid), leaf_size, sah_bins, queue_capacity, blocks_per_sm,
                      paths_in_flight, 1 if bvh_in_host_memory else 0, int(cell_cache_bytes),
                      1 if continue_cells else 0, int(handoff_waves))
        _check(lib.sddm_build(self._h, C.byref(o)))
        self.build_opts = o

    # -- render -------------------------------------------------------------
    def _descs(self, specs, method, bsdf, outs, aov_x, aov_p):
        keep = []
        arr = (RenderDesc * len(specs))()
        for r, sp in enumerate(specs):
            cam = sp.camera if sp.camera is not None else self.scene.camera
            d = arr[r]
            d.width, d.height, d.spp, d.max_depth = sp.width, sp.height, sp.spp, sp.max_depth
            d.seed, d.render_id = sp.seed & 0xFFFFFFFF, sp.render_id & 0xFFFFFFFF
            d.nee = 1 if sp.nee else 0
            d.bsdf_mode = BSDFS[bsdf]
            d.method = METHODS[method]
            d.camera = Camera((C.c_float * 3)(*cam.pos), (C.c_float * 3)(*cam.look), (C.c_float * 3)(*cam.up),
                              float(cam.vfov_deg), float(cam.ortho_height))
            if sp.glass_s:
                s = np.full(self.n_mat, -1.0, np.float32)
                for m, v in sp.glass_s.items():
                    s[int(m)] = float(v)
                keep.append(s)
                d.glass_s = s.ctypes.data
            else:
                d.glass_s = None
            d.xyz_out = outs[r]
            d.aov_sample_xyz = aov_x[r] if aov_x else None
            d.aov_first_prim = aov_p[r] if aov_p else None
        return arr, keep

    def render(self, specs, method="ddm", bsdf="exact", aov=False):
        """sddm_render into fresh CUDA tensors. Returns (images, stats[, aov]):
        images [H,W,3] float32 per render; aov = (sample_xyz [H*W*spp,3], first_prim)."""
        import torch
        if not isinstance(specs, (list, tuple)):
            specs = [specs]
        dev = torch.device("cuda", self.device)
        imgs = [torch.empty((sp.height, sp.width, 3), dtype=torch.float32, device=dev) for sp in specs]
        ax = ap = None
        if aov:
            ax = [torch.empty((sp.n_paths, 3), dtype=torch.float32, device=dev) for sp in specs]
            ap = [torch.empty((sp.n_paths,), dtype=torch.int32, device=dev) for sp in specs]
        arr, _keep = self._descs(specs, method, bsdf, [t.data_ptr() for t in imgs],
                                 [t.data_ptr() for t in ax] if ax else None,
                                 [t.data_ptr() for t in ap] if ap else None)
        st = Stats()
        _check(lib.sddm_render(self._h, arr, len(specs), C.byref(st)))
        self.last_stats = st.as_dict()
        if aov:
            return imgs, self.last_stats, (ax, ap)
        return imgs, self.last_stats

    def render_into(self, specs, outs, method="ddm", bsdf="exact"):
        """sddm_render into caller-provided CUDA tensors (no allocation)."""
        arr, _keep = self._descs(specs, method, bsdf, [t.data_ptr() for t in outs], None, None)
        st = Stats()
        _check(lib.sddm_render(self._h, arr, len(specs), C.byref(st)))
        self.last_stats = st.as_dict()
        return self.last_stats

    def render_noalloc(self, spec, out):
        """sddm_render_noalloc: one megakernel render into the caller's CUDA tensor
        ``out`` [H,W,3] float32; the library allocates nothing during the call."""
        arr, _keep = self._descs([spec], "megakernel", "exact", [out.data_ptr()], None, None)
        st = Stats()
        _check(lib.sddm_render_noalloc(self._h, arr, C.byref(st)))
        self.last_stats = st.as_dict()
        return self.last_stats

    def render_photon_map(self, spec, n_photons, radius, method="ddm", bsdf="exact", caustic_radius=0.0):
        """sddm_render_photon_map: photon pass of n_photons from the lights, then
        the camera pass gathering the map within ``radius`` at the first diffuse
        vertex, both by ``method``; with ``caustic_radius`` > 0 the caustic
        photons form a second map gathered within it. Returns (image [H,W,3]
        CUDA float32, stats, photon stats)."""
        import torch
        img = torch.empty((spec.height, spec.width, 3), dtype=torch.float32, device=torch.device("cuda", self.device))
        arr, _keep = self._descs([spec], method, bsdf, [img.data_ptr()], None, None)
        st, pst = Stats(), PhotonStats()
        _check(lib.sddm_render_photon_map(self._h, arr, int(n_photons), float(radius), float(caustic_radius),
                                          C.byref(st), C.byref(pst)))
        self.last_stats = st.as_dict()
        return img, self.last_stats, pst.as_dict()

    def render_progressive_photon_map(self, spec, n_passes, n_photons, radius, alpha=0.7, method="ddm",
                                      bsdf="exact", caustic_radius=0.0):
        """sddm_render_progressive_photon_map: the mean of n_passes photon-mapping
        renders (render ids spec.render_id + j - 1) with gather radii shrinking
        by (j + alpha) / (j + 1) in area per pass. Returns (image, stats, photon stats)."""
        import torch
        img = torch.empty((spec.height, spec.width, 3), dtype=torch.float32, device=torch.device("cuda", self.device))
        arr, _keep = self._descs([spec], method, bsdf, [img.data_ptr()], None, None)
        st, pst = Stats(), PhotonStats()
        _check(lib.sddm_render_progressive_photon_map(self._h, arr, int(n_passes), int(n_photons), float(radius),
                                                      float(caustic_radius), float(alpha), C.byref(st),
                                                      C.byref(pst)))
        self.last_stats = st.as_dict()
        return img, self.last_stats, pst.as_dict()

    def render_host(self, specs, outs: Sequence[np.ndarray], method="ddm", bsdf="exact"):
        """sddm_render_host: outputs are host (pinned or pageable) float32 arrays [H,W,3]."""
        ptrs = []
        for o in outs:
            if isinstance(o, np.ndarray):
                assert o.dtype == np.float32 and o.flags.c_contiguous
                ptrs.append(o.ctypes.data)
            else:   # a CPU torch tensor (possibly pinned)
                assert o.dtype.is_floating_point and o.is_contiguous() and o.device.type == "cpu"
                ptrs.append(o.data_ptr())
        arr, _keep = self._descs(specs, method, bsdf, ptrs, None, None)
        st = Stats()
        _check(lib.sddm_render_host(self._h, arr, len(specs), C.byref(st)))
        self.last_stats = st.as_dict()
        return self.last_stats

    def autotune(self, specs, method="ddm", bsdf="exact"):
        import torch
        dev = torch.device("cuda", self.device)
        imgs = [torch.empty((sp.height, sp.width, 3), dtype=torch.float32, device=dev) for sp in specs]
        arr, _keep = self._descs(specs, method, bsdf, [t.data_ptr() for t in imgs], None, None)
        best = BuildOpts()
        _check(lib.sddm_autotune(self._h, arr, len(specs), C.byref(best)))
        self.build_opts = best
        return dict(grid=tuple(best.grid), leaf_size=best.leaf_size, sah_bins=best.sah_bins,
                    queue_capacity=best.queue_capacity, blocks_per_sm=best.blocks_per_sm,
                    paths_in_flight=best.paths_in_flight, bvh_in_host_memory=bool(best.bvh_in_host_memory),
                    cell_cache_bytes=best.cell_cache_bytes, continue_cells=bool(best.continue_cells),
                    handoff_waves=best.handoff_waves)

    def set_profiling(self, time_trace=False, count_traversal=False, eager=False, test_mlp_timeout=False):
        """sddm_set_profiling: per-launch trace-kernel events, traversal counters,
        or eager launches (all three disable CUDA graph replay); test_mlp_timeout
        makes the surrogate network's wait on the tensor core run out (a test
        of the failure path)."""
        _check(lib.sddm_set_profiling(self._h, (1 if time_trace else 0) | (2 if count_traversal else 0)
                                      | (4 if eager else 0) | (8 if test_mlp_timeout else 0)))

    # -- learned glass surrogate ------------------------------------------------
    def mlp_train(self, mat, samples=0, steps=0, batch=0, lr=0.0, seed=0, thick_min=0.0, thick_max=0.0,
                  resume=False):
        """sddm_mlp_train: train the surrogate of glass material ``mat``; returns the report."""
        o = MlpTrainOpts(samples, steps, batch, lr, seed & 0xFFFFFFFF, thick_min, thick_max, 1 if resume else 0)
        r = MlpReport()
        _check(lib.sddm_mlp_train(self._h, int(mat), C.byref(o), C.byref(r)))
        return r.as_dict()

    def mlp_get_weights(self, mat):
        p = np.zeros(MLP_PARAMS, np.float32)
        _check(lib.sddm_mlp_get_weights(self._h, int(mat), _ptr(p)))
        return p

    def mlp_set_weights(self, mat, params, thick_min=0.002, thick_max=0.010):
        p = _f32(params)
        assert p.shape == (MLP_PARAMS,)
        _check(lib.sddm_mlp_set_weights(self._h, int(mat), _ptr(p), float(thick_min), float(thick_max)))

    def mlp_save(self, mat, path):
        _check(lib.sddm_mlp_save(self._h, int(mat), os.fsencode(path)))

    def mlp_load(self, mat, path):
        _check(lib.sddm_mlp_load(self._h, int(mat), os.fsencode(path)))

    def mlp_grad(self, X, Y, params):
        """sddm_mlp_grad on CUDA tensors X [n,4], Y [n,2], params [8770]; returns (grad, loss)."""
        import torch
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib.sddm_mlp_grad(self._h, int(X.shape[0]), X.data_ptr(), Y.data_ptr(), params.data_ptr(),
                                 grad.data_ptr(), loss.data_ptr()))
        return grad, loss

    # -- test hooks -----------------------------------------------------------
    def glass_eval(self, mat, cos_t, bins, s, thick, mode="exact"):
        """sddm_glass_eval on CUDA tensors; returns (R, T) tensors."""
        import torch
        n = int(cos_t.numel())
        R = torch.empty(n, dtype=torch.float32, device=cos_t.device)
        T = torch.empty_like(R)
        _check(lib.sddm_glass_eval(self._h, int(mat), n, cos_t.data_ptr(), bins.data_ptr(), s.data_ptr(),
                                   thick.data_ptr(), R.data_ptr(), T.data_ptr(), BSDFS[mode]))
        return R, T

    def rgb_to_spectrum(self, rgb, rgb_to_xyz=None, clamp=False):
        """sddm_rgb_to_spectrum: spectra [n, L] (numpy float32) of RGB values [n, 3]
        on the spectrum of the current scene (set_scene first)."""
        rgb = np.ascontiguousarray(np.atleast_2d(rgb), np.float32)
        out = np.zeros((rgb.shape[0], self.scene.L), np.float32)
        m = None if rgb_to_xyz is None else np.ascontiguousarray(rgb_to_xyz, np.float32)
        _check(lib.sddm_rgb_to_spectrum(self._h, int(rgb.shape[0]), _ptr(rgb), _ptr(m) if m is not None else None,
                                        _ptr(out), 1 if clamp else 0))
        return out

    def philox(self, ctr, key0, key1):
        """sddm_philox on a CUDA int32/uint32 tensor [n,4]; returns [n,4] words (int32 view)."""
        import torch
        out = torch.empty_like(ctr)
        _check(lib.sddm_philox(self._h, int(ctr.shape[0]), ctr.data_ptr(), key0 & 0xFFFFFFFF,
                               key1 & 0xFFFFFFFF, out.data_ptr()))
        return out
