"""Python binding of the RTSDF C ABI (argument marshalling only).

Every step of the pipeline runs in librtsdf's CUDA kernels; PyTorch provides
device memory for caller-owned buffers and the CUDA stream.  Method names
follow the C entry points of ``include/rtsdf.h``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import call


class _CudaView:
    """Zero-copy descriptor of a device buffer (``__cuda_array_interface__``)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _host_or_device(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            t = a.detach().contiguous()
            want = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
            if t.dtype != want:
                t = t.to(want)
            return t.data_ptr(), int(t.is_cuda), t
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, 0, arr


def make_config(coarse_n, bmin=(0.0, 0.0, 0.0), extent=1.0, beta_vox=0.5, alpha=1.0, seed=0, stream=0):
    cfg = _abi.Config()
    cfg.bmin = (ctypes.c_float * 3)(*[float(b) for b in bmin])
    cfg.extent = float(extent)
    cfg.coarse_n = int(coarse_n)
    cfg.beta_vox = float(beta_vox)
    cfg.alpha = float(alpha)
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    cfg.stream = stream
    return cfg


class RTSDF:
    """One SDF generator context (coarse grid N^3, fine grid (2N)^3) on one GPU.

    Sec. 2 of the paper: voxelize -> jump flood (coarse SDF, Sec. 2.1) ->
    mask + ray trace with Eq. 1 accumulation (fine SDF, Sec. 2.2) -> soft
    shadows (Sec. 2.3).
    """

    def __init__(self, coarse_n: int, bmin=(0.0, 0.0, 0.0), extent: float = 1.0, beta_vox: float = 0.5,
                 alpha: float = 1.0, seed: int = 0, stream=None, device=None, _borrowed=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("RTSDF needs a CUDA device (sm_103a); there is no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._owned = _borrowed is None
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            if _borrowed is not None:
                h = _borrowed
            else:
                cfg = make_config(coarse_n, bmin, extent, beta_vox, alpha, seed, self.stream.cuda_stream)
                h = ctypes.c_void_p()
                call("rtsdf_create", ctypes.byref(cfg), ctypes.byref(h))
        self._h = h
        self.coarse_n = int(coarse_n)
        self.fine_n = 2 * int(coarse_n)
        self.bmin = tuple(float(b) for b in bmin)
        self.extent = float(extent)
        self.beta_vox, self.alpha, self.seed = float(beta_vox), float(alpha), int(seed)

    # ------------------------------------------------------------ lifecycle
    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            if self._owned:
                _abi.lib().rtsdf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def set_stream(self, stream) -> None:
        call("rtsdf_set_stream", self._h, stream.cuda_stream)
        self.stream = stream

    # ------------------------------------------------------------ scene
    def upload_mesh(self, verts, tris) -> None:
        pv, dv, kv = _host_or_device(verts, np.float32)
        pt, dt, kt = _host_or_device(tris, np.int32)
        if dv != dt:
            raise ValueError("verts and tris must both be host or both be device buffers")
        nv = int(np.prod(kv.shape)) // 3
        nt = int(np.prod(kt.shape)) // 3
        call("rtsdf_upload_mesh", self._h, pv, nv, pt, nt, dv)
        self._nt = nt

    def set_objects(self, vert_object, n_objects: int) -> None:
        p, d, k = _host_or_device(vert_object, np.int32)
        call("rtsdf_set_objects", self._h, p, int(n_objects), d)

    def move_objects(self, translations) -> None:
        p, d, k = _host_or_device(translations, np.float32)
        call("rtsdf_move_objects", self._h, p, d)
        self._keep = k   # device buffers must outlive the enqueued copy

    def transform_objects(self, xforms) -> None:
        """Rigid transform per object: float32 [n_objects, 3, 4] (rows of
        [R | t]) or [n_objects, 12]; see rtsdf_transform_objects."""
        p, d, k = _host_or_device(xforms, np.float32)
        call("rtsdf_transform_objects", self._h, p, d)
        self._keep = k   # device buffers must outlive the enqueued copy

    def set_reset(self, on: bool) -> None:
        """Reset in changed regions after moves (default on); see rtsdf_set_reset."""
        call("rtsdf_set_reset", self._h, int(bool(on)))

    def get_reset(self) -> bool:
        v = ctypes.c_int32()
        call("rtsdf_get_reset", self._h, ctypes.byref(v))
        return bool(v.value)

    def build_bvh(self, refit: bool = False) -> None:
        call("rtsdf_build_bvh", self._h, int(bool(refit)))

    BVH_BUILDERS = {"lbvh": 0, "sah": 1, "two_level": 2}

    def set_bvh_builder(self, builder: str) -> None:
        """Topology of the next full build: "sah" (binned surface-area
        heuristic, the default), "lbvh" (Morton radix tree) or "two_level"
        (an SAH subtree per object under a top tree that every refit
        rebuilds)."""
        call("rtsdf_set_bvh_builder", self._h, self.BVH_BUILDERS[builder])

    def get_bvh_builder(self) -> str:
        v = ctypes.c_int32()
        call("rtsdf_get_bvh_builder", self._h, ctypes.byref(v))
        return {0: "lbvh", 1: "sah", 2: "two_level"}[v.value]

    def bvh_topology(self):
        """(children int32 [nt-1, 2], leaf_tri int32 [nt], root) of the last
        build; a child < 0 is ~(leaf position)."""
        nt = getattr(self, "_nt", 0)
        ch = np.zeros((max(nt - 1, 0), 2), np.int32)
        lt = np.zeros(nt, np.int32)
        root = ctypes.c_int32()
        call("rtsdf_get_bvh_topology", self._h, ch.ctypes.data if ch.size else None,
             lt.ctypes.data if lt.size else None, ctypes.byref(root))
        return ch, lt, root.value

    # ------------------------------------------------------------ Sec. 2.1-2.2
    def voxelize(self) -> None:
        call("rtsdf_voxelize", self._h)

    def jfa(self) -> None:
        call("rtsdf_jfa", self._h)

    def trace(self, d_vox: float, rays_per_texel: int, frame: int) -> None:
        call("rtsdf_trace", self._h, float(d_vox), int(rays_per_texel), int(frame))

    def update(self, d_vox: float, rays_per_texel: int, frame: int) -> None:
        """One frame of Sec. 2.1-2.2: voxelize, jump flood, mask and trace."""
        self.voxelize()
        self.jfa()
        self.trace(d_vox, rays_per_texel, frame)

    # ------------------------------------------------------------ Sec. 2.3
    @staticmethod
    def _light3(light):
        import torch
        if isinstance(light, torch.Tensor):
            light = light.detach().double().cpu().numpy()
        l = [float(x) for x in np.asarray(light, dtype=np.float64).reshape(3)]
        return (ctypes.c_float * 3)(*l)

    def shadow(self, pos, nrm, light, k: float = 8.0, steps: int = 64, step_max_vox: float = 4.0,
               eps_vox: float = 1.0, sdf=None, out=None, jitter_vox: float = 0.0, frame: int = 0):
        """Soft-shadow visibility per shading point; jitter_vox > 0 jitters
        each ray origin toward the light (rtsdf_shadow_jittered)."""
        import torch
        pos = pos.contiguous()
        nrm = nrm.contiguous()
        npix = pos.numel() // 3
        vis = out if out is not None else torch.empty(pos.shape[:-1], device=pos.device, dtype=torch.float32)
        sp = 0 if sdf is None else sdf.contiguous().data_ptr()
        if jitter_vox:
            call("rtsdf_shadow_jittered", self._h, sp, pos.data_ptr(), nrm.data_ptr(), npix, self._light3(light),
                 float(k), int(steps), float(step_max_vox), float(eps_vox), float(jitter_vox), int(frame),
                 vis.data_ptr())
        else:
            call("rtsdf_shadow", self._h, sp, pos.data_ptr(), nrm.data_ptr(), npix, self._light3(light), float(k),
                 int(steps), float(step_max_vox), float(eps_vox), vis.data_ptr())
        return vis

    def shadow_fallback(self, pos, nrm, light, vis=None, eps_vox: float = 1.0, blocked=None):
        """Thin-surface fallback: exact occlusion toward the light from the
        march's origin; blocked points get ``vis`` = 0 in place.  ``blocked``
        (uint8 [npix] device, optional) receives the occlusion flags."""
        pos = pos.contiguous()
        nrm = nrm.contiguous()
        if vis is not None and not vis.is_contiguous():
            raise ValueError("vis must be contiguous (it is updated in place)")
        call("rtsdf_shadow_fallback", self._h, pos.data_ptr(), nrm.data_ptr(), pos.numel() // 3,
             self._light3(light), float(eps_vox), vis.data_ptr() if vis is not None else None,
             blocked.data_ptr() if blocked is not None else None)
        return vis

    def taa_resolve(self, cur, hist, blend: float = 0.1):
        """In-place temporal anti-aliasing of ``hist`` [H, W] toward ``cur``."""
        if cur.dim() != 2 or tuple(cur.shape) != tuple(hist.shape) or not hist.is_contiguous():
            raise ValueError("cur and hist must be [H, W] and hist contiguous")
        cur = cur.contiguous()
        call("rtsdf_taa_resolve", self._h, cur.data_ptr(), hist.data_ptr(), int(cur.shape[1]), int(cur.shape[0]),
             float(blend))
        return hist

    def shadow_backward(self, pos, nrm, light, dvis, dsdf, dlight, k: float = 8.0, steps: int = 64,
                        step_max_vox: float = 4.0, eps_vox: float = 1.0, sdf=None) -> None:
        pos = pos.contiguous()
        nrm = nrm.contiguous()
        dvis = dvis.contiguous()
        sp = 0 if sdf is None else sdf.contiguous().data_ptr()
        call("rtsdf_shadow_backward", self._h, sp, pos.data_ptr(), nrm.data_ptr(), pos.numel() // 3,
             self._light3(light), float(k), int(steps), float(step_max_vox), float(eps_vox), dvis.data_ptr(),
             dsdf.data_ptr(), dlight.data_ptr())

    # ------------------------------------------------------------ inspection
    def grids(self) -> dict:
        """Zero-copy torch views of the context's grids (valid while it lives)."""
        import torch
        g = _abi.Grids()
        call("rtsdf_get_grids", self._h, ctypes.byref(g))
        nc3, nf3 = self.coarse_n ** 3, self.fine_n ** 3
        dev = self.device

        def view(ptr, n, ts):
            return torch.as_tensor(_CudaView(ptr, (n,), ts), device=dev)

        return {
            "seeds": view(g.seeds, nc3, "<u4"),
            "coarse": view(g.coarse, nc3, "<f4"),
            "fine": view(g.fine, nf3, "<f4"),
            "accum": view(g.accum, nf3, "<f4"),
            "counts": view(g.counts, nf3, "<u4"),
            "masked": view(g.masked, max(self.masked_count(), 1), "<u4"),
        }

    def masked_count(self) -> int:
        n = ctypes.c_int64()
        call("rtsdf_get_masked_count", self._h, ctypes.byref(n))
        return int(n.value)

    def set_profiling(self, on: bool) -> None:
        call("rtsdf_set_profiling", self._h, int(bool(on)))

    def get_tuning(self) -> dict:
        t = _abi.Tuning()
        call("rtsdf_get_tuning", self._h, ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in _abi.Tuning._fields_}

    def set_tuning(self, **kw) -> None:
        cur = self.get_tuning()
        cur.update(kw)
        t = _abi.Tuning(**cur)
        call("rtsdf_set_tuning", self._h, ctypes.byref(t))

    def autotune(self, d_vox: float, rays_per_texel: int, frame: int, use_cache: bool = True) -> dict:
        """Time candidate launch parameters on this scene and keep the fastest
        (the accumulated SDF is saved and restored)."""
        t = _abi.Tuning()
        call("rtsdf_autotune", self._h, float(d_vox), int(rays_per_texel), int(frame), int(bool(use_cache)),
             ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in _abi.Tuning._fields_}

    SIGN_MODES = {"vote": 0, "nearest": 1}

    def set_sign_mode(self, mode: str) -> None:
        """"vote" (Sec. 2.2's front/back vote) or "nearest" (the face of the
        nearest hit; rays capped at the texel's accumulated distance).
        Changing the mode restarts the accumulation."""
        call("rtsdf_set_sign_mode", self._h, self.SIGN_MODES[mode])

    def get_sign_mode(self) -> str:
        v = ctypes.c_int32()
        call("rtsdf_get_sign_mode", self._h, ctypes.byref(v))
        return {0: "vote", 1: "nearest"}[v.value]

    def set_counting(self, on: bool) -> None:
        call("rtsdf_set_counting", self._h, int(bool(on)))

    def stats(self) -> dict:
        """Counters and per-stage device ms since the previous call."""
        s = _abi.Stats()
        call("rtsdf_get_stats", self._h, ctypes.byref(s))
        out = {name: getattr(s, name) for name in ("launches", "n_masked_texels", "jfa_passes", "bvh_depth",
                                                    "rays", "node_visits", "tri_tests", "lane_slots",
                                                    "leaf_slots")}
        out["stage_ms"] = {k: float(s.stage_ms[i]) for i, k in enumerate(_abi.STAGES)}
        out["stage_calls"] = {k: int(s.stage_calls[i]) for i, k in enumerate(_abi.STAGES)}
        return out

    def save_state(self) -> bytes:
        n = ctypes.c_size_t()
        call("rtsdf_state_size", self._h, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        call("rtsdf_save_state", self._h, ctypes.addressof(buf), n.value)
        return buf.raw

    def load_state(self, data: bytes) -> None:
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        call("rtsdf_load_state", self._h, ctypes.addressof(buf), len(data))

    def sync(self) -> None:
        call("rtsdf_sync", self._h)


class RTSDFBatch:
    """Many independent scenes updated by one persistent launch per frame
    (``rtsdf_batch_*``).  ``scenes`` is a list of dicts with the RTSDF
    constructor's keyword arguments (coarse_n, bmin, extent, beta_vox,
    alpha, seed)."""

    def __init__(self, scenes, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("RTSDFBatch needs a CUDA device (sm_103a); there is no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device())
        n = len(scenes)
        arr = (_abi.Config * n)()
        sptr = 0 if stream is None else stream.cuda_stream
        for i, sc in enumerate(scenes):
            arr[i] = make_config(stream=sptr, **sc)
        h = ctypes.c_void_p()
        call("rtsdf_batch_create", arr, n, ctypes.byref(h))
        self._h = h
        self.scenes = []
        for i, sc in enumerate(scenes):
            ch = ctypes.c_void_p()
            call("rtsdf_batch_context", h, i, ctypes.byref(ch))
            kw = dict(sc)
            self.scenes.append(RTSDF(_borrowed=ch, **kw))

    def frame(self, d_vox: float, rays_per_texel: int, frame: int) -> None:
        call("rtsdf_batch_frame", self._h, float(d_vox), int(rays_per_texel), int(frame))

    def sync(self) -> None:
        call("rtsdf_batch_sync", self._h)

    def get_tuning(self) -> dict:
        t = _abi.BatchTuning()
        call("rtsdf_batch_get_tuning", self._h, ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in _abi.BatchTuning._fields_}

    def set_tuning(self, **kw) -> None:
        cur = self.get_tuning()
        cur.update(kw)
        t = _abi.BatchTuning(**cur)
        call("rtsdf_batch_set_tuning", self._h, ctypes.byref(t))

    def autotune(self, d_vox: float, rays_per_texel: int, frame: int, use_cache: bool = True) -> dict:
        t = _abi.BatchTuning()
        call("rtsdf_batch_autotune", self._h, float(d_vox), int(rays_per_texel), int(frame), int(bool(use_cache)),
             ctypes.byref(t))
        return {k: getattr(t, k) for k, _ in _abi.BatchTuning._fields_}

    def stats(self) -> dict:
        s = _abi.BatchInfo()
        call("rtsdf_batch_stats", self._h, ctypes.byref(s))
        out = {k: getattr(s, k) for k, _ in _abi.BatchInfo._fields_ if k != "stage_ms"}
        names = ("clear", "voxelize", "voxelize_large", "jfa", "mask", "trace", "finalize")
        out["stage_ms"] = {n: round(float(s.stage_ms[i]), 4) for i, n in enumerate(names)}
        return out

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            for sc in self.scenes:
                sc._h = ctypes.c_void_p()
            _abi.lib().rtsdf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
