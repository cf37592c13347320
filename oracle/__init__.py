"""RTSDF CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.

A plain, slow and obviously-correct CPU restatement of the method of
"RTSDF: Generating Signed Distance Fields in Real Time for Soft Shadow
Rendering" (Tan, Chua, Koh, Bhojan, Pacific Graphics 2020):

* Sec. 2.1 -- conservative voxelization, 3D jump flooding, coarse SDF with
  the bias beta subtracted;
* Sec. 2.2 -- the near-surface mask (Eq. 1's case split), random sphere
  directions from a counter-based Philox stream, brute-force closest-hit ray
  casting, the Eq. 1 temporal minimum and the front/back vote for the sign;
* Sec. 2.3 -- the sphere-traced soft-shadow visibility and its reverse-mode
  derivative.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
implementation (``paper_2210_04449_gb300``) and never imports it.

Loops live in ``rtsdf_oracle.c`` (built by :func:`build` with gcc,
``-ffp-contract=off``); the elementwise steps (coarse SDF, mask, Eq. 1, the
reset rule) are numpy below.  Floating point is fp64, except where a
floating-point result decides an integer result; there both sides use
fp32 with the operation order written out in the C file.

Grids are flat arrays in x-fastest order (index ``x + n*(y + n*z)``).
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtsdf_oracle.c")
LIB_PATH = os.path.join(_HERE, "librtsdf_oracle.so")
_lib = None
_lock = threading.Lock()

i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle's C part (gcc, -O2, OpenMP, no FP contraction)."""
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(_SRC):
        return LIB_PATH
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-fopenmp", "-o", LIB_PATH + ".tmp", _SRC, "-lm"]
    if platform.machine() in ("x86_64", "AMD64"):
        # fmaf() is correctly rounded either way; the hardware FMA is faster.
        cmd.insert(1, "-mfma")
    subprocess.run(cmd, check=True)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        L = ctypes.CDLL(LIB_PATH)
        c_i64, c_int, c_f, c_d, c_u32, c_u64 = (ctypes.c_int64, ctypes.c_int, ctypes.c_float,
                                                 ctypes.c_double, ctypes.c_uint32, ctypes.c_uint64)
        sig = {
            "orc_quant_scale": (c_f, [c_int, c_f]),
            "orc_quantise_vertices": (c_int, [f32p, c_i64, f32p, c_f, c_int, i64p]),
            "orc_voxelize": (c_int, [f32p, c_i64, i32p, c_i64, f32p, c_f, c_int, i32p]),
            "orc_tri_voxel_overlap": (c_int, [i64p, c_int, c_int, c_int]),
            "orc_jfa_passes": (c_int, [c_int]),
            "orc_jfa": (c_int, [i32p, c_int, i32p]),
            "orc_seed_d2": (None, [i32p, c_int, i64p]),
            "orc_edt_brute": (None, [i32p, c_int, i64p]),
            "orc_edt_separable": (None, [i32p, c_int, i64p]),
            "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
            "orc_philox4x64_10": (None, [u64p, u64p, u64p]),
            "orc_sphere_dir": (c_int, [c_u64, c_u32, c_u32, c_u32, f32p]),
            "orc_ray_triangle": (c_int, [f32p, f32p, f32p, f32p, f32p,
                                         ctypes.POINTER(c_f), ctypes.POINTER(c_int)]),
            "orc_texel_centre": (None, [f32p, c_f, c_int, c_i64, f32p]),
            "orc_trace": (None, [f32p, i32p, c_i64, f32p, c_f, c_int, c_u64, c_int, c_int,
                                 i64p, c_i64, f32p, i32p, i32p, i64p, i32p]),
            "orc_trace_bvh": (None, [f32p, i32p, c_i64, f32p, c_f, c_int, c_u64, c_int, c_int,
                                     i64p, c_i64, f32p, i32p, i32p, i64p, i32p]),
            "orc_cast_rays": (None, [f32p, i32p, c_i64, f32p, f32p, c_i64, f32p, i32p, i64p]),
            "orc_cast_rays_bvh": (None, [f32p, i32p, c_i64, f32p, f32p, c_i64, f32p, i32p, i64p]),
            "orc_point_mesh_distance": (None, [f32p, i32p, c_i64, f64p, c_i64, f64p]),
            "orc_sample": (c_d, [f32p, c_int, f64p, c_d, f64p]),
            "orc_shadow": (None, [f32p, c_int, f64p, c_d, f32p, f32p, c_i64, f64p, c_d, c_int,
                                  c_d, c_d, f64p, ctypes.c_void_p, ctypes.c_void_p]),
            "orc_shadow_jitter": (None, [c_u64, c_u32, c_i64, f64p]),
            "orc_shadow_margin": (None, [f32p, c_int, f64p, c_d, f32p, f32p, c_i64, f64p, c_d, c_int,
                                         c_d, c_d, f64p]),
            "orc_shadow_exact": (None, [f32p, i32p, c_i64, f32p, f32p, c_i64, f32p, c_f, i32p]),
            "orc_shadow_grad": (None, [f32p, c_int, f64p, c_d, f32p, f32p, c_i64, f64p, c_d, c_int,
                                       c_d, c_d, f64p, f64p, f64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleError(ValueError):
    pass


# ---------------------------------------------------------------------------
# Sec. 2.1 -- voxelization and jump flooding
# ---------------------------------------------------------------------------

def quant_scale(n: int, extent: float) -> np.float32:
    return np.float32(_load().orc_quant_scale(n, extent))


def quantise_vertices(verts, bmin, extent, n):
    v = _f32(verts)
    q = np.zeros(v.size, dtype=np.int64)
    if _load().orc_quantise_vertices(v.reshape(-1), v.shape[0], _f32(bmin), extent, n, q):
        raise OracleError("vertex outside [bmin - extent/2, bmin + 3 extent/2] or not finite")
    return q.reshape(-1, 3)


def voxelize(verts, tris, bmin, extent, n):
    """Occupancy grid: int32 [n^3], linear index where occupied, else -1."""
    v, t = _f32(verts), _i32(tris)
    occ = np.empty(n ** 3, dtype=np.int32)
    rc = _load().orc_voxelize(v.reshape(-1), v.shape[0], t.reshape(-1), t.shape[0],
                              _f32(bmin), extent, n, occ)
    if rc == -1:
        raise OracleError("vertex outside [bmin - extent/2, bmin + 3 extent/2] or not finite")
    if rc == -2:
        raise OracleError("triangle index out of range")
    return occ


def tri_voxel_overlap(qtri, x, y, z) -> bool:
    return bool(_load().orc_tri_voxel_overlap(np.ascontiguousarray(qtri, np.int64).reshape(-1), x, y, z))


def jfa_passes(n: int) -> int:
    return int(_load().orc_jfa_passes(n))


def jfa(occ, n):
    """Jump flooding: nearest-seed linear index per voxel (-1: no seed)."""
    out = np.empty(n ** 3, dtype=np.int32)
    passes = _load().orc_jfa(_i32(occ), n, out)
    return out, passes


def seed_d2(seeds, n):
    d2 = np.empty(n ** 3, dtype=np.int64)
    _load().orc_seed_d2(_i32(seeds), n, d2)
    return d2


def edt_brute(occ, n):
    d2 = np.empty(n ** 3, dtype=np.int64)
    _load().orc_edt_brute(_i32(occ), n, d2)
    return d2


def edt_separable(occ, n):
    d2 = np.empty(n ** 3, dtype=np.int64)
    _load().orc_edt_separable(_i32(occ), n, d2)
    return d2


def coarse_sdf(seeds, n, extent, beta_vox):
    """Sec. 2.1: distance to the nearest seed voxel (centre to centre) minus
    beta (in coarse voxels); fp64; +inf where the grid has no seed."""
    h = extent / n
    d2 = seed_d2(seeds, n)
    c = np.full(n ** 3, np.inf)
    ok = d2 >= 0
    c[ok] = h * np.sqrt(d2[ok].astype(np.float64)) - beta_vox * h
    return c


# ---------------------------------------------------------------------------
# Sec. 2.2 -- near-surface mask (Eq. 1's case split)
# ---------------------------------------------------------------------------

def mask_threshold(d_vox: float, beta_vox: float) -> int:
    """c <= d (coarse voxels) with c = sqrt(D2) - beta  <=>  D2 <= floor((d+beta)^2).
    Returns -1 when no D2 can satisfy it (d + beta < 0)."""
    s = float(np.float32(d_vox)) + float(np.float32(beta_vox))
    if s < 0:
        return -1
    return int(math.floor(s * s))


def parent_index(nc: int):
    """Coarse parent (linear index) of every fine texel of the 2*nc grid."""
    nf = 2 * nc
    j = np.arange(nf ** 3, dtype=np.int64)
    x, y, z = j % nf, (j // nf) % nf, j // (nf * nf)
    return (x >> 1) + nc * ((y >> 1) + nc * (z >> 1))


def mask_fill(seeds, nc, d_vox, beta_vox, c):
    """Fine texel j (grid 2*nc) is masked iff its parent coarse voxel has
    D2 <= T (Eq. 1, first case); unmasked texels take the coarse value c
    (Eq. 1, second case).  Returns (mask bool [nf^3], f_unmasked fp64 with
    NaN at masked texels)."""
    T = mask_threshold(d_vox, beta_vox)
    d2 = seed_d2(seeds, nc)
    par = parent_index(nc)
    pd2 = d2[par]
    mask = (pd2 >= 0) & (pd2 <= T)
    f = np.where(mask, np.nan, c[par])
    return mask, f


# ---------------------------------------------------------------------------
# Sec. 2.2 -- Philox directions, ray casting
# ---------------------------------------------------------------------------

def philox4x32(ctr, key):
    out = np.empty(4, dtype=np.uint32)
    _load().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32), np.ascontiguousarray(key, np.uint32), out)
    return out


def philox4x64(ctr, key):
    out = np.empty(4, dtype=np.uint64)
    _load().orc_philox4x64_10(np.ascontiguousarray(ctr, np.uint64), np.ascontiguousarray(key, np.uint64), out)
    return out


def sphere_dir(seed, texel, frame, ray):
    d = np.empty(3, dtype=np.float32)
    pairs = _load().orc_sphere_dir(int(seed) & (2 ** 64 - 1), int(texel), int(frame), int(ray), d)
    return d, pairs


def ray_triangle(o, d, v0, v1, v2):
    t = ctypes.c_float()
    f = ctypes.c_int()
    hit = _load().orc_ray_triangle(_f32(o), _f32(d), _f32(v0), _f32(v1), _f32(v2),
                                   ctypes.byref(t), ctypes.byref(f))
    return bool(hit), float(t.value), bool(f.value)


def texel_centre(bmin, extent, nf, j):
    o = np.empty(3, dtype=np.float32)
    _load().orc_texel_centre(_f32(bmin), extent, nf, int(j), o)
    return o


def trace(verts, tris, bmin, extent, nf, seed, frame, R, texels, nearest=False, accel="brute"):
    """One frame of Sec. 2.2 tracing for the given fine texels: (r_t fp32,
    #front, #back, triangle of r_t), plus with ``nearest`` the face of the
    nearest hit (1 = back; on equal distances a front hit wins).

    ``accel``: "brute" tests every ray against every triangle (the
    definition); "bvh" finds the same closest hits through a bounding-volume
    hierarchy that only skips triangles a ray cannot reach before its best
    hit (same fp32 test and tie rule; pinned bit for bit to "brute")."""
    if accel not in ("brute", "bvh"):
        raise ValueError(accel)
    v, t = _f32(verts), _i32(tris)
    tx = np.ascontiguousarray(texels, dtype=np.int64)
    m = tx.size
    r = np.empty(m, np.float32)
    nf_ = np.empty(m, np.int32)
    nb = np.empty(m, np.int32)
    bt = np.empty(m, np.int64)
    rb = np.empty(m, np.int32)
    fn = _load().orc_trace if accel == "brute" else _load().orc_trace_bvh
    fn(v.reshape(-1), t.reshape(-1), t.shape[0], _f32(bmin), extent, nf,
       int(seed) & (2 ** 64 - 1), frame, R, tx, m, r, nf_, nb, bt, rb)
    if nearest:
        return r, nf_, nb, bt, rb
    return r, nf_, nb, bt


def cast_rays(verts, tris, orig, dirs, accel="brute"):
    """Closest hit of arbitrary rays: (t fp32, +inf on a miss; front face;
    triangle index or -1).  ``accel`` as in :func:`trace`."""
    if accel not in ("brute", "bvh"):
        raise ValueError(accel)
    v, t = _f32(verts), _i32(tris)
    o, d = _f32(orig).reshape(-1, 3), _f32(dirs).reshape(-1, 3)
    n = o.shape[0]
    tout = np.empty(n, np.float32)
    fr = np.empty(n, np.int32)
    tri = np.empty(n, np.int64)
    fn = _load().orc_cast_rays if accel == "brute" else _load().orc_cast_rays_bvh
    fn(v.reshape(-1), t.reshape(-1), t.shape[0], o.reshape(-1), d.reshape(-1), n, tout, fr, tri)
    return tout, fr.astype(bool), tri


def point_mesh_distance(verts, tris, pts):
    p = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty(p.shape[0])
    t = _i32(tris)
    _load().orc_point_mesh_distance(_f32(verts).reshape(-1), t.reshape(-1), t.shape[0],
                                    p.reshape(-1), p.shape[0], out)
    return out


# ---------------------------------------------------------------------------
# Sec. 2.2 -- Eq. 1 accumulation, sign vote, region reset
# ---------------------------------------------------------------------------

def eq1_update(u_prev, c_t, r_t, alpha):
    """Eq. 1, first case, on the unsigned accumulator:
    u_t = min(alpha u_{t-1} + (1 - alpha) c_t, r_t)  (fp64).
    alpha = 1 keeps the plain minimum; alpha = 0 uses c_t (no 0*inf)."""
    u_prev = np.asarray(u_prev, dtype=np.float64)
    c_t = np.asarray(c_t, dtype=np.float64)
    r_t = np.asarray(r_t, dtype=np.float64)
    if alpha == 1.0:
        prev = u_prev
    elif alpha == 0.0:
        prev = c_t
    else:
        with np.errstate(invalid="ignore"):
            prev = np.where(np.isinf(u_prev), np.inf, alpha * u_prev + (1.0 - alpha) * c_t)
    return np.minimum(prev, r_t)


def signed_output(u, c_parent, nfront, nback):
    """Fine SDF value of a masked texel: the accumulated minimum (the coarse
    value while no ray has hit yet), negative when back-face hits outnumber
    front-face hits (Sec. 2.2, last paragraph)."""
    mag = np.where(np.isfinite(u), u, c_parent)
    return np.where(np.asarray(nback) > np.asarray(nfront), -mag, mag)


def reset_rule(centres, u_prev, aabb_lo, aabb_hi):
    """Reset in changed regions: a texel whose centre lies within its current
    accumulated distance of a moved object's previous bounding box restarts
    its accumulation.  fp32 (the decision precision):
    dx = max(max(lo - p, p - hi), 0) per axis, d2 = (dx*dx + dy*dy) + dz*dz,
    reset iff d2 <= u*u for some moved object."""
    p = np.asarray(centres, dtype=np.float32).reshape(-1, 3)
    u = np.asarray(u_prev, dtype=np.float32)
    uu = u * u
    out = np.zeros(p.shape[0], dtype=bool)
    lo = np.asarray(aabb_lo, dtype=np.float32).reshape(-1, 3)
    hi = np.asarray(aabb_hi, dtype=np.float32).reshape(-1, 3)
    zero = np.float32(0)
    for k in range(lo.shape[0]):
        d = [np.maximum(np.maximum(lo[k, a] - p[:, a], p[:, a] - hi[k, a]), zero) for a in range(3)]
        d2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
        out |= d2 <= uu
    return out


def texel_centres(bmin, extent, nf, texels):
    """fp32 centres of the given fine texels (same arithmetic as texel_centre)."""
    b = _f32(bmin)
    hf = np.float32(extent) / np.float32(nf)
    j = np.asarray(texels, dtype=np.int64)
    idx = np.stack([j % nf, (j // nf) % nf, j // (nf * nf)], axis=1).astype(np.float32)
    return b[None, :] + (idx + np.float32(0.5)) * hf


class FinePipeline:
    """Sec. 2.1 -> Sec. 2.2 over frames, for the whole fine grid or a subset
    of fine texels (state kept only for the tracked texels).

    Per frame: voxelize, jump flood, coarse SDF, mask; unmasked texels take
    c and restart their accumulator; masked tracked texels may be reset
    (moved objects), then are traced and updated by Eq. 1."""

    def __init__(self, bmin, extent, nc, beta_vox, d_vox, alpha, seed, track=None, sign="vote", accel="brute"):
        """sign: "vote" (Sec. 2.2: negative when back-face hits outnumber
        front-face hits, counts kept over frames) or "nearest" (the variant
        that keeps the face of the nearest hit found so far; on equal
        distances a front hit wins).  accel: how :func:`trace` finds the
        closest hits ("brute" or "bvh", same results)."""
        if sign not in ("vote", "nearest"):
            raise ValueError(sign)
        if accel not in ("brute", "bvh"):
            raise ValueError(accel)
        self.accel = accel
        self.bmin = np.asarray(bmin, np.float32)
        self.extent = float(extent)
        self.nc, self.nf = nc, 2 * nc
        self.beta, self.d, self.alpha, self.seed = beta_vox, d_vox, alpha, seed
        self.sign = sign
        self.track = None if track is None else np.asarray(track, np.int64)
        m = self.nf ** 3 if track is None else self.track.size
        self.u = np.full(m, np.inf)
        self.nF = np.zeros(m, np.int64)
        self.nB = np.zeros(m, np.int64)
        self.back = np.zeros(m, np.int64)   # "nearest": face of the accumulated minimum
        self.f = np.zeros(m)

    def texels(self):
        return np.arange(self.nf ** 3, dtype=np.int64) if self.track is None else self.track

    def frame(self, verts, tris, frame, R, moved_aabbs=None):
        occ = voxelize(verts, tris, self.bmin, self.extent, self.nc)
        seeds, _ = jfa(occ, self.nc)
        c = coarse_sdf(seeds, self.nc, self.extent, self.beta)
        mask, fun = mask_fill(seeds, self.nc, self.d, self.beta, c)
        tx = self.texels()
        cpar = c[parent_index(self.nc)][tx]
        m = mask[tx]
        # unmasked: f = c, accumulator restarts
        self.u[~m] = np.inf
        self.nF[~m] = 0
        self.nB[~m] = 0
        self.back[~m] = 0
        self.f[~m] = fun[tx][~m]
        sel = np.nonzero(m)[0]
        if moved_aabbs is not None and sel.size:
            lo, hi = moved_aabbs
            rs = reset_rule(texel_centres(self.bmin, self.extent, self.nf, tx[sel]),
                            self.u[sel], lo, hi)
            self.u[sel[rs]] = np.inf
            self.nF[sel[rs]] = 0
            self.nB[sel[rs]] = 0
            self.back[sel[rs]] = 0
        if sel.size:
            r, cf, cb, _, rb = trace(verts, tris, self.bmin, self.extent, self.nf, self.seed, frame, R, tx[sel],
                                     nearest=True, accel=self.accel)
            if self.sign == "vote":
                self.u[sel] = eq1_update(self.u[sel], cpar[sel], r, self.alpha)
                self.nF[sel] += cf
                self.nB[sel] += cb
                self.f[sel] = signed_output(self.u[sel], cpar[sel], self.nF[sel], self.nB[sel])
            else:
                # Eq. 1's minimum, keeping the face of whichever term is smaller
                # (the decayed previous value or this frame's nearest hit)
                prev = eq1_update(self.u[sel], cpar[sel], np.full(sel.size, np.inf), self.alpha)
                r64 = r.astype(np.float64)
                bp = self.back[sel]
                back = np.where(r64 < prev, rb, np.where(prev < r64, bp, np.minimum(bp, rb)))
                u = np.minimum(prev, r64)
                self.u[sel] = u
                self.back[sel] = np.where(np.isfinite(u), back, 0)
                mag = np.where(np.isfinite(u), u, cpar[sel])
                self.f[sel] = np.where(self.back[sel] == 1, -mag, mag)
        return dict(occ=occ, seeds=seeds, c=c, mask=mask)


# ---------------------------------------------------------------------------
# Sec. 2.3 -- soft shadows and their derivative
# ---------------------------------------------------------------------------

def shadow(sdf, n, bmin, extent, pos, nrm, light_v, k, steps, step_max, eps, info=False, shift=None):
    """Visibility per shading point (fp64).  ``sdf`` float32 [n^3].  ``shift``
    (fp64 [npix], world units, optional) moves each ray origin toward the
    light: the jitter of Sec. 2.3."""
    s = _f32(sdf).reshape(-1)
    p, q = _f32(pos).reshape(-1, 3), _f32(nrm).reshape(-1, 3)
    npix = p.shape[0]
    vis = np.empty(npix)
    inf = np.empty(3 * npix, np.int32) if info else None
    sh = None if shift is None else np.ascontiguousarray(shift, np.float64).reshape(-1)
    if sh is not None and sh.size != npix:
        raise ValueError("shift needs one value per shading point")
    _load().orc_shadow(s, n, np.asarray(bmin, np.float64), float(extent), p.reshape(-1), q.reshape(-1),
                       npix, np.asarray(light_v, np.float64), float(k), int(steps), float(step_max),
                       float(eps), vis, inf.ctypes.data if info else None,
                       sh.ctypes.data if sh is not None else None)
    if info:
        return vis, inf.reshape(-1, 3)
    return vis


def shadow_margin(sdf, n, bmin, extent, pos, nrm, light_v, k, steps, step_max, eps):
    """Per shading point, the smallest relative gap over its march between
    the two sides of any discrete decision (inside the volume, h < eps,
    t - y > 0, a new minimum of the penumbra estimate, h < step_max, the
    root's argument > 0), fp64.  A march with a margin well above the
    rounding of another precision takes the same discrete path there."""
    s = _f32(sdf).reshape(-1)
    p, q = _f32(pos).reshape(-1, 3), _f32(nrm).reshape(-1, 3)
    out = np.empty(p.shape[0])
    _load().orc_shadow_margin(s, n, np.asarray(bmin, np.float64), float(extent), p.reshape(-1), q.reshape(-1),
                              p.shape[0], np.asarray(light_v, np.float64), float(k), int(steps), float(step_max),
                              float(eps), out)
    return out


def unit_light(light_v):
    """The fp32 unit light direction: normalised in fp64 ((x^2 + y^2) + z^2,
    then each component divided by the root), rounded to fp32."""
    x, y, z = (float(np.float32(c)) for c in light_v)
    nv = math.sqrt(x * x + y * y + z * z)
    return np.array([x / nv, y / nv, z / nv], np.float32)


def shadow_exact(verts, tris, pos, nrm, light_v, eps):
    """Thin-surface fallback (Sec. 3: the march steps through surfaces
    thinner than its epsilon and leaves holes in the umbra; the paper would
    shadow-map those regions), read as an exact occlusion test toward the
    light.  blocked[i] is True iff some triangle meets the ray from the
    march's origin fmaf(nrm, 2 eps, pos) (fp32, one rounding) along the
    fp32 unit light direction, by the tracer's fp32 ray/triangle test.
    ``eps``: the march epsilon in world units (fp32)."""
    v, t = _f32(verts), _i32(tris)
    p, q = _f32(pos).reshape(-1, 3), _f32(nrm).reshape(-1, 3)
    out = np.empty(p.shape[0], np.int32)
    two_eps = float(np.float32(2.0) * np.float32(eps))
    _load().orc_shadow_exact(v.reshape(-1), t.reshape(-1), t.shape[0], p.reshape(-1), q.reshape(-1),
                             p.shape[0], unit_light(light_v), two_eps, out)
    return out.astype(bool)


def shadow_fallback(vis, blocked):
    """Visibility after the thin-surface fallback: 0 where the exact test
    is blocked, the march's value elsewhere (min(vis, 1 - blocked))."""
    return np.where(np.asarray(blocked, bool), 0.0, np.asarray(vis, np.float64))


def shadow_jitter(seed, frame, npix):
    """Per-pixel jitter fractions xi in [0, 1) of one frame (Sec. 2.3: the
    shadow ray origin is jittered toward the light): Philox-4x32-10 with
    counter (pixel lo, pixel hi, frame, 0x53484457) and key (seed lo, seed
    hi), top 24 bits of the first output word times 2^-24."""
    xi = np.empty(int(npix))
    _load().orc_shadow_jitter(int(seed) & (2 ** 64 - 1), int(frame) & 0xFFFFFFFF, int(npix), xi)
    return xi


def taa_resolve(cur, hist, blend):
    """Temporal anti-aliasing of a visibility image (Sec. 2.3 stabilises the
    jitter noise with TAA), static camera: the history is clamped to the
    min / max of the current frame's 3x3 neighbourhood (clamped at the image
    border) and blended toward the current value, out = h + blend (cur - h).
    ``cur``, ``hist``: [H, W]; fp64 result."""
    c = np.asarray(cur, np.float64)
    h = np.asarray(hist, np.float64)
    H, W = c.shape
    pad = np.pad(c, 1, mode="edge")
    win = np.stack([pad[dy:dy + H, dx:dx + W] for dy in range(3) for dx in range(3)])
    hc = np.clip(h, win.min(axis=0), win.max(axis=0))
    return hc + float(blend) * (c - hc)


def shadow_grad(sdf, n, bmin, extent, pos, nrm, light_v, k, steps, step_max, eps, dvis):
    """Reverse-mode derivative: (dLoss/dsdf fp64 [n^3], dLoss/dlight_v fp64 [3])."""
    s = _f32(sdf).reshape(-1)
    p, q = _f32(pos).reshape(-1, 3), _f32(nrm).reshape(-1, 3)
    npix = p.shape[0]
    g = np.zeros(n ** 3)
    gl = np.zeros(3)
    _load().orc_shadow_grad(s, n, np.asarray(bmin, np.float64), float(extent), p.reshape(-1),
                            q.reshape(-1), npix, np.asarray(light_v, np.float64), float(k), int(steps),
                            float(step_max), float(eps),
                            np.ascontiguousarray(dvis, np.float64).reshape(-1), g, gl)
    return g, gl


def sample(sdf, n, bmin, extent, q):
    return float(_load().orc_sample(_f32(sdf).reshape(-1), n, np.asarray(bmin, np.float64), float(extent),
                                    np.asarray(q, np.float64)))
