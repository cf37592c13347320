"""Seeded synthetic scenes, shading points and motion for the RTSDF pipeline.

This module only *creates inputs*: triangle meshes, rigid per-object
translations and G-buffer style shading points.  It holds none of the SDF
method's arithmetic (no voxelization, jump flooding, ray generation, tracing
or marching), so both the CPU oracle and the CUDA path can be fed from it.

The paper measures on "The Modern Living Room" (teaser caption), a scene that
is not available here; procedural rooms and object clouds with the same
character (a floor and walls plus many closed objects of mixed size) stand in
for it.  Every generator is deterministic in its ``seed``.

Conventions
-----------
* vertices: float32 [V, 3]; triangles: int32 [T, 3].
* every closed object is wound counter-clockwise seen from outside (outward
  normals ``(v1 - v0) x (v2 - v0)``); room quads face the room interior.
* scene bounds are the unit cube ``[0, 1]^3`` unless stated otherwise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "box_mesh", "icosphere_mesh", "uv_sphere_mesh", "room_quads",
    "random_rotation", "merge", "tiny_scene", "room_scene", "animated_scene",
    "batch_scenes", "floor_gbuffer", "object_translations", "random_soup",
    "sphere_grid_sdf", "box_grid_sdf",
]


@dataclass
class Mesh:
    verts: np.ndarray            # float32 [V, 3]
    tris: np.ndarray             # int32 [T, 3]
    vert_object: np.ndarray = field(default=None)   # int32 [V], object id per vertex
    n_objects: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def nt(self) -> int:
        return int(self.tris.shape[0])


# --------------------------------------------------------------------------
# primitive meshes (float64 internally, cast at the end)
# --------------------------------------------------------------------------

def _box_unit():
    v = np.array([[x, y, z] for z in (-1, 1) for y in (-1, 1) for x in (-1, 1)],
                 dtype=np.float64)
    # vertex id = x + 2y + 4z with x,y,z in {0,1}; faces wound outward
    quads = [
        (0, 2, 3, 1),  # z = -1, normal -z
        (4, 5, 7, 6),  # z = +1
        (0, 1, 5, 4),  # y = -1
        (2, 6, 7, 3),  # y = +1
        (0, 4, 6, 2),  # x = -1
        (1, 3, 7, 5),  # x = +1
    ]
    t = []
    for a, b, c, d in quads:
        t.append((a, b, c))
        t.append((a, c, d))
    return v, np.array(t, dtype=np.int64)


def _icosphere_unit(subdiv: int):
    p = (1.0 + 5 ** 0.5) / 2.0
    v = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    v = [np.array(x, dtype=np.float64) / np.linalg.norm(x) for x in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = nf
    v = np.array(v)
    f = np.array(f, dtype=np.int64)
    # make the winding outward
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", n, v[f].mean(axis=1)) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def _uv_sphere_unit(n_lon: int, n_lat: int):
    """Unit UV sphere with ``n_lat`` latitude bands: 2*n_lon*(n_lat-1) tris."""
    verts = [(0.0, 0.0, 1.0)]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2 * math.pi * j / n_lon
            verts.append((math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)))
    verts.append((0.0, 0.0, -1.0))
    v = np.array(verts)
    south = len(verts) - 1

    def ring(i, j):
        return 1 + (i - 1) * n_lon + (j % n_lon)

    f = []
    for j in range(n_lon):
        f.append((0, ring(1, j), ring(1, j + 1)))
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            a, b = ring(i, j), ring(i, j + 1)
            c, d = ring(i + 1, j), ring(i + 1, j + 1)
            f.append((a, c, d))
            f.append((a, d, b))
    for j in range(n_lon):
        f.append((south, ring(n_lat - 1, j + 1), ring(n_lat - 1, j)))
    f = np.array(f, dtype=np.int64)
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", n, v[f].mean(axis=1)) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation matrix (normalised quaternion of 4 normals)."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _place(v, f, center, scale, rot=None):
    v = v * scale
    if rot is not None:
        v = v @ rot.T
    return v + np.asarray(center, dtype=np.float64), f


def box_mesh(center, half, rot=None):
    v, f = _box_unit()
    return _place(v, f, center, np.asarray(half, dtype=np.float64), rot)


def icosphere_mesh(subdiv, center, r, rot=None):
    v, f = _icosphere_unit(subdiv)
    return _place(v, f, center, r, rot)


def _hash_u32(x):
    """Integer mixer (an avalanche hash) over uint64 arrays -> uint32."""
    x = (x ^ (x >> np.uint64(33))) * np.uint64(0xFF51AFD7ED558CCD)
    x = (x ^ (x >> np.uint64(33))) * np.uint64(0xC4CEB9FE1A85EC53)
    x = x ^ (x >> np.uint64(33))
    return (x & np.uint64(0xFFFFFFFF)).astype(np.uint64)


def _gradient_noise(p, seed):
    """3D gradient noise in [-1, 1]-ish with hashed lattice gradients.

    The lattice gradient at integer point g is a hashed unit vector; the
    value is the quintic-faded trilinear blend of g_i . (p - g_i).
    """
    p = np.asarray(p, dtype=np.float64)
    g0 = np.floor(p).astype(np.int64)
    fr = p - g0
    fade = fr * fr * fr * (fr * (fr * 6 - 15) + 10)
    out = np.zeros(p.shape[0])
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                g = g0 + np.array([dx, dy, dz])
                key = ((g[:, 0] & 0x1FFFFF) | ((g[:, 1] & 0x1FFFFF) << 21)
                       | ((g[:, 2] & 0x1FFFFF) << 42)).astype(np.uint64)
                key = key ^ np.uint64(seed * 0x9E3779B97F4A7C15 & 0xFFFFFFFFFFFFFFFF)
                h1 = _hash_u32(key)
                h2 = _hash_u32(key ^ np.uint64(0x5851F42D4C957F2D))
                z = h1.astype(np.float64) / 2 ** 31 - 1.0
                phi = h2.astype(np.float64) / 2 ** 32 * 2 * math.pi
                rr = np.sqrt(np.maximum(0.0, 1 - z * z))
                grad = np.stack([rr * np.cos(phi), rr * np.sin(phi), z], axis=1)
                d = fr - np.array([dx, dy, dz])
                w = ((fade[:, 0] if dx else 1 - fade[:, 0])
                     * (fade[:, 1] if dy else 1 - fade[:, 1])
                     * (fade[:, 2] if dz else 1 - fade[:, 2]))
                out += w * np.einsum("ij,ij->i", grad, d)
    return out


def uv_sphere_mesh(center, r, n_lon=50, n_lat=21, displace=0.0, noise_freq=4.0,
                   noise_seed=0, rot=None):
    v, f = _uv_sphere_unit(n_lon, n_lat)
    if displace:
        nz = _gradient_noise(v * noise_freq, noise_seed)
        v = v * (1.0 + displace * nz)[:, None]
    return _place(v, f, center, r, rot)


def room_quads(lo=0.02, hi=0.98):
    """Floor y=lo and walls x=lo, x=hi, z=lo as 2 tris each, facing inward."""
    quads = [
        # floor (normal +y)
        [(0, lo, 0), (0, lo, 1), (1, lo, 1), (1, lo, 0)],
        # wall x = lo (normal +x)
        [(lo, 0, 0), (lo, 1, 0), (lo, 1, 1), (lo, 0, 1)],
        # wall x = hi (normal -x)
        [(hi, 0, 0), (hi, 0, 1), (hi, 1, 1), (hi, 1, 0)],
        # wall z = lo (normal +z)
        [(0, 0, lo), (1, 0, lo), (1, 1, lo), (0, 1, lo)],
    ]
    v, f = [], []
    for q in quads:
        b = len(v)
        v += q
        f += [(b, b + 1, b + 2), (b, b + 2, b + 3)]
    return np.array(v, dtype=np.float64), np.array(f, dtype=np.int64)


def merge(parts, meta=None) -> Mesh:
    """Concatenate (verts, tris) parts; each part becomes one object."""
    vs, fs, objs = [], [], []
    base = 0
    for k, (v, f) in enumerate(parts):
        vs.append(v)
        fs.append(f + base)
        objs.append(np.full(len(v), k, dtype=np.int32))
        base += len(v)
    verts = np.concatenate(vs).astype(np.float32)
    tris = np.concatenate(fs).astype(np.int32)
    return Mesh(verts, tris, np.concatenate(objs), len(parts), dict(meta or {}))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def tiny_scene() -> Mesh:
    """Axis-aligned box (half 0.2 at 0.3) + icosphere (subdiv 2, r 0.15)."""
    parts = [box_mesh((0.3, 0.3, 0.3), 0.2),
             icosphere_mesh(2, (0.7, 0.6, 0.65), 0.15)]
    return merge(parts, dict(name="tiny", box=((0.3, 0.3, 0.3), 0.2),
                             sphere=((0.7, 0.6, 0.65), 0.15)))


def room_scene(seed: int = 1, n_objects: int = 200, n_spheres: int = 78,
               subdiv: int = 3) -> Mesh:
    """Room (floor + 3 walls) and ``n_objects`` boxes/icospheres."""
    rng = np.random.default_rng(seed)
    parts = [room_quads()]
    kinds = np.array([1] * n_spheres + [0] * (n_objects - n_spheres))
    rng.shuffle(kinds)
    for kind in kinds:
        c = rng.uniform(0.1, 0.9, 3)
        s = math.exp(rng.uniform(math.log(0.02), math.log(0.1)))
        rot = random_rotation(rng)
        if kind:
            parts.append(icosphere_mesh(subdiv, c, s, rot))
        else:
            parts.append(box_mesh(c, s, rot))
    return merge(parts, dict(name="room", seed=seed))


def animated_scene(seed: int = 2, n_objects: int = 500, n_lon: int = 50,
                   n_lat: int = 21) -> Mesh:
    """``n_objects`` displaced UV spheres (2*n_lon*(n_lat-1) tris each)."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(n_objects):
        c = rng.uniform(0.1, 0.9, 3)
        r = math.exp(rng.uniform(math.log(0.02), math.log(0.05)))
        parts.append(uv_sphere_mesh(c, r, n_lon, n_lat, displace=0.1,
                                    noise_seed=seed * 100003 + i,
                                    rot=random_rotation(rng)))
    return merge(parts, dict(name="animated", seed=seed))


def object_translations(seed: int, frame: int, n_objects: int, max_len: float):
    """Per-object translation for one frame: uniform in a ball of radius max_len."""
    rng = np.random.default_rng([seed, frame, 0x7A11])
    d = rng.standard_normal((n_objects, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = max_len * rng.uniform(0.0, 1.0, n_objects) ** (1.0 / 3.0)
    return (d * rad[:, None]).astype(np.float32)


def batch_scenes(seed: int = 3, count: int = 64, sizes=(32, 48, 64, 80, 96, 112, 128),
                 tri_median: float = 14000.0, tri_sigma: float = 1.2,
                 tri_clip=(1000, 200000)):
    """``count`` scenes of uneven grid size and triangle budget."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        n = int(rng.choice(sizes))
        t = float(np.clip(math.exp(math.log(tri_median) + tri_sigma * rng.standard_normal()),
                          *tri_clip))
        n_obj = int(math.ceil(t / 166.0))
        parts = []
        for _ in range(n_obj):
            c = rng.uniform(0.1, 0.9, 3)
            s = math.exp(rng.uniform(math.log(0.02), math.log(0.1)))
            rot = random_rotation(rng)
            if rng.uniform() < 0.5:
                parts.append(box_mesh(c, s, rot))
            else:
                parts.append(icosphere_mesh(2, c, s, rot))
        m = merge(parts, dict(name=f"batch{i}", seed=seed + i, coarse_n=n))
        out.append(m)
    return out


def random_soup(seed: int, n_tris: int, lo=0.05, hi=0.95, size=0.08) -> Mesh:
    """Random independent triangles (for property tests)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(lo, hi, (n_tris, 1, 3))
    v = c + rng.uniform(-size, size, (n_tris, 3, 3))
    verts = v.reshape(-1, 3).astype(np.float32)
    tris = np.arange(3 * n_tris, dtype=np.int32).reshape(-1, 3)
    return Mesh(verts, tris, np.arange(n_tris, dtype=np.int32).repeat(3), n_tris,
                dict(name="soup", seed=seed))


def floor_gbuffer(w: int, h: int, y: float = 0.02, lo: float = 0.0, hi: float = 1.0):
    """Orthographic top-down G-buffer of the floor plane y = ``y``.

    Returns positions and normals as float32 [h, w, 3] (pixel centres over
    the square [lo, hi]^2 in x and z; normal +y).
    """
    xs = lo + (np.arange(w) + 0.5) * (hi - lo) / w
    zs = lo + (np.arange(h) + 0.5) * (hi - lo) / h
    X, Z = np.meshgrid(xs, zs)
    pos = np.stack([X, np.full_like(X, y), Z], axis=-1).astype(np.float32)
    nrm = np.zeros_like(pos)
    nrm[..., 1] = 1.0
    return pos, nrm


def sphere_grid_sdf(n: int, center, r, bmin=(0.0, 0.0, 0.0), extent=1.0, floor_y=None):
    """Analytic sphere (and optional floor half-space) SDF sampled at cell centres.

    float32 [n, n, n] indexed [z, y, x].  Used as a synthetic fine grid for
    the shadow pass.
    """
    b = np.asarray(bmin, dtype=np.float64)
    c = (np.arange(n) + 0.5) * extent / n
    Z, Y, X = np.meshgrid(b[2] + c, b[1] + c, b[0] + c, indexing="ij")
    d = np.sqrt((X - center[0]) ** 2 + (Y - center[1]) ** 2 + (Z - center[2]) ** 2) - r
    if floor_y is not None:
        d = np.minimum(d, Y - floor_y)
    return d.astype(np.float32)


def box_grid_sdf(n: int, center, half, bmin=(0.0, 0.0, 0.0), extent=1.0, floor_y=None):
    """Analytic axis-aligned box SDF sampled at cell centres, float32 [z, y, x]."""
    b = np.asarray(bmin, dtype=np.float64)
    c = (np.arange(n) + 0.5) * extent / n
    Z, Y, X = np.meshgrid(b[2] + c, b[1] + c, b[0] + c, indexing="ij")
    q = np.stack([np.abs(X - center[0]), np.abs(Y - center[1]), np.abs(Z - center[2])], -1) - half
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(q.max(axis=-1), 0.0)
    d = outside + inside
    if floor_y is not None:
        d = np.minimum(d, Y - floor_y)
    return d.astype(np.float32)
