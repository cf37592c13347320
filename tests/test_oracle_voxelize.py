"""Pins for the oracle's conservative voxelization (Sec. 2.1).

The oracle's int64 separating-axis test is checked against an independent
exact method (Sutherland-Hodgman clipping of the quantised triangle by the
six closed slabs of the voxel, in rational arithmetic), against the
analytic voxel set of an axis-aligned box, and against geometric facts
(every point of a triangle lies in an occupied voxel; an occupied voxel's
centre is within half a voxel diagonal of the mesh).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth import scenes as S

BMIN = np.zeros(3, np.float32)


def _clip_nonempty(tri_q, x, y, z, sub=256):
    """Closed triangle meets closed cube [x,x+1]x[y,y+1]x[z,z+1] (voxel
    units, vertices in 1/sub units) -- exact polygon clipping."""
    poly = [tuple(Fraction(int(c)) for c in v) for v in tri_q]
    lo = (x * sub, y * sub, z * sub)
    for axis in range(3):
        for side in (0, 1):
            bound = Fraction(lo[axis] + side * sub)

            def inside(p):
                return p[axis] >= bound if side == 0 else p[axis] <= bound

            out = []
            m = len(poly)
            for i in range(m):
                a, b = poly[i], poly[(i + 1) % m]
                ia, ib = inside(a), inside(b)
                if ia:
                    out.append(a)
                if ia != ib:
                    t = (bound - a[axis]) / (b[axis] - a[axis])
                    out.append(tuple(a[k] + t * (b[k] - a[k]) for k in range(3)))
            poly = out
            if not poly:
                return False
    return True


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_overlap_matches_exact_clipping(seed):
    n = 6
    rng = np.random.default_rng(seed)
    checked = hits = 0
    for _ in range(60):
        c = rng.uniform(0.1, 0.9, 3)
        size = rng.choice([0.02, 0.1, 0.3])
        v = (c + rng.uniform(-size, size, (3, 3))).astype(np.float32)
        if rng.uniform() < 0.2:     # degenerate: collinear or repeated vertices
            v[2] = v[0] + (v[1] - v[0]) * np.float32(rng.choice([0.0, 0.5, 1.0]))
        q = oracle.quantise_vertices(v, BMIN, 1.0, n)
        lo = np.maximum(q.min(0) // 256 - 1, 0)
        hi = np.minimum(q.max(0) // 256 + 1, n - 1)
        for zz in range(lo[2], hi[2] + 1):
            for yy in range(lo[1], hi[1] + 1):
                for xx in range(lo[0], hi[0] + 1):
                    a = oracle.tri_voxel_overlap(q, xx, yy, zz)
                    b = _clip_nonempty(q, xx, yy, zz)
                    assert a == b, (v, xx, yy, zz)
                    checked += 1
                    hits += a
    assert checked > 500 and 0 < hits < checked


def test_touching_faces_count():
    # Triangle lying exactly in the plane x = 2 voxels touches voxels 1 and 2.
    n = 8
    h = 1.0 / n
    v = np.array([[2 * h, 3.1 * h, 3.1 * h], [2 * h, 3.6 * h, 3.2 * h], [2 * h, 3.3 * h, 3.7 * h]], np.float32)
    occ = oracle.voxelize(v, np.array([[0, 1, 2]]), BMIN, 1.0, n).reshape(n, n, n)
    xs = sorted(set(np.nonzero(occ >= 0)[2].tolist()))
    assert xs == [1, 2]


def test_axis_aligned_box_exact_set():
    # Box [0.1, 0.5]^3 at n = 32: faces at 3.2 and 16 voxels.  Closed sets:
    # voxel i is occupied iff [i, i+1] meets the surface of the box.
    n = 32
    m = S.merge([S.box_mesh((0.3, 0.3, 0.3), 0.2)])
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, n).reshape(n, n, n) >= 0
    lo = 819 / 256.0   # 0.1 * 8192 rounded to a 1/256 step
    hi = 16.0
    i = np.arange(n)
    inside_span = (i + 1 >= lo) & (i <= hi)            # [i, i+1] meets [lo, hi]
    touches_lo = (i <= lo) & (i + 1 >= lo)
    touches_hi = (i <= hi) & (i + 1 >= hi)
    face = touches_lo | touches_hi
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    # z-major storage: occ[z, y, x]
    span = inside_span[X] & inside_span[Y] & inside_span[Z]
    on_face = face[X] | face[Y] | face[Z]
    expect = (span & on_face).transpose(2, 1, 0)
    assert np.array_equal(occ, expect)


@pytest.mark.parametrize("n", [16, 32])
def test_conservative_and_tight_tiny_scene(n):
    m = S.tiny_scene()
    h = 1.0 / n
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, n)
    # (1) every vertex and random surface points lie in an occupied voxel
    rng = np.random.default_rng(5)
    tri = m.verts[m.tris].astype(np.float64)
    w = rng.dirichlet([1, 1, 1], size=(tri.shape[0], 20))
    pts = np.einsum("tsk,tkd->tsd", w, tri).reshape(-1, 3)
    pts = np.concatenate([pts, m.verts.astype(np.float64)])
    g = np.floor(pts / h).astype(np.int64)
    interior = np.all((np.abs(pts / h - np.round(pts / h)) > 3e-3), axis=1)
    g = g[interior]
    lin = g[:, 0] + n * (g[:, 1] + n * g[:, 2])
    assert np.all(occ[lin] >= 0)
    # (2) every occupied voxel centre is within h*sqrt(3)/2 (+ quantisation) of the mesh
    j = np.nonzero(occ >= 0)[0]
    cen = np.stack([j % n, (j // n) % n, j // (n * n)], 1) * h + h / 2
    d = oracle.point_mesh_distance(m.verts, m.tris, cen)
    assert np.all(d <= h * np.sqrt(3) / 2 + h * np.sqrt(3) / 512 + 1e-7)


def test_soup_tight_against_distance():
    n = 24
    h = 1.0 / n
    m = S.random_soup(7, 40, size=0.1)
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, n)
    j = np.nonzero(occ >= 0)[0]
    cen = np.stack([j % n, (j // n) % n, j // (n * n)], 1) * h + h / 2
    d = oracle.point_mesh_distance(m.verts, m.tris, cen)
    assert np.all(d <= h * np.sqrt(3) / 2 + h * np.sqrt(3) / 512 + 1e-7)


def test_bad_inputs():
    v = np.array([[0.1, 0.1, 0.1], [0.2, 0.1, 0.1], [0.1, 0.2, np.nan]], np.float32)
    with pytest.raises(oracle.OracleError):
        oracle.voxelize(v, np.array([[0, 1, 2]]), BMIN, 1.0, 8)
    v[2, 2] = 0.1
    with pytest.raises(oracle.OracleError):
        oracle.voxelize(v, np.array([[0, 1, 3]]), BMIN, 1.0, 8)
    v[2, 2] = 5.0     # beyond bmin + 3/2 extent
    with pytest.raises(oracle.OracleError):
        oracle.voxelize(v, np.array([[0, 1, 2]]), BMIN, 1.0, 8)
    # empty mesh: nothing occupied
    occ = oracle.voxelize(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32), BMIN, 1.0, 4)
    assert np.all(occ == -1)
