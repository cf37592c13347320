"""Pins for the oracle's ray generation and ray casting (Sec. 2.2).

* Philox: both widths reproduce the published known-answer vectors of
  Salmon et al. (SC'11) stored in ``tests/golden/philox_kat.txt``; the
  shared round structure is also checked bit-for-bit against numpy's
  independent Philox-4x64-10, and the 4x32 outputs for uniformity and
  avalanche.
* Directions: unit length, uniform on the sphere (moments; Archimedes: the
  z component is uniform on [-1, 1]).
* Ray/triangle: hand-derived hits, and agreement with an fp64 ray-plane +
  barycentric computation on random cases.
* Closest hit + minimum over rays: the distribution law of the minimum over
  R uniform rays above a plane, P(min <= d0/u) = 1 - ((1+u)/2)^R; the
  front/back convention; and "traced minimum >= exact distance".
"""
import math
import os

import numpy as np
import pytest

import oracle
from synth import scenes as S

BMIN = np.zeros(3, np.float32)


def _kat_vectors():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")
    out = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, rounds, *words = line.split()
            w = [int(x, 16) for x in words]
            out.append((name, int(rounds), w[0:4], w[4:6], w[6:10]))
    return out


def test_philox_known_answer_vectors():
    """Random123's published Philox-4x32-10 and 4x64-10 vectors: a wrong
    multiplier, Weyl constant, word permutation or round count fails."""
    kat = _kat_vectors()
    assert sum(1 for k in kat if k[0] == "philox4x32") == 3
    assert sum(1 for k in kat if k[0] == "philox4x64") == 3
    for name, rounds, ctr, key, expect in kat:
        assert rounds == 10
        if name == "philox4x32":
            got = oracle.philox4x32(np.array(ctr, np.uint32), np.array(key, np.uint32))
        else:
            got = oracle.philox4x64(np.array(ctr, np.uint64), np.array(key, np.uint64))
        assert [int(x) for x in got] == expect, (name, ctr, key)


def test_philox_structure_matches_numpy_4x64():
    rng = np.random.default_rng(0)
    for _ in range(20):
        ctr = rng.integers(0, 2 ** 63, 4, dtype=np.uint64)
        key = rng.integers(0, 2 ** 63, 2, dtype=np.uint64)
        bg = np.random.Philox(counter=ctr, key=key)
        ref = bg.random_raw(4).astype(np.uint64)
        # numpy increments the counter before each block
        c1 = ctr.copy()
        c1[0] += np.uint64(1)
        assert np.array_equal(oracle.philox4x64(c1, key), ref)


def test_philox4x32_statistics():
    outs = np.array([oracle.philox4x32([i, 7, 0, 0], [1234, 5678]) for i in range(20000)])
    bits = np.unpackbits(outs.view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.002
    by = outs.view(np.uint8).ravel()
    hist = np.bincount(by, minlength=256)
    exp = by.size / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 5 * math.sqrt(2 * 255)
    # avalanche: flipping one counter bit flips ~half the output bits
    flips = []
    for b in range(32):
        a = oracle.philox4x32([5, 6, 7, 8], [9, 10])
        c = oracle.philox4x32([5 ^ (1 << b), 6, 7, 8], [9, 10])
        flips.append(np.unpackbits((a ^ c).view(np.uint8)).sum())
    assert 50 < np.mean(flips) < 78
    # key sensitivity
    assert not np.array_equal(oracle.philox4x32([1, 2, 3, 4], [0, 0]), oracle.philox4x32([1, 2, 3, 4], [0, 1]))


def _dirs(n, seed=11):
    return np.array([oracle.sphere_dir(seed, i // 64, 3, i % 64)[0] for i in range(n)], np.float64)


def test_directions_uniform_on_sphere():
    n = 60000
    d = _dirs(n)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-6)
    sig = 1 / math.sqrt(3 * n)
    assert np.all(np.abs(d.mean(0)) < 5 * sig)
    cov = d.T @ d / n
    assert np.allclose(cov, np.eye(3) / 3, atol=6 / math.sqrt(n))
    # Archimedes: each coordinate is uniform on [-1, 1]; KS test on z and x
    for k in (0, 2):
        z = np.sort(d[:, k])
        ecdf = np.arange(1, n + 1) / n
        ks = np.max(np.abs(ecdf - (z + 1) / 2))
        assert ks < 1.8 / math.sqrt(n)


def test_direction_is_a_function_of_its_counter():
    a, _ = oracle.sphere_dir(5, 100, 2, 7)
    b, _ = oracle.sphere_dir(5, 100, 2, 7)
    assert np.array_equal(a, b)
    others = [oracle.sphere_dir(5, 101, 2, 7)[0], oracle.sphere_dir(5, 100, 3, 7)[0],
              oracle.sphere_dir(5, 100, 2, 8)[0], oracle.sphere_dir(6, 100, 2, 7)[0]]
    for o in others:
        assert not np.array_equal(a, o)


def test_ray_triangle_closed_forms():
    v0, v1, v2 = [0, 0, 0], [1, 0, 0], [0, 1, 0]      # normal +z
    hit, t, front = oracle.ray_triangle([0.25, 0.25, 1], [0, 0, -1], v0, v1, v2)
    assert hit and t == 1.0 and front
    hit, t, front = oracle.ray_triangle([0.25, 0.25, -2], [0, 0, 1], v0, v1, v2)
    assert hit and t == 2.0 and not front
    # vertex and edge are part of the closed triangle
    assert oracle.ray_triangle([0, 0, 1], [0, 0, -1], v0, v1, v2)[0]
    assert oracle.ray_triangle([0.5, 0.5, 1], [0, 0, -1], v0, v1, v2)[0]
    # outside, parallel, behind
    assert not oracle.ray_triangle([0.75, 0.75, 1], [0, 0, -1], v0, v1, v2)[0]
    assert not oracle.ray_triangle([0.25, 0.25, 1], [1, 0, 0], v0, v1, v2)[0]
    assert not oracle.ray_triangle([0.25, 0.25, 1], [0, 0, 1], v0, v1, v2)[0]
    # origin on the surface: t = 0 counts
    hit, t, _ = oracle.ray_triangle([0.25, 0.25, 0], [0, 0, 1], v0, v1, v2)
    assert hit and t == 0.0


def test_ray_triangle_matches_fp64_plane_intersection():
    rng = np.random.default_rng(3)
    agree = 0
    for _ in range(4000):
        tri = rng.uniform(-1, 1, (3, 3)).astype(np.float32)
        o = rng.uniform(-2, 2, 3).astype(np.float32)
        target = (tri.T @ rng.dirichlet([1, 1, 1]) + rng.normal(0, 0.3, 3))
        d = (target - o)
        d = (d / np.linalg.norm(d)).astype(np.float32)
        hit, t, front = oracle.ray_triangle(o, d, *tri)
        a, b, c = tri.astype(np.float64)
        n = np.cross(b - a, c - a)
        dd, oo = d.astype(np.float64), o.astype(np.float64)
        den = n @ dd
        if abs(den) < 1e-6:
            continue
        t64 = n @ (a - oo) / den
        p = oo + t64 * dd
        # barycentrics by sub-areas
        area = np.linalg.norm(n)
        w1 = np.dot(np.cross(p - a, c - a), n) / area ** 2
        w2 = np.dot(np.cross(b - a, p - a), n) / area ** 2
        w0 = 1 - w1 - w2
        margin = min(w0, w1, w2)
        if t64 > 1e-4 and margin > 1e-4:
            assert hit and abs(t - t64) <= 1e-5 * max(1.0, t64)
            assert front == (den < 0)
            agree += 1
        elif t64 < -1e-4 or margin < -1e-4:
            assert not hit
    assert agree > 500


def test_min_over_rays_plane_law():
    # Floor only (huge quad at y = 0, normal +y); texel j at height d0 =
    # (jy + 0.5) h.  U = d0 / r_min has CDF ((1+u)/2)^R on [0, 1].
    R, nf = 8, 64
    v = np.array([[-1e3, 0, -1e3], [-1e3, 0, 1e3], [1e3, 0, 1e3], [1e3, 0, -1e3]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    rng = np.random.default_rng(1)
    jx, jz = rng.integers(0, nf, 3000), rng.integers(0, nf, 3000)
    jy = rng.integers(0, 8, 3000)
    tex = jx + nf * (jy + nf * jz)
    tex = np.unique(tex)
    r, cf, cb, _ = oracle.trace(v, t, BMIN, 1.0, nf, 99, 0, R, tex)
    d0 = ((tex // nf) % nf + 0.5) / nf
    U = np.where(np.isfinite(r), d0 / r, 0.0)
    U = np.sort(np.minimum(U, 1.0))
    n = U.size
    F = ((1 + U) / 2) ** R
    ks = max(np.max(np.arange(1, n + 1) / n - F), np.max(F - np.arange(0, n) / n))
    assert ks < 1.63 / math.sqrt(n)      # 1 % critical value
    # every hit is a front hit (rays come from above the upward floor)
    assert np.all(cb == 0) and cf.sum() > 0
    # from below the floor every hit is a back hit
    vb = v.copy()
    vb[:, 1] = 0.9
    r2, cf2, cb2, _ = oracle.trace(vb, t, BMIN, 1.0, nf, 99, 0, R, tex)
    assert np.all(cf2 == 0) and cb2.sum() > 0


def test_inside_box_back_hits_and_lower_bound():
    m = S.merge([S.box_mesh((0.5, 0.5, 0.5), 0.3)])
    nf = 32
    j = np.arange(nf ** 3)
    cen = (np.stack([j % nf, (j // nf) % nf, j // (nf * nf)], 1) + 0.5) / nf
    inside = np.all(np.abs(cen - 0.5) < 0.29, axis=1)
    tex = np.random.default_rng(2).choice(np.nonzero(inside)[0], 400, replace=False)
    r, cf, cb, _ = oracle.trace(m.verts, m.tris, BMIN, 1.0, nf, 5, 0, 16, tex)
    assert np.all(cf == 0) and np.all(cb == 16)     # every ray escapes through a back face
    d = oracle.point_mesh_distance(m.verts, m.tris, cen[tex])
    assert np.all(r >= d - 1e-6)


def test_traced_minimum_bounds_and_convergence():
    m = S.tiny_scene()
    nc, nf = 16, 32
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, nc)
    seeds, _ = oracle.jfa(occ, nc)
    c = oracle.coarse_sdf(seeds, nc, 1.0, 0.5)
    mask, _ = oracle.mask_fill(seeds, nc, 2.0, 0.5, c)
    tex = np.random.default_rng(4).choice(np.nonzero(mask)[0], 300, replace=False)
    cen = oracle.texel_centres(BMIN, 1.0, nf, tex).astype(np.float64)
    d = oracle.point_mesh_distance(m.verts, m.tris, cen)
    u = np.full(tex.size, np.inf)
    med = []
    for frame in range(16):
        r, *_ = oracle.trace(m.verts, m.tris, BMIN, 1.0, nf, 0, frame, 16, tex)
        un = oracle.eq1_update(u, 0.0, r, 1.0)
        assert np.all(un <= u)                      # non-increasing (alpha = 1)
        u = un
        fin = np.isfinite(u)
        assert np.all(u[fin] >= d[fin] - 1e-6)      # never below the true distance
        if frame in (0, 3, 15):
            med.append(np.median((u[fin] - d[fin]) / np.maximum(d[fin], 1e-3)))
    assert med[0] > med[1] > med[2]


def test_eq1_and_sign_and_reset_rules():
    u = np.array([np.inf, 0.3, 0.3, np.inf])
    c = np.array([0.1, 0.1, -0.02, 0.2])
    r = np.array([0.5, 0.2, np.inf, np.inf])
    assert np.array_equal(oracle.eq1_update(u, c, r, 1.0), [0.5, 0.2, 0.3, np.inf])
    assert np.allclose(oracle.eq1_update(u, c, r, 0.0), [0.1, 0.1, -0.02, 0.2])
    assert np.allclose(oracle.eq1_update(u, c, r, 0.5), [0.5, 0.2, 0.14, np.inf])
    s = oracle.signed_output(np.array([0.2, np.inf, 0.1]), np.array([0.3, 0.3, 0.3]),
                             np.array([3, 0, 2]), np.array([1, 0, 5]))
    assert np.allclose(s, [0.2, 0.3, -0.1])
    p = np.array([[0.5, 0.5, 0.5], [0.9, 0.5, 0.5]], np.float32)
    lo = np.array([[0.6, 0.4, 0.4]], np.float32)
    hi = np.array([[0.7, 0.6, 0.6]], np.float32)
    assert list(oracle.reset_rule(p, np.array([0.11, 0.1]), lo, hi)) == [True, False]
    assert list(oracle.reset_rule(p, np.array([0.09, 0.21]), lo, hi)) == [False, True]


# --------------------------------------------------------------------------
# The nearest-hit sign variant (the face of the nearest hit found so far)
# --------------------------------------------------------------------------

def _box_pipeline(mesh, nc, sign, R=16, frames=2):
    pipe = oracle.FinePipeline(BMIN, 1.0, nc, 0.5, 2.0, 1.0, 9, sign=sign)
    for f in range(frames):
        pipe.frame(mesh.verts, mesh.tris, f, R)
    return pipe


def test_nearest_sign_inside_and_outside_a_closed_box():
    # every first hit from inside a closed, outward-facing box is a back face
    # and every first hit from outside one is a front face
    m = S.merge([S.box_mesh((0.5, 0.5, 0.5), 0.25)])
    nc = 16
    vote = _box_pipeline(m, nc, "vote")
    near = _box_pipeline(m, nc, "nearest")
    tx = near.texels()
    hit = np.isfinite(near.u)
    assert hit.sum() > 1000
    assert np.array_equal(near.u, vote.u)               # same rays, same minimum
    nf = 2 * nc
    cen = (np.stack([tx % nf, (tx // nf) % nf, tx // (nf * nf)], 1) + 0.5) / nf
    inside = np.all(np.abs(cen - 0.5) < 0.25, axis=1)
    assert np.all(near.f[hit & inside] < 0) and np.all(near.f[hit & ~inside] > 0)


def test_nearest_sign_follows_the_closest_ray_not_the_vote():
    # texels inside a big closed box, just behind a small front-facing plate:
    # most rays end on the box walls (back faces), so the vote is negative,
    # while the nearest hit is the plate's front face whenever some ray meets it
    plate = (np.array([[0.40, 0.5, 0.40], [0.62, 0.5, 0.45], [0.45, 0.5, 0.62]], np.float64),
             np.array([[0, 1, 2]], np.int64))                    # normal -y (faces the texels below)
    m = S.merge([S.box_mesh((0.5, 0.5, 0.5), 0.45), plate])
    nc, R = 16, 4            # few rays: some texels meet the plate in one frame only
    nf = 2 * nc
    vote = _box_pipeline(m, nc, "vote", R=R, frames=2)
    near = _box_pipeline(m, nc, "nearest", R=R, frames=2)
    tx = near.texels()
    cen = (np.stack([tx % nf, (tx // nf) % nf, tx // (nf * nf)], 1) + 0.5) / nf
    below = (np.abs(cen[:, 1] - 0.47) < 0.02) & (np.abs(cen[:, 0] - 0.48) < 0.03) & \
            (np.abs(cen[:, 2] - 0.48) < 0.03) & np.isfinite(near.u)
    assert below.sum() >= 4
    # independent check: cast the texel's rays of both frames one by one and
    # take the face of the closest one (ties: front)
    for i in np.nonzero(below)[0]:
        o = cen[i].astype(np.float32)
        dirs = np.stack([oracle.sphere_dir(9, int(tx[i]), f, r)[0] for f in range(2) for r in range(R)])
        t, front, _ = oracle.cast_rays(m.verts, m.tris, np.repeat(o[None], 2 * R, 0), dirs)
        tmin = t.min()
        want_back = 0 if np.any(front[t == tmin]) else 1
        assert near.u[i] == tmin
        assert (near.f[i] < 0) == bool(want_back)
    assert np.any(near.f[below] > 0) and np.any(vote.f[below] < 0)
    assert np.any((near.f[below] > 0) & (vote.f[below] < 0))   # the two statistics differ here


# --------------------------------------------------------------------------
# The hierarchy path of the oracle's closest hit equals the brute-force one
# --------------------------------------------------------------------------

def _masked_sample(mesh, nc, count, seed):
    occ = oracle.voxelize(mesh.verts, mesh.tris, BMIN, 1.0, nc)
    seeds, _ = oracle.jfa(occ, nc)
    c = oracle.coarse_sdf(seeds, nc, 1.0, 0.5)
    mask, _ = oracle.mask_fill(seeds, nc, 2.0, 0.5, c)
    tx = np.nonzero(mask)[0]
    return np.sort(np.random.default_rng(seed).choice(tx, min(count, tx.size), replace=False))


@pytest.mark.parametrize("scene", ["tiny", "room", "soup", "spheres"])
def test_bvh_trace_equals_brute_force(scene):
    # masked texels (the tracer's real origins, next to surfaces) and
    # uniformly random ones; every output bit for bit
    if scene == "tiny":
        m, nc, n = S.tiny_scene(), 32, 1500
    elif scene == "room":
        m, nc, n = S.room_scene(1, n_objects=60, n_spheres=20), 64, 300
    elif scene == "soup":
        m, nc, n = S.random_soup(4, 3000), 32, 600
    else:
        m, nc, n = S.animated_scene(3, n_objects=30, n_lon=16, n_lat=9), 48, 600
    nf = 2 * nc
    tex = np.unique(np.concatenate([_masked_sample(m, nc, n, 1),
                                    np.random.default_rng(2).choice(nf ** 3, n // 3, replace=False)]))
    for frame in (0, 1):
        a = oracle.trace(m.verts, m.tris, BMIN, 1.0, nf, 7, frame, 16, tex, nearest=True)
        b = oracle.trace(m.verts, m.tris, BMIN, 1.0, nf, 7, frame, 16, tex, nearest=True, accel="bvh")
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.isfinite(a[0]).mean() > 0.5


def test_bvh_cast_rays_grazing_and_axis_parallel():
    # rays in the planes of axis-aligned box faces and along their edges,
    # rays through vertices, zero direction components, origins on faces,
    # and random near-grazing directions: the hierarchy must not skip a
    # triangle that the fp32 test accepts
    m = S.merge([S.box_mesh((0.5, 0.5, 0.5), 0.25), S.box_mesh((0.3, 0.7, 0.3), 0.1),
                 S.icosphere_mesh(2, (0.7, 0.3, 0.6), 0.12)])
    rng = np.random.default_rng(8)
    o, d = [], []
    for _ in range(3000):
        axis = rng.integers(0, 3)
        p = rng.uniform(0.2, 0.8, 3)
        p[axis] = rng.choice([0.25, 0.75, 0.2, 0.4, 0.5])        # on a face plane
        q = rng.normal(size=3)
        q[axis] = rng.choice([0.0, 1e-7, -1e-7, 1e-4])            # in or next to that plane
        o.append(p)
        d.append(q / np.linalg.norm(q))
    for vtx in m.verts[::7]:
        p = rng.uniform(0, 1, 3)
        o.append(p)
        d.append((vtx - p) / np.linalg.norm(vtx - p))              # aimed at a vertex
    for k in range(300):
        q = np.zeros(3)
        q[k % 3] = 1.0 if k % 2 else -1.0                          # two zero components
        o.append(rng.uniform(0.1, 0.9, 3))
        d.append(q)
    o = np.array(o, np.float32)
    d = np.array(d, np.float32)
    a = oracle.cast_rays(m.verts, m.tris, o, d)
    b = oracle.cast_rays(m.verts, m.tris, o, d, accel="bvh")
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert np.isfinite(a[0]).mean() > 0.3


def test_bvh_exact_distance_ties_keep_the_smaller_index():
    # a floor of 8 x 8 quads on a dyadic grid, each split along a diagonal,
    # triangles in shuffled order; rays straight down onto shared edges and
    # vertices hit several triangles at exactly the same fp32 distance, and
    # the smaller triangle index must win whatever order the hierarchy
    # visits them in
    g = 8
    verts = np.array([[i / g, 0.5, k / g] for k in range(g + 1) for i in range(g + 1)], np.float32)
    tris = []
    for k in range(g):
        for i in range(g):
            a, b, c, d = k * (g + 1) + i, k * (g + 1) + i + 1, (k + 1) * (g + 1) + i + 1, (k + 1) * (g + 1) + i
            tris += [[a, c, b], [a, d, c]]
    tris = np.array(tris, np.int32)[np.random.default_rng(3).permutation(2 * g * g)]
    o, d = [], []
    for k in range(g):
        for i in range(g):
            for s in (0.25, 0.5, 0.75):
                o.append([(i + s) / g, 0.75, (k + s) / g])         # on a diagonal
            o.append([(i + 0.5) / g, 0.75, k / g])                # on a shared grid edge
            o.append([i / g, 0.75, k / g])                        # on a shared vertex
    o = np.array(o, np.float32)
    d = np.tile(np.array([[0.0, -1.0, 0.0]], np.float32), (o.shape[0], 1))
    a = oracle.cast_rays(verts, tris, o, d)
    b = oracle.cast_rays(verts, tris, o, d, accel="bvh")
    assert np.all(a[0] == np.float32(0.25))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
