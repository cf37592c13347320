"""Pins for the oracle's soft-shadow march and its derivative (Sec. 2.3).

* Trilinear sampling reproduces linear fields exactly and the texel values
  at texel centres.
* A ray running parallel to a plane sees a constant h = H, so the penumbra
  term has the closed form k H (sqrt 3 / 2) / (t - H/2) at every step after
  the first, and the visibility is its value at the last step inside the
  volume -- this pins the step rule, the exit rule and the Aaltonen-style
  penumbra estimate together.
* Umbra and fully-lit special cases.
* The reverse-mode derivative agrees with fp64 central finite differences
  (step 1e-4) of the forward march, kinks excluded.
* The jitter of the ray origin toward the light: 24-bit fractions, uniform
  on [0, 1) and independent across frames; a shifted origin keeps the
  closed form above and moves the exit step by exactly the shift.
* The TAA resolve: constant images are fixed points, blend 1 returns the
  current frame, results stay inside the current 3x3 range, a far history
  clamps to that range, and an unclamped history decays as (1 - blend)^t.
"""
import math

import numpy as np
import pytest

import oracle
from synth import scenes as S

BMIN = np.zeros(3)


def _linear_grid(n, grad, c0):
    c = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    return (grad[0] * X + grad[1] * Y + grad[2] * Z + c0).astype(np.float32)


def test_trilinear_exact_on_linear_fields():
    n = 16
    g = _linear_grid(n, (0.3, -0.7, 0.2), 0.05)
    rng = np.random.default_rng(0)
    for _ in range(200):
        q = rng.uniform(0.5 / n, 1 - 0.5 / n, 3)
        v = oracle.sample(g, n, BMIN, 1.0, q)
        assert abs(v - (0.3 * q[0] - 0.7 * q[1] + 0.2 * q[2] + 0.05)) < 1e-6
    # texel centre returns the texel value
    j = (3, 7, 11)
    q = (np.array(j) + 0.5) / n
    assert oracle.sample(g, n, BMIN, 1.0, q) == pytest.approx(float(g[j[2], j[1], j[0]]), abs=1e-12)


@pytest.mark.parametrize("H,k,smax_vox,steps", [(0.06, 8.0, 4.0, 64), (0.04, 4.0, 2.0, 64), (0.03, 4.0, 2.0, 64),
                                                (0.05, 8.0, 1.0, 20), (0.2, 2.0, 8.0, 64)])
def test_march_parallel_to_plane_closed_form(H, k, smax_vox, steps):
    n = 32
    h = 1.0 / n
    y0 = 0.1
    grid = _linear_grid(n, (0, 1, 0), -y0)          # SDF = y - y0
    eps = h
    smax = smax_vox * h
    # start point o = p + 2 eps nrm at height H above the plane, x = 0.1
    p = np.array([[0.1, y0 + H - 2 * eps, 0.5]], np.float32)
    nrm = np.array([[0, 1, 0]], np.float32)
    vis = oracle.shadow(grid, n, BMIN, 1.0, p, nrm, (1.0, 0.0, 0.0), k, steps, smax, eps)[0]
    o = p[0].astype(np.float64) + 2 * eps * nrm[0]
    Hf = o[1] - y0
    step = min(Hf, smax)
    res = 1.0
    for i in range(steps):
        t = i * step
        if o[0] + t > 1.0:
            break
        if i >= 1 and t - Hf / 2 > 0:
            res = min(res, k * Hf * math.sqrt(3) / 2 / (t - Hf / 2))
    if Hf < eps:
        res = 0.0                                   # h < eps at the first sample
    assert vis == pytest.approx(res, rel=2e-6, abs=1e-12)   # grid values are fp32


def test_umbra_and_lit():
    n = 32
    h = 1.0 / n
    grid = S.box_grid_sdf(n, (0.5, 0.5, 0.5), 0.25, floor_y=0.1)
    pos, nrm = S.floor_gbuffer(16, 16, y=0.1, lo=0.4, hi=0.6)
    vis = oracle.shadow(grid, n, BMIN, 1.0, pos, nrm, (0, 1, 0), 8.0, 64, 4 * h, h)
    assert np.all(vis == 0.0)                 # straight under the box: umbra
    pos, nrm = S.floor_gbuffer(16, 16, y=0.1, lo=0.0, hi=0.2)
    vis = oracle.shadow(grid, n, BMIN, 1.0, pos, nrm, (0, 1, 0), 8.0, 64, 4 * h, h)
    assert np.all(vis == 1.0)                 # far from the box, light overhead


def _fd_setup(n=32, k=2.0):
    h = 1.0 / n
    grid = np.minimum(S.sphere_grid_sdf(n, (0.5, 0.35, 0.5), 0.12),
                      S.box_grid_sdf(n, (0.3, 0.3, 0.65), 0.06)).astype(np.float32)
    grid = np.minimum(grid, _linear_grid(n, (0, 1, 0), -0.1))       # floor y = 0.1
    pos, nrm = S.floor_gbuffer(24, 24, y=0.1, lo=0.1, hi=0.9)
    cfg = dict(k=k, steps=64, step_max=4 * h, eps=h)
    return n, grid, pos, nrm, cfg


def test_gradient_matches_finite_differences():
    n, grid, pos, nrm, cfg = _fd_setup()
    Lv = np.array([0.4, 1.0, 0.3])
    rng = np.random.default_rng(7)
    w = rng.normal(size=pos.shape[0] * pos.shape[1])

    def loss(g, lv):
        return float(w @ oracle.shadow(g, n, BMIN, 1.0, pos, nrm, lv, **cfg))

    gs, gl = oracle.shadow_grad(grid, n, BMIN, 1.0, pos, nrm, Lv, dvis=w, **cfg)
    nz = np.nonzero(gs)[0]
    assert nz.size > 50
    pick = np.concatenate([nz[np.argsort(-np.abs(gs[nz]))[:60]], rng.choice(nz, 60, replace=False)])
    ok = kinks = 0
    flat = grid.reshape(-1)
    for j in np.unique(pick):
        hstep = 1e-4
        gp = flat.copy(); gp[j] += np.float32(hstep)
        gm = flat.copy(); gm[j] -= np.float32(hstep)
        dp = float(gp[j]) - float(flat[j])
        dm = float(flat[j]) - float(gm[j])
        l0 = loss(flat, Lv)
        fp = (loss(gp, Lv) - l0) / dp
        fm = (l0 - loss(gm, Lv)) / dm
        if abs(fp - fm) > 0.1 * max(abs(fp), abs(fm), 1e-12):
            kinks += 1
            continue
        fd = (loss(gp, Lv) - loss(gm, Lv)) / (dp + dm)
        assert abs(fd - gs[j]) <= 1e-3 * max(abs(fd), 1e-3 * np.max(np.abs(gs))), (j, fd, gs[j])
        ok += 1
    assert ok >= 60 and kinks <= ok
    # light direction: FD over the pixels whose march is smooth around L (the
    # same discrete path -- samples taken, arg-min step, termination -- and
    # one-sided slopes that agree, so no step-limit or cell-boundary kink)
    vis0, info0 = oracle.shadow(flat, n, BMIN, 1.0, pos, nrm, Lv, info=True, **cfg)
    smooth = np.ones(info0.shape[0], bool)
    central = []
    for a in range(3):
        e = np.zeros(3); e[a] = 1e-4
        vp, ip = oracle.shadow(flat, n, BMIN, 1.0, pos, nrm, Lv + e, info=True, **cfg)
        vm, im = oracle.shadow(flat, n, BMIN, 1.0, pos, nrm, Lv - e, info=True, **cfg)
        sp, sm = (vp - vis0) / 1e-4, (vis0 - vm) / 1e-4
        smooth &= np.all(ip == info0, axis=1) & np.all(im == info0, axis=1)
        smooth &= np.abs(sp - sm) <= 1e-2 * np.maximum(np.maximum(np.abs(sp), np.abs(sm)), 1e-3)
        central.append((vp - vm) / 2e-4)
    assert smooth.mean() > 0.8
    ws = np.where(smooth, w, 0.0)
    _, gl = oracle.shadow_grad(grid, n, BMIN, 1.0, pos, nrm, Lv, dvis=ws, **cfg)
    for a in range(3):
        fd = float(ws @ central[a])
        assert abs(fd - gl[a]) <= 1e-3 * max(abs(fd), 1e-6), (a, fd, gl[a])


# --------------------------------------------------------------------------
# Sec. 2.3's jittered ray origin and the temporal anti-aliasing resolve
# --------------------------------------------------------------------------

def test_jitter_fractions_uniform_and_per_frame():
    n = 200_000
    xi = oracle.shadow_jitter(11, 3, n)
    assert np.all((xi >= 0) & (xi < 1))
    assert np.all(xi * 2 ** 24 == np.floor(xi * 2 ** 24))      # 24-bit fractions
    assert np.array_equal(xi, oracle.shadow_jitter(11, 3, n))  # a function of (seed, frame, pixel)
    # uniform on [0, 1): Kolmogorov-Smirnov distance against the identity
    s = np.sort(xi)
    ks = np.max(np.maximum(np.arange(1, n + 1) / n - s, s - np.arange(n) / n))
    assert ks < 1.63 / math.sqrt(n)                             # p > 0.01
    assert abs(xi.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    other = oracle.shadow_jitter(11, 4, n)                      # another frame
    assert abs(np.corrcoef(xi, other)[0, 1]) < 5 / math.sqrt(n)
    assert not np.array_equal(xi, oracle.shadow_jitter(12, 3, n))


@pytest.mark.parametrize("shift", [0.0, 0.05, 0.13, 0.31])
def test_jittered_march_parallel_to_plane_closed_form(shift):
    # as the closed form above, with the origin moved by `shift` along L:
    # the march samples o + (shift + t) L, so it leaves the volume after
    # fewer steps while h and the penumbra terms (in t) stay the same
    n, H, k, smax_vox, steps = 32, 0.06, 8.0, 4.0, 64
    h = 1.0 / n
    y0 = 0.1
    grid = _linear_grid(n, (0, 1, 0), -y0)
    eps, smax = h, smax_vox * h
    p = np.array([[0.1, y0 + H - 2 * eps, 0.5]], np.float32)
    nrm = np.array([[0, 1, 0]], np.float32)
    vis = oracle.shadow(grid, n, BMIN, 1.0, p, nrm, (1.0, 0.0, 0.0), k, steps, smax, eps,
                        shift=np.array([shift]))[0]
    o = p[0].astype(np.float64) + 2 * eps * nrm[0]
    Hf = o[1] - y0
    step = min(Hf, smax)
    res, last = 1.0, -1
    for i in range(steps):
        t = i * step
        if o[0] + shift + t > 1.0:
            break
        last = i
        if i >= 1 and t - Hf / 2 > 0:
            res = min(res, k * Hf * math.sqrt(3) / 2 / (t - Hf / 2))
    assert vis == pytest.approx(res, rel=2e-6, abs=1e-12)
    # the exit step moves with the shift: ceil((1 - o_x - shift) / step) samples
    assert last == math.floor((1.0 - o[0] - shift) / step + 1e-12)


def test_taa_resolve_rules():
    rng = np.random.default_rng(5)
    H, W = 9, 13
    cur = rng.random((H, W))
    # a constant image is a fixed point, blend 1 returns the current frame
    const = np.full((H, W), 0.37)
    assert np.array_equal(oracle.taa_resolve(const, const, 0.1), const)
    assert np.allclose(oracle.taa_resolve(cur, rng.random((H, W)), 1.0), cur, atol=0, rtol=0)
    # the result stays inside the current 3x3 neighbourhood's range
    hist = rng.uniform(-2, 3, (H, W))
    out = oracle.taa_resolve(cur, hist, 0.25)
    for y in range(H):
        for x in range(W):
            win = cur[max(y - 1, 0):y + 2, max(x - 1, 0):x + 2]
            assert win.min() - 1e-15 <= out[y, x] <= win.max() + 1e-15
    # checkerboard of 0/1 with the history far above: the history clamps to
    # the neighbourhood maximum 1, so out = 1 + b (cur - 1)
    cb = (np.add.outer(np.arange(H), np.arange(W)) % 2).astype(np.float64)
    out = oracle.taa_resolve(cb, np.full((H, W), 10.0), 0.2)
    assert np.allclose(out, 1.0 + 0.2 * (cb - 1.0), rtol=0, atol=1e-15)
    # a history inside the range decays geometrically toward a static frame
    h = np.minimum(cur + 0.01, 1.0)
    d0 = h - cur
    for _ in range(6):
        h = oracle.taa_resolve(cur, h, 0.1)
    pad = np.pad(cur, 1, mode="edge")
    mx = np.max([pad[dy:dy + H, dx:dx + W] for dy in range(3) for dx in range(3)], axis=0)
    inside = (cur + 0.01 <= mx)            # pixels whose first history was not clamped
    assert np.allclose((h - cur)[inside], (0.9 ** 6 * d0)[inside], rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- thin-surface fallback (Sec. 3)

def _one_triangle(z=1.0):
    v = np.array([[0.0, 0.0, z], [1.0, 0.0, z], [0.0, 1.0, z]], np.float32)
    return v, np.array([[0, 1, 2]], np.int32)


@pytest.mark.parametrize("light", [(0.0, 0.0, 1.0), (0.3, -0.2, 1.0), (-0.5, 0.4, 0.8)])
def test_exact_occlusion_closed_form(light):
    # floor points below the triangle x, y >= 0, x + y <= 1 at z = 1: the ray
    # toward L meets z = 1 at (x, y) + (1 - oz) (Lx, Ly) / Lz; blocked iff that
    # point is inside the triangle (points within 1e-3 of an edge skipped)
    v, t = _one_triangle()
    rng = np.random.default_rng(3)
    pos = np.zeros((4000, 3), np.float32)
    pos[:, :2] = rng.uniform(-0.6, 1.4, (4000, 2)).astype(np.float32)
    nrm = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (4000, 1))
    eps = np.float32(0.01)
    blocked = oracle.shadow_exact(v, t, pos, nrm, light, eps)
    L = np.asarray(light, np.float64) / np.linalg.norm(light)
    oz = 2.0 * float(eps)
    hx = pos[:, 0].astype(np.float64) + (1.0 - oz) * L[0] / L[2]
    hy = pos[:, 1].astype(np.float64) + (1.0 - oz) * L[1] / L[2]
    margin = np.minimum(np.minimum(hx, hy), 1.0 - hx - hy)
    clear = np.abs(margin) > 1e-3
    assert clear.sum() > 3500
    np.testing.assert_array_equal(blocked[clear], (margin > 0)[clear])
    assert 0 < blocked.sum() < blocked.size


def test_exact_occlusion_only_ahead_of_the_origin():
    # a light below the floor points away from the triangle: nothing blocks;
    # a triangle below the origin never blocks a ray going up
    v, t = _one_triangle(z=1.0)
    pos = np.array([[0.2, 0.2, 0.0], [0.1, 0.3, 0.0]], np.float32)
    nrm = np.tile(np.array([0.0, 0.0, 1.0], np.float32), (2, 1))
    assert not oracle.shadow_exact(v, t, pos, nrm, (0.0, 0.0, -1.0), 0.01).any()
    assert oracle.shadow_exact(v, t, pos, nrm, (0.0, 0.0, 1.0), 0.01).all()
    vb, tb = _one_triangle(z=-0.5)
    assert not oracle.shadow_exact(vb, tb, pos, nrm, (0.0, 0.0, 1.0), 0.01).any()


def test_exact_occlusion_is_the_any_hit_of_cast_rays():
    # the same decision as the tracer's closest-hit cast from the march origin
    m = S.random_soup(12, 300)
    rng = np.random.default_rng(4)
    pos = rng.uniform(0.0, 1.0, (500, 3)).astype(np.float32)
    nrm = rng.normal(size=(500, 3)).astype(np.float32)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    eps = np.float32(2.0 ** -8)
    blocked = oracle.shadow_exact(m.verts, m.tris, pos, nrm, (0.2, 1.0, 0.4), eps)
    L = oracle.unit_light((0.2, 1.0, 0.4))
    # 2 eps is a power of two, so n * 2 eps is exact in fp32 and the fp64 sum
    # of two fp32 values this close in magnitude is exact: rounding it once to
    # fp32 is fmaf(n, 2 eps, p)
    o = (pos.astype(np.float64) + nrm.astype(np.float64) * (2.0 * float(eps))).astype(np.float32)
    tout, _, tri = oracle.cast_rays(m.verts, m.tris, o, np.tile(L, (500, 1)))
    np.testing.assert_array_equal(blocked, tri >= 0)
    assert 0 < blocked.sum() < blocked.size


def test_fallback_takes_the_umbra_only_where_blocked():
    vis = np.array([0.0, 0.3, 1.0, 0.7])
    blocked = np.array([True, True, False, False])
    np.testing.assert_array_equal(oracle.shadow_fallback(vis, blocked), [0.0, 0.0, 1.0, 0.7])


def test_decision_margin_predicts_a_stable_march_path():
    # A point whose march keeps every discrete decision at a relative gap
    # above 1e-2 must take the same path (step count, minimising step,
    # termination) when the grid is perturbed by 1e-4 relative noise; the
    # noise must change the path of some points, and only of points with a
    # small margin.
    nf = 64
    g = np.minimum(S.sphere_grid_sdf(nf, (0.5, 0.35, 0.5), 0.12), S.box_grid_sdf(nf, (0.3, 0.3, 0.65), 0.06))
    c = (np.arange(nf) + 0.5) / nf
    grid = np.minimum(g, (c[None, :, None] - 0.1) * np.ones((nf, nf, nf))).astype(np.float32)
    pos, nrm = S.floor_gbuffer(256, 256, y=0.1, lo=0.05, hi=0.95)
    L, h = (0.4, 1.0, 0.3), 1.0 / nf
    cfg = (8.0, 64, 4 * h, h)
    m = oracle.shadow_margin(grid, nf, BMIN, 1.0, pos, nrm, L, *cfg)
    _, i0 = oracle.shadow(grid, nf, BMIN, 1.0, pos, nrm, L, *cfg, info=True)
    rng = np.random.default_rng(4)
    changed = np.zeros(m.size, bool)
    for _ in range(4):
        noisy = (grid.astype(np.float64) * (1 + rng.normal(0, 1e-4, grid.shape))).astype(np.float32)
        _, i1 = oracle.shadow(noisy, nf, BMIN, 1.0, pos, nrm, L, *cfg, info=True)
        changed |= np.any(i0 != i1, axis=1)
    assert changed.sum() >= 5
    assert np.all(m[changed] <= 1e-2)
    assert 0.9 < np.mean(m > 1e-2) < 1.0
