"""Pins for the oracle's jump flooding, coarse SDF and mask (Sec. 2.1-2.2).

Checked against brute-force exact Euclidean distance transforms (all
seeds), a separable exact EDT (itself checked against brute force), the
known exactness of jump flooding for a single seed, hand-built tie cases,
the analytic box/sphere distance bound, and the real-valued form of Eq. 1's
case split.
"""
import math

import numpy as np
import pytest

import oracle
from synth import scenes as S

BMIN = np.zeros(3, np.float32)


def _random_seeds(n, k, seed):
    rng = np.random.default_rng(seed)
    occ = np.full(n ** 3, -1, np.int32)
    idx = rng.choice(n ** 3, size=k, replace=False)
    occ[idx] = idx
    return occ


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 16, 17, 31])
def test_single_seed_is_exact(n):
    rng = np.random.default_rng(n)
    for _ in range(3):
        occ = _random_seeds(n, 1, int(rng.integers(1 << 30)))
        seeds, passes = oracle.jfa(occ, n)
        assert passes == math.ceil(math.log2(n)) if n > 1 else passes == 0
        s = occ[occ >= 0][0]
        assert np.all(seeds == s)


def test_corner_seed_reaches_far_corner():
    n = 32
    occ = np.full(n ** 3, -1, np.int32)
    occ[0] = 0
    seeds, passes = oracle.jfa(occ, n)
    assert passes == 5 and seeds[-1] == 0


@pytest.mark.parametrize("n,k", [(8, 3), (12, 10), (16, 40), (24, 30), (32, 200)])
def test_jfa_not_below_exact_and_rarely_wrong(n, k):
    occ = _random_seeds(n, k, 100 + n)
    seeds, _ = oracle.jfa(occ, n)
    d_jfa = oracle.seed_d2(seeds, n)
    d_ex = oracle.edt_brute(occ, n)
    assert np.all(d_jfa >= d_ex)
    rate = np.mean(d_jfa != d_ex)
    assert rate < 0.01, rate
    # every seed voxel keeps itself
    s = np.nonzero(occ >= 0)[0]
    assert np.all(seeds[s] == s)


@pytest.mark.parametrize("n", [7, 16, 20])
def test_separable_edt_equals_brute(n):
    occ = _random_seeds(n, 9, n)
    assert np.array_equal(oracle.edt_separable(occ, n), oracle.edt_brute(occ, n))
    empty = np.full(n ** 3, -1, np.int32)
    assert np.all(oracle.edt_separable(empty, n) == -1)


def test_tie_goes_to_smaller_linear_index():
    n = 8
    occ = np.full(n ** 3, -1, np.int32)
    a = 2 + n * (3 + n * 3)
    b = 6 + n * (3 + n * 3)
    occ[a] = a
    occ[b] = b
    seeds, _ = oracle.jfa(occ, n)
    mid = 4 + n * (3 + n * 3)
    assert seeds[mid] == a
    # tie across z: seeds above and below
    occ = np.full(n ** 3, -1, np.int32)
    a = 4 + n * (4 + n * 1)
    b = 4 + n * (4 + n * 5)
    occ[a] = a
    occ[b] = b
    seeds, _ = oracle.jfa(occ, n)
    assert seeds[4 + n * (4 + n * 3)] == a


def test_empty_grid():
    n = 8
    seeds, _ = oracle.jfa(np.full(n ** 3, -1, np.int32), n)
    assert np.all(seeds == -1)
    c = oracle.coarse_sdf(seeds, n, 1.0, 0.5)
    assert np.all(np.isinf(c))


def test_scene_mismatch_rate_and_edt():
    n = 32
    m = S.tiny_scene()
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, n)
    seeds, _ = oracle.jfa(occ, n)
    d_jfa = oracle.seed_d2(seeds, n)
    d_ex = oracle.edt_separable(occ, n)
    assert np.all(d_jfa >= d_ex)
    assert np.mean(d_jfa != d_ex) < 0.01


def test_coarse_sdf_against_mesh_distance():
    # Outside objects, where the JFA seed is an exact nearest seed,
    # |c - d_mesh| <= h (sqrt(3)/2 + beta) + quantisation (Sec. 2.1: the
    # coarse SDF is the distance to the nearest voxel minus beta).
    n, beta = 32, 0.5
    h = 1.0 / n
    m = S.tiny_scene()
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, n)
    seeds, _ = oracle.jfa(occ, n)
    c = oracle.coarse_sdf(seeds, n, 1.0, beta)
    exact = oracle.seed_d2(seeds, n) == oracle.edt_separable(occ, n)
    j = np.arange(n ** 3)
    cen = np.stack([j % n, (j // n) % n, j // (n * n)], 1) * h + h / 2
    (bc, bh), (sc, sr) = m.meta["box"], m.meta["sphere"]
    outside_box = np.any(np.abs(cen - np.array(bc)) > bh, axis=1)
    outside_sph = np.linalg.norm(cen - np.array(sc), axis=1) > sr
    sel = np.nonzero(exact & outside_box & outside_sph)[0]
    rng = np.random.default_rng(0)
    sel = rng.choice(sel, size=3000, replace=False)
    d = oracle.point_mesh_distance(m.verts, m.tris, cen[sel])
    err = c[sel] - d
    q = h * math.sqrt(3) / 512
    assert np.all(err <= h * (math.sqrt(3) / 2 - beta) + q + 1e-9)
    assert np.all(err >= -h * (math.sqrt(3) / 2 + beta) - q - 1e-9)
    # the analytic box SDF (exact for the box mesh) agrees with the mesh distance
    # where the box is the nearest object
    qb = np.maximum(np.abs(cen[sel] - np.array(bc)) - bh, 0)
    dbox = np.linalg.norm(qb, axis=1)
    dsph = np.linalg.norm(cen[sel] - np.array(sc), axis=1) - sr
    near_box = dbox < dsph - 0.02
    assert np.allclose(d[near_box], dbox[near_box], atol=1e-6)


@pytest.mark.parametrize("d_vox,beta", [(2.0, 0.5), (1.0, 0.25), (3.0, 0.0), (0.0, 0.5)])
def test_mask_matches_real_valued_case_split(d_vox, beta):
    # Eq. 1: fine texel is traced iff c_t <= d, with c_t the coarse value at
    # its parent voxel.  The integer test D2 <= floor((d+beta)^2) must give
    # the same set as the real comparison.
    n = 16
    m = S.tiny_scene()
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, n)
    seeds, _ = oracle.jfa(occ, n)
    c = oracle.coarse_sdf(seeds, n, 1.0, beta)
    mask, f = oracle.mask_fill(seeds, n, d_vox, beta, c)
    par = oracle.parent_index(n)
    real = c[par] <= d_vox / n + 1e-12
    assert np.array_equal(mask, real)
    assert np.all(np.isnan(f[mask])) and np.array_equal(f[~mask], c[par][~mask])


def test_parent_index():
    nc = 4
    par = oracle.parent_index(nc)
    nf = 8
    j = 5 + nf * (2 + nf * 7)   # fine (5, 2, 7) -> coarse (2, 1, 3)
    assert par[j] == 2 + nc * (1 + nc * 3)
