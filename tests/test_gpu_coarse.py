"""GPU parity of Sec. 2.1 (voxelization, jump flooding, coarse SDF) and the
Eq. 1 mask: integer outputs bit-exact against the oracle, the coarse SDF
within fp32 rounding (|dc| <= 1e-6 extent)."""
import numpy as np
import pytest

import oracle
from synth import scenes as S
from tests._util import seeds_to_linear

pytestmark = pytest.mark.gpu

BMIN = np.zeros(3, np.float32)


def _ctx(nc, beta=0.5, **kw):
    from paper_2210_04449_gb300 import RTSDF
    return RTSDF(nc, beta_vox=beta, **kw)


def _scenes():
    tiny = S.tiny_scene()
    soup = S.random_soup(3, 300, size=0.08)
    big = S.merge([S.room_quads()])                       # large floor/wall triangles
    one = S.Mesh(np.array([[0.2, 0.3, 0.4], [0.7, 0.35, 0.45], [0.4, 0.8, 0.6]], np.float32),
                 np.array([[0, 1, 2]], np.int32))
    sliver = S.Mesh(np.array([[0.1, 0.5, 0.5], [0.9, 0.5001, 0.5], [0.5, 0.5002, 0.5001]], np.float32),
                    np.array([[0, 1, 2]], np.int32))
    return {"tiny": tiny, "soup": soup, "room": big, "one": one, "sliver": sliver}


@pytest.mark.parametrize("tile", [0, 4])
@pytest.mark.parametrize("name", ["tiny", "soup", "room", "one", "sliver"])
@pytest.mark.parametrize("nc", [1, 2, 3, 16, 37, 48])
def test_voxelize_and_jfa_bit_exact(name, nc, tile):
    # tile 0: one voxel per thread; tile 4: four voxels per thread sharing
    # their z-slices (ragged z-lattices at nc = 3, 37, 48)
    m = _scenes()[name]
    rt = _ctx(nc)
    rt.set_tuning(jfa_tile=tile)
    rt.upload_mesh(m.verts, m.tris)
    rt.voxelize()
    occ_g = seeds_to_linear(rt.grids()["seeds"].cpu().numpy(), nc)
    occ_o = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, nc)
    assert np.array_equal(occ_g, occ_o)
    rt.jfa()
    g = rt.grids()
    seeds_g = seeds_to_linear(g["seeds"].cpu().numpy(), nc)
    seeds_o, passes = oracle.jfa(occ_o, nc)
    assert np.array_equal(seeds_g, seeds_o)
    assert rt.stats()["jfa_passes"] == passes
    c_o = oracle.coarse_sdf(seeds_o, nc, 1.0, 0.5)
    c_g = g["coarse"].cpu().numpy().astype(np.float64)
    fin = np.isfinite(c_o)
    assert np.array_equal(fin, np.isfinite(c_g))
    assert np.all(np.abs(c_g[fin] - c_o[fin]) <= 1e-6)
    rt.sync()


def test_empty_scene():
    rt = _ctx(8)
    rt.upload_mesh(np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32))
    rt.build_bvh()
    rt.update(2.0, 4, 0)
    g = rt.grids()
    assert np.all(g["seeds"].cpu().numpy() == 0xFFFFFFFF)
    assert np.all(np.isinf(g["coarse"].cpu().numpy()))
    assert rt.masked_count() == 0
    assert np.all(np.isinf(g["fine"].cpu().numpy()))
    rt.sync()


@pytest.mark.parametrize("nc", [128, 256])
def test_full_size_room_and_sphere_cloud(nc):
    # the coarse grids of the workloads (the 256^3 one is the benchmark scene,
    # 1,000,000 triangles): bit-exact voxels and seeds under every pass
    # kernel, and the coarse SDF of the last pass
    m = S.room_scene(1) if nc == 128 else S.animated_scene(2, n_objects=500)
    rt = _ctx(nc)
    rt.upload_mesh(m.verts, m.tris)
    rt.voxelize()
    occ_g = seeds_to_linear(rt.grids()["seeds"].cpu().numpy(), nc)
    occ_o = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, nc)
    assert np.array_equal(occ_g, occ_o)
    seeds_o, _ = oracle.jfa(occ_o, nc)
    for tile in range(5):   # every pass kernel the tuner can pick
        rt.set_tuning(jfa_tile=tile)
        rt.voxelize()
        rt.jfa()
        seeds_g = seeds_to_linear(rt.grids()["seeds"].cpu().numpy(), nc)
        assert np.array_equal(seeds_g, seeds_o), tile
    c_g = rt.grids()["coarse"].cpu().numpy().astype(np.float64)
    c_o = oracle.coarse_sdf(seeds_o, nc, 1.0, 0.5)
    fin = np.isfinite(c_o)
    assert np.array_equal(fin, np.isfinite(c_g))
    assert np.max(np.abs(c_g[fin] - c_o[fin])) <= 1e-6
    rt.sync()


@pytest.mark.parametrize("d_vox,beta", [(2.0, 0.5), (1.0, 0.0), (3.5, 1.0), (0.0, 0.5)])
def test_mask_and_fill(d_vox, beta):
    nc = 24
    m = S.tiny_scene()
    rt = _ctx(nc, beta=beta)
    rt.upload_mesh(m.verts, m.tris)
    rt.build_bvh()
    rt.update(d_vox, 1, 0)
    g = rt.grids()
    n_m = rt.masked_count()
    masked_g = np.sort(g["masked"].cpu().numpy()[:n_m].astype(np.int64))
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, nc)
    seeds, _ = oracle.jfa(occ, nc)
    c = oracle.coarse_sdf(seeds, nc, 1.0, beta)
    mask, fill = oracle.mask_fill(seeds, nc, d_vox, beta, c)
    par = oracle.parent_index(nc)
    masked_o = np.unique(par[mask])
    assert np.array_equal(masked_g, masked_o)
    f = g["fine"].cpu().numpy().astype(np.float64)
    assert np.all(np.abs(f[~mask] - fill[~mask]) <= 1e-6)
    rt.sync()
