"""GPU parity of the thin-surface fallback (an exact occlusion test toward
the light from the march's origin, the reading of the paper's Sec. 3 future
work) and of tracing meshes with one or two triangles.

Bar: the occlusion flags are bit-identical to the oracle's brute-force test
(both sides decide in fp32 with the same origin, direction and ray/triangle
arithmetic); visibility after the fallback is exactly 0 where blocked and
the march's own value elsewhere.
"""
import numpy as np
import pytest

import oracle
from synth import scenes as S

pytestmark = pytest.mark.gpu

BMIN = np.zeros(3, np.float32)


def _ctx(mesh, nc=32, objects=False):
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(nc, seed=3)
    rt.upload_mesh(mesh.verts, mesh.tris)
    if objects:
        rt.set_objects(mesh.vert_object, mesh.n_objects)
    rt.build_bvh()
    return rt


def _points(seed, n, lo=0.02, hi=0.98):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    nrm = rng.normal(size=(n, 3)).astype(np.float32)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return pos, nrm


def _fallback(rt, pos, nrm, light, eps_vox, vis0):
    import torch
    dev = rt.device
    tp, tn = torch.tensor(pos, device=dev), torch.tensor(nrm, device=dev)
    vis = torch.tensor(vis0, device=dev, dtype=torch.float32)
    blocked = torch.zeros(pos.shape[0], device=dev, dtype=torch.uint8)
    rt.shadow_fallback(tp, tn, light, vis, eps_vox=eps_vox, blocked=blocked)
    rt.sync()
    return vis.cpu().numpy(), blocked.cpu().numpy().astype(bool)


@pytest.mark.parametrize("scene,light", [("soup", (0.2, 1.0, 0.4)), ("room", (0.3, 1.0, -0.2)),
                                         ("animated", (-0.4, 0.9, 0.1))])
def test_occlusion_flags_match_oracle(scene, light):
    mesh = {"soup": lambda: S.random_soup(21, 3000),
            "room": lambda: S.room_scene(22, n_objects=12, n_spheres=6),
            "animated": lambda: S.animated_scene(23, n_objects=20, n_lon=20, n_lat=11)}[scene]()
    nc, eps_vox = 32, 1.0
    rt = _ctx(mesh, nc)
    pos, nrm = _points(24, 6000)
    vis0 = np.random.default_rng(25).uniform(0.0, 1.0, pos.shape[0]).astype(np.float32)
    vis, blocked = _fallback(rt, pos, nrm, light, eps_vox, vis0)
    eps = np.float32(eps_vox) * (np.float32(1.0) / np.float32(2 * nc))
    want = oracle.shadow_exact(mesh.verts, mesh.tris, pos, nrm, light, eps)
    assert np.array_equal(blocked, want)
    assert 0 < want.sum() < want.size
    np.testing.assert_array_equal(vis, oracle.shadow_fallback(vis0, want).astype(np.float32))
    rt.close()


@pytest.mark.parametrize("n_tris", [1, 2])
def test_occlusion_with_one_or_two_triangles(n_tris):
    v = np.array([[0.2, 0.6, 0.2], [0.8, 0.6, 0.2], [0.2, 0.6, 0.8], [0.8, 0.6, 0.8]], np.float32)
    tris = np.array([[0, 1, 2], [1, 3, 2]], np.int32)[:n_tris]
    mesh = S.Mesh(v, tris)
    rt = _ctx(mesh, 16)
    pos, nrm = S.floor_gbuffer(64, 64, y=0.05)
    pos, nrm = pos.reshape(-1, 3), nrm.reshape(-1, 3)
    vis0 = np.ones(pos.shape[0], np.float32)
    vis, blocked = _fallback(rt, pos, nrm, (0.0, 1.0, 0.0), 1.0, vis0)
    eps = np.float32(1.0) * (np.float32(1.0) / np.float32(32))
    want = oracle.shadow_exact(v, tris, pos, nrm, (0.0, 1.0, 0.0), eps)
    assert np.array_equal(blocked, want) and want.any() and not want.all()
    rt.close()


def test_fallback_closes_the_umbra_under_a_thin_plate():
    # a plate of zero thickness over a floor: the fine SDF is traced, the
    # march gives the soft shadow, and the fallback makes every point whose
    # exact ray meets the plate fully shadowed
    import torch
    from paper_2210_04449_gb300 import RTSDF
    plate = np.array([[0.3, 0.5, 0.3], [0.7, 0.5, 0.3], [0.3, 0.5, 0.7], [0.7, 0.5, 0.7]], np.float32)
    floor = np.array([[0.0, 0.02, 0.0], [1.0, 0.02, 0.0], [0.0, 0.02, 1.0], [1.0, 0.02, 1.0]], np.float32)
    verts = np.concatenate([plate, floor])
    tris = np.array([[0, 2, 1], [1, 2, 3], [4, 6, 5], [5, 6, 7]], np.int32)
    nc = 32
    rt = RTSDF(nc, seed=4)
    rt.upload_mesh(verts, tris)
    rt.build_bvh()
    for t in range(4):
        rt.update(2.0, 16, t)
    pos, nrm = S.floor_gbuffer(96, 96, y=0.02)
    tp = torch.tensor(pos.reshape(-1, 3), device=rt.device)
    tn = torch.tensor(nrm.reshape(-1, 3), device=rt.device)
    light = (0.1, 1.0, 0.05)
    vis = rt.shadow(tp, tn, light, k=8.0, steps=64, step_max_vox=4.0, eps_vox=1.0)
    before = vis.cpu().numpy().copy()
    blocked = torch.zeros(tp.shape[0], device=rt.device, dtype=torch.uint8)
    rt.shadow_fallback(tp, tn, light, vis, eps_vox=1.0, blocked=blocked)
    rt.sync()
    after, b = vis.cpu().numpy(), blocked.cpu().numpy().astype(bool)
    assert b.sum() > 500                                   # the plate's exact shadow on the floor
    assert np.all(after[b] == 0.0)
    np.testing.assert_array_equal(after[~b], before[~b])
    eps = np.float32(1.0) * (np.float32(1.0) / np.float32(2 * nc))
    assert np.array_equal(b, oracle.shadow_exact(verts, tris, pos.reshape(-1, 3), nrm.reshape(-1, 3), light, eps))
    print(f"points the march left lit inside the plate's exact shadow: {(before[b] > 0).sum()} of {b.sum()}")
    rt.close()


def test_fallback_needs_a_current_bvh():
    from paper_2210_04449_gb300 import RTSDF, RtsdfError
    import torch
    m = S.animated_scene(26, n_objects=3, n_lon=12, n_lat=7)
    rt = RTSDF(16)
    rt.upload_mesh(m.verts, m.tris)
    rt.set_objects(m.vert_object, m.n_objects)
    pos, nrm = _points(27, 16)
    tp, tn = torch.tensor(pos, device=rt.device), torch.tensor(nrm, device=rt.device)
    vis = torch.ones(16, device=rt.device)
    with pytest.raises(RtsdfError):
        rt.shadow_fallback(tp, tn, (0.0, 1.0, 0.0), vis)          # no BVH yet
    rt.build_bvh()
    rt.shadow_fallback(tp, tn, (0.0, 1.0, 0.0), vis)
    rt.move_objects(np.full((3, 3), 0.01, np.float32))
    with pytest.raises(RtsdfError):
        rt.shadow_fallback(tp, tn, (0.0, 1.0, 0.0), vis)          # moved: the BVH needs a rebuild
    with pytest.raises(RtsdfError):
        rt.shadow_fallback(tp, tn, (0.0, 1.0, 0.0), None, blocked=None)
    rt.sync()
    rt.close()


@pytest.mark.parametrize("n_tris", [1, 2])
def test_trace_with_one_or_two_triangles(n_tris):
    # a one-triangle mesh has no BVH node: its only leaf starts parked
    from paper_2210_04449_gb300 import RTSDF
    v = np.array([[0.3, 0.4, 0.3], [0.7, 0.45, 0.35], [0.4, 0.5, 0.7], [0.75, 0.55, 0.7]], np.float32)
    tris = np.array([[0, 1, 2], [1, 3, 2]], np.int32)[:n_tris]
    nc, d, beta, R = 16, 2.0, 0.5, 16
    rt = RTSDF(nc, beta_vox=beta, seed=0)
    rt.upload_mesh(v, tris)
    rt.build_bvh()
    pipe = oracle.FinePipeline(BMIN, 1.0, nc, beta, d, 1.0, 0)
    for t in range(2):
        rt.update(d, R, t)
        pipe.frame(v, tris, t, R)
    rt.sync()
    g = rt.grids()
    tx = pipe.texels()
    u = g["accum"].cpu().numpy()[tx]
    cnt = g["counts"].cpu().numpy()[tx].astype(np.int64)
    assert tx.size > 0
    assert np.array_equal(np.isinf(u), np.isinf(pipe.u))
    fin = np.isfinite(u)
    assert np.max(np.abs(u[fin] - pipe.u[fin]), initial=0.0) <= 2e-5 * np.sqrt(3.0)
    assert np.array_equal(cnt & 0xFFFF, pipe.nF) and np.array_equal(cnt >> 16, pipe.nB)
    rt.close()


def test_full_size_flags_sampled():
    # the benchmark scene (500 spheres, 1,000,000 triangles) and a 1920x1080
    # floor G-buffer: every flag from the GPU, 512 sampled points from the
    # oracle's brute-force test over all triangles
    import torch
    from paper_2210_04449_gb300 import RTSDF
    mesh = S.animated_scene(2, n_objects=500)
    rt = RTSDF(256, seed=2)
    rt.upload_mesh(mesh.verts, mesh.tris)
    rt.build_bvh()
    pos, nrm = S.floor_gbuffer(1920, 1080, y=0.02)
    pos, nrm = pos.reshape(-1, 3), nrm.reshape(-1, 3)
    light = (0.4, 1.0, 0.3)
    tp, tn = torch.tensor(pos, device=rt.device), torch.tensor(nrm, device=rt.device)
    blocked = torch.zeros(pos.shape[0], device=rt.device, dtype=torch.uint8)
    rt.shadow_fallback(tp, tn, light, None, blocked=blocked)
    rt.sync()
    b = blocked.cpu().numpy().astype(bool)
    pick = np.random.default_rng(5).choice(pos.shape[0], 512, replace=False)
    eps = np.float32(1.0) * (np.float32(1.0) / np.float32(512))
    want = oracle.shadow_exact(mesh.verts, mesh.tris, pos[pick], nrm[pick], light, eps)
    assert np.array_equal(b[pick], want)
    assert 0.05 < b.mean() < 0.95
    rt.close()
