"""The two node-fetch paths of the BVH traversal give the same results.

The tracers take the z planes and child ids of every 4-wide node through the
texture pipe when the node array fits a linear texture, and plain loads
otherwise (arrays beyond the device's texture width).  The scenes here are
small enough for textures, so the plain-load path is forced with the test
switch rtsdf_debug_texture_fetch; the per-scene tracer (with object motion
and the reset), the exact-occlusion fallback and the batched tracer (split
launches) must give bit-identical outputs either way.  And the texture
object follows a node array that grows: a context, or a batch, re-used with
a larger mesh gives a fresh one's result.
"""
import numpy as np
import pytest

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _scene_run(mesh, n_obj):
    import torch
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(48, beta_vox=0.5, seed=11)
    rt.upload_mesh(mesh.verts, mesh.tris)
    rt.set_objects(mesh.vert_object, n_obj)
    rt.build_bvh()
    for t in range(3):
        if t:
            rt.move_objects(S.object_translations(5, t, n_obj, 1.0 / 48))
            rt.build_bvh()
        rt.update(2.0, 16, t)
    rt.sync()
    g = rt.grids()
    out = {k: g[k].cpu().numpy().copy() for k in ("accum", "counts", "fine")}
    pos, nrm = S.floor_gbuffer(64, 48, y=0.05)
    dev = torch.device("cuda")
    blocked = torch.zeros(64 * 48, device=dev, dtype=torch.uint8)
    rt.shadow_fallback(torch.tensor(pos, device=dev), torch.tensor(nrm, device=dev), (0.4, 1.0, 0.3), None,
                       blocked=blocked)
    rt.sync()
    out["blocked"] = blocked.cpu().numpy()
    rt.close()
    return out


def _batch_run(items):
    from paper_2210_04449_gb300 import RTSDFBatch
    b = RTSDFBatch([cfg for cfg, _ in items])
    b.set_tuning(split_trace=1)
    for sc, (_, mesh) in zip(b.scenes, items):
        sc.upload_mesh(mesh.verts, mesh.tris)
        sc.build_bvh()
    for f in range(2):
        b.frame(2.0, 16, f)
    b.sync()
    out = [{k: sc.grids()[k].cpu().numpy().copy() for k in ("accum", "counts", "fine")} for sc in b.scenes]
    b.close()
    return out


def test_texture_and_plain_node_fetch_agree():
    from paper_2210_04449_gb300 import _abi
    lib = _abi.lib()
    mesh = S.animated_scene(6, n_objects=30, n_lon=16, n_lat=9)
    items = [(dict(coarse_n=32, beta_vox=0.5, seed=2), S.room_scene(4, n_objects=10, n_spheres=4, subdiv=2)),
             (dict(coarse_n=40, beta_vox=0.5, seed=3), S.animated_scene(8, n_objects=12, n_lon=16, n_lat=9))]
    try:
        lib.rtsdf_debug_texture_fetch(1)
        tex = _scene_run(mesh, mesh.n_objects)
        tex_b = _batch_run(items)
        lib.rtsdf_debug_texture_fetch(0)
        plain = _scene_run(mesh, mesh.n_objects)
        plain_b = _batch_run(items)
    finally:
        lib.rtsdf_debug_texture_fetch(1)
    assert np.isfinite(tex["accum"]).sum() > 1000 and tex["blocked"].any()
    for k in tex:
        assert np.array_equal(tex[k], plain[k]), k
    for i, (a, b) in enumerate(zip(tex_b, plain_b)):
        for k in a:
            assert np.array_equal(a[k], b[k]), (i, k)


def test_node_texture_follows_a_growing_tree():
    # a context that first builds a small tree and then a tree several times
    # larger reallocates its node array; the texture object over it is
    # replaced, and the frame equals a fresh context's bit for bit
    from paper_2210_04449_gb300 import RTSDF
    small = S.tiny_scene()
    big = S.animated_scene(3, n_objects=25, n_lon=16, n_lat=9)

    def frame(rt, mesh):
        rt.upload_mesh(mesh.verts, mesh.tris)
        rt.build_bvh()
        rt.update(2.0, 16, 0)
        rt.sync()
        return {k: v.cpu().numpy().copy() for k, v in rt.grids().items() if k in ("accum", "counts", "fine")}

    rt = RTSDF(32, beta_vox=0.5, seed=4)
    frame(rt, small)
    rt.load_state(_fresh_state(32))
    got = frame(rt, big)
    rt.close()
    ref = RTSDF(32, beta_vox=0.5, seed=4)
    want = frame(ref, big)
    ref.close()
    for k in want:
        assert np.array_equal(got[k], want[k]), k


def _fresh_state(n):
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(n, beta_vox=0.5, seed=4)
    s = rt.save_state()
    rt.close()
    return s


def test_batch_node_texture_follows_a_growing_tree():
    # the batch's concatenated node array (and its texture) grows when a
    # scene's mesh does; the frame equals a fresh batch's
    from paper_2210_04449_gb300 import RTSDFBatch
    cfgs = [dict(coarse_n=24, beta_vox=0.5, seed=5), dict(coarse_n=32, beta_vox=0.5, seed=6)]
    small = S.tiny_scene()
    big = S.animated_scene(4, n_objects=20, n_lon=16, n_lat=9)

    def run(b, meshes, frame):
        for sc, m in zip(b.scenes, meshes):
            sc.upload_mesh(m.verts, m.tris)
            sc.build_bvh()
        b.frame(2.0, 16, frame)
        b.sync()
        return [{k: sc.grids()[k].cpu().numpy().copy() for k in ("accum", "counts", "fine")} for sc in b.scenes]

    b = RTSDFBatch(cfgs)
    b.set_tuning(split_trace=1)
    run(b, [small, small], 0)
    for sc in b.scenes:
        sc.load_state(_fresh_state_of(sc))
    got = run(b, [big, small], 0)
    b.close()
    f = RTSDFBatch(cfgs)
    f.set_tuning(split_trace=1)
    want = run(f, [big, small], 0)
    f.close()
    for i, (a, w) in enumerate(zip(got, want)):
        for k in w:
            assert np.array_equal(a[k], w[k]), (i, k)


def _fresh_state_of(sc):
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(sc.coarse_n, beta_vox=0.5, seed=0)
    s = rt.save_state()
    rt.close()
    return s
