"""The two node-fetch paths of the BVH traversal give the same results.

The tracers take the z planes and child ids of every 4-wide node through the
texture pipe when the node array fits a linear texture, and plain loads
otherwise (arrays beyond the device's texture width).  The scenes here are
small enough for textures, so the plain-load path is forced with the test
switch rtsdf_debug_texture_fetch; the per-scene tracer (with object motion
and the reset), the exact-occlusion fallback and the batched tracer (split
launches) must give bit-identical outputs either way.
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
