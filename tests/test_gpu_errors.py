"""Error behaviour of the C ABI with a GPU: bad meshes (E_MESH), calls out
of order (E_STATE), bad arguments (E_ARG), a failed allocation (E_OOM), a
cyclic tree stopped by the traversal's bounds (E_OVERFLOW), and that a
context is usable again after each.  Nothing here provokes a device fault:
every error is a host-side argument check or a device validation word (bad
indices are rewritten to 0 and bad vertices clamped before any kernel reads
them; the cyclic tree's node ids are valid indices, and every traversal
loop and stack access is bounded)."""
import numpy as np
import pytest

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _name(fn, *a, **k):
    from paper_2210_04449_gb300 import RtsdfError
    with pytest.raises(RtsdfError) as ei:
        fn(*a, **k)
    return ei.value.name


def _fine_after_frame(rt, m, d=2.0, R=8):
    rt.upload_mesh(m.verts, m.tris)
    rt.build_bvh()
    rt.update(d, R, 0)
    rt.sync()
    return rt.grids()["fine"].cpu().numpy().copy()


def test_mesh_validation_then_recovery():
    from paper_2210_04449_gb300 import RTSDF
    m = S.tiny_scene()
    rt = RTSDF(16, seed=1)
    bad_index = m.tris.copy()
    bad_index[5, 1] = m.verts.shape[0]                  # one past the last vertex
    assert _name(rt.upload_mesh, m.verts, bad_index) == "RTSDF_E_MESH"
    negative = m.tris.copy()
    negative[0, 0] = -1
    assert _name(rt.upload_mesh, m.verts, negative) == "RTSDF_E_MESH"
    nan_vert = m.verts.copy()
    nan_vert[3, 0] = np.nan
    assert _name(rt.upload_mesh, nan_vert, m.tris) == "RTSDF_E_MESH"
    far_vert = m.verts.copy()
    far_vert[0] = (5.0, 5.0, 5.0)                       # outside [bmin - E/2, bmin + 3E/2]
    assert _name(rt.upload_mesh, far_vert, m.tris) == "RTSDF_E_MESH"
    # a rejected mesh leaves the context without a mesh
    assert _name(rt.voxelize) == "RTSDF_E_STATE"
    assert _name(rt.build_bvh) == "RTSDF_E_STATE"
    # a valid mesh afterwards gives exactly a fresh context's result
    got = _fine_after_frame(rt, m)
    want = _fine_after_frame(RTSDF(16, seed=1), m)
    assert np.array_equal(got, want)
    rt.close()


def test_calls_out_of_order():
    from paper_2210_04449_gb300 import RTSDF
    m = S.animated_scene(3, n_objects=4, n_lon=12, n_lat=7)
    rt = RTSDF(16)
    assert _name(rt.voxelize) == "RTSDF_E_STATE"         # no mesh yet
    assert _name(rt.bvh_topology) == "RTSDF_E_STATE"     # no BVH yet
    rt.upload_mesh(m.verts, m.tris)
    assert _name(rt.jfa) == "RTSDF_E_STATE"              # before voxelize
    assert _name(rt.build_bvh, refit=True) == "RTSDF_E_STATE"   # refit before a build
    assert _name(rt.trace, 2.0, 8, 0) == "RTSDF_E_STATE"         # before jfa
    assert _name(rt.move_objects, np.zeros((4, 3), np.float32)) == "RTSDF_E_STATE"   # no objects
    rt.voxelize()
    rt.jfa()
    assert _name(rt.trace, 2.0, 8, 0) == "RTSDF_E_STATE"         # no BVH yet
    rt.set_objects(m.vert_object, m.n_objects)
    rt.build_bvh()
    rt.trace(2.0, 8, 0)
    rt.move_objects(np.full((4, 3), 0.01, np.float32))
    assert _name(rt.trace, 2.0, 8, 1) == "RTSDF_E_STATE"         # moved: the BVH needs a refit
    rt.build_bvh(refit=True)
    rt.update(2.0, 8, 1)
    rt.sync()
    rt.close()


def test_argument_checks():
    import torch
    from paper_2210_04449_gb300 import RTSDF
    m = S.tiny_scene()
    rt = RTSDF(16)
    rt.upload_mesh(m.verts, m.tris)
    rt.build_bvh()
    rt.voxelize()
    rt.jfa()
    for rays in (0, 3, 2048):
        assert _name(rt.trace, 2.0, rays, 0) == "RTSDF_E_ARG"
    assert _name(rt.trace, float("nan"), 8, 0) == "RTSDF_E_ARG"
    assert _name(rt.trace, 2.0, 8, -1) == "RTSDF_E_ARG"
    rt.trace(2.0, 1, 0)                                   # the extremes of the ray count are valid
    rt.trace(2.0, 1024, 1)
    pos, nrm = S.floor_gbuffer(8, 8, y=0.05)
    tp, tn = torch.tensor(pos, device=rt.device), torch.tensor(nrm, device=rt.device)
    assert _name(rt.shadow, tp, tn, (0.4, 1.0, 0.3), steps=0) == "RTSDF_E_ARG"
    assert _name(rt.shadow, tp, tn, (0.4, 1.0, 0.3), steps=257) == "RTSDF_E_ARG"
    assert _name(rt.shadow, tp, tn, (0.4, 1.0, 0.3), k=0.0) == "RTSDF_E_ARG"
    assert _name(rt.shadow, tp, tn, (0.0, 0.0, 0.0)) == "RTSDF_E_ARG"
    assert _name(rt.shadow, tp, tn, (0.4, 1.0, 0.3), jitter_vox=-1.0) == "RTSDF_E_ARG"
    img = torch.zeros((8, 8), device=rt.device)
    assert _name(rt.taa_resolve, img, img, 0.1) == "RTSDF_E_ARG"           # cur and hist overlap
    assert _name(rt.taa_resolve, img.clone(), img, 0.0) == "RTSDF_E_ARG"   # blend outside (0, 1]
    assert _name(rt.set_tuning, refill_min=0) == "RTSDF_E_ARG"
    from paper_2210_04449_gb300 import _abi
    assert _abi.lib().rtsdf_set_bvh_builder(rt._h, 7) == 1                 # unknown builder
    assert rt.get_bvh_builder() == "sah"
    assert _name(rt.set_tuning, jfa_tile=9) == "RTSDF_E_ARG"
    state = rt.save_state()
    assert _name(rt.load_state, state[:-1]) == "RTSDF_E_ARG"              # truncated
    other = RTSDF(8)
    assert _name(other.load_state, state) == "RTSDF_E_ARG"                # another grid size
    rt.sync()
    other.close()
    rt.close()


def test_motion_leaving_the_volume_is_reported_and_cleared():
    from paper_2210_04449_gb300 import RTSDF
    m = S.animated_scene(5, n_objects=3, n_lon=12, n_lat=7)
    rt = RTSDF(16)
    rt.upload_mesh(m.verts, m.tris)
    rt.set_objects(m.vert_object, m.n_objects)
    rt.build_bvh()
    rt.update(2.0, 4, 0)
    rt.sync()
    far = np.zeros((3, 3), np.float32)
    far[1] = (10.0, 0.0, 0.0)                             # object 1 leaves the accepted box
    rt.move_objects(far)
    rt.build_bvh(refit=True)
    rt.update(2.0, 4, 1)
    assert _name(rt.sync) == "RTSDF_E_MESH"               # clamped, reported once
    rt.sync()                                             # the status word was cleared
    rt.close()


def test_allocation_failure_returns_oom_and_recovers():
    # host-side fault injection: the context allocator fails the n-th
    # allocation (no device allocation is attempted for it); the call returns
    # RTSDF_E_OOM and frees what it allocated, and everything works again
    from paper_2210_04449_gb300 import RTSDF, _abi
    lib = _abi.lib()
    m = S.tiny_scene()
    ref = _fine_after_frame(RTSDF(16, seed=1), m)
    for after in (0, 3, 12):
        lib.rtsdf_debug_fail_allocation(after)
        assert _name(RTSDF, 16, seed=1) == "RTSDF_E_OOM"
    lib.rtsdf_debug_fail_allocation(-1)
    rt = RTSDF(16, seed=1)
    # fail inside the mesh upload (its vertex / index buffers), then retry
    lib.rtsdf_debug_fail_allocation(0)
    assert _name(rt.upload_mesh, m.verts, m.tris) == "RTSDF_E_OOM"
    lib.rtsdf_debug_fail_allocation(-1)
    assert np.array_equal(_fine_after_frame(rt, m), ref)
    rt.sync()
    rt.close()


def test_cyclic_tree_reports_overflow_and_recovers():
    # the root's children rewritten to name the root (valid node ids closing a
    # cycle): every walk that enters it stops at its step bound or stack
    # limit, the tracer and the exact-occlusion fallback report
    # RTSDF_E_OVERFLOW, and a rebuilt tree plus the saved accumulation give
    # the uninterrupted result bit for bit
    import torch
    from paper_2210_04449_gb300 import RTSDF, _abi
    lib = _abi.lib()
    m = S.tiny_scene()
    ref = RTSDF(16, seed=1)
    ref.upload_mesh(m.verts, m.tris)
    ref.build_bvh()
    for t in range(2):
        ref.update(2.0, 8, t)
    ref.sync()
    want = {k: v.cpu().numpy().copy() for k, v in ref.grids().items() if k in ("accum", "counts", "fine")}
    rt = RTSDF(16, seed=1)
    assert _abi.STATUS_NAMES[lib.rtsdf_debug_bvh_cycle(rt._h)] == "RTSDF_E_STATE"   # no tree yet
    rt.upload_mesh(m.verts, m.tris)
    rt.build_bvh()
    rt.update(2.0, 8, 0)
    rt.sync()
    state = rt.save_state()
    assert _abi.STATUS_NAMES[lib.rtsdf_debug_bvh_cycle(rt._h)] == "RTSDF_OK"
    rt.update(2.0, 8, 1)
    assert _name(rt.sync) == "RTSDF_E_OVERFLOW"
    pos, nrm = S.floor_gbuffer(16, 16, y=0.05)
    dev = torch.device("cuda")
    blocked = torch.zeros(16 * 16, device=dev, dtype=torch.uint8)
    rt.shadow_fallback(torch.tensor(pos, device=dev), torch.tensor(nrm, device=dev), (0.4, 1.0, 0.3), None,
                       blocked=blocked)
    assert _name(rt.sync) == "RTSDF_E_OVERFLOW"
    rt.build_bvh()
    rt.load_state(state)
    rt.update(2.0, 8, 1)
    rt.sync()
    got = rt.grids()
    for k, v in want.items():
        assert np.array_equal(got[k].cpu().numpy(), v), k
    rt.close()
    ref.close()


def test_stream_switch_orders_later_calls():
    # frames alternate between two streams; rtsdf_set_stream waits for the
    # old stream, so the result equals a context that stays on one stream
    import torch
    from paper_2210_04449_gb300 import RTSDF
    m = S.animated_scene(2, n_objects=12, n_lon=16, n_lat=9)
    ref = RTSDF(32, seed=3)
    want = None
    for t in range(3):
        if t == 0:
            ref.upload_mesh(m.verts, m.tris)
            ref.build_bvh()
        ref.update(2.0, 16, t)
    ref.sync()
    want = ref.grids()["fine"].cpu().numpy().copy()
    ref.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    rt = RTSDF(32, seed=3)
    rt.set_stream(streams[0])
    rt.upload_mesh(m.verts, m.tris)
    rt.build_bvh()
    for t in range(3):
        rt.set_stream(streams[t % 2])
        rt.update(2.0, 16, t)
    rt.sync()
    assert np.array_equal(rt.grids()["fine"].cpu().numpy(), want)
    rt.close()
