"""Launch tuning changes speed only: every jump-flood tile and tracer setting
gives bit-identical grids, and the autotuners leave the accumulated SDF as
they found it (they save and restore the temporal state)."""
import numpy as np
import pytest

from synth import scenes as S

pytestmark = pytest.mark.gpu

KEYS = ("seeds", "coarse", "accum", "counts", "fine")


def _snap(rt):
    g = rt.grids()
    return {k: g[k].cpu().numpy().copy() for k in KEYS}


def _ctx(mesh, nc=48, seed=4):
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(nc, beta_vox=0.5, seed=seed)
    rt.upload_mesh(mesh.verts, mesh.tris)
    rt.build_bvh()
    return rt


@pytest.mark.parametrize("tuning", [dict(jfa_tile=1), dict(jfa_tile=2), dict(jfa_tile=3), dict(jfa_tile=4),
                                    dict(refill_min=1, ray_chunk=32), dict(refill_min=16, ray_chunk=4096),
                                    dict(trace_blocks_per_sm=2)])
def test_tuning_does_not_change_results(tuning):
    mesh = S.room_scene(3, n_objects=30, n_spheres=10, subdiv=2)
    ref = _ctx(mesh)
    alt = _ctx(mesh)
    alt.set_tuning(**tuning)
    for f in range(2):
        ref.update(2.0, 16, f)
        alt.update(2.0, 16, f)
    ref.sync()
    alt.sync()
    a, b = _snap(ref), _snap(alt)
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


def test_autotune_keeps_state_and_results():
    mesh = S.room_scene(3, n_objects=30, n_spheres=10, subdiv=2)
    ref = _ctx(mesh)
    tuned = _ctx(mesh)
    for f in range(2):
        ref.update(2.0, 16, f)
        tuned.update(2.0, 16, f)
    tuned.sync()
    before = _snap(tuned)
    best = tuned.autotune(2.0, 16, 2, use_cache=False)
    assert 0 <= best["jfa_tile"] <= 4 and best["refill_min"] >= 1 and best["ray_chunk"] >= 32
    after = _snap(tuned)
    for k in ("accum", "counts", "fine"):
        assert np.array_equal(before[k], after[k]), k
    assert tuned.autotune(2.0, 16, 2, use_cache=True) == best       # cached
    for f in (2, 3):
        ref.update(2.0, 16, f)
        tuned.update(2.0, 16, f)
    ref.sync()
    tuned.sync()
    a, b = _snap(ref), _snap(tuned)
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


def test_batch_autotune_keeps_state():
    from paper_2210_04449_gb300 import RTSDFBatch
    meshes = [S.tiny_scene(), S.random_soup(2, 300, size=0.05), S.room_scene(5, n_objects=10, n_spheres=4, subdiv=2)]
    cfgs = [dict(coarse_n=n, beta_vox=0.5, seed=i) for i, n in enumerate((16, 40, 64))]
    b = RTSDFBatch(cfgs)
    for sc, m in zip(b.scenes, meshes):
        sc.upload_mesh(m.verts, m.tris)
        sc.build_bvh()
    b.frame(2.0, 8, 0)
    b.sync()
    before = [_snap(sc) for sc in b.scenes]
    best = b.autotune(2.0, 8, 1, use_cache=False)
    assert best["refill_min"] >= 1 and best["ray_chunk"] >= 32
    for sc, snap in zip(b.scenes, before):
        after = _snap(sc)
        for k in ("accum", "counts", "fine"):
            assert np.array_equal(snap[k], after[k]), k
    b.close()
