"""BVH builders on the GPU.  Every topology (binned SAH, Morton, two-level)
must be a binary tree over every triangle, the one-tree builders with the
leaves in position order; the SAH tree must have the lower surface-area
cost; the build must be deterministic; a two-level tree must stay valid and
close to a fresh SAH tree in cost as its objects move; and the traced SDF
must not depend on the builder (every ray keeps its closest hit, equal
distances the smaller triangle index), so all builders give bit-identical
grids."""
import numpy as np
import pytest

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _identical_tris(n):
    v = np.array([[0.3, 0.4, 0.5], [0.35, 0.4, 0.5], [0.3, 0.45, 0.52]], np.float32)
    return S.Mesh(v, np.zeros((n, 3), np.int32))


def _flat_soup(seed, n):
    m = S.random_soup(seed, n)
    v = m.verts.copy()
    v[:, 2] = 0.5                                         # every triangle in one plane
    return S.Mesh(v, m.tris)


SCENES = {
    "two": lambda: S.random_soup(1, 2),
    "three": lambda: S.random_soup(2, 3),
    "33": lambda: S.random_soup(3, 33),
    "1025": lambda: S.random_soup(4, 1025),
    "5000": lambda: S.random_soup(5, 5000),
    "animated": lambda: S.animated_scene(6, n_objects=12, n_lon=24, n_lat=13),
    "identical": lambda: _identical_tris(3000),
    "flat": lambda: _flat_soup(7, 2500),
}


def _build(mesh, builder, nc=16):
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(nc)
    rt.set_bvh_builder(builder)
    assert rt.get_bvh_builder() == builder
    rt.upload_mesh(mesh.verts, mesh.tris)
    if mesh.vert_object is not None:
        rt.set_objects(mesh.vert_object, mesh.n_objects)
    rt.build_bvh()
    return rt


def _check_tree(ch, lt, root, nt, in_order=True):
    """Every node and leaf reached once from the root; leaf_tri is a
    permutation of the triangles; with in_order, the in-order leaves are
    positions 0..nt-1 (the one-tree builders; a two-level tree orders its
    objects by the top tree)."""
    assert np.array_equal(np.sort(lt), np.arange(nt))
    if nt < 2:
        assert root == -1
        return
    seen = np.zeros(nt - 1, bool)
    order = []
    stack = [root]
    while stack:
        x = stack.pop()
        if x < 0:
            order.append(~x)
            continue
        assert 0 <= x < nt - 1 and not seen[x]
        seen[x] = True
        stack.append(int(ch[x, 1]))                        # right after left: left pops first
        stack.append(int(ch[x, 0]))
    assert seen.all()
    assert sorted(order) == list(range(nt))
    if in_order:
        assert order == list(range(nt))


def _sah_cost(ch, lt, root, mesh):
    """Sum over internal nodes of area(node) / area(root) (leaves: one
    triangle each, the same for every tree)."""
    tv = mesh.verts[mesh.tris].astype(np.float64)         # [nt, 3, 3]
    lo_t, hi_t = tv.min(axis=1), tv.max(axis=1)
    nt = len(lt)
    lo = np.zeros((nt - 1, 3))
    hi = np.zeros((nt - 1, 3))
    post = []
    stack = [(root, False)]
    while stack:
        x, done = stack.pop()
        if done:
            post.append(x)
            continue
        stack.append((x, True))
        for c in ch[x]:
            if c >= 0:
                stack.append((int(c), False))
    for x in post:
        bl, bh = [], []
        for c in ch[x]:
            if c >= 0:
                bl.append(lo[c])
                bh.append(hi[c])
            else:
                t = lt[~c]
                bl.append(lo_t[t])
                bh.append(hi_t[t])
        lo[x] = np.minimum(*bl)
        hi[x] = np.maximum(*bh)
    d = hi - lo
    area = d[:, 0] * d[:, 1] + d[:, 1] * d[:, 2] + d[:, 2] * d[:, 0]
    return float(area.sum() / area[root])


@pytest.mark.parametrize("builder", ["sah", "lbvh", "two_level"])
@pytest.mark.parametrize("scene", list(SCENES))
def test_topology_is_a_tree_over_every_triangle(builder, scene):
    mesh = SCENES[scene]()
    rt = _build(mesh, builder)
    ch, lt, root = rt.bvh_topology()
    _check_tree(ch, lt, root, mesh.tris.shape[0], in_order=builder != "two_level")
    st = rt.stats()
    assert 1 <= st["bvh_depth"] <= mesh.tris.shape[0]
    rt.sync()
    rt.close()


@pytest.mark.parametrize("scene", ["5000", "animated", "flat"])
def test_sah_tree_has_lower_cost(scene):
    mesh = SCENES[scene]()
    costs = {}
    for b in ("sah", "lbvh"):
        rt = _build(mesh, b)
        costs[b] = _sah_cost(*rt.bvh_topology(), mesh)
        rt.close()
    assert costs["sah"] < costs["lbvh"]


def test_sah_build_is_deterministic():
    mesh = SCENES["animated"]()
    rt = _build(mesh, "sah")
    a = rt.bvh_topology()
    rt.build_bvh()
    b = rt.bvh_topology()
    other = _build(mesh, "sah")
    c = other.bvh_topology()
    for x, y in ((a, b), (a, c)):
        assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1]) and x[2] == y[2]
    rt.close()
    other.close()


def test_identical_triangles_stay_shallow():
    # no split separates equal centroids: ranges split at the middle
    mesh = SCENES["identical"]()
    rt = _build(mesh, "sah")
    assert rt.stats()["bvh_depth"] <= 16
    rt.close()


def test_two_level_falls_back_to_one_sah_tree():
    # 1025 one-triangle objects: more than one top-tree block holds, so the
    # build makes the single SAH tree (leaves in position order)
    mesh = SCENES["1025"]()
    rt = _build(mesh, "two_level")
    ch, lt, root = rt.bvh_topology()
    _check_tree(ch, lt, root, mesh.tris.shape[0], in_order=True)
    ref = _build(mesh, "sah")
    want = ref.bvh_topology()
    assert np.array_equal(ch, want[0]) and np.array_equal(lt, want[1]) and root == want[2]
    rt.close()
    ref.close()


def _objects_scene():
    # 40 spheres, one more object that is a single triangle, one without triangles
    m = S.animated_scene(9, n_objects=40, n_lon=16, n_lat=9)
    nv = m.verts.shape[0]
    extra = np.array([[0.5, 0.5, 0.5], [0.52, 0.5, 0.5], [0.5, 0.53, 0.5]], np.float32)
    verts = np.concatenate([m.verts, extra])
    tris = np.concatenate([m.tris, np.array([[nv, nv + 1, nv + 2]], np.int32)])
    vo = np.concatenate([m.vert_object, np.full(3, m.n_objects, np.int32)])
    return S.Mesh(verts, tris, vo, m.n_objects + 2)


def test_two_level_refit_keeps_a_valid_tree_of_sah_quality():
    mesh = _objects_scene()
    rt = _build(mesh, "two_level", nc=24)
    nt = mesh.tris.shape[0]
    verts = mesh.verts.copy()
    for t in range(1, 6):
        tr = S.object_translations(10, t, mesh.n_objects, 0.02).astype(np.float32)
        rt.move_objects(tr)
        rt.build_bvh(refit=True)
        ch, lt, root = rt.bvh_topology()
        _check_tree(ch, lt, root, nt, in_order=False)
        verts = verts + tr[mesh.vert_object]             # the library's per-frame fp32 move
        moved = S.Mesh(verts, mesh.tris, mesh.vert_object, mesh.n_objects)
        two = _sah_cost(ch, lt, root, moved)
        ref = _build(moved, "sah", nc=24)
        fresh = _sah_cost(*ref.bvh_topology(), moved)
        ref.close()
        assert two <= 1.15 * fresh
    rt.close()


@pytest.mark.parametrize("refit", [False, True])
def test_traced_sdf_does_not_depend_on_the_builder(refit):
    from paper_2210_04449_gb300 import RTSDF
    mesh = S.animated_scene(8, n_objects=6, n_lon=20, n_lat=11)
    out = {}
    for b in ("sah", "lbvh", "two_level"):
        rt = RTSDF(24, seed=5)
        rt.set_bvh_builder(b)
        rt.upload_mesh(mesh.verts, mesh.tris)
        rt.set_objects(mesh.vert_object, mesh.n_objects)
        rt.build_bvh()
        for t in range(3):
            if t > 0:
                rt.move_objects(S.object_translations(8, t, mesh.n_objects, 0.5 / 24))
                rt.build_bvh(refit=refit)
            rt.update(2.0, 16, t)
        rt.sync()
        g = rt.grids()
        out[b] = {k: g[k].cpu().numpy().copy() for k in ("fine", "accum", "counts")}
        rt.close()
    for k in ("fine", "accum", "counts"):
        assert np.array_equal(out["sah"][k], out["lbvh"][k]), k
        assert np.array_equal(out["sah"][k], out["two_level"][k]), k


def test_full_size_sah_tree():
    # the benchmark scene: the SAH tree is a tree over all 1,000,000
    # triangles with the leaves in position order, and cheaper than the
    # Morton tree by the surface-area cost
    mesh = S.animated_scene(2, n_objects=500)
    costs = {}
    for b in ("sah", "lbvh"):
        rt = _build(mesh, b, nc=64)
        ch, lt, root = rt.bvh_topology()
        if b == "sah":
            _check_tree(ch, lt, root, mesh.tris.shape[0])
        costs[b] = _sah_cost(ch, lt, root, mesh)
        rt.close()
    assert costs["sah"] < 0.95 * costs["lbvh"]

