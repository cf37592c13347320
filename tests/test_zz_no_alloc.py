"""rtsdf_jfa_noalloc: the jump flood for callers that cannot allocate device
memory (their host owns the memory budget or bans allocation in its frame
loop).  Called through the C ABI on caller-owned buffers, it must reproduce
rtsdf_jfa -- seeds bit-exact, coarse SDF within 1e-6 -- on two calls in a row
(the second call finds the first call's data in the shared scratch array).
This file runs last so that a failure here leaves every other test run."""
import ctypes

import numpy as np
import pytest

from synth import scenes as S

pytestmark = pytest.mark.gpu


def _reference(mesh, nc, beta):
    """Voxelized input grid and rtsdf_jfa's output for it."""
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(nc, beta_vox=beta)
    rt.upload_mesh(mesh.verts, mesh.tris)
    rt.voxelize()
    occ = rt.grids()["seeds"].clone()
    rt.jfa()
    g = rt.grids()
    seeds, coarse = g["seeds"].clone(), g["coarse"].clone()
    rt.sync()
    rt.close()
    return occ, seeds, coarse


def _noalloc(occ, nc, beta):
    import torch
    from paper_2210_04449_gb300 import _abi
    out_s = torch.full_like(occ, 7)
    out_c = torch.full((nc ** 3,), -5.0, device=occ.device)
    stream = torch.cuda.current_stream(occ.device).cuda_stream
    rc = _abi.lib().rtsdf_jfa_noalloc(occ.data_ptr(), out_s.data_ptr(), out_c.data_ptr(), nc, 1.0, beta, stream)
    assert rc == 0, _abi.STATUS_NAMES.get(rc)
    torch.cuda.synchronize(occ.device)
    return out_s, out_c


def test_noalloc_matches_rtsdf_jfa_on_two_calls():
    # pass counts 7 (odd, last pass reads the scratch array), 6 (even), 5,
    # 1 (a single pass straight into seeds_out), 2, and 0 (n = 1: copy and
    # coarse SDF only)
    cases = [(S.room_scene(1, n_objects=40), 128, 0.5), (S.tiny_scene(), 48, 0.25),
             (S.tiny_scene(), 32, 0.5), (S.tiny_scene(), 2, 0.5), (S.tiny_scene(), 3, 0.5),
             (S.tiny_scene(), 1, 0.5)]
    for mesh, nc, beta in cases:
        occ, seeds, coarse = _reference(mesh, nc, beta)
        out_s, out_c = _noalloc(occ, nc, beta)
        assert np.array_equal(out_s.cpu().numpy(), seeds.cpu().numpy())
        c_ref, c_new = coarse.cpu().numpy().astype(np.float64), out_c.cpu().numpy().astype(np.float64)
        fin = np.isfinite(c_ref)
        assert np.array_equal(fin, np.isfinite(c_new))
        assert np.max(np.abs(c_new[fin] - c_ref[fin])) <= 1e-6


def test_noalloc_rejects_oversize_and_aliasing():
    import torch
    from paper_2210_04449_gb300 import _abi
    lib = _abi.lib()
    buf = torch.zeros(3 * 8 ** 3, dtype=torch.int32, device="cuda")
    p = buf.data_ptr()
    # n beyond the scratch array's 128^3 capacity
    big = torch.zeros(2, dtype=torch.int32, device="cuda")
    assert lib.rtsdf_jfa_noalloc(big.data_ptr(), big.data_ptr() + 4, big.data_ptr(), 129, 1.0, 0.5, None) == 1
    # overlapping input and output
    assert lib.rtsdf_jfa_noalloc(p, p + 4, p + 2 * 4 * 8 ** 3, 8, 1.0, 0.5, None) == 1
    assert lib.rtsdf_jfa_noalloc(p, p + 4 * 8 ** 3, p + 2 * 4 * 8 ** 3, 8, 1.0, 0.5, None) == 0
    torch.cuda.synchronize()
