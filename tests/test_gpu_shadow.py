"""GPU parity of Sec. 2.3 (soft-shadow march) and of its adjoint.

Forward: fp32 kernel vs the fp64 oracle on the same synthetic fine grid.
Points where a discrete decision of the march (h < eps, leaving the cube,
which step sets the minimum) differs between fp32 and fp64 are counted; all
others agree to |dvis| <= 1e-4 (fp32 rounding amplified by at most ~1e3 in
k dd / (t - y) near the first steps).  The flip count must stay below 1 %.
Backward: dLoss/dsdf and dLoss/dlight against the oracle's fp64 derivative
on points whose march path is identical, relative error <= 1e-3 of the
largest entry; plus torch autograd through ShadowFn.
"""
import numpy as np
import pytest

import oracle
from synth import scenes as S

pytestmark = pytest.mark.gpu

BMIN = np.zeros(3)


def _grid(nf):
    g = np.minimum(S.sphere_grid_sdf(nf, (0.5, 0.35, 0.5), 0.12),
                   S.box_grid_sdf(nf, (0.3, 0.3, 0.65), 0.06))
    c = (np.arange(nf) + 0.5) / nf
    floor = (c[None, :, None] - 0.1) * np.ones((nf, nf, nf))
    return np.minimum(g, floor).astype(np.float32)


def _setup(nf, w, k):
    import torch
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(nf // 2)
    grid = _grid(nf)
    pos, nrm = S.floor_gbuffer(w, w, y=0.1, lo=0.05, hi=0.95)
    dev = rt.device
    return rt, grid, pos, nrm, torch.tensor(grid.reshape(-1), device=dev), torch.tensor(pos, device=dev), \
        torch.tensor(nrm, device=dev)


@pytest.mark.parametrize("nf,k,steps,smax", [(64, 8.0, 64, 4.0), (128, 2.0, 64, 4.0), (64, 4.0, 16, 1.0),
                                             (128, 8.0, 256, 8.0)])
def test_shadow_forward(nf, k, steps, smax):
    rt, grid, pos, nrm, tg, tp, tn = _setup(nf, 96, k)
    L = (0.4, 1.0, 0.3)
    h = 1.0 / nf
    vis_g = rt.shadow(tp, tn, L, k=k, steps=steps, step_max_vox=smax, eps_vox=1.0, sdf=tg).cpu().numpy().ravel()
    vis_o, info = oracle.shadow(grid, nf, BMIN, 1.0, pos, nrm, L, k, steps, smax * h, h, info=True)
    d = np.abs(vis_g - vis_o)
    flips = d > 1e-4
    print(f"nf={nf} k={k}: max|d|={d.max():.2e} flips={flips.sum()}/{d.size} "
          f"shadowed={np.mean(vis_o < 1):.2f}")
    assert flips.mean() < 0.01
    assert np.median(d) < 1e-6


def test_shadow_lit_and_umbra_cases():
    import torch
    from paper_2210_04449_gb300 import RTSDF
    nf = 64
    rt = RTSDF(nf // 2)
    grid = S.box_grid_sdf(nf, (0.5, 0.5, 0.5), 0.25, floor_y=0.1)
    tg = torch.tensor(grid.reshape(-1), device=rt.device)
    pos, nrm = S.floor_gbuffer(16, 16, y=0.1, lo=0.4, hi=0.6)
    v = rt.shadow(torch.tensor(pos, device=rt.device), torch.tensor(nrm, device=rt.device), (0, 1, 0), sdf=tg)
    assert torch.all(v == 0)
    pos, nrm = S.floor_gbuffer(16, 16, y=0.1, lo=0.0, hi=0.1)     # >= 0.15 from the box
    v = rt.shadow(torch.tensor(pos, device=rt.device), torch.tensor(nrm, device=rt.device), (0, 1, 0), sdf=tg)
    assert torch.all(v == 1)
    # no shading points
    e = torch.zeros((0, 3), device=rt.device)
    assert rt.shadow(e, e, (0, 1, 0), sdf=tg).numel() == 0


@pytest.mark.parametrize("nf,k", [(64, 2.0), (128, 2.0)])
def test_shadow_backward_against_oracle(nf, k):
    import torch
    rt, grid, pos, nrm, tg, tp, tn = _setup(nf, 64, k)
    L = np.array([0.4, 1.0, 0.3])
    h = 1.0 / nf
    cfg = dict(k=k, steps=64, step_max=4 * h, eps=h)
    vis_o, info = oracle.shadow(grid, nf, BMIN, 1.0, pos, nrm, L, info=True, **cfg)
    vis_g = rt.shadow(tp, tn, L, k=k, steps=64, step_max_vox=4.0, eps_vox=1.0, sdf=tg).cpu().numpy().ravel()
    same = np.abs(vis_g - vis_o) <= 1e-5        # identical discrete path
    w = np.random.default_rng(0).normal(size=vis_o.size) * same
    gs_o, gl_o = oracle.shadow_grad(grid, nf, BMIN, 1.0, pos, nrm, L, dvis=w, **cfg)
    dsdf = torch.zeros(nf ** 3, device=rt.device)
    dl = torch.zeros(3, device=rt.device)
    rt.shadow_backward(tp, tn, L, torch.tensor(w, dtype=torch.float32, device=rt.device), dsdf, dl, k=k,
                       steps=64, step_max_vox=4.0, eps_vox=1.0, sdf=tg)
    gs_g = dsdf.cpu().numpy().astype(np.float64)
    gl_g = dl.cpu().numpy().astype(np.float64)
    scale = np.max(np.abs(gs_o))
    assert scale > 0
    err = np.max(np.abs(gs_g - gs_o)) / scale
    lerr = np.max(np.abs(gl_g - gl_o)) / np.max(np.abs(gl_o))
    print(f"nf={nf}: grid rel err {err:.2e}, light rel err {lerr:.2e}")
    assert err <= 1e-3
    assert lerr <= 1e-3


def test_autograd_shadow_fn():
    import torch
    from paper_2210_04449_gb300 import soft_shadow
    nf = 64
    rt, grid, pos, nrm, tg, tp, tn = _setup(nf, 48, 2.0)
    sdf = tg.clone().requires_grad_(True)
    light = torch.tensor([0.4, 1.0, 0.3], dtype=torch.float64, requires_grad=True)
    target = soft_shadow(rt, tg, torch.tensor([0.5, 1.0, 0.2]), tp, tn, k=2.0).detach()
    vis = soft_shadow(rt, sdf, light, tp, tn, k=2.0)
    loss = ((vis - target) ** 2).mean()
    loss.backward()
    assert sdf.grad is not None and light.grad is not None
    assert torch.isfinite(sdf.grad).all() and torch.isfinite(light.grad).all()
    # against the oracle derivative of the same loss
    h = 1.0 / nf
    dvis = (2 * (vis - target) / vis.numel()).detach().cpu().numpy().astype(np.float64)
    gs_o, gl_o = oracle.shadow_grad(grid, nf, BMIN, 1.0, pos, nrm, light.detach().numpy(), k=2.0, steps=64,
                                    step_max=4 * h, eps=h, dvis=dvis)
    assert np.max(np.abs(sdf.grad.cpu().numpy() - gs_o)) <= 2e-3 * np.max(np.abs(gs_o)) + 1e-12


# --------------------------------------------------------------------------
# Sec. 2.3's jittered ray origin and the TAA resolve
# --------------------------------------------------------------------------

def _jitter_setup(nf, w, seed):
    import torch
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(nf // 2, seed=seed)
    grid = _grid(nf)
    pos, nrm = S.floor_gbuffer(w, w, y=0.1, lo=0.05, hi=0.95)
    dev = rt.device
    return rt, grid, pos, nrm, torch.tensor(grid.reshape(-1), device=dev), torch.tensor(pos, device=dev), \
        torch.tensor(nrm, device=dev)


def test_jitter_zero_is_the_plain_march():
    from paper_2210_04449_gb300.context import call
    rt, grid, pos, nrm, tg, tp, tn = _jitter_setup(64, 64, 3)
    L = (0.4, 1.0, 0.3)
    plain = rt.shadow(tp, tn, L, sdf=tg)
    jit0 = plain.clone().fill_(-1.0)
    call("rtsdf_shadow_jittered", rt._h, tg.data_ptr(), tp.data_ptr(), tn.data_ptr(), tp.numel() // 3,
         rt._light3(L), 8.0, 64, 4.0, 1.0, 0.0, 7, jit0.data_ptr())
    assert np.array_equal(plain.cpu().numpy(), jit0.cpu().numpy())


@pytest.mark.parametrize("nf,jit,frame,seed", [(64, 2.0, 0, 1), (128, 4.0, 5, 2), (64, 0.5, 1 << 20, 3)])
def test_jittered_shadow_matches_oracle(nf, jit, frame, seed):
    rt, grid, pos, nrm, tg, tp, tn = _jitter_setup(nf, 96, seed)
    L = (0.4, 1.0, 0.3)
    h = 1.0 / nf
    vis_g = rt.shadow(tp, tn, L, sdf=tg, jitter_vox=jit, frame=frame).cpu().numpy().ravel()
    shift = oracle.shadow_jitter(seed, frame, pos.reshape(-1, 3).shape[0]) * jit * h
    vis_o = oracle.shadow(grid, nf, BMIN, 1.0, pos, nrm, L, 8.0, 64, 4 * h, h, shift=shift)
    plain_o = oracle.shadow(grid, nf, BMIN, 1.0, pos, nrm, L, 8.0, 64, 4 * h, h)
    d = np.abs(vis_g - vis_o)
    flips = d > 1e-4
    print(f"jitter nf={nf} jit={jit}: max|d|={d.max():.2e} flips={flips.sum()}/{d.size} "
          f"changed-by-jitter={np.mean(np.abs(vis_o - plain_o) > 1e-3):.2f}")
    assert flips.mean() < 0.01
    assert np.median(d) < 1e-6
    assert np.mean(np.abs(vis_o - plain_o) > 1e-3) > 0.01     # the jitter did move the march


@pytest.mark.parametrize("H,W", [(1, 1), (3, 5), (23, 37), (1080, 1920)])
@pytest.mark.parametrize("blend", [0.1, 1.0])
def test_taa_resolve_matches_oracle(H, W, blend):
    import torch
    from paper_2210_04449_gb300 import RTSDF
    rt = RTSDF(8)
    rng = np.random.default_rng(H * 7 + W)
    cur = rng.random((H, W)).astype(np.float32)
    hist = rng.uniform(-0.5, 1.5, (H, W)).astype(np.float32)
    tc = torch.tensor(cur, device=rt.device)
    th = torch.tensor(hist, device=rt.device)
    rt.taa_resolve(tc, th, blend)
    want = oracle.taa_resolve(cur, hist, blend)
    assert np.max(np.abs(th.cpu().numpy() - want)) <= 1e-6


def test_jittered_shadows_with_taa_over_frames():
    import torch
    nf, w, seed, jit = 64, 96, 4, 2.0
    rt, grid, pos, nrm, tg, tp, tn = _jitter_setup(nf, w, seed)
    L = (0.4, 1.0, 0.3)
    h = 1.0 / nf
    hist_g = torch.zeros((w, w), device=rt.device)
    hist_o = np.zeros((w, w))
    for f in range(6):
        vg = rt.shadow(tp, tn, L, sdf=tg, jitter_vox=jit, frame=f).reshape(w, w)
        rt.taa_resolve(vg, hist_g, 1.0 if f == 0 else 0.2)
        shift = oracle.shadow_jitter(seed, f, pos.reshape(-1, 3).shape[0]) * jit * h
        vo = oracle.shadow(grid, nf, BMIN, 1.0, pos, nrm, L, 8.0, 64, 4 * h, h, shift=shift).reshape(w, w)
        hist_o = oracle.taa_resolve(vo, hist_o, 1.0 if f == 0 else 0.2)
    d = np.abs(hist_g.cpu().numpy() - hist_o)
    print(f"6 jittered frames + TAA: max|d|={d.max():.2e} frac>1e-4={np.mean(d > 1e-4):.4f}")
    assert np.median(d) < 1e-6
    assert np.mean(d > 1e-4) < 0.03      # march branch flips, spread by the 3x3 clamp
