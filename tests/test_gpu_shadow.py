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
