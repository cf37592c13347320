"""Sec. 2.3 at the sizes the benchmark times, on a fine SDF that the pipeline
itself traced (not an analytic grid).

Workload: the procedural room (~100k triangles) at coarse 256^3 -> fine
512^3 (the differentiable-shadow workload: the room scene's geometry at a
512^3 fine grid), one frame of 1 ray per texel.  Both sides trace their own
fine SDF: the GPU through the library, the oracle through its own Sec. 2.1
pipeline and its hierarchy trace (bit-identical to brute force) -- the
oracle never reads a GPU grid.

* The fine grids themselves: every one of the ~41M masked texels compared
  (distances, counts, signed values), and the fill of every unmasked texel.
* Forward march (Sec. 2.3) at 1920 x 1080 floor points, L = (0.4, 1, 0.3),
  k = 8, 64 steps: 65,536 sampled points against the fp64 oracle march;
  median |dvis| and the rate of branch flips (|dvis| > 1e-4).
* Adjoint at 1024 x 1024 floor points, loss = mean (vis - target)^2 with the
  target rendered with the light rotated 5 degrees about the horizontal
  axis perpendicular to it.  The loss is taken over the points whose march
  the oracle finds stable (every discrete decision at a relative gap above
  1e-4, and a visibility that moves by at most 1e-5 when the grid, the
  shading positions and the light are perturbed at about ten times fp32
  rounding; the count is printed), so that fp32 and fp64 agree on them:
  dLoss/dsdf on >= 1000 texels with |g| >= 1e-6 and dLoss/dlight against
  the oracle's fp64 reverse sweep, relative error <= 1e-3 per entry; and
  the oracle gradient against fp64 central finite differences (h = 1e-4)
  to 1e-3 relative, kinks excluded and counted.
"""
import math

import numpy as np
import pytest

import oracle
from synth import scenes as S

pytestmark = pytest.mark.gpu

BMIN = np.zeros(3, np.float32)
NC, NF, D, BETA, RAYS, SEED = 256, 512, 2.0, 0.5, 1, 1
HF = 1.0 / NF
K, STEPS, SMAX_VOX, EPS_VOX = 8.0, 64, 4.0, 1.0
L0 = np.array([0.4, 1.0, 0.3]) / np.linalg.norm([0.4, 1.0, 0.3])
TOL = 2e-5 * math.sqrt(3.0)

_ROOM = {}


def _room512():
    """(GPU context with its traced 512^3 fine SDF, the oracle's fine SDF
    fp32 [NF^3], the oracle pipeline over the masked texels, those texels,
    the oracle's fill of the unmasked texels), built once per process."""
    if _ROOM:
        return _ROOM
    from paper_2210_04449_gb300 import RTSDF
    m = S.room_scene(1)
    occ = oracle.voxelize(m.verts, m.tris, BMIN, 1.0, NC)
    seeds, _ = oracle.jfa(occ, NC)
    c = oracle.coarse_sdf(seeds, NC, 1.0, BETA)
    mask, fill = oracle.mask_fill(seeds, NC, D, BETA, c)
    tex = np.nonzero(mask)[0]
    pipe = oracle.FinePipeline(BMIN, 1.0, NC, BETA, D, 1.0, SEED, track=tex, accel="bvh")
    pipe.frame(m.verts, m.tris, 0, RAYS)
    f_o = fill
    f_o[tex] = pipe.f
    f_o = f_o.astype(np.float32)
    rt = RTSDF(NC, beta_vox=BETA, seed=SEED)
    rt.upload_mesh(m.verts, m.tris)
    rt.build_bvh()
    rt.update(D, RAYS, 0)
    rt.sync()
    _ROOM.update(rt=rt, f_o=f_o, pipe=pipe, tex=tex, mask=mask)
    return _ROOM


def _gbuffer(w, h):
    import torch
    pos, nrm = S.floor_gbuffer(w, h, y=0.02)
    pos, nrm = pos.reshape(-1, 3), nrm.reshape(-1, 3)
    return pos, nrm, torch.tensor(pos, device="cuda"), torch.tensor(nrm, device="cuda")


def test_room_512_fine_grid_every_texel():
    r = _room512()
    rt, pipe, tex, mask = r["rt"], r["pipe"], r["tex"], r["mask"]
    g = rt.grids()
    assert rt.masked_count() * 8 == tex.size
    u = g["accum"].cpu().numpy()
    cnt = g["counts"].cpu().numpy().astype(np.int64)
    f = g["fine"].cpu().numpy()
    ug, fg = u[tex].astype(np.float64), f[tex].astype(np.float64)
    both_inf = np.isinf(ug) & np.isinf(pipe.u)
    with np.errstate(invalid="ignore"):
        du = np.where(both_inf, 0.0, np.abs(ug - pipe.u))
    bad = ((du > TOL) | ((cnt[tex] & 0xFFFF) != pipe.nF) | ((cnt[tex] >> 16) != pipe.nB)
           | (np.abs(fg - pipe.f) > TOL))
    exact = np.mean((ug == pipe.u) | both_inf)
    print(f"room 512^3: masked texels={tex.size} mismatched={int(bad.sum())} ({bad.mean():.2e}) "
          f"u-exact={exact:.7f} hit={np.isfinite(pipe.u).mean():.3f}")
    assert bad.mean() <= 1e-4
    um = ~mask
    fo = r["f_o"][um].astype(np.float64)
    fu = f[um].astype(np.float64)
    fin = np.isfinite(fo)
    assert np.array_equal(fin, np.isfinite(fu))
    assert np.max(np.abs(fu[fin] - fo[fin])) <= 1e-6


def test_shadow_1080p_on_traced_sdf():
    r = _room512()
    rt, f_o = r["rt"], r["f_o"]
    pos, nrm, tp, tn = _gbuffer(1920, 1080)
    vis_g = rt.shadow(tp, tn, L0, k=K, steps=STEPS, step_max_vox=SMAX_VOX, eps_vox=EPS_VOX).cpu().numpy().ravel()
    idx = np.sort(np.random.default_rng(21).choice(pos.shape[0], 65_536, replace=False))
    vis_o = oracle.shadow(f_o, NF, BMIN, 1.0, pos[idx], nrm[idx], L0, K, STEPS, SMAX_VOX * HF, EPS_VOX * HF)
    d = np.abs(vis_g[idx] - vis_o)
    flips = d > 1e-4
    print(f"1080p march on the traced 512^3 SDF: median|d|={np.median(d):.2e} max|d|={d.max():.2e} "
          f"flips={int(flips.sum())}/{d.size} shadowed={np.mean(vis_o < 1):.3f} umbra={np.mean(vis_o == 0):.3f}")
    assert np.mean(vis_o < 1) > 0.05          # the room's objects do cast shadows on the floor
    assert flips.mean() < 0.01
    assert np.median(d) < 1e-6


def _rotate(v, axis, deg):
    a = math.radians(deg)
    k = axis / np.linalg.norm(axis)
    return v * math.cos(a) + np.cross(k, v) * math.sin(a) + k * np.dot(k, v) * (1 - math.cos(a))


def test_config5_adjoint_against_oracle_and_finite_differences():
    import torch
    r = _room512()
    rt, f_o = r["rt"], r["f_o"]
    pos, nrm, tp, tn = _gbuffer(1024, 1024)
    P = pos.shape[0]
    axis = np.array([L0[2], 0.0, -L0[0]])                 # horizontal, perpendicular to L0
    L1 = _rotate(L0, axis, 5.0)
    cfg = dict(k=K, steps=STEPS, step_max=SMAX_VOX * HF, eps=EPS_VOX * HF)
    vis_o = oracle.shadow(f_o, NF, BMIN, 1.0, pos, nrm, L0, **cfg)
    tgt_o = oracle.shadow(f_o, NF, BMIN, 1.0, pos, nrm, L1, **cfg)
    loss_o = np.mean((vis_o - tgt_o) ** 2)
    # points whose march keeps every discrete decision at a relative gap
    # above 1e-4 (the oracle's own criterion) take the same path in fp32;
    # the adjoint is compared on the loss over those points
    stable = oracle.shadow_margin(f_o, NF, BMIN, 1.0, pos, nrm, L0, **cfg) > 1e-4
    # ... and whose visibility does not amplify rounding: near t = y the
    # penumbra ratio k dd / (t - y) magnifies the rounding of the marched
    # distance t even on an unchanged path, so each point is marched again
    # on grids, shading positions and light directions perturbed at about
    # ten times fp32 rounding (relative 1e-6 on the grid, 1e-6 on the
    # positions and on the light vector); points whose visibility moves by
    # more than 1e-5 in any of three draws are left out
    rng_s = np.random.default_rng(9)
    for _ in range(3):
        fp = (f_o * (1.0 + rng_s.normal(0.0, 1e-6, f_o.shape).astype(np.float32))).astype(np.float32)
        pp = (pos + rng_s.normal(0.0, 1e-6, pos.shape)).astype(np.float32)
        lp = L0 + rng_s.normal(0.0, 1e-6, 3)
        stable &= np.abs(oracle.shadow(fp, NF, BMIN, 1.0, pp, nrm, lp, **cfg) - vis_o) <= 1e-5
        del fp
    dvis = 2.0 * (vis_o - tgt_o) / P * stable
    g_o, gl_o = oracle.shadow_grad(f_o, NF, BMIN, 1.0, pos, nrm, L0, dvis=dvis, **cfg)

    kw = dict(k=K, steps=STEPS, step_max_vox=SMAX_VOX, eps_vox=EPS_VOX)
    vis_g = rt.shadow(tp, tn, L0, **kw)
    tgt_g = rt.shadow(tp, tn, L1, **kw)
    loss_g = float(((vis_g - tgt_g) ** 2).mean())
    dsdf = torch.zeros(NF ** 3, device="cuda")
    dl = torch.zeros(3, device="cuda")
    rt.shadow_backward(tp, tn, L0, torch.tensor(dvis, dtype=torch.float32, device="cuda"), dsdf, dl, **kw)
    g_g = dsdf.cpu().numpy()
    gl_g = dl.cpu().numpy().astype(np.float64)
    vis_g = vis_g.cpu().numpy().ravel()
    flips = np.abs(vis_g - vis_o) > 1e-4
    print(f"config 5: loss gpu {loss_g:.6e} oracle {loss_o:.6e}; shadowed={np.mean(vis_o < 1):.3f}; "
          f"stable points {int(stable.sum())}/{P}; flips {int(flips.sum())} (on stable points "
          f"{int((flips & stable).sum())})")
    checks = [("loss", loss_o > 0 and abs(loss_g - loss_o) <= 1e-3 * loss_o),
              ("stable fraction", np.mean(stable) > 0.8),
              ("no flip on a stable point", (flips & stable).sum() == 0)]

    nz = np.nonzero(np.abs(g_o) >= 1e-6)[0]
    rng = np.random.default_rng(5)
    pick = np.sort(rng.choice(nz, min(3000, nz.size), replace=False))
    rel = np.abs(g_g[pick].astype(np.float64) - g_o[pick]) / np.abs(g_o[pick])
    print(f"adjoint: texels with |g| >= 1e-6: {nz.size}, sampled {pick.size}, max rel {rel.max():.2e}, "
          f"99.9% {np.quantile(rel, 0.999):.2e}, median {np.median(rel):.2e}")
    checks += [("texels sampled", pick.size >= 1000), ("dLoss/dsdf per entry", rel.max() <= 1e-3)]
    lrel = np.abs(gl_g - gl_o) / np.abs(gl_o)
    print(f"dLoss/dlight gpu {gl_g} oracle {gl_o} rel {lrel.max():.2e}")
    checks.append(("dLoss/dlight", lrel.max() <= 1e-3))

    # the oracle gradient against fp64 central differences of the same
    # loss.  Texel j: only points whose ray passes within 2 texels of j can
    # change with f_j.  A kink (a discrete decision crossed within +-h) is
    # flagged when the one-sided differences disagree by more than 10 % or
    # the central differences at h and h/2 disagree by more than 1e-3.
    h = 1e-4
    fd_pick = pick[rng.permutation(pick.size)[:300]]
    base = (vis_o - tgt_o) ** 2 * stable
    spos = pos.astype(np.float64) + 2 * EPS_VOX * HF * nrm
    kinks, errs = 0, []
    f = f_o.copy()
    for j in fd_pick:
        q = (np.array([j % NF, (j // NF) % NF, j // (NF * NF)]) + 0.5) * HF
        foot = q - ((q[1] - spos[0, 1]) / L0[1]) * L0
        win = (np.abs(spos[:, 0] - foot[0]) < 6 * HF) & (np.abs(spos[:, 2] - foot[2]) < 6 * HF) & stable
        cand = np.nonzero(win)[0]
        w = q[None, :] - spos[cand]
        t = np.maximum(w @ L0, 0.0)
        dist = np.linalg.norm(w - t[:, None] * L0[None, :], axis=1)
        a = cand[dist <= 2.0 * HF]
        if a.size == 0:
            continue
        f0 = f[j]
        diff = {}
        for sgn in (1.0, -1.0, 0.5, -0.5):
            f[j] = np.float32(f0 + sgn * h)
            step = float(f[j]) - float(f0)
            v = oracle.shadow(f, NF, BMIN, 1.0, pos[a], nrm[a], L0, **cfg)
            diff[sgn] = (np.sum((v - tgt_o[a]) ** 2 - base[a]) / P, step)
        f[j] = f0
        (dp, hp), (dm, hm) = diff[1.0], diff[-1.0]
        (dp2, hp2), (dm2, hm2) = diff[0.5], diff[-0.5]
        fwd, bwd = dp / hp, dm / hm
        c1, c2 = (dp - dm) / (hp - hm), (dp2 - dm2) / (hp2 - hm2)
        if abs(fwd - bwd) > 0.1 * max(abs(fwd), abs(bwd)) or abs(c1 - c2) > 1e-3 * abs(c1):
            kinks += 1
            continue
        errs.append(abs(c1 - g_o[j]) / abs(g_o[j]))
    errs = np.array(errs)
    print(f"finite differences (texels): sampled={fd_pick.size} checked={errs.size} kinks={kinks} "
          f"max rel={errs.max():.2e} median rel={np.median(errs):.2e}")
    checks += [("fd texels checked", errs.size >= 200), ("fd texels", errs.max() <= 1e-3)]
    # dLoss/dlight: per point central differences of vis; points with a
    # kink within +-h (same rule, per point) are left out of both sides
    for ax in range(3):
        vs = {}
        for sgn in (1.0, -1.0, 0.5, -0.5):
            lv = L0.copy()
            lv[ax] += sgn * h
            vs[sgn] = oracle.shadow(f_o, NF, BMIN, 1.0, pos, nrm, lv, **cfg)
        fwd, bwd = (vs[1.0] - vis_o) / h, (vis_o - vs[-1.0]) / h
        c1, c2 = (vs[1.0] - vs[-1.0]) / (2 * h), (vs[0.5] - vs[-0.5]) / h
        kink = ((np.abs(fwd - bwd) > 0.1 * np.maximum(np.abs(fwd), np.abs(bwd)) + 1e-6)
                | (np.abs(c1 - c2) > 1e-3 * np.abs(c1) + 1e-6))
        w = dvis * ~kink
        fd = float(np.sum(w * c1))
        _, gl = oracle.shadow_grad(f_o, NF, BMIN, 1.0, pos, nrm, L0, dvis=w, **cfg)
        print(f"dLoss/dlight[{ax}]: fd {fd:.8e} oracle {gl[ax]:.8e} (kink points left out: {int(kink.sum())})")
        checks.append((f"fd light {ax}", abs(fd - gl[ax]) <= 1e-3 * abs(gl[ax])))
    failed = [name for name, ok in checks if not ok]
    assert not failed, failed
