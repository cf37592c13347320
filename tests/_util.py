"""Shared helpers for the tests (no method arithmetic here)."""
from __future__ import annotations

import numpy as np

EMPTY = 0xFFFFFFFF


def seeds_to_linear(s, n):
    """Packed GPU seeds (x | y << 8 | z << 16, all ones = none) -> linear index / -1."""
    s = np.asarray(s).astype(np.int64)
    lin = (s & 0xFF) + n * (((s >> 8) & 0xFF) + n * ((s >> 16) & 0xFF))
    return np.where(s == EMPTY, -1, lin)


def child_texels(masked_coarse, nc):
    """Fine texels (linear, grid 2nc) of the given coarse voxels, 8 each."""
    v = np.asarray(masked_coarse, dtype=np.int64)
    x, y, z = v % nc, (v // nc) % nc, v // (nc * nc)
    nf = 2 * nc
    out = []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                out.append((2 * x + dx) + nf * ((2 * y + dy) + nf * (2 * z + dz)))
    return np.sort(np.concatenate(out))


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False
