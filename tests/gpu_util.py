"""Helpers for the GPU tests: pinned host operands filled from the seeded generator."""
import numpy as np
import torch

import synth


def pinned(rows, cols, dtype=torch.float64, ld=None, fill=None):
    """A pinned rows x cols host tensor (a view of rows x ld storage when ld > cols)."""
    ld = cols if ld is None else ld
    base = torch.empty((max(rows, 1), max(ld, 1)), dtype=dtype, pin_memory=True)
    if fill is not None:
        base.fill_(fill)
    return base[:rows, :cols]


def pinned_from(seed, stream, rows, cols, kind, param=0.0, dtype=torch.float64, ld=None, pad=np.nan):
    t = pinned(rows, cols, dtype=dtype, ld=ld, fill=pad if ld is not None else None)
    if rows and cols:
        synth.fill(t, seed, stream, kind, param)
    return t


def np64(t):
    return t.numpy().astype(np.float64, copy=True)
