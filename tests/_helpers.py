"""Shared helpers for the tests (no method arithmetic)."""
import numpy as np

import inputs


def cylinder_case(mech, ni=48, nj=32, mach=10.0, T=300.0, p=500.0):
    nodes = inputs.cylinder_ogrid(ni, nj)
    fs = inputs.freestream(mech, T=T, p=p, mach=mach)
    return nodes, inputs.cylinder_bc(), fs


def rel_err(a, b, axis=None):
    """max |a-b| / max |b| (per row if axis given)."""
    a = np.asarray(a)
    b = np.asarray(b)
    if axis is None:
        return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
    return np.max(np.abs(a - b), axis=axis) / np.maximum(np.max(np.abs(b), axis=axis), 1e-300)


def rel(a, b, ns=0):
    """Per-variable error of a vs b ([nvar][n]); species rows (first ns) share one scale."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        a, b = a[None], b[None]
    scale = np.abs(b).max(axis=1)
    if ns:
        scale[:ns] = np.max(scale[:ns])
    scale = np.maximum(scale, 1e-300)
    return float(np.max(np.abs(a - b).max(axis=1) / scale))
