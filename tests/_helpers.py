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
