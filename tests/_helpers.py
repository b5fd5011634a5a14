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


def oracle_run_to(case, tol=1e-8, chunk=100, max_iters=20000, scheme=0, correction=1):
    """Run the oracle on a half-cylinder case (dict with ni, nj, mech, mach, dr1, limiter, cfl,
    cfl_start, ramp) from the freestream until both residual monitors have dropped by `tol`,
    checked after the first iteration and then every `chunk` iterations (the GPU driver's
    schedule).  Runs in a worker process of its own; imports only the oracle."""
    import oracle
    nodes = inputs.cylinder_half(case["ni"], case["nj"], dr1=case["dr1"])
    fs = inputs.freestream(case["mech"], T=300.0, p=500.0, mach=case["mach"])
    g = oracle.OracleGrid(nodes, inputs.cylinder_half_bc(), case["mech"], limiter=case["limiter"])
    g.set_boundary(fs, Tw=500.0)
    g.set_state(g.freestream_state())
    kw = dict(scheme=scheme, correction=correction, clip=1, cfl=case["cfl"],
              cfl_start=case["cfl_start"], ramp_iters=case["ramp"])
    st = g.step(iters=1, **kw)
    r0 = (st["r_species"], st["r_energy"])
    done, hist = 1, [(1, 1.0, 1.0, st["q_stag"])]
    status = "max_iters"
    while done < max_iters:
        st = g.step(iters=chunk, **kw)
        done += st["iters_done"]
        hist.append((done, st["r_species"] / r0[0], st["r_energy"] / r0[1], st["q_stag"]))
        if hist[-1][1] <= tol and hist[-1][2] <= tol:
            status = "converged"
            break
    return dict(status=status, iterations=done, q_stag=float(st["q_stag"]), history=hist)
