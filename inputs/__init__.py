"""Seeded synthetic input generators shared by the oracle tests, the CUDA tests and bench.py.

This module holds grid node coordinates, freestream descriptions and seeded random
perturbation fields only.  It contains none of the method's arithmetic (no thermodynamics,
no fluxes, no implicit operator): every quantity derived from these inputs is computed
separately by the oracle and by the CUDA library.

Node arrays are struct-of-arrays: ``nodes[d, k, j, i]`` for 3D and ``nodes[d, j, i]`` for 2D,
flattened in C order, with (ni+1) x (nj+1) [x (nk+1)] nodes for ni x nj [x nk] cells.  For a
periodic direction the last node layer is an exact copy of the first one.
"""
import math
import numpy as np

# Boundary condition codes (same integers as the library and the oracle use).
BC_PERIODIC, BC_WALL, BC_FARFIELD, BC_OUTFLOW, BC_AXIS = 0, 1, 2, 3, 4
# Gas models: 0 = single-species perfect diatomic gas (tests only), 1 = 5-species air 1T,
# 2 = 11-species ionised air 2T.
MECH_PERFECT, MECH_AIR5, MECH_AIR11 = 0, 1, 2
SPECIES = {
    MECH_PERFECT: ["A2"],
    MECH_AIR5: ["N2", "O2", "NO", "N", "O"],
    MECH_AIR11: ["N2", "O2", "NO", "N", "O", "NO+", "N2+", "O2+", "N+", "O+", "e-"],
}


def geometric_ratio(n, first, total):
    """Ratio q with first*(1+q+...+q^(n-1)) == total, by bisection."""
    if abs(first * n - total) < 1e-15 * total:
        return 1.0
    lo, hi = (1.0 + 1e-12, 2.0) if first * n < total else (1e-6, 1.0 - 1e-12)
    f = lambda q: first * (q ** n - 1.0) / (q - 1.0) - total
    if first * n < total:
        while f(hi) < 0:
            hi *= 1.5
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (f(mid) < 0) == (f(lo) < 0):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def cylinder_ogrid(ni, nj, radius=0.05, r_out=0.2, dr1=5e-5):
    """2D O-grid around a cylinder: i circumferential (clockwise, periodic), j radial outward.

    Cell i=0 is centred on the windward stagnation line (angle pi); the grid is mirror
    symmetric about the x axis.  Radial spacing is geometric with first spacing dr1.
    Returns nodes of shape (2, nj+1, ni+1).
    """
    q = geometric_ratio(nj, dr1, r_out - radius)
    r = np.empty(nj + 1)
    r[0] = radius
    for j in range(nj):
        r[j + 1] = r[j] + dr1 * q ** j
    r[nj] = r_out
    theta = math.pi + math.pi / ni - 2.0 * math.pi * np.arange(ni + 1) / ni
    nodes = np.empty((2, nj + 1, ni + 1))
    nodes[0] = r[:, None] * np.cos(theta)[None, :]
    nodes[1] = r[:, None] * np.sin(theta)[None, :]
    nodes[:, :, ni] = nodes[:, :, 0]
    return nodes


def cylinder_bc():
    """imin, imax, jmin, jmax, kmin, kmax boundary codes of the O-grid."""
    return [BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_FARFIELD, BC_PERIODIC, BC_PERIODIC]


def cylinder_half(ni, nj, radius=0.05, r_out=0.2, dr1=5e-5):
    """2D grid over the windward half of a cylinder: i circumferential (clockwise, from the
    upper shoulder to the lower one), j radial outward.  Both i ends are supersonic outflow
    boundaries, so the grid holds no wake and the flow has a steady state.

    The span is 180 degrees shifted by half a cell so that cell i = ni/2 is centred on the
    windward stagnation line (angle pi) for even ni.  Returns nodes of shape (2, nj+1, ni+1).
    """
    q = geometric_ratio(nj, dr1, r_out - radius)
    r = np.empty(nj + 1)
    r[0] = radius
    for j in range(nj):
        r[j + 1] = r[j] + dr1 * q ** j
    r[nj] = r_out
    dth = math.pi / ni
    theta = math.pi + (ni // 2 + 0.5 - np.arange(ni + 1)) * dth
    nodes = np.empty((2, nj + 1, ni + 1))
    nodes[0] = r[:, None] * np.cos(theta)[None, :]
    nodes[1] = r[:, None] * np.sin(theta)[None, :]
    return nodes


def cylinder_half_bc():
    """imin, imax, jmin, jmax, kmin, kmax boundary codes of the half-cylinder grid."""
    return [BC_OUTFLOW, BC_OUTFLOW, BC_WALL, BC_FARFIELD, BC_PERIODIC, BC_PERIODIC]


def sphere_cone(ni, nj, nk, nose=0.05, half_angle_deg=7.0, length=0.5, standoff=None, dr1=None):
    """3D sphere-cone grid: i along the body from the nose (axis) to the base, j normal to the
    wall, k circumferential (periodic).  Nodes at i=0 lie on the symmetry axis (degenerate
    i-faces of zero area).  Returns nodes of shape (3, nk+1, nj+1, ni+1).

    The body surface is parametrised by arc length s from the nose; the outer boundary is a
    scaled copy of the body (an ellipse-like shell) so that every j-line is straight along the
    local body normal.
    """
    a = math.radians(half_angle_deg)
    s_sph = nose * (math.pi / 2 - a)                       # arc length of the spherical cap
    x_tan = nose * (1 - math.sin(a))                       # tangency point (x from nose)
    r_tan = nose * math.cos(a)
    l_cone = (length - x_tan) / math.cos(a)
    s_tot = s_sph + l_cone
    if dr1 is None:
        dr1 = 5e-5 * 48.0 / nj * 32.0 / 48.0
    if standoff is None:
        standoff = 0.6 * nose
    # body points and outward normals
    s = s_tot * (np.arange(ni + 1) / ni) ** 1.0
    xb, rb, nx, nr = (np.empty(ni + 1) for _ in range(4))
    for i, si in enumerate(s):
        if si <= s_sph:
            phi = si / nose                                # angle from the axis
            xb[i] = nose * (1 - math.cos(phi))
            rb[i] = nose * math.sin(phi)
            nx[i], nr[i] = -math.cos(phi), math.sin(phi)
        else:
            t = si - s_sph
            xb[i] = x_tan + t * math.cos(a)
            rb[i] = r_tan + t * math.sin(a)
            nx[i], nr[i] = -math.sin(a), math.cos(a)
    rb[0] = 0.0
    nr[0] = 0.0
    nx[0] = -1.0
    # normal distance of the outer boundary grows along the body
    h = standoff * (1.5 + 3.0 * np.arange(ni + 1) / ni)
    nodes = np.empty((3, nk + 1, nj + 1, ni + 1))
    phik = 2.0 * math.pi * np.arange(nk + 1) / nk
    for i in range(ni + 1):
        q = geometric_ratio(nj, dr1, h[i])
        d = np.empty(nj + 1)
        d[0] = 0.0
        for j in range(nj):
            d[j + 1] = d[j] + dr1 * q ** j
        d[nj] = h[i]
        xs = xb[i] + d * nx[i]
        rs = rb[i] + d * nr[i]
        nodes[0, :, :, i] = xs[None, :]
        nodes[1, :, :, i] = rs[None, :] * np.cos(phik)[:, None]
        nodes[2, :, :, i] = rs[None, :] * np.sin(phik)[:, None]
    nodes[:, nk] = nodes[:, 0]
    return nodes


def sphere_cone_bc():
    return [BC_AXIS, BC_OUTFLOW, BC_WALL, BC_FARFIELD, BC_PERIODIC, BC_PERIODIC]


def box_grid(ni, nj, nk=0, lx=1.0, ly=1.0, lz=1.0, seed=None, wiggle=0.0):
    """Cartesian box (optionally with smooth seeded interior node displacement).

    2D if nk == 0.  With wiggle > 0 the interior nodes are displaced by a smooth field of
    relative amplitude ``wiggle`` (boundary nodes fixed), giving a curvilinear grid.
    """
    rng = np.random.default_rng(seed)
    if nk == 0:
        x = np.linspace(0, lx, ni + 1)
        y = np.linspace(0, ly, nj + 1)
        X, Y = np.meshgrid(x, y, indexing="xy")
        nodes = np.stack([X, Y])
        if wiggle > 0:
            ph = rng.uniform(0, 2 * math.pi, 4)
            bx = np.sin(math.pi * X / lx) * np.sin(math.pi * Y / ly)
            nodes[0] += wiggle * lx / ni * bx * np.sin(3 * Y / ly + ph[0]) * 2
            nodes[1] += wiggle * ly / nj * bx * np.cos(2 * X / lx + ph[1]) * 2
        return nodes
    x = np.linspace(0, lx, ni + 1)
    y = np.linspace(0, ly, nj + 1)
    z = np.linspace(0, lz, nk + 1)
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    nodes = np.stack([X, Y, Z])
    if wiggle > 0:
        ph = rng.uniform(0, 2 * math.pi, 6)
        b = np.sin(math.pi * X / lx) * np.sin(math.pi * Y / ly) * np.sin(math.pi * Z / lz)
        nodes[0] += wiggle * lx / ni * b * np.sin(3 * Y / ly + ph[0]) * 2
        nodes[1] += wiggle * ly / nj * b * np.cos(2 * Z / lz + ph[1]) * 2
        nodes[2] += wiggle * lz / nk * b * np.sin(2 * X / lx + ph[2]) * 2
    return nodes


def freestream(mech, T=300.0, p=500.0, mach=10.0, Tv=None, Y=None, direction=(1.0, 0.0, 0.0)):
    """Freestream description (primitive quantities only)."""
    names = SPECIES[mech]
    Yv = np.zeros(len(names))
    if Y is None:
        if mech == MECH_PERFECT:
            Yv[0] = 1.0
        else:
            Yv[0], Yv[1] = 0.767, 0.233
    else:
        for k, v in Y.items():
            Yv[names.index(k)] = v
    return dict(T=T, Tv=T if Tv is None else Tv, p=p, mach=mach, Y=Yv,
                dir=np.asarray(direction, dtype=np.float64))


def smooth_field(shape, seed, amplitude, modes=3):
    """Seeded smooth random field in [-amplitude, amplitude] on a cell array of ``shape``
    (C order, last axis = i)."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.linspace(0, 1, n) for n in shape], indexing="ij")
    f = np.zeros(shape)
    for _ in range(modes):
        ph = rng.uniform(0, 2 * math.pi, len(shape))
        kk = rng.integers(1, 4, len(shape))
        term = np.ones(shape)
        for g, k, p in zip(grids, kk, ph):
            term = term * np.sin(math.pi * k * g + p)
        f += rng.uniform(-1, 1) * term
    m = np.max(np.abs(f))
    return amplitude * f / m if m > 0 else f


def perturbed_primitive(mech, cell_shape, seed, T=1500.0, Tv=None, p=2000.0,
                        speed=1500.0, Y=None, amp=0.3, ndim=2, dissociated=True):
    """Seeded non-uniform primitive state on the cells (SoA): returns dict with
    rho_s[ns, ...], u[ndim, ...], T[...], Tv[...].  Densities come from an ideal-gas
    estimate with a fixed molar mass; the exact thermodynamic state is whatever the
    conserved variables built from these primitives imply."""
    names = SPECIES[mech]
    ns = len(names)
    rng_seed = seed * 7919 + 13
    Yb = np.zeros(ns)
    if Y is not None:
        Yb[:] = Y
    elif mech == MECH_PERFECT:
        Yb[0] = 1.0
    elif mech == MECH_AIR5:
        Yb[:] = [0.6, 0.15, 0.05, 0.1, 0.1] if dissociated else [0.767, 0.233, 0, 0, 0]
    else:
        Yb[:] = [0.55, 0.1, 0.05, 0.12, 0.12, 0.02, 0.015, 0.01, 0.008, 0.007, 0.0]
        if dissociated:
            Yb[10] = 5.4858e-4 * (0.02 / 30.0 + 0.015 / 28.0 + 0.01 / 32.0 + 0.008 / 14.0 + 0.007 / 16.0)
        else:
            Yb[:] = 0.0
            Yb[0], Yb[1] = 0.767, 0.233
    Yb = Yb / Yb.sum()
    fields = [smooth_field(cell_shape, rng_seed + k, 1.0) for k in range(ns + ndim + 3)]
    Yc = np.empty((ns,) + tuple(cell_shape))
    for s in range(ns):
        Yc[s] = Yb[s] * (1.0 + 0.5 * amp * fields[s]) if Yb[s] > 0 else 0.0
    Yc /= Yc.sum(axis=0, keepdims=True)
    Tc = T * (1.0 + amp * fields[ns])
    Tvc = (T if Tv is None else Tv) * (1.0 + amp * fields[ns + 1])
    pc = p * (1.0 + amp * fields[ns + 2])
    rho = pc / (287.0 * Tc)
    u = np.empty((ndim,) + tuple(cell_shape))
    for d in range(ndim):
        u[d] = speed * (0.8 if d == 0 else 0.2) * (1.0 + fields[ns + 3 + d])
    return dict(rho_s=Yc * rho[None], u=u, T=Tc, Tv=Tvc)


def batch_cases(n=64, seed=0):
    """Seeded list of independent 2D half-cylinder cases of uneven size for batched runs:
    grid (64 s) x (48 s) with s uniform in 1..8, Mach uniform in [6, 20], CFL log-uniform in
    [5, 200], 5-species 1T or 11-species 2T air with probability 1/2 each."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        s = int(rng.integers(1, 9))
        mach = float(rng.uniform(6.0, 20.0))
        cfl = float(math.exp(rng.uniform(math.log(5.0), math.log(200.0))))
        mech = MECH_AIR5 if rng.random() < 0.5 else MECH_AIR11
        out.append(dict(ni=64 * s, nj=48 * s, mach=mach, cfl=cfl, mech=mech))
    return out


def mlp_init(seed=0):
    """Seeded initial parameters of the 14-128-128-128-22 surrogate network as one float32
    vector (W1, b1, W2, b2, W3, b3, W4, b4; W row-major [out][in]): weights uniform in
    +-1/sqrt(fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for nout, nin in ((128, 14), (128, 128), (128, 128), (22, 128)):
        a = 1.0 / math.sqrt(nin)
        parts.append(rng.uniform(-a, a, nout * nin))
        parts.append(np.zeros(nout))
    return np.concatenate(parts).astype(np.float32)


def species_box(ns, seed=0, n=(10, 10, 10), size=(1.0, 1.0, 1.0)):
    """Uniform non-reacting flow of ns species in a Cartesian box, far field on every side
    (the species-count scaling test of Sec. 3.1).  Species s has molar mass M[s] (kg/kmol,
    log-uniform in [2, 100]) and dof[s] translational-rotational degrees of freedom (3 or 5,
    equally likely); mass fractions Y are a seeded Dirichlet(1) draw.  The flow: T = 300 K,
    p = 1e4 Pa, velocity (600, 300, 150) m/s, so that it crosses every face family."""
    rng = np.random.default_rng(seed)
    M = np.exp(rng.uniform(math.log(2.0), math.log(100.0), ns))
    dof = np.where(rng.uniform(size=ns) < 0.5, 3.0, 5.0)
    Y = rng.dirichlet(np.ones(ns))
    return dict(ns=ns, M=M, dof=dof, Y=Y, T=300.0, p=1.0e4, u=np.array([600.0, 300.0, 150.0]),
                n=tuple(n), size=tuple(size))


def species_box_rhs(ns, ncell, seed=0):
    """Seeded right-hand side [ns + 4][ncell] (rho_1..rho_ns, m_x, m_y, m_z, rho E) for the
    implicit operator of the species box: uniform in [-1, 1] times 1e-4 (species), 1e-1
    (momentum) and 1e2 (energy) per unit volume scale."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(-1.0, 1.0, (ns + 4, ncell))
    r[:ns] *= 1e-4
    r[ns:ns + 3] *= 1e-1
    r[ns + 3] *= 1e2
    return r
