"""Plain numpy restatement of one implicit LU-SGS step of the split (CS) and coupled (CI)
operators for a non-reacting mixture of ns calorically perfect species on a uniform Cartesian
box: the species-count scaling test of Sec. 3.1 (a uniform flow in a box, far field on every
side, no chemistry, ns from 16 upwards; the cost of one implicit step is compared).

TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and the CPU legs of the benchmark may
import this module.  It shares no code with the CUDA path.

Gas (reading: the paper leaves the species of this test unspecified): species s has molar
mass M_s and f_s translational-rotational degrees of freedom, c_v,s = (f_s / 2) R_u / M_s,
R_s = R_u / M_s, no vibrational energy, no formation energy.  Conserved variables
Q = (rho_1 .. rho_ns, m_x, m_y, m_z, rho E); p = (sum_s rho_s R_s) T with
T = (rho E - |m|^2 / (2 rho)) / sum_s rho_s c_v,s.  Euler flux through a face vector S:
(rho_s U, m U + p S, (rho E + p) U), U = m.S / rho.

Operators (Sec. 2.2-2.3, as the 2D/3D path computes them, inviscid radii: the flow is
uniform, so viscous fluxes vanish; the viscous radius would add a per-cell scalar and does not
change the cost's dependence on ns):
  radii per cell and direction d, with S_d the mean of the cell's two d-faces:
    flow / coupled  lambda_F,d = |u.S_d| + c |S_d|,   species  lambda_C,d = |u.S_d|;
  V / dtau = sum_d lambda_F,d / CFL;
  diagonals D_F = V/dtau + sum_d lambda_F,d, D_s = V/dtau + sum_d lambda_C,d (every species),
    D_CI = (V/dtau + sum_d lambda_F,d) I (n_c x n_c: no source Jacobian without chemistry);
  split: flow block (rho, m, rho E) with the frozen-composition flux Jacobian (the species
    perturbed as Y_s d rho) and one scalar equation per species with the Jacobian U I;
  coupled: n_c = ns + 4 unknowns (rho, m, rho E, rho_2 .. rho_ns), rho_1 = rho - sum_{r>1} rho_r;
  forward sweep in cell order c = i + ni (j + nj k):
    D x_c = rhs_c + sum_{lower nb} 1/2 (A(S) x_nb + lambda_nb x_nb),
  backward sweep in reverse order:
    D y_c = D x_c - sum_{upper nb} 1/2 (A(S) y_nb - lambda_nb y_nb),
  with S the face vector between c and nb (oriented +d) and A(S) x the flux Jacobian of the
  neighbour's state applied to x.  Boundary neighbours (far field) contribute nothing.
  Flux Jacobian-vector products are directional derivatives of the flux function, taken here
  by the complex step F(Q + i h x).imag / h (exact to rounding for this rational flux).

Parity pins: tests/test_oracle_species_box.py.
"""
import numpy as np

RU = 8314.462618           # J/(kmol K)
H_CS = 1e-30               # complex-step size


class Box:
    """Geometry, gas and uniform state of the species box."""

    def __init__(self, case):
        self.ns = ns = int(case["ns"])
        self.n = tuple(int(x) for x in case["n"])
        self.size = tuple(float(x) for x in case["size"])
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.Rs = RU / np.asarray(case["M"], dtype=np.float64)
        self.cvs = 0.5 * np.asarray(case["dof"], dtype=np.float64) * self.Rs
        Y = np.asarray(case["Y"], dtype=np.float64)
        T, p, u = float(case["T"]), float(case["p"]), np.asarray(case["u"], dtype=np.float64)
        rho = p / (np.dot(Y, self.Rs) * T)
        q = np.empty(ns + 4)
        q[:ns] = rho * Y
        q[ns:ns + 3] = rho * u
        q[ns + 3] = rho * np.dot(Y, self.cvs) * T + 0.5 * rho * np.dot(u, u)
        self.q = q                                   # uniform conserved state
        h = [self.size[d] / self.n[d] for d in range(3)]
        self.V = h[0] * h[1] * h[2]
        # face vectors of the three face families (uniform box)
        self.S = [np.array([h[1] * h[2], 0.0, 0.0]), np.array([0.0, h[0] * h[2], 0.0]),
                  np.array([0.0, 0.0, h[0] * h[1]])]

    def cell(self, i, j, k):
        return i + self.n[0] * (j + self.n[1] * k)

    def coords(self, c):
        i = c % self.n[0]
        j = (c // self.n[0]) % self.n[1]
        return i, j, c // (self.n[0] * self.n[1])


def flux(box, q, S):
    """Euler flux of a conserved state q (real or complex) through face vector S."""
    ns = box.ns
    rhos = q[:ns]
    rho = rhos.sum()
    m = q[ns:ns + 3]
    K = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho
    T = (q[ns + 3] - K) / np.dot(rhos, box.cvs)
    p = np.dot(rhos, box.Rs) * T
    U = (m[0] * S[0] + m[1] * S[1] + m[2] * S[2]) / rho
    F = np.empty(ns + 4, dtype=q.dtype)
    F[:ns] = rhos * U
    F[ns:ns + 3] = m * U + p * np.asarray(S)
    F[ns + 3] = (q[ns + 3] + p) * U
    return F


def jvp_full(box, q, S, dq):
    """d F / d Q (q) applied to dq (full layout), by the complex step."""
    return flux(box, q + 1j * H_CS * dq, S).imag / H_CS


def primitives(box, q):
    ns = box.ns
    rho = q[:ns].sum()
    u = q[ns:ns + 3] / rho
    cv = np.dot(q[:ns], box.cvs) / rho
    R = np.dot(q[:ns], box.Rs) / rho
    T = (q[ns + 3] / rho - 0.5 * np.dot(u, u)) / cv
    p = rho * R * T
    c = np.sqrt((1.0 + R / cv) * p / rho)
    return rho, u, p, c


def radii(box, q):
    """(lambda_F[3], lambda_C[3]) of a cell in the uniform box (all faces alike)."""
    rho, u, p, c = primitives(box, q)
    lF, lC = np.empty(3), np.empty(3)
    for d in range(3):
        Sb = box.S[d]                 # mean of the two d-faces (equal in a uniform box)
        U = np.dot(u, Sb)
        lF[d] = abs(U) + c * np.linalg.norm(Sb)
        lC[d] = abs(U)
    return lF, lC


def neighbours(box, c, lower):
    """(neighbour cell, face vector, direction, side) of the lower (or upper) neighbours."""
    i, j, k = box.coords(c)
    o = [i, j, k]
    out = []
    for d in range(3):
        for s in (-1, 1):
            p = list(o)
            p[d] += s
            if p[d] < 0 or p[d] >= box.n[d]:
                continue
            if (s < 0) != lower:
                continue
            out.append((box.cell(*p), box.S[d], d, s))
    return out


def split_operator(box, rhs, cfl):
    """Split LU-SGS increments, layout (rho, m_x, m_y, m_z, rho E, rho_1 .. rho_ns) x cells.
    rhs: [ns + 4][N] in the conserved layout (rho_1 .. rho_ns, m, rho E)."""
    ns, N = box.ns, box.N
    q = box.q
    lF, lC = radii(box, q)
    Vdt = lF.sum() / cfl
    DF = Vdt + lF.sum()
    Ds = Vdt + lC.sum()
    Y = q[:ns] / q[:ns].sum()

    def jvp_flow(xf, S):
        dq = np.concatenate([Y * xf[0], xf[1:4], xf[4:5]])
        a = jvp_full(box, q, S, dq)
        return np.concatenate([[a[:ns].sum()], a[ns:ns + 4]])

    def U_face(S):
        return np.dot(q[ns:ns + 3] / q[:ns].sum(), S)

    xF = np.zeros((5, N))
    xS = np.zeros((ns, N))
    for c in range(N):
        acc = np.concatenate([[rhs[:ns, c].sum()], rhs[ns:ns + 4, c]])
        accs = rhs[:ns, c].copy()
        for nb, S, d, s in neighbours(box, c, True):
            acc += 0.5 * (jvp_flow(xF[:, nb], S) + lF[d] * xF[:, nb])
            accs += 0.5 * (U_face(S) * xS[:, nb] + lC[d] * xS[:, nb])
        xF[:, c] = acc / DF
        xS[:, c] = accs / Ds
    yF = np.zeros((5, N))
    yS = np.zeros((ns, N))
    for c in range(N - 1, -1, -1):
        acc = np.zeros(5)
        accs = np.zeros(ns)
        for nb, S, d, s in neighbours(box, c, False):
            acc -= 0.5 * (jvp_flow(yF[:, nb], S) - lF[d] * yF[:, nb])
            accs -= 0.5 * (U_face(S) * yS[:, nb] - lC[d] * yS[:, nb])
        yF[:, c] = xF[:, c] + acc / DF
        yS[:, c] = xS[:, c] + accs / Ds
    return np.concatenate([yF, yS])


def coupled_operator(box, rhs, cfl):
    """Coupled LU-SGS increments, layout (rho, m_x, m_y, m_z, rho E, rho_2 .. rho_ns) x cells."""
    ns, N = box.ns, box.N
    nc = ns + 4
    q = box.q
    lF, _ = radii(box, q)
    Vdt = lF.sum() / cfl
    D = (Vdt + lF.sum()) * np.eye(nc)

    def to_full(x):
        dq = np.empty(ns + 4)
        dq[0] = x[0] - x[5:].sum()
        dq[1:ns] = x[5:]
        dq[ns:ns + 4] = x[1:5]
        return dq

    def jvp_ci(x, S):
        a = jvp_full(box, q, S, to_full(x))
        return np.concatenate([[a[:ns].sum()], a[ns:ns + 4], a[1:ns]])

    def rhs_ci(c):
        return np.concatenate([[rhs[:ns, c].sum()], rhs[ns:ns + 4, c], rhs[1:ns, c]])

    x = np.zeros((nc, N))
    for c in range(N):
        acc = rhs_ci(c)
        for nb, S, d, s in neighbours(box, c, True):
            acc += 0.5 * (jvp_ci(x[:, nb], S) + lF[d] * x[:, nb])
        x[:, c] = np.linalg.solve(D, acc)
    y = np.zeros((nc, N))
    for c in range(N - 1, -1, -1):
        acc = np.zeros(nc)
        for nb, S, d, s in neighbours(box, c, False):
            acc -= 0.5 * (jvp_ci(y[:, nb], S) - lF[d] * y[:, nb])
        y[:, c] = x[:, c] + np.linalg.solve(D, acc)
    return y
