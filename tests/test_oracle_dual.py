"""Pins of the oracle's dual time stepping (Sec. 2.3, the dual-time form of the implicit scheme:
physical-time term (1+theta)(Q - Q^n) - theta (Q^n - Q^{n-1}) over dt added to the residual,
(1+theta) V / dt added to every diagonal of the operator).

The workload is a zero-dimensional reactor: a spatially uniform, moving, chemically and
thermally out-of-equilibrium 11-species 2T air state on a box that is periodic in both
directions, so that every flux cancels and the spatial residual is -V S(Q).  There:
  * the converged inner iterate of every physical step must solve the time-discrete equation
    (1+theta)(Q - Q^n) - theta (Q^n - Q^{n-1}) = dt S(Q), with S from a separate steady
    evaluation of the residual (a wrong sign, coefficient, volume factor or level fails it);
  * over several steps the result must converge to the solution of the ODE dQ/dt = S(Q) from
    scipy's Radau integrator at tight tolerance, at first order for theta = 0 and at second
    order for theta = 1/2 (the three-level backward difference); theta = 2 is first order;
  * with dual time stepping off, or no physical step begun, the scheme is the steady one.
"""
import math

import numpy as np
import pytest

import inputs
import oracle

MECH = inputs.MECH_AIR11
ME = 5.48579909e-4
NODES = inputs.box_grid(3, 3)
BC = [0, 0, 0, 0, 0, 0]            # periodic in i and in j
T_END = 8e-6


def reactor_freestream():
    ions = {"NO+": 1e-5, "N2+": 1e-6, "O2+": 1e-6, "N+": 1e-6, "O+": 1e-6}
    M = {"NO+": 30.006, "N2+": 28.013, "O2+": 31.998, "N+": 14.006, "O+": 15.999}
    Y = {"O2": 0.2, "NO": 0.02, "N": 0.01, "O": 0.0299, **ions}
    Y["e-"] = ME * sum(v / M[k] for k, v in ions.items())      # charge neutral
    Y["N2"] = 1.0 - sum(Y.values())
    return inputs.freestream(MECH, T=6000.0, Tv=1500.0, p=1e4, mach=0.3, Y=Y)


def reactor(dt=0.0, theta=0.0):
    g = oracle.OracleGrid(NODES, BC, MECH)
    g.set_boundary(reactor_freestream(), Tw=500.0)
    g.set_state(g.freestream_state())
    if dt > 0.0:
        g.set_dual(dt, theta)
    return g


@pytest.fixture(scope="module")
def source():
    """S(q) of a uniform state q, from the steady residual of the periodic box."""
    g = reactor()
    V = 1.0 / 9.0

    def S(q):
        g.set_state(np.repeat(np.asarray(q)[:, None], 9, axis=1))
        R, _ = g.residual()
        return -R[:, 0] / V
    return S


def inner(g, iters):
    for _ in range(iters):
        g.step(scheme=0, correction=1, clip=1, cfl=1e3, cfl_start=1e3, ramp_iters=0, iters=1)


def test_uniform_box_is_a_reactor(source):
    g = reactor()
    Q = g.freestream_state()
    R, _ = g.residual()
    # all cells alike, momentum and total energy conserved, the rest driven by the source
    assert np.allclose(R, R[:, :1], rtol=1e-12, atol=1e-12 * np.abs(R).max())
    s = source(Q[:, 0])
    assert np.all(np.abs(s[11:14]) <= 1e-9 * np.abs(s).max())
    assert abs(s[:11].sum()) <= 1e-10 * np.abs(s[:11]).max()       # mass
    assert s[14] > 0.0                                               # Tv < T: e_v grows


@pytest.mark.parametrize("theta", [0.0, 0.5, 2.0])
def test_converged_step_solves_the_time_discrete_equation(source, theta):
    dt = 5e-7
    g = reactor(dt, theta)
    Qnm1 = Qn = None
    for n in range(3):
        Qprev = g.get_state()[:, 0]
        g.dual_advance()
        Qnm1, Qn = Qn, Qprev
        inner(g, 25)
        Q = g.get_state()
        # stays uniform (to rounding; the second momentum is zero up to rounding noise)
        tol = 1e-12 * np.maximum(np.abs(Q).max(axis=1), np.abs(Q[11]).max())
        assert np.all(np.abs(Q - Q[:, :1]).max(axis=1) <= tol)
        q = Q[:, 0]
        th = theta if n >= 1 else 0.0          # the first step has no Q^{n-1}: implicit Euler
        lhs = (1.0 + th) * (q - Qn) - (th * (Qn - Qnm1) if n >= 1 else 0.0)
        res = lhs - dt * source(q)
        scale = np.abs(q - Qn).max()
        assert np.abs(res).max() <= 1e-9 * scale, (n, np.abs(res).max() / scale)


@pytest.fixture(scope="module")
def reference(source):
    from scipy.integrate import solve_ivp
    Q0 = reactor().freestream_state()[:, 0]
    atol = 1e-13 * (np.abs(Q0) + 1e-3 * Q0[:11].sum())
    sol = solve_ivp(lambda t, q: source(q), (0.0, T_END), Q0, method="Radau", rtol=1e-11,
                    atol=atol)
    assert sol.status == 0
    return sol.y[:, -1]


def march(dt, theta):
    g = reactor(dt, theta)
    for _ in range(int(round(T_END / dt))):
        g.dual_advance()
        inner(g, 12)
    return g.get_state()[:, 0]


def observed_orders(theta, dts, reference):
    err = [np.abs(march(dt, theta) - reference)[:11].max() for dt in dts]
    return err, [math.log2(err[k] / err[k + 1]) for k in range(len(err) - 1)]


def test_theta_zero_is_first_order(reference):
    err, p = observed_orders(0.0, [1e-6, 5e-7, 2.5e-7], reference)
    assert all(0.85 < x < 1.15 for x in p), p


def test_theta_half_is_second_order(reference):
    err, p = observed_orders(0.5, [2.5e-7, 1.25e-7, 6.25e-8], reference)
    assert p[-1] > 1.8 and p[-1] > p[0], p
    # and far more accurate than implicit Euler at the same step
    e0, _ = observed_orders(0.0, [2.5e-7, 1.25e-7], reference)
    assert err[0] < 0.2 * e0[0]


def test_theta_two_is_first_order(reference):
    err, p = observed_orders(2.0, [1e-6, 5e-7, 2.5e-7], reference)
    assert all(0.6 < x < 1.4 for x in p), p


def test_dual_off_or_not_begun_is_the_steady_scheme():
    nodes = inputs.cylinder_half(16, 12)
    fs = inputs.freestream(MECH, T=300.0, p=500.0, mach=10.0)
    out = []
    for mode in ("never", "off", "not begun"):
        g = oracle.OracleGrid(nodes, inputs.cylinder_half_bc(), MECH)
        g.set_boundary(fs, Tw=500.0)
        g.set_state(g.freestream_state())
        if mode == "off":
            g.set_dual(1e-6, 0.5)
            g.set_dual(0.0, 0.0)
        elif mode == "not begun":
            g.set_dual(1e-6, 0.5)
        g.step(scheme=0, correction=1, clip=1, cfl=2.0, cfl_start=0.5, ramp_iters=10, iters=5)
        out.append(g.get_state())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_dual_rejects_bad_arguments():
    g = reactor()
    with pytest.raises(oracle.OracleError):
        g.set_dual(-1.0, 0.0)
    with pytest.raises(oracle.OracleError):
        g.set_dual(1e-6, -0.5)
    with pytest.raises(oracle.OracleError):
        g.dual_advance()                     # dual time stepping not on
