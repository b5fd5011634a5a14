"""ctypes front end of the FP64 CPU oracle (``oracle/cs_oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle is the plain restatement of the method (arXiv:2403.03440,
Sec. 2) that the CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  It never imports the CUDA
package and the CUDA package never imports it.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cs_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libcs_oracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "libcs_oracle_omp.so")
_lib = None
_openmp = False


def use_openmp():
    """Load the OpenMP build (all host cores; used only to time the oracle) instead of the
    serial one.  Must be called before the first oracle call of the process."""
    global _openmp
    if _lib is not None:
        raise RuntimeError("the oracle library is already loaded")
    _openmp = True

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def build(force=False, openmp=None):
    """Compile the oracle with gcc (FP64, -O3, no contraction into FMA, no host-specific
    instruction set: the same results on every host); openmp=True builds the variant whose
    independent per-cell and per-face loops run on all host cores (timing only)."""
    if openmp is None:
        openmp = _openmp
    out = _OUT_OMP if openmp else _OUT
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O3", "-ffp-contract=off", "-std=c11", "-fPIC", "-shared"]
    if openmp:
        cmd.append("-fopenmp")
    cmd += ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _ip, C.c_int, C.c_int,
                                 C.c_double, _dp, C.POINTER(C.c_void_p)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_reacting.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_hcorr.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_viscous.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_transport.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_update_limit.argtypes = [C.c_void_p, C.c_double]
        L.orc_set_dual.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.orc_set_ci_splitting.argtypes = [C.c_void_p, C.c_int]
        L.orc_set_dtau_source.argtypes = [C.c_void_p, C.c_int]
        L.orc_dual_advance.argtypes = [C.c_void_p]
        L.orc_set_boundary.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                                       _dp, _dp, C.c_double]
        L.orc_freestream_state.argtypes = [C.c_void_p, _dp]
        L.orc_set_state.argtypes = [C.c_void_p, _dp]
        L.orc_get_state.argtypes = [C.c_void_p, _dp]
        L.orc_residual.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_lusgs_split.argtypes = [C.c_void_p, C.c_double, _dp]
        L.orc_lusgs_coupled.argtypes = [C.c_void_p, C.c_double, _dp]
        L.orc_correct.argtypes = [C.c_void_p, C.c_int, C.c_int, _dp, _ip]
        L.orc_step.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                               C.c_int, C.c_int, _dp]
        L.orc_last_error.argtypes = [C.c_void_p]
        L.orc_last_error.restype = C.c_char_p
        L.orc_dims.argtypes = [C.c_void_p, _ip]
        L.orc_field.argtypes = [C.c_void_p, C.c_char_p, _dp]
        L.orc_build_diagonals.argtypes = [C.c_void_p, C.c_double]
        L.orc_coupling_block.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _ip]
        L.orc_gas_info.argtypes = [C.c_int, _dp, _dp, _ip]
        L.orc_state_prim.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.orc_state_cons.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double, _dp]
        L.orc_state_flux.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
        L.orc_state_roe.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, C.c_double, _dp]
        L.orc_state_jvp.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_int, _dp, _dp]
        L.orc_state_chem.argtypes = [C.c_int, _dp, C.c_double, C.c_double, _dp, _dp]
        L.orc_lnKc.argtypes = [C.c_int, C.c_int, C.c_double, _dp]
        L.orc_gibbs.argtypes = [C.c_int, C.c_int, C.c_double, _dp]
        L.orc_state_vib.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.orc_species_energy.argtypes = [C.c_int, C.c_double, C.c_double, _dp]
        L.orc_state_source_jac.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
    return _lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def gas_info(mech):
    M = np.zeros(16)
    hf = np.zeros(16)
    dims = np.zeros(3, dtype=np.int32)
    lib().orc_gas_info(mech, _p(M), _p(hf), dims.ctypes.data_as(_ip))
    ns = int(dims[0])
    return dict(ns=ns, nr=int(dims[1]), ntemp=int(dims[2]), M=M[:ns].copy(), hf=hf[:ns].copy())


PRIM_KEYS = ["T", "Tv", "p", "c", "beta", "rho", "Gam", "H", "mu", "kt", "kv", "rhoD",
             "cvtr", "cvve", "cv", "prev"]


def state_prim(mech, nd, q):
    q = _f64(q)
    out = np.zeros(16 + 16)
    st = lib().orc_state_prim(mech, nd, _p(q), _p(out))
    if st:
        raise OracleError(f"state_prim status {st}")
    ns = gas_info(mech)["ns"]
    d = {k: out[i] for i, k in enumerate(PRIM_KEYS)}
    d["prs"] = out[16:16 + ns].copy()
    return d


def state_cons(mech, nd, rhos, u, T, Tv=None):
    info = gas_info(mech)
    q = np.zeros(info["ns"] + nd + 1 + (info["ntemp"] == 2))
    lib().orc_state_cons(mech, nd, _p(_f64(rhos)), _p(_f64(u)), float(T),
                         float(T if Tv is None else Tv), _p(q))
    return q


def state_flux(mech, nd, q, S):
    q = _f64(q)
    F = np.zeros_like(q)
    st = lib().orc_state_flux(mech, nd, _p(q), _p(_f64(np.resize(S, 3))), _p(F))
    if st:
        raise OracleError(f"flux status {st}")
    return F


def state_roe(mech, nd, qL, qR, S, efix=0.1):
    qL, qR = _f64(qL), _f64(qR)
    F = np.zeros_like(qL)
    st = lib().orc_state_roe(mech, nd, _p(qL), _p(qR), _p(_f64(np.resize(S, 3))), efix, _p(F))
    if st:
        raise OracleError(f"roe status {st}")
    return F


def state_jvp(mech, nd, q, S, which, dq):
    q, dq = _f64(q), _f64(dq)
    out = np.zeros(32)
    st = lib().orc_state_jvp(mech, nd, _p(q), _p(_f64(np.resize(S, 3))), which, _p(dq), _p(out))
    if st:
        raise OracleError(f"jvp status {st}")
    return out[:len(dq)].copy()


def state_chem(mech, rhos, T, Tv=None):
    rhos = _f64(rhos)
    ns = len(rhos)
    om = np.zeros(ns)
    J = np.zeros(ns * ns)
    lib().orc_state_chem(mech, _p(rhos), float(T), float(T if Tv is None else Tv), _p(om), _p(J))
    return om, J.reshape(ns, ns)


def state_source_jac(mech, nd, q):
    q = _f64(q)
    ns = gas_info(mech)["ns"]
    om = np.zeros(ns)
    J = np.zeros(ns * len(q))
    st = lib().orc_state_source_jac(mech, nd, _p(q), _p(om), _p(J))
    if st:
        raise OracleError(f"source_jac status {st}")
    return om, J.reshape(ns, len(q))


def lnKc(mech, r, T):
    out = np.zeros(1)
    if lib().orc_lnKc(mech, r, float(T), _p(out)):
        raise OracleError("bad reaction")
    return float(out[0])


def gibbs_RT(mech, s, T):
    out = np.zeros(1)
    if lib().orc_gibbs(mech, s, float(T), _p(out)):
        raise OracleError("bad species")
    return float(out[0])


def state_vib(mech, nd, q):
    ns = gas_info(mech)["ns"]
    out = np.zeros(2 + ns)
    st = lib().orc_state_vib(mech, nd, _p(_f64(q)), _p(out))
    if st:
        raise OracleError(f"vib status {st}")
    return dict(omega_v=out[0], relax=out[1], tau=out[2:].copy())


def species_energy(mech, T, Tv=None):
    ns = gas_info(mech)["ns"]
    out = np.zeros(ns)
    lib().orc_species_energy(mech, float(T), float(T if Tv is None else Tv), _p(out))
    return out


class OracleGrid:
    """One structured grid + state in the oracle.  Arrays are numpy float64, SoA [var][cell]."""

    def __init__(self, nodes, bc, mech, limiter=1, efix=0.1):
        nodes = _f64(nodes)
        nd = nodes.shape[0]
        if nd == 2:
            nj, ni = nodes.shape[1] - 1, nodes.shape[2] - 1
            nk = 1
        else:
            nk, nj, ni = nodes.shape[1] - 1, nodes.shape[2] - 1, nodes.shape[3] - 1
        self.nd, self.ni, self.nj, self.nk, self.mech = nd, ni, nj, nk, mech
        bca = np.asarray(bc, dtype=np.int32)
        h = C.c_void_p()
        st = lib().orc_create(nd, ni, nj, nk, bca.ctypes.data_as(_ip), mech, limiter, efix,
                              _p(nodes), C.byref(h))
        if st:
            raise OracleError(f"orc_create status {st}")
        self._h = h
        dims = np.zeros(8, dtype=np.int32)
        lib().orc_dims(h, dims.ctypes.data_as(_ip))
        (self.ncell, self.nq, self.nsplit, self.nci, self.ns, self.ntemp, self.nF,
         self.stag_cell) = [int(x) for x in dims]

    def __del__(self):
        if getattr(self, "_h", None) is not None and lib is not None:
            try:
                lib().orc_destroy(self._h)
            except Exception:
                pass
            self._h = None

    def _check(self, st, what):
        if st:
            raise OracleError(f"{what}: status {st}: {lib().orc_last_error(self._h).decode()}")

    def set_reacting(self, on):
        lib().orc_set_reacting(self._h, int(bool(on)))

    def set_hcorr(self, on):
        lib().orc_set_hcorr(self._h, int(bool(on)))

    def set_viscous(self, on):
        """Viscous and diffusive fluxes and radii on (default) or off (inviscid flow)."""
        lib().orc_set_viscous(self._h, int(bool(on)))

    def set_transport(self, model):
        """Transport model: 0 Sutherland / constant Pr, Sc; 1 Blottner-Eucken-Wilke-Blanc."""
        self._check(lib().orc_set_transport(self._h, int(model)), "set_transport")

    def set_update_limit(self, f):
        self._check(lib().orc_set_update_limit(self._h, float(f)), "set_update_limit")

    def set_ci_splitting(self, mode):
        """Flux-Jacobian splitting of the coupled operator: 0 spectral, 1 eigenvalue."""
        self._check(lib().orc_set_ci_splitting(self._h, int(mode)), "set_ci_splitting")

    def set_dtau_source(self, on):
        """Source radius lambda_S in the local time step's denominator (Sec. 2.2): 0 / 1."""
        self._check(lib().orc_set_dtau_source(self._h, int(on)), "set_dtau_source")

    def set_dual(self, dt, theta=0.0):
        """Dual time stepping with physical step dt (0: steady) and coefficient theta."""
        self._check(lib().orc_set_dual(self._h, float(dt), float(theta)), "set_dual")

    def dual_advance(self):
        """Begin a physical time step from the current state (Q^{n-1} <- Q^n <- Q)."""
        self._check(lib().orc_dual_advance(self._h), "dual_advance")

    def set_boundary(self, fs, Tw=500.0):
        Y = _f64(fs["Y"])
        d = _f64(np.resize(fs["dir"], 3))
        self._check(lib().orc_set_boundary(self._h, fs["T"], fs["Tv"], fs["p"], fs["mach"],
                                           _p(Y), _p(d), Tw), "set_boundary")
        dims = np.zeros(8, dtype=np.int32)
        lib().orc_dims(self._h, dims.ctypes.data_as(_ip))
        self.stag_cell = int(dims[7])

    def freestream_state(self):
        Q = np.zeros((self.nq, self.ncell))
        lib().orc_freestream_state(self._h, _p(Q))
        return Q

    def set_state(self, Q):
        Q = _f64(Q).reshape(self.nq, self.ncell)
        self._check(lib().orc_set_state(self._h, _p(Q)), "set_state")

    def get_state(self):
        Q = np.zeros((self.nq, self.ncell))
        lib().orc_get_state(self._h, _p(Q))
        return Q

    def residual(self):
        R = np.zeros((self.nq, self.ncell))
        norms = np.zeros(3)
        self._check(lib().orc_residual(self._h, _p(R), _p(norms)), "residual")
        return R, norms

    def lusgs_split(self, cfl):
        dQ = np.zeros((self.nsplit, self.ncell))
        self._check(lib().orc_lusgs_split(self._h, cfl, _p(dQ)), "lusgs_split")
        return dQ

    def lusgs_coupled(self, cfl):
        dQ = np.zeros((self.nci, self.ncell))
        self._check(lib().orc_lusgs_coupled(self._h, cfl, _p(dQ)), "lusgs_coupled")
        return dQ

    def correct(self, mode, clip, dQ=None):
        n = C.c_int(0)
        ptr = _p(_f64(dQ)) if dQ is not None else C.cast(None, _dp)
        keep = _f64(dQ) if dQ is not None else None
        if keep is not None:
            ptr = _p(keep)
        self._check(lib().orc_correct(self._h, mode, clip, ptr, C.byref(n)), "correct")
        return n.value

    def step(self, scheme=0, correction=1, clip=1, cfl=10.0, cfl_start=1.0, ramp_iters=0,
             iters=1):
        stats = np.zeros(5)
        self._check(lib().orc_step(self._h, scheme, correction, clip, cfl, cfl_start, ramp_iters,
                                   iters, _p(stats)), "step")
        return dict(iters_done=int(stats[0]), r_species=stats[1], r_energy=stats[2],
                    q_stag=stats[3], nclip=int(stats[4]))

    def field(self, name, size=None):
        if size is None:
            size = max(self.ncell * 64 * 3, self.ncell * self.nci * self.nci, 3 * (self.ni + 1) *
                       (self.nj + 1) * (self.nk + 1) * self.nq)
        out = np.zeros(size)
        n = lib().orc_field(self._h, name.encode(), _p(out))
        if n < 0:
            raise KeyError(name)
        return out[:n].copy()

    def build_diagonals(self, cfl):
        self._check(lib().orc_build_diagonals(self._h, cfl), "build_diagonals")

    def coupling_block(self, c, d, side, scheme):
        nv = self.nF if scheme == 0 else self.ns if scheme == 1 else self.nci
        out = np.zeros(nv * nv)
        nb = C.c_int(-1)
        st = lib().orc_coupling_block(self._h, c, d, side, scheme, _p(out), C.byref(nb))
        if st:
            return None, -1
        return out.reshape(nv, nv), nb.value


def prim_to_cons_field(mech, nd, prim):
    """Conserved SoA state from a primitive field dict (rho_s, u, T, Tv) — oracle arithmetic."""
    rho_s = np.asarray(prim["rho_s"])
    ns = rho_s.shape[0]
    shape = rho_s.shape[1:]
    ncell = int(np.prod(shape))
    rs = rho_s.reshape(ns, ncell)
    u = np.asarray(prim["u"]).reshape(nd, ncell)
    T = np.asarray(prim["T"]).reshape(ncell)
    Tv = np.asarray(prim.get("Tv", prim["T"])).reshape(ncell)
    info = gas_info(mech)
    nq = ns + nd + 1 + (info["ntemp"] == 2)
    Q = np.zeros((nq, ncell))
    for c in range(ncell):
        Q[:, c] = state_cons(mech, nd, rs[:, c], u[:, c], T[c], Tv[c])
    return Q
