"""Python binding of the GB300 component-splitting LU-SGS library (``include/cs.h``).

Argument marshalling only: every step of the iteration runs in the library's CUDA kernels.
Arrays may be numpy arrays (host memory) or CUDA torch tensors (device memory); both are
passed to the C ABI as plain pointers.  The library must have been built (``build()``); if it
is missing, loading raises — there is no CPU fallback.
"""
import ctypes as C
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libcs_gb300.so")
SOURCES = ["launch_air11_2d.cu", "launch_air11_3d.cu", "launch_air5_2d.cu", "launch_air5_3d.cu",
           "launch_perfect_2d.cu", "launch_perfect_3d.cu", "capi.cu", "noalloc.cu", "probe.cu", "mlp.cu",
           "species_box.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC"]

CS_OK, CS_ERR_ARG, CS_ERR_OOM, CS_ERR_CUDA, CS_ERR_NONPHYSICAL, CS_ERR_NEWTON, \
    CS_ERR_TIMEOUT, CS_ERR_STATE = range(8)
SCHEME_SPLIT, SCHEME_COUPLED = 0, 1
STATUS_NAMES = {0: "CS_OK", 1: "CS_ERR_ARG", 2: "CS_ERR_OOM", 3: "CS_ERR_CUDA",
                4: "CS_ERR_NONPHYSICAL", 5: "CS_ERR_NEWTON", 6: "CS_ERR_TIMEOUT",
                7: "CS_ERR_STATE"}


def _nvcc():
    for cand in ("nvcc", "/usr/local/cuda/bin/nvcc"):
        try:
            subprocess.run([cand, "--version"], check=True, capture_output=True)
            return cand
        except (OSError, subprocess.CalledProcessError):
            continue
    raise RuntimeError("nvcc not found")


def build(force=False, jobs=8):
    """Compile the CUDA sources for sm_103a (in parallel) and link the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [os.path.join(_CSRC, f) for f in os.listdir(_CSRC)]
    deps.append(os.path.join(_HERE, "..", "include", "cs.h"))
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(_BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(_CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj

    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp,
                        *objs, "-lcudart"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class cs_grid_desc(C.Structure):
    _fields_ = [("ndim", C.c_int), ("ni", C.c_int), ("nj", C.c_int), ("nk", C.c_int),
                ("bc", C.c_int * 6), ("mech", C.c_int), ("limiter", C.c_int),
                ("entropy_fix", C.c_double), ("reacting", C.c_int)]


class cs_freestream(C.Structure):
    _fields_ = [("T", C.c_double), ("Tv", C.c_double), ("p", C.c_double), ("mach", C.c_double),
                ("Y", C.c_double * 16), ("dir", C.c_double * 3)]


class cs_wall(C.Structure):
    _fields_ = [("Tw", C.c_double), ("catalytic", C.c_int)]


class cs_step_opts(C.Structure):
    _fields_ = [("scheme", C.c_int), ("correction", C.c_int), ("clip", C.c_int),
                ("cfl", C.c_double), ("cfl_start", C.c_double), ("ramp_iters", C.c_int),
                ("precision", C.c_int), ("iters", C.c_int)]


class cs_step_stats(C.Structure):
    _fields_ = [("iters_done", C.c_int), ("r_species", C.c_double), ("r_energy", C.c_double),
                ("q_stag", C.c_double), ("nclip", C.c_int), ("status_cell", C.c_int)]


EXPORTS = ["cs_grid_create", "cs_grid_destroy", "cs_grid_dims", "cs_set_boundary",
           "cs_set_state", "cs_load_state", "cs_init_freestream", "cs_get_state", "cs_residual",
           "cs_lusgs_split", "cs_lusgs_coupled", "cs_correct", "cs_step", "cs_get_field",
           "cs_gas_info", "cs_profile", "cs_sweep_info", "cs_measure_fp64_rate", "cs_set_option", "cs_set_dual", "cs_dual_advance",
           "cs_residual_norms_static",
           "cs_last_error", "cs_batch_create", "cs_batch_destroy", "cs_batch_tune",
           "cs_batch_step", "cs_batch_stream", "cs_batch_last_error", "cs_mlp_create",
           "cs_mlp_destroy", "cs_mlp_get_params", "cs_mlp_forward", "cs_mlp_grad",
           "cs_mlp_train_step", "cs_mlp_last_error", "cs_surrogate_sample",
           "cs_surrogate_attach", "cs_surrogate_detach", "cs_species_box_create", "cs_species_box_destroy",
           "cs_species_box_state", "cs_species_box_step", "cs_species_box_time",
           "cs_species_box_last_error"]

_lib = None


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} (call build())")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    L.cs_grid_create.argtypes = [C.POINTER(cs_grid_desc), vp, vp, C.POINTER(vp)]
    L.cs_grid_destroy.argtypes = [vp]
    L.cs_grid_dims.argtypes = [vp, ip]
    L.cs_set_boundary.argtypes = [vp, C.POINTER(cs_freestream), C.POINTER(cs_wall)]
    L.cs_set_state.argtypes = [vp, vp]
    L.cs_load_state.argtypes = [vp, vp]
    L.cs_measure_fp64_rate.argtypes = [vp, dp]
    L.cs_init_freestream.argtypes = [vp]
    L.cs_get_state.argtypes = [vp, vp]
    L.cs_residual.argtypes = [vp, vp, dp]
    L.cs_lusgs_split.argtypes = [vp, C.c_double, C.c_int, vp]
    L.cs_lusgs_coupled.argtypes = [vp, C.c_double, vp]
    L.cs_correct.argtypes = [vp, C.c_int, C.c_int, vp, ip]
    L.cs_step.argtypes = [vp, C.POINTER(cs_step_opts), C.POINTER(cs_step_stats)]
    L.cs_get_field.argtypes = [vp, C.c_char_p, vp, ip]
    L.cs_gas_info.argtypes = [C.c_int, dp, dp, ip]
    L.cs_profile.argtypes = [vp, C.c_int, dp, C.POINTER(C.c_long)]
    L.cs_sweep_info.argtypes = [vp, ip]
    L.cs_set_option.argtypes = [vp, C.c_char_p, C.c_double]
    L.cs_set_dual.argtypes = [vp, C.c_double, C.c_double]
    dp = C.POINTER(C.c_double)
    L.cs_species_box_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp,
                                        C.c_double, C.c_double, dp, C.POINTER(vp)]
    L.cs_species_box_destroy.argtypes = [vp]
    L.cs_species_box_state.argtypes = [vp, vp]
    L.cs_species_box_step.argtypes = [vp, C.c_int, C.c_double, vp, vp]
    L.cs_species_box_time.argtypes = [vp, C.c_int, C.c_double, vp, vp, C.c_int, vp, C.c_size_t, dp]
    L.cs_species_box_last_error.argtypes = [vp]
    L.cs_species_box_last_error.restype = C.c_char_p
    L.cs_dual_advance.argtypes = [vp]
    L.cs_last_error.argtypes = [vp]
    L.cs_batch_create.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp)]
    L.cs_batch_destroy.argtypes = [vp]
    L.cs_batch_tune.argtypes = [vp, C.c_int, C.c_int, ip]
    L.cs_batch_step.argtypes = [vp, C.POINTER(cs_step_opts), C.c_int, C.c_int, C.POINTER(cs_step_stats)]
    L.cs_batch_stream.argtypes = [vp, C.POINTER(vp)]
    L.cs_batch_last_error.argtypes = [vp]
    fp = C.POINTER(C.c_float)
    L.cs_mlp_create.argtypes = [C.c_int, fp, C.POINTER(vp)]
    L.cs_mlp_destroy.argtypes = [vp]
    L.cs_mlp_get_params.argtypes = [vp, fp]
    L.cs_mlp_forward.argtypes = [vp, vp, C.c_int, vp]
    L.cs_mlp_grad.argtypes = [vp, vp, vp, C.c_int, fp, dp]
    L.cs_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, C.c_float, dp]
    L.cs_mlp_last_error.argtypes = [vp]
    L.cs_surrogate_sample.argtypes = [vp, vp, vp]
    L.cs_surrogate_attach.argtypes = [vp, vp, vp]
    L.cs_surrogate_detach.argtypes = [vp]
    for name in EXPORTS:
        getattr(L, name).restype = C.c_char_p if name.endswith("last_error") else C.c_int
    _lib = L
    return L


class CSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (device or host)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or a.dtype.itemsize != 8:
            raise ValueError("tensor must be contiguous float64")
        return C.c_void_p(a.data_ptr())
    if not (a.flags["C_CONTIGUOUS"] and a.dtype == np.float64):
        raise ValueError("array must be C-contiguous float64")
    return C.c_void_p(a.ctypes.data)


def gas_info(mech):
    M = np.zeros(16)
    hf = np.zeros(16)
    dims = np.zeros(3, dtype=np.int32)
    st = lib().cs_gas_info(mech, M.ctypes.data_as(C.POINTER(C.c_double)),
                           hf.ctypes.data_as(C.POINTER(C.c_double)),
                           dims.ctypes.data_as(C.POINTER(C.c_int)))
    if st:
        raise CSError(st, "cs_gas_info")
    ns = int(dims[0])
    return dict(ns=ns, nr=int(dims[1]), ntemp=int(dims[2]), M=M[:ns].copy(), hf=hf[:ns].copy())


def measure_fp64_rate(stream=None):
    """FP64 FMA throughput of the current device, GFLOP/s (cs_measure_fp64_rate)."""
    out = C.c_double()
    st = lib().cs_measure_fp64_rate(C.c_void_p(stream) if stream else None, C.byref(out))
    if st:
        raise CSError(st, "cs_measure_fp64_rate")
    return out.value


class Grid:
    """A structured grid with its state on the current CUDA device (one C-ABI grid object)."""

    def __init__(self, nodes, bc, mech, limiter=1, efix=0.1, reacting=True, stream=None):
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        nd = nodes.shape[0]
        d = cs_grid_desc()
        d.ndim = nd
        if nd == 2:
            d.nj, d.ni, d.nk = nodes.shape[1] - 1, nodes.shape[2] - 1, 1
        else:
            d.nk, d.nj, d.ni = nodes.shape[1] - 1, nodes.shape[2] - 1, nodes.shape[3] - 1
        for k in range(6):
            d.bc[k] = int(bc[k])
        d.mech, d.limiter, d.entropy_fix, d.reacting = mech, limiter, efix, int(bool(reacting))
        h = C.c_void_p()
        st = lib().cs_grid_create(C.byref(d), C.c_void_p(nodes.ctypes.data),
                                  C.c_void_p(stream) if stream else None, C.byref(h))
        if st:
            raise CSError(st, "cs_grid_create")
        self._h = h
        self.nd, self.ni, self.nj, self.nk, self.mech = nd, d.ni, d.nj, d.nk, mech
        self._dims()

    def _dims(self):
        dims = (C.c_int * 8)()
        lib().cs_grid_dims(self._h, dims)
        (self.ncell, self.nq, self.nsplit, self.nci, self.ns, self.ntemp, self.nF,
         self.stag_cell) = list(dims)

    def close(self):
        if getattr(self, "_h", None):
            lib().cs_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st:
            raise CSError(st, f"{what}: {lib().cs_last_error(self._h).decode()}")

    def set_boundary(self, fs, Tw=500.0):
        f = cs_freestream()
        f.T, f.Tv, f.p, f.mach = fs["T"], fs["Tv"], fs["p"], fs["mach"]
        for s, y in enumerate(fs["Y"]):
            f.Y[s] = float(y)
        for q in range(3):
            f.dir[q] = float(fs["dir"][q]) if q < len(fs["dir"]) else 0.0
        w = cs_wall()
        w.Tw, w.catalytic = Tw, 0
        self._check(lib().cs_set_boundary(self._h, C.byref(f), C.byref(w)), "cs_set_boundary")
        self._dims()

    def set_state(self, Q):
        self._check(lib().cs_set_state(self._h, _ptr(Q)), "cs_set_state")

    def load_state(self, Q):
        """Replace the state, keeping the iteration counter and temperature warm starts."""
        self._check(lib().cs_load_state(self._h, _ptr(Q)), "cs_load_state")

    def init_freestream(self):
        self._check(lib().cs_init_freestream(self._h), "cs_init_freestream")

    def get_state(self, out=None):
        if out is None:
            out = np.zeros((self.nq, self.ncell))
        self._check(lib().cs_get_state(self._h, _ptr(out)), "cs_get_state")
        return out

    def residual(self, R_out=None, want_R=True):
        if R_out is None and want_R:
            R_out = np.zeros((self.nq, self.ncell))
        norms = (C.c_double * 3)()
        self._check(lib().cs_residual(self._h, _ptr(R_out), norms), "cs_residual")
        return R_out, np.array(list(norms))

    def lusgs_split(self, cfl, out=None, want=True, precision=0):
        if out is None and want:
            out = np.zeros((self.nsplit, self.ncell))
        self._check(lib().cs_lusgs_split(self._h, cfl, precision, _ptr(out)), "cs_lusgs_split")
        return out

    def lusgs_coupled(self, cfl, out=None, want=True):
        if out is None and want:
            out = np.zeros((self.nci, self.ncell))
        self._check(lib().cs_lusgs_coupled(self._h, cfl, _ptr(out)), "cs_lusgs_coupled")
        return out

    def correct(self, mode, clip, dQ=None):
        n = C.c_int(0)
        self._check(lib().cs_correct(self._h, mode, clip, _ptr(dQ), C.byref(n)), "cs_correct")
        return n.value

    def step(self, scheme=0, correction=1, clip=1, cfl=10.0, cfl_start=1.0, ramp_iters=0,
             iters=1, precision=0):
        o = cs_step_opts()
        o.scheme, o.correction, o.clip, o.cfl, o.cfl_start = scheme, correction, clip, cfl, cfl_start
        o.ramp_iters, o.precision, o.iters = ramp_iters, precision, iters
        s = cs_step_stats()
        self._check(lib().cs_step(self._h, C.byref(o), C.byref(s)), "cs_step")
        return dict(iters_done=s.iters_done, r_species=s.r_species, r_energy=s.r_energy,
                    q_stag=s.q_stag, nclip=s.nclip)

    def surrogate_sample(self, X, T):
        """Raw features / targets of every cell into device float32 tensors [N][14], [N][22]."""
        self._check(lib().cs_surrogate_sample(self._h, X.data_ptr(), T.data_ptr()), "cs_surrogate_sample")

    def attach_surrogate(self, net, norm):
        nrm = np.ascontiguousarray(norm, dtype=np.float64)
        assert nrm.size == 72
        self._check(lib().cs_surrogate_attach(self._h, net._h, _ptr(nrm)), "cs_surrogate_attach")
        self._surrogate = net      # keep the network alive while attached

    def detach_surrogate(self):
        self._check(lib().cs_surrogate_detach(self._h), "cs_surrogate_detach")
        self._surrogate = None

    PHASES = ["primitive", "gradient", "flux", "assemble", "spectral", "sweep_fwd",
              "sweep_bwd", "correct"]

    def set_option(self, name, value):
        self._check(lib().cs_set_option(self._h, name.encode(), float(value)), "cs_set_option")

    def set_dual(self, dt, theta=0.0):
        """Dual time stepping with physical step dt (0: steady) and coefficient theta."""
        self._check(lib().cs_set_dual(self._h, float(dt), float(theta)), "cs_set_dual")

    def dual_advance(self):
        """Begin a physical time step from the current state (Q^{n-1} <- Q^n <- Q)."""
        self._check(lib().cs_dual_advance(self._h), "cs_dual_advance")

    def profile(self, enable):
        """Return {phase: (ms, launches)} accumulated since the last call; (re)arm timing."""
        ms = (C.c_double * 8)()
        nl = (C.c_long * 8)()
        self._check(lib().cs_profile(self._h, int(enable), ms, nl), "cs_profile")
        return {p: (ms[k], nl[k]) for k, p in enumerate(self.PHASES)}

    def sweep_info(self):
        """(kernel, CTAs per cluster) of the last split sweep ("cluster_sweep" numbering)."""
        out = (C.c_int * 2)()
        self._check(lib().cs_sweep_info(self._h, out), "cs_sweep_info")
        return out[0], out[1]

    def field(self, name, size=None):
        if size is None:
            size = max(64 * 3 * self.ncell, 3 * (self.ni + 1) * (self.nj + 1) * (self.nk + 1) * self.nq)
        out = np.zeros(size)
        n = C.c_int(0)
        self._check(lib().cs_get_field(self._h, name.encode(), _ptr(out), C.byref(n)), "cs_get_field")
        return out[:n.value].copy()


class Batch:
    """Independent grids stepped together: K iterations of every case captured into one CUDA
    graph and replayed (cs_batch_* of the C ABI).  The grids must outlive the batch."""

    def __init__(self, grids):
        self.grids = list(grids)
        arr = (C.c_void_p * len(self.grids))(*[g._h for g in self.grids])
        h = C.c_void_p()
        st = lib().cs_batch_create(len(self.grids), arr, C.byref(h))
        if st:
            raise CSError(st, "cs_batch_create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            lib().cs_batch_destroy(self._h)
            self._h = None

    def _check(self, st, what):
        if st:
            raise CSError(st, f"{what}: {lib().cs_batch_last_error(self._h).decode()}")

    def stream(self):
        """Address of the batch's cudaStream_t (for CUDA events around step())."""
        h = C.c_void_p()
        self._check(lib().cs_batch_stream(self._h, C.byref(h)), "cs_batch_stream")
        return h.value

    def tune(self, precision=0, trials=3):
        """Time the split sweep per case over cluster kernels and sizes; returns [(kind, C)]."""
        out = (C.c_int * (2 * len(self.grids)))()
        self._check(lib().cs_batch_tune(self._h, int(precision), int(trials), out), "cs_batch_tune")
        return [(out[2 * c], out[2 * c + 1]) for c in range(len(self.grids))]

    def step(self, opts, iters, iters_per_graph=1):
        """opts: one dict of cs_step options per case (keys as Grid.step, without iters)."""
        n = len(self.grids)
        arr = (cs_step_opts * n)()
        for c, o in enumerate(opts):
            arr[c].scheme = o.get("scheme", 0)
            arr[c].correction = o.get("correction", 1)
            arr[c].clip = o.get("clip", 1)
            arr[c].cfl = o.get("cfl", 10.0)
            arr[c].cfl_start = o.get("cfl_start", 1.0)
            arr[c].ramp_iters = o.get("ramp_iters", 0)
            arr[c].precision = o.get("precision", 0)
            arr[c].iters = iters
        stats = (cs_step_stats * n)()
        st = lib().cs_batch_step(self._h, arr, int(iters), int(iters_per_graph), stats)
        out = [dict(iters_done=s.iters_done, r_species=s.r_species, r_energy=s.r_energy,
                    q_stag=s.q_stag, nclip=s.nclip, status_cell=s.status_cell) for s in stats]
        self._check(st, "cs_batch_step")
        return out


MLP_NPARAM = 37782


class MLP:
    """The chemistry surrogate network (cs_mlp_* of the C ABI).  Inputs and targets are device
    tensors (torch float32, contiguous), passed by address."""

    def __init__(self, params, max_batch):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == MLP_NPARAM
        h = C.c_void_p()
        st = lib().cs_mlp_create(int(max_batch), p.ctypes.data_as(C.POINTER(C.c_float)), C.byref(h))
        if st:
            raise CSError(st, "cs_mlp_create")
        self._h = h
        self.max_batch = int(max_batch)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().cs_mlp_destroy(self._h)
            self._h = None

    def _check(self, st, what):
        if st:
            raise CSError(st, f"{what}: {lib().cs_mlp_last_error(self._h).decode()}")

    def params(self):
        out = np.zeros(MLP_NPARAM, dtype=np.float32)
        self._check(lib().cs_mlp_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float))),
                    "cs_mlp_get_params")
        return out

    def forward(self, X, Y):
        """X: device float32 [n][14]; Y: device float32 [n][22] (written)."""
        self._check(lib().cs_mlp_forward(self._h, X.data_ptr(), X.shape[0], Y.data_ptr()), "cs_mlp_forward")

    def grad(self, X, T):
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        loss = C.c_double()
        self._check(lib().cs_mlp_grad(self._h, X.data_ptr(), T.data_ptr(), X.shape[0],
                                      g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)), "cs_mlp_grad")
        return loss.value, g

    def train_step(self, X, T, lr):
        loss = C.c_double()
        self._check(lib().cs_mlp_train_step(self._h, X.data_ptr(), T.data_ptr(), X.shape[0],
                                            float(lr), C.byref(loss)), "cs_mlp_train_step")
        return loss.value


class SpeciesBox:
    """Uniform non-reacting flow of ns species in a box: one implicit step of the split or
    coupled operator (cs_species_box_* of the C ABI; the species-count scaling test)."""

    def __init__(self, case):
        ns = int(case["ns"])
        self.ns = ns
        self.n = tuple(int(x) for x in case["n"])
        self.ncell = self.n[0] * self.n[1] * self.n[2]

        def arr(a, k):
            a = np.ascontiguousarray(a, dtype=np.float64)
            assert a.shape == (k,)
            return a
        self._keep = [arr(case["size"], 3), arr(case["M"], ns), arr(case["dof"], ns),
                      arr(case["Y"], ns), arr(case["u"], 3)]
        size, M, dof, Y, u = self._keep
        P = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
        h = C.c_void_p()
        st = lib().cs_species_box_create(ns, *self.n, P(size), P(M), P(dof), P(Y),
                                         float(case["T"]), float(case["p"]), P(u), C.byref(h))
        if st:
            raise CSError(st, "cs_species_box_create")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            try:
                lib().cs_species_box_destroy(self._h)
            except Exception:
                pass
            self._h = None

    def _check(self, st, what):
        if st:
            raise CSError(st, f"{what}: {lib().cs_species_box_last_error(self._h).decode()}")

    def state(self):
        import torch
        Q = torch.empty((self.ns + 4, self.ncell), dtype=torch.float64, device="cuda")
        self._check(lib().cs_species_box_state(self._h, Q.data_ptr()), "cs_species_box_state")
        return Q

    def step(self, scheme, cfl, rhs, out=None):
        """rhs: device float64 [ns + 4][ncell]; returns the device increments."""
        import torch
        n = self.ns + 5 if scheme == 0 else self.ns + 4
        if out is None:
            out = torch.empty((n, self.ncell), dtype=torch.float64, device="cuda")
        self._check(lib().cs_species_box_step(self._h, scheme, float(cfl), rhs.data_ptr(),
                                              out.data_ptr()), "cs_species_box_step")
        return out

    def time(self, scheme, cfl, rhs, reps, flush=None):
        """Mean device ms of `reps` steps; flush: a device tensor written before each step."""
        import torch
        n = self.ns + 5 if scheme == 0 else self.ns + 4
        out = torch.empty((n, self.ncell), dtype=torch.float64, device="cuda")
        ms = C.c_double()
        fp = flush.data_ptr() if flush is not None else None
        fb = flush.numel() * flush.element_size() if flush is not None else 0
        self._check(lib().cs_species_box_time(self._h, scheme, float(cfl), rhs.data_ptr(),
                                              out.data_ptr(), int(reps), fp, fb, C.byref(ms)),
                    "cs_species_box_time")
        return ms.value
