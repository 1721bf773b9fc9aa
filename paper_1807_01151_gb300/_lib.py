"""ctypes binding of include/emg.h (argument marshalling only).

Loads the in-tree libemg.so built by ``paper_1807_01151_gb300.build``.  There is no
fallback: if the library is missing, loading raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libemg.so")

STATUS = {0: "EMG_OK", 1: "EMG_ERR_ARG", 2: "EMG_ERR_OOM", 3: "EMG_ERR_CUDA", 4: "EMG_ERR_NONFINITE",
          5: "EMG_ERR_UNPHYSICAL", 6: "EMG_ERR_NOT_CONVERGED", 7: "EMG_ERR_TIMEOUT", 8: "EMG_CANCELLED"}


class MeshDescC(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_nodes", C.c_int64), ("xyz", C.POINTER(C.c_double)),
                ("n_elems", C.c_int64), ("elem_nodes", C.POINTER(C.c_int64)),
                ("face_bc", C.POINTER(C.c_int32)), ("wall_normal", C.POINTER(C.c_double))]


class ParamsC(C.Structure):
    _fields_ = [("gamma", C.c_double), ("mach", C.c_double), ("alpha_deg", C.c_double),
                ("p_max", C.c_int32), ("rk_stages", C.c_int32), ("krylov_m", C.c_int32),
                ("cfl_max", C.c_double), ("exp_dt_factor", C.c_double), ("pre_smooth", C.c_int32),
                ("prec", C.c_int32), ("cuda_stream", C.c_void_p), ("lag_blocks", C.c_int32),
                ("use_graph", C.c_int32), ("autotune", C.c_int32), ("coop_krylov", C.c_int32),
                ("krylov_tol", C.c_double), ("exp_dt_global", C.c_int32), ("jac_freeze", C.c_int32),
                ("quad_extra", C.c_int32), ("omega", C.c_double * 3), ("block_kernels", C.c_int32), ("krylov_f32", C.c_int32)]


class CycleInfoC(C.Structure):
    _fields_ = [("n", C.c_int64), ("res_rho", C.c_double), ("res", C.c_double * 5), ("cfl", C.c_double),
                ("krylov_dim", C.c_int32)]


class SolveReportC(C.Structure):
    _fields_ = [("cycles", C.c_int64), ("res0", C.c_double), ("res_final", C.c_double),
                ("converged", C.c_int32)]


class ServerParamsC(C.Structure):
    _fields_ = [("mem_budget", C.c_int64), ("max_active", C.c_int32), ("drop", C.c_double),
                ("max_cycles", C.c_int64), ("keep_state", C.c_int32), ("stall_cycles", C.c_int64)]


class RequestResultC(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("cycles", C.c_int64), ("res0", C.c_double),
                ("res_final", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double), ("device_bytes", C.c_int64)]


EXPORTS = {
    "emg_default_params": (None, [C.POINTER(ParamsC)]),
    "emg_create_mesh": (C.c_int, [C.POINTER(MeshDescC), C.POINTER(ParamsC), C.POINTER(C.c_void_p)]),
    "emg_destroy": (C.c_int, [C.c_void_p]),
    "emg_last_error": (C.c_char_p, [C.c_void_p]),
    "emg_device_bytes": (C.c_int64, [C.c_void_p]),
    "emg_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "emg_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "emg_set_cycle": (C.c_int, [C.c_void_p, C.c_int64, C.c_double]),
    "emg_get_cycle": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "emg_vcycle": (C.c_int, [C.c_void_p, C.POINTER(CycleInfoC)]),
    "emg_solve_steady": (C.c_int, [C.c_void_p, C.c_double, C.c_int64, C.POINTER(SolveReportC)]),
    "emg_residual_norm": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "emg_residual": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]),
    "emg_jacobian_diag": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]),
    "emg_prk_step": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                               C.c_int32]),
    "emg_jacobian_p0": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "emg_exp1_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.POINTER(C.c_int32), C.c_int32]),
    "emg_element_geometry": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "emg_block_operator": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_void_p,
                                     C.c_int32]),
    "emg_probe_peaks": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "emg_profile_enable": (C.c_int, [C.c_void_p, C.c_int32]),
    "emg_profile_read": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "emg_profile_class_name": (C.c_char_p, [C.c_int32]),
    "emg_launch_count": (C.c_int64, [C.c_void_p]),
    "emg_graph_kernels": (C.c_int64, [C.c_void_p]),
    "emg_tuning": (C.c_char_p, [C.c_void_p]),
    "emg_selftest_wait_timeout": (C.c_int, [C.c_void_p]),
    "emg_exp1_step_noalloc": (C.c_int, [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                        C.POINTER(C.c_int32)]),
    "emg_estimate_device_bytes": (C.c_int, [C.POINTER(MeshDescC), C.POINTER(ParamsC), C.POINTER(C.c_int64)]),
    "emg_server_create": (C.c_int, [C.POINTER(ServerParamsC), C.POINTER(C.c_void_p)]),
    "emg_server_destroy": (C.c_int, [C.c_void_p]),
    "emg_server_last_error": (C.c_char_p, [C.c_void_p]),
    "emg_server_clock": (C.c_double, [C.c_void_p]),
    "emg_server_submit": (C.c_int, [C.c_void_p, C.POINTER(MeshDescC), C.POINTER(ParamsC), C.c_void_p,
                                    C.POINTER(C.c_int64)]),
    "emg_server_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "emg_server_results": (C.c_int, [C.c_void_p, C.POINTER(RequestResultC), C.c_int32, C.POINTER(C.c_int32)]),
    "emg_server_take_state": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]),
    "emg_server_cancel": (C.c_int, [C.c_void_p, C.c_int64]),
    "emg_build_info": (C.c_char_p, []),
}

PROFILE_CLASSES = 13

_lib = None


def load():
    """Load libemg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} not built: run paper_1807_01151_gb300.build.build() (nvcc, sm_103a)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class EmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _ptr(a):
    """Host numpy array -> (pointer, 0); torch CUDA tensor -> (data_ptr, 1)."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data), 0
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr()), 1
    raise TypeError("expected a numpy array or a CUDA tensor")


def mesh_desc(mesh):
    """emg_mesh_desc of a workloads.MeshDesc; returns (desc, arrays it points into)."""
    xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
    en = np.ascontiguousarray(mesh.elem_nodes, dtype=np.int64)
    fb = np.ascontiguousarray(mesh.face_bc, dtype=np.int32)
    wn = getattr(mesh, "wall_normal", None)
    wn = None if wn is None else np.ascontiguousarray(wn, dtype=np.float64)
    d = MeshDescC(int(mesh.dim), xyz.shape[1], xyz.ctypes.data_as(C.POINTER(C.c_double)), int(mesh.n_elems),
                  en.ctypes.data_as(C.POINTER(C.c_int64)), fb.ctypes.data_as(C.POINTER(C.c_int32)),
                  None if wn is None else wn.ctypes.data_as(C.POINTER(C.c_double)))
    return d, (xyz, en, fb, wn)


def make_params(p_max=2, mach=0.3, alpha_deg=0.0, gamma=1.4, rk_stages=4, krylov_m=30, cfl_max=100.0,
                exp_dt_factor=0.0, pre_smooth=2, prec=0, stream=None, lag_blocks=0, use_graph=1, autotune=1,
                coop_krylov=1, krylov_tol=0.0, exp_dt_global=0, jac_freeze=1, quad_extra=2, omega=(0.0, 0.0, 0.0),
                block_kernels=0, krylov_f32=-1):
    prm = ParamsC()
    load().emg_default_params(C.byref(prm))
    prm.gamma, prm.mach, prm.alpha_deg = gamma, mach, alpha_deg
    prm.p_max, prm.rk_stages, prm.krylov_m = p_max, rk_stages, krylov_m
    prm.cfl_max, prm.exp_dt_factor, prm.pre_smooth, prm.prec = cfl_max, exp_dt_factor, pre_smooth, prec
    prm.cuda_stream = C.c_void_p(stream) if stream else None
    prm.lag_blocks = int(lag_blocks)
    prm.use_graph = int(use_graph)
    prm.autotune = int(autotune)
    prm.coop_krylov = int(coop_krylov)
    prm.krylov_tol = float(krylov_tol)
    prm.exp_dt_global = int(exp_dt_global)
    prm.jac_freeze = int(jac_freeze)
    prm.quad_extra = int(quad_extra)
    for k in range(3):
        prm.omega[k] = float(omega[k])
    prm.block_kernels = int(block_kernels)
    prm.krylov_f32 = int(krylov_f32)
    return prm


def estimate_device_bytes(mesh, **params):
    """Device bytes a Solver of this mesh and these parameters would hold (host-only call)."""
    d, keep = mesh_desc(mesh)
    prm = make_params(**params)
    b = C.c_int64()
    st = load().emg_estimate_device_bytes(C.byref(d), C.byref(prm), C.byref(b))
    if st != 0:
        raise EmgError(st, "emg_estimate_device_bytes")
    return b.value


class Solver:
    """One eMG context (device-resident mesh, basis tables, state and work arrays)."""

    def __init__(self, mesh, p_max=2, **params):
        self.lib = load()
        self.dim = int(mesh.dim)
        self.E = int(mesh.n_elems)
        self.p_max = int(p_max)
        self.prec = int(params.get("prec", 0))
        d, self._keep = mesh_desc(mesh)
        prm = make_params(p_max=p_max, **params)
        h = C.c_void_p()
        st = self.lib.emg_create_mesh(C.byref(d), C.byref(prm), C.byref(h))
        self.h = h
        if st != 0:
            msg = self.lib.emg_last_error(h).decode() if h.value else ""
            if h.value:
                self.lib.emg_destroy(h)
            self.h = None
            raise EmgError(st, msg)

    def close(self):
        if getattr(self, "h", None):
            self.lib.emg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise EmgError(st, self.lib.emg_last_error(self.h).decode())

    def n_modes(self, p):
        return (p + 1) * (p + 2) // 2 if self.dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6

    @property
    def device_bytes(self):
        return int(self.lib.emg_device_bytes(self.h))

    def set_state(self, U=None):
        if U is None:
            self._check(self.lib.emg_set_state(self.h, None, 0))
            return
        p, dev = _ptr(U)
        self._check(self.lib.emg_set_state(self.h, p, dev))

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.E, 5, self.n_modes(self.p_max)))
        p, dev = _ptr(out)
        self._check(self.lib.emg_get_state(self.h, p, dev))
        return out

    def set_cycle(self, n, res_ref=0.0):
        self._check(self.lib.emg_set_cycle(self.h, int(n), float(res_ref)))

    def get_cycle(self):
        n, r = C.c_int64(), C.c_double()
        self._check(self.lib.emg_get_cycle(self.h, C.byref(n), C.byref(r)))
        return n.value, r.value

    def vcycle(self, info=True):
        if not info:
            self._check(self.lib.emg_vcycle(self.h, None))
            return None
        ci = CycleInfoC()
        self._check(self.lib.emg_vcycle(self.h, C.byref(ci)))
        return dict(n=ci.n, res_rho=ci.res_rho, res=list(ci.res), cfl=ci.cfl, krylov_dim=ci.krylov_dim)

    def solve_steady(self, drop=1e-10, max_cycles=1000, raise_on_fail=True):
        rep = SolveReportC()
        st = self.lib.emg_solve_steady(self.h, drop, max_cycles, C.byref(rep))
        out = dict(cycles=rep.cycles, res0=rep.res0, res_final=rep.res_final, converged=bool(rep.converged))
        if st != 0 and (raise_on_fail or st != 6):
            self._check(st)
        return out

    def residual_norm(self):
        r, r5 = C.c_double(), (C.c_double * 5)()
        self._check(self.lib.emg_residual_norm(self.h, C.byref(r), r5))
        return r.value, list(r5)

    def residual(self, p, u, out=None):
        u = np.ascontiguousarray(u, dtype=np.float64) if isinstance(u, np.ndarray) else u
        if out is None:
            out = np.empty((self.E, 5, self.n_modes(p)))
        pu, du = _ptr(u)
        po, do = _ptr(out)
        if du != do:
            raise ValueError("u and out must both be host or both be device")
        self._check(self.lib.emg_residual(self.h, p, pu, po, du))
        return out

    def jacobian_diag(self, p, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        b = 5 * self.n_modes(p)
        out = np.empty((self.E, b, b))
        self._check(self.lib.emg_jacobian_diag(self.h, p, _ptr(u)[0], _ptr(out)[0], 0))
        return out

    def prk_step(self, p, u, tau=None, cfl=1.0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.empty_like(u)
        tp = _ptr(np.ascontiguousarray(tau, dtype=np.float64))[0] if tau is not None else None
        self._check(self.lib.emg_prk_step(self.h, p, _ptr(u)[0], tp, float(cfl), _ptr(out)[0], 0))
        return out

    def block_operator(self, p, u, cfl=1.0, which=0, out=None):
        """P_e (which = 0) or the float32 explicit P_e^{-1} (which = 1) of level p at state u,
        as [E][5N][5N] float64 row-major (emg_block_operator)."""
        u = np.ascontiguousarray(u, dtype=np.float64) if isinstance(u, np.ndarray) else u
        b = 5 * self.n_modes(p)
        if out is None:
            out = np.empty((self.E, b, b))
        pu, du = _ptr(u)
        po, do = _ptr(out)
        if du != do:
            raise ValueError("u and out must both be host or both be device")
        self._check(self.lib.emg_block_operator(self.h, int(p), pu, float(cfl), int(which), po, du))
        return out

    def jacobian_p0(self, u0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        nf = 2 * self.dim
        diag = np.empty((self.E, 5, 5))
        off = np.empty((self.E, nf, 5, 5))
        nbr = np.empty((self.E, nf), dtype=np.int64)
        self._check(self.lib.emg_jacobian_p0(self.h, _ptr(u0)[0], _ptr(diag)[0], _ptr(off)[0],
                                             C.c_void_p(nbr.ctypes.data), 0))
        return diag, off, nbr

    def exp1_step(self, u0, dt, tau0=None):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        dt = np.ascontiguousarray(dt, dtype=np.float64)
        out = np.empty_like(u0)
        k = C.c_int32()
        tp = _ptr(np.ascontiguousarray(tau0, dtype=np.float64))[0] if tau0 is not None else None
        self._check(self.lib.emg_exp1_step(self.h, _ptr(u0)[0], tp, _ptr(dt)[0], _ptr(out)[0], C.byref(k), 0))
        return out, k.value

    def profile(self, on=True):
        self._check(self.lib.emg_profile_enable(self.h, 1 if on else 0))

    def profile_read(self):
        """{class name: (total ms, launches)} since profiling was enabled (synchronises)."""
        out = {}
        for k in range(PROFILE_CLASSES):
            ms, n = C.c_double(), C.c_int64()
            self._check(self.lib.emg_profile_read(self.h, k, C.byref(ms), C.byref(n)))
            out[self.lib.emg_profile_class_name(k).decode()] = (ms.value, n.value)
        return out

    @property
    def launch_count(self):
        return int(self.lib.emg_launch_count(self.h))

    @property
    def graph_kernels(self):
        return int(self.lib.emg_graph_kernels(self.h))

    @property
    def tuning(self):
        return self.lib.emg_tuning(self.h).decode()

    def element_geometry(self):
        vol = np.empty(self.E)
        h = np.empty(self.E)
        self._check(self.lib.emg_element_geometry(self.h, _ptr(vol)[0], _ptr(h)[0]))
        return vol, h


class Server:
    """Request loop with continuous batching (emg_server_*): solves of different meshes,
    orders and Mach numbers run concurrently, each in a context of its own."""

    def __init__(self, max_active=8, mem_budget=0, drop=1e-10, max_cycles=2000, keep_state=False, stall_cycles=0):
        self.lib = load()
        sp = ServerParamsC(int(mem_budget), int(max_active), float(drop), int(max_cycles), int(bool(keep_state)),
                           int(stall_cycles))
        h = C.c_void_p()
        st = self.lib.emg_server_create(C.byref(sp), C.byref(h))
        if st != 0:
            raise EmgError(st, "emg_server_create")
        self.h = h
        self._shape = {}

    def close(self):
        if getattr(self, "h", None):
            self.lib.emg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise EmgError(st, self.lib.emg_server_last_error(self.h).decode())

    def clock(self):
        return float(self.lib.emg_server_clock(self.h))

    def submit(self, mesh, U0=None, **params):
        """Queue one steady solve; returns its request id."""
        d, keep = mesh_desc(mesh)
        prm = make_params(**params)
        u = None
        if U0 is not None:
            u = np.ascontiguousarray(U0, dtype=np.float64)
        rid = C.c_int64()
        self._check(self.lib.emg_server_submit(self.h, C.byref(d), C.byref(prm),
                                               None if u is None else C.c_void_p(u.ctypes.data), C.byref(rid)))
        p = int(params.get("p_max", 2))
        nm = (p + 1) * (p + 2) // 2 if mesh.dim == 2 else (p + 1) * (p + 2) * (p + 3) // 6
        self._shape[rid.value] = (int(mesh.n_elems), 5, nm)
        return rid.value

    def step(self):
        """One non-blocking scheduling round; returns (active, queued)."""
        a, q = C.c_int32(), C.c_int32()
        self._check(self.lib.emg_server_step(self.h, C.byref(a), C.byref(q)))
        return a.value, q.value

    def results(self):
        """Finished requests since the last call, as dicts, in completion order."""
        out = []
        buf = (RequestResultC * 64)()
        while True:
            n = C.c_int32()
            self._check(self.lib.emg_server_results(self.h, buf, 64, C.byref(n)))
            for k in range(n.value):
                r = buf[k]
                out.append(dict(id=r.id, status=r.status, status_name=STATUS.get(r.status, str(r.status)),
                                cycles=r.cycles, res0=r.res0, res_final=r.res_final, t_submit=r.t_submit,
                                t_admit=r.t_admit, t_done=r.t_done, device_bytes=r.device_bytes))
            if n.value < 64:
                return out

    def cancel(self, rid):
        """Withdraw a queued or active request (its result reports EMG_CANCELLED)."""
        self._check(self.lib.emg_server_cancel(self.h, int(rid)))

    def take_state(self, rid):
        U = np.empty(self._shape[rid])
        self._check(self.lib.emg_server_take_state(self.h, int(rid), C.c_void_p(U.ctypes.data), U.size))
        return U


def exp1_step_noalloc(dim, diag, off, nbr, r0, dt, u0, u_out, krylov_m=30, stream=None):
    """emg_exp1_step_noalloc on CUDA tensors (device pointers only); returns the Krylov
    dimension.  Raises EmgError on a non-zero status."""
    lib = load()
    ptrs = []
    for t in (diag, off, nbr, r0, dt, u0, u_out):
        if not (hasattr(t, "data_ptr") and getattr(t, "is_cuda", False) and t.is_contiguous()):
            raise TypeError("exp1_step_noalloc takes contiguous CUDA tensors")
        ptrs.append(C.c_void_p(t.data_ptr()))
    k = C.c_int32()
    st = lib.emg_exp1_step_noalloc(int(dim), int(diag.shape[0]), *ptrs[:6], int(krylov_m),
                                   C.c_void_p(stream) if stream else None, ptrs[6], C.byref(k))
    if st != 0:
        raise EmgError(st, "emg_exp1_step_noalloc")
    return k.value


def probe_peaks():
    """Measured float64 / float32 FMA throughput of the current device (TFLOP/s) and the SM
    clock of the run (MHz), from the library's register-only probe kernels."""
    f64, f32, mhz = C.c_double(), C.c_double(), C.c_double()
    st = load().emg_probe_peaks(C.byref(f64), C.byref(f32), C.byref(mhz))
    if st != 0:
        raise EmgError(st, "emg_probe_peaks")
    return dict(fp64_tflops=f64.value, fp32_tflops=f32.value, sm_mhz=mhz.value)


def build_info():
    return load().emg_build_info().decode()
