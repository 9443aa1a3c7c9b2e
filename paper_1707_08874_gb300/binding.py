"""Thin ctypes binding of ``libclselinv.so`` (C ABI in ``include/clselinv.h``).

Argument marshalling only: every step of the drift evaluation runs in the CUDA
library.  Device arrays are torch tensors (complex128, CUDA, contiguous); the
stream is torch's current stream unless one is given.  There is no CPU path:
if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

CL_OK = 0
CL_ERR_INVALID_ARG = 1
CL_ERR_OOM = 2
CL_ERR_CUDA = 3
CL_ERR_SINGULAR = 4
CL_ERR_NONFINITE = 5
CL_ERR_TIMEOUT = 6
CL_ERR_UNSUPPORTED = 7
CL_FP64 = 0
CL_MIXED_FP32 = 1
CL_FP64_EMU = 2
CL_MIXED_BF16X3 = 3

_lib = None


class CLError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (what, error_string(code) if _lib else "?", code))


class PlanInfo(ctypes.Structure):
    _fields_ = [("Ns", ctypes.c_int), ("Nt", ctypes.c_int), ("V", ctypes.c_int), ("N", ctypes.c_int),
                ("batch", ctypes.c_int), ("precision", ctypes.c_int), ("n_supernodes", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("max_front", ctypes.c_int), ("max_pivot_block", ctypes.c_int),
                ("panel", ctypes.c_int), ("factor_flops", ctypes.c_double), ("selinv_flops", ctypes.c_double),
                ("front_bytes", ctypes.c_double), ("device_bytes", ctypes.c_double),
                ("launches_per_eval", ctypes.c_int), ("workspace_bytes", ctypes.c_double),
                ("n_shapes", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double)]


class TraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("phase", ctypes.c_int), ("op", ctypes.c_int), ("stream", ctypes.c_int),
                ("level", ctypes.c_int), ("t0_us", ctypes.c_double), ("t1_us", ctypes.c_double)]


class LangevinParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("m", ctypes.c_double), ("mu", ctypes.c_double), ("nf", ctypes.c_double),
                ("eps_max", ctypes.c_double), ("kappa", ctypes.c_double), ("alpha_cool", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("n_cool", ctypes.c_int), ("fermions", ctypes.c_int),
                ("renorm_det", ctypes.c_int), ("reunit", ctypes.c_int)]


OBS_FIELDS = ["plaq_s_re", "plaq_s_im", "plaq_t_re", "plaq_t_im", "poly_re", "poly_im", "poly_inv_re",
              "poly_inv_im", "cond_re", "cond_im", "unitarity", "kmax", "eps", "t", "step", "spare",
              "density_re", "density_im", "spare2", "spare3"]
OBS_LEN = len(OBS_FIELDS)


def obs_dict(row) -> dict:
    """One replica's observables record (20 doubles) as a dict of complex / float values."""
    r = [float(x) for x in row]
    return dict(plaq_s=complex(r[0], r[1]), plaq_t=complex(r[2], r[3]), poly=complex(r[4], r[5]),
                poly_inv=complex(r[6], r[7]), condensate=complex(r[8], r[9]), unitarity=r[10], kmax=r[11],
                eps=r[12], t=r[13], step=r[14], density=complex(r[16], r[17]))


EXPORTS = ["cl_analyze", "cl_analyze_symbolic", "cl_factor", "cl_selinv_blocks", "cl_fermion_drift",
           "cl_drift_eval", "cl_get_status", "cl_plan_get_info", "cl_plan_get_node", "cl_profile_enable",
           "cl_profile_read", "cl_profile_trace", "cl_plan_pivot_growth", "cl_measure_peak", "cl_drift_eval_noalloc", "cl_gauge_drift", "cl_link_update", "cl_gauge_cool",
           "cl_observables", "cl_langevin_step", "cl_analyze_ex", "cl_group_create", "cl_group_drift_eval",
           "cl_group_capture", "cl_group_launch", "cl_group_destroy", "cl_destroy_plan", "cl_error_string",
           "cl_zgemm_emu_workspace", "cl_zgemm_emu", "cl_plan_check_schedule",
           "cl_analyze_symbolic_ex", "cl_plan_export", "cl_plan_set_wait_limit", "cl_analyze_ragged",
           "cl_analyze_ragged_ex", "cl_analyze_ragged_symbolic", "cl_stochastic_workspace", "cl_left_solve",
           "cl_stochastic_drift"]

# cl_plan_export tables (include/clselinv.h) and their int64 row widths
TABLES = {"meta": (0, 11), "factor_ops": (1, 11), "selinv_ops": (2, 11), "gemm": (3, 20), "panel": (4, 9),
          "copy": (5, 14), "extadd": (6, 11), "gather": (7, 7), "maps": (8, 1), "off": (9, 1), "ld": (10, 1),
          "segments": (11, 8), "vnodes": (12, 18), "vsites": (13, 1), "unperm": (14, 6),
          "node_panels": (15, 1)}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError("libclselinv.so is not built: run paper_1707_08874_gb300.build.build()")
        _build.build()
    L = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.cl_analyze.argtypes = [I, I, I, I, ctypes.POINTER(P)]
    L.cl_analyze_symbolic.argtypes = [I, I, I, ctypes.POINTER(P)]
    L.cl_analyze_symbolic_ex.argtypes = [I, I, I, I, ctypes.POINTER(P)]
    L.cl_factor.argtypes = [P, P, D, D, P]
    L.cl_selinv_blocks.argtypes = [P, P, P, P, P]
    L.cl_fermion_drift.argtypes = [P, P, P, P, D, D, P, P]
    L.cl_drift_eval.argtypes = [P, P, D, D, D, P, P, P, P, P]
    L.cl_get_status.argtypes = [P, P, ctypes.POINTER(I), ctypes.POINTER(I)]
    L.cl_plan_get_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
    L.cl_plan_get_node.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I),
                                   ctypes.POINTER(I), P, P]
    L.cl_profile_enable.argtypes = [P, I]
    L.cl_profile_read.argtypes = [P, ctypes.POINTER(ProfileEntry), I, ctypes.POINTER(I)]
    L.cl_profile_trace.argtypes = [P, ctypes.POINTER(TraceEntry), I, ctypes.POINTER(I)]
    L.cl_plan_pivot_growth.argtypes = [P, P, ctypes.POINTER(D)]
    L.cl_measure_peak.argtypes = [I, ctypes.POINTER(D)]
    L.cl_drift_eval_noalloc.argtypes = [I, I, P, D, D, D, P, P, P, P, P]
    L.cl_gauge_drift.argtypes = [P, P, D, P, P]
    L.cl_link_update.argtypes = [P, P, P, D, ctypes.c_ulonglong, ctypes.c_longlong, P]
    L.cl_gauge_cool.argtypes = [P, P, I, D, P]
    L.cl_observables.argtypes = [P, P, P, P, P, D, D, P, P]
    L.cl_langevin_step.argtypes = [P, P, ctypes.POINTER(LangevinParams), P, P, P]
    L.cl_analyze_ex.argtypes = [I, I, I, I, I, ctypes.POINTER(P)]
    PP = ctypes.POINTER(P)
    L.cl_group_create.argtypes = [I, PP, PP]
    L.cl_group_drift_eval.argtypes = [P, PP, D, D, D, PP, PP, PP, P]
    L.cl_group_capture.argtypes = [P, PP, D, D, D, PP, PP, PP, P]
    L.cl_group_launch.argtypes = [P, P]
    L.cl_group_destroy.argtypes = [P]
    L.cl_group_destroy.restype = None
    L.cl_zgemm_emu_workspace.argtypes = [I, I, I, ctypes.POINTER(ctypes.c_size_t)]
    L.cl_plan_check_schedule.argtypes = [P, I, ctypes.POINTER(ctypes.c_longlong), ctypes.c_char_p, I]
    L.cl_plan_export.argtypes = [P, I, P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
    L.cl_zgemm_emu.argtypes = [I, I, I, P, I, P, I, P, I, I, I, P, ctypes.c_size_t, P, P]
    L.cl_plan_set_wait_limit.argtypes = [P, D]
    IA = ctypes.POINTER(I)
    L.cl_analyze_ragged.argtypes = [I, IA, IA, IA, I, ctypes.POINTER(P)]
    L.cl_analyze_ragged_ex.argtypes = [I, IA, IA, IA, I, I, ctypes.POINTER(P)]
    L.cl_analyze_ragged_symbolic.argtypes = [I, IA, IA, IA, I, I, ctypes.POINTER(P)]
    L.cl_stochastic_workspace.argtypes = [P, I, ctypes.POINTER(ctypes.c_size_t)]
    L.cl_left_solve.argtypes = [P, P, I, P, P, ctypes.c_size_t, P]
    L.cl_stochastic_drift.argtypes = [P, P, D, D, D, P, I, P, P, P, P, P, P, ctypes.c_size_t, P]
    L.cl_destroy_plan.argtypes = [P]
    L.cl_destroy_plan.restype = None
    L.cl_error_string.argtypes = [I]
    L.cl_error_string.restype = ctypes.c_char_p
    for f in EXPORTS:
        if f not in ("cl_destroy_plan", "cl_error_string", "cl_group_destroy"):
            getattr(L, f).restype = I
    _lib = L
    return L


def error_string(code: int) -> str:
    return load().cl_error_string(code).decode()


def measure_peak(unit: int) -> float:
    """GFLOP/s of the current device: 0 = FP64 MMA, 1 = FP64 FMA, 2 = FP32 FMA."""
    g = ctypes.c_double()
    _check(load().cl_measure_peak(unit, ctypes.byref(g)), "cl_measure_peak")
    return g.value


def drift_eval_noalloc(Ns: int, Nt: int, links, m: float, mu: float, nf: float, Gdiag, Gfwd, Gbwd, Kf,
                       stream=None) -> int:
    """cl_drift_eval_noalloc (no device allocation; small lattices); returns the status code."""
    return load().cl_drift_eval_noalloc(Ns, Nt, _dev(links, "links"), float(m), float(mu), float(nf),
                                        _dev(Gdiag, "Gdiag"), _dev(Gfwd, "Gfwd"), _dev(Gbwd, "Gbwd"),
                                        _dev(Kf, "Kf"), _stream(stream))


def zgemm_emu(A, B, C=None, beta: bool = False, neg: bool = False, stream=None):
    """C = [C] +/- A @ B through cl_zgemm_emu (complex128 CUDA tensors, 2-D,
    row-major with unit column stride).  Returns (C, status code of the
    device status word)."""
    import torch
    L = load()
    M, K = A.shape
    K2, N = B.shape
    if K2 != K:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.zeros((M, N), dtype=torch.complex128, device=A.device)
    nbytes = ctypes.c_size_t()
    _check(L.cl_zgemm_emu_workspace(M, N, K, ctypes.byref(nbytes)), "cl_zgemm_emu_workspace")
    work = torch.empty(nbytes.value, dtype=torch.uint8, device=A.device)
    status = torch.zeros(4, dtype=torch.int32, device=A.device)
    for t, n in ((A, "A"), (B, "B"), (C, "C")):
        if not (t.is_cuda and t.dtype == torch.complex128 and t.dim() == 2 and t.stride(1) == 1):
            raise TypeError("%s must be a 2-D complex128 CUDA tensor with unit column stride" % n)
    _check(L.cl_zgemm_emu(M, N, K, ctypes.c_void_p(A.data_ptr()), A.stride(0), ctypes.c_void_p(B.data_ptr()),
                          B.stride(0), ctypes.c_void_p(C.data_ptr()), C.stride(0), int(beta), int(neg),
                          ctypes.c_void_p(work.data_ptr()), nbytes.value, ctypes.c_void_p(status.data_ptr()),
                          _stream(stream)), "cl_zgemm_emu")
    torch.cuda.synchronize()
    return C, int(status[0].item())


def _check(code: int, what: str):
    if code != CL_OK:
        raise CLError(code, what)


def _dev(t, name, shape_tail=None):
    """data_ptr of a contiguous complex128 CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous complex128 CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A plan of cl_analyze: one lattice shape, `batch` replicas, one precision."""

    def __init__(self, handle, symbolic: bool):
        self._h = handle
        self.symbolic = symbolic
        self.info = self.get_info()

    # -- construction ----------------------------------------------------
    @classmethod
    def analyze(cls, Ns: int, Nt: int, batch: int = 1, precision: int = CL_FP64) -> "Plan":
        h = ctypes.c_void_p()
        _check(load().cl_analyze(Ns, Nt, batch, precision, ctypes.byref(h)), "cl_analyze")
        return cls(h, False)

    @classmethod
    def analyze_ex(cls, Ns: int, Nt: int, batch: int, precision: int, panel: int) -> "Plan":
        h = ctypes.c_void_p()
        _check(load().cl_analyze_ex(Ns, Nt, batch, precision, panel, ctypes.byref(h)), "cl_analyze_ex")
        return cls(h, False)

    @classmethod
    def analyze_ragged(cls, shapes, precision: int = CL_FP64_EMU, panel: int = 0, symbolic: bool = False) -> "Plan":
        """cl_analyze_ragged_ex (or its host half) over shapes = [(Ns, Nt,
        count), ...]: the site-indexed arrays of every lattice concatenated in
        shape order."""
        n = len(shapes)
        arr = lambda k: (ctypes.c_int * n)(*[int(sh[k]) for sh in shapes])
        h = ctypes.c_void_p()
        fn = load().cl_analyze_ragged_symbolic if symbolic else load().cl_analyze_ragged_ex
        _check(fn(n, arr(0), arr(1), arr(2), precision, panel, ctypes.byref(h)), "cl_analyze_ragged")
        plan = cls(h, symbolic)
        plan.shapes = [tuple(int(x) for x in sh) for sh in shapes]
        return plan

    @classmethod
    def analyze_symbolic(cls, Ns: int, Nt: int, precision: int = CL_FP64, panel: int = 0) -> "Plan":
        h = ctypes.c_void_p()
        _check(load().cl_analyze_symbolic_ex(Ns, Nt, precision, panel, ctypes.byref(h)), "cl_analyze_symbolic_ex")
        return cls(h, True)

    def close(self):
        if self._h:
            load().cl_destroy_plan(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- host queries ------------------------------------------------------
    def get_info(self) -> dict:
        inf = PlanInfo()
        _check(load().cl_plan_get_info(self._h, ctypes.byref(inf)), "cl_plan_get_info")
        return inf.as_dict()

    def check_schedule(self, ignore_waits: bool = False):
        """Host race check of the two-stream factor schedule: (conflicts, first)."""
        n = ctypes.c_longlong()
        buf = ctypes.create_string_buffer(256)
        _check(load().cl_plan_check_schedule(self._h, int(ignore_waits), ctypes.byref(n), buf, 256),
               "cl_plan_check_schedule")
        return n.value, buf.value.decode()

    def export_tables(self) -> dict:
        """The plan's schedule tables (cl_plan_export) as int64 numpy arrays,
        one row per descriptor."""
        import numpy as np
        L = load()
        out = {}
        for name, (table, width) in TABLES.items():
            n = ctypes.c_longlong()
            _check(L.cl_plan_export(self._h, table, None, 0, ctypes.byref(n)), "cl_plan_export")
            a = np.zeros(max(n.value, 1), dtype=np.int64)
            _check(L.cl_plan_export(self._h, table, ctypes.c_void_p(a.ctypes.data), n.value, ctypes.byref(n)),
                   "cl_plan_export")
            out[name] = a[:n.value].reshape(-1, width) if width > 1 else a[:n.value]
        return out

    def node(self, i: int) -> dict:
        L = load()
        par, lev, ns, nb = (ctypes.c_int() for _ in range(4))
        _check(L.cl_plan_get_node(self._h, i, ctypes.byref(par), ctypes.byref(lev), ctypes.byref(ns),
                                  ctypes.byref(nb), None, None), "cl_plan_get_node")
        sep = np.empty(ns.value, np.int32)
        bnd = np.empty(nb.value, np.int32)
        _check(L.cl_plan_get_node(self._h, i, None, None, None, None, sep.ctypes.data_as(ctypes.c_void_p),
                                  bnd.ctypes.data_as(ctypes.c_void_p)), "cl_plan_get_node")
        return dict(parent=par.value, level=lev.value, sep=sep, bnd=bnd)

    # -- compute calls (stream-ordered, no host sync) -----------------------
    def factor(self, links, m: float, mu: float, stream=None):
        _check(load().cl_factor(self._h, _dev(links, "links"), float(m), float(mu), _stream(stream)), "cl_factor")

    def selinv_blocks(self, Gdiag, Gfwd, Gbwd, stream=None):
        _check(load().cl_selinv_blocks(self._h, _dev(Gdiag, "Gdiag"), _dev(Gfwd, "Gfwd"), _dev(Gbwd, "Gbwd"),
                                       _stream(stream)), "cl_selinv_blocks")

    def fermion_drift(self, links, Gfwd, Gbwd, mu: float, nf: float, Kf, stream=None):
        _check(load().cl_fermion_drift(self._h, _dev(links, "links"), _dev(Gfwd, "Gfwd"), _dev(Gbwd, "Gbwd"),
                                       float(mu), float(nf), _dev(Kf, "Kf"), _stream(stream)),
               "cl_fermion_drift")

    def drift_eval(self, links, m: float, mu: float, nf: float, Gdiag, Gfwd, Gbwd, Kf, stream=None):
        _check(load().cl_drift_eval(self._h, _dev(links, "links"), float(m), float(mu), float(nf),
                                    _dev(Gdiag, "Gdiag"), _dev(Gfwd, "Gfwd"), _dev(Gbwd, "Gbwd"),
                                    _dev(Kf, "Kf"), _stream(stream)), "cl_drift_eval")

    # -- stochastic estimator (Eq. 7) -----------------------------------------
    def _stoch_work(self, n: int):
        import torch
        nbytes = ctypes.c_size_t()
        _check(load().cl_stochastic_workspace(self._h, int(n), ctypes.byref(nbytes)), "cl_stochastic_workspace")
        return torch.empty(max(16, nbytes.value), dtype=torch.uint8, device="cuda"), nbytes.value

    def left_solve(self, eta, w, stream=None):
        """cl_left_solve: w_i = eta_i^dag D^{-1} after factor(); eta, w [n][sites][3]."""
        work, nb = self._stoch_work(eta.shape[0])
        _check(load().cl_left_solve(self._h, _dev(eta, "eta"), int(eta.shape[0]), _dev(w, "w"),
                                    ctypes.c_void_p(work.data_ptr()), nb, _stream(stream)), "cl_left_solve")
        return work

    def stochastic_drift(self, links, m: float, mu: float, nf: float, eta, w, Gdiag, Gfwd, Gbwd, Kf, stream=None):
        """cl_stochastic_drift (Eq. 7): factor, left solves, estimated blocks, drift.
        Returns the workspace tensor (keep it alive until the stream is done)."""
        work, nb = self._stoch_work(eta.shape[0])
        _check(load().cl_stochastic_drift(self._h, _dev(links, "links"), float(m), float(mu), float(nf),
                                          _dev(eta, "eta"), int(eta.shape[0]), _dev(w, "w"), _dev(Gdiag, "Gdiag"),
                                          _dev(Gfwd, "Gfwd"), _dev(Gbwd, "Gbwd"), _dev(Kf, "Kf"),
                                          ctypes.c_void_p(work.data_ptr()), nb, _stream(stream)),
               "cl_stochastic_drift")
        return work

    def set_wait_limit(self, seconds: float):
        """cl_plan_set_wait_limit: limit of the tensor-core GEMM waits (< 0: default 0.5 s)."""
        _check(load().cl_plan_set_wait_limit(self._h, float(seconds)), "cl_plan_set_wait_limit")

    def get_status(self, stream=None):
        info = ctypes.c_int()
        detail = (ctypes.c_int * 2)()
        _check(load().cl_get_status(self._h, _stream(stream), ctypes.byref(info), detail), "cl_get_status")
        return info.value, (detail[0], detail[1])

    # -- Langevin pieces ---------------------------------------------------
    def _dbl(self, t, name):
        import torch
        if t is None:
            return None
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
        return ctypes.c_void_p(t.data_ptr())

    def gauge_drift(self, links, beta: float, Kg, stream=None):
        _check(load().cl_gauge_drift(self._h, _dev(links, "links"), float(beta), _dev(Kg, "Kg"), _stream(stream)),
               "cl_gauge_drift")

    def link_update(self, links, K, eps: float, seed: int, step: int, stream=None):
        _check(load().cl_link_update(self._h, _dev(links, "links"), _dev(K, "K"), float(eps), int(seed), int(step),
                                     _stream(stream)), "cl_link_update")

    def gauge_cool(self, links, n_cool: int, alpha0: float, stream=None):
        _check(load().cl_gauge_cool(self._h, _dev(links, "links"), int(n_cool), float(alpha0), _stream(stream)),
               "cl_gauge_cool")

    def observables(self, links, Gdiag, Gfwd, Gbwd, mu: float, nf: float, obs, stream=None):
        _check(load().cl_observables(self._h, _dev(links, "links"), _dev(Gdiag, "Gdiag"), _dev(Gfwd, "Gfwd"),
                                     _dev(Gbwd, "Gbwd"), float(mu), float(nf), self._dbl(obs, "obs"),
                                     _stream(stream)), "cl_observables")

    def langevin_step(self, links, params: dict, state, obs, stream=None):
        prm = LangevinParams(**params)
        _check(load().cl_langevin_step(self._h, _dev(links, "links"), ctypes.byref(prm), self._dbl(state, "state"),
                                       self._dbl(obs, "obs"), _stream(stream)), "cl_langevin_step")

    def profile_enable(self, on: bool = True):
        _check(load().cl_profile_enable(self._h, 1 if on else 0), "cl_profile_enable")

    def profile_read(self) -> dict:
        buf = (ProfileEntry * 16)()
        n = ctypes.c_int()
        _check(load().cl_profile_read(self._h, buf, 16, ctypes.byref(n)), "cl_profile_read")
        return {buf[i].name.decode(): dict(launches=buf[i].launches, total_ms=buf[i].total_ms,
                                           flops=buf[i].flops, bytes=buf[i].bytes) for i in range(n.value)}

    def pivot_growth(self, stream=None) -> float:
        """cl_plan_pivot_growth: the largest max|entry| / min|pivot| over the
        panel blocks of the latest factorisation."""
        g = ctypes.c_double()
        _check(load().cl_plan_pivot_growth(self._h, _stream(stream), ctypes.byref(g)), "cl_plan_pivot_growth")
        return g.value

    def profile_trace(self) -> list:
        """Per-launch timeline of the profiled calls since profile_enable: one
        dict per launch (name, phase, op, stream, level, t0_us, t1_us)."""
        n = ctypes.c_int()
        _check(load().cl_profile_trace(self._h, None, 0, ctypes.byref(n)), "cl_profile_trace")
        buf = (TraceEntry * max(1, n.value))()
        _check(load().cl_profile_trace(self._h, buf, n.value, ctypes.byref(n)), "cl_profile_trace")
        return [dict(name=b.name.decode(), phase=b.phase, op=b.op, stream=b.stream, level=b.level,
                     t0_us=b.t0_us, t1_us=b.t1_us) for b in buf[:n.value]]

    # -- convenience: allocate outputs and run one evaluation --------------
    def alloc_outputs(self):
        """Output arrays of a drift evaluation: [batch][V]... for one shape, one
        [sites of all lattices]... row (leading dimension 1) for a ragged plan."""
        import torch
        B, V = self.info["batch"], self.info["V"]
        if self.info["n_shapes"] > 1 or getattr(self, "shapes", None):
            B = 1  # ragged: V counts the sites of all lattices
        kw = dict(dtype=torch.complex128, device="cuda")
        return dict(Gdiag=torch.empty((B, V, 3, 3), **kw), Gfwd=torch.empty((B, V, 4, 3, 3), **kw),
                    Gbwd=torch.empty((B, V, 4, 3, 3), **kw), Kf=torch.empty((B, V, 4, 8), **kw))


class Group:
    """cl_group: plans of several lattice shapes evaluated side by side, with
    optional CUDA-graph capture of the whole schedule."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        self._h = ctypes.c_void_p()
        _check(load().cl_group_create(len(self.plans), arr, ctypes.byref(self._h)), "cl_group_create")

    @staticmethod
    def _ptrs(ts, name):
        return (ctypes.c_void_p * len(ts))(*[_dev(t, name).value for t in ts])

    def drift_eval(self, links, m, mu, nf, Gfwd, Gbwd, Kf, stream=None):
        _check(load().cl_group_drift_eval(self._h, self._ptrs(links, "links"), float(m), float(mu), float(nf),
                                          self._ptrs(Gfwd, "Gfwd"), self._ptrs(Gbwd, "Gbwd"),
                                          self._ptrs(Kf, "Kf"), _stream(stream)), "cl_group_drift_eval")

    def capture(self, links, m, mu, nf, Gfwd, Gbwd, Kf, stream=None):
        _check(load().cl_group_capture(self._h, self._ptrs(links, "links"), float(m), float(mu), float(nf),
                                       self._ptrs(Gfwd, "Gfwd"), self._ptrs(Gbwd, "Gbwd"),
                                       self._ptrs(Kf, "Kf"), _stream(stream)), "cl_group_capture")

    def launch(self, stream=None):
        _check(load().cl_group_launch(self._h, _stream(stream)), "cl_group_launch")

    def close(self):
        if self._h:
            load().cl_group_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
