"""ctypes binding of libgrprec.so (include/grprec.h), argument marshalling only.

The functions keep the C names.  Every step of the scheme runs in the CUDA
library; this module never computes any part of it.  Loading fails loudly when
the library is missing (there is no CPU fallback).  ``Solver`` wraps one
context for numpy (host) or torch CUDA (device) buffers.
"""
import ctypes
import os

import numpy as np

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))

GRP_ADVECTION, GRP_EULER_IDEAL = 0, 1
GRP_BC_PERIODIC, GRP_BC_TRANSMISSIVE = 0, 1
GRP_GUESS_PVRS, GRP_GUESS_TRRS, GRP_GUESS_MLP = 0, 1, 2
GRP_LAUNCH_AUTO, GRP_LAUNCH_FLAT, GRP_LAUNCH_FUSED, GRP_LAUNCH_SPLIT, GRP_LAUNCH_TILED = 0, 1, 2, 3, 4
GRP_OK = 0
GRP_NSTATS = 9
(STAT_STEPS, STAT_NEWTON_SUM, STAT_NEWTON_MAX, STAT_RECON_FB, STAT_FLUX_FB, STAT_RS_CALLS,
 STAT_LOW_ORDER, STAT_GUESS_USED, STAT_GUESS_REJECTED) = range(9)


class grp_problem(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int), ("lambda_", ctypes.c_double), ("gamma", ctypes.c_double),
                ("M", ctypes.c_int), ("cfl", ctypes.c_double), ("n_domains", ctypes.c_int),
                ("n_cells", ctypes.POINTER(ctypes.c_int)), ("x_left", ctypes.POINTER(ctypes.c_double)),
                ("x_right", ctypes.POINTER(ctypes.c_double)), ("bc", ctypes.POINTER(ctypes.c_int)),
                ("newton_rtol", ctypes.c_double), ("newton_max_iter", ctypes.c_int),
                ("guess", ctypes.c_int), ("dt_hold", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("recon", ctypes.c_int), ("solver", ctypes.c_int),
                ("source", ctypes.c_int), ("source_coef", ctypes.c_double)]


class GrpError(RuntimeError):
    pass


_lib = None
_vp = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def load(build_if_missing=True):
    """Load libgrprec.so (building it with nvcc when absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.path.join(HERE, "libgrprec.so")
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise GrpError("libgrprec.so is missing: build it with paper_2602_21911_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.grp_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(grp_problem)]
    L.grp_set_initial.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int]
    L.grp_step.argtypes = [_vp, ctypes.c_int, ctypes.c_double]
    L.grp_advance_to.argtypes = [_vp, ctypes.c_double, ctypes.c_int]
    L.grp_get_state.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int]
    L.grp_get_stats.argtypes = [_vp, _vp, _vp]
    L.grp_error_norms.argtypes = [_vp, _vp, ctypes.c_int, _vp, _vp, _vp]
    L.grp_launch_count.argtypes = [_vp]
    L.grp_launch_count.restype = ctypes.c_longlong
    L.grp_set_kernel_timing.argtypes = [_vp, ctypes.c_int]
    L.grp_get_kernel_timing.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]
    L.grp_probe_fp64_peak.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.grp_set_launch.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    _ip = ctypes.POINTER(ctypes.c_int)
    L.grp_get_launch.argtypes = [_vp, _ip, _ip, _ip, _ip, _ip]
    L.grp_step_noalloc.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), _vp]
    L.grp_set_guess_model.argtypes = [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int]
    L.grp_set_harvest.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, ctypes.c_int]
    L.grp_mlp_forward.argtypes = [_vp, _vp, ctypes.c_longlong, _vp, _vp]
    L.grp_mlp_loss_grad.argtypes = [_vp, _vp, _vp, ctypes.c_longlong, _vp, _vp, _vp, _vp]
    L.grp_mlp_adam.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, _vp]
    L.grp_riemann_batch.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, _vp, _vp,
                                    ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.grp_set_graph.argtypes = [_vp, ctypes.c_int]
    L.grp_destroy.argtypes = [_vp]
    L.grp_destroy.restype = None
    L.grp_status_string.argtypes = [ctypes.c_int]
    L.grp_status_string.restype = ctypes.c_char_p
    _lib = L
    return L


def grp_probe_fp64_peak(device=0):
    """Measured FP64 FLOP/s of the device (FMA chains; an FMA counts 2)."""
    v = ctypes.c_double(0.0)
    _check(load().grp_probe_fp64_peak(int(device), ctypes.byref(v)), "grp_probe_fp64_peak")
    return v.value


GRP_NOALLOC_MAX_CELLS = 65536
GRP_RECON_GRPREC, GRP_RECON_GRPRECNL = 0, 1
GRP_SOLVER_TT, GRP_SOLVER_DET = 0, 1
GRP_SOURCE_NONE, GRP_SOURCE_LINEAR, GRP_SOURCE_GRAVITY = 0, 1, 2
GRP_MLP_NPARAM = 4673


def mlp_work_floats(n):
    return int(n) * 257


def _dev(x, what):
    p, dev = _ptr(x)
    if not dev:
        raise GrpError("%s must be a device tensor" % what)
    return p


def grp_mlp_forward(weights, x, y, stream=None):
    _check(load().grp_mlp_forward(_dev(weights, "weights"), _dev(x, "x"), int(x.shape[0]), _dev(y, "y"),
                                  stream), "grp_mlp_forward")


def grp_mlp_loss_grad(weights, x, target, grad, loss, work, stream=None):
    _check(load().grp_mlp_loss_grad(_dev(weights, "weights"), _dev(x, "x"), _dev(target, "target"),
                                    int(x.shape[0]), _dev(grad, "grad"), _dev(loss, "loss"),
                                    _dev(work, "work"), stream), "grp_mlp_loss_grad")


def grp_mlp_adam(weights, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().grp_mlp_adam(_dev(weights, "weights"), _dev(grad, "grad"), _dev(m, "m"), _dev(v, "v"),
                               int(step), float(lr), float(beta1), float(beta2), float(eps), stream),
           "grp_mlp_adam")


def grp_riemann_batch(QL, QR, ps, iters, status, used=None, gamma=1.4, guess=0, weights=None, box=None,
                      p_start=None, newton_rtol=1e-12, newton_max_iter=50, stream=None):
    """Star pressures of n independent Riemann problems.  QL, QR: device float64
    [3, n] (rho, m, E); p_start: None or device float64 [n] explicit starts;
    ps float64 [n], iters and status int32 [n], used uint8 [n] or None: device
    outputs."""
    n = int(QL.shape[-1])
    _check(load().grp_riemann_batch(float(gamma), int(guess), float(newton_rtol), int(newton_max_iter),
                                    _dev(weights, "weights") if weights is not None else None,
                                    _dev(box, "box") if box is not None else None, n,
                                    _dev(QL, "QL"), _dev(QR, "QR"),
                                    _dev(p_start, "p_start") if p_start is not None else None,
                                    _dev(ps, "ps"), _dev(iters, "iters"),
                                    _dev(status, "status"), _dev(used, "used") if used is not None else None,
                                    stream), "grp_riemann_batch")


def noalloc_check_buffers(prob, avg_in, iface_in, avg_out, iface_out, current_device=None):
    """Reject, before any call into the library, buffers the allocation-free
    step cannot take: each must be a contiguous float64 CUDA tensor on the
    current device (the library resolves its scratch on the current device),
    holding C planes of n_cells (averages) or n_ifaces (interface data)
    doubles, and the outputs must not overlap the inputs.  Returns the four
    device addresses."""
    n = np.asarray(prob["n_cells"]).reshape(-1)
    if n.size != 1:
        raise GrpError("grp_step_noalloc advances one domain")
    C = 3 if int(prob["system"]) == GRP_EULER_IDEAL else 1
    N = int(n[0])
    nif = N + (1 if int(np.asarray(prob["bc"]).reshape(-1)[0]) == GRP_BC_TRANSMISSIVE else 0)
    spans = []
    for name, x, size in (("avg_in", avg_in, C * N), ("iface_in", iface_in, C * nif),
                          ("avg_out", avg_out, C * N), ("iface_out", iface_out, C * nif)):
        if not hasattr(x, "data_ptr") or not getattr(x, "is_cuda", False):
            raise GrpError("grp_step_noalloc: %s must be a CUDA tensor" % name)
        if str(x.dtype) != "torch.float64":
            raise GrpError("grp_step_noalloc: %s must be float64" % name)
        if not x.is_contiguous():
            raise GrpError("grp_step_noalloc: %s must be contiguous" % name)
        if x.numel() != size:
            raise GrpError("grp_step_noalloc: %s holds %d doubles, %d expected" % (name, x.numel(), size))
        if current_device is None:
            import torch
            current_device = torch.cuda.current_device()
        if x.device.index != current_device:
            raise GrpError("grp_step_noalloc: %s is on cuda:%s, the current device is cuda:%d"
                           % (name, x.device.index, current_device))
        spans.append((x.data_ptr(), x.data_ptr() + 8 * size))
    for o in (2, 3):
        for i in (0, 1):
            if spans[o][0] < spans[i][1] and spans[i][0] < spans[o][1]:
                raise GrpError("grp_step_noalloc: outputs must not overlap the inputs")
    return [sp[0] for sp in spans]


def grp_step_noalloc(prob, avg_in, iface_in, avg_out, iface_out, t, t_end=float("inf"), stream=None):
    """One step of a single-domain problem through the allocation-free entry
    point; the four buffers are device tensors the caller owns (checked by
    noalloc_check_buffers).  Returns (t_new, status)."""
    ptrs = noalloc_check_buffers(prob, avg_in, iface_in, avg_out, iface_out)
    n = np.asarray(prob["n_cells"]).reshape(-1)
    t_out, st = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(load().grp_step_noalloc(int(prob["system"]), float(prob.get("lam", 1.0)),
                                   float(prob.get("gamma", 1.4)), int(prob["M"]), float(prob["cfl"]),
                                   int(n[0]), float(np.asarray(prob["x_left"]).reshape(-1)[0]),
                                   float(np.asarray(prob["x_right"]).reshape(-1)[0]),
                                   int(np.asarray(prob["bc"]).reshape(-1)[0]),
                                   *ptrs, float(t), float(t_end), ctypes.byref(t_out), ctypes.byref(st),
                                   stream), "grp_step_noalloc")
    return t_out.value, st.value


def grp_status_string(code):
    return load().grp_status_string(int(code)).decode()


def _check(rc, what):
    if rc != GRP_OK:
        raise GrpError("%s failed: %s (%d)" % (what, grp_status_string(rc), rc))


def _ptr(x):
    """(address, is_device) of a numpy array or a torch tensor."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise GrpError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    return x.ctypes.data, 0


class Solver:
    """One grp_ctx.  ``prob`` uses the keys of ``inputs`` problems."""

    def __init__(self, prob, device=0, stream=None, guess=None, dt_hold=None):
        L = load()
        self._keep = dict(n=np.ascontiguousarray(prob["n_cells"], dtype=np.int32),
                          xl=np.ascontiguousarray(prob["x_left"], dtype=np.float64),
                          xr=np.ascontiguousarray(prob["x_right"], dtype=np.float64),
                          bc=np.ascontiguousarray(prob["bc"], dtype=np.int32))
        k = self._keep
        p = grp_problem()
        p.system = int(prob["system"])
        p.lambda_ = float(prob.get("lam", 1.0))
        p.gamma = float(prob.get("gamma", 1.4))
        p.M = int(prob["M"])
        p.cfl = float(prob["cfl"])
        p.n_domains = len(k["n"])
        p.n_cells = k["n"].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        p.x_left = k["xl"].ctypes.data_as(_D)
        p.x_right = k["xr"].ctypes.data_as(_D)
        p.bc = k["bc"].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        p.newton_rtol = float(prob.get("newton_rtol", 1e-12))
        p.newton_max_iter = int(prob.get("newton_max_iter", 50))
        p.guess = int(prob.get("guess", 0) if guess is None else guess)
        p.dt_hold = int(prob.get("dt_hold", 1) if dt_hold is None else dt_hold)
        p.device = int(device)
        p.stream = stream
        p.recon = int(prob.get("recon", GRP_RECON_GRPREC))
        p.solver = int(prob.get("solver", GRP_SOLVER_TT))
        p.source = int(prob.get("source", GRP_SOURCE_NONE))
        p.source_coef = float(prob.get("source_coef", 0.0))
        self.prob = prob
        self.C = 3 if p.system == GRP_EULER_IDEAL else 1
        self.D = p.n_domains
        self.ncell = int(k["n"].sum())
        self.nif = int(np.sum(k["n"] + (k["bc"] == GRP_BC_TRANSMISSIVE)))
        h = _vp()
        _check(L.grp_create(ctypes.byref(h), ctypes.byref(p)), "grp_create")
        self.h = h
        self.L = L

    def close(self):
        if getattr(self, "h", None):
            self.L.grp_destroy(self.h)
            self.h = None

    __del__ = close

    def set_initial(self, avg, lim_minus, lim_plus=None):
        a, da = _ptr(avg)
        m, dm = _ptr(lim_minus)
        q, dq = _ptr(lim_plus)
        if not (da == dm and (q is None or dq == da)):
            raise GrpError("all initial buffers must live on the same side")
        for x, n in ((avg, self.C * self.ncell), (lim_minus, self.C * self.nif), (lim_plus, self.C * self.nif)):
            if x is not None and (x.dtype != np.float64 if isinstance(x, np.ndarray) else str(x.dtype) != "torch.float64"):
                raise GrpError("buffers must be float64")
            if x is not None and (x.size if isinstance(x, np.ndarray) else x.numel()) != n:
                raise GrpError("buffer size mismatch")
        _check(self.L.grp_set_initial(self.h, a, m, q, da), "grp_set_initial")

    def step(self, n, t_end=np.inf):
        _check(self.L.grp_step(self.h, int(n), float(t_end)), "grp_step")

    def advance_to(self, t_end, max_steps=10 ** 7):
        _check(self.L.grp_advance_to(self.h, float(t_end), int(max_steps)), "grp_advance_to")

    def get_state(self, avg=None, iface=None, t=None):
        """Host numpy copies (allocated here when not given) or device tensors."""
        if avg is None and iface is None and t is None:
            avg = np.empty((self.C, self.ncell))
            iface = np.empty((self.C, self.nif))
            t = np.empty(self.D)
        a, da = _ptr(avg)
        i, di = _ptr(iface)
        tt, dt = _ptr(t)
        dev = max(da, di, dt)
        _check(self.L.grp_get_state(self.h, a, i, tt, dev), "grp_get_state")
        return avg, iface, t

    def get_stats(self):
        stats = np.zeros((self.D, GRP_NSTATS), dtype=np.uint64)
        status = np.zeros(self.D, dtype=np.int32)
        _check(self.L.grp_get_stats(self.h, stats.ctypes.data, status.ctypes.data), "grp_get_stats")
        return stats, status

    def error_norms(self, exact):
        e, de = _ptr(exact)
        l1, l2, li = np.zeros(self.D), np.zeros(self.D), np.zeros(self.D)
        _check(self.L.grp_error_norms(self.h, e, de, l1.ctypes.data, l2.ctypes.data, li.ctypes.data),
               "grp_error_norms")
        return l1, l2, li

    def set_kernel_timing(self, on=True):
        _check(self.L.grp_set_kernel_timing(self.h, 1 if on else 0), "grp_set_kernel_timing")

    def kernel_timing(self):
        """(summed flux-kernel milliseconds, timed launches) since the last call."""
        ms, n = ctypes.c_double(0.0), ctypes.c_longlong(0)
        _check(self.L.grp_get_kernel_timing(self.h, ctypes.byref(ms), ctypes.byref(n)), "grp_get_kernel_timing")
        return ms.value, n.value

    def set_launch(self, mode=GRP_LAUNCH_AUTO, threads=256, cells_per_block=2048, steps_per_launch=8):
        _check(self.L.grp_set_launch(self.h, int(mode), int(threads), int(cells_per_block),
                                     int(steps_per_launch)), "grp_set_launch")

    def set_graph(self, steps_per_graph=16):
        """CUDA graphs of steps_per_graph steps for grp_step (0: direct launches)."""
        _check(self.L.grp_set_graph(self.h, int(steps_per_graph)), "grp_set_graph")

    def get_launch(self):
        v = [ctypes.c_int(0) for _ in range(5)]
        _check(self.L.grp_get_launch(self.h, *[ctypes.byref(x) for x in v]), "grp_get_launch")
        return dict(zip(("form", "threads", "cells_per_block", "steps_per_launch", "blocks"),
                        [x.value for x in v]))

    def set_guess_model(self, weights, box):
        w, dw = _ptr(weights)
        b, db = _ptr(box)
        if dw != db:
            raise GrpError("weights and box must live on the same side")
        _check(self.L.grp_set_guess_model(self.h, w, GRP_MLP_NPARAM, b, dw), "grp_set_guess_model")

    def set_harvest(self, records=None, count=None, log2_stride=0):
        if records is None:
            _check(self.L.grp_set_harvest(self.h, None, None, 0, 0), "grp_set_harvest")
            return
        _check(self.L.grp_set_harvest(self.h, _dev(records, "records"), _dev(count, "count"),
                                      int(records.shape[0]), int(log2_stride)), "grp_set_harvest")

    def launch_count(self):
        return int(self.L.grp_launch_count(self.h))
