"""Python binding of the sm_103a tensor-train multigroup S_N transport library.

Argument marshalling only: every computation runs in the CUDA kernels of
``libtt_gb300.so`` behind the C ABI of ``include/tt.h``.  PyTorch provides device memory
and the CUDA stream.  If the shared library is missing or no CUDA device is present, the
calls raise; there is no CPU fallback.

Functions keep the C names: ``tt_step``, ``tt_round``, ``tt_apply_transport``,
``tt_axpy``, ``tt_dot``, ``tt_energy_density``, ``tt_plan_create``, ``tt_sync``.
"""
from __future__ import annotations

import ctypes
import sys
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtt_gb300.so")
MAX_CORES = 8

TT_OK, TT_ERR_ARG, TT_ERR_SHAPE, TT_ERR_CAPACITY, TT_ERR_CUDA = 0, 1, 2, 3, 4
TT_ERR_NONFINITE, TT_ERR_TIMEOUT, TT_ERR_UNSUPPORTED, TT_ERR_WORKSPACE = 5, 6, 7, 8
TT_F64, TT_F32 = 0, 1
TT_PREC_FP64, TT_PREC_MIXED = 0, 1
TT_QUAD_GAUSS_LEGENDRE_MU, TT_QUAD_LATLONG_MIDPOINT = 0, 1
TT_PREC_MIXED_3XTF32 = 2
PRECISIONS = {"fp64": TT_PREC_FP64, "mixed": TT_PREC_MIXED, "mixed_3xtf32": TT_PREC_MIXED_3XTF32}
ROUNDINGS = {"tsqr": 0, "gram": 1, "randomized": 2}

EXPORTS = ("tt_status_string", "tt_context_create", "tt_context_destroy", "tt_sync", "tt_workspace_query",
           "tt_plan_create", "tt_plan_destroy", "tt_plan_array", "tt_axpy", "tt_dot", "tt_round",
           "tt_apply_transport", "tt_step", "tt_energy_density", "tt_context_set_timing",
           "tt_context_counters", "tt_context_diagnostics", "tt_dot_noalloc", "tt_batch_create",
           "tt_batch_step", "tt_batch_sync", "tt_batch_info", "tt_batch_destroy", "tt_context_set_rounding",
           "tt_internal_ranks", "tt_context_set_sketch", "tt_context_set_tsqr", "tt_context_get_tsqr",
           "tt_autotune", "tt_context_set_graphs", "tt_tsqr_geometry", "tt_context_set_limits",
           "tt_tc_gemm", "tt_peak_probe")
TSQR_VARIANTS = {"column": 0, "rowsplit": 1, "column_dense": 2, "blocked": 3}
TIMER_NAMES = ("tsqr_leaf", "tsqr_merge", "small", "update", "other", "tsqr_leaf_source", "update_source")


class TTError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status})")


class _Tensor(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("n", ctypes.c_int32 * MAX_CORES),
                ("rcap", ctypes.c_int32 * (MAX_CORES + 1)), ("rank", ctypes.c_void_p),
                ("core", ctypes.c_void_p * MAX_CORES), ("dtype", ctypes.c_int)]


class _Problem(ctypes.Structure):
    _fields_ = [("ndim_x", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("ngroup", ctypes.c_int32), ("quadrature", ctypes.c_int32),
                ("ntheta", ctypes.c_int32), ("nphi", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("c", ctypes.c_double), ("dt", ctypes.c_double), ("a_rad", ctypes.c_double),
                ("group_edges", ctypes.c_void_p), ("temperature", ctypes.c_void_p),
                ("rho_kappa_a", ctypes.c_void_p), ("rho_kappa_s", ctypes.c_void_p),
                ("inflow_temperature", ctypes.c_double * 6), ("flux", ctypes.c_int32),
                ("rho_cv", ctypes.c_void_p), ("topology", ctypes.c_int32)]


TOPOLOGIES = {"merged": 0, "merged_nux_y": 1, "split_x": 2}


_lib = None


def library_path():
    return LIB_PATH


def lib():
    """Load libtt_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2602_00290_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, dbl, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
        L.tt_status_string.restype = ctypes.c_char_p
        L.tt_status_string.argtypes = [ctypes.c_int]
        sigs = {
            "tt_context_create": [ctypes.POINTER(vp), ctypes.c_int, vp, sz],
            "tt_context_destroy": [vp],
            "tt_sync": [vp],
            "tt_workspace_query": [vp, vp, ctypes.POINTER(_Tensor), ctypes.c_int, ctypes.POINTER(sz)],
            "tt_plan_create": [vp, ctypes.POINTER(_Problem), ctypes.POINTER(vp)],
            "tt_plan_destroy": [vp],
            "tt_plan_array": [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64)],
            "tt_axpy": [vp, dbl, ctypes.POINTER(_Tensor), ctypes.POINTER(_Tensor)],
            "tt_dot": [vp, ctypes.POINTER(_Tensor), ctypes.POINTER(_Tensor), vp],
            "tt_round": [vp, ctypes.POINTER(_Tensor), dbl, i32, ctypes.c_int],
            "tt_apply_transport": [vp, vp, ctypes.POINTER(_Tensor), ctypes.POINTER(_Tensor)],
            "tt_step": [vp, vp, ctypes.POINTER(_Tensor), dbl, i32, ctypes.c_int, vp],
            "tt_energy_density": [vp, vp, ctypes.POINTER(_Tensor), vp],
            "tt_context_set_timing": [vp, ctypes.c_int],
            "tt_context_set_graphs": [vp, ctypes.c_int],
            "tt_context_counters": [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), ctypes.c_int],
            "tt_context_diagnostics": [vp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int],
            "tt_dot_noalloc": [vp, ctypes.POINTER(_Tensor), ctypes.POINTER(_Tensor), vp],
            "tt_batch_create": [vp, ctypes.c_int32, ctypes.POINTER(vp), ctypes.POINTER(_Tensor),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                ctypes.c_int32, ctypes.POINTER(vp)],
            "tt_batch_step": [vp, ctypes.c_int32],
            "tt_batch_sync": [vp, ctypes.POINTER(ctypes.c_int32)],
            "tt_batch_info": [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_size_t),
                              ctypes.POINTER(ctypes.c_int32)],
            "tt_batch_destroy": [vp],
            "tt_context_set_rounding": [vp, ctypes.c_int],
            "tt_context_set_sketch": [vp, vp, ctypes.c_int32, ctypes.c_int32],
            "tt_context_set_tsqr": [vp, ctypes.c_int, i32, i32, i32],
            "tt_context_get_tsqr": [vp, ctypes.c_int, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)],
            "tt_autotune": [vp, vp, ctypes.POINTER(_Tensor), dbl, i32, ctypes.c_int, i32, ctypes.POINTER(i32),
                            ctypes.POINTER(ctypes.c_float)],
            "tt_context_set_limits": [vp, i32, ctypes.c_int64, i32],
            "tt_tc_gemm": [vp, ctypes.c_int64, i32, i32, vp, vp, vp, i32, vp],
            "tt_peak_probe": [vp, i32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)],
            "tt_tsqr_geometry": [ctypes.c_int, i32, i32, ctypes.c_int64, i32, i32, i32,
                                 ctypes.POINTER(ctypes.c_int64), i32],
            "tt_internal_ranks": [vp, vp, ctypes.POINTER(_Tensor), ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                  ctypes.c_int64],
        }
        for name, args in sigs.items():
            f = getattr(L, name)
            f.restype = ctypes.c_int
            f.argtypes = args
        _lib = L
    return _lib


GEOMETRY_KEYS = ("leaves", "rows_per_leaf", "block_rows", "leaf_threads", "leaf_smem", "merge_threads",
                 "merge_smem", "merge_levels", "ws_a_doubles", "ws_b_doubles", "variant", "merge_rows")


def tsqr_geometry(precision, variant, ncap, nrows, num_sms, per_sm, max_leaves=0):
    """Launch geometry of the TSQR over the merged core (tt_tsqr_geometry; host only, no GPU)."""
    out = (ctypes.c_int64 * len(GEOMETRY_KEYS))()
    v = TSQR_VARIANTS[variant] if isinstance(variant, str) else int(variant)
    _check(lib().tt_tsqr_geometry(PRECISIONS[precision], v, ncap, nrows, num_sms, per_sm, max_leaves, out,
                                  len(GEOMETRY_KEYS)), "tt_tsqr_geometry")
    return dict(zip(GEOMETRY_KEYS, list(out)))


def tc_gemm(A, B, passes=3, stream=None, status=None):
    """D = A B^T on the tensor cores (tt_tc_gemm): A (M x K), B (N x K) FP32 CUDA tensors."""
    torch = _torch()
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty(M, N, dtype=torch.float32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().tt_tc_gemm(ctypes.c_void_p(s.cuda_stream), M, N, K, ctypes.c_void_p(A.data_ptr()),
                            ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(D.data_ptr()), passes,
                            ctypes.c_void_p(status.data_ptr() if status is not None else 0)), "tt_tc_gemm")
    return D


PEAK_KINDS = {"fp64": 0, "fp32": 1, "tf32_tensor": 2}


def peak_probe(kind, iters, stream=None):
    """(flops, ms) of one probe of an arithmetic pipe (tt_peak_probe)."""
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    flops = ctypes.c_double()
    ms = ctypes.c_float()
    _check(lib().tt_peak_probe(ctypes.c_void_p(s.cuda_stream), PEAK_KINDS[kind], int(iters), ctypes.byref(flops),
                               ctypes.byref(ms)), "tt_peak_probe")
    return flops.value, ms.value


def status_string(st):
    try:
        return lib().tt_status_string(int(st)).decode()
    except Exception:  # library not loadable: still describe the code
        return f"status {st}"


def _check(st, where):
    if st != TT_OK:
        raise TTError(st, where)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the tensor-train transport library runs on the GPU only")
    return torch


# --------------------------------------------------------------------------------------------

class Context:
    """A library context bound to the current CUDA device and torch's current stream."""

    def __init__(self, device: Optional[int] = None, stream=None, workspace_bytes: int = 0):
        torch = _torch()
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(lib().tt_context_create(ctypes.byref(h), self.device, ctypes.c_void_p(self.stream.cuda_stream),
                                       int(workspace_bytes)), "tt_context_create")
        self.handle = h

    def sync(self):
        _check(lib().tt_sync(self.handle), "tt_sync")

    def set_limits(self, jacobi_sweeps: int = 0, barrier_spins: int = 0, barrier_extra: int = 0):
        """Bounded device-side iterations (tt_context_set_limits; 0 restores a default)."""
        _check(lib().tt_context_set_limits(self.handle, int(jacobi_sweeps), int(barrier_spins), int(barrier_extra)),
               "tt_context_set_limits")

    def set_sketch(self, omega):
        """Sketch of randomized rounding: omega (n_1...n_{d-1} x l) as a numpy or torch array."""
        torch = _torch()
        om = torch.as_tensor(np.asarray(omega, dtype=np.float64), device=torch.device("cuda", self.device)).contiguous()
        self._sketch = om
        _check(lib().tt_context_set_sketch(self.handle, ctypes.c_void_p(om.data_ptr()), int(om.shape[0]),
                                           int(om.shape[1])), "tt_context_set_sketch")

    def set_graphs(self, enable: bool = True):
        """tt_step replays a captured CUDA graph of the step while its arguments stay the same."""
        _check(lib().tt_context_set_graphs(self.handle, 1 if enable else 0), "tt_context_set_graphs")

    def set_rounding(self, method: str):
        """"tsqr" (Householder TSQR, default), "gram" (Gram matrix + pivoted-Cholesky root) or
        "randomized" (sketch of set_sketch, TSQR of the sketch, C = Q^T A)."""
        _check(lib().tt_context_set_rounding(self.handle, ROUNDINGS[method]), "tt_context_set_rounding")

    def set_tsqr(self, prec: str, ncap: int, variant: str = "column", leaves: int = 0):
        """TSQR kernels for passes of ncap columns at precision prec ("fp64" / "mixed"):
        variant "column" (one thread per column), "rowsplit" (four lanes per column) or
        "column_dense" (FP32, 32-row blocks, four CTAs per SM), leaves = cap on the TSQR leaves
        (0: the default wave).  ncap <= 0 clears every entry."""
        _check(lib().tt_context_set_tsqr(self.handle, PRECISIONS[prec], int(ncap), TSQR_VARIANTS[variant],
                                         int(leaves)), "tt_context_set_tsqr")

    def get_tsqr(self, prec: str, ncap: int):
        """(variant, leaf cap) a pass of ncap columns at precision prec runs with."""
        v, l = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tt_context_get_tsqr(self.handle, PRECISIONS[prec], int(ncap), ctypes.byref(v), ctypes.byref(l)),
               "tt_context_get_tsqr")
        names = {i: k for k, i in TSQR_VARIANTS.items()}
        return names[v.value], l.value

    def autotune(self, plan: "Plan", I: "TT", tol: float, rmax: int, prec: str = "mixed", steps: int = 3):
        """Time the TSQR choices of tt_step's two passes on a copy of I and keep the fastest
        (tt_autotune).  Returns {"transport": (variant, leaves), "source": (...),
        "ms_default": ..., "ms_tuned": ...}."""
        ch = (ctypes.c_int32 * 4)()
        ms = (ctypes.c_float * 2)()
        _check(lib().tt_autotune(self.handle, plan.handle, ctypes.byref(I._struct()), float(tol), int(rmax),
                                 PRECISIONS[prec], int(steps), ch, ms), "tt_autotune")
        names = {i: k for k, i in TSQR_VARIANTS.items()}
        return {"transport": (names[ch[0]], ch[1]), "source": (names[ch[2]], ch[3]),
                "ms_default": float(ms[0]), "ms_tuned": float(ms[1])}

    def set_timing(self, enable: bool):
        _check(lib().tt_context_set_timing(self.handle, 1 if enable else 0), "tt_context_set_timing")

    def diagnostics(self, reset: bool = False):
        """Statistics since the last reset: Jacobi max sweeps, SVD count, total sweeps; tt_step
        graph replays, captures and refused captures (tt_context_diagnostics)."""
        out = (ctypes.c_int64 * 6)()
        _check(lib().tt_context_diagnostics(self.handle, out, 6, 1 if reset else 0), "tt_context_diagnostics")
        return {"jacobi_sweeps_max": out[0], "jacobi_svds": out[1], "jacobi_sweeps_total": out[2],
                "graph_replays": out[3], "graph_captures": out[4], "graph_failures": out[5]}

    def counters(self, reset: bool = False):
        """(ms per category, launches per category) since the last reset (tt_context_counters)."""
        ms = (ctypes.c_double * len(TIMER_NAMES))()
        n = (ctypes.c_int64 * len(TIMER_NAMES))()
        _check(lib().tt_context_counters(self.handle, ms, n, 1 if reset else 0), "tt_context_counters")
        return dict(zip(TIMER_NAMES, list(ms))), dict(zip(TIMER_NAMES, list(n)))

    def close(self):
        if getattr(self, "handle", None):
            lib().tt_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        # no CUDA teardown while the interpreter shuts down (the driver may already be gone)
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class TT:
    """TT tensor in capacity layout: core j is a torch tensor [rcap_{j-1}*n_j, rcap_j] on the GPU,
    live ranks in a device int32 tensor."""

    def __init__(self, n: Sequence[int], rcap: Sequence[int], dtype="f64", device="cuda"):
        torch = _torch()
        self.d = len(n)
        self.n = list(n)
        self.rcap = [1] + list(rcap) + [1]
        assert len(self.rcap) == self.d + 1
        self.dtype = dtype
        tdt = torch.float64 if dtype == "f64" else torch.float32
        self.cores = [torch.zeros(self.rcap[j] * self.n[j], self.rcap[j + 1], dtype=tdt, device=device)
                      for j in range(self.d)]
        self.rank = torch.ones(self.d + 1, dtype=torch.int32, device=device)
        self._s = None

    @classmethod
    def from_cores(cls, cores, rcap=None, dtype="f64", device="cuda"):
        """Copy cores given with live shapes (r_{j-1}, n_j, r_j) into capacity layout."""
        torch = _torch()
        cores = [np.asarray(c, dtype=np.float64) for c in cores]
        n = [c.shape[1] for c in cores]
        live = [c.shape[2] for c in cores[:-1]]
        rcap = list(live) if rcap is None else list(rcap)
        x = cls(n, rcap, dtype, device)
        tdt = torch.float64 if dtype == "f64" else torch.float32
        for j, c in enumerate(cores):
            r0, nj, r1 = c.shape
            buf = np.zeros((x.rcap[j], nj, x.rcap[j + 1]))
            buf[:r0, :, :r1] = c
            x.cores[j].copy_(torch.from_numpy(buf.reshape(x.rcap[j] * nj, x.rcap[j + 1])).to(tdt))
        x.rank.copy_(torch.tensor([1] + live + [1], dtype=torch.int32))
        return x

    def ranks(self) -> List[int]:
        return [int(v) for v in self.rank.cpu().tolist()]

    def to_cores(self):
        """Live cores as float64 numpy arrays of shape (r_{j-1}, n_j, r_j)."""
        r = self.ranks()
        out = []
        for j in range(self.d):
            a = self.cores[j].double().cpu().numpy().reshape(self.rcap[j], self.n[j], self.rcap[j + 1])
            out.append(a[:r[j], :, :r[j + 1]].copy())
        return out

    def _struct(self):
        s = _Tensor()
        s.d = self.d
        for j in range(self.d):
            s.n[j] = self.n[j]
        for j in range(self.d + 1):
            s.rcap[j] = self.rcap[j]
        s.rank = self.rank.data_ptr()
        for j in range(self.d):
            s.core[j] = self.cores[j].data_ptr()
        s.dtype = TT_F64 if self.dtype == "f64" else TT_F32
        self._s = s
        return s


class Plan:
    """Device-side per-problem coefficients (tt_plan_create) for a raw workload."""

    def __init__(self, ctx: Context, wl):
        torch = _torch()
        dev = torch.device("cuda", ctx.device)
        self.wl = wl
        self._arrays = [torch.as_tensor(np.asarray(a, dtype=np.float64), device=dev).contiguous()
                        for a in (wl.group_edges, wl.temperature, wl.rho_kappa_a, wl.rho_kappa_s)]
        p = _Problem()
        p.ndim_x, p.nx, p.ny, p.nz, p.ngroup = wl.ndim, wl.nx, wl.ny, wl.nz, wl.ngroup
        p.quadrature = TT_QUAD_GAUSS_LEGENDRE_MU if wl.quad == "gauss_legendre_mu" else TT_QUAD_LATLONG_MIDPOINT
        p.ntheta, p.nphi = wl.ntheta, wl.nphi
        p.dx, p.dy, p.dz = wl.spacing
        p.c, p.dt, p.a_rad = wl.c, wl.dt, wl.a_rad
        p.group_edges, p.temperature, p.rho_kappa_a, p.rho_kappa_s = [a.data_ptr() for a in self._arrays]
        for f in range(6):
            t = wl.inflow_temperature[f] if f < len(wl.inflow_temperature) else None
            p.inflow_temperature[f] = -1.0 if t is None else float(t)
        p.flux = {"upwind": 0, "rusanov": 1, "central": 2}[getattr(wl, "flux", "upwind")]
        p.topology = TOPOLOGIES[getattr(wl, "topology", "merged")]
        rcv = getattr(wl, "rho_cv", None)
        if rcv is not None:
            self._arrays.append(torch.as_tensor(np.asarray(rcv, dtype=np.float64), device=dev).contiguous())
            p.rho_cv = self._arrays[-1].data_ptr()
        else:
            p.rho_cv = None
        h = ctypes.c_void_p()
        _check(lib().tt_plan_create(ctx.handle, ctypes.byref(p), ctypes.byref(h)), "tt_plan_create")
        self.handle = h
        self.ctx = ctx
        self.d = 2 if wl.ndim == 1 else 3
        self.n = [wl.nrow, wl.ntheta] + ([wl.nphi] if self.d == 3 else [])

    def array(self, which):
        """Copy of a plan array (see tt_plan_array) as a numpy array."""
        ptr = ctypes.c_void_p()
        n = ctypes.c_int64()
        _check(lib().tt_plan_array(self.handle, int(which), ctypes.byref(ptr), ctypes.byref(n)), "tt_plan_array")
        self.ctx.sync()
        if n.value == 0:
            return np.empty(0)
        return _wrap_device_ptr(ptr.value, n.value).cpu().numpy().copy()

    def temperature(self):
        """Material temperature per cell (advanced by tt_step when the problem is coupled)."""
        return self.array(7)

    def t_dagger(self):
        """T^dagger of the last coupled step per cell."""
        return self.array(8)

    def new_state(self, rcap: Sequence[int], dtype="f64"):
        return TT(self.n, rcap, dtype)

    def close(self):
        if getattr(self, "handle", None):
            lib().tt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        # no CUDA teardown while the interpreter shuts down (the driver may already be gone)
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def _wrap_device_ptr(ptr, count):
    """A torch float64 view of `count` doubles of device memory owned by the library."""
    torch = _torch()

    class _Holder:
        pass

    h = _Holder()
    h.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f8", "data": (ptr, False), "version": 3}
    return torch.as_tensor(h, device="cuda")


# --- C ABI names --------------------------------------------------------------------------------

def tt_plan_create(ctx: Context, wl) -> Plan:
    return Plan(ctx, wl)


def tt_sync(ctx: Context):
    ctx.sync()


def tt_axpy(ctx: Context, alpha: float, x: TT, y: TT):
    _check(lib().tt_axpy(ctx.handle, float(alpha), ctypes.byref(x._struct()), ctypes.byref(y._struct())), "tt_axpy")


def tt_dot(ctx: Context, x: TT, y: TT, out=None):
    torch = _torch()
    if out is None:
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
    _check(lib().tt_dot(ctx.handle, ctypes.byref(x._struct()), ctypes.byref(y._struct()),
                        ctypes.c_void_p(out.data_ptr())), "tt_dot")
    return out


def tt_dot_noalloc(stream, x: TT, y: TT, out):
    """<x, y> into the device double `out` without any device allocation (see tt.h); `stream`
    is a torch CUDA stream (or None for the legacy default stream)."""
    h = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(lib().tt_dot_noalloc(h, ctypes.byref(x._struct()), ctypes.byref(y._struct()),
                                ctypes.c_void_p(out.data_ptr())), "tt_dot_noalloc")
    return out


class Batch:
    """Independent problems stepped together (tt_batch_*): plans[i] with states[i] (TT objects,
    kept alive by the batch), tolerances and rank caps per problem, one precision."""

    def __init__(self, ctx: Context, plans, states, tol, rmax, prec="fp64", nstreams=0):
        n = len(plans)
        assert len(states) == n
        tol = [float(t) for t in (tol if hasattr(tol, "__len__") else [tol] * n)]
        rmax = [int(r) for r in (rmax if hasattr(rmax, "__len__") else [rmax] * n)]
        self.ctx, self.plans, self.states = ctx, list(plans), list(states)
        self._structs = (_Tensor * n)(*[s._struct() for s in states])
        hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
        h = ctypes.c_void_p()
        _check(lib().tt_batch_create(ctx.handle, n, hp, self._structs, (ctypes.c_double * n)(*tol),
                                     (ctypes.c_int32 * n)(*rmax), PRECISIONS[prec], int(nstreams), ctypes.byref(h)),
               "tt_batch_create")
        self.handle = h
        self.n = n

    def step(self, nsteps=1):
        _check(lib().tt_batch_step(self.handle, int(nsteps)), "tt_batch_step")

    def sync(self):
        """Per-problem latched statuses (raises on the first error)."""
        st = (ctypes.c_int32 * self.n)()
        rc = lib().tt_batch_sync(self.handle, st)
        _check(rc, "tt_batch_sync")
        return list(st)

    def info(self):
        n = ctypes.c_int64()
        b = ctypes.c_size_t()
        k = ctypes.c_int32()
        _check(lib().tt_batch_info(self.handle, ctypes.byref(n), ctypes.byref(b), ctypes.byref(k)), "tt_batch_info")
        return {"launches_per_step": n.value, "workspace_bytes": b.value, "streams": k.value}

    def close(self):
        if getattr(self, "handle", None):
            lib().tt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        # no CUDA teardown while the interpreter shuts down (the driver may already be gone)
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def tt_internal_ranks(ctx: Context, plan: "Plan", x: TT, delta_rel: float, with_status: bool = False):
    """(r1, r1x, sigma_nu, sigma_x): internal delta-ranks of the merged core (tt_internal_ranks).
    with_status: a TT_ERR_TIMEOUT (a Jacobi sweep cap reached; the ranks of the last sweep) is
    returned as a fifth element instead of raised."""
    G = plan.wl.ngroup
    ncx = G * x.rcap[1]
    nX = x.n[0] // G
    r = (ctypes.c_int32 * 2)()
    snu = (ctypes.c_double * G)()
    nsx = min(nX, ncx)
    sx = (ctypes.c_double * nsx)()
    st = lib().tt_internal_ranks(ctx.handle, plan.handle, ctypes.byref(x._struct()), float(delta_rel), r, snu, G,
                                 sx, nsx)
    if not (with_status and st == TT_ERR_TIMEOUT):
        _check(st, "tt_internal_ranks")
    out = (int(r[0]), int(r[1]), np.array(snu[:]), np.array(sx[:]))
    return out + (st,) if with_status else out


def tt_round(ctx: Context, x: TT, tol: float, rmax: int, prec="fp64"):
    _check(lib().tt_round(ctx.handle, ctypes.byref(x._struct()), float(tol), int(rmax), PRECISIONS[prec]),
           "tt_round")


def tt_apply_transport(ctx: Context, plan: Plan, x: TT, out: TT):
    _check(lib().tt_apply_transport(ctx.handle, plan.handle, ctypes.byref(x._struct()), ctypes.byref(out._struct())),
           "tt_apply_transport")


def tt_step(ctx: Context, plan: Plan, I: TT, tol: float, rmax: int, prec="fp64", energy=None):
    ptr = ctypes.c_void_p(energy.data_ptr()) if energy is not None else None
    _check(lib().tt_step(ctx.handle, plan.handle, ctypes.byref(I._struct()), float(tol), int(rmax),
                         PRECISIONS[prec], ptr), "tt_step")


def tt_energy_density(ctx: Context, plan: Plan, x: TT, out=None):
    torch = _torch()
    if out is None:
        out = torch.empty(x.n[0], dtype=torch.float64, device="cuda")
    _check(lib().tt_energy_density(ctx.handle, plan.handle, ctypes.byref(x._struct()),
                                   ctypes.c_void_p(out.data_ptr())), "tt_energy_density")
    return out


def tt_workspace_query(ctx: Context, plan: Optional[Plan], x: TT, prec="fp64") -> int:
    n = ctypes.c_size_t()
    _check(lib().tt_workspace_query(ctx.handle, plan.handle if plan is not None else None,
                                    ctypes.byref(x._struct()), PRECISIONS[prec], ctypes.byref(n)),
           "tt_workspace_query")
    return int(n.value)


def initial_state(plan: Plan, rcap: Sequence[int], dtype="f64") -> TT:
    """Rank-1 isotropic TT with Z = epsilon_f(T) per row computed by the plan (I^0 = epsilon)."""
    torch = _torch()
    x = TT(plan.n, rcap, dtype)
    ptr = ctypes.c_void_p()
    n = ctypes.c_int64()
    _check(lib().tt_plan_array(plan.handle, 0, ctypes.byref(ptr), ctypes.byref(n)), "tt_plan_array")
    eps = _wrap_device_ptr(ptr.value, n.value)
    x.cores[0][:, 0].copy_(eps)
    for j in range(1, x.d):
        x.cores[j].view(x.rcap[j], x.n[j], x.rcap[j + 1])[0, :, 0] = 1.0
    return x
