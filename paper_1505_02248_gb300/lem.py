"""Thin ctypes binding of liblem.so (include/lem.h): argument marshalling only.

Every step of the LEM path runs in the library's CUDA kernels; this module only turns
Python values into the C descriptor and passes device pointers (torch tensors) or host
buffers (numpy arrays) through. There is no fallback: if liblem.so is missing or fails to
load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblem.so")

LEM_OK, LEM_EINVAL, LEM_ENOMEM, LEM_ECUDA, LEM_EBUSY, LEM_ENOTREADY, LEM_ETIMEOUT, LEM_ENUMERIC = range(8)
BC = {"dirichlet": 0, "periodic": 1}
MODE = {"phi": 0, "exp": 1}
PREC = {"fp64": 0, "split": 1, "split_fast": 2}
SCHEME = {"euler": 0, "rb3": 1}


class LemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class ProblemDesc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int),
        ("n", C.c_int64 * 2),
        ("bc", C.c_int * 2),
        ("coef", C.POINTER(C.c_double) * 5),
        ("coef_stride", C.c_int64),
        ("reaction", C.c_int),
        ("dt", C.c_double),
        ("tile", C.c_int * 2),
        ("overlap", C.c_int * 2),
        ("mode", C.c_int),
        ("prec", C.c_int),
        ("refresh", C.c_int),
        ("scheme", C.c_int),
        ("complex_values", C.c_int),
        ("coef_im", C.POINTER(C.c_double) * 5),
        ("porous_m", C.c_double),
    ]


class Info(C.Structure):
    _fields_ = [
        ("ntiles", C.c_int64), ("nclasses", C.c_int64), ("n_loc", C.c_int64), ("n_int", C.c_int64),
        ("squarings_max", C.c_int), ("built", C.c_int), ("split_path", C.c_int),
        ("device_bytes", C.c_int64), ("apply_path", C.c_int),
    ]


APPLY_PATHS = {0: "fp64_gemm", 1: "fp64_gemv", 2: "f32_gemv", 3: "tc_split", 4: "fp64_band", 5: "f32_band"}


class BatchCandidate(C.Structure):
    _fields_ = [("fused", C.c_int), ("lanes", C.c_int), ("n_cap", C.c_int), ("ms", C.c_double), ("chosen", C.c_int)]


class ServerStats(C.Structure):
    _fields_ = [
        ("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
        ("queued", C.c_int64), ("active", C.c_int64), ("dof_steps", C.c_int64),
        ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("first_admit_to_last_done_s", C.c_double),
        ("device_bytes", C.c_int64), ("ctx_hits", C.c_int64), ("ctx_misses", C.c_int64),
        ("ctx_adopted", C.c_int64), ("worker_admit_s", C.c_double), ("worker_issue_s", C.c_double),
        ("worker_build_s", C.c_double), ("ctx_built", C.c_int64), ("adopt_failed", C.c_int64),
        ("tier_completed", C.c_int64 * 2), ("tier_dof_steps", C.c_int64 * 2),
        ("tier_p50_ms", C.c_double * 2), ("tier_p99_ms", C.c_double * 2),
    ]


_lib = None

# (name, restype, argtypes) for every entry point of include/lem.h
SIGNATURES = [
    ("lem_create", C.c_int, [C.POINTER(ProblemDesc), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("lem_build_propagators", C.c_int, [C.c_void_p, C.c_void_p]),
    ("lem_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("lem_step_host", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("lem_get_propagator", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    ("lem_get_propagator_phi3", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    ("lem_set_propagators", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lem_tile_class", C.c_int64, [C.c_void_p, C.c_int64]),
    ("lem_class_squarings", C.c_int, [C.c_void_p, C.c_int64]),
    ("lem_get_info", C.c_int, [C.c_void_p, C.POINTER(Info)]),
    ("lem_plan_query", C.c_int, [C.POINTER(ProblemDesc), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_void_p]),
    ("lem_step_fp64_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    ("lem_set_truncation", C.c_int, [C.c_void_p, C.c_double]),
    ("lem_get_band", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.POINTER(C.c_int64)]),
    ("lem_set_timing", C.c_int, [C.c_void_p, C.c_int]),
    ("lem_get_timing", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    ("lem_sync", C.c_int, [C.c_void_p]),
    ("lem_destroy", None, [C.c_void_p]),
    ("lem_batch_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int,
                                   C.c_void_p, C.POINTER(C.c_void_p)]),
    ("lem_batch_run", C.c_int, [C.c_void_p, C.c_int]),
    ("lem_batch_schedule", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("lem_batch_destroy", None, [C.c_void_p]),
    ("lem_batch_info", C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("lem_batch_sync", C.c_int, [C.c_void_p]),
    ("lem_batch_candidates", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int)]),
    ("lem_batch_gemm_work", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("lem_batch_profile", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("lem_server_create", C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
    ("lem_server_reset_stats", C.c_int, [C.c_void_p]),
    ("lem_submit", C.c_int, [C.c_void_p, C.POINTER(ProblemDesc), C.c_double, C.c_void_p, C.c_int,
                             C.POINTER(C.c_uint64)]),
    ("lem_poll", C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_int)]),
    ("lem_wait", C.c_int, [C.c_void_p, C.c_uint64, C.c_double]),
    ("lem_server_get_stats", C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    ("lem_server_destroy", None, [C.c_void_p]),
    ("lem_status_str", C.c_char_p, [C.c_int]),
    ("lem_last_error", C.c_char_p, []),
]


def load(path: str = LIB_PATH):
    """Load liblem.so (raises if it is missing: there is no non-CUDA implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblem.so not built at {path}: run __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(status: int, what: str = "") -> None:
    if status != LEM_OK:
        lib = load()
        raise LemError(status, f"{what}: {lib.lem_status_str(status).decode()}: {lib.lem_last_error().decode()}")


def make_desc(shape, bc, coef: dict, dt: float, tile, overlap, mode="phi", prec="fp64",
              reaction=False, refresh=0, scheme="euler", porous_m=0.0):
    """Build a ProblemDesc; returns (desc, keepalive) -- keep the second alive while used.
    porous_m > 0 selects the porous-medium nonlinearity (reaction 2) with that exponent."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    d = ProblemDesc()
    d.ndim = nd
    for a in range(2):
        d.n[a] = shape[a] if a < nd else 0
        d.bc[a] = BC[bc[a]] if a < nd else 0
        d.tile[a] = int(tile[a]) if a < nd else 0
        d.overlap[a] = int(overlap[a]) if a < nd else 0
    keep = []
    names = ["C", "W", "E", "S", "N"][: 3 if nd == 1 else 5]
    raw = [np.asarray(coef[k]).ravel() for k in names]
    cplx = any(np.iscomplexobj(a) for a in raw)
    arrays = [np.ascontiguousarray(a.real, dtype=np.float64) for a in raw]
    imags = [np.ascontiguousarray(a.imag, dtype=np.float64) if np.iscomplexobj(a) else np.zeros(a.size)
             for a in raw]
    stride = 0 if all(a.size == 1 for a in arrays) else 1
    npts = int(np.prod(shape))
    for k, (a, b) in enumerate(zip(arrays, imags)):
        if stride == 1 and a.size == 1:
            a, b = np.full(npts, float(a[0])), np.full(npts, float(b[0]))
        keep += [a, b]
        d.coef[k] = a.ctypes.data_as(C.POINTER(C.c_double))
        if cplx:
            d.coef_im[k] = b.ctypes.data_as(C.POINTER(C.c_double))
    d.coef_stride = stride
    d.complex_values = 1 if cplx else 0
    d.reaction = 2 if porous_m else (1 if reaction else 0)
    d.porous_m = float(porous_m)
    d.dt = float(dt)
    d.mode = MODE[mode]
    d.prec = PREC[prec]
    d.refresh = int(refresh)
    d.scheme = SCHEME[scheme]
    return d, keep


def plan_query(shape, bc, coef, dt, tile, overlap, **kw):
    """Host-only decomposition (no device): dict with ntiles, nclasses, n_loc, n_int, tiles."""
    lib = load()
    d, keep = make_desc(shape, bc, coef, dt, tile, overlap, **kw)
    nt, nc, nl, ni = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    check(lib.lem_plan_query(C.byref(d), C.byref(nt), C.byref(nc), C.byref(nl), C.byref(ni), None), "plan")
    info = np.zeros((nt.value, 11), dtype=np.int32)
    check(lib.lem_plan_query(C.byref(d), None, None, None, None, info.ctypes.data_as(C.c_void_p)), "plan")
    return dict(ntiles=nt.value, nclasses=nc.value, n_loc=nl.value, n_int=ni.value, tiles=info)


def check_device_state(state, npts: int, complex_: bool = False, device=None):
    """Raise unless `state` is a contiguous CUDA tensor of npts float64 (complex128 for a
    complex problem) values, on `device` when given: the library dereferences its pointer on
    the GPU, so a host or mis-sized buffer must never reach it."""
    if not getattr(state, "is_cuda", False):
        raise TypeError("the state must be a CUDA tensor")
    if not state.is_contiguous():
        raise ValueError("the state must be contiguous")
    if state.dtype.itemsize != (16 if complex_ else 8) or state.is_complex() != complex_ or \
            not (state.is_complex() or state.is_floating_point()):
        raise TypeError("the state must be complex128" if complex_ else "the state must be float64")
    if state.numel() != npts:
        raise ValueError(f"the state has {state.numel()} values, the mesh {npts}")
    if device is not None and state.device.index != int(device):
        raise ValueError(f"the state is on {state.device}, the context on cuda:{int(device)}")


def check_host_state(state, npts: int, complex_: bool = False):
    """Raise unless `state` is a C-contiguous numpy array of npts float64 (complex128) values."""
    want = np.complex128 if complex_ else np.float64
    if not isinstance(state, np.ndarray) or state.dtype != want:
        raise TypeError(f"the state must be a numpy {np.dtype(want).name} array")
    if not state.flags.c_contiguous or state.size != npts:
        raise ValueError(f"the state must be C-contiguous with {npts} values")


class Lem:
    """One LEM context (lem_create ... lem_destroy) on a CUDA device."""

    def __init__(self, shape, bc, coef, dt, tile, overlap, mode="phi", prec="fp64",
                 reaction=False, refresh=0, device=0, stream=None, scheme="euler", porous_m=0.0):
        lib = load()
        self._lib = lib
        d, keep = make_desc(shape, bc, coef, dt, tile, overlap, mode, prec, reaction, refresh, scheme, porous_m)
        self.shape = tuple(int(s) for s in shape)
        self.npts = int(np.prod(self.shape))
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream is not None else None
        check(lib.lem_create(C.byref(d), int(device), st, C.byref(h)), "lem_create")
        self.complex = bool(d.complex_values)
        self.device = int(device)
        del keep
        self._h = h

    @classmethod
    def from_workload(cls, wl: dict, **kw):
        args = dict(mode="phi", prec="fp64", reaction=wl.get("reaction", False),
                    refresh=wl.get("refresh", 0), porous_m=wl.get("porous_m", 0.0))
        args.update(kw)
        return cls(wl["shape"], wl["bc"], wl["coef"], wl["dt"], wl["tile"], wl["overlap"], **args)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls -------------------------------------------------------------------------
    def build(self, state=None):
        if state is not None:
            check_device_state(state, self.npts, self.complex, self.device)
        ptr = None if state is None else C.c_void_p(state.data_ptr())
        check(self._lib.lem_build_propagators(self._h, ptr), "lem_build_propagators")

    def step(self, state, nsteps: int):
        """Advance a CUDA tensor in place: float64 (npts values), or complex128 (npts values,
        interleaved re/im) for a complex problem."""
        check_device_state(state, self.npts, self.complex, self.device)
        check(self._lib.lem_step(self._h, C.c_void_p(state.data_ptr()), int(nsteps)), "lem_step")

    def step_noalloc(self, state, nsteps: int):
        """lem_step_fp64_noalloc: the FP64 step with static scratch (no device allocation)."""
        check_device_state(state, self.npts, False, self.device)
        check(self._lib.lem_step_fp64_noalloc(self._h, C.c_void_p(state.data_ptr()), int(nsteps)),
              "lem_step_fp64_noalloc")

    def step_host(self, state: np.ndarray, nsteps: int):
        """Advance a host float64 (complex128 for a complex problem) array in place (copies in
        and out inside the call)."""
        check_host_state(state, self.npts, self.complex)
        check(self._lib.lem_step_host(self._h, state.ctypes.data_as(C.c_void_p), int(nsteps)),
              "lem_step_host")

    def propagator(self, cls: int) -> np.ndarray:
        inf = self.info()
        out = np.zeros((inf["n_int"], inf["n_loc"]))
        check(self._lib.lem_get_propagator(self._h, int(cls), out.ctypes.data_as(C.c_void_p)),
              "lem_get_propagator")
        return out

    def propagator_phi3(self, cls: int) -> np.ndarray:
        """The phi_3 propagator of a class (third-order Rosenbrock contexts)."""
        inf = self.info()
        out = np.zeros((inf["n_int"], inf["n_loc"]))
        check(self._lib.lem_get_propagator_phi3(self._h, int(cls), out.ctypes.data_as(C.c_void_p)),
              "lem_get_propagator_phi3")
        return out

    def set_propagators(self, P: np.ndarray, squarings=None):
        """Load all classes' propagators (nclasses x n_int x n_loc, float64) instead of building."""
        P = np.ascontiguousarray(P, dtype=np.float64)
        sq = None if squarings is None else np.ascontiguousarray(squarings, dtype=np.int32)
        check(self._lib.lem_set_propagators(self._h, P.ctypes.data_as(C.c_void_p),
                                            None if sq is None else sq.ctypes.data_as(C.c_void_p)),
              "lem_set_propagators")

    def tile_class(self, t: int) -> int:
        return int(self._lib.lem_tile_class(self._h, int(t)))

    def squarings(self, cls: int) -> int:
        return int(self._lib.lem_class_squarings(self._h, int(cls)))

    def info(self) -> dict:
        i = Info()
        check(self._lib.lem_get_info(self._h, C.byref(i)), "lem_get_info")
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def set_truncation(self, tol: float):
        """lem_set_truncation: keep each owner row's box of window nodes (tol >= 0), or turn
        truncation off (tol < 0)."""
        check(self._lib.lem_set_truncation(self._h, float(tol)), "lem_set_truncation")

    def band(self, cls: int):
        """lem_get_band: ((ly, hy, lx, hx), values stored per owner row) of class cls."""
        ext = (C.c_int32 * 4)()
        nv = C.c_int64()
        check(self._lib.lem_get_band(self._h, int(cls), ext, C.byref(nv)), "lem_get_band")
        return tuple(int(e) for e in ext), int(nv.value)

    def band_total(self) -> int:
        """Values stored for all classes' boxes together (lem_get_band with cls = -1)."""
        ext = (C.c_int32 * 4)()
        nv = C.c_int64()
        check(self._lib.lem_get_band(self._h, -1, ext, C.byref(nv)), "lem_get_band")
        return int(nv.value)

    def set_timing(self, on, period: int = 1):
        """Bracket every `period`-th apply-kernel launch with CUDA events (on: True/False)."""
        check(self._lib.lem_set_timing(self._h, max(1, int(period)) if on else 0), "lem_set_timing")

    def get_timing(self):
        """(total_ms, launches) of the apply kernel since the last call."""
        t, n = C.c_double(), C.c_int64()
        check(self._lib.lem_get_timing(self._h, C.byref(t), C.byref(n)), "lem_get_timing")
        return t.value, n.value

    def sync(self):
        check(self._lib.lem_sync(self._h), "lem_sync")


class Server:
    """lem_server: continuous batching of independent LEM requests on one device."""

    def __init__(self, budget_bytes: int = 0, device: int = 0):
        lib = load()
        self._lib = lib
        h = C.c_void_p()
        check(lib.lem_server_create(C.c_size_t(int(budget_bytes)), int(device), C.byref(h)), "lem_server_create")
        self._h = h
        self._keep = {}

    def submit(self, shape, bc, coef, dt, tile, overlap, state: np.ndarray, nsteps: int, tol: float = 1e-6,
               mode="phi", reaction=False, refresh=0) -> int:
        """Queue `state` (float64, C-contiguous, updated in place when done); returns a ticket."""
        check_host_state(state, int(np.prod([int(v) for v in shape])))
        d, keep = make_desc(shape, bc, coef, dt, tile, overlap, mode, "fp64", reaction, refresh)
        t = C.c_uint64()
        check(self._lib.lem_submit(self._h, C.byref(d), float(tol), state.ctypes.data_as(C.c_void_p), int(nsteps),
                                   C.byref(t)), "lem_submit")
        self._keep[t.value] = state  # the server writes into it until done
        return t.value

    def poll(self, ticket: int) -> bool:
        done = C.c_int()
        check(self._lib.lem_poll(self._h, C.c_uint64(ticket), C.byref(done)), "lem_poll")
        return bool(done.value)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        check(self._lib.lem_wait(self._h, C.c_uint64(ticket), float(timeout_s)), "lem_wait")

    def status(self, ticket: int) -> int:
        done = C.c_int()
        return int(self._lib.lem_poll(self._h, C.c_uint64(ticket), C.byref(done)))

    def stats(self) -> dict:
        st = ServerStats()
        check(self._lib.lem_server_get_stats(self._h, C.byref(st)), "lem_server_get_stats")
        out = {}
        for f, _ in ServerStats._fields_:
            v = getattr(st, f)
            out[f] = list(v) if f.startswith("tier_") else v
        return out

    def reset_stats(self):
        check(self._lib.lem_server_reset_stats(self._h), "lem_server_reset_stats")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lem_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """lem_batch: one CUDA graph advancing many contexts' device states together."""

    def __init__(self, ctxs, states, steps_per_launch: int = 1, lanes: int = 8, stream=None):
        lib = load()
        self._lib = lib
        n = len(ctxs)
        if n != len(states):
            raise ValueError("one state per context")
        for c, s in zip(ctxs, states):
            check_device_state(s, c.npts, c.complex, c.device)
        self._ctxs = list(ctxs)
        self._states = list(states)  # keep the captured tensors alive
        hc = (C.c_void_p * n)(*[c._h.value for c in ctxs])
        hs = (C.c_void_p * n)(*[s.data_ptr() for s in states])
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream is not None else None
        check(lib.lem_batch_create(hc, hs, n, int(steps_per_launch), int(lanes), st, C.byref(h)), "lem_batch_create")
        self._h = h
        self.n = n

    def run(self, launches: int = 1):
        check(self._lib.lem_batch_run(self._h, int(launches)), "lem_batch_run")

    def schedule(self):
        est = np.zeros(self.n)
        lane = np.zeros(self.n, dtype=np.int32)
        check(self._lib.lem_batch_schedule(self._h, est.ctypes.data_as(C.c_void_p), lane.ctypes.data_as(C.c_void_p)),
              "lem_batch_schedule")
        return est, lane

    def info(self):
        f, lm, fm = C.c_int(), C.c_double(), C.c_double()
        check(self._lib.lem_batch_info(self._h, C.byref(f), C.byref(lm), C.byref(fm)), "lem_batch_info")
        return {"fused": bool(f.value), "lanes_ms": lm.value, "fused_ms": fm.value}

    def sync(self):
        check(self._lib.lem_batch_sync(self._h), "lem_batch_sync")

    def candidates(self):
        """The autotuner's timed candidates: list of dicts (fused, lanes, n_cap, ms, chosen)."""
        n = C.c_int()
        check(self._lib.lem_batch_candidates(self._h, 0, None, C.byref(n)), "lem_batch_candidates")
        arr = (BatchCandidate * max(1, n.value))()
        check(self._lib.lem_batch_candidates(self._h, n.value, arr, C.byref(n)), "lem_batch_candidates")
        return [{f: getattr(arr[k], f) for f, _ in BatchCandidate._fields_} for k in range(n.value)]

    def gemm_work(self):
        """(algorithmic, executed) FLOPs of one fused GEMM launch (fused schedule only)."""
        a, e = C.c_double(), C.c_double()
        check(self._lib.lem_batch_gemm_work(self._h, C.byref(a), C.byref(e)), "lem_batch_gemm_work")
        return a.value, e.value

    def profile(self, nsteps: int = 1):
        g, r, o, f = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        check(self._lib.lem_batch_profile(self._h, int(nsteps), C.byref(g), C.byref(r), C.byref(o), C.byref(f)),
              "lem_batch_profile")
        return {"gemm_ms": g.value, "residual_ms": r.value, "other_ms": o.value, "gemm_flops": f.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.lem_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
