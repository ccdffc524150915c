"""Python binding of libpmmm.so, the GB300 particle mesh multipole method library.

Argument marshalling only: every step of a force evaluation runs in the CUDA
kernels of ``csrc/`` behind the C ABI of ``include/pmmm.h``.  PyTorch supplies
device memory and the stream.  There is no CPU fallback: if the compiled
library is missing, loading fails with an error naming the build step.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpmmm.so")

OK = 0
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_OUT_OF_BOX, ERR_NONFINITE_INPUT = -1, -2, -3, -4
ERR_CUDA, ERR_TIMEOUT, ERR_OOM = -5, -6, -7
OPEN, PERIODIC = 0, 1
FP64, FP32, FP32_SPLITBF16_M2L = 0, 1, 2
NEAR_AUTO, NEAR_CELL_ITEMS, NEAR_PER_TARGET, NEAR_CELL_ITEMS_SPLIT = 0, 1, 2, 3
NEAR_AUTO_OCCUPANCY = 8
EXPORT_PERM, EXPORT_SORTED_CELL, EXPORT_CELL_START = 1, 2, 3
EXPORT_MULTIPOLE, EXPORT_LOCAL, EXPORT_CORR, EXPORT_FAR = 4, 5, 6, 7
INFO_K, INFO_C, INFO_CG, INFO_KH, INFO_N, INFO_WORKSPACE_BYTES, INFO_LAUNCHES = 1, 2, 3, 4, 5, 6, 7
INFO_SYSTEMS = 8
INFO_TUNED_NEAR, INFO_M2L_TILE, INFO_REFINE, INFO_M2L_ARITH, INFO_SPLIT = 9, 10, 11, 12, 13
M2L_ARITH_FP64_SIMT, M2L_ARITH_FP32_SIMT, M2L_ARITH_SPLITBF16_TC = 0, 1, 2
MAX_SYSTEMS = 65535
SUR_PARAMS, SUR_ADAM_M, SUR_ADAM_V, SUR_IN_SCALE, SUR_OUT_SCALE = 1, 2, 3, 4, 5
SUR_INFO_STEP, SUR_INFO_FALLBACK, SUR_INFO_CLOW, SUR_INFO_CHIGH, SUR_INFO_ROWS = 1, 2, 3, 4, 5
SUR_IN, SUR_OUT_ROWS, SUR_NPARAM = 432, 128, 209536


class PmmmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = _lib().pmmm_strerror(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


class _Config(ctypes.Structure):
    _fields_ = [
        ("box_lo", ctypes.c_double * 3),
        ("box_len", ctypes.c_double * 3),
        ("mesh", ctypes.c_int32 * 3),
        ("p", ctypes.c_int32),
        ("cutoff", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("near_field", ctypes.c_int32),
        ("sign", ctypes.c_double),
        ("ewald_alpha", ctypes.c_double),
        ("ewald_nmax", ctypes.c_int32),
        ("refine", ctypes.c_int32),
        ("reserved", ctypes.c_int32 * 6),
    ]


_LIB = None

# Every function the C ABI declares, with its ctypes signature.
_SIGS = {
    "pmmm_abi_version": (ctypes.c_int, []),
    "pmmm_config_init": (None, [ctypes.POINTER(_Config)]),
    "pmmm_plan_create": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "pmmm_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pmmm_plan_reserve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "pmmm_compute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pmmm_compute_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pmmm_compute_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pmmm_compute_batched_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
    "pmmm_compute_batched_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p]),
    "pmmm_plan_reserve_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64]),
    "pmmm_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32]),
    "pmmm_plan_status": (ctypes.c_int, [ctypes.c_void_p]),
    "pmmm_plan_export": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "pmmm_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "pmmm_plan_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pmmm_plan_stage_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "pmmm_stage_name": (ctypes.c_char_p, [ctypes.c_int]),
    "pmmm_bin_sort_static": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "pmmm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pmmm_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "pmmm_surrogate_create": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_void_p)]),
    "pmmm_surrogate_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "pmmm_surrogate_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]),
    "pmmm_surrogate_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]),
    "pmmm_surrogate_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "pmmm_surrogate_set_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "pmmm_surrogate_set_fallback": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "pmmm_surrogate_training_pair": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "pmmm_surrogate_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "pmmm_surrogate_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pmmm_surrogate_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
    "pmmm_probe_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "pmmm_surrogate_compute": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
}


def library_path() -> str:
    return LIB_PATH


def _lib():
    """Loads libpmmm.so; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                               f"g.build()\"` (nvcc, sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def build(force: bool = False) -> str:
    """Compiles libpmmm.so in-tree (see buildlib.py)."""
    from . import buildlib
    return buildlib.build(force=force)


STATIC_SORT_MAX_N = 65536


def bin_sort_static(cfg: Config, pos, perm, cell_start, stream=None) -> int:
    """Binning and stable cell sort with no device allocation (pmmm_bin_sort_static):
    pos (n, 3) CUDA tensor in the precision's dtype; perm int32 (>= n elements) and
    cell_start int32 (>= K+1 elements) CUDA tensors receive the results.  All three
    must be contiguous and on the current device; anything else raises ValueError
    before the library is called.  Returns the status code."""
    import torch
    dt = torch.float64 if int(cfg.precision) == FP64 else torch.float32
    dev = torch.cuda.current_device()
    K = int(cfg.mesh[0]) * int(cfg.mesh[1]) * int(cfg.mesh[2])
    for t, nm in ((pos, "pos"), (perm, "perm"), (cell_start, "cell_start")):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError(f"{nm} must be a contiguous CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{nm} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    if pos.dtype != dt:
        raise ValueError(f"pos must be {dt} for this precision")
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError("pos must have shape (n, 3)")
    n = int(pos.shape[0])
    if perm.dtype != torch.int32 or perm.numel() < n:
        raise ValueError("perm must be an int32 tensor of at least n elements")
    if cell_start.dtype != torch.int32 or cell_start.numel() < K + 1:
        raise ValueError("cell_start must be an int32 tensor of at least K + 1 elements")
    c = cfg.to_c()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(_lib().pmmm_bin_sort_static(ctypes.byref(c), n, ctypes.c_void_p(pos.data_ptr()),
                                           ctypes.c_void_p(perm.data_ptr()), ctypes.c_void_p(cell_start.data_ptr()),
                                           ctypes.c_void_p(stream.cuda_stream)))


PROBE_FP32_FMA, PROBE_FP32X2_FMA, PROBE_FP64_FMA = 0, 1, 2


def probe_peak(what: int, stream=None) -> float:
    """pmmm_probe_peak: measured FMA rate of the current GPU in flop/s (2 x FMAs/s)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    v = ctypes.c_double(0.0)
    _check(_lib().pmmm_probe_peak(int(what), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(v)),
           "pmmm_probe_peak")
    return float(v.value)


def selftest_wait_timeout(polls: int = 1 << 16, stream=None) -> int:
    """pmmm_selftest_wait_timeout: a bounded device-side wait that runs out; returns the status."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(_lib().pmmm_selftest_wait_timeout(ctypes.c_void_p(stream.cuda_stream), int(polls)))


def stage_names():
    out, i = [], 0
    while True:
        s = _lib().pmmm_stage_name(i)
        if s is None:
            return out
        out.append(s.decode())
        i += 1


@dataclass
class Config:
    """Mirror of pmmm_config (include/pmmm.h)."""
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_len: tuple = (1.0, 1.0, 1.0)
    mesh: tuple = (8, 8, 8)
    p: int = 4
    cutoff: int = 1
    boundary: int = OPEN
    precision: int = FP64
    sign: float = 1.0
    ewald_alpha: float = 0.0
    ewald_nmax: int = 0
    near_field: int = NEAR_AUTO
    refine: int = 0  # two-level PMMM (Sec. 5): r >= 2 -> every r^3 block of the mesh is one coarse cell

    def to_c(self) -> _Config:
        c = _Config()
        _lib().pmmm_config_init(ctypes.byref(c))
        for a in range(3):
            c.box_lo[a] = float(self.box_lo[a])
            c.box_len[a] = float(self.box_len[a])
            c.mesh[a] = int(self.mesh[a])
        c.p, c.cutoff, c.boundary, c.precision = int(self.p), int(self.cutoff), int(self.boundary), int(self.precision)
        c.sign, c.ewald_alpha, c.ewald_nmax = float(self.sign), float(self.ewald_alpha), int(self.ewald_nmax)
        c.near_field = int(self.near_field)
        c.refine = int(self.refine)
        return c

    @property
    def fp64(self) -> bool:
        return self.precision == FP64


def _check(st: int, what: str):
    if st != OK:
        raise PmmmError(st, what)


class Plan:
    """A PMMM plan: geometry, order, precision, precomputed kernel spectra and workspace.

    ``compute`` takes CUDA tensors (float64 for FP64, float32 otherwise):
    pos (n, 3), q (n,), and returns (phi (n,), force (n, 3), energy or None).
    """

    def __init__(self, cfg: Config, stream=None):
        import torch
        self.cfg = cfg
        self._c = cfg.to_c()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = ctypes.c_void_p()
        _check(_lib().pmmm_plan_create(ctypes.byref(self._c), ctypes.c_void_p(stream.cuda_stream),
                                       ctypes.byref(handle)), "pmmm_plan_create")
        self._h = handle
        self.dtype = torch.float64 if cfg.fp64 else torch.float32
        self.np_dtype = np.float64 if cfg.fp64 else np.float32

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().pmmm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------ compute
    def reserve(self, n: int):
        _check(_lib().pmmm_plan_reserve(self._h, int(n)), "pmmm_plan_reserve")

    def compute(self, pos, q, phi=None, force=None, energy: bool = False, check: bool = False):
        import torch
        n = int(q.shape[0])
        for t, nm in ((pos, "pos"), (q, "q")):
            if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
                raise ValueError(f"{nm} must be a contiguous CUDA {self.dtype} tensor")
        if pos.shape != (n, 3):
            raise ValueError("pos must have shape (n, 3)")
        if phi is None:
            phi = torch.empty(n, dtype=self.dtype, device=q.device)
        if force is None:
            force = torch.empty((n, 3), dtype=self.dtype, device=q.device)
        e = ctypes.c_double(0.0)
        st = _lib().pmmm_compute(self._h, n, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                 ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(force.data_ptr()),
                                 ctypes.byref(e) if energy else None)
        _check(st, "pmmm_compute")
        if check and not energy:
            _check(_lib().pmmm_plan_status(self._h), "pmmm_compute (device status)")
        return phi, force, (e.value if energy else None)

    def compute_raw(self, n: int, pos_ptr: int, q_ptr: int, phi_ptr: int, force_ptr: int) -> int:
        """Queue one evaluation on raw device pointers; returns the status."""
        return _lib().pmmm_compute(self._h, int(n), ctypes.c_void_p(pos_ptr), ctypes.c_void_p(q_ptr),
                                   ctypes.c_void_p(phi_ptr), ctypes.c_void_p(force_ptr), None)

    def compute_host(self, pos, q, phi=None, force=None, energy: bool = False):
        """Host arrays in and out (numpy or pinned CPU tensors); synchronous."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        n = int(q.shape[0])
        if phi is None:
            phi = np.empty(n, dtype=self.np_dtype)
        if force is None:
            force = np.empty((n, 3), dtype=self.np_dtype)
        e = ctypes.c_double(0.0)
        st = _lib().pmmm_compute_host(self._h, n, ctypes.c_void_p(ptr(pos)), ctypes.c_void_p(ptr(q)),
                                      ctypes.c_void_p(ptr(phi)), ctypes.c_void_p(ptr(force)),
                                      ctypes.byref(e) if energy else None)
        _check(st, "pmmm_compute_host")
        return phi, force, (e.value if energy else None)

    # ------------------------------------------------------------------ batched form
    @staticmethod
    def _offsets(counts):
        off = np.zeros(len(counts) + 1, dtype=np.int64)
        off[1:] = np.cumsum(np.asarray(counts, dtype=np.int64))
        return off

    def reserve_batched(self, nsys: int, n: int):
        _check(_lib().pmmm_plan_reserve_batched(self._h, int(nsys), int(n)), "pmmm_plan_reserve_batched")

    def compute_batched(self, counts, pos, q, phi=None, force=None, energies: bool = False):
        """Systems of counts[s] particles, concatenated in pos (n, 3) and q (n,) CUDA
        tensors; returns (phi, force, per-system energies as numpy or None)."""
        import torch
        off = self._offsets(counts)
        n = int(off[-1])
        for t, nm in ((pos, "pos"), (q, "q")):
            if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
                raise ValueError(f"{nm} must be a contiguous CUDA {self.dtype} tensor")
        if pos.shape != (n, 3) or q.shape != (n,):
            raise ValueError("pos must be (n, 3) and q (n,) with n = sum(counts)")
        if phi is None:
            phi = torch.empty(n, dtype=self.dtype, device=q.device)
        if force is None:
            force = torch.empty((n, 3), dtype=self.dtype, device=q.device)
        e = np.zeros(len(counts), dtype=np.float64)
        st = _lib().pmmm_compute_batched(self._h, len(counts), ctypes.c_void_p(off.ctypes.data),
                                         ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                         ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(force.data_ptr()),
                                         ctypes.c_void_p(e.ctypes.data) if energies else None)
        _check(st, "pmmm_compute_batched")
        return phi, force, (e if energies else None)

    def compute_batched_raw(self, offsets: np.ndarray, pos_ptr: int, q_ptr: int, phi_ptr: int, force_ptr: int,
                            graph: bool = False) -> int:
        """Queue one batched evaluation on raw device pointers (offsets: int64 numpy, nsys+1);
        graph=True replays a CUDA graph of the evaluation (pmmm_compute_batched_graph)."""
        f = _lib().pmmm_compute_batched_graph if graph else _lib().pmmm_compute_batched
        return f(self._h, len(offsets) - 1, ctypes.c_void_p(offsets.ctypes.data), ctypes.c_void_p(pos_ptr),
                 ctypes.c_void_p(q_ptr), ctypes.c_void_p(phi_ptr), ctypes.c_void_p(force_ptr), None)

    def compute_batched_graph(self, counts, pos, q, phi, force, energies: bool = False):
        """compute_batched through a CUDA graph (pmmm_compute_batched_graph); phi and
        force must be given, and the same tensors reused to replay without a new capture."""
        off = self._offsets(counts)
        e = np.zeros(len(counts), dtype=np.float64)
        st = _lib().pmmm_compute_batched_graph(self._h, len(counts), ctypes.c_void_p(off.ctypes.data),
                                               ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                               ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(force.data_ptr()),
                                               ctypes.c_void_p(e.ctypes.data) if energies else None)
        _check(st, "pmmm_compute_batched_graph")
        return phi, force, (e if energies else None)

    def compute_batched_host(self, counts, pos, q, phi=None, force=None):
        """Host arrays in and out (numpy or pinned CPU tensors); synchronous; returns
        (phi, force, per-system energies)."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        off = self._offsets(counts)
        n = int(off[-1])
        if phi is None:
            phi = np.empty(n, dtype=self.np_dtype)
        if force is None:
            force = np.empty((n, 3), dtype=self.np_dtype)
        e = np.zeros(len(counts), dtype=np.float64)
        st = _lib().pmmm_compute_batched_host(self._h, len(counts), ctypes.c_void_p(off.ctypes.data),
                                              ctypes.c_void_p(ptr(pos)), ctypes.c_void_p(ptr(q)),
                                              ctypes.c_void_p(ptr(phi)), ctypes.c_void_p(ptr(force)),
                                              ctypes.c_void_p(e.ctypes.data))
        _check(st, "pmmm_compute_batched_host")
        return phi, force, e

    def autotune(self, counts, pos, q, reps: int = 3):
        """pmmm_plan_autotune on these inputs (counts: particles per system); returns the
        (near-field kernel, tensor-core M2L tile) chosen."""
        off = self._offsets(counts)
        _check(_lib().pmmm_plan_autotune(self._h, len(counts), ctypes.c_void_p(off.ctypes.data),
                                         ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(q.data_ptr()), int(reps)),
               "pmmm_plan_autotune")
        return self.info(INFO_TUNED_NEAR), self.info(INFO_M2L_TILE)

    def status(self) -> int:
        return int(_lib().pmmm_plan_status(self._h))

    # ------------------------------------------------------------------ diagnostics
    def info(self, what: int) -> int:
        v = ctypes.c_int64(0)
        _check(_lib().pmmm_plan_info(self._h, int(what), ctypes.byref(v)), "pmmm_plan_info")
        return int(v.value)

    def export(self, what: int) -> np.ndarray:
        n, C, B = self.info(INFO_N), self.info(INFO_C), self.info(INFO_SYSTEMS)
        K = self.info(INFO_K) * B
        shapes = {
            EXPORT_PERM: ((n,), np.int32),
            EXPORT_SORTED_CELL: ((n,), np.int32),
            EXPORT_CELL_START: ((K + 1,), np.int32),
            EXPORT_MULTIPOLE: ((C, K), np.float64),
            EXPORT_LOCAL: ((C, K), np.float64),
            EXPORT_CORR: ((8,) if B == 1 else (B, 8), np.float64),
            EXPORT_FAR: ((n, 4), np.float64),
        }
        shape, dt = shapes[what]
        out = np.zeros(shape, dtype=dt)
        _check(_lib().pmmm_plan_export(self._h, int(what), ctypes.c_void_p(out.ctypes.data), out.nbytes),
               "pmmm_plan_export")
        return out

    def set_timing(self, on: bool = True):
        _check(_lib().pmmm_plan_set_timing(self._h, int(bool(on))), "pmmm_plan_set_timing")

    def stage_times(self) -> dict:
        names = stage_names()
        buf = (ctypes.c_float * len(names))()
        k = _lib().pmmm_plan_stage_times(self._h, buf, len(names))
        if k < 0:
            raise PmmmError(k, "pmmm_plan_stage_times")
        return {names[i]: float(buf[i]) for i in range(k)}


class Surrogate:
    """Learned local-expansion correction (pmmm_surrogate_* of include/pmmm.h): an
    order-3 plan whose locals are corrected toward order p_high by a multilayer
    perceptron before L2P, with the plain order-p_high plan as training target and
    fallback.  cfg must have p = 3, cutoff 1 and FP32 precision."""

    def __init__(self, cfg: Config, p_high: int = 10, stream=None):
        import torch
        self.cfg = cfg
        self.p_high = int(p_high)
        c = cfg.to_c()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(_lib().pmmm_surrogate_create(ctypes.byref(c), self.p_high, ctypes.c_void_p(stream.cuda_stream),
                                            ctypes.byref(h)), "pmmm_surrogate_create")
        self._h = h
        self.rows = self.info(SUR_INFO_ROWS)
        self.c_high = self.info(SUR_INFO_CHIGH)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().pmmm_surrogate_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, what: int) -> int:
        v = ctypes.c_int64(0)
        _check(_lib().pmmm_surrogate_info(self._h, int(what), ctypes.byref(v)), "pmmm_surrogate_info")
        return int(v.value)

    def _count(self, what):
        return {SUR_PARAMS: SUR_NPARAM, SUR_ADAM_M: SUR_NPARAM, SUR_ADAM_V: SUR_NPARAM, SUR_IN_SCALE: 16,
                SUR_OUT_SCALE: self.c_high}[what]

    def get(self, what: int) -> np.ndarray:
        out = np.zeros(self._count(what), dtype=np.float32)
        _check(_lib().pmmm_surrogate_get(self._h, int(what), ctypes.c_void_p(out.ctypes.data), out.size),
               "pmmm_surrogate_get")
        return out

    def set(self, what: int, values):
        a = np.ascontiguousarray(values, dtype=np.float32).reshape(-1)
        _check(_lib().pmmm_surrogate_set(self._h, int(what), ctypes.c_void_p(a.ctypes.data), a.size),
               "pmmm_surrogate_set")

    @property
    def step(self) -> int:
        return self.info(SUR_INFO_STEP)

    @step.setter
    def step(self, v: int):
        _check(_lib().pmmm_surrogate_set_step(self._h, int(v)), "pmmm_surrogate_set_step")

    @property
    def fallback(self) -> bool:
        return bool(self.info(SUR_INFO_FALLBACK))

    @fallback.setter
    def fallback(self, on: bool):
        _check(_lib().pmmm_surrogate_set_fallback(self._h, int(bool(on))), "pmmm_surrogate_set_fallback")

    def training_pair(self, pos, q, X, T, stats: np.ndarray = None):
        """Features X (CUDA bfloat16 [rows, 432] view) and targets T (CUDA float32 [rows, 128])."""
        st = _lib().pmmm_surrogate_training_pair(
            self._h, int(q.shape[0]), ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(q.data_ptr()),
            ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
            ctypes.c_void_p(stats.ctypes.data) if stats is not None else None)
        _check(st, "pmmm_surrogate_training_pair")

    def forward(self, X, out):
        rows = int(X.shape[0])
        _check(_lib().pmmm_surrogate_forward(self._h, ctypes.c_void_p(X.data_ptr()), rows,
                                             ctypes.c_void_p(out.data_ptr())), "pmmm_surrogate_forward")
        return out

    def gradients(self, X, T):
        g = np.zeros(SUR_NPARAM, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(_lib().pmmm_surrogate_gradients(self._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                               int(X.shape[0]), ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)),
               "pmmm_surrogate_gradients")
        return float(loss.value), g

    def train_step_raw(self, x_ptr: int, t_ptr: int, rows: int, lr: float, want_loss: bool = False):
        loss = ctypes.c_double(0.0)
        st = _lib().pmmm_surrogate_train_step(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(rows),
                                              float(lr), ctypes.byref(loss) if want_loss else None)
        _check(st, "pmmm_surrogate_train_step")
        return float(loss.value) if want_loss else None

    def compute(self, pos, q, phi=None, force=None, energy: bool = False):
        import torch
        n = int(q.shape[0])
        if phi is None:
            phi = torch.empty(n, dtype=torch.float32, device=q.device)
        if force is None:
            force = torch.empty((n, 3), dtype=torch.float32, device=q.device)
        e = ctypes.c_double(0.0)
        st = _lib().pmmm_surrogate_compute(self._h, n, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                           ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(force.data_ptr()),
                                           ctypes.byref(e) if energy else None)
        _check(st, "pmmm_surrogate_compute")
        return phi, force, (e.value if energy else None)

    def compute_raw(self, n: int, pos_ptr: int, q_ptr: int, phi_ptr: int, force_ptr: int) -> int:
        return _lib().pmmm_surrogate_compute(self._h, int(n), ctypes.c_void_p(pos_ptr), ctypes.c_void_p(q_ptr),
                                             ctypes.c_void_p(phi_ptr), ctypes.c_void_p(force_ptr), None)
