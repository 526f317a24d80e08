"""Python binding of libttice (include/ttice.h): argument marshalling only.

Every entry point of the C ABI has a function of the same name here; each converts torch tensors to
device pointers and the current torch CUDA stream to a cudaStream_t and calls the library.  All the
arithmetic of the update runs in the library's CUDA kernels; there is no Python or CPU path.  If the
shared library has not been built, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_void_p

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libttice.so")

# constants mirrored from include/ttice.h
TTICE_OK, TTICE_EINVAL, TTICE_ENOMEM, TTICE_ECAPACITY = 0, -1, -2, -3
TTICE_ENONFINITE, TTICE_ETIMEOUT, TTICE_ECUDA, TTICE_EINTERNAL = -4, -5, -6, -7
TTICE_SKIP_NONE, TTICE_SKIP_EXACT, TTICE_SKIP_MEAN = 0, 1, 2
TTICE_EPSUPD_EXACT, TTICE_EPSUPD_APPROX = 0, 1
TTICE_FP64, TTICE_FP32, TTICE_TF32, TTICE_BF16, TTICE_SPLIT_BF16 = 0, 1, 2, 3, 4
TTICE_F32, TTICE_F64 = 0, 1
TTICE_NOALLOC_MAX_ELEMS = 4 * 1024 * 1024

PRECISIONS = {"fp64": TTICE_FP64, "fp32": TTICE_FP32, "tf32": TTICE_TF32, "bf16": TTICE_BF16,
              "split_bf16": TTICE_SPLIT_BF16}
SKIP_MODES = {"none": TTICE_SKIP_NONE, "exact": TTICE_SKIP_EXACT, "mean": TTICE_SKIP_MEAN}


class ttice_heuristics(ctypes.Structure):
    _fields_ = [("skip_mode", c_int), ("subselect", c_int), ("eps_upd_mode", c_int),
                ("occupancy_tau", c_double), ("precision", c_int), ("input_dtype", c_int)]


class ttice_capacity(ctypes.Structure):
    _fields_ = [("max_batch", c_int64), ("max_rank", c_int64), ("obs_reserve", c_int64)]


class ttice_update_stats(ctypes.Structure):
    _fields_ = [("skipped", c_int32), ("n_selected", c_int32), ("rel_err_before", c_double),
                ("eps_upd", c_double), ("eps_core", c_double), ("ranks", c_int64 * 18),
                ("new_dirs", c_int32 * 16), ("n_obs", c_int64), ("core_elems", c_int64),
                ("eig_sweep_limit", c_int32), ("eig_sweeps", c_int32),
                ("krylov_solves", c_int32), ("krylov_fallbacks", c_int32)]


TTICE_NPHASES = 8
PHASE_NAMES = ["k1_stage1", "chain", "residual", "gram", "eig", "orth_append", "d_project", "final"]


class ttice_profile(ctypes.Structure):
    _fields_ = [("ms", c_double * TTICE_NPHASES), ("bytes", c_double * TTICE_NPHASES),
                ("flops", c_double * TTICE_NPHASES), ("count", c_int64 * TTICE_NPHASES),
                ("updates", c_int64)]


class TTICEError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = f"{what}: {ttice_strerror(code)} ({code})"
        if code in (TTICE_ECUDA, TTICE_ENOMEM):
            msg += f" [{ttice_last_cuda_error()}]"
        super().__init__(msg)
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2211_12487_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P = POINTER
    sig = {
        "ttice_default_heuristics": (None, [P(ttice_heuristics)]),
        "ttice_default_capacity": (None, [P(ttice_capacity)]),
        "ttice_create": (c_int, [P(c_int64), c_int, c_double, P(ttice_heuristics), P(ttice_capacity),
                                 P(c_void_p)]),
        "ttice_update": (c_int, [c_void_p, c_void_p, c_int64, c_void_p]),
        "ttice_project": (c_int, [c_void_p, c_void_p, c_int64, c_void_p, c_void_p, c_void_p]),
        "ttice_ranks": (c_int, [c_void_p, P(c_int64)]),
        "ttice_reconstruct": (c_int, [c_void_p, c_int64, c_int64, c_void_p, c_int, c_void_p]),
        "ttice_stats": (c_int, [c_void_p, P(ttice_update_stats)]),
        "ttice_info": (c_int, [c_void_p, P(c_int), P(c_int64), P(c_int)]),
        "ttice_get_core": (c_int, [c_void_p, c_int, c_void_p, P(c_int64), P(c_int64)]),
        "ttice_get_last_core": (c_int, [c_void_p, c_void_p, P(c_int64), P(c_int64)]),
        "ttice_load": (c_int, [c_void_p, P(c_int64), P(c_void_p), c_void_p, c_int64]),
        "ttice_capacities": (c_int, [c_void_p, P(c_int64)]),
        "ttice_device_bytes": (c_int, [c_void_p, P(c_int64)]),
        "ttice_capacity_miss": (c_int, [c_void_p, P(c_int), P(c_int64)]),
        "ttice_projected_bytes": (c_int, [P(c_int64), c_int, P(ttice_heuristics), P(ttice_capacity), P(c_int64),
                                          P(c_int64)]),
        "ttice_reserve_rank": (c_int, [c_void_p, c_int, c_int64]),
        "ttice_checkpoint_write": (c_int, [ctypes.c_char_p, c_int, P(c_int64), c_double, P(ttice_heuristics),
                                           P(c_int64), P(c_void_p), c_void_p, c_int64]),
        "ttice_checkpoint_read": (c_int, [ctypes.c_char_p, P(c_int), P(c_int64), P(c_double),
                                          P(ttice_heuristics), P(c_int64), P(c_int64), P(c_void_p), c_void_p]),
        "ttice_save": (c_int, [c_void_p, ctypes.c_char_p]),
        "ttice_open": (c_int, [ctypes.c_char_p, P(ttice_capacity), P(c_void_p)]),
        "ttice_profile_enable": (c_int, [c_void_p, c_int]),
        "ttice_profile_read": (c_int, [c_void_p, P(ttice_profile)]),
        "ttice_kernel_launches": (c_int64, []),
        "ttice_reconstruct_noalloc": (c_int, [c_void_p, c_int64, c_int64, c_void_p, c_int, c_void_p]),
        "ttice_destroy": (None, [c_void_p]),
        "ttice_strerror": (ctypes.c_char_p, [c_int]),
        "ttice_last_cuda_error": (ctypes.c_char_p, []),
        "ttice_test_fail_alloc": (None, [c_int64]),
        "ttice_test_wait_limit_ns": (None, [ctypes.c_uint64]),
        "ttice_test_drop_copy": (None, [c_int64]),
        "ttice_test_tc_cgs_min": (None, [c_double]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def ttice_strerror(code: int) -> str:
    return _lib.ttice_strerror(int(code)).decode()


def ttice_last_cuda_error() -> str:
    return _lib.ttice_last_cuda_error().decode()


def ttice_test_fail_alloc(n: int) -> None:
    _lib.ttice_test_fail_alloc(int(n))


def ttice_test_wait_limit_ns(ns: int) -> None:
    _lib.ttice_test_wait_limit_ns(int(ns))


def ttice_test_drop_copy(chunk: int) -> None:
    _lib.ttice_test_drop_copy(int(chunk))


def ttice_test_tc_cgs_min(flops: float) -> None:
    _lib.ttice_test_tc_cgs_min(float(flops))


def _check(code: int, what: str):
    if code != TTICE_OK:
        raise TTICEError(code, what)


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def ttice_default_heuristics() -> ttice_heuristics:
    h = ttice_heuristics()
    _lib.ttice_default_heuristics(ctypes.byref(h))
    return h


def ttice_default_capacity() -> ttice_capacity:
    c = ttice_capacity()
    _lib.ttice_default_capacity(ctypes.byref(c))
    return c


def ttice_create(dims, eps: float, heuristics: ttice_heuristics | None = None,
                 capacity: ttice_capacity | None = None) -> int:
    arr = (c_int64 * len(dims))(*[int(n) for n in dims])
    out = c_void_p()
    _check(_lib.ttice_create(arr, len(dims), float(eps),
                             ctypes.byref(heuristics) if heuristics is not None else None,
                             ctypes.byref(capacity) if capacity is not None else None,
                             ctypes.byref(out)), "ttice_create")
    return out.value


def ttice_update(h: int, Y: torch.Tensor, batch: int | None = None, stream=None) -> None:
    assert Y.is_cuda and Y.is_contiguous()
    b = Y.shape[0] if batch is None else batch
    _check(_lib.ttice_update(h, Y.data_ptr(), int(b), _stream_ptr(stream)), "ttice_update")


def ttice_project(h: int, Y: torch.Tensor, coeffs: torch.Tensor | None, rel_err: torch.Tensor | None,
                  stream=None) -> None:
    assert Y.is_cuda and Y.is_contiguous()
    _check(_lib.ttice_project(h, Y.data_ptr(), int(Y.shape[0]),
                              coeffs.data_ptr() if coeffs is not None else None,
                              rel_err.data_ptr() if rel_err is not None else None,
                              _stream_ptr(stream)), "ttice_project")


def ttice_ranks(h: int, d: int) -> list[int]:
    arr = (c_int64 * (d + 2))()
    _check(_lib.ttice_ranks(h, arr), "ttice_ranks")
    return list(arr)


def ttice_info(h: int) -> tuple[list[int], int]:
    """(dims, device index) of handle h."""
    d = c_int()
    dims = (c_int64 * 16)()
    dev = c_int()
    _check(_lib.ttice_info(h, ctypes.byref(d), dims, ctypes.byref(dev)), "ttice_info")
    return [int(dims[i]) for i in range(d.value)], int(dev.value)


def _check_out(h: int, count: int, out: torch.Tensor, what: str) -> int:
    """The output of a reconstruction must be a contiguous FP32/FP64 tensor on the handle's device
    holding exactly count observations (the library writes count * n_1 ... n_d elements)."""
    if not (out.is_cuda and out.is_contiguous() and out.dtype in (torch.float32, torch.float64)):
        raise ValueError(f"{what}: out must be a contiguous float32/float64 CUDA tensor")
    dims, dev = ttice_info(h)
    n = 1
    for x in dims:
        n *= x
    if out.numel() != int(count) * n:
        raise ValueError(f"{what}: out holds {out.numel()} elements, {int(count)} observations need {int(count) * n}")
    if out.device.index != dev:
        raise ValueError(f"{what}: out is on cuda:{out.device.index}, the handle on cuda:{dev}")
    return TTICE_F32 if out.dtype == torch.float32 else TTICE_F64


def ttice_reconstruct(h: int, first: int, count: int, out: torch.Tensor, stream=None) -> None:
    dt = _check_out(h, count, out, "ttice_reconstruct")
    _check(_lib.ttice_reconstruct(h, int(first), int(count), out.data_ptr(), dt, _stream_ptr(stream)),
           "ttice_reconstruct")


def ttice_reconstruct_noalloc(h: int, first: int, count: int, out: torch.Tensor, stream=None) -> None:
    """Same result as ttice_reconstruct, computed without any device allocation (fixed library
    scratch; see include/ttice.h for the size limit and the sharing rules)."""
    dt = _check_out(h, count, out, "ttice_reconstruct_noalloc")
    _check(_lib.ttice_reconstruct_noalloc(h, int(first), int(count), out.data_ptr(), dt,
                                          _stream_ptr(stream)), "ttice_reconstruct_noalloc")


def ttice_stats(h: int) -> dict:
    s = ttice_update_stats()
    _check(_lib.ttice_stats(h, ctypes.byref(s)), "ttice_stats")
    return s


def ttice_get_core(h: int, i: int) -> np.ndarray:
    rows, cols = c_int64(), c_int64()
    _check(_lib.ttice_get_core(h, i, None, ctypes.byref(rows), ctypes.byref(cols)), "ttice_get_core")
    out = np.zeros((rows.value, cols.value), dtype=np.float64)
    if out.size:
        _check(_lib.ttice_get_core(h, i, out.ctypes.data, ctypes.byref(rows), ctypes.byref(cols)),
               "ttice_get_core")
    return out


def ttice_get_last_core(h: int) -> np.ndarray:
    n, r = c_int64(), c_int64()
    _check(_lib.ttice_get_last_core(h, None, ctypes.byref(n), ctypes.byref(r)), "ttice_get_last_core")
    out = np.zeros((n.value, r.value), dtype=np.float64)
    if out.size:
        _check(_lib.ttice_get_last_core(h, out.ctypes.data, ctypes.byref(n), ctypes.byref(r)),
               "ttice_get_last_core")
    return out


def ttice_load(h: int, ranks, cores, last: np.ndarray) -> None:
    rk = (c_int64 * len(ranks))(*[int(r) for r in ranks])
    keep = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
    ptrs = (c_void_p * len(keep))(*[k.ctypes.data if k.size else None for k in keep])
    lastc = np.ascontiguousarray(last, dtype=np.float64)
    _check(_lib.ttice_load(h, rk, ptrs, lastc.ctypes.data if lastc.size else None, int(lastc.shape[0])),
           "ttice_load")


def ttice_checkpoint_write(path: str, dims, eps: float, heuristics: ttice_heuristics, ranks, cores,
                           last: np.ndarray) -> None:
    d = len(dims)
    dm = (c_int64 * d)(*[int(n) for n in dims])
    rk = (c_int64 * (d + 1))(*[int(r) for r in ranks])
    keep = [np.ascontiguousarray(c, dtype=np.float64) for c in cores]
    ptrs = (c_void_p * d)(*[k.ctypes.data if k.size else None for k in keep])
    lastc = np.ascontiguousarray(last, dtype=np.float64)
    _check(_lib.ttice_checkpoint_write(os.fsencode(path), d, dm, float(eps), ctypes.byref(heuristics), rk, ptrs,
                                       lastc.ctypes.data if lastc.size else None, int(lastc.shape[0])),
           "ttice_checkpoint_write")


def ttice_checkpoint_read(path: str) -> dict:
    d = c_int()
    dims = (c_int64 * 16)()
    eps = c_double()
    heur = ttice_heuristics()
    ranks = (c_int64 * 17)()
    n_obs = c_int64()
    args = (os.fsencode(path), ctypes.byref(d), dims, ctypes.byref(eps), ctypes.byref(heur), ranks,
            ctypes.byref(n_obs))
    _check(_lib.ttice_checkpoint_read(*args, None, None), "ttice_checkpoint_read")
    dd = d.value
    rk = [int(ranks[i]) for i in range(dd + 1)]
    dm = [int(dims[i]) for i in range(dd)]
    cores = [np.zeros((rk[i] * dm[i], rk[i + 1])) for i in range(dd)]
    last = np.zeros((n_obs.value, rk[dd]))
    ptrs = (c_void_p * dd)(*[c.ctypes.data if c.size else None for c in cores])
    _check(_lib.ttice_checkpoint_read(*args, ptrs, last.ctypes.data if last.size else None),
           "ttice_checkpoint_read")
    return {"dims": dm, "eps": eps.value, "heuristics": heur, "ranks": rk, "cores": cores, "last": last}


def ttice_checkpoint_read_header(path: str) -> dict:
    """dims, eps, heuristics, ranks and n_obs of a checkpoint, without its arrays."""
    d = c_int()
    dims = (c_int64 * 16)()
    eps = c_double()
    heur = ttice_heuristics()
    ranks = (c_int64 * 17)()
    n_obs = c_int64()
    _check(_lib.ttice_checkpoint_read(os.fsencode(path), ctypes.byref(d), dims, ctypes.byref(eps),
                                      ctypes.byref(heur), ranks, ctypes.byref(n_obs), None, None),
           "ttice_checkpoint_read")
    dd = d.value
    return {"dims": [int(dims[i]) for i in range(dd)], "eps": eps.value, "heuristics": heur,
            "ranks": [int(ranks[i]) for i in range(dd + 1)], "n_obs": int(n_obs.value)}


def ttice_save(h: int, path: str) -> None:
    _check(_lib.ttice_save(h, os.fsencode(path)), "ttice_save")


def ttice_open(path: str, capacity: ttice_capacity | None = None) -> int:
    out = c_void_p()
    _check(_lib.ttice_open(os.fsencode(path), ctypes.byref(capacity) if capacity is not None else None,
                           ctypes.byref(out)), "ttice_open")
    return out.value


def ttice_capacities(h: int, d: int) -> list[int]:
    arr = (c_int64 * (d + 1))()
    _check(_lib.ttice_capacities(h, arr), "ttice_capacities")
    return list(arr)


def ttice_device_bytes(h: int) -> int:
    v = c_int64()
    _check(_lib.ttice_device_bytes(h, ctypes.byref(v)), "ttice_device_bytes")
    return int(v.value)


def ttice_projected_bytes(dims, heuristics: ttice_heuristics | None = None,
                          capacity: ttice_capacity | None = None, caps=None) -> int:
    d = len(dims)
    dm = (c_int64 * d)(*[int(n) for n in dims])
    cp = (c_int64 * (d + 1))(*[int(c) for c in caps]) if caps is not None else None
    v = c_int64()
    _check(_lib.ttice_projected_bytes(dm, d, ctypes.byref(heuristics) if heuristics is not None else None,
                                      ctypes.byref(capacity) if capacity is not None else None, cp,
                                      ctypes.byref(v)), "ttice_projected_bytes")
    return int(v.value)


def ttice_capacity_miss(h: int) -> tuple[int, int]:
    k, need = c_int(), c_int64()
    _check(_lib.ttice_capacity_miss(h, ctypes.byref(k), ctypes.byref(need)), "ttice_capacity_miss")
    return int(k.value), int(need.value)


def ttice_reserve_rank(h: int, k: int, cap: int) -> None:
    _check(_lib.ttice_reserve_rank(h, int(k), int(cap)), "ttice_reserve_rank")


def ttice_profile_enable(h: int, on: bool = True) -> None:
    _check(_lib.ttice_profile_enable(h, int(bool(on))), "ttice_profile_enable")


def ttice_profile_read(h: int) -> dict:
    p = ttice_profile()
    _check(_lib.ttice_profile_read(h, ctypes.byref(p)), "ttice_profile_read")
    return {name: {"ms": p.ms[i], "bytes": p.bytes[i], "flops": p.flops[i], "count": p.count[i]}
            for i, name in enumerate(PHASE_NAMES)} | {"updates": p.updates}


def ttice_kernel_launches() -> int:
    return int(_lib.ttice_kernel_launches())


def ttice_destroy(h: int) -> None:
    _lib.ttice_destroy(h)


class TTICE:
    """One incremental TT decomposition living on the current CUDA device."""

    def __init__(self, dims, eps: float, *, skip_mode: str = "exact", subselect: bool = True,
                 eps_upd: str = "exact", tau: float = 1.0, precision: str = "fp64",
                 input_dtype=torch.float32, max_batch: int = 32, max_rank: int = 512,
                 obs_reserve: int = 1024):
        self.dims = [int(n) for n in dims]
        self.d = len(self.dims)
        self.input_dtype = input_dtype
        h = ttice_default_heuristics()
        h.skip_mode = SKIP_MODES[skip_mode]
        h.subselect = int(bool(subselect))
        h.eps_upd_mode = TTICE_EPSUPD_EXACT if eps_upd == "exact" else TTICE_EPSUPD_APPROX
        h.occupancy_tau = float(tau)
        h.precision = PRECISIONS[precision]
        h.input_dtype = TTICE_F32 if input_dtype == torch.float32 else TTICE_F64
        c = ttice_default_capacity()
        c.max_batch, c.max_rank, c.obs_reserve = int(max_batch), int(max_rank), int(obs_reserve)
        self.h = ttice_create(self.dims, eps, h, c)

    def update(self, Y: torch.Tensor, stream=None) -> ttice_update_stats:
        assert Y.dtype == self.input_dtype and tuple(Y.shape[1:]) == tuple(self.dims)
        ttice_update(self.h, Y, Y.shape[0], stream)
        return ttice_stats(self.h)

    def project(self, Y: torch.Tensor, stream=None):
        assert Y.dtype == self.input_dtype and tuple(Y.shape[1:]) == tuple(self.dims)
        rd = self.ranks()[self.d]
        coeffs = torch.zeros((Y.shape[0], rd), dtype=torch.float64, device=Y.device)
        rel = torch.zeros((Y.shape[0],), dtype=torch.float64, device=Y.device)
        ttice_project(self.h, Y, coeffs, rel, stream)
        return coeffs, rel

    def ranks(self) -> list[int]:
        return ttice_ranks(self.h, self.d)

    def reconstruct(self, first: int, count: int, dtype=torch.float64, device="cuda") -> torch.Tensor:
        out = torch.empty((count, *self.dims), dtype=dtype, device=device)
        ttice_reconstruct(self.h, first, count, out)
        return out

    def stats(self):
        return ttice_stats(self.h)

    def core(self, i: int) -> np.ndarray:
        return ttice_get_core(self.h, i)

    def last_core(self) -> np.ndarray:
        return ttice_get_last_core(self.h)

    def load(self, ranks, cores, last) -> None:
        ttice_load(self.h, ranks, cores, last)

    def save(self, path: str) -> None:
        ttice_save(self.h, path)

    @classmethod
    def open(cls, path: str, *, max_batch: int = 32, max_rank: int = 512, obs_reserve: int = 1024) -> "TTICE":
        """A decomposition resumed from a checkpoint written by save() (its dims, eps, heuristics
        and state); capacities as in the constructor, each rank's at least its saved rank."""
        hdr = ttice_checkpoint_read_header(path)
        c = ttice_default_capacity()
        c.max_batch, c.max_rank, c.obs_reserve = int(max_batch), int(max_rank), int(obs_reserve)
        self = cls.__new__(cls)
        self.dims = hdr["dims"]
        self.d = len(self.dims)
        self.input_dtype = torch.float32 if hdr["heuristics"].input_dtype == TTICE_F32 else torch.float64
        self.h = ttice_open(path, c)
        return self

    def capacities(self) -> list[int]:
        return ttice_capacities(self.h, self.d)

    def device_bytes(self) -> int:
        return ttice_device_bytes(self.h)

    def capacity_miss(self) -> tuple[int, int]:
        """(k, need) after an update that failed with TTICE_ECAPACITY: rank r_k needed `need`."""
        return ttice_capacity_miss(self.h)

    def reserve_rank(self, k: int, cap: int) -> None:
        ttice_reserve_rank(self.h, k, cap)

    def profile(self, on: bool = True) -> None:
        ttice_profile_enable(self.h, on)

    def profile_read(self) -> dict:
        return ttice_profile_read(self.h)

    def close(self) -> None:
        if self.h:
            ttice_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
