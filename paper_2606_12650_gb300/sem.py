"""Thin Python binding of libsem (argument marshalling only).

The functions carry the names of the C-ABI in ``include/sem.h``:
``init``, ``update``, ``run``, ``sync``, ``finalize``, ``last_error``,
``set_allocator``, ``set_stream``, ``launch_count``.  Every step of the
computation runs in libsem's CUDA kernels; this module converts Python values
to ``sem_arg`` records:

* ``int`` -> SEM_ARG_INT, ``float`` -> SEM_ARG_DOUBLE, ``None`` -> SEM_ARG_NONE
* a CUDA ``torch.Tensor`` -> SEM_ARG_DEVICE (its data pointer)
* a numpy array or CPU tensor -> SEM_ARG_MAPPED (its host address, which must
  lie inside a mirror created with ``update``)
* ``OutInt()`` / ``OutDouble()`` -> SEM_ARG_OUT_INT / SEM_ARG_OUT_DOUBLE

PyTorch provides device memory (libsem's allocator hooks are pointed at the
caching allocator by ``init``) and the stream.  There is no fallback: if
``libsem.so`` is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsem.so")

# status codes and constants (mirrors include/sem.h)
SEM_OK = 0
SEM_EINIT = -1
SEM_EARG = -2
SEM_ENOMAP = -3
SEM_ERANGE = -4
SEM_ENOMEM = -5
SEM_EKERNEL = -6
SEM_ETIMEDOUT = -7
SEM_ECUDA = -8
SEM_EMESH = -9
SEM_EHANDLE = -10

SEM_ALLOC, SEM_TO, SEM_FROM, SEM_FREE = 0, 1, 2, 3

ARG_INT, ARG_DOUBLE, ARG_MAPPED, ARG_DEVICE, ARG_OUT_DOUBLE, ARG_OUT_INT, ARG_NONE, ARG_HOST = range(8)

EXPORTS = ("sem_init", "sem_update", "sem_run", "sem_sync", "sem_finalize", "sem_last_error",
           "sem_set_allocator", "sem_set_stream", "sem_launch_count", "sem_dot_noalloc")


class SemError(RuntimeError):
    """A libsem call returned a negative status."""

    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where} failed with status {code}: {message}")
        self.code = code
        self.message = message


class _V(ctypes.Union):
    _fields_ = [("i", ctypes.c_int64), ("d", ctypes.c_double), ("ptr", ctypes.c_void_p)]


class SemArg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("v", _V)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None
_keep = {}          # ctypes callbacks and the torch stream must outlive their use


def _open(path: str):
    if not os.path.exists(path):
        raise RuntimeError(f"libsem.so not found at {path}: build it with "
                           "paper_2606_12650_gb300.build.build() (nvcc, sm_103a)")
    return ctypes.CDLL(path)


def load(path: str | None = None):
    """Load libsem.so (no GPU needed).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = _open(path or LIB_PATH)
        lib.sem_init.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p)]
        lib.sem_update.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_size_t,
                                   ctypes.c_size_t, ctypes.c_int]
        lib.sem_run.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(SemArg)]
        lib.sem_sync.argtypes = []
        lib.sem_finalize.argtypes = []
        lib.sem_last_error.argtypes = []
        lib.sem_last_error.restype = ctypes.c_char_p
        lib.sem_set_allocator.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.sem_set_stream.argtypes = [ctypes.c_void_p]
        lib.sem_launch_count.argtypes = []
        lib.sem_launch_count.restype = ctypes.c_int64
        lib.sem_dot_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        lib.sem_dot_noalloc.restype = ctypes.c_int
        for name in ("sem_init", "sem_update", "sem_run", "sem_sync", "sem_finalize",
                     "sem_set_allocator", "sem_set_stream"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def last_error() -> str:
    return load().sem_last_error().decode(errors="replace")


def _check(rc: int, where: str) -> int:
    if rc != SEM_OK:
        raise SemError(rc, where, last_error())
    return rc


class OutInt:
    """Receives an int64 result of ``run``."""

    def __init__(self):
        self._c = ctypes.c_int64(0)

    @property
    def value(self) -> int:
        return int(self._c.value)


class OutDouble:
    """Receives a double result of ``run``."""

    def __init__(self):
        self._c = ctypes.c_double(0.0)

    @property
    def value(self) -> float:
        return float(self._c.value)


class DevicePtr(int):
    """A raw device address (SEM_ARG_DEVICE)."""


class HostPtr(int):
    """The address of a host object (a ctypes structure) passed for the
    duration of the call (SEM_ARG_HOST)."""


class HostArray:
    """A small host numpy array passed by address for the duration of the
    call (SEM_ARG_HOST): read and/or written by libsem."""

    def __init__(self, arr):
        if not arr.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        self.arr = arr


def _is_torch_tensor(a) -> bool:
    t = type(a)
    return t.__module__.startswith("torch") and t.__name__ in ("Tensor", "Parameter")


def _marshal(a) -> SemArg:
    arg = SemArg()
    if a is None:
        arg.kind = ARG_NONE
    elif isinstance(a, OutInt):
        arg.kind = ARG_OUT_INT
        arg.v.ptr = ctypes.cast(ctypes.pointer(a._c), ctypes.c_void_p).value
    elif isinstance(a, OutDouble):
        arg.kind = ARG_OUT_DOUBLE
        arg.v.ptr = ctypes.cast(ctypes.pointer(a._c), ctypes.c_void_p).value
    elif isinstance(a, HostArray):
        arg.kind = ARG_HOST
        arg.v.ptr = a.arr.__array_interface__["data"][0]
    elif isinstance(a, HostPtr):
        arg.kind = ARG_HOST
        arg.v.ptr = int(a)
    elif isinstance(a, DevicePtr):
        arg.kind = ARG_DEVICE
        arg.v.ptr = int(a)
    elif isinstance(a, bool):
        raise TypeError("bool is not a libsem argument")
    elif isinstance(a, int):
        arg.kind = ARG_INT
        arg.v.i = a
    elif isinstance(a, float):
        arg.kind = ARG_DOUBLE
        arg.v.d = a
    elif _is_torch_tensor(a):
        if not a.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        arg.kind = ARG_DEVICE if a.is_cuda else ARG_MAPPED
        arg.v.ptr = a.data_ptr()
    elif hasattr(a, "__array_interface__"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arguments must be C-contiguous")
        arg.kind = ARG_MAPPED
        arg.v.ptr = a.__array_interface__["data"][0]
    else:
        raise TypeError(f"cannot pass {type(a).__name__} to libsem")
    return arg


def _host_ptr_and_size(arr):
    if _is_torch_tensor(arr):
        if arr.is_cuda:
            raise ValueError("update() maps host arrays; pass a CPU tensor or numpy array")
        return arr.data_ptr(), arr.numel(), arr.element_size()
    if not arr.flags["C_CONTIGUOUS"]:
        raise ValueError("update() needs a C-contiguous array")
    return arr.__array_interface__["data"][0], arr.size, arr.itemsize


# ---------------------------------------------------------------- the C-ABI calls
def init(argv=(), use_torch_allocator: bool = True, torch_stream=None) -> None:
    """sem_init(argv); then route device allocations through PyTorch's caching
    allocator and run on ``torch_stream`` (a new torch.cuda.Stream if None)."""
    lib = load()
    if _keep.get("initialised"):
        raise SemError(SEM_EINIT, "sem_init", "already initialised")
    args = [a.encode() for a in argv]
    arr = (ctypes.c_char_p * max(len(args), 1))(*args)
    if not use_torch_allocator:
        _check(lib.sem_init(len(args), arr), "sem_init")
        _keep["initialised"] = True
        return
    import torch
    dev = 0
    for a in argv:
        if a.startswith("--device="):
            dev = int(a.split("=", 1)[1])
    stream = torch_stream or torch.cuda.Stream(device=dev)

    def _alloc(nbytes, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream))
        except Exception:  # libsem reports the failure as SEM_ENOMEM
            return 0

    def _free(ptr, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    alloc_cb, free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
    _check(lib.sem_set_allocator(ctypes.cast(alloc_cb, ctypes.c_void_p),
                                 ctypes.cast(free_cb, ctypes.c_void_p), None), "sem_set_allocator")
    _keep.update(alloc=alloc_cb, free=free_cb, stream=stream)
    _check(lib.sem_init(len(args), arr), "sem_init")
    _keep["initialised"] = True
    _check(lib.sem_set_stream(ctypes.c_void_p(stream.cuda_stream)), "sem_set_stream")


def update(arr, op: int, start: int = 0, end: int | None = None) -> None:
    """sem_update on a host array (numpy or CPU tensor), elements [start, end)."""
    ptr, n, es = _host_ptr_and_size(arr)
    _check(load().sem_update(ctypes.c_void_p(ptr), start, n if end is None else end, es, op),
           "sem_update")


def run(kernel: str, *args) -> None:
    """sem_run(kernel, args); OUT arguments are filled in place."""
    recs = (SemArg * max(len(args), 1))(*[_marshal(a) for a in args])
    _check(load().sem_run(kernel.encode(), len(args), recs), f"sem_run('{kernel}')")


def sync() -> None:
    _check(load().sem_sync(), "sem_sync")


def finalize() -> None:
    lib = load()
    _check(lib.sem_finalize(), "sem_finalize")
    _check(lib.sem_set_allocator(None, None, None), "sem_set_allocator")
    _keep.clear()


def set_stream(stream_handle: int | None) -> None:
    _check(load().sem_set_stream(ctypes.c_void_p(stream_handle)), "sem_set_stream")


def launch_count() -> int:
    return int(load().sem_launch_count())


def dot_noalloc(c, u, v, n: int, out, stream_handle: int | None = None) -> None:
    """sem_dot_noalloc: out[0] = sum c*u*v over n entries, with no device
    allocation (c may be None).  Arguments are CUDA tensors; the call does not
    synchronise ``stream_handle`` (a cudaStream_t, None = default stream)."""
    ptr = lambda t: None if t is None else t.data_ptr()
    _check(load().sem_dot_noalloc(ptr(c), ptr(u), ptr(v), int(n), ptr(out),
                                  None if stream_handle is None else ctypes.c_void_p(stream_handle)),
           "sem_dot_noalloc")


def stream():
    """The torch.cuda.Stream libsem runs on (when ``init`` created one)."""
    return _keep.get("stream")


# ---------------------------------------------------------------- operator tuner
TUNE_F64, TUNE_F32_G32, TUNE_F32_G16 = 0, 1, 2           # what is tuned
VARIANT_COLUMNS, VARIANT_LINES, VARIANT_PERSISTENT, VARIANT_LINES_PREFETCH, VARIANT_LINES_STAGED = 0, 1, 2, 3, 4
VARIANT_NAMES = {VARIANT_COLUMNS: "columns", VARIANT_LINES: "lines", VARIANT_PERSISTENT: "persistent",
                 VARIANT_LINES_PREFETCH: "lines_prefetch", VARIANT_LINES_STAGED: "lines_staged"}


def autotune(handle: int, kind: int, reps: int = 10):
    """Time every operator variant of `kind` on problem `handle` (its order)
    and keep the fastest.  Returns [(variant, elements_per_block, us), ...]."""
    import numpy as np
    cand = np.zeros(3 * 32, dtype=np.float64)
    n = OutInt()
    run("autotune", int(handle), int(kind), int(reps), HostArray(cand), 32, n)
    return [(int(cand[3 * c]), int(cand[3 * c + 1]), float(cand[3 * c + 2])) for c in range(n.value)]


def autotune_get(kind: int, N: int):
    """The variant in use for (kind, N): (variant, elements_per_block, us)."""
    v, e, u = OutInt(), OutInt(), OutDouble()
    run("autotune_get", int(kind), int(N), v, e, u)
    return v.value, e.value, u.value


def autotune_set(kind: int, N: int, variant: int, epb: int = 0) -> None:
    run("autotune_set", int(kind), int(N), int(variant), int(epb))


def _path_arg(path: str):
    import numpy as np
    b = np.frombuffer(str(path).encode() + b"\0", dtype=np.uint8).copy()
    return HostArray(b)


def autotune_save(path: str) -> None:
    run("autotune_save", _path_arg(path))


def autotune_load(path: str) -> None:
    run("autotune_load", _path_arg(path))
