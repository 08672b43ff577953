"""Python binding of libnvpit.so: Nievergelt parallel-in-time propagators on GB300.

Argument marshalling only.  Every step of the method runs in the CUDA kernels
behind the C ABI declared in include/nvpit.h; the functions here have the same
names without the ``nv_`` prefix.  Device buffers are torch CUDA tensors
(float64, contiguous); the stream defaults to torch's current stream.

The library must have been built (``paper_1304_6514_gb300._build.build()``);
importing a function that needs it raises if it is missing.  There is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, Structure, byref, c_char, c_double, c_int32, c_int64, c_void_p

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libnvpit.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "nvpit.h")

# enums (include/nvpit.h)
NV_OK, NV_EINVAL, NV_ENOMEM, NV_ECUDA, NV_EDOMAIN, NV_EBADMAP, NV_ETIMEOUT, NV_ENOTSUP = range(8)
RHS = {"linear_scalar": 0, "square": 1, "cos_cubic": 2, "heat1d": 3, "vdp": 4, "chain3": 5,
       "advdiff2d": 6, "heat1d_varcoef": 7, "wave": 8}
SCHEME = {"euler": 0, "rk4": 1, "leapfrog": 2}
MAP = {"pl1d": 0, "bilinear2d": 1, "affine": 2}
PREC = {"fp64": 0, "fp32": 1, "tf32_refine": 2, "bf16_refine": 3, "fp32_refine": 4}
OOB = {"extrapolate": 0, "error": 1}


class NvRhs(Structure):
    _fields_ = [("kind", c_int32), ("dim", c_int32), ("params", POINTER(c_double)),
                ("nparams", c_int32)]


class NvSamples(Structure):
    _fields_ = [("map", c_int32), ("per_dim", c_int32), ("lo", c_double * 2),
                ("hi", c_double * 2), ("oob_policy", c_int32)]


class NvSteps(Structure):
    _fields_ = [("scheme", c_int32), ("dt", c_double), ("steps_per_slice", c_int64),
                ("prec", c_int32)]


class NvMapsDesc(Structure):
    _fields_ = [("map", c_int32), ("prec", c_int32), ("scheme", c_int32), ("S", c_int32),
                ("dim", c_int32), ("per_dim", c_int32), ("steps_per_slice", c_int64),
                ("h", c_double), ("elems_per_slice", c_int64), ("bytes", c_int64),
                ("elem_bytes", c_int32), ("band", c_int32), ("work_per_slice", c_int64),
                ("build_kernel", c_char * 64)]


class NvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"nvpit status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnvpit.so and declare its prototypes.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1304_6514_gb300._build.build()"
                           " (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P = c_void_p
    sig = {
        "nv_build_propagators": [POINTER(NvRhs), c_double, c_double, c_int32, POINTER(NvSamples),
                                 POINTER(NvSteps), POINTER(c_void_p), P],
        "nv_compose": [P, P, P, P, P],
        "nv_solve": [POINTER(NvRhs), c_double, c_double, c_int32, POINTER(NvSamples),
                     POINTER(NvSteps), P, P, P],
        "nv_serial_fine": [POINTER(NvRhs), c_double, c_double, c_int32, POINTER(NvSteps), P, P, P],
        "nv_maps_destroy": [P],
        "nv_maps_info": [P, POINTER(NvMapsDesc)],
        "nv_maps_copy_out": [P, P, c_int64, P],
        "nv_maps_copy_range": [P, P, c_int64, c_int64, P],
        "nv_maps_check": [P, P, POINTER(c_int64)],
        "nv_tune_set": [c_int32, c_int32],
        "nv_compose_affine_noalloc": [P, c_int32, c_int32, c_int32, P, P, P, P, P],
        "nv_build_batch": [c_int32, c_int32, c_int32, P, c_int32, P, P, P, POINTER(NvSamples),
                           POINTER(NvSteps), POINTER(c_void_p), P],
        "nv_batch_rebuild": [P, P],
        "nv_batch_compose": [P, P, P, P],
        "nv_batch_run": [P, P, P, P],
        "nv_batch_autotune": [P, P, POINTER(c_int32)],
        "nv_batch_info": [P, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64), POINTER(c_int32)],
        "nv_batch_copy_out": [P, P, c_int64, P],
        "nv_batch_check": [P, P, POINTER(c_int64)],
        "nv_batch_destroy": [P],
        "nv_build_pairs": [POINTER(NvRhs), c_double, c_double, c_int32, POINTER(NvSteps), c_int64,
                           ctypes.c_uint64, c_double, c_double, P, P, P],
        "nv_propagate": [POINTER(NvRhs), c_double, c_double, c_int32, POINTER(NvSteps), c_int32, c_int32,
                         c_int64, P, P],
        "nv_mlp_create": [ctypes.c_uint64, POINTER(c_void_p)],
        "nv_mlp_destroy": [P],
        "nv_mlp_set_scales": [P, P, P],
        "nv_mlp_params": [P, P, POINTER(c_int64)],
        "nv_mlp_set_params": [P, P],
        "nv_mlp_grads": [P, P, P, c_int32, P, POINTER(c_double), P],
        "nv_mlp_train": [P, P, P, c_int32, c_int64, c_int64, c_int32, c_double, P, POINTER(c_double)],
        "nv_mlp_validate": [P, P, P, c_int32, c_int64, P, P],
        "nv_mlp_compose": [P, POINTER(NvRhs), c_double, c_double, c_int32, POINTER(NvSteps), P, c_int64, P, P, P],
        "nv_mlp_parareal": [P, POINTER(NvRhs), c_double, c_double, c_int32, POINTER(NvSteps), c_int32, c_int64,
                            P, P, P, P],
        "nv_plan_steps": [c_double, c_double, c_int32, c_double, c_int64, POINTER(c_int64),
                          POINTER(c_double)],
        "nv_alu_rate": [c_int32, POINTER(c_double), P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = c_int32
    lib.nv_last_error.argtypes = []
    lib.nv_last_error.restype = ctypes.c_char_p
    lib.nv_version.argtypes = []
    lib.nv_version.restype = c_int32
    _lib = lib
    return lib


def header_functions(path: str = HEADER_PATH) -> list[str]:
    """Names of the functions include/nvpit.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nv_[a-z_0-9]+)\s*\(", text)))


def last_error() -> str:
    return load_library().nv_last_error().decode()


def _check(status: int):
    if status != NV_OK:
        raise NvError(status, last_error())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("device buffers must be contiguous float64 CUDA tensors")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ------------------------------------------------------------------ descriptors

def rhs(kind: str, dim: int, params=()):
    arr = (c_double * max(1, len(params)))(*params)
    r = NvRhs(RHS[kind], dim, arr if params else None, len(params))
    r._keep = arr
    return r


def samples(map: str, per_dim: int = 0, lo=(0.0, 0.0), hi=(0.0, 0.0), oob: str = "extrapolate"):
    lo = tuple(lo) + (0.0,) * (2 - len(lo))
    hi = tuple(hi) + (0.0,) * (2 - len(hi))
    return NvSamples(MAP[map], per_dim, (c_double * 2)(*lo), (c_double * 2)(*hi), OOB[oob])


def steps(scheme: str, dt: float = 0.0, steps_per_slice: int = 0, prec: str = "fp64"):
    return NvSteps(SCHEME[scheme], dt, steps_per_slice, PREC[prec])


class Maps:
    """Library-owned slice maps (nv_maps); freed by destroy() or garbage collection."""

    def __init__(self, handle: int):
        self.handle = handle

    def info(self) -> NvMapsDesc:
        return maps_info(self)

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(load_library().nv_maps_destroy(h))

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.nv_maps_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


# ------------------------------------------------------------------ entry points

def build_propagators(rhs_, t0, T, S, samples_, steps_, maps: Maps | None = None, stream=None) -> Maps:
    """nv_build_propagators: the computation phase (Figure "pseudocode")."""
    lib = load_library()
    h = c_void_p(maps.handle if maps is not None else None)
    _check(lib.nv_build_propagators(byref(rhs_), t0, T, S, byref(samples_), byref(steps_),
                                    byref(h), _stream(stream)))
    if maps is not None:
        return maps
    return Maps(h.value)


def compose(maps: Maps, y0, yT, lambdas=None, stream=None):
    """nv_compose: the communication phase (Figure "pseudocode")."""
    _check(load_library().nv_compose(maps.handle, _ptr(y0), _ptr(yT), _ptr(lambdas), _stream(stream)))


def solve(rhs_, t0, T, S, samples_, steps_, y0, yT, stream=None):
    _check(load_library().nv_solve(byref(rhs_), t0, T, S, byref(samples_), byref(steps_), _ptr(y0),
                                   _ptr(yT), _stream(stream)))


def serial_fine(rhs_, t0, T, S, steps_, y0, yT, stream=None):
    _check(load_library().nv_serial_fine(byref(rhs_), t0, T, S, byref(steps_), _ptr(y0), _ptr(yT),
                                         _stream(stream)))


def compose_affine_noalloc(maps_dev, prec: str, dim: int, S: int, y0, yT, lambdas=None,
                           status=None, stream=None):
    """nv_compose_affine_noalloc: the affine chain over caller-owned maps, with
    its scratch in the library's fixed static device array (no allocation).
    maps_dev: CUDA tensor holding the maps in the AFFINE layout (float64 for
    prec "fp64", float32 for "fp32"); status: optional int32 CUDA tensor."""
    import torch
    want = torch.float64 if prec == "fp64" else torch.float32
    if not (maps_dev.is_cuda and maps_dev.dtype == want and maps_dev.is_contiguous()):
        raise ValueError("maps_dev must be a contiguous CUDA tensor of the maps' precision")
    if maps_dev.numel() < S * dim * (dim + 1):
        raise ValueError("maps_dev holds fewer than S * dim * (dim + 1) values")
    st = None
    if status is not None:
        if not (status.is_cuda and status.dtype == torch.int32):
            raise ValueError("status must be an int32 CUDA tensor")
        st = status.data_ptr()
    _check(load_library().nv_compose_affine_noalloc(maps_dev.data_ptr(), PREC[prec], dim, S, _ptr(y0),
                                                    _ptr(yT), _ptr(lambdas), st, _stream(stream)))


def maps_info(maps: Maps) -> NvMapsDesc:
    d = NvMapsDesc()
    _check(load_library().nv_maps_info(maps.handle, byref(d)))
    return d


def maps_copy_out(maps: Maps, dst, stream=None):
    """Copy the map data into a torch tensor (host or device) of at least info().bytes bytes."""
    nbytes = dst.numel() * dst.element_size()
    _check(load_library().nv_maps_copy_out(maps.handle, dst.data_ptr(), min(nbytes, maps_info(maps).bytes),
                                           _stream(stream)))


def maps_check(maps: Maps, stream=None) -> int:
    """Synchronise and raise NvError on a recorded device status; returns the out-of-range count."""
    n = c_int64(0)
    _check(load_library().nv_maps_check(maps.handle, _stream(stream), byref(n)))
    return n.value


def maps_data(maps: Maps):
    """The map data as a new CUDA tensor (float64, float32 or bfloat16, flat)."""
    import torch
    d = maps_info(maps)
    dt = {8: torch.float64, 4: torch.float32, 2: torch.bfloat16}[d.elem_bytes]
    out = torch.empty(d.bytes // d.elem_bytes, dtype=dt, device="cuda")
    _check(load_library().nv_maps_copy_out(maps.handle, out.data_ptr(), d.bytes, _stream(None)))
    return out


def maps_slice(maps: Maps, j: int, count: int = 1):
    """Map data of slices j .. j+count-1 as a new flat CUDA tensor."""
    import torch
    d = maps_info(maps)
    dt = {8: torch.float64, 4: torch.float32, 2: torch.bfloat16}[d.elem_bytes]
    out = torch.empty(d.elems_per_slice * count, dtype=dt, device="cuda")
    _check(load_library().nv_maps_copy_range(maps.handle, out.data_ptr(), j * d.elems_per_slice * d.elem_bytes,
                                             count * d.elems_per_slice * d.elem_bytes, _stream(None)))
    return out


def plan_steps(t0, T, S, dt=0.0, steps_per_slice=0):
    m, h = c_int64(0), c_double(0.0)
    _check(load_library().nv_plan_steps(t0, T, S, dt, steps_per_slice, byref(m), byref(h)))
    return m.value, h.value


def alu_rate(prec: str = "fp64", stream=None) -> float:
    """Measured FMA throughput of the device's float64 / float32 pipe (FLOP/s)."""
    out = c_double(0.0)
    _check(load_library().nv_alu_rate(PREC[prec], byref(out), _stream(stream)))
    return out.value


def tune_set(key: int, value: int):
    _check(load_library().nv_tune_set(key, value))


def version() -> int:
    return load_library().nv_version()


# ------------------------------------------------------------------ batched instances

class Batch:
    """Library-owned batch of independent instances (nv_batch)."""

    def __init__(self, handle: int):
        self.handle = handle

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(load_library().nv_batch_destroy(h))

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.nv_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def build_batch(kind: str, dim: int, params, t0, T, S, samples_, steps_, stream=None) -> Batch:
    """nv_build_batch: params (B, nparams), t0/T (B,), S (B,) host arrays."""
    import numpy as np
    params = np.ascontiguousarray(params, dtype=np.float64)
    if params.ndim == 1:
        params = params[:, None]
    t0 = np.ascontiguousarray(t0, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.int32)
    B = len(T)
    h = c_void_p()
    _check(load_library().nv_build_batch(RHS[kind], dim, B, params.ctypes.data, params.shape[1],
                                         t0.ctypes.data, T.ctypes.data, S.ctypes.data, byref(samples_),
                                         byref(steps_), byref(h), _stream(stream)))
    return Batch(h.value)


def batch_rebuild(batch: Batch, stream=None):
    _check(load_library().nv_batch_rebuild(batch.handle, _stream(stream)))


def batch_compose(batch: Batch, y0, yT, stream=None):
    _check(load_library().nv_batch_compose(batch.handle, _ptr(y0), _ptr(yT), _stream(stream)))


def batch_run(batch: Batch, y0, yT, stream=None):
    _check(load_library().nv_batch_run(batch.handle, _ptr(y0), _ptr(yT), _stream(stream)))


def batch_autotune(batch: Batch, stream=None) -> int:
    best = c_int32(0)
    _check(load_library().nv_batch_autotune(batch.handle, _stream(stream), byref(best)))
    return best.value


def batch_info(batch: Batch) -> dict:
    a, b, c, d = c_int64(0), c_int64(0), c_int64(0), c_int32(0)
    _check(load_library().nv_batch_info(batch.handle, byref(a), byref(b), byref(c), byref(d)))
    return {"total_slices": a.value, "traj_steps": b.value, "table_bytes": c.value, "threads": d.value}


def batch_tables(batch: Batch, dtype):
    """The tables of every instance as a new flat CUDA tensor of `dtype`."""
    import torch
    nbytes = batch_info(batch)["table_bytes"]
    out = torch.empty(nbytes // torch.empty((), dtype=dtype).element_size(), dtype=dtype, device="cuda")
    _check(load_library().nv_batch_copy_out(batch.handle, out.data_ptr(), nbytes, _stream(None)))
    return out


def batch_check(batch: Batch, stream=None) -> int:
    n = c_int64(0)
    _check(load_library().nv_batch_check(batch.handle, _stream(stream), byref(n)))
    return n.value


# ------------------------------------------------------------------ learned propagator

def _dptr(t):
    """Device pointer of any contiguous CUDA tensor (float32 / float64)."""
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def build_pairs(rhs_, t0, T, S, steps_, M, seed, lo, hi, y0, yend, stream=None):
    """nv_build_pairs into y0 / yend (S*M*6 float32 or float64 CUDA tensors)."""
    _check(load_library().nv_build_pairs(byref(rhs_), t0, T, S, byref(steps_), M, seed, lo, hi, _dptr(y0),
                                         _dptr(yend), _stream(stream)))


def propagate(rhs_, t0, T, S, steps_, j0, nslices, y, stream=None):
    """nv_propagate: float64 fine integration of the states y (count x 6, in place)."""
    _check(load_library().nv_propagate(byref(rhs_), t0, T, S, byref(steps_), j0, nslices, y.shape[0], _ptr(y),
                                       _stream(stream)))


class MLP:
    """The slice-conditioned MLP propagator (nv_mlp)."""

    def __init__(self, seed: int = 0):
        h = c_void_p()
        _check(load_library().nv_mlp_create(seed, byref(h)))
        self.handle = h.value

    def destroy(self):
        if self.handle:
            h, self.handle = self.handle, None
            _check(load_library().nv_mlp_destroy(h))

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.nv_mlp_destroy(self.handle)
                self.handle = None
        except Exception:
            pass

    def set_scales(self, sx, sd):
        a = (c_double * 6)(*sx)
        b = (c_double * 6)(*sd)
        _check(load_library().nv_mlp_set_scales(self.handle, a, b))

    def params(self):
        import numpy as np
        n = c_int64(0)
        _check(load_library().nv_mlp_params(self.handle, None, byref(n)))
        out = np.empty(n.value, dtype=np.float32)
        _check(load_library().nv_mlp_params(self.handle, out.ctypes.data, byref(n)))
        return out

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(load_library().nv_mlp_set_params(self.handle, p.ctypes.data))

    def grads(self, X, Y, stream=None):
        import torch
        n = c_int64(0)
        _check(load_library().nv_mlp_params(self.handle, None, byref(n)))
        g = torch.empty(n.value, dtype=torch.float32, device="cuda")
        loss = c_double(0.0)
        _check(load_library().nv_mlp_grads(self.handle, _dptr(X), _dptr(Y), X.shape[0], _dptr(g), byref(loss),
                                           _stream(stream)))
        return g, loss.value

    def train(self, y0, yend, S, M, steps, batch, lr, stream=None):
        loss = c_double(0.0)
        _check(load_library().nv_mlp_train(self.handle, _dptr(y0), _dptr(yend), S, M, steps, batch, lr,
                                           _stream(stream), byref(loss)))
        return loss.value

    def validate(self, y0, yend, S, Mv, stream=None):
        import numpy as np
        err = np.zeros(S, dtype=np.float64)
        _check(load_library().nv_mlp_validate(self.handle, _dptr(y0), _dptr(yend), S, Mv, err.ctypes.data,
                                              _stream(stream)))
        return err

    def compose(self, rhs_, t0, T, S, steps_, y0, yT, fallback=None, stream=None):
        import numpy as np
        fb = None
        if fallback is not None:
            fb = np.ascontiguousarray(fallback, dtype=np.int32)
        _check(load_library().nv_mlp_compose(self.handle, byref(rhs_), t0, T, S, byref(steps_),
                                             fb.ctypes.data if fb is not None else None, y0.shape[0], _ptr(y0),
                                             _ptr(yT), _stream(stream)))

    def parareal(self, rhs_, t0, T, S, steps_, iters, y0, yT, lambdas=None, stream=None):
        """nv_mlp_parareal: this network as the coarse map of a float64 residual
        correction (float64 defects of every slice, a correction chained over
        the network's Jacobians), `iters` iterations."""
        _check(load_library().nv_mlp_parareal(self.handle, byref(rhs_), t0, T, S, byref(steps_), iters,
                                              y0.shape[0], _ptr(y0), _ptr(yT),
                                              _ptr(lambdas) if lambdas is not None else None, _stream(stream)))
