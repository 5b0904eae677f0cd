"""Python binding of libtpf (ctypes; argument marshalling only).

Every step of a solve runs in libtpf's CUDA kernels; this module only checks shapes and dtypes,
passes device pointers and the current CUDA stream, and turns status codes into exceptions.
PyTorch is used for device memory and streams.  There is no CPU fallback: if libtpf.so cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ESINGULAR, ENOMEM, ECUDA, ETIMEOUT, ENOCONV, EUNSUPPORTED = range(8)
PREC_FP64, PREC_MIXED = 0, 1
METHOD_DENSE, METHOD_SPARSE = 0, 1
START_FLAT, START_GIVEN, START_WARM = 0, 1, 2

# Every entry point declared in include/tpf.h.
EXPORTS = (
    "tpf_default_opts", "tpf_strerror", "tpf_create", "tpf_create_poly", "tpf_destroy", "tpf_n_pq", "tpf_precompute_host",
    "tpf_solve", "tpf_solve_host", "tpf_solve_ex", "tpf_solve_batch", "tpf_batch_create", "tpf_batch_launch",
    "tpf_batch_wait", "tpf_batch_destroy", "tpf_set_zip", "tpf_autotune", "tpf_last_stats", "tpf_selftest_gemm",
    "tpf_selftest_gemm_wait", "tpf_solve_fp64_noalloc",
    "tpf_mlp_create", "tpf_mlp_destroy", "tpf_mlp_param_count", "tpf_mlp_get_params", "tpf_mlp_set_params",
    "tpf_mlp_fit_normalization", "tpf_mlp_get_normalization", "tpf_mlp_train_step", "tpf_mlp_gradients",
    "tpf_mlp_predict", "tpf_solve_learned", "tpf_solve_learned_host",
)

# Size of the built-in scratch array of tpf_solve_fp64_noalloc (include/tpf.h).
NOALLOC_SCRATCH_BYTES = 64 << 20


class TpfError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {strerror(status)}")


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("start", ctypes.c_int), ("switch_tol", ctypes.c_double), ("profile", ctypes.c_int),
                ("method", ctypes.c_int)]


class Outputs(ctypes.Structure):
    _fields_ = [("s_complex64", ctypes.c_int), ("v_complex64", ctypes.c_int), ("v_min", ctypes.c_double),
                ("v_max", ctypes.c_double), ("col_vmin", ctypes.c_void_p), ("col_vmax", ctypes.c_void_p),
                ("col_viol", ctypes.c_void_p), ("bus_under", ctypes.c_void_p), ("bus_over", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("precise_sweeps", ctypes.c_int), ("converged", ctypes.c_int64),
                ("columns", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("gemm_ms", ctypes.c_double),
                ("residual_ms", ctypes.c_double), ("other_ms", ctypes.c_double), ("gemm_launches", ctypes.c_int64),
                ("gemm_columns", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = False):
    """Load libtpf.so (optionally building it first).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libtpf.so not built ({path}); run __graft_entry__.build() or "
                               "python -m paper_2403_04578_gb300.build")
        _build.build()
    L = ctypes.CDLL(path)
    vp, i32p, f64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)
    L.tpf_default_opts.argtypes = [ctypes.POINTER(Opts)]
    L.tpf_default_opts.restype = None
    L.tpf_strerror.argtypes = [ctypes.c_int]
    L.tpf_strerror.restype = ctypes.c_char_p
    L.tpf_create.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, f64p, ctypes.c_int, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int, i32p, ctypes.POINTER(vp)]
    L.tpf_create.restype = ctypes.c_int
    L.tpf_destroy.argtypes = [vp]
    L.tpf_destroy.restype = None
    L.tpf_n_pq.argtypes = [vp]
    L.tpf_n_pq.restype = ctypes.c_int
    L.tpf_precompute_host.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, f64p, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, i32p, f64p, f64p]
    L.tpf_precompute_host.restype = ctypes.c_int
    L.tpf_solve.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.POINTER(Opts), vp]
    L.tpf_solve.restype = ctypes.c_int
    L.tpf_solve_host.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.POINTER(Opts), vp]
    L.tpf_solve_host.restype = ctypes.c_int
    L.tpf_create_poly.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p, f64p, ctypes.c_int, f64p,
                                  ctypes.c_int, i32p, ctypes.POINTER(vp)]
    L.tpf_create_poly.restype = ctypes.c_int
    L.tpf_autotune.argtypes = [vp, ctypes.c_int64, vp, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_int), vp]
    L.tpf_autotune.restype = ctypes.c_int
    L.tpf_set_zip.argtypes = [vp, vp]
    L.tpf_set_zip.restype = ctypes.c_int
    L.tpf_solve_ex.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.POINTER(Outputs), ctypes.POINTER(Opts), vp]
    L.tpf_solve_ex.restype = ctypes.c_int
    L.tpf_solve_batch.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Opts), vp,
                                  ctypes.POINTER(Stats), vp]
    L.tpf_solve_batch.restype = ctypes.c_int
    L.tpf_batch_create.argtypes = [ctypes.c_int, vp, vp, vp, vp, vp, vp, ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    L.tpf_batch_create.restype = ctypes.c_int
    L.tpf_batch_launch.argtypes = [vp, vp]
    L.tpf_batch_launch.restype = ctypes.c_int
    L.tpf_batch_wait.argtypes = [vp, vp, ctypes.POINTER(Stats)]
    L.tpf_batch_wait.restype = ctypes.c_int
    L.tpf_batch_destroy.argtypes = [vp]
    L.tpf_batch_destroy.restype = None
    L.tpf_last_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.tpf_last_stats.restype = ctypes.c_int
    L.tpf_selftest_gemm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
    L.tpf_selftest_gemm.restype = ctypes.c_int
    L.tpf_selftest_gemm_wait.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp,
                                         ctypes.c_double, ctypes.c_int, vp]
    L.tpf_selftest_gemm_wait.restype = ctypes.c_int
    L.tpf_solve_fp64_noalloc.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int64, vp, vp, vp, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, vp]
    L.tpf_solve_fp64_noalloc.restype = ctypes.c_int
    f32p = ctypes.POINTER(ctypes.c_float)
    L.tpf_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                 ctypes.POINTER(vp)]
    L.tpf_mlp_destroy.argtypes = [vp]
    L.tpf_mlp_destroy.restype = None
    L.tpf_mlp_param_count.argtypes = [vp]
    L.tpf_mlp_param_count.restype = ctypes.c_int64
    L.tpf_mlp_get_params.argtypes = [vp, f32p]
    L.tpf_mlp_set_params.argtypes = [vp, f32p]
    L.tpf_mlp_fit_normalization.argtypes = [vp, ctypes.c_int64, vp, vp, vp]
    L.tpf_mlp_get_normalization.argtypes = [vp, f32p, f32p, f32p, f32p]
    L.tpf_mlp_train_step.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double), vp]
    L.tpf_mlp_gradients.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_double), f32p, vp]
    L.tpf_mlp_predict.argtypes = [vp, ctypes.c_int64, vp, vp, ctypes.POINTER(ctypes.c_int64), vp]
    L.tpf_solve_learned.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.POINTER(Opts),
                                    ctypes.POINTER(ctypes.c_int64), vp]
    L.tpf_solve_learned.restype = ctypes.c_int
    L.tpf_solve_learned_host.argtypes = L.tpf_solve_learned.argtypes
    L.tpf_solve_learned_host.restype = ctypes.c_int
    for name in ("tpf_mlp_create", "tpf_mlp_get_params", "tpf_mlp_set_params", "tpf_mlp_fit_normalization",
                 "tpf_mlp_get_normalization", "tpf_mlp_train_step", "tpf_mlp_gradients", "tpf_mlp_predict"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def strerror(status: int) -> str:
    try:
        return lib().tpf_strerror(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _z(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_opts(precision: str | int = "mixed", tol: float = 1e-10, max_iter: int = 100, start: str | int = "flat",
              switch_tol: float = 1e-4, profile: bool = False, method: str | int = "dense") -> Opts:
    o = Opts()
    lib().tpf_default_opts(ctypes.byref(o))
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.precision = {"fp64": PREC_FP64, "mixed": PREC_MIXED}.get(precision, precision)
    o.start = {"flat": START_FLAT, "given": START_GIVEN, "warm": START_WARM}.get(start, start)
    o.switch_tol = float(switch_tol)
    o.profile = 1 if profile else 0
    o.method = {"dense": METHOD_DENSE, "sparse": METHOD_SPARSE}.get(method, method)
    return o


def precompute_host(n_bus, from_bus, to_bus, z_pu, slack=0, v0=1.0 + 0j, pq_bus=None):
    """K = -Y_dd^{-1} and W = K Y_ds v_s as computed by tpf_create (host only, no device)."""
    if pq_bus is None:
        pq_bus = [b for b in range(n_bus) if b != slack]
    fa, fp = _i32(from_bus)
    ta, tp = _i32(to_bus)
    za, zp = _z(z_pu)
    pa, pp = _i32(pq_bus)
    n = len(pa)
    K = np.zeros((n, n), dtype=np.complex128)
    W = np.zeros(n, dtype=np.complex128)
    st = lib().tpf_precompute_host(int(n_bus), len(fa), fp, tp, zp, int(slack), float(np.real(v0)), float(np.imag(v0)),
                                   n, pp, K.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   W.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != OK:
        raise TpfError(st, "tpf_precompute_host")
    return K, W


def _host_buffer(a, name, dtype, shape):
    """Check a host buffer handed to tpf_solve_host: a C-contiguous numpy array or CPU torch tensor
    of the given dtype and shape (the library reads and writes exactly that many bytes)."""
    if hasattr(a, "is_cuda"):
        import torch

        tdt = {np.complex128: torch.complex128, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        ok = not a.is_cuda and a.dtype == tdt and a.is_contiguous() and tuple(a.shape) == shape
    else:
        ok = isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous and a.shape == shape
    if not ok:
        raise ValueError(f"{name} must be a C-contiguous host {np.dtype(dtype).name} array of shape {shape}")


def _device_tensors(specs):
    """specs: (name, tensor, torch dtype, shape) each.  Every tensor must have its dtype and shape
    (the kernels read and write exactly that many elements through its pointer), then be
    contiguous and on the device; dtypes and shapes are checked first."""
    import torch

    for name, X, dtype, shape in specs:
        if not isinstance(X, torch.Tensor) or X.dtype != dtype or tuple(X.shape) != tuple(shape):
            raise ValueError(f"{name} must be a {dtype} tensor of shape {tuple(shape)}")
    for name, X, _, _ in specs:
        if not X.is_contiguous() or not X.is_cuda:
            raise ValueError(f"{name} must be a contiguous CUDA tensor")


def _batch_outputs(S, V, iters, mismatch):
    """Caller-supplied batch outputs, per feeder f: V[f] complex128 shaped like S[f], iters[f] int32
    and mismatch[f] float64 of length T_f, all contiguous on the device (the batch kernels write
    through these pointers).  One pass of plain comparisons (a few microseconds per feeder); the
    precise message, dtypes and shapes of all feeders before placement, only on failure."""
    import torch

    if not (len(V) == len(iters) == len(mismatch) == len(S)):
        raise ValueError("one V, iters and mismatch tensor per feeder")
    c128, i32, f64, Tn = torch.complex128, torch.int32, torch.float64, torch.Tensor
    for s, v, i, m in zip(S, V, iters, mismatch):
        n = (s.shape[0],)
        if not (isinstance(v, Tn) and isinstance(i, Tn) and isinstance(m, Tn)
                and v.dtype == c128 and i.dtype == i32 and m.dtype == f64
                and v.shape == s.shape and i.shape == n and m.shape == n
                and v.is_cuda and i.is_cuda and m.is_cuda
                and v.is_contiguous() and i.is_contiguous() and m.is_contiguous()):
            break
    else:
        return
    specs = []
    for f, s in enumerate(S):
        n = (s.shape[0],)
        specs += [(f"V[{f}]", V[f], c128, s.shape), (f"iters[{f}]", iters[f], i32, n),
                  (f"mismatch[{f}]", mismatch[f], f64, n)]
    _device_tensors(specs)


def _one_device(named, want=None):
    """The index of the one CUDA device that holds every tensor in `named` ((name, tensor) pairs;
    None entries are skipped) and, when given, equals `want` (the device of the Feeder or network the
    call runs on).  The library passes raw pointers to kernels launched on that device, so a tensor on
    another GPU is refused here rather than read through a foreign pointer."""
    dev, first = want, None
    for name, X in named:
        if X is None:
            continue
        idx = X.device.index
        if dev is None:
            dev, first = idx, name
        elif idx != dev:
            where = f"the device of {first}" if first else "the device this object was created on"
            raise ValueError(f"{name} is on cuda:{idx}, but {where} is cuda:{dev}: "
                             "every tensor of a call must be on one device")
        if first is None:
            first = name
    return dev


def _stream_ptr(stream, device=None):
    """The cudaStream_t to pass: `stream`, or the current torch stream of `device`.  A given stream
    must belong to `device`."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream(device)
    elif device is not None and stream.device.index != device:
        raise ValueError(f"the stream belongs to cuda:{stream.device.index}, the tensors to cuda:{device}")
    return ctypes.c_void_p(stream.cuda_stream)


def _on_device(device):
    """Context in which torch's current device (and the CUDA runtime's) is `device`."""
    import torch

    return torch.cuda.device(device)


def _current_device():
    import torch

    return torch.cuda.current_device()


class Feeder:
    """A feeder uploaded to the GPU (a tpf_handle) of the current device; every later call takes
    tensors on that device and runs there."""

    def __init__(self, n_bus, from_bus, to_bus, z_pu, slack=0, v0=1.0 + 0j, pq_bus=None):
        if pq_bus is None:
            pq_bus = [b for b in range(n_bus) if b != slack]
        fa, fp = _i32(from_bus)
        ta, tp = _i32(to_bus)
        za, zp = _z(z_pu)
        pa, pp = _i32(pq_bus)
        h = ctypes.c_void_p()
        st = lib().tpf_create(int(n_bus), len(fa), fp, tp, zp, int(slack), float(np.real(v0)), float(np.imag(v0)),
                              len(pa), pp, ctypes.byref(h))
        if st != OK:
            raise TpfError(st, "tpf_create")
        self._h = h
        self.n_pq = lib().tpf_n_pq(h)
        self.device = _current_device()  # tpf_create builds the feeder on the current device

    @classmethod
    def poly(cls, n_bus, from_bus, to_bus, z_blocks, phases=3, slack=0, v0=None, pq_bus=None):
        """A polyphase feeder: z_blocks [n_branch][phases][phases] complex; v0 [phases]."""
        if pq_bus is None:
            pq_bus = [b for b in range(n_bus) if b != slack]
        if v0 is None:
            v0 = np.exp(-2j * np.pi * np.arange(phases) / phases)
        fa, fp = _i32(from_bus)
        ta, tp = _i32(to_bus)
        z = np.ascontiguousarray(np.asarray(z_blocks, np.complex128).reshape(len(fa), phases, phases))
        zr = z.view(np.float64).reshape(-1)
        v = np.ascontiguousarray(np.asarray(v0, np.complex128)).view(np.float64)
        pa, pp = _i32(pq_bus)
        h = ctypes.c_void_p()
        st = lib().tpf_create_poly(int(n_bus), len(fa), int(phases), fp, tp,
                                   zr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(slack),
                                   v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(pa), pp, ctypes.byref(h))
        if st != OK:
            raise TpfError(st, "tpf_create_poly")
        obj = cls.__new__(cls)
        obj._h = h
        obj.n_pq = lib().tpf_n_pq(h)
        obj.device = _current_device()
        obj._keep = (fa, ta, z, v, pa)
        return obj

    @classmethod
    def from_inputs(cls, f):
        """From a ``paper_2403_04578_gb300.inputs.Feeder``."""
        return cls(f.n_bus, f.from_bus, f.to_bus, f.z_pu, f.slack, f.v0, f.pq_bus)

    def close(self):
        if getattr(self, "_h", None):
            lib().tpf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def autotune(self, S, tol=1e-10, max_iter=100, switch_tol=1e-4, stream=None) -> int:
        """tpf_autotune on the CUDA complex128 sample S [T, n_pq]; returns the chosen buses per thread."""
        import torch

        shape = tuple(getattr(S, "shape", ()))
        _device_tensors([("S", S, torch.complex128, (shape[0] if len(shape) == 2 else -1, self.n_pq))])
        dev = _one_device([("S", S)], getattr(self, "device", None))
        o = make_opts("mixed", tol, max_iter, "flat", switch_tol, False, "sparse")
        b = ctypes.c_int(0)
        with _on_device(dev):
            st = lib().tpf_autotune(self._h, S.shape[0], ctypes.c_void_p(S.data_ptr()), ctypes.byref(o),
                                    ctypes.byref(b), _stream_ptr(stream, dev))
        if st != OK:
            raise TpfError(st, "tpf_autotune")
        return b.value

    def set_zip(self, alpha=None):
        """ZIP load coefficients (Eq. 3): alpha = [alpha_P, alpha_I, alpha_Z], each [n_pq] (or None)."""
        if alpha is None:
            st = lib().tpf_set_zip(self._h, None)
        else:
            a = np.ascontiguousarray(alpha, dtype=np.float64).reshape(3, self.n_pq)
            st = lib().tpf_set_zip(self._h, ctypes.c_void_p(a.ctypes.data))
        if st != OK:
            raise TpfError(st, "tpf_set_zip")

    def stats(self) -> dict:
        s = Stats()
        lib().tpf_last_stats(self._h, ctypes.byref(s))
        return s.as_dict()

    def solve(self, S, V=None, iters=None, mismatch=None, precision="mixed", tol=1e-10, max_iter=100, start=None,
              switch_tol=1e-4, stream=None, check=True, profile=False, method="dense"):
        """Solve every column of the device tensor S (complex128 [T][n_pq]).

        Returns (V, iters, mismatch, status); outputs are allocated when not given.  With
        ``start='given'`` (default when V is passed) V is read as the starting point and anchored at
        once; ``start='warm'`` reads it as an approximate start (FP32 sweeps first).
        """
        import torch

        if not (isinstance(S, torch.Tensor) and S.is_cuda and S.dtype == torch.complex128 and S.dim() == 2):
            raise TypeError("S must be a CUDA complex128 tensor [T, n_pq]")
        if S.shape[1] != self.n_pq or not S.is_contiguous():
            raise ValueError(f"S must be contiguous with {self.n_pq} columns")
        T = S.shape[0]
        if start is None:
            start = "given" if V is not None else "flat"
        if V is None:
            V = torch.empty_like(S)
        if iters is None:
            iters = torch.empty(T, dtype=torch.int32, device=S.device)
        if mismatch is None:
            mismatch = torch.empty(T, dtype=torch.float64, device=S.device)
        for t_, dt, shape in ((V, torch.complex128, S.shape), (iters, torch.int32, (T,)),
                              (mismatch, torch.float64, (T,))):
            if not (t_.is_cuda and t_.dtype == dt and t_.is_contiguous() and t_.shape == shape):
                raise ValueError("V must be shaped like S, iters and mismatch [T]: contiguous CUDA tensors "
                                 "(complex128, int32, float64)")
        dev = _one_device([("S", S), ("V", V), ("iters", iters), ("mismatch", mismatch)],
                          getattr(self, "device", None))
        o = make_opts(precision, tol, max_iter, start, switch_tol, profile, method)
        with _on_device(dev):
            st = lib().tpf_solve(self._h, T, ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(V.data_ptr()),
                                 ctypes.c_void_p(iters.data_ptr()), ctypes.c_void_p(mismatch.data_ptr()),
                                 ctypes.byref(o), _stream_ptr(stream, dev))
        if check and st not in (OK, ENOCONV):
            raise TpfError(st, "tpf_solve")
        return V, iters, mismatch, st

    def solve_learned(self, net, S, V=None, iters=None, mismatch=None, tol=1e-10, max_iter=100, switch_tol=1e-4,
                      stream=None, check=True, profile=False):
        """tpf_solve_learned: V_0 from the LearnedStart network ``net`` (fused inference), then the
        sparse mixed solve from it.  Returns (V, iters, mismatch, fallback columns, status)."""
        import torch

        if not (isinstance(S, torch.Tensor) and S.is_cuda and S.dtype == torch.complex128 and S.dim() == 2):
            raise TypeError("S must be a CUDA complex128 tensor [T, n_pq]")
        if S.shape[1] != self.n_pq or not S.is_contiguous():
            raise ValueError(f"S must be contiguous with {self.n_pq} columns")
        if net.n_pq != self.n_pq:
            raise ValueError(f"the network is for {net.n_pq} demand buses, the feeder has {self.n_pq}")
        T = S.shape[0]
        V = torch.empty_like(S) if V is None else V
        iters = torch.empty(T, dtype=torch.int32, device=S.device) if iters is None else iters
        mismatch = torch.empty(T, dtype=torch.float64, device=S.device) if mismatch is None else mismatch
        _device_tensors([("V", V, torch.complex128, S.shape), ("iters", iters, torch.int32, (T,)),
                         ("mismatch", mismatch, torch.float64, (T,))])
        dev = _one_device([("S", S), ("V", V), ("iters", iters), ("mismatch", mismatch)],
                          getattr(self, "device", None))
        _one_device([("S", S)], getattr(net, "device", None))
        o = make_opts("mixed", tol, max_iter, "warm", switch_tol, profile, "sparse")
        fb = ctypes.c_int64(0)
        with _on_device(dev):
            st = lib().tpf_solve_learned(self._h, net._h, T, ctypes.c_void_p(S.data_ptr()),
                                         ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(iters.data_ptr()),
                                         ctypes.c_void_p(mismatch.data_ptr()), ctypes.byref(o), ctypes.byref(fb),
                                         _stream_ptr(stream, dev))
        if check and st not in (OK, ENOCONV):
            raise TpfError(st, "tpf_solve_learned")
        return V, iters, mismatch, fb.value, st

    def solve_learned_host(self, net, S, tol=1e-10, max_iter=100, switch_tol=1e-4, stream=None, out=None,
                           check=True, profile=False):
        """tpf_solve_learned_host on host arrays (numpy or pinned torch CPU tensors, complex128
        [T][n_pq]): the learned-start solve with the host-to-device copies, the solve and the copies
        back pipelined inside the library.  Returns (V, iters, mismatch, fallback columns, status)."""
        T = S.shape[0]
        _host_buffer(S, "S", np.complex128, (T, self.n_pq))
        if net.n_pq != self.n_pq:
            raise ValueError(f"the network is for {net.n_pq} demand buses, the feeder has {self.n_pq}")
        if out is None:
            V = np.empty((T, self.n_pq), dtype=np.complex128)
            it = np.empty(T, dtype=np.int32)
            mm = np.empty(T, dtype=np.float64)
        else:
            V, it, mm = out
            _host_buffer(V, "V", np.complex128, (T, self.n_pq))
            _host_buffer(it, "iters", np.int32, (T,))
            _host_buffer(mm, "mismatch", np.float64, (T,))

        def ptr(a):
            return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)

        dev = getattr(self, "device", None)
        if dev is not None and getattr(net, "device", dev) != dev:
            raise ValueError(f"the network is on cuda:{net.device}, the feeder on cuda:{dev}")
        o = make_opts("mixed", tol, max_iter, "warm", switch_tol, profile, "sparse")
        fb = ctypes.c_int64(0)
        with _on_device(dev):
            st = lib().tpf_solve_learned_host(self._h, net._h, T, ptr(S), ptr(V), ptr(it), ptr(mm), ctypes.byref(o),
                                              ctypes.byref(fb), _stream_ptr(stream, dev))
        if check and st not in (OK, ENOCONV):
            raise TpfError(st, "tpf_solve_learned_host")
        return V, it, mm, fb.value, st

    def solve_tensor(self, S, V=None, want_V=True, v_complex64=None, v_band=(0.95, 1.05), bus_counts=None,
                     tol=1e-10, max_iter=100, start=None, switch_tol=1e-4, stream=None, check=True, profile=False):
        """tpf_solve_ex on a load tensor of any leading shape [..., n_pq] (complex64 or complex128).

        Returns a dict: V (same leading shape; None when want_V is False), iters, mismatch, vmin, vmax
        (per column |V| extremes), viol (buses outside v_band per column), bus_under / bus_over
        (columns below / above the band per bus, added to `bus_counts` when given) and status.
        """
        import torch

        if not (isinstance(S, torch.Tensor) and S.is_cuda and S.dtype in (torch.complex64, torch.complex128)):
            raise TypeError("S must be a CUDA complex64 or complex128 tensor")
        if S.shape[-1] != self.n_pq or not S.is_contiguous():
            raise ValueError(f"S must be contiguous with last dimension {self.n_pq}")
        lead = S.shape[:-1]
        T = int(np.prod(lead)) if len(lead) else 1
        dev = S.device
        if start is None:
            start = "given" if V is not None else "flat"
        v32 = (S.dtype == torch.complex64) if v_complex64 is None else bool(v_complex64)
        vdt = torch.complex64 if v32 else torch.complex128
        if V is None and (want_V or start in ("given", "warm")):
            V = torch.empty(S.shape, dtype=vdt, device=dev)
        if V is not None and (V.dtype != vdt or V.shape != S.shape or not V.is_contiguous()):
            raise ValueError("V must be contiguous, shaped like S, complex64 iff v_complex64")
        it = torch.empty(lead, dtype=torch.int32, device=dev)
        mm = torch.empty(lead, dtype=torch.float64, device=dev)
        vmin = torch.empty(lead, dtype=torch.float32, device=dev)
        vmax = torch.empty(lead, dtype=torch.float32, device=dev)
        viol = torch.empty(lead, dtype=torch.int32, device=dev)
        if bus_counts is None:
            bus_counts = (torch.zeros(self.n_pq, dtype=torch.int32, device=dev),
                          torch.zeros(self.n_pq, dtype=torch.int32, device=dev))
        else:  # the kernels add n_pq counters into each
            if len(bus_counts) != 2:
                raise ValueError("bus_counts must be a pair (under, over)")
            _device_tensors([("bus_counts[0]", bus_counts[0], torch.int32, (self.n_pq,)),
                             ("bus_counts[1]", bus_counts[1], torch.int32, (self.n_pq,))])
        out = Outputs(1 if S.dtype == torch.complex64 else 0, 1 if v32 else 0, float(v_band[0]), float(v_band[1]),
                      vmin.data_ptr(), vmax.data_ptr(), viol.data_ptr(), bus_counts[0].data_ptr(),
                      bus_counts[1].data_ptr())
        dev = _one_device([("S", S), ("V", V), ("bus_counts[0]", bus_counts[0]), ("bus_counts[1]", bus_counts[1])],
                          getattr(self, "device", None))
        o = make_opts("mixed", tol, max_iter, start, switch_tol, profile, "sparse")
        vp = ctypes.c_void_p
        with _on_device(dev):
            st = lib().tpf_solve_ex(self._h, T, vp(S.data_ptr()), vp(V.data_ptr() if V is not None else 0),
                                    vp(it.data_ptr()), vp(mm.data_ptr()), ctypes.byref(out), ctypes.byref(o),
                                    _stream_ptr(stream, dev))
        if check and st not in (OK, ENOCONV):
            raise TpfError(st, "tpf_solve_ex")
        return {"V": V, "iters": it, "mismatch": mm, "vmin": vmin, "vmax": vmax, "viol": viol,
                "bus_under": bus_counts[0], "bus_over": bus_counts[1], "status": st}

    def solve_host(self, S, V0=None, precision="mixed", tol=1e-10, max_iter=100, switch_tol=1e-4, stream=None,
                   out=None, check=True, profile=False, method="dense", start=None):
        """tpf_solve_host on host arrays (numpy or pinned torch CPU tensors, complex128 [T][n_pq]).
        With V0, start is 'given' (default) or 'warm'."""
        T = S.shape[0]
        _host_buffer(S, "S", np.complex128, (T, self.n_pq))
        if V0 is not None:
            _host_buffer(V0, "V0", np.complex128, (T, self.n_pq))
        if out is None:
            V = np.empty((T, self.n_pq), dtype=np.complex128) if V0 is None else V0
            it = np.empty(T, dtype=np.int32)
            mm = np.empty(T, dtype=np.float64)
        else:
            V, it, mm = out
            _host_buffer(V, "V", np.complex128, (T, self.n_pq))
            _host_buffer(it, "iters", np.int32, (T,))
            _host_buffer(mm, "mismatch", np.float64, (T,))
        if V0 is not None and V is not V0:
            V[...] = V0

        def ptr(a):
            return ctypes.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)

        if start is None:
            start = "given" if V0 is not None else "flat"
        o = make_opts(precision, tol, max_iter, start, switch_tol, profile, method)
        dev = getattr(self, "device", None)
        with _on_device(dev):
            st = lib().tpf_solve_host(self._h, T, ptr(S), ptr(V), ptr(it), ptr(mm), ctypes.byref(o),
                                      _stream_ptr(stream, dev))
        if check and st not in (OK, ENOCONV):
            raise TpfError(st, "tpf_solve_host")
        return V, it, mm, st


def _batch_device(feeders, S, V, iters, mismatch):
    """The one device of a batch: every feeder's and every tensor's.  With a single visible GPU every
    CUDA tensor is on it, and the per-tensor pass (thousands of tensors in a large batch) is skipped."""
    import torch

    if torch.cuda.device_count() == 1 and len(S):
        return S[0].device.index
    named = []
    for f in range(len(S)):
        named += [(f"S[{f}]", S[f]), (f"V[{f}]", V[f]), (f"iters[{f}]", iters[f]), (f"mismatch[{f}]", mismatch[f])]
    devs = {getattr(fd, "device", None) for fd in feeders} - {None}
    if len(devs) > 1:
        raise ValueError("the feeders of a batch must be on one device")
    return _one_device(named, devs.pop() if devs else None)


def solve_batch(feeders, S, V=None, iters=None, mismatch=None, precision="mixed", tol=1e-10, max_iter=100,
                start=None, switch_tol=1e-4, method="sparse", stream=None, check=True, profile=False):
    """tpf_solve_batch over a list of Feeder objects with their CUDA complex128 load tensors.

    Outputs (V, iters, mismatch lists) are allocated when not given.  Returns
    (V, iters, mismatch, converged per feeder (numpy int64), stats dict, status).
    """
    import torch

    F = len(feeders)
    if len(S) != F:
        raise ValueError("one load tensor per feeder")
    if start is None:
        start = "given" if V is not None else "flat"
    supplied = V is not None or iters is not None or mismatch is not None
    V = list(V) if V is not None else [torch.empty_like(s) for s in S]
    iters = list(iters) if iters is not None else [torch.empty(s.shape[0], dtype=torch.int32, device=s.device)
                                                    for s in S]
    mismatch = list(mismatch) if mismatch is not None else [
        torch.empty(s.shape[0], dtype=torch.float64, device=s.device) for s in S]
    for f in range(F):
        s = S[f]
        if not (isinstance(s, torch.Tensor) and s.is_cuda and s.dtype == torch.complex128 and s.dim() == 2
                and s.shape[1] == feeders[f].n_pq and s.is_contiguous()):
            raise ValueError(f"S[{f}] must be a contiguous CUDA complex128 [T, n_pq] tensor")
    if supplied:
        _batch_outputs(S, V, iters, mismatch)
    dev = _batch_device(feeders, S, V, iters, mismatch)
    P = ctypes.c_void_p * F
    hs = P(*[fd._h.value for fd in feeders])
    Ts = (ctypes.c_int64 * F)(*[int(s.shape[0]) for s in S])
    Sp = P(*[s.data_ptr() for s in S])
    Vp = P(*[v.data_ptr() for v in V])
    Ip = P(*[i.data_ptr() for i in iters])
    Mp = P(*[m.data_ptr() for m in mismatch])
    conv = (ctypes.c_int64 * F)()
    st_ = Stats()
    o = make_opts(precision, tol, max_iter, start, switch_tol, profile, method)
    with _on_device(dev):
        st = lib().tpf_solve_batch(F, hs, Ts, Sp, Vp, Ip, Mp, ctypes.byref(o), conv, ctypes.byref(st_),
                                   _stream_ptr(stream, dev))
    if check and st not in (OK, ENOCONV):
        raise TpfError(st, "tpf_solve_batch")
    return V, iters, mismatch, np.array(conv[:], dtype=np.int64), st_.as_dict(), st


class BatchGraph:
    """tpf_batch_*: a batch of radial feeders prepared once (sparse method, mixed precision) and
    solved by replaying one captured CUDA graph.  Rewrite the tensors of S in place and call
    launch() / wait() again to solve new loads.  The feeders and tensors must outlive the object.
    """

    def __init__(self, feeders, S, V=None, iters=None, mismatch=None, tol=1e-10, max_iter=100, start=None,
                 switch_tol=1e-4):
        import torch

        F = len(feeders)
        if len(S) != F:
            raise ValueError("one load tensor per feeder")
        if start is None:
            start = "given" if V is not None else "flat"
        self.V = list(V) if V is not None else [torch.empty_like(s) for s in S]
        self.iters = list(iters) if iters is not None else [
            torch.empty(s.shape[0], dtype=torch.int32, device=s.device) for s in S]
        self.mismatch = list(mismatch) if mismatch is not None else [
            torch.empty(s.shape[0], dtype=torch.float64, device=s.device) for s in S]
        for f in range(F):
            s = S[f]
            if not (isinstance(s, torch.Tensor) and s.is_cuda and s.dtype == torch.complex128 and s.dim() == 2
                    and s.shape[1] == feeders[f].n_pq and s.is_contiguous()):
                raise ValueError(f"S[{f}] must be a contiguous CUDA complex128 [T, n_pq] tensor")
        _batch_outputs(S, self.V, self.iters, self.mismatch)
        self.device = _batch_device(feeders, S, self.V, self.iters, self.mismatch)
        self.F, self.S, self.feeders = F, list(S), list(feeders)
        P = ctypes.c_void_p * F
        hs = P(*[fd._h.value for fd in feeders])
        Ts = (ctypes.c_int64 * F)(*[int(s.shape[0]) for s in S])
        o = make_opts("mixed", tol, max_iter, start, switch_tol, False, "sparse")
        self._b = ctypes.c_void_p()
        with _on_device(self.device):
            st = lib().tpf_batch_create(F, hs, Ts, P(*[s.data_ptr() for s in S]), P(*[v.data_ptr() for v in self.V]),
                                        P(*[i.data_ptr() for i in self.iters]),
                                        P(*[m.data_ptr() for m in self.mismatch]), ctypes.byref(o),
                                        ctypes.byref(self._b))
        if st != OK:
            raise TpfError(st, "tpf_batch_create")

    def launch(self, stream=None):
        with _on_device(self.device):
            st = lib().tpf_batch_launch(self._b, _stream_ptr(stream, self.device))
        if st != OK:
            raise TpfError(st, "tpf_batch_launch")

    def wait(self, check=True):
        """(converged per feeder (numpy int64), stats dict, status) of the last launch."""
        conv = (ctypes.c_int64 * self.F)()
        st_ = Stats()
        st = lib().tpf_batch_wait(self._b, conv, ctypes.byref(st_))
        if check and st not in (OK, ENOCONV):
            raise TpfError(st, "tpf_batch_wait")
        return np.array(conv[:], dtype=np.int64), st_.as_dict(), st

    def close(self):
        if self._b:
            lib().tpf_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_fp64_noalloc(K, W, S, V, iters=None, tol=1e-10, max_iter=100, given_start=False, stream=None):
    """tpf_solve_fp64_noalloc: the FP64 solve without any allocation by the library.

    For callers whose device memory all comes from their own pool: K (complex128 [n, n]), W
    (complex128 [n]), S and V (complex128 [T, n]) and iters (int32 [T], optional) are the caller's
    CUDA tensors; the solve's scratch is libtpf's built-in 64 MiB array.  Returns the status.
    """
    import torch

    n = K.shape[0]
    T = S.shape[0]
    c128 = torch.complex128
    _device_tensors([("K", K, c128, (n, n)), ("W", W, c128, (n,)), ("S", S, c128, (T, n)), ("V", V, c128, (T, n))]
                    + ([("iters", iters, torch.int32, (T,))] if iters is not None else []))
    dev = _one_device([("K", K), ("W", W), ("S", S), ("V", V), ("iters", iters)])
    with _on_device(dev):  # the library solves on the current device
        return lib().tpf_solve_fp64_noalloc(
            int(n), ctypes.c_void_p(K.data_ptr()), ctypes.c_void_p(W.data_ptr()), int(T),
            ctypes.c_void_p(S.data_ptr()), ctypes.c_void_p(V.data_ptr()),
            ctypes.c_void_p(iters.data_ptr() if iters is not None else 0), float(tol), int(max_iter),
            1 if given_start else 0, _stream_ptr(stream, dev))


def selftest_gemm(Ar, Ai, Br, Bi, stream=None, wait_s=None, withhold_loads=False, check=True):
    """D = A B^T over complex numbers with the library's tcgen05 kernel (fp16 in, FP32 out).

    wait_s / withhold_loads: tpf_selftest_gemm_wait, the test of the kernel's bounded waits (with
    withhold_loads the waits run out and the status is ETIMEOUT).  Returns (Dr, Di), or
    (Dr, Di, status) when check is False."""
    import torch

    M, K = Ar.shape
    N = Br.shape[0]
    f16 = torch.float16
    _device_tensors([("Ar", Ar, f16, (M, K)), ("Ai", Ai, f16, (M, K)), ("Br", Br, f16, (N, K)), ("Bi", Bi, f16, (N, K))])
    dev = _one_device([("Ar", Ar), ("Ai", Ai), ("Br", Br), ("Bi", Bi)])
    Dr = torch.empty((N, M), dtype=torch.float32, device=Ar.device)
    Di = torch.empty((N, M), dtype=torch.float32, device=Ar.device)
    ptrs = [ctypes.c_void_p(x.data_ptr()) for x in (Ar, Ai, Br, Bi, Dr, Di)]
    with _on_device(dev):
        if wait_s is None and not withhold_loads:
            st = lib().tpf_selftest_gemm(M, N, K, *ptrs, _stream_ptr(stream, dev))
        else:
            st = lib().tpf_selftest_gemm_wait(M, N, K, *ptrs, float(2.0 if wait_s is None else wait_s),
                                              1 if withhold_loads else 0, _stream_ptr(stream, dev))
    if not check:
        return Dr, Di, st
    if st != OK:
        raise TpfError(st, "tpf_selftest_gemm")
    return Dr, Di


class LearnedStart:
    """The learned warm-start network of libtpf (tpf_mlp_*): BF16 tensor-core training and inference.

    Inputs are a column's loads (P then Q of the n demand buses), outputs Re V - 1 and Im V; both
    z-scored with statistics fitted on training columns.  All arithmetic runs in libtpf's kernels.
    """

    def __init__(self, n_pq, hidden=256, hidden_layers=3, max_batch=1024, seed=1):
        h = ctypes.c_void_p()
        st = lib().tpf_mlp_create(int(n_pq), int(hidden), int(hidden_layers), int(max_batch), int(seed),
                                  ctypes.byref(h))
        if st != OK:
            raise TpfError(st, "tpf_mlp_create")
        self._h = h
        self.n_pq = int(n_pq)
        self.max_batch = int(max_batch)
        self.device = _current_device()  # tpf_mlp_create allocates on the current device
        self.sizes = [2 * n_pq] + [hidden] * hidden_layers + [2 * n_pq]

    def close(self):
        if getattr(self, "_h", None):
            lib().tpf_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _f32(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))

    def params(self):
        """Flat FP32 parameters: per layer W (out x in, row-major) then b."""
        out = np.empty(lib().tpf_mlp_param_count(self._h), dtype=np.float32)
        st = lib().tpf_mlp_get_params(self._h, self._f32(out))
        if st != OK:
            raise TpfError(st, "tpf_mlp_get_params")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        st = lib().tpf_mlp_set_params(self._h, self._f32(flat))
        if st != OK:
            raise TpfError(st, "tpf_mlp_set_params")

    def unflatten(self, flat):
        Ws, bs, off = [], [], 0
        for i in range(len(self.sizes) - 1):
            o, k = self.sizes[i + 1], self.sizes[i]
            Ws.append(flat[off:off + o * k].reshape(o, k))
            off += o * k
            bs.append(flat[off:off + o])
            off += o
        return Ws, bs

    def _columns(self, S, V=None, vname="V"):
        """S (and V) must be contiguous CUDA complex128 [T, n_pq] tensors, V shaped like S: the
        kernels read T x n_pq values from each.  Dtypes and shapes are checked before placement."""
        import torch

        pairs = [("S", S)] + ([(vname, V)] if V is not None else [])
        for name, X in pairs:
            if not isinstance(X, torch.Tensor) or X.dtype != torch.complex128:
                raise TypeError(f"{name} must be a complex128 torch tensor")
            if X.dim() != 2 or X.shape[1] != self.n_pq or X.shape != S.shape:
                raise ValueError(f"{name} must have shape [T, {self.n_pq}]" + (" like S" if name != "S" else ""))
        for name, X in pairs:
            if not X.is_contiguous() or not X.is_cuda:
                raise ValueError(f"{name} must be a contiguous CUDA tensor")
        return _one_device(pairs, getattr(self, "device", None))

    def fit_normalization(self, S, V, stream=None):
        dev = self._columns(S, V)
        with _on_device(dev):
            st = lib().tpf_mlp_fit_normalization(self._h, S.shape[0], ctypes.c_void_p(S.data_ptr()),
                                                 ctypes.c_void_p(V.data_ptr()), _stream_ptr(stream, dev))
        if st != OK:
            raise TpfError(st, "tpf_mlp_fit_normalization")

    def normalization(self):
        a = [np.empty(2 * self.n_pq, dtype=np.float32) for _ in range(4)]
        st = lib().tpf_mlp_get_normalization(self._h, *(self._f32(x) for x in a))
        if st != OK:
            raise TpfError(st, "tpf_mlp_get_normalization")
        return tuple(a)

    def train_step(self, S, V, lr=1e-3, want_loss=True, stream=None):
        dev = self._columns(S, V)
        loss = ctypes.c_double(0.0)
        with _on_device(dev):
            st = lib().tpf_mlp_train_step(self._h, S.shape[0], ctypes.c_void_p(S.data_ptr()),
                                          ctypes.c_void_p(V.data_ptr()), float(lr),
                                          ctypes.byref(loss) if want_loss else None, _stream_ptr(stream, dev))
        if st != OK:
            raise TpfError(st, "tpf_mlp_train_step")
        return loss.value if want_loss else None

    def gradients(self, S, V, stream=None):
        dev = self._columns(S, V)
        loss = ctypes.c_double(0.0)
        g = np.empty(lib().tpf_mlp_param_count(self._h), dtype=np.float32)
        with _on_device(dev):
            st = lib().tpf_mlp_gradients(self._h, S.shape[0], ctypes.c_void_p(S.data_ptr()),
                                         ctypes.c_void_p(V.data_ptr()), ctypes.byref(loss), self._f32(g),
                                         _stream_ptr(stream, dev))
        if st != OK:
            raise TpfError(st, "tpf_mlp_gradients")
        return loss.value, g

    def predict(self, S, V0=None, stream=None):
        """Predicted starting voltages (complex128 CUDA tensor like S) and the fallback count."""
        import torch

        if V0 is None:
            dev = self._columns(S)
            V0 = torch.empty_like(S)
        else:
            dev = self._columns(S, V0, "V0")
        fb = ctypes.c_int64(0)
        with _on_device(dev):
            st = lib().tpf_mlp_predict(self._h, S.shape[0], ctypes.c_void_p(S.data_ptr()),
                                       ctypes.c_void_p(V0.data_ptr()), ctypes.byref(fb), _stream_ptr(stream, dev))
        if st != OK:
            raise TpfError(st, "tpf_mlp_predict")
        return V0, fb.value
