"""libtpf's C ABI on the host (no GPU): symbols, host-side precomputation, argument checks."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tpf_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(tpf_lib):
    names = declared_symbols()
    assert "tpf_solve" in names and "tpf_create" in names
    for name in names:
        assert hasattr(tpf_lib, name), f"{name} not exported"
    assert set(tpf.EXPORTS) <= names


def test_strerror_and_defaults(tpf_lib):
    for st in range(8):
        assert tpf.strerror(st).startswith("TPF_")
    o = tpf.Opts()
    tpf_lib.tpf_default_opts(ctypes.byref(o))
    assert o.tol == 1e-10 and o.max_iter == 100 and o.precision == tpf.PREC_MIXED and o.start == tpf.START_FLAT


@pytest.mark.parametrize("n_bus,seed", [(2, 1), (34, 1), (150, 9)])
def test_precompute_host_matches_oracle_radial(tpf_lib, n_bus, seed):
    f = G.make_feeder(n_bus, seed)
    c = O.Case.from_feeder(f)
    K, W = tpf.precompute_host(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    assert np.abs(K - c.K).max() <= 1e-12 * np.abs(c.K).max()
    assert np.abs(W - c.W).max() <= 1e-13


def test_precompute_host_meshed_and_reordered(tpf_lib):
    f = G.make_feeder(50, 4)
    fb = np.r_[f.from_bus, 10, 3]
    tb = np.r_[f.to_bus, 40, 22]
    z = np.r_[f.z_pu, 0.01 + 0.02j, 0.03 + 0.01j]
    vs = 1.02 + 0.01j
    pq = np.array([b for b in range(50) if b != 0])[::-1].copy()  # reversed bus order
    c = O.Case(50, fb, tb, z, vs=vs, pq=pq)
    K, W = tpf.precompute_host(50, fb, tb, z, v0=vs, pq_bus=pq)
    assert np.abs(K - c.K).max() <= 1e-12 * np.abs(c.K).max()
    assert np.abs(W - c.W).max() <= 1e-13


def test_precompute_host_argument_errors(tpf_lib):
    z = [0.01 + 0.01j, 0.02 + 0.01j]
    with pytest.raises(tpf.TpfError) as e:
        tpf.precompute_host(3, [0, 0], [1, 1], z)  # bus 2 isolated: Y_dd singular
    assert e.value.status == tpf.ESINGULAR
    with pytest.raises(tpf.TpfError) as e:
        tpf.precompute_host(3, [0, 1], [1, 7], z)  # index out of range
    assert e.value.status == tpf.EINVAL
    with pytest.raises(tpf.TpfError) as e:
        tpf.precompute_host(3, [0, 1], [1, 2], [0.01 + 0.01j, 0.0])  # zero impedance
    assert e.value.status == tpf.EINVAL
    with pytest.raises(tpf.TpfError) as e:
        tpf.precompute_host(3, [0, 1], [1, 2], z, pq_bus=[1, 1])  # repeated bus
    assert e.value.status == tpf.EINVAL
    with pytest.raises(tpf.TpfError) as e:
        tpf.precompute_host(3, [0, 1], [1, 2], z, pq_bus=[0, 1])  # slack listed as PQ
    assert e.value.status == tpf.EINVAL


def test_create_fails_loudly_without_a_device(tpf_lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    f = G.make_feeder(10, 1)
    with pytest.raises(tpf.TpfError) as e:
        tpf.Feeder.from_inputs(f)
    assert e.value.status == tpf.ECUDA


def test_batch_entry_points_argument_errors(tpf_lib):
    """The prepared-batch entry points reject bad arguments before touching a device."""
    vp = ctypes.c_void_p
    out = vp(123)
    h = (vp * 1)(vp(0))
    T = (ctypes.c_int64 * 1)(4)
    ptrs = (vp * 1)(vp(0))
    o = tpf.Opts()
    tpf_lib.tpf_default_opts(ctypes.byref(o))
    assert tpf_lib.tpf_batch_create(1, h, T, ptrs, ptrs, None, None, ctypes.byref(o), None) == tpf.EINVAL
    assert tpf_lib.tpf_batch_create(0, h, T, ptrs, ptrs, None, None, ctypes.byref(o), ctypes.byref(out)) == tpf.EINVAL
    assert out.value is None  # cleared on failure
    assert tpf_lib.tpf_batch_create(1, None, T, ptrs, ptrs, None, None, ctypes.byref(o), ctypes.byref(out)) == tpf.EINVAL
    assert tpf_lib.tpf_batch_create(1, h, T, ptrs, ptrs, None, None, ctypes.byref(o), ctypes.byref(out)) == tpf.EINVAL
    assert tpf_lib.tpf_batch_launch(None, None) == tpf.EINVAL
    assert tpf_lib.tpf_batch_wait(None, None, None) == tpf.EINVAL
    tpf_lib.tpf_batch_destroy(None)


def test_make_opts_maps_names_to_abi_constants(tpf_lib):
    o = tpf.make_opts("fp64", tol=1e-9, max_iter=50, start="warm", switch_tol=1e-3, profile=True, method="sparse")
    assert (o.precision, o.start, o.method) == (tpf.PREC_FP64, tpf.START_WARM, tpf.METHOD_SPARSE)
    assert o.tol == 1e-9 and o.max_iter == 50 and o.switch_tol == 1e-3 and o.profile == 1
    o = tpf.make_opts()
    assert (o.precision, o.start, o.method, o.profile) == (tpf.PREC_MIXED, tpf.START_FLAT, tpf.METHOD_DENSE, 0)
    assert tpf.make_opts(start="given").start == tpf.START_GIVEN
    assert tpf.make_opts(precision=tpf.PREC_FP64, method=tpf.METHOD_DENSE).precision == tpf.PREC_FP64
    with pytest.raises(TypeError):
        tpf.make_opts(precision="bf16")
    with pytest.raises(TypeError):
        tpf.make_opts(method="newton")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libtpf.so every entry point of the binding raises; there is no CPU fallback."""
    monkeypatch.setattr(tpf, "_lib", None)
    monkeypatch.setattr(tpf._build, "LIB", str(tmp_path / "libtpf.so"))
    with pytest.raises(RuntimeError, match="not built"):
        tpf.lib()
    with pytest.raises(RuntimeError, match="not built"):
        tpf.make_opts()
    with pytest.raises(RuntimeError, match="not built"):
        tpf.Feeder.from_inputs(G.make_feeder(10, 1))
    with pytest.raises(RuntimeError, match="not built"):
        tpf.precompute_host(2, [0], [1], [0.1 + 0.05j])


def test_noalloc_argument_errors_before_any_device_call(tpf_lib):
    """tpf_solve_fp64_noalloc checks its arguments and its 64 MiB scratch bound on the host first.
    The pointers below are stand-ins that none of these calls dereferences."""
    import math

    import torch

    f = tpf_lib.tpf_solve_fp64_noalloc
    p = ctypes.c_void_p(0x1000)

    def call(n=33, K=p, W=p, T=8, S=p, V=p, tol=1e-10, max_iter=100):
        return f(n, K, W, T, S, V, None, ctypes.c_double(tol), max_iter, 0, None)

    for kw in ({"n": 0}, {"T": -1}, {"tol": -1.0}, {"tol": math.nan}, {"max_iter": 0}, {"max_iter": 100001},
               {"K": None}, {"W": None}, {"S": None}, {"V": None}):
        assert call(**kw) == tpf.EINVAL, kw
    assert call(T=0, K=None, W=None, S=None, V=None) == tpf.OK  # nothing to do
    # Scratch = 1024 + 16 T_128 (n + 1) bytes <= 64 MiB: at n = 33 the largest T is 963 x 128.
    assert call(n=33, T=963 * 128 + 1) == tpf.EINVAL
    assert call(n=999, T=5000) == tpf.EINVAL
    if not torch.cuda.is_available():
        assert call(n=33, T=963 * 128) == tpf.ECUDA  # within the bound: it goes on to the (absent) device


def test_entry_points_refuse_null_handles_and_bad_arguments_on_the_host(tpf_lib):
    """Every entry point that takes a handle refuses NULL, and option, size and pointer errors are
    returned before any handle is read or any device call is made."""
    L = tpf_lib
    vp = ctypes.c_void_p
    p = vp(0x1000)  # a stand-in pointer that these calls never dereference
    o = tpf.Opts()
    L.tpf_default_opts(ctypes.byref(o))
    bad = tpf.Opts()
    L.tpf_default_opts(ctypes.byref(bad))
    bad.tol = -1.0
    st = tpf.Stats()
    out = tpf.Outputs(0, 0, 0.95, 1.05, None, None, None, None, None)
    E = tpf.EINVAL

    assert L.tpf_solve(None, 8, p, p, None, None, ctypes.byref(o), None) == E
    assert L.tpf_solve_host(None, 8, p, p, None, None, ctypes.byref(o), None) == E
    assert L.tpf_solve_ex(None, 8, p, p, None, None, None, ctypes.byref(o), None) == E
    assert L.tpf_solve_ex(None, 8, p, p, None, None, ctypes.byref(out), ctypes.byref(o), None) == E
    assert L.tpf_autotune(None, 8, p, ctypes.byref(o), None, None) == E
    assert L.tpf_set_zip(None, None) == E
    assert L.tpf_last_stats(None, ctypes.byref(st)) == E
    assert L.tpf_n_pq(None) == -1
    L.tpf_destroy(None)

    # tpf_solve_batch: sizes and pointer arrays first, options before the empty-batch return.
    assert L.tpf_solve_batch(-1, None, None, None, None, None, None, ctypes.byref(o), None, None, None) == E
    assert L.tpf_solve_batch(1, None, None, None, None, None, None, ctypes.byref(o), None, None, None) == E
    assert L.tpf_solve_batch(0, None, None, None, None, None, None, ctypes.byref(bad), None, None, None) == E
    st.columns = 99
    assert L.tpf_solve_batch(0, None, None, None, None, None, None, ctypes.byref(o), None, ctypes.byref(st),
                             None) == tpf.OK
    assert st.columns == 0  # statistics cleared

    # The tensor-core self-test: tile multiples and pointers.
    assert L.tpf_selftest_gemm(100, 128, 64, p, p, p, p, p, p, None) == E
    assert L.tpf_selftest_gemm(128, 128, 64, p, None, p, p, p, p, None) == E

    # Learned start.
    h = vp(123)
    assert L.tpf_mlp_create(10, 256, 3, 1024, 1, None) == E
    assert L.tpf_mlp_create(0, 256, 3, 1024, 1, ctypes.byref(h)) == E and h.value is None
    assert L.tpf_mlp_create(10, 256, 17, 1024, 1, ctypes.byref(h)) == E
    assert L.tpf_mlp_create(10, 256, 3, 100, 1, ctypes.byref(h)) == E
    assert L.tpf_mlp_param_count(None) == -1
    f32 = (ctypes.c_float * 4)()
    assert L.tpf_mlp_get_params(None, f32) == E
    assert L.tpf_mlp_set_params(None, f32) == E
    assert L.tpf_mlp_fit_normalization(None, 8, p, p, None) == E
    assert L.tpf_mlp_get_normalization(None, f32, f32, f32, f32) == E
    assert L.tpf_mlp_train_step(None, 128, p, p, 1e-3, None, None) == E
    assert L.tpf_mlp_gradients(None, 128, p, p, None, f32, None) == E
    assert L.tpf_mlp_predict(None, 8, p, p, None, None) == E
    L.tpf_mlp_destroy(None)

    # The learned-start solve from host buffers: handles, sizes and options before any device call.
    fb = ctypes.c_int64(7)
    assert L.tpf_solve_learned_host(None, p, 8, p, p, None, None, ctypes.byref(o), ctypes.byref(fb), None) == E
    assert fb.value == 0
    assert L.tpf_solve_learned_host(p, None, 8, p, p, None, None, ctypes.byref(o), None, None) == E
    assert L.tpf_solve_learned_host(p, p, -1, p, p, None, None, ctypes.byref(o), None, None) == E
    assert L.tpf_solve_learned_host(p, p, 8, p, p, None, None, ctypes.byref(bad), None, None) == E
    dense = tpf.make_opts("mixed", 1e-10, 100, "warm", 1e-4, False, "dense")
    assert L.tpf_solve_learned_host(p, p, 8, p, p, None, None, ctypes.byref(dense), None, None) == tpf.EUNSUPPORTED
    fp64 = tpf.make_opts("fp64", 1e-10, 100, "warm", 1e-4, False, "sparse")
    assert L.tpf_solve_learned_host(p, p, 8, p, p, None, None, ctypes.byref(fp64), None, None) == tpf.EUNSUPPORTED


def test_solve_host_checks_its_host_buffers_before_the_library():
    """tpf_solve_host reads and writes T x n_pq complex128 values: the binding refuses buffers of
    another dtype, shape or layout, and device tensors, before any library call."""
    import torch

    fd = object.__new__(tpf.Feeder)  # no device here: the checks come first
    fd._h, fd.n_pq = None, 5
    T = 4
    S = np.zeros((T, 5), np.complex128)
    bad_S = [S.astype(np.complex64), np.zeros((T, 6), np.complex128), np.zeros((5, T), np.complex128).T,
             torch.zeros((T, 5), dtype=torch.complex64)]
    for b in bad_S:
        with pytest.raises(ValueError, match="S must be"):
            fd.solve_host(b)
    with pytest.raises(ValueError, match="V0 must be"):
        fd.solve_host(S, V0=np.ones((T, 5), np.complex64))
    good = (torch.zeros((T, 5), dtype=torch.complex128), torch.zeros(T, dtype=torch.int32),
            torch.zeros(T, dtype=torch.float64))
    for k, b in ((1, torch.zeros(T, dtype=torch.int64)), (2, np.zeros(T, np.float32)),
                 (0, torch.zeros((T, 4), dtype=torch.complex128))):
        out = list(good)
        out[k] = b
        with pytest.raises(ValueError, match="must be a C-contiguous host"):
            fd.solve_host(S, out=tuple(out))
    # Well-formed buffers pass the checks and fail loudly further on: without a CUDA driver at the
    # stream lookup, otherwise in the library, which refuses the missing handle.
    with pytest.raises((tpf.TpfError, RuntimeError)) as e:
        fd.solve_host(torch.from_numpy(S), out=good)
    if isinstance(e.value, tpf.TpfError):
        assert e.value.status == tpf.EINVAL


def test_learned_start_checks_its_tensors_before_the_library():
    """The network's kernels read T x n_pq complex128 values: other dtypes, widths, mismatched V and
    host tensors are refused in the binding."""
    import torch

    net = object.__new__(tpf.LearnedStart)  # no device here: the checks come first
    net._h, net.n_pq, net.max_batch = None, 6, 1024
    S = torch.zeros((128, 6), dtype=torch.complex128)
    with pytest.raises(TypeError, match="S must be a complex128"):
        net.predict(S.to(torch.complex64))
    with pytest.raises(ValueError, match=r"S must have shape \[T, 6\]"):
        net.train_step(torch.zeros((128, 7), dtype=torch.complex128), S)
    with pytest.raises(ValueError, match="V must have shape"):
        net.gradients(S, torch.zeros((256, 6), dtype=torch.complex128))
    with pytest.raises(ValueError, match="V must have shape"):
        net.fit_normalization(S, torch.zeros((128, 5), dtype=torch.complex128))
    with pytest.raises(ValueError, match="contiguous CUDA"):
        net.fit_normalization(S, S)  # host tensors
    with pytest.raises(ValueError, match="contiguous CUDA"):
        net.predict(torch.zeros((128, 12), dtype=torch.complex128)[:, ::2])  # strided columns
    with pytest.raises(ValueError, match="V0 must have shape"):
        net.predict(S, torch.zeros((64, 6), dtype=torch.complex128))


def test_noalloc_and_gemm_bindings_check_their_tensors():
    """The allocation-free solve and the GEMM self-test pass raw pointers: the binding checks that
    every tensor has the dtype and shape the kernels assume, and lives on the device."""
    import torch

    c = torch.complex128
    K, W = torch.zeros((4, 4), dtype=c), torch.zeros(4, dtype=c)
    S = torch.zeros((8, 4), dtype=c)
    cases = [((torch.zeros((4, 5), dtype=c), W, S, S), "K must be"),
             ((K, torch.zeros(5, dtype=c), S, S), "W must be"),
             ((K, W, torch.zeros((8, 3), dtype=c), S), "S must be"),
             ((K, W, S, torch.zeros((8, 4), dtype=torch.complex64)), "V must be"),
             ((K, W, S, S, torch.zeros(8, dtype=torch.int64)), "iters must be"),
             ((K, W, S, S), "contiguous CUDA")]
    for args, msg in cases:
        with pytest.raises(ValueError, match=msg):
            tpf.solve_fp64_noalloc(*args)
    h = torch.zeros((128, 64), dtype=torch.float16)
    with pytest.raises(ValueError, match="Ai must be"):
        tpf.selftest_gemm(h, torch.zeros((128, 32), dtype=torch.float16), h, h)
    with pytest.raises(ValueError, match="Br must be"):
        tpf.selftest_gemm(h, h, h.float(), h)
    with pytest.raises(ValueError, match="contiguous CUDA"):
        tpf.selftest_gemm(h, h, h, h)


def test_batch_output_lists_are_checked():
    """Caller-supplied batch outputs must match each feeder's loads in count, dtype and shape."""
    import torch

    S = [torch.zeros((8, 4), dtype=torch.complex128), torch.zeros((3, 6), dtype=torch.complex128)]
    V = [torch.zeros_like(s) for s in S]
    it = [torch.zeros(s.shape[0], dtype=torch.int32) for s in S]
    mm = [torch.zeros(s.shape[0], dtype=torch.float64) for s in S]
    with pytest.raises(ValueError, match="one V, iters and mismatch"):
        tpf._batch_outputs(S, V[:1], it, mm)
    with pytest.raises(ValueError, match=r"V\[1\] must be"):
        tpf._batch_outputs(S, [V[0], torch.zeros((3, 5), dtype=torch.complex128)], it, mm)
    with pytest.raises(ValueError, match=r"iters\[0\] must be"):
        tpf._batch_outputs(S, V, [torch.zeros(8, dtype=torch.int64), it[1]], mm)
    with pytest.raises(ValueError, match=r"mismatch\[1\] must be"):
        tpf._batch_outputs(S, V, it, [mm[0], torch.zeros(4, dtype=torch.float64)])
    with pytest.raises(ValueError, match="contiguous CUDA"):
        tpf._batch_outputs(S, V, it, mm)  # well-formed, but host tensors


def test_autotune_and_tensor_counters_are_checked():
    import torch

    fd = object.__new__(tpf.Feeder)
    fd._h, fd.n_pq = None, 5
    with pytest.raises(ValueError, match="S must be"):
        fd.autotune(torch.zeros((16, 4), dtype=torch.complex128))
    with pytest.raises(ValueError, match="S must be"):
        fd.autotune(torch.zeros(16, dtype=torch.complex128))
    with pytest.raises(ValueError, match="contiguous CUDA"):
        fd.autotune(torch.zeros((16, 5), dtype=torch.complex128))
    with pytest.raises(ValueError, match="S must be"):
        fd.autotune(np.zeros((16, 5), np.complex128))


def test_solve_host_accepts_the_buffers_callers_use():
    """Row slices of a C-contiguous array, a V0 copy and CPU torch outputs pass the checks; the call
    then fails only for want of a device (a CUDA driver here, the handle in the library)."""
    import torch

    fd = object.__new__(tpf.Feeder)
    fd._h, fd.n_pq = None, 5
    big = np.zeros((40, 5), np.complex128)
    S = big[10:30]  # a row slice stays C-contiguous
    out = (torch.zeros((20, 5), dtype=torch.complex128), torch.zeros(20, dtype=torch.int32),
           torch.zeros(20, dtype=torch.float64))
    for kw in ({}, {"V0": (S + 1.0).copy(), "start": "warm"}, {"out": out}):
        with pytest.raises((tpf.TpfError, RuntimeError)) as e:
            fd.solve_host(S, **kw)
        assert not isinstance(e.value, ValueError)


def test_tensors_on_another_device_are_refused():
    """The library launches on one device and passes raw pointers: a tensor on another GPU than
    the call's other tensors, or than the feeder's or network's device, is refused in the binding,
    and so is a stream of another device (CPU stand-ins carry only a device)."""
    from types import SimpleNamespace

    import torch

    def on(k):
        return SimpleNamespace(device=torch.device("cuda", k))

    assert tpf._one_device([("S", on(1)), ("V", on(1)), ("iters", None)]) == 1
    assert tpf._one_device([("S", on(0))], want=0) == 0
    with pytest.raises(ValueError, match=r"V is on cuda:1, but the device of S is cuda:0"):
        tpf._one_device([("S", on(0)), ("V", on(1))])
    with pytest.raises(ValueError, match=r"S is on cuda:2, but the device this object was created on is cuda:0"):
        tpf._one_device([("S", on(2))], want=0)
    with pytest.raises(ValueError, match="belongs to cuda:1"):
        tpf._stream_ptr(SimpleNamespace(device=torch.device("cuda", 1), cuda_stream=0), 0)
    feeders = [SimpleNamespace(device=0), SimpleNamespace(device=1)]
    t = [on(0), on(0)]
    with pytest.raises(ValueError, match="feeders of a batch must be on one device"):
        tpf._batch_device(feeders, t, t, t, t)
    with pytest.raises(ValueError, match=r"mismatch\[1\] is on cuda:1"):
        tpf._batch_device(feeders[:1] * 2, t, t, t, [on(0), on(1)])
    assert tpf._batch_device(feeders[:1] * 2, t, t, t, t) == 0


def test_gemm_wait_selftest_refuses_bad_limits_on_the_host(tpf_lib):
    """tpf_selftest_gemm_wait checks its sizes, pointers and wait limit before any device call."""
    p = ctypes.c_void_p(16)
    f = ctypes.c_void_p(16)
    for M, N, K, w in ((128, 128, 64, 0.0), (128, 128, 64, 11.0), (128, 128, 64, float("nan")),
                       (100, 128, 64, 0.01), (128, 128, 60, 0.01)):
        assert tpf_lib.tpf_selftest_gemm_wait(M, N, K, p, p, p, p, f, f, w, 1, None) == tpf.EINVAL
    assert tpf_lib.tpf_selftest_gemm_wait(128, 128, 64, None, p, p, p, f, f, 0.01, 1, None) == tpf.EINVAL
