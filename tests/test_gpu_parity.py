"""GPU parity: libtpf (through its C ABI) against the FP64 CPU oracle.

Tolerances (stated once here, used below):
  * FP64 path: max |V - V_oracle| <= 1e-9 pu (oracle iterated to 1e-13).
  * mixed path: max |V - V_oracle| <= 1e-8 pu.
  * iteration counts: FP64 path equal to the oracle's at the same tol, except columns whose
    deciding step lies within 1% of tol (rounding can move them by one); mixed path within +-1.
  * GEMM self-test: fp16 operands are exact in FP32, so only the FP32 summation order differs:
    |D - D_ref| <= 1e-4 * (1 + |D_ref|).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9
TOL_MIXED = 1e-8


def _case(nb, T, seed=1, t0=0):
    f = G.make_feeder(nb, seed)
    c = O.Case.from_feeder(f)
    S = G.load_tensor(f, T, seed, t0=t0)
    return f, c, S


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _iters_close(it_gpu, it_ref, delta_ref_prev, tol, slack):
    bad = np.flatnonzero(np.abs(it_gpu - it_ref) > slack)
    return bad


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (1024, 256, 1024)])
def test_gemm_selftest(cuda, M, N, K):
    import torch

    g = torch.Generator(device="cpu").manual_seed(M + N + K)
    A = [torch.rand((M, K), generator=g).mul(2).sub(1).half().cuda() for _ in range(2)]
    B = [torch.rand((N, K), generator=g).mul(2).sub(1).half().cuda() for _ in range(2)]
    Dr, Di = tpf.selftest_gemm(A[0], A[1], B[0], B[1])
    torch.cuda.synchronize()
    a = [x.double() for x in A]
    b = [x.double() for x in B]
    ref_r = (b[0] @ a[0].T - b[1] @ a[1].T)
    ref_i = (b[1] @ a[0].T + b[0] @ a[1].T)
    for got, ref in ((Dr, ref_r), (Di, ref_i)):
        err = (got.double() - ref).abs() / (1 + ref.abs())
        assert err.max().item() <= 1e-4, f"max scaled error {err.max().item()}"


def test_gemm_bounded_wait_expires_cleanly(cuda):
    """Failure detection without a fault: the GEMM's copy producer withholds its loads, so the MMA
    and epilogue waits (limited to 20 ms here) run out.  The kernel flags the error, drains its own
    work, frees its tensor memory and returns: the call reports ETIMEOUT within a second, and the
    same process then computes a correct product and a solve that matches the oracle."""
    import time

    import torch

    g = torch.Generator(device="cpu").manual_seed(7)
    M, N, K = 256, 384, 192
    A = [torch.rand((M, K), generator=g).mul(2).sub(1).half().cuda() for _ in range(2)]
    B = [torch.rand((N, K), generator=g).mul(2).sub(1).half().cuda() for _ in range(2)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, _, st = tpf.selftest_gemm(A[0], A[1], B[0], B[1], wait_s=0.02, withhold_loads=True, check=False)
    dt = time.perf_counter() - t0
    assert st == tpf.ETIMEOUT, tpf.strerror(st)
    assert dt < 1.0, f"the expired waits took {dt:.2f} s to return"
    # The context is intact: a product with the same short limit but real loads, then a solve.
    Dr, Di, st = tpf.selftest_gemm(A[0], A[1], B[0], B[1], wait_s=1.0, check=False)
    assert st == tpf.OK
    a = [x.double() for x in A]
    b = [x.double() for x in B]
    ref_r = b[0] @ a[0].T - b[1] @ a[1].T
    assert ((Dr.double() - ref_r).abs() / (1 + ref_r.abs())).max().item() <= 1e-4
    f, c, S = _case(34, 100)
    _check(f, c, S, "mixed", TOL_MIXED, 1)


def _check(f, c, S, precision, tol_v, it_slack, tol=1e-10, **kw):
    Vo, _, _ = c.solve(S, tol=1e-13)
    _, it_ref, d_ref = c.solve(S, tol=tol)
    fd = tpf.Feeder.from_inputs(f)
    V, it, mm, st = fd.solve(_dev(S), precision=precision, tol=tol, **kw)
    assert st == tpf.OK
    V = V.cpu().numpy()
    it = it.cpu().numpy()
    mm = mm.cpu().numpy()
    err = np.abs(V - Vo).max()
    assert err <= tol_v, f"max |V - V_oracle| = {err:.3e}"
    assert (it > 0).all()
    bad = np.flatnonzero(np.abs(it - it_ref) > it_slack)
    assert bad.size == 0, f"iteration counts differ in {bad.size} columns, e.g. {it[bad[:5]]} vs {it_ref[bad[:5]]}"
    # Mismatch at the returned V agrees with the oracle's evaluation of the same V.
    mm_ref = c.mismatch(S, V)
    assert np.all(np.abs(mm - mm_ref) <= 1e-9 + 1e-3 * mm_ref)
    st_ = fd.stats()
    assert st_["converged"] == S.shape[0]
    fd.close()
    return err, it


@pytest.mark.parametrize("nb,T", [(34, 1440), (2, 7), (3, 1), (35, 129), (100, 200), (200, 300)])
def test_fp64_vs_oracle(cuda, nb, T):
    f, c, S = _case(nb, T)
    _check(f, c, S, "fp64", TOL_FP64, 0)


@pytest.mark.parametrize("nb,T", [(34, 1440), (2, 7), (3, 1), (35, 129), (100, 200), (200, 300), (400, 257)])
def test_mixed_vs_oracle(cuda, nb, T):
    f, c, S = _case(nb, T)
    _check(f, c, S, "mixed", TOL_MIXED, 1)


def test_mixed_peak_hours_1000(cuda):
    """1,000-bus feeder, evening peak columns (lowest voltages), ragged T."""
    f = G.make_feeder(1000, 1)
    c = O.Case.from_feeder(f)
    S = G.load_tensor(f, 4096, 1)[1080:1080 + 300]
    _check(f, c, S, "mixed", TOL_MIXED, 1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_empty_and_given_start(cuda, precision):
    import torch

    f, c, S = _case(34, 50)
    fd = tpf.Feeder.from_inputs(f)
    V, it, mm, st = fd.solve(_dev(S[:0]), precision=precision)
    assert st == tpf.OK and V.shape[0] == 0
    Vo, _, _ = c.solve(S, tol=1e-13)
    V0 = _dev(Vo)
    V, it, mm, st = fd.solve(_dev(S), V=V0.clone(), precision=precision, tol=1e-10)
    assert st == tpf.OK
    assert (it.cpu().numpy() == 1).all()  # the oracle's solution is already a fixed point
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-12


@pytest.mark.parametrize("method", ["dense", "sparse"])
def test_warm_start(cuda, method):
    """start='warm' reads V as an approximate V_0: from the oracle's solution perturbed by up to
    2e-3 pu it reaches the same tolerance in fewer sweeps than the flat start; from the exact
    solution it converges too (its low words are dropped, so after a few sweeps rather than one)."""
    f = G.make_feeder(1000, 1)
    c = O.Case.from_feeder(f)
    S = G.load_tensor(f, 4096, 1)[1080:1080 + 200]
    Vo, _, _ = c.solve(S, tol=1e-13)
    _, it_flat, _ = c.solve(S, tol=1e-10)
    rng = np.random.default_rng(3)
    Vp = Vo + 1e-3 * (rng.uniform(-1, 1, Vo.shape) + 1j * rng.uniform(-1, 1, Vo.shape))
    fd = tpf.Feeder.from_inputs(f)
    for V0, most in ((Vp, it_flat.mean() - 1.0), (Vo, 6)):
        V, it, mm, st = fd.solve(_dev(S), V=_dev(V0), precision="mixed", tol=1e-10, method=method, start="warm")
        assert st == tpf.OK
        assert np.abs(V.cpu().numpy() - Vo).max() <= TOL_MIXED
        assert it.cpu().numpy().mean() <= most
    # Host buffers take the same warm start.
    Vh, ith, _, st = fd.solve_host(S, V0=Vp.copy(), precision="mixed", tol=1e-10, method=method, start="warm")
    assert st == tpf.OK and np.abs(Vh - Vo).max() <= TOL_MIXED
    # FP64: warm is the given start.
    V, it, mm, st = fd.solve(_dev(S), V=_dev(Vo), precision="fp64", tol=1e-10, start="warm")
    assert st == tpf.OK and (it.cpu().numpy() == 1).all()
    with pytest.raises(tpf.TpfError):
        fd.solve(_dev(S), precision="mixed", method=method, start=7)
    fd.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_infeasible_and_nan_columns(cuda, precision):
    f, c, S = _case(34, 64)
    S = S.copy()
    S[3] *= 400.0  # far beyond the loadability of the feeder: no solution
    S[10, 5] = np.nan
    fd = tpf.Feeder.from_inputs(f)
    V, it, mm, st = fd.solve(_dev(S), precision=precision, max_iter=60)
    assert st == tpf.ENOCONV
    it = it.cpu().numpy()
    assert it[3] == -60 and it[10] == -60
    good = np.setdiff1d(np.arange(64), [3, 10])
    Vo, _, _ = c.solve(S[good], tol=1e-13)
    tol_v = TOL_FP64 if precision == "fp64" else TOL_MIXED
    assert np.abs(V.cpu().numpy()[good] - Vo).max() <= tol_v
    assert fd.stats()["converged"] == 62


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_host_buffers_match_device(cuda, precision):
    f, c, S = _case(100, 333)
    fd = tpf.Feeder.from_inputs(f)
    Vd, itd, mmd, _ = fd.solve(_dev(S), precision=precision)
    Vh, ith, mmh, st = fd.solve_host(S, precision=precision)
    assert st == tpf.OK
    assert np.array_equal(Vh, Vd.cpu().numpy())
    assert np.array_equal(ith, itd.cpu().numpy())


def test_chunked_host_solve_matches_device(cuda):
    """tpf_solve_host splits large T into chunks whose copies overlap the solve of other chunks."""
    import torch

    f = G.make_feeder(34, 1)
    T = 70001  # four chunks, ragged last one
    S = G.load_tensor(f, T, 3)
    fd = tpf.Feeder.from_inputs(f)
    Vd, itd, mmd, _ = fd.solve(_dev(S), precision="mixed")
    Sh = torch.from_numpy(S).pin_memory()
    out = (torch.empty((T, f.n_pq), dtype=torch.complex128).pin_memory(),
           torch.empty(T, dtype=torch.int32).pin_memory(), torch.empty(T, dtype=torch.float64).pin_memory())
    Vh, ith, mmh, st = fd.solve_host(Sh, precision="mixed", out=out)
    assert st == tpf.OK
    assert torch.equal(Vh, Vd.cpu()) and torch.equal(ith, itd.cpu()) and torch.equal(mmh, mmd.cpu())
    assert fd.stats()["converged"] == T
    fd.close()


def test_create_errors(cuda):
    with pytest.raises(tpf.TpfError) as e:
        tpf.Feeder(3, [0, 0], [1, 1], [0.01 + 0.01j, 0.02 + 0.01j])  # bus 2 not connected
    assert e.value.status == tpf.ESINGULAR
    with pytest.raises(tpf.TpfError) as e:
        tpf.Feeder(3, [0, 1], [1, 5], [0.01 + 0.01j, 0.02 + 0.01j])
    assert e.value.status == tpf.EINVAL


# --- sparse formulation (Algorithm 2, Eq. 13-14): tree substitution instead of the dense K ---

@pytest.mark.parametrize("nb,T", [(34, 1440), (2, 7), (3, 1), (35, 129), (100, 200), (400, 257)])
def test_sparse_vs_oracle(cuda, nb, T):
    f, c, S = _case(nb, T)
    _check(f, c, S, "mixed", TOL_MIXED, 1, method="sparse")


def test_sparse_peak_hours_1000(cuda):
    f = G.make_feeder(1000, 1)
    c = O.Case.from_feeder(f)
    S = G.load_tensor(f, 4096, 1)[1080:1080 + 300]
    err, _ = _check(f, c, S, "mixed", TOL_MIXED, 1, method="sparse")
    # The anchored sweeps reach the FP64 fixed point to about 1e-11 pu.  Losing the low word of S
    # or V in the FP64 <-> FP32-pair conversions leaves errors near 1e-9..1e-8 pu, inside the bar
    # above: this bound catches that.
    assert err <= 1e-10, f"max |V - V_oracle| = {err:.3e}"


def test_sparse_chain_feeder(cuda):
    """A 150-bus chain (149 depth levels of one bus each: the longest level walk per sweep), with
    the slack at the far end and a shuffled demand-bus order."""
    import torch

    nb = 150
    rng = np.random.default_rng(11)
    frm, to = np.arange(nb - 1, 0, -1), np.arange(nb - 2, -1, -1)  # slack = bus 149
    z = (4e-4 + 3e-4j) * rng.uniform(0.5, 1.5, nb - 1)
    pq = rng.permutation(nb - 1)
    c = O.Case(nb, frm, to, z, slack=nb - 1, vs=1.02 + 0.01j, pq=pq)
    S = (rng.uniform(1e-3, 6e-3, (130, nb - 1)) * (1 + 0.3j)).astype(np.complex128)
    Vo, _, _ = c.solve(S, tol=1e-13)
    _, it_ref, _ = c.solve(S, tol=1e-10)
    fd = tpf.Feeder(nb, frm, to, z, slack=nb - 1, v0=1.02 + 0.01j, pq_bus=pq)
    V, it, mm, st = fd.solve(_dev(S), precision="mixed", tol=1e-10, method="sparse")
    assert st == tpf.OK
    assert np.abs(V.cpu().numpy() - Vo).max() <= TOL_MIXED
    assert np.abs(it.cpu().numpy() - it_ref).max() <= 1
    fd.close()


def test_sparse_largest_feeder_vs_newton(cuda):
    """3,500 buses (the shared-memory limit of one column is 3,657 demand buses): a few columns
    against the sparse Newton-Raphson solution, which does not need the dense K."""
    f = G.make_feeder(3500, 2)
    S = G.load_tensor(f, 4096, 2)[[0, 700, 1100, 4095]]
    Ysp = O.ybus(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    fd = tpf.Feeder.from_inputs(f)
    V, it, mm, st = fd.solve(_dev(S), precision="mixed", tol=1e-10, method="sparse")
    assert st == tpf.OK
    V = V.cpu().numpy()
    for k in range(S.shape[0]):
        # Power mismatch 1e-11 pu is at the rounding floor of a 3,500-bus sum; the voltage error it
        # leaves is below 1e-11 * max|K_ij| (about 1e-12 pu here).
        Vn, _, ok = O.nr_solve(Ysp, f.slack, f.v0, f.pq_bus, S[k], tol=1e-11)
        assert ok
        assert np.abs(V[k] - Vn).max() <= TOL_MIXED
    fd.close()


def test_sparse_matches_dense_iterates(cuda):
    """Same iterates as the dense form: equal iteration counts up to rounding (+-1) and the same V."""
    f, c, S = _case(200, 600, seed=3)
    fd = tpf.Feeder.from_inputs(f)
    Vd, itd, _, _ = fd.solve(_dev(S), precision="mixed")
    Vs, its, _, st = fd.solve(_dev(S), precision="mixed", method="sparse")
    assert st == tpf.OK
    assert np.abs(itd.cpu().numpy() - its.cpu().numpy()).max() <= 1
    assert np.abs(Vd.cpu().numpy() - Vs.cpu().numpy()).max() <= 2 * TOL_MIXED
    fd.close()


def test_sparse_empty_given_and_failures(cuda):
    f, c, S = _case(34, 64)
    fd = tpf.Feeder.from_inputs(f)
    V, it, mm, st = fd.solve(_dev(S[:0]), precision="mixed", method="sparse")
    assert st == tpf.OK and V.shape[0] == 0
    Vo, _, _ = c.solve(S, tol=1e-13)
    V, it, mm, st = fd.solve(_dev(S), V=_dev(Vo), precision="mixed", tol=1e-10, method="sparse")
    assert st == tpf.OK
    assert (it.cpu().numpy() == 1).all()
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-12
    S2 = S.copy()
    S2[3] *= 400.0
    S2[10, 5] = np.nan
    V, it, mm, st = fd.solve(_dev(S2), precision="mixed", max_iter=60, method="sparse")
    assert st == tpf.ENOCONV
    it = it.cpu().numpy()
    assert it[3] == -60 and it[10] == -60
    good = np.setdiff1d(np.arange(64), [3, 10])
    assert np.abs(V.cpu().numpy()[good] - Vo[good]).max() <= TOL_MIXED
    assert fd.stats()["converged"] == 62
    # Host buffers through the same method.
    Vh, ith, mmh, st = fd.solve_host(S, precision="mixed", method="sparse")
    Vd, itd, mmd, _ = fd.solve(_dev(S), precision="mixed", method="sparse")
    assert st == tpf.OK and np.array_equal(Vh, Vd.cpu().numpy()) and np.array_equal(ith, itd.cpu().numpy())
    fd.close()


def test_sparse_unsupported(cuda):
    """The sparse formulation takes radial feeders only, in either precision."""
    mesh = tpf.Feeder(3, [0, 1, 0], [1, 2, 2], [0.01 + 0.01j, 0.02 + 0.01j, 0.03 + 0.02j])
    for precision in ("mixed", "fp64"):
        _, _, _, st = mesh.solve(_dev(np.full((4, 2), 0.01 + 0.005j)), precision=precision, method="sparse",
                                 check=False)
        assert st == tpf.EUNSUPPORTED
    mesh.close()


def test_autotune_keeps_results(cuda):
    """tpf_autotune picks a launch shape on a sample; solves afterwards still match the oracle,
    also with ZIP coefficients laid out again for the new shape."""
    f, c, S = _case(300, 1500, seed=6)
    fd = tpf.Feeder.from_inputs(f)
    b = fd.autotune(_dev(S[:1024]))
    assert b in (2, 4, 8)
    Vo, _, _ = c.solve(S, tol=1e-13)
    V, it, mm, st = fd.solve(_dev(S), method="sparse")
    assert st == tpf.OK and np.abs(V.cpu().numpy() - Vo).max() <= TOL_MIXED
    a = np.random.default_rng(1).dirichlet([2, 1, 1], f.n_pq).T.copy()
    fd.set_zip(a)
    assert fd.autotune(_dev(S[:512])) in (2, 4, 8)
    Vz, _, _ = c.solve_zip(S[:200], a, tol=1e-13)
    V, _, _, st = fd.solve(_dev(S[:200]), method="sparse")
    assert st == tpf.OK and np.abs(V.cpu().numpy() - Vz).max() <= TOL_MIXED
    fd.close()


@pytest.mark.parametrize("nb", [33, 97, 161, 290, 481, 700, 1021, 1500, 2100, 2900, 4097])
def test_sparse_block_shapes(cuda, nb):
    """Feeders whose demand-bus counts land on block sizes of every kind: whole warps that are not
    powers of two (runtime-size kernels), the compile-time power-of-two sizes, 8 buses per thread
    above 2,048, and the 4,096-bus limit.  A few peak columns against the oracle (FPI up to 1,500
    buses, sparse Newton-Raphson beyond)."""
    f = G.make_feeder(nb, 3)
    S = G.load_tensor(f, 4096, 3)[[1080, 1140, 2400]]
    fd = tpf.Feeder.from_inputs(f)
    V, it, mm, st = fd.solve(_dev(S), precision="mixed", tol=1e-10, method="sparse")
    assert st == tpf.OK
    V = V.cpu().numpy()
    if nb <= 1500:
        Vo, _, _ = O.Case.from_feeder(f).solve(S, tol=1e-13)
        assert np.abs(V - Vo).max() <= TOL_MIXED
    else:
        Ysp = O.ybus(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
        for k in range(S.shape[0]):
            Vn, _, ok = O.nr_solve(Ysp, f.slack, f.v0, f.pq_bus, S[k], tol=1e-11)
            assert ok
            assert np.abs(V[k] - Vn).max() <= TOL_MIXED
    fd.close()


def test_sparse_large_feeders_beyond_4096(cuda):
    """16 buses per thread with device scratch and chunked launches (4,097 to 6,144 demand buses):
    a 5,000-bus feeder against sparse Newton-Raphson, over more columns than one launch takes
    (the repeated columns agree bit for bit); ZIP loads on it against the oracle's ZIP power
    balance; the 6,145-bus limit and one bus past it."""
    import torch

    f = G.make_feeder(5000, 2)
    S3 = G.load_tensor(f, 4096, 2)[[0, 1100, 4095]]
    S = np.concatenate([S3, np.repeat(S3[1:2], 9000, axis=0)])  # 9,003 columns: two launches
    fd = tpf.Feeder.from_inputs(f)
    V, it, mm, st = fd.solve(_dev(S), precision="mixed", tol=1e-10, method="sparse")
    assert st == tpf.OK
    assert fd.stats()["kernel_launches"] == 2
    assert torch.equal(V[1], V[-1]) and torch.equal(V[1], V[8500])
    Vh = V[:3].cpu().numpy()
    Y = O.ybus(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    for k in range(3):
        Vn, _, ok = O.nr_solve(Y, f.slack, f.v0, f.pq_bus, S3[k], tol=1e-11)
        assert ok
        assert np.abs(Vh[k] - Vn).max() <= TOL_MIXED
    # In a batch with a small feeder: the large one is solved on its own, with the same results.
    fs = G.make_feeder(60, 4)
    fds = tpf.Feeder.from_inputs(fs)
    Ss = G.load_tensor(fs, 40, 4)
    Vb, itb, _, conv, _, st = tpf.solve_batch([fd, fds], [_dev(S3), _dev(Ss)])
    assert st == tpf.OK and list(conv) == [3, 40]
    assert np.array_equal(Vb[0].cpu().numpy(), Vh)
    fds.close()
    alpha = np.random.default_rng(5).dirichlet([2, 1, 1], fd.n_pq).T.copy()
    fd.set_zip(alpha)
    Vz, _, _, st = fd.solve(_dev(S3), precision="mixed", tol=1e-10, method="sparse")
    assert st == tpf.OK
    mz = O.mismatch_zip(Y, f.slack, f.v0, f.pq_bus, alpha, S3, Vz.cpu().numpy())
    assert mz.max() <= 1e-8, mz
    fd.close()
    for nb, ok_ in ((6145, True), (6146, False)):
        f2 = G.make_feeder(nb, 4)
        fd2 = tpf.Feeder.from_inputs(f2)
        S2 = G.load_tensor(f2, 4096, 4)[[1100]]
        V2, _, _, st = fd2.solve(_dev(S2), precision="mixed", tol=1e-10, method="sparse", check=False)
        if ok_:
            assert st == tpf.OK
            Vn, _, ok = O.nr_solve(O.ybus(f2.n_bus, f2.from_bus, f2.to_bus, f2.z_pu), f2.slack, f2.v0, f2.pq_bus,
                                   S2[0], tol=1e-11)
            assert ok and np.abs(V2.cpu().numpy()[0] - Vn).max() <= TOL_MIXED
        else:
            assert st == tpf.EUNSUPPORTED
        fd2.close()
