"""GPU parity at the headline's full size: the 1,000-bus feeder over the one-minute year (525,600
columns), solved in the launch configuration bench.py times (sparse formulation, block shape
autotuned on the first 16,384 columns; the flat start, then the learned start), with sampled
columns checked one by one against the FP64 oracle and properties that hold at any size checked on
every column.

Bars: max |V - V_oracle| <= 1e-8 pu on the sampled columns (the mixed path's bar; the oracle
iterated to 1e-13); the flat start's sweep counts within +-1 of the oracle's on those columns;
every column converged (its final step <= tol, its count in [1, max_iter]); the reported mismatch
within 1e-9 + 1e-3 of the oracle's mismatch of the same V on the samples, finite everywhere; the
learned start's mean sweep count below the flat start's.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

pytestmark = pytest.mark.gpu

T_YEAR = 525_600
TOL = 1e-10
THREADS = os.cpu_count() or 1


def _samples(rng):
    """256 columns evenly spaced over the year, and the 64 minutes around one day's evening peak."""
    even = np.linspace(0, T_YEAR - 1, 256).astype(np.int64)
    day = int(rng.integers(0, 365))
    peak = day * 1440 + 1110 + np.arange(64)
    return np.unique(np.concatenate([even, peak]))


def _check_columns(c, S_dev, V, it, mm, idx, iters_exact):
    S = S_dev[idx].cpu().numpy()
    Vg = V[idx].cpu().numpy()
    Vo, ito, _ = c.solve(S, tol=1e-13, threads=THREADS)
    err = float(np.abs(Vg - Vo).max())
    assert err <= 1e-8, f"max |V - V_oracle| = {err:.3e} on {len(idx)} sampled columns"
    mm_g = mm[idx].cpu().numpy()
    mm_ref = c.mismatch(S, Vg)
    assert np.all(np.abs(mm_g - mm_ref) <= 1e-9 + 1e-3 * mm_ref)
    if iters_exact:
        _, ito_t, _ = c.solve(S, tol=TOL, threads=THREADS)
        assert np.all(np.abs(it[idx].cpu().numpy() - ito_t) <= 1)
    return err


def _check_all(fd, V, it, mm, T):
    import torch

    assert fd.stats()["converged"] == T
    itc = it.cpu().numpy()
    assert itc.min() >= 1 and itc.max() <= 100
    assert bool(torch.isfinite(mm).all()) and bool(torch.isfinite(torch.view_as_real(V)).all())
    mag = V.abs()
    assert float(mag.min()) > 0.7 and float(mag.max()) < 1.1


def test_headline_year_flat_and_learned(cuda):
    import torch

    rng = np.random.default_rng(2026)
    f = G.make_feeder(1000, 1)
    c = O.Case.from_feeder(f)
    fd = tpf.Feeder.from_inputs(f)
    dev = torch.device("cuda:0")
    S = G.load_tensor_device(f, T_YEAR, 1, dev)
    V = torch.empty_like(S)
    it = torch.empty(T_YEAR, dtype=torch.int32, device=dev)
    mm = torch.empty(T_YEAR, dtype=torch.float64, device=dev)
    fd.autotune(S[:16384], tol=TOL)
    idx = _samples(rng)

    # Flat start: one launch over the year.
    _, _, _, st = fd.solve(S, V, it, mm, precision="mixed", tol=TOL, start="flat", method="sparse")
    assert st == tpf.OK
    _check_all(fd, V, it, mm, T_YEAR)
    _check_columns(c, S, V, it, mm, idx, iters_exact=True)
    flat_sweeps = it.float().mean().item()

    # Learned start: a network trained briefly on 16,384 other columns, then the fused prediction
    # and the warm solve over the year.
    S_tr = G.load_tensor_device(f, 16384, 101, dev)
    V_tr, _, _, st = fd.solve(S_tr, precision="mixed", tol=TOL, method="sparse")
    assert st == tpf.OK
    net = tpf.LearnedStart(f.n_pq, hidden=256, hidden_layers=3, max_batch=1024, seed=1)
    net.fit_normalization(S_tr, V_tr)
    for epoch in range(8):
        for k in range(0, 16384, 1024):
            net.train_step(S_tr[k:k + 1024], V_tr[k:k + 1024], lr=1e-3, want_loss=False)
    del S_tr, V_tr
    V.zero_()
    _, _, _, fallback, st = fd.solve_learned(net, S, V, it, mm, tol=TOL)
    assert st == tpf.OK and 0 <= fallback < T_YEAR
    _check_all(fd, V, it, mm, T_YEAR)
    _check_columns(c, S, V, it, mm, idx, iters_exact=False)
    assert it.float().mean().item() < flat_sweeps - 0.5
    net.close()
    fd.close()
    del S, V
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_learned_start_config5_year(cuda):
    """Config 5 at full size: the 200-bus feeder, the network trained on 100,000 library-solved
    columns of another load draw, evaluated on the unseen one-minute year through
    tpf_solve_learned."""
    import torch

    rng = np.random.default_rng(5)
    f = G.make_feeder(200, 1)
    c = O.Case.from_feeder(f)
    fd = tpf.Feeder.from_inputs(f)
    dev = torch.device("cuda:0")
    S_tr = G.load_tensor_device(f, 100_000, 201, dev)
    V_tr, _, _, st = fd.solve(S_tr, precision="mixed", tol=TOL, method="sparse")
    assert st == tpf.OK
    net = tpf.LearnedStart(f.n_pq, hidden=256, hidden_layers=3, max_batch=1024, seed=1)
    net.fit_normalization(S_tr, V_tr)
    for epoch in range(10):
        for k in range(0, 99_328, 1024):
            net.train_step(S_tr[k:k + 1024], V_tr[k:k + 1024], lr=1e-3, want_loss=False)
    del S_tr, V_tr
    S = G.load_tensor_device(f, T_YEAR, 200, dev)
    fd.autotune(S[:16384], tol=TOL)
    V, it, mm, st = fd.solve(S, precision="mixed", tol=TOL, start="flat", method="sparse")
    assert st == tpf.OK
    flat_sweeps = it.float().mean().item()
    V, it, mm, fallback, st = fd.solve_learned(net, S, V, it, mm, tol=TOL)
    assert st == tpf.OK and 0 <= fallback <= T_YEAR // 100
    _check_all(fd, V, it, mm, T_YEAR)
    _check_columns(c, S, V, it, mm, _samples(rng), iters_exact=False)
    assert it.float().mean().item() < flat_sweeps - 1.0
    net.close()
    fd.close()
    torch.cuda.synchronize()


def test_scenario_tensor_config3(cuda):
    """Config 3 at full size: the 500-bus feeder and the [200 scenarios x 8,760 hours] complex64 load
    tensor in one tpf_solve_ex call with the voltage-band statistics (V written in complex128).
    Sampled columns: V against the oracle, and the per-column statistics against the oracle's V
    (a bus within 1e-7 pu of a band edge may fall either way); all columns: converged, and the
    per-bus band counts summing to the per-column ones."""
    import torch

    rng = np.random.default_rng(3)
    f = G.make_feeder(500, 1, peak_factor=1.8)
    c = O.Case.from_feeder(f)
    fd = tpf.Feeder.from_inputs(f)
    dev = torch.device("cuda:0")
    S = G.scenario_tensor_device(f, 200, 8760, 1, dev)
    T = 200 * 8760
    band = (0.95, 1.05)
    r = fd.solve_tensor(S, v_complex64=False, start="flat", v_band=band, tol=TOL)
    assert r["status"] == tpf.OK
    it = r["iters"].reshape(T)
    assert int((it > 0).sum()) == T and int(it.max()) <= 100
    viol = r["viol"].reshape(T)
    assert int(viol.sum()) == int(r["bus_under"].sum()) + int(r["bus_over"].sum())
    idx = np.unique(np.concatenate([np.linspace(0, T - 1, 256).astype(np.int64), rng.integers(0, T, 64)]))
    Sf = S.reshape(T, -1)[torch.from_numpy(idx).to(dev)]
    Vo, _, _ = c.solve(Sf.cpu().numpy().astype(np.complex128), tol=1e-13, threads=THREADS)
    Vg = r["V"].reshape(T, -1)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    assert np.abs(Vg - Vo).max() <= 1e-8
    mag = np.abs(Vo)
    vmin = r["vmin"].reshape(T)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    vmax = r["vmax"].reshape(T)[torch.from_numpy(idx).to(dev)].cpu().numpy()
    assert np.all(np.abs(vmin - mag.min(axis=1)) <= 1e-6) and np.all(np.abs(vmax - mag.max(axis=1)) <= 1e-6)
    out = (mag < band[0]) | (mag > band[1])
    edge = (np.abs(mag - band[0]) <= 1e-7) | (np.abs(mag - band[1]) <= 1e-7)
    vg = viol[torch.from_numpy(idx).to(dev)].cpu().numpy()
    lo, hi = (out & ~edge).sum(axis=1), (out | edge).sum(axis=1)
    assert np.all((vg >= lo) & (vg <= hi))
    fd.close()
    del S, r
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def test_feeder_batch_config4(cuda):
    """Config 4 at full size: 4,096 feeders (bus counts log-uniform in [20, 2,000], T in
    {96, 288, 1,440}) in one tpf_solve_batch call.  Every column of every feeder converged; 4
    columns of each of 48 feeders spread over the bus counts (the largest included) against the
    oracle; the CUDA-graph replay of the prepared batch gives the same V bit for bit."""
    import torch

    dev = torch.device("cuda:0")
    specs = G.batch_specs(4096)
    feeders = [G.make_feeder(nb, sd) for nb, _, sd in specs]
    fds = [tpf.Feeder.from_inputs(f) for f in feeders]
    S = [G.load_tensor_device(f, T, sd, dev, step_minutes=G.step_minutes_for(T))
         for f, (_, T, sd) in zip(feeders, specs)]
    V, it, mm, conv, stats, st = tpf.solve_batch(fds, S, start="flat", tol=TOL)
    assert st == tpf.OK
    Ts = np.array([T for _, T, _ in specs])
    assert np.array_equal(conv, Ts)
    order = np.argsort([f.n_bus for f in feeders], kind="stable")
    pick = np.unique(np.concatenate([order[np.linspace(0, len(order) - 1, 47).astype(int)], order[-1:]]))
    worst = 0.0
    for k in pick:
        cc = torch.linspace(0, S[k].shape[0] - 1, 4, device=dev).long()
        Vo, _, _ = O.Case.from_feeder(feeders[k]).solve(S[k][cc].cpu().numpy(), tol=1e-13, threads=THREADS)
        worst = max(worst, float(np.abs(V[k][cc].cpu().numpy() - Vo).max()))
    assert worst <= 1e-8, worst
    bg = tpf.BatchGraph(fds, S, start="flat", tol=TOL)
    bg.launch()
    gconv, _, gst = bg.wait()
    assert gst == tpf.OK and np.array_equal(gconv, Ts)
    for k in pick:
        assert torch.equal(bg.V[k], V[k]), k
    bg.close()
    for fd in fds:
        fd.close()
    torch.cuda.synchronize()
