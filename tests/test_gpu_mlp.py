"""The learned warm start on the GPU: BF16 tensor-core gradients against the FP64 reference, training,
and what the trained network saves the fixed-point iteration.

Tolerances: the GPU runs every product in BF16 (8-bit significand) with FP32 accumulation, so its
gradient is compared with the FP64 reference (same weights, same normalised batch) by relative L2
error <= 2e-2 and cosine similarity >= 0.999; the loss within 2 %.
"""
import numpy as np
import pytest

from oracle import mlp as OM
from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _features(S):
    return np.concatenate([S.real, S.imag], axis=1)


def _targets(V):
    return np.concatenate([V.real - 1.0, V.imag], axis=1)


def _zscore_stats(A):
    mu = A.mean(axis=0)
    sd = A.std(axis=0)
    return mu, sd


def _norm(A, mu, sd):
    return np.where(sd > 0, (A - mu) / np.where(sd > 0, sd, 1.0), 0.0)


@pytest.fixture(scope="module")
def feeder200():
    f = G.make_feeder(200, 5)
    c = O.Case.from_feeder(f)
    return f, c


def test_gradients_match_the_fp64_reference(cuda, feeder200):
    f, c = feeder200
    S = G.load_tensor(f, 4096, 5)[::32][:128]  # 128 columns spread over the day
    V, it, _ = c.solve(S, tol=1e-12)
    assert (it > 0).all()
    net = tpf.LearnedStart(f.n_pq, hidden=256, hidden_layers=3, max_batch=128, seed=3)
    Sd, Vd = _dev(S), _dev(V)
    net.fit_normalization(Sd, Vd)
    X, Y = _features(S), _targets(V)
    xm, xs = _zscore_stats(X)
    ym, ys = _zscore_stats(Y)
    gm, gs, hm, hs = net.normalization()
    assert np.allclose(gm, xm, rtol=1e-5, atol=1e-9) and np.allclose(gs, xs, rtol=1e-4, atol=1e-9)
    assert np.allclose(hm, ym, rtol=1e-5, atol=1e-9) and np.allclose(hs, ys, rtol=1e-4, atol=1e-9)
    rng = np.random.default_rng(11)
    sizes = net.sizes
    Ws = [rng.uniform(-1, 1, (sizes[i + 1], sizes[i])) * np.sqrt(6.0 / (sizes[i] + sizes[i + 1]))
          for i in range(len(sizes) - 1)]
    bs = [rng.normal(0, 0.05, sizes[i + 1]) for i in range(len(sizes) - 1)]
    flat = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)]).astype(np.float32)
    net.set_params(flat)
    assert np.array_equal(net.params(), flat)
    loss_gpu, g_gpu = net.gradients(Sd, Vd)
    ref = OM.MLP([w.astype(np.float32).astype(np.float64) for w in Ws], [b.astype(np.float32) for b in bs])
    loss_ref, gW, gb = ref.gradients(_norm(X, xm, xs), _norm(Y, ym, ys))
    g_ref = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(gW, gb)])
    assert loss_gpu == pytest.approx(loss_ref, rel=2e-2)
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    cos = float(g_gpu @ g_ref / (np.linalg.norm(g_gpu) * np.linalg.norm(g_ref)))
    assert rel <= 2e-2, rel
    assert cos >= 0.999, cos
    net.close()


def test_prediction_matches_the_fp64_reference(cuda, feeder200):
    """Inference (bias and GELU in the GEMM epilogue, FP32 output) against the FP64 network on the
    same weights: the normalised outputs agree to BF16 accuracy, and V_0 is their denormalisation."""
    f, c = feeder200
    S = G.load_tensor(f, 4096, 7)[::16][:256]
    V, it, _ = c.solve(S, tol=1e-12)
    net = tpf.LearnedStart(f.n_pq, hidden=256, hidden_layers=3, max_batch=128, seed=3)
    Sd, Vd = _dev(S), _dev(V)
    net.fit_normalization(Sd, Vd)
    xm, xs, ym, ys = (np.asarray(a, dtype=np.float64) for a in net.normalization())
    rng = np.random.default_rng(12)
    sizes = net.sizes
    Ws = [rng.uniform(-1, 1, (sizes[i + 1], sizes[i])) * np.sqrt(6.0 / (sizes[i] + sizes[i + 1]))
          for i in range(len(sizes) - 1)]
    bs = [rng.normal(0, 0.05, sizes[i + 1]) for i in range(len(sizes) - 1)]
    Ws[-1] *= 0.05  # small outputs: every prediction stays inside the |V| guard
    flat = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)]).astype(np.float32)
    net.set_params(flat)
    V0, fallback = net.predict(Sd)  # 256 columns: two batches of 128
    assert fallback == 0
    ref = OM.MLP([w.astype(np.float32).astype(np.float64) for w in Ws], [b.astype(np.float32) for b in bs])
    y_ref, _ = ref.forward(_norm(_features(S), xm, xs))
    V0 = V0.cpu().numpy()
    ok = ys > 0  # outputs with spread (all of them here)
    y_gpu = (np.concatenate([V0.real - 1.0, V0.imag], axis=1)[:, ok] - ym[ok]) / ys[ok]
    y_ref = y_ref[:, ok]
    rel = np.linalg.norm(y_gpu - y_ref) / np.linalg.norm(y_ref)
    cos = float((y_gpu * y_ref).sum() / (np.linalg.norm(y_gpu) * np.linalg.norm(y_ref)))
    assert rel <= 2e-2, rel
    assert cos >= 0.999, cos
    net.close()


def test_training_reduces_the_loss(cuda, feeder200):
    f, c = feeder200
    S = G.load_tensor(f, 4096, 6)
    V, it, _ = c.solve(S, tol=1e-12)
    Sd, Vd = _dev(S), _dev(V)
    net = tpf.LearnedStart(f.n_pq, max_batch=1024, seed=4)
    net.fit_normalization(Sd, Vd)
    first = None
    last = []
    for step in range(400):
        k = (step % 4) * 1024
        loss = net.train_step(Sd[k:k + 1024], Vd[k:k + 1024], lr=1e-3)
        first = loss if first is None else first
        last.append(loss)
    assert np.isfinite(last).all()
    assert np.mean(last[-8:]) < 0.02 * first
    net.close()


def test_learned_start_saves_sweeps(cuda, feeder200):
    """Trained on GPU-solved columns of one load draw, evaluated on unseen columns of another."""
    import torch

    f, c = feeder200
    fd = tpf.Feeder.from_inputs(f)
    S_tr = _dev(G.load_tensor(f, 16384, 21))
    V_tr, _, _, st = fd.solve(S_tr, precision="mixed", tol=1e-10)
    assert st == tpf.OK
    net = tpf.LearnedStart(f.n_pq, max_batch=1024, seed=5)
    net.fit_normalization(S_tr, V_tr)
    for epoch in range(25):
        for k in range(0, 16384, 1024):
            net.train_step(S_tr[k:k + 1024], V_tr[k:k + 1024], lr=1e-3, want_loss=False)
    S_np = G.load_tensor(f, 4096, 22)
    S_ev = _dev(S_np)
    V0, fallback = net.predict(S_ev)
    assert fallback == 0
    Vo, _, _ = c.solve(S_np, tol=1e-13)
    start_err = np.abs(V0.cpu().numpy() - Vo).max()
    flat_err = np.abs(1.0 - Vo).max()
    assert start_err < 0.1 * flat_err, (start_err, flat_err)
    V_l, it_l, _, st_l = fd.solve(S_ev, V=V0.clone(), precision="mixed", tol=1e-10)
    V_f, it_f, _, st_f = fd.solve(S_ev, precision="mixed", tol=1e-10)
    assert st_l == tpf.OK and st_f == tpf.OK
    assert np.abs(V_l.cpu().numpy() - Vo).max() <= 1e-8
    assert np.abs(V_f.cpu().numpy() - Vo).max() <= 1e-8
    assert it_l.float().mean().item() < it_f.float().mean().item() - 1.0
    # The sparse formulation from the prediction as a warm start (FP32 sweeps first, one anchor).
    V_w, it_w, _, st_w = fd.solve(S_ev, V=V0.clone(), precision="mixed", tol=1e-10, method="sparse", start="warm")
    V_s, it_s, _, st_s = fd.solve(S_ev, precision="mixed", tol=1e-10, method="sparse")
    assert st_w == tpf.OK and st_s == tpf.OK
    assert np.abs(V_w.cpu().numpy() - Vo).max() <= 1e-8
    assert it_w.float().mean().item() < it_s.float().mean().item() - 1.0
    net.close()
    fd.close()
    torch.cuda.synchronize()


def test_learned_start_in_the_batch_path(cuda):
    """One network per feeder (a family of feeders of different sizes), each trained on its own
    library-solved columns; their predictions start one tpf_solve_batch call (warm start).  The
    batch reaches the oracle's solutions in fewer sweeps than from the flat start."""
    import torch

    specs = [(60, 31), (120, 32), (200, 33)]
    feeders = [G.make_feeder(nb, sd) for nb, sd in specs]
    fds = [tpf.Feeder.from_inputs(f) for f in feeders]
    S_ev, V0s, nets = [], [], []
    for f, fd, (_, sd) in zip(feeders, fds, specs):
        S_tr = _dev(G.load_tensor(f, 8192, sd))
        V_tr, _, _, st = fd.solve(S_tr, precision="mixed", tol=1e-10, method="sparse")
        assert st == tpf.OK
        net = tpf.LearnedStart(f.n_pq, max_batch=1024, seed=sd)
        net.fit_normalization(S_tr, V_tr)
        for epoch in range(20):
            for k in range(0, 8192, 1024):
                net.train_step(S_tr[k:k + 1024], V_tr[k:k + 1024], lr=1e-3, want_loss=False)
        S = _dev(G.load_tensor(f, 4096, sd + 100)[::8])
        V0, fallback = net.predict(S)
        assert fallback == 0
        S_ev.append(S)
        V0s.append(V0)
        nets.append(net)
    Vw, itw, _, conv, _, st = tpf.solve_batch(fds, S_ev, V=[v.clone() for v in V0s], start="warm")
    assert st == tpf.OK and list(conv) == [s.shape[0] for s in S_ev]
    Vf, itf, _, _, _, st = tpf.solve_batch(fds, S_ev)
    assert st == tpf.OK
    for f, S, V, it_w, it_f in zip(feeders, S_ev, Vw, itw, itf):
        Vo, _, _ = O.Case.from_feeder(f).solve(S.cpu().numpy(), tol=1e-13)
        assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-8
        # (a 60-bus feeder needs only about 5 sweeps from the flat start, so the saving is smaller)
        assert it_w.float().mean().item() < it_f.float().mean().item() - 0.5
    for net in nets:
        net.close()
    for fd in fds:
        fd.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("hidden,layers,T", [(256, 3, 1000), (128, 1, 300), (256, 2, 129)])
def test_fused_prediction_matches_the_fp64_reference(cuda, feeder200, hidden, layers, T):
    """The fused inference kernel (all layers of a 128-column tile in one tcgen05 kernel, hidden
    activations in shared memory) against the FP64 network on the same weights, over several
    tiles with a ragged last one; then outputs pushed outside the |V| guard send every column to
    the flat start."""
    f, c = feeder200
    S = G.load_tensor(f, 4096, 9)[:T]
    V, _, _ = c.solve(S, tol=1e-12)
    net = tpf.LearnedStart(f.n_pq, hidden=hidden, hidden_layers=layers, max_batch=128, seed=3)
    Sd, Vd = _dev(S), _dev(V)
    net.fit_normalization(Sd, Vd)
    xm, xs, ym, ys = (np.asarray(a, dtype=np.float64) for a in net.normalization())
    rng = np.random.default_rng(hidden + layers)
    sizes = net.sizes
    Ws = [rng.uniform(-1, 1, (sizes[i + 1], sizes[i])) * np.sqrt(6.0 / (sizes[i] + sizes[i + 1]))
          for i in range(len(sizes) - 1)]
    bs = [rng.normal(0, 0.05, sizes[i + 1]) for i in range(len(sizes) - 1)]
    Ws[-1] *= 0.05
    flat = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)]).astype(np.float32)
    net.set_params(flat)
    V0, fallback = net.predict(Sd)
    assert fallback == 0
    ref = OM.MLP([w.astype(np.float32).astype(np.float64) for w in Ws], [b.astype(np.float32) for b in bs])
    y_ref, _ = ref.forward(_norm(_features(S), xm, xs))
    V0 = V0.cpu().numpy()
    ok = ys > 0
    y_gpu = (np.concatenate([V0.real - 1.0, V0.imag], axis=1)[:, ok] - ym[ok]) / ys[ok]
    rel = np.linalg.norm(y_gpu - y_ref[:, ok]) / np.linalg.norm(y_ref[:, ok])
    rows = np.linalg.norm(y_gpu - y_ref[:, ok], axis=1) / np.linalg.norm(y_ref[:, ok], axis=1)
    assert rel <= 2e-2 and rows.max() <= 5e-2, (rel, rows.max())
    bs_far = [b.copy() for b in bs]
    bs_far[-1][: f.n_pq] += 1e4  # Re V far above the band at every bus (1e4 standard deviations)
    net.set_params(np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs_far)]).astype(np.float32))
    V0, fallback = net.predict(Sd)
    assert fallback == T
    assert np.array_equal(V0.cpu().numpy(), np.ones_like(S))
    net.close()


@pytest.mark.parametrize("hidden,layers", [(256, 3), (128, 1)])
def test_fused_prediction_with_several_tiles_per_cta(cuda, feeder200, hidden, layers):
    """More 128-column tiles than SMs: each persistent CTA takes several tiles in turn and the rings
    of the weights and of the converted features wrap many times.  Every column's prediction equals
    the one computed in a launch with one tile per CTA (a column's outputs depend on its own row of
    the products only, so the two agree bit for bit), and sampled columns match the FP64 network."""
    import torch

    f, c = feeder200
    S_fit = G.load_tensor(f, 4096, 9)
    V_fit, _, _ = c.solve(S_fit, tol=1e-12)
    net = tpf.LearnedStart(f.n_pq, hidden=hidden, hidden_layers=layers, max_batch=128, seed=5)
    net.fit_normalization(_dev(S_fit), _dev(V_fit))
    xm, xs, ym, ys = (np.asarray(a, dtype=np.float64) for a in net.normalization())
    rng = np.random.default_rng(17 + layers)
    sizes = net.sizes
    Ws = [rng.uniform(-1, 1, (sizes[i + 1], sizes[i])) * np.sqrt(6.0 / (sizes[i] + sizes[i + 1]))
          for i in range(len(sizes) - 1)]
    bs = [rng.normal(0, 0.05, sizes[i + 1]) for i in range(len(sizes) - 1)]
    Ws[-1] *= 0.05
    net.set_params(np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)]).astype(np.float32))
    T = 48_037  # 376 tiles over at most 152 CTAs, the last one ragged
    S = G.load_tensor(f, T, 10)
    Sd = _dev(S)
    V0, fallback = net.predict(Sd)
    assert fallback == 0
    for k in (0, 128 * 151 + 5, T - 2000):
        part, fb = net.predict(Sd[k:k + 2000])  # 16 tiles: one per CTA
        assert fb == 0 and torch.equal(part, V0[k:k + 2000]), k
    idx = np.sort(rng.choice(T, 512, replace=False))
    ref = OM.MLP([w.astype(np.float32).astype(np.float64) for w in Ws], [b.astype(np.float32) for b in bs])
    y_ref, _ = ref.forward(_norm(_features(S[idx]), xm, xs))
    V0s = V0.cpu().numpy()[idx]
    ok = ys > 0
    y_gpu = (np.concatenate([V0s.real - 1.0, V0s.imag], axis=1)[:, ok] - ym[ok]) / ys[ok]
    rel = np.linalg.norm(y_gpu - y_ref[:, ok]) / np.linalg.norm(y_ref[:, ok])
    assert rel <= 2e-2, rel
    net.close()


def test_learned_host_solve_matches_the_device_solve(cuda, feeder200):
    """tpf_solve_learned_host (host buffers, copies and chunked solves pipelined in the library):
    70,000 columns go in four chunks, and every column's V, sweep count and mismatch equal the
    device-resident tpf_solve_learned's bit for bit (a column's prediction and solve do not depend on
    the other columns); sampled columns match the oracle within 1e-8 pu; the fallback counts agree."""
    import torch

    f, c = feeder200
    fd = tpf.Feeder.from_inputs(f)
    S_fit = G.load_tensor(f, 4096, 9)
    V_fit, _, _ = c.solve(S_fit, tol=1e-12)
    net = tpf.LearnedStart(f.n_pq, hidden=256, hidden_layers=3, max_batch=128, seed=5)
    net.fit_normalization(_dev(S_fit), _dev(V_fit))
    rng = np.random.default_rng(23)
    sizes = net.sizes
    Ws = [rng.uniform(-1, 1, (sizes[i + 1], sizes[i])) * np.sqrt(6.0 / (sizes[i] + sizes[i + 1]))
          for i in range(len(sizes) - 1)]
    bs = [rng.normal(0, 0.05, sizes[i + 1]) for i in range(len(sizes) - 1)]
    Ws[-1] *= 0.05
    net.set_params(np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)]).astype(np.float32))
    T = 70_000
    S = G.load_tensor(f, T, 11)
    Sh = torch.from_numpy(S).pin_memory()
    Vh, ith, mmh, fb_h, st_h = fd.solve_learned_host(net, Sh, tol=1e-10)
    assert st_h == tpf.OK
    assert fd.stats()["converged"] == T
    V, it, mm, fb, st = fd.solve_learned(net, _dev(S), tol=1e-10)
    assert st == tpf.OK and fb_h == fb
    assert np.array_equal(Vh, V.cpu().numpy())
    assert np.array_equal(ith, it.cpu().numpy())
    assert np.array_equal(mmh, mm.cpu().numpy())
    idx = np.sort(rng.choice(T, 256, replace=False))
    Vo, ito, _ = c.solve(S[idx], tol=1e-13)
    assert np.abs(Vh[idx] - Vo).max() <= 1e-8
    # Empty input.
    _, _, _, fb0, st0 = fd.solve_learned_host(net, S[:0])
    assert st0 == tpf.OK and fb0 == 0
    net.close()
    fd.close()
    torch.cuda.synchronize()


def test_learned_solve_with_infeasible_and_non_finite_columns(cuda, feeder200):
    """Bad columns through the learned start: a load far beyond the feeder's loadability, a NaN, a
    load of 1e300 (beyond FP32: the converter's infinity) and an infinite one.  The NaN and infinite
    predictions fail the |V| band and start flat; every bad column is reported unconverged
    (-max_iter, TPF_ENOCONV); the other columns match the oracle."""
    f, c = feeder200
    fd = tpf.Feeder.from_inputs(f)
    S_fit = G.load_tensor(f, 4096, 9)
    V_fit, _, _ = c.solve(S_fit, tol=1e-12)
    net = tpf.LearnedStart(f.n_pq, hidden=256, hidden_layers=3, max_batch=128, seed=5)
    net.fit_normalization(_dev(S_fit), _dev(V_fit))
    rng = np.random.default_rng(31)
    sizes = net.sizes
    Ws = [rng.uniform(-1, 1, (sizes[i + 1], sizes[i])) * np.sqrt(6.0 / (sizes[i] + sizes[i + 1]))
          for i in range(len(sizes) - 1)]
    bs = [rng.normal(0, 0.05, sizes[i + 1]) for i in range(len(sizes) - 1)]
    Ws[-1] *= 0.05
    net.set_params(np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)]).astype(np.float32))
    S = G.load_tensor(f, 4096, 12).copy()
    bad = [3, 10, 20, 30]
    S[3] *= 400.0
    S[10, 5] = np.nan
    S[20, 7] = 1e300
    S[30, 0] = np.inf
    V, it, mm, fallback, st = fd.solve_learned(net, _dev(S), tol=1e-10, max_iter=60)
    assert st == tpf.ENOCONV
    itc = it.cpu().numpy()
    assert all(itc[k] == -60 for k in bad), itc[bad]
    assert fallback >= 3  # the NaN, 1e300 and infinite columns at least
    assert fd.stats()["converged"] == 4096 - len(bad)
    good = np.setdiff1d(np.arange(4096), bad)
    idx = good[:: 16]
    Vo, _, _ = c.solve(S[idx], tol=1e-13)
    assert np.abs(V.cpu().numpy()[idx] - Vo).max() <= 1e-8
    assert np.all(itc[good] > 0)
    net.close()
    fd.close()


def test_learned_solve_matches_the_oracle(cuda, feeder200):
    """tpf_solve_learned (fused prediction into complex64 starting voltages, then the sparse mixed
    solve from them): the oracle's solution within 1e-8 pu, fewer sweeps than the flat start, no
    column sent to the flat start; argument errors on the host."""
    import torch

    f, c = feeder200
    fd = tpf.Feeder.from_inputs(f)
    S_tr = _dev(G.load_tensor(f, 16384, 41))
    V_tr, _, _, st = fd.solve(S_tr, precision="mixed", tol=1e-10, method="sparse")
    assert st == tpf.OK
    net = tpf.LearnedStart(f.n_pq, max_batch=1024, seed=7)
    net.fit_normalization(S_tr, V_tr)
    for epoch in range(25):
        for k in range(0, 16384, 1024):
            net.train_step(S_tr[k:k + 1024], V_tr[k:k + 1024], lr=1e-3, want_loss=False)
    S_np = G.load_tensor(f, 4096, 42)[:3001]
    S_ev = _dev(S_np)
    V, it, mm, fb, st = fd.solve_learned(net, S_ev, tol=1e-10)
    assert st == tpf.OK and fb == 0
    Vo, _, _ = c.solve(S_np, tol=1e-13)
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-8
    assert fd.stats()["converged"] == S_np.shape[0]
    mm_ref = c.mismatch(S_np, V.cpu().numpy())
    assert np.all(np.abs(mm.cpu().numpy() - mm_ref) <= 1e-9 + 1e-3 * mm_ref)
    _, it_f, _, _ = fd.solve(S_ev, precision="mixed", tol=1e-10, method="sparse")
    assert it.float().mean().item() < it_f.float().mean().item() - 1.0
    # Predictions pushed outside the |V| band: every column starts flat (the solver's guard), with
    # the flat start's results.
    params = net.params()
    Ws, bs = net.unflatten(params.copy())
    bs[-1][: f.n_pq] += 1e4
    net.set_params(np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(Ws, bs)]))
    V2, it2, _, fb2, st2 = fd.solve_learned(net, S_ev, tol=1e-10)
    assert st2 == tpf.OK and fb2 == S_np.shape[0]
    assert torch.equal(it2, it_f)
    assert np.abs(V2.cpu().numpy() - Vo).max() <= 1e-8
    net.set_params(params)
    # Empty input, and a network for another feeder size.
    _, _, _, fb, st = fd.solve_learned(net, S_ev[:0])
    assert st == tpf.OK and fb == 0
    other = tpf.LearnedStart(30, max_batch=128, seed=1)
    with pytest.raises(ValueError, match="demand buses"):
        fd.solve_learned(other, S_ev)
    other.close()
    net.close()
    fd.close()
    torch.cuda.synchronize()
