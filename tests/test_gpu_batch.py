"""GPU: tpf_solve_batch over feeders of different sizes against the FP64 oracle.

Tolerances as in test_gpu_parity: max |V - V_oracle| <= 1e-8 pu (mixed path), iteration counts
within +-1 of the oracle's.  A batched feeder runs exactly the arithmetic of its own sparse solve,
so batch and single results are compared bit for bit.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

pytestmark = pytest.mark.gpu

TOL_MIXED = 1e-8


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _batch(specs):
    feeders, S, cases = [], [], []
    for n_bus, T, seed in specs:
        f = G.make_feeder(n_bus, seed)
        feeders.append(f)
        S.append(G.load_tensor(f, T, seed, step_minutes=G.step_minutes_for(max(T, 96))))
    return feeders, S


def test_batch_matches_oracle_and_single_solves(cuda):
    # Sizes spanning block sizes from 32 to 512 threads, ragged and empty column counts.
    specs = [(2, 7, 1), (20, 96, 2), (35, 129, 3), (130, 96, 4), (300, 288, 5), (20, 0, 6), (700, 96, 7),
             (1100, 40, 8), (57, 288, 9), (3, 1, 11)]
    feeders, S = _batch(specs)
    fds = [tpf.Feeder.from_inputs(f) for f in feeders]
    Sd = [_dev(s) for s in S]
    V, it, mm, conv, stats, st = tpf.solve_batch(fds, Sd)
    assert st == tpf.OK
    assert list(conv) == [s.shape[0] for s in S]
    assert stats["converged"] == sum(s.shape[0] for s in S)
    for k, f in enumerate(feeders):
        if S[k].shape[0] == 0:
            continue
        c = O.Case.from_feeder(f)
        Vo, _, _ = c.solve(S[k], tol=1e-13)
        _, it_ref, _ = c.solve(S[k], tol=1e-10)
        Vk = V[k].cpu().numpy()
        assert np.abs(Vk - Vo).max() <= TOL_MIXED, f"feeder {k} (n_bus {f.n_bus})"
        assert np.abs(it[k].cpu().numpy() - it_ref).max() <= 1
        mm_ref = c.mismatch(S[k], Vk)
        assert np.all(np.abs(mm[k].cpu().numpy() - mm_ref) <= 1e-9 + 1e-3 * mm_ref)
        Vs, its, mms, st1 = fds[k].solve(Sd[k], precision="mixed", method="sparse")
        assert st1 == tpf.OK
        assert np.array_equal(Vs.cpu().numpy(), Vk) and np.array_equal(its.cpu().numpy(), it[k].cpu().numpy())
    for fd in fds:
        fd.close()


def test_batch_meshed_feeder_falls_back(cuda):
    f = G.make_feeder(40, 3)
    fr, to, z = list(f.from_bus), list(f.to_bus), list(f.z_pu)
    fr.append(5), to.append(30), z.append(0.02 + 0.01j)  # a loop: not radial
    mesh = tpf.Feeder(f.n_bus, fr, to, z, f.slack, f.v0, f.pq_bus)
    rad = tpf.Feeder.from_inputs(G.make_feeder(60, 4))
    S_mesh = G.load_tensor(f, 50, 3)
    S_rad = G.load_tensor(G.make_feeder(60, 4), 70, 4)
    V, it, mm, conv, stats, st = tpf.solve_batch([mesh, rad], [_dev(S_mesh), _dev(S_rad)])
    assert st == tpf.OK and list(conv) == [50, 70]
    cm = O.Case(f.n_bus, fr, to, z, f.slack, f.v0, f.pq_bus)
    Vo, _, _ = cm.solve(S_mesh, tol=1e-13)
    assert np.abs(V[0].cpu().numpy() - Vo).max() <= TOL_MIXED
    Vo2, _, _ = O.Case.from_feeder(G.make_feeder(60, 4)).solve(S_rad, tol=1e-13)
    assert np.abs(V[1].cpu().numpy() - Vo2).max() <= TOL_MIXED
    mesh.close()
    rad.close()


def test_batch_unconverged_and_given_start(cuda):
    feeders, S = _batch([(30, 64, 1), (90, 32, 2)])
    S[0] = S[0].copy()
    S[0][7] *= 400.0  # infeasible column
    fds = [tpf.Feeder.from_inputs(f) for f in feeders]
    V, it, mm, conv, stats, st = tpf.solve_batch(fds, [_dev(s) for s in S], max_iter=60)
    assert st == tpf.ENOCONV
    assert list(conv) == [63, 32]
    assert it[0].cpu().numpy()[7] == -60
    # Given start at the oracle's solution: one sweep per column.
    Vo = [O.Case.from_feeder(f).solve(s, tol=1e-13)[0] for f, s in zip(feeders, S)]
    Vg = [_dev(Vo[1])]
    V, it, mm, conv, stats, st = tpf.solve_batch(fds[1:], [_dev(S[1])], V=Vg, start="given")
    assert st == tpf.OK and (it[0].cpu().numpy() == 1).all()
    assert np.abs(V[0].cpu().numpy() - Vo[1]).max() <= 1e-12
    for fd in fds:
        fd.close()


def test_batch_errors(cuda):
    f = G.make_feeder(30, 1)
    fd = tpf.Feeder.from_inputs(f)
    S = _dev(G.load_tensor(f, 8, 1))
    with pytest.raises(tpf.TpfError) as e:
        tpf.solve_batch([fd, fd], [S, S])  # the same handle twice
    assert e.value.status == tpf.EINVAL
    V, it, mm, conv, stats, st = tpf.solve_batch([], [])
    assert st == tpf.OK and conv.size == 0
    fd.close()


def test_batch_graph_replays_match_solve_batch(cuda):
    """tpf_batch_*: the batch is prepared once and solved by replaying one captured CUDA graph;
    each replay reads the current loads.  Its results are those of tpf_solve_batch bit for bit."""
    import torch

    specs = [(2, 7, 1), (35, 129, 3), (130, 96, 4), (20, 0, 6), (700, 96, 7), (57, 288, 9)]
    feeders, S = _batch(specs)
    fds = [tpf.Feeder.from_inputs(f) for f in feeders]
    alpha = np.random.default_rng(2).dirichlet([2, 1, 1], fds[2].n_pq).T.copy()
    fds[2].set_zip(alpha)  # a ZIP feeder takes a launch of its own
    Sd = [_dev(s) for s in S]
    Vr, itr, mmr, convr, _, st = tpf.solve_batch(fds, Sd)
    assert st == tpf.OK
    bg = tpf.BatchGraph(fds, Sd)
    _, _, st = bg.wait(check=False)
    assert st == tpf.EINVAL  # nothing launched yet
    for _ in range(2):
        bg.launch()
        conv, stats, st = bg.wait()
        assert st == tpf.OK and list(conv) == list(convr) and stats["converged"] == sum(convr)
        for f in range(len(fds)):
            assert torch.equal(bg.V[f], Vr[f]) and torch.equal(bg.iters[f], itr[f])
            assert torch.equal(bg.mismatch[f], mmr[f])
    # New loads written in place are solved by the next replay.
    for s in Sd:
        s.mul_(0.8)
    Vr2, itr2, _, convr2, _, _ = tpf.solve_batch(fds, Sd)
    bg.launch()
    conv, _, st = bg.wait()
    assert st == tpf.OK and list(conv) == list(convr2)
    assert all(torch.equal(bg.V[f], Vr2[f]) and torch.equal(bg.iters[f], itr2[f]) for f in range(len(fds)))
    # A feeder re-laid out after creation (autotune) makes the launch refuse.
    fds[4].autotune(Sd[4][:64].contiguous())
    with pytest.raises(tpf.TpfError) as e:
        bg.launch()
    assert e.value.status == tpf.EINVAL
    bg.close()
    # Meshed feeders have no tree layout: unsupported.
    f = feeders[1]
    fr, to, z = list(f.from_bus), list(f.to_bus), list(f.z_pu)
    fr.append(5), to.append(30), z.append(0.02 + 0.01j)
    mesh = tpf.Feeder(f.n_bus, fr, to, z, f.slack, f.v0, f.pq_bus)
    with pytest.raises(tpf.TpfError) as e:
        tpf.BatchGraph([mesh], [Sd[1]])
    assert e.value.status == tpf.EUNSUPPORTED
    mesh.close()
    for fd in fds:
        fd.close()
