"""GPU: scenario x time load tensors (complex64) through tpf_solve_ex with fused statistics.

The oracle solves the same complex64 loads widened to complex128 (the input's exact values).
Bars: V within 1e-8 pu when V is written as complex128, within 2e-7 pu (the FP32 rounding of a
value near 1) when written as complex64; per-column |V| extremes within 1e-6; violation counts
exact except at buses within 1e-6 of a band edge.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

pytestmark = pytest.mark.gpu


def _case(n_bus=120, n_scen=6, n_hours=48, seed=3):
    f = G.make_feeder(n_bus, seed, peak_factor=1.8)
    S = G.scenario_tensor(f, n_scen, n_hours, seed)
    return f, S


def _check_stats(res, Vo, band, T, n):
    absV = np.abs(Vo).reshape(T, n)
    vmin = res["vmin"].cpu().numpy().reshape(T)
    vmax = res["vmax"].cpu().numpy().reshape(T)
    assert np.abs(vmin - absV.min(1)).max() <= 1e-6
    assert np.abs(vmax - absV.max(1)).max() <= 1e-6
    under, over = absV < band[0], absV > band[1]
    edge = (np.abs(absV - band[0]) < 1e-6) | (np.abs(absV - band[1]) < 1e-6)
    clean = ~edge.any(1)
    viol = res["viol"].cpu().numpy().reshape(T)
    assert np.array_equal(viol[clean], (under | over).sum(1)[clean])
    cols_clean = ~edge.any(0)
    assert np.array_equal(res["bus_under"].cpu().numpy()[cols_clean], under.sum(0)[cols_clean])
    assert np.array_equal(res["bus_over"].cpu().numpy()[cols_clean], over.sum(0)[cols_clean])


def test_scenario_tensor_complex64(cuda):
    import torch

    f, S = _case()
    n_scen, n_hours, n = S.shape
    T = n_scen * n_hours
    fd = tpf.Feeder.from_inputs(f)
    c = O.Case.from_feeder(f)
    S128 = S.astype(np.complex128).reshape(T, n)
    Vo, _, _ = c.solve(S128, tol=1e-13)
    Sd = torch.from_numpy(S).cuda()
    band = (0.96, 1.02)
    res = fd.solve_tensor(Sd, v_complex64=False, v_band=band)
    assert res["status"] == tpf.OK
    V = res["V"].cpu().numpy().reshape(T, n)
    assert res["V"].shape == S.shape
    assert np.abs(V - Vo).max() <= 1e-8
    mm_ref = c.mismatch(S128, V)
    assert np.all(np.abs(res["mismatch"].cpu().numpy().reshape(T) - mm_ref) <= 1e-9 + 1e-3 * mm_ref)
    _check_stats(res, Vo, band, T, n)
    # complex64 V and statistics-only runs agree with the complex128 one.
    r32 = fd.solve_tensor(Sd, v_band=band)
    assert r32["V"].dtype == torch.complex64
    assert np.abs(r32["V"].cpu().numpy().reshape(T, n) - Vo).max() <= 2e-7
    r0 = fd.solve_tensor(Sd, want_V=False, v_band=band)
    assert r0["V"] is None
    for k in ("iters", "vmin", "vmax", "viol", "bus_under", "bus_over"):
        assert torch.equal(r0[k], res[k]), k
    fd.close()


def test_scenario_counts_accumulate(cuda):
    import torch

    f, S = _case(n_bus=60, n_scen=4, n_hours=24, seed=5)
    fd = tpf.Feeder.from_inputs(f)
    Sd = torch.from_numpy(S).cuda()
    band = (0.97, 1.01)
    whole = fd.solve_tensor(Sd, want_V=False, v_band=band)
    counts = (torch.zeros(f.n_pq, dtype=torch.int32, device="cuda"),
              torch.zeros(f.n_pq, dtype=torch.int32, device="cuda"))
    for s in range(S.shape[0]):  # one scenario at a time into the same per-bus counters
        fd.solve_tensor(Sd[s].contiguous(), want_V=False, v_band=band, bus_counts=counts)
    assert torch.equal(counts[0], whole["bus_under"]) and torch.equal(counts[1], whole["bus_over"])
    fd.close()


def test_tensor_requires_sparse(cuda):
    import torch

    f, S = _case(n_bus=20, n_scen=1, n_hours=4)
    fr, to, z = list(f.from_bus), list(f.to_bus), list(f.z_pu)
    fr.append(2), to.append(9), z.append(0.03 + 0.02j)
    mesh = tpf.Feeder(f.n_bus, fr, to, z, f.slack, f.v0, f.pq_bus)
    res = mesh.solve_tensor(torch.from_numpy(S).cuda(), check=False)
    assert res["status"] == tpf.EUNSUPPORTED
    mesh.close()


def test_tensor_statistics_in_every_launch_chunk(cuda):
    """A 5,000-bus feeder over 8,200 complex64 columns: the large-feeder kernel solves them in two
    launches, each writing its own columns' statistics.  The per-column |V| extremes and band
    counts agree with the returned V in both, and the per-bus counts add up over all columns."""
    import torch

    f = G.make_feeder(5000, 2, peak_factor=1.6)
    T, n = 8200, f.n_pq
    Sd = G.load_tensor_device(f, T, 2, torch.device("cuda"), dtype=torch.complex64)
    fd = tpf.Feeder.from_inputs(f)
    band = (0.95, 1.02)
    res = fd.solve_tensor(Sd, v_complex64=False, v_band=band)
    assert res["status"] == tpf.OK
    assert fd.stats()["kernel_launches"] == 2
    absV = res["V"].abs()
    vmin, vmax = absV.min(1).values.float(), absV.max(1).values.float()
    assert (res["vmin"] - vmin).abs().max().item() <= 1e-6
    assert (res["vmax"] - vmax).abs().max().item() <= 1e-6
    under, over = absV < band[0], absV > band[1]
    edge = ((absV - band[0]).abs() < 1e-6) | ((absV - band[1]).abs() < 1e-6)
    clean = ~edge.any(1)
    assert torch.equal(res["viol"][clean], (under | over).sum(1).to(res["viol"].dtype)[clean])
    cols_clean = ~edge.any(0)
    assert torch.equal(res["bus_under"][cols_clean], under.sum(0).to(res["bus_under"].dtype)[cols_clean])
    assert torch.equal(res["bus_over"][cols_clean], over.sum(0).to(res["bus_over"].dtype)[cols_clean])
    fd.close()


def test_tensor_three_phase_complex64(cuda):
    """A three-phase feeder through tpf_solve_ex with complex64 loads: V against the polyphase
    oracle on the widened loads, and the statistics against that V."""
    import torch

    pf = G.make_feeder_poly(60, 3)
    T = 96
    S = G.load_tensor_poly(pf, T, 3).reshape(T, -1).astype(np.complex64)
    pc = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, vs=pf.v0)
    Vo, _, _ = pc.solve(S.astype(np.complex128), tol=1e-13)
    fd = tpf.Feeder.poly(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, v0=pf.v0)
    band = (0.97, 1.03)
    res = fd.solve_tensor(torch.from_numpy(S).cuda(), v_complex64=False, v_band=band)
    assert res["status"] == tpf.OK
    V = res["V"].cpu().numpy()
    assert np.abs(V - Vo).max() <= 1e-8
    _check_stats(res, Vo, band, T, S.shape[1])
    fd.close()
