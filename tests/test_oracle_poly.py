"""Pins of the oracle's polyphase network (Eq. 1 with phases = 3): two reductions to the
single-phase oracle that hold exactly, and the power balance at the returned solution."""
import numpy as np

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G


def _rot(ph):
    return np.exp(-2j * np.pi * np.arange(ph) / ph)


def test_balanced_network_is_the_positive_sequence_solution():
    # Self z + z_m, mutual z_m, balanced loads s on every phase: the voltages are the single-phase
    # solution with impedance z and load s, rotated by the phase angles.
    f = G.make_feeder(40, 3)
    pf = G.make_feeder_poly(40, 3, unbalance=0.0)
    pc = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3)
    c = O.Case.from_feeder(f)
    S1 = G.load_tensor(f, 5, 3) * 0.7
    S3 = np.repeat(S1[:, :, None], 3, axis=2).reshape(5, -1)
    V3, it3, _ = pc.solve(S3)
    V1, it1, _ = c.solve(S1)
    assert (it3 > 0).all()
    expect = (V1[:, :, None] * _rot(3)[None, None, :]).reshape(5, -1)
    assert np.abs(V3 - expect).max() <= 1e-12
    assert (pc.mismatch(S3, V3) <= 1e-10).all()


def test_uncoupled_phases_are_three_single_phase_feeders():
    pf = G.make_feeder_poly(30, 5, mutual=0.0, unbalance=0.3)
    pc = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3)
    S = G.load_tensor_poly(pf, 4, 5)  # [T][n][3]
    V3, _, _ = pc.solve(S.reshape(4, -1))
    V3 = V3.reshape(4, pf.n_pq, 3)
    for p in range(3):
        c = O.Case(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks[:, p, p], vs=_rot(3)[p])
        Vp, _, _ = c.solve(S[:, :, p])
        assert np.abs(V3[:, :, p] - Vp).max() <= 1e-12


def test_coupled_unbalanced_power_balance_and_certificate():
    pf = G.make_feeder_poly(60, 7, mutual=0.4, unbalance=0.3)
    pc = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3)
    S = G.load_tensor_poly(pf, 24, 7).reshape(24, -1)
    V, it, _ = pc.solve(S)
    assert (it > 0).all()
    assert (pc.mismatch(S, V) <= 1e-10).all()
    # Eq. 9-11 contraction certificate at the solution stays below one.
    for t in range(0, 24, 6):
        assert O.contraction_certificate(pc.K, S[t], V[t]) < 1.0
    # A planted mistake (mutual coupling dropped) breaks the balance of the true network.
    z0 = pf.z_blocks.copy()
    for p in range(3):
        for q in range(3):
            if p != q:
                z0[:, p, q] = 0.0
    wrong = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, z0, 3)
    Vw, _, _ = wrong.solve(S)
    assert (pc.mismatch(S, Vw) > 1e-6).all()
