"""GPU: polyphase feeders (Eq. 1 with phases = 3) against the oracle's polyphase Algorithm 1.

Bars: max |V - V_oracle| <= 1e-8 pu on the sparse formulation (FP32 sweeps with double-float
anchors) and <= 1e-9 pu on the FP64 path; iteration counts within one of the oracle's (the tree
substitution with 3 x 3 branch blocks is the oracle's K = -Y_dd^-1 product); the power balance
of the returned voltages as the oracle evaluates it.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _poly(nb, T, seed, **kw):
    pf = G.make_feeder_poly(nb, seed, **kw)
    pc = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, vs=pf.v0)
    S = G.load_tensor_poly(pf, T, seed).reshape(T, -1)
    fd = tpf.Feeder.poly(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, v0=pf.v0)
    return pf, pc, S, fd


@pytest.mark.parametrize("nb,T", [(40, 128), (2, 9), (120, 65), (300, 40)])
@pytest.mark.parametrize("precision,method,tol_v", [("mixed", "sparse", 1e-8), ("fp64", "dense", 1e-9)])
def test_poly_vs_oracle(cuda, nb, T, precision, method, tol_v):
    pf, pc, S, fd = _poly(nb, T, seed=nb)
    assert fd.n_pq == 3 * pf.n_pq
    Vo, _, _ = pc.solve(S, tol=1e-13)
    _, it_ref, _ = pc.solve(S, tol=1e-10)
    V, it, mm, st = fd.solve(_dev(S), precision=precision, method=method, tol=1e-10)
    assert st == tpf.OK
    V = V.cpu().numpy()
    assert np.abs(V - Vo).max() <= tol_v
    assert np.abs(it.cpu().numpy() - it_ref).max() <= 1
    mm_ref = pc.mismatch(S, V)
    assert np.all(np.abs(mm.cpu().numpy() - mm_ref) <= 1e-9 + 1e-3 * mm_ref)
    fd.close()


def test_poly_balanced_equals_rotated_single_phase(cuda):
    f = G.make_feeder(60, 4)
    pf = G.make_feeder_poly(60, 4, unbalance=0.0)
    S1 = G.load_tensor(f, 50, 4) * 0.7
    S3 = np.repeat(S1[:, :, None], 3, axis=2).reshape(50, -1)
    fd3 = tpf.Feeder.poly(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, v0=pf.v0)
    V3, _, _, st = fd3.solve(_dev(S3), method="sparse")
    assert st == tpf.OK
    V1o, _, _ = O.Case.from_feeder(f).solve(S1, tol=1e-13)
    rot = np.exp(-2j * np.pi * np.arange(3) / 3)
    assert np.abs(V3.cpu().numpy().reshape(50, -1, 3) - V1o[:, :, None] * rot).max() <= 1e-8
    fd3.close()


def test_poly_given_start_batch_and_errors(cuda):
    pf, pc, S, fd = _poly(50, 40, seed=9)
    Vo, _, _ = pc.solve(S, tol=1e-13)
    V, it, _, st = fd.solve(_dev(S), V=_dev(Vo), method="sparse", start="given")
    assert st == tpf.OK and (it.cpu().numpy() == 1).all()
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-12
    # A batch mixing the polyphase feeder with single-phase ones.
    f1 = G.make_feeder(70, 3)
    fd1 = tpf.Feeder.from_inputs(f1)
    S1 = G.load_tensor(f1, 30, 3)
    Vb, itb, _, conv, _, st = tpf.solve_batch([fd, fd1], [_dev(S), _dev(S1)])
    assert st == tpf.OK and list(conv) == [40, 30]
    assert np.abs(Vb[0].cpu().numpy() - Vo).max() <= 1e-8
    assert np.abs(Vb[1].cpu().numpy() - O.Case.from_feeder(f1).solve(S1, tol=1e-13)[0]).max() <= 1e-8
    # Unsupported and invalid requests.
    _, _, _, st = fd.solve(_dev(S), precision="mixed", method="dense", check=False)
    assert st == tpf.EUNSUPPORTED
    with pytest.raises(tpf.TpfError) as e:
        fd.set_zip(np.ones((3, fd.n_pq)))
    assert e.value.status == tpf.EUNSUPPORTED
    with pytest.raises(tpf.TpfError) as e:
        tpf.Feeder.poly(pf.n_bus, pf.from_bus, pf.to_bus, np.zeros((pf.n_bus - 1, 3, 3)), 3)
    assert e.value.status == tpf.EINVAL  # singular branch blocks
    fd.close()
    fd1.close()


def test_poly_large_feeder_eight_buses_per_thread(cuda):
    """1,000 three-phase buses (2,997 unknowns): 8 positions per thread, 384 threads, the impedance
    rows read through the cache; against the oracle on a few columns."""
    pf, pc, S, fd = _poly(1000, 6, seed=4)
    Vo, it_o, _ = pc.solve(S, tol=1e-13)
    V, it, mm, st = fd.solve(_dev(S), method="sparse", tol=1e-10)
    assert st == tpf.OK
    assert np.abs(V.cpu().numpy() - Vo).max() <= 1e-8
    fd.close()


def test_poly_large_feeder_sixteen_buses_per_thread(cuda):
    """1,700 three-phase buses (5,097 unknowns, past 4,096): 16 positions per thread with device
    scratch; the oracle's power balance of the returned voltages."""
    pf = G.make_feeder_poly(1700, 6)
    S = G.load_tensor_poly(pf, 4, 6).reshape(4, -1)
    pc = O.PolyCase(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, vs=pf.v0, with_k=False)
    fd = tpf.Feeder.poly(pf.n_bus, pf.from_bus, pf.to_bus, pf.z_blocks, 3, v0=pf.v0)
    V, it, mm, st = fd.solve(_dev(S), method="sparse", tol=1e-10)
    assert st == tpf.OK
    assert pc.mismatch(S, V.cpu().numpy()).max() <= 1e-8
    fd.close()
