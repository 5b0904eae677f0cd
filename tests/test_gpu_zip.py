"""GPU: ZIP loads (Eq. 3) on the sparse formulation and the FP64 path against the oracle.

The oracle iterates Eq. 3 literally (per-column F = -B^-1 A, w = -B^-1 c); the library keeps the
shared K and evaluates the ZIP current from the iterate.  Both reach the same fixed point, so the
bars are on V (1e-8 pu mixed, 1e-9 pu FP64) and on the power balance, not on iteration counts.
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


def _zip_case(nb, T, seed):
    f = G.make_feeder(nb, seed)
    c = O.Case.from_feeder(f)
    S = G.load_tensor(f, T, seed)
    a = np.random.default_rng(seed).dirichlet([2, 1, 1], f.n_pq).T.copy()  # per-bus shares
    return f, c, S, a


@pytest.mark.parametrize("nb,T", [(34, 200), (100, 64), (300, 20), (2, 5)])
@pytest.mark.parametrize("precision,method,tol_v", [("mixed", "sparse", 1e-8), ("fp64", "dense", 1e-9)])
def test_zip_vs_oracle(cuda, nb, T, precision, method, tol_v):
    f, c, S, a = _zip_case(nb, T, seed=nb)
    Vo, ito, _ = c.solve_zip(S, a, tol=1e-13)
    assert (ito > 0).all()
    fd = tpf.Feeder.from_inputs(f)
    fd.set_zip(a)
    V, it, mm, st = fd.solve(_dev(S), precision=precision, method=method, tol=1e-10)
    assert st == tpf.OK
    V = V.cpu().numpy()
    assert np.abs(V - Vo).max() <= tol_v
    mm_ref = c.mismatch_zip(S, a, V)
    assert np.all(np.abs(mm.cpu().numpy() - mm_ref) <= 1e-9 + 1e-3 * mm_ref)
    assert (mm_ref <= 1e-8).all()
    fd.close()


def test_zip_constant_power_and_reset(cuda):
    f, c, S, _ = _zip_case(60, 40, 3)
    fd = tpf.Feeder.from_inputs(f)
    V0, it0, _, _ = fd.solve(_dev(S), method="sparse")
    fd.set_zip(np.stack([np.ones(f.n_pq), np.zeros(f.n_pq), np.zeros(f.n_pq)]))
    V1, it1, _, _ = fd.solve(_dev(S), method="sparse")
    assert np.abs(V1.cpu().numpy() - V0.cpu().numpy()).max() <= 1e-14
    assert np.array_equal(it1.cpu().numpy(), it0.cpu().numpy())
    fd.set_zip(None)
    V2, it2, _, _ = fd.solve(_dev(S), method="sparse")
    assert np.array_equal(V2.cpu().numpy(), V0.cpu().numpy())
    fd.close()


def test_zip_unsupported_and_invalid(cuda):
    f, c, S, a = _zip_case(30, 8, 5)
    fd = tpf.Feeder.from_inputs(f)
    fd.set_zip(a)
    _, _, _, st = fd.solve(_dev(S), precision="mixed", method="dense", check=False)
    assert st == tpf.EUNSUPPORTED
    bad = a.copy()
    bad[1, 3] = np.nan
    with pytest.raises(tpf.TpfError) as e:
        fd.set_zip(bad)
    assert e.value.status == tpf.EINVAL
    fd.close()


def test_zip_in_a_batch_and_given_start(cuda):
    specs = [(40, 30, 11), (90, 20, 12), (25, 50, 13)]
    fds, S, refs = [], [], []
    for k, (nb, T, seed) in enumerate(specs):
        f, c, s, a = _zip_case(nb, T, seed)
        fd = tpf.Feeder.from_inputs(f)
        if k != 1:  # feeder 1 stays constant power
            fd.set_zip(a)
            refs.append(c.solve_zip(s, a, tol=1e-13)[0])
        else:
            refs.append(c.solve(s, tol=1e-13)[0])
        fds.append(fd)
        S.append(_dev(s))
    V, it, mm, conv, stats, st = tpf.solve_batch(fds, S)
    assert st == tpf.OK
    for k in range(3):
        assert np.abs(V[k].cpu().numpy() - refs[k]).max() <= 1e-8
    # Starting at the oracle's ZIP solution: one sweep.
    Vg, itg, _, st = fds[0].solve(S[0], V=_dev(refs[0]), method="sparse", start="given")
    assert st == tpf.OK and (itg.cpu().numpy() == 1).all()
    assert np.abs(Vg.cpu().numpy() - refs[0]).max() <= 1e-12
    for fd in fds:
        fd.close()


@pytest.mark.parametrize("nb", [2500, 3500])
def test_zip_large_feeders(cuda, nb):
    """ZIP loads at 8 buses per thread (2,500 buses: 2,499 demand buses, 320 threads, 179 KB of
    shared memory) and at 3,500 buses, which would need more than 227 KB at 8 buses per thread and
    is laid out at 16 while coefficients are set: the oracle's ZIP power balance at the returned V,
    and the same V as the FP64 dense path (Eq. 3's current from the iterate, a different kernel).
    Dropping the coefficients returns the feeder to constant power with its default layout."""
    f = G.make_feeder(nb, 7)
    S = G.load_tensor(f, 4096, 7)[[0, 1100, 2500]]
    a = np.random.default_rng(nb).dirichlet([2, 1, 1], f.n_pq).T.copy()
    fd = tpf.Feeder.from_inputs(f)
    V0, _, _, st = fd.solve(_dev(S), precision="mixed", method="sparse")  # constant power first
    assert st == tpf.OK
    fd.set_zip(a)
    V, it, mm, st = fd.solve(_dev(S), precision="mixed", method="sparse", tol=1e-10)
    assert st == tpf.OK, tpf.strerror(st)
    V = V.cpu().numpy()
    Y = O.ybus(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    mz = O.mismatch_zip(Y, f.slack, f.v0, f.pq_bus, a, S, V)
    assert mz.max() <= 1e-8, mz
    assert np.all(np.abs(mm.cpu().numpy() - mz) <= 1e-9 + 1e-3 * mz)
    V64, _, _, st = fd.solve(_dev(S), precision="fp64", method="dense", tol=1e-10)
    assert st == tpf.OK
    assert np.abs(V64.cpu().numpy() - V).max() <= 1e-8
    fd.set_zip(None)
    V1, _, _, st = fd.solve(_dev(S), precision="mixed", method="sparse")
    assert st == tpf.OK and np.array_equal(V1.cpu().numpy(), V0.cpu().numpy())
    fd.close()
