"""The seeded input generator: determinism, structure of the recipe, chunked regeneration."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G


def test_feeder_is_a_seeded_tree():
    a = G.make_feeder(300, 7)
    b = G.make_feeder(300, 7)
    c = G.make_feeder(300, 8)
    assert np.array_equal(a.from_bus, b.from_bus) and np.array_equal(a.z_pu, b.z_pu)
    assert not np.array_equal(a.from_bus, c.from_bus)
    assert a.n_branch == a.n_bus - 1
    assert (a.from_bus < a.to_bus).all()  # each bus hangs off an earlier one
    assert a.depth.max() <= 12
    r = a.z_pu.real * G.Z_BASE_OHM
    x = a.z_pu.imag * G.Z_BASE_OHM
    assert (r > 0.1 * 0.2 - 1e-12).all() and (r < 0.6 * 1.5 + 1e-12).all()
    assert (x > 0.05 * 0.2 - 1e-12).all() and (x < 0.4 * 1.5 + 1e-12).all()
    assert a.base_kw[0] == 0.0 and (a.base_kw[1:] >= 20).all() and (a.base_kw[1:] <= 150).all()


def test_load_tensor_recipe():
    f = G.make_feeder(40, 3)
    S = G.load_tensor(f, 2000, 3)
    assert S.shape == (2000, 39) and S.dtype == np.complex128
    base, pf = f.pq_params()
    # Q = P tan(acos(pf)) exactly, per bus
    assert np.allclose(S.imag / S.real, np.tan(np.arccos(pf))[None, :], rtol=1e-12)
    # the noise is lognormal(0, 0.2): log of P / (lam * base * shape) has sd 0.2
    hours = (np.arange(2000) / 60.0) % 24
    ratio = S.real / (f.load_scale * base[None, :] / 1000.0 * G.daily_shape(hours)[:, None])
    lr = np.log(ratio)
    assert abs(lr.mean()) < 0.01 and abs(lr.std() - 0.2) < 0.01
    assert G.daily_shape(np.linspace(0, 24, 10001)).max() == pytest.approx(1.0, abs=1e-6)


def test_chunks_regenerate_independently():
    f = G.make_feeder(20, 1)
    full = G.load_tensor(f, 3 * G.CHUNK, 5)
    mid = G.load_tensor(f, G.CHUNK, 5, t0=G.CHUNK)
    assert np.array_equal(full[G.CHUNK:2 * G.CHUNK], mid)
    with pytest.raises(ValueError):
        G.load_tensor(f, 10, 5, t0=3)


@pytest.mark.parametrize("n_bus,seed", [(34, 1), (200, 2), (1000, 1)])
def test_load_scale_puts_the_peak_column_near_090(n_bus, seed):
    """The recipe's load scale keeps the heaviest column solvable, around 0.90 pu."""
    f = G.make_feeder(n_bus, seed)
    base, pf = f.pq_params()
    p = f.load_scale * base / 1000.0
    S = (p + 1j * p * np.tan(np.arccos(pf)))[None, :]
    c = O.Case.from_feeder(f)
    V, it, _ = c.solve(S, tol=1e-10)
    assert it[0] > 0
    vmin = np.abs(V).min()
    if f.load_scale < 1.0:
        assert 0.88 <= vmin <= 0.92
    else:
        assert vmin >= 0.88


def test_scenario_tensor_and_batch_specs():
    f = G.make_feeder(60, 4, peak_factor=1.8)
    S = G.scenario_tensor(f, 5, 48, 4)
    assert S.shape == (5, 48, 59) and S.dtype == np.complex64
    # PV only lowers P in daylight; Q is untouched by PV
    night = np.arange(48) % 24 < 6
    assert (S.real[:, night, :] > 0).all()
    specs = G.batch_specs(500)
    n = np.array([s[0] for s in specs])
    T = np.array([s[1] for s in specs])
    assert n.min() >= 20 and n.max() <= 2000 and set(T) <= {96, 288, 1440}
    assert specs == G.batch_specs(500)
