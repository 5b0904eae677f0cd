"""CPU: the torch-drawn input recipes (used for the largest workloads on the GPU) follow the same
recipe as the host generators -- checked on a CPU device -- and the polyphase inputs keep the
properties the polyphase tests rely on."""
import numpy as np
import pytest

from paper_2403_04578_gb300 import inputs as G

torch = pytest.importorskip("torch")


def test_device_load_tensor_follows_the_host_recipe():
    f = G.make_feeder(60, 3)
    T = 8192
    S = G.load_tensor_device(f, T, 3, "cpu").numpy()
    assert S.shape == (T, f.n_pq) and S.dtype == np.complex128
    base, pf = f.pq_params()
    # Power factor per bus exactly as drawn: Q = P tan(acos pf).
    assert np.allclose(S.imag, S.real * np.tan(np.arccos(pf))[None, :], rtol=1e-12, atol=0)
    # P = lam base shape(hour) lognormal(0, 0.2): the log of the noise has mean 0 and std 0.2.
    hours = (np.arange(T) / 60.0) % 24.0
    det = f.load_scale * base[None, :] / G.S_BASE_KW * G.daily_shape(hours)[:, None]
    z = np.log(S.real / det)
    assert abs(z.mean()) < 0.005 and abs(z.std() - 0.2) < 0.005
    # The host recipe draws the same distribution.
    zh = np.log(G.load_tensor(f, T, 3).real / det)
    assert abs(zh.mean()) < 0.005 and abs(zh.std() - 0.2) < 0.005
    # Reproducible for a seed, different across seeds.
    assert np.array_equal(S, G.load_tensor_device(f, T, 3, "cpu").numpy())
    assert not np.array_equal(S, G.load_tensor_device(f, T, 4, "cpu").numpy())
    # complex64 on request, same values rounded.
    S32 = G.load_tensor_device(f, 64, 3, "cpu", dtype=torch.complex64)
    assert S32.dtype == torch.complex64
    assert np.allclose(S32.numpy(), S[:64], rtol=1e-6, atol=0)


def test_device_scenario_tensor_shape_and_scenario_factors():
    f = G.make_feeder(40, 5, peak_factor=1.8)
    n_scen, n_hours = 6, 48
    S = G.scenario_tensor_device(f, n_scen, n_hours, 5, "cpu")
    assert tuple(S.shape) == (n_scen, n_hours, f.n_pq) and S.dtype == torch.complex64
    Sh = G.scenario_tensor(f, n_scen, n_hours, 5)
    assert Sh.shape == (n_scen, n_hours, f.n_pq)
    # Same recipe: the PV buses (negative net load at midday somewhere) and the load level agree.
    for X in (S.numpy(), Sh):
        assert np.isfinite(X).all()
        assert (X.real < 0).any()  # PV exports at some bus and hour
    ratio = np.abs(S.numpy()).mean() / np.abs(Sh).mean()
    assert 0.8 < ratio < 1.25


def test_polyphase_inputs():
    pf = G.make_feeder_poly(50, 9)
    f = G.make_feeder(50, 9)
    assert pf.z_blocks.shape == (49, 3, 3)
    # Symmetric blocks whose positive-sequence impedance (self - mutual) is the single-phase z.
    assert np.allclose(pf.z_blocks, pf.z_blocks.transpose(0, 2, 1))
    assert np.allclose(pf.z_blocks[:, 0, 0] - pf.z_blocks[:, 0, 1], f.z_pu, rtol=1e-14, atol=0)
    # Phase shares average to one per bus: the bus total is the single-phase base load.
    assert np.allclose(pf.base_kw.sum(axis=1), 3 * f.base_kw, rtol=1e-12)
    bal = G.make_feeder_poly(50, 9, unbalance=0.0)
    assert np.allclose(bal.base_kw, bal.base_kw[:, :1])
    S = G.load_tensor_poly(pf, 100, 9)
    assert S.shape == (100, 49, 3) and S.dtype == np.complex128
    assert np.allclose(S.imag, S.real * np.tan(np.arccos(pf.pf[1:]))[None], rtol=1e-12, atol=0)
