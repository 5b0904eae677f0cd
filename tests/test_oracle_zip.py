"""Pins of the oracle's ZIP load model (Eq. 3): cases with closed forms, the reduction to the
constant-power iteration, an independent root finder, and a planted mistake."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G


def _case(nb=30, seed=2, T=6):
    f = G.make_feeder(nb, seed)
    return f, O.Case.from_feeder(f), G.load_tensor(f, T, seed, t0=0)


def _alpha(n, p, i, z):
    return np.stack([np.full(n, p), np.full(n, i), np.full(n, z)])


def _ydd(c):
    pq = c.pq
    return c.Y[np.ix_(pq, pq)], c.Y[pq, c.slack]


def test_constant_impedance_is_linear():
    # alpha_Z = 1: i_d = conj(s) v, so (Y_dd + diag(conj(s))) v = -Y_ds v_s exactly.
    f, c, S = _case()
    n = f.n_pq
    V, it, _ = c.solve_zip(S, _alpha(n, 0, 0, 1))
    Ydd, Yds = _ydd(c)
    for t in range(S.shape[0]):
        v = np.linalg.solve(Ydd + np.diag(np.conj(S[t])), -Yds * c.vs)
        assert np.abs(V[t] - v).max() <= 1e-12
    assert (it == 2).all()  # F = 0: the first update lands on w, the second confirms it


def test_constant_current_is_linear():
    # alpha_I = 1: i_d = conj(s), so v = -Y_dd^{-1} (Y_ds v_s + conj(s)).
    f, c, S = _case()
    V, it, _ = c.solve_zip(S, _alpha(f.n_pq, 0, 1, 0))
    Ydd, Yds = _ydd(c)
    for t in range(S.shape[0]):
        v = np.linalg.solve(Ydd, -(Yds * c.vs + np.conj(S[t])))
        assert np.abs(V[t] - v).max() <= 1e-12


def test_constant_power_reduces_to_algorithm_1():
    f, c, S = _case()
    Vz, itz, _ = c.solve_zip(S, _alpha(f.n_pq, 1, 0, 0), tol=1e-10)
    V, it, _ = c.solve(S, tol=1e-10)
    assert np.array_equal(itz, it)
    assert np.abs(Vz - V).max() <= 1e-13
    mz = c.mismatch_zip(S, _alpha(f.n_pq, 1, 0, 0), V)
    assert np.allclose(mz, c.mismatch(S, V), rtol=1e-9, atol=1e-15)


def test_mixed_zip_matches_an_independent_root_finder():
    scipy_opt = pytest.importorskip("scipy.optimize")
    f, c, S = _case(nb=12, seed=4, T=3)
    n = f.n_pq
    rng = np.random.default_rng(0)
    a = rng.dirichlet([1, 1, 1], n).T  # per-bus coefficients summing to 1
    V, it, _ = c.solve_zip(S, a)
    assert (it > 0).all()
    assert (c.mismatch_zip(S, a, V) <= 1e-12).all()
    Ydd, Yds = _ydd(c)
    for t in range(S.shape[0]):
        s = S[t]

        def F(x):
            v = x[:n] + 1j * x[n:]
            r = Ydd @ v + Yds * c.vs + a[0] * np.conj(s / v) + a[1] * np.conj(s) + a[2] * np.conj(s) * v
            return np.r_[r.real, r.imag]

        def J(x):
            # Wirtinger derivatives of the residual: A = dr/dv, B = dr/dconj(v); then
            # dr/dRe(v) = A + B and dr/dIm(v) = j (A - B).
            v = x[:n] + 1j * x[n:]
            A = Ydd + np.diag(a[2] * np.conj(s))
            B = np.diag(-a[0] * np.conj(s) / np.conj(v) ** 2)
            dr, di = A + B, 1j * (A - B)
            return np.block([[dr.real, di.real], [dr.imag, di.imag]])

        x, info, ier, msg = scipy_opt.fsolve(F, np.r_[np.ones(n), np.zeros(n)], fprime=J, xtol=1e-10,
                                             full_output=True)
        assert ier == 1, msg  # the root finder itself converged
        assert np.abs(F(x)).max() <= 1e-10  # admittances are ~2e3 pu: 1e-13 relative
        assert np.abs(x[:n] + 1j * x[n:] - V[t]).max() <= 1e-12


def test_planted_mistake_in_the_load_model_is_seen():
    # The constant-power solution does not balance a ZIP load: the ZIP mismatch sees it.
    f, c, S = _case()
    a = _alpha(f.n_pq, 0.5, 0.3, 0.2)
    Vp, _, _ = c.solve(S)
    Vz, _, _ = c.solve_zip(S, a)
    assert (c.mismatch_zip(S, a, Vz) <= 1e-12).all()
    assert (c.mismatch_zip(S, a, Vp) > 1e-5).all()
