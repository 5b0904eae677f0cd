"""Pins of the CPU oracle to facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: the paper's two-bus example
(tests/golden/two_bus_fig2.json, Sec. III Fig. 2), the closed-form roots of the two-bus quadratic,
the Sec. III circle geometry of the load impedances (Eq. 6-7, their intersections and tangency)
and its parabola of critical loads,
the feasibility condition of Eq. 10, the contraction factor of Eq. 11, the radial path-sum form of
Y_dd^{-1}, an independent sparse Newton-Raphson, the power-balance residual of Eq. 1 and brute
force on tiny feeders.  The last test plants mistakes in the oracle's inputs (a sign, a dropped
conjugate, a dropped W) and shows that the pins catch each of them.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2403_04578_gb300 import inputs as G

HERE = os.path.dirname(os.path.abspath(__file__))


def fig2():
    with open(os.path.join(HERE, "golden", "two_bus_fig2.json")) as fh:
        g = json.load(fh)
    return complex(*g["z_s"]), complex(g["p_l"], g["q_l"]), complex(g["v0_abs"], 0.0)


def two_bus_case(z, v0=1.0 + 0j):
    return O.Case(2, [0], [1], [z], slack=0, vs=v0)


def power_balance(v, z, s, v0):
    """Eq. 1 for two buses: injection at bus 1 is v conj((v - v0)/z); it must equal -s."""
    return abs(v * np.conj((v - v0) / z) + s)


def test_closed_form_roots_solve_the_two_bus_power_flow():
    z, s, v0 = fig2()
    hi, lo = O.two_bus_roots(z, s, v0)
    assert power_balance(hi, z, s, v0) < 1e-14
    assert power_balance(lo, z, s, v0) < 1e-14
    assert abs(hi) > abs(lo)
    # |v_high| = 0.62115..., |v_low| = 0.37970... for the Fig. 2 load.
    assert abs(abs(hi) - 0.621150) < 5e-6 and abs(abs(lo) - 0.379697) < 5e-6


def test_fpi_reaches_the_high_voltage_root_fig2():
    z, s, v0 = fig2()
    c = two_bus_case(z, v0)
    assert abs(c.K[0, 0] + z) < 1e-15  # K = -Y_dd^{-1} = -z_s
    assert abs(c.W[0] - v0) < 1e-15  # W = K Y_ds v_s = v_s
    V, it, d = c.solve(np.array([[s]]), tol=1e-14, max_iter=500)
    hi, lo = O.two_bus_roots(z, s, v0)
    assert it[0] > 0
    assert abs(V[0, 0] - hi) < 1e-13


def test_contraction_ratio_matches_eq11():
    """Eq. 11 for two buses: the FPI step shrinks by k = |z_s| / |z_l| = |z||s| / |v|^2."""
    z, s, v0 = fig2()
    c = two_bus_case(z, v0)
    hi, _ = O.two_bus_roots(z, s, v0)
    k = O.two_bus_contraction(z, s, hi)
    assert abs(k - 0.6113) < 1e-3
    S = np.array([[s]])
    iterates = [c.solve(S, tol=0.0, max_iter=m)[0][0, 0] for m in range(1, 40)]
    steps = np.abs(np.diff(iterates))
    ratios = steps[1:] / steps[:-1]
    # The map is anti-holomorphic (v -> v0 - z conj(s)/conj(v)), so the step ratio tends to k.
    assert abs(ratios[-1] - k) < 1e-4


def test_low_root_is_repelling_and_nr_can_find_it():
    z, s, v0 = fig2()
    hi, lo = O.two_bus_roots(z, s, v0)
    assert O.two_bus_contraction(z, s, lo) > 1.0  # Eq. 11: k > 1 at the low-voltage root
    c = two_bus_case(z, v0)
    V, it, _ = c.solve(np.array([[s]]), V0=np.array([[lo * (1 + 1e-6)]]), tol=1e-13, max_iter=2000)
    assert it[0] > 0 and abs(V[0, 0] - hi) < 1e-11
    # Newton-Raphson started next to the low root converges to it (Fig. 4(a)).
    vnr, nit, ok = O.nr_solve(c.ybus_sparse(), 0, v0, [1], [s], v_init=[lo * (1 + 1e-3)], tol=1e-13)
    assert ok and abs(vnr[0] - lo) < 1e-10


def test_fpi_basin_covers_the_plane():
    """Fig. 4(c): the FPI reaches the high root from starts all over the complex plane."""
    z, s, v0 = fig2()
    hi, lo = O.two_bus_roots(z, s, v0)
    c = two_bus_case(z, v0)
    mags = np.linspace(0.05, 2.0, 14)
    angs = np.linspace(-np.pi, np.pi, 13, endpoint=False)
    starts = (mags[:, None] * np.exp(1j * angs[None, :])).ravel()
    starts = starts[np.abs(starts - lo) > 1e-3]
    S = np.full((starts.size, 1), s)
    V, it, _ = c.solve(S, V0=starts[:, None], tol=1e-13, max_iter=3000)
    assert (it > 0).all()
    assert np.abs(V[:, 0] - hi).max() < 1e-11


def sec3_circles(z_s: complex, s: complex, v0_abs: float):
    """Eq. 6-7: the load impedances z_l = r_l + j x_l that draw p_l (resp. q_l) from the source lie
    on a circle in the (r_l, x_l) plane; centres and radii from the two-bus power expression."""
    rs, xs, p, q = z_s.real, z_s.imag, s.real, s.imag
    c_p = np.array([v0_abs ** 2 / (2 * p) - rs, -xs])
    r_p = v0_abs / (2 * p) * np.sqrt(v0_abs ** 2 - 4 * rs * p)
    c_q = np.array([-rs, v0_abs ** 2 / (2 * q) - xs])
    r_q = v0_abs / (2 * q) * np.sqrt(v0_abs ** 2 - 4 * xs * q)
    return c_p, r_p, c_q, r_q


def sec3_load_impedances(z_s: complex, s: complex, v0_abs: float):
    """Both solutions z_l as the intersections of the Eq. 6-7 circles, found on their radical line
    (the line through both intersections, perpendicular to the line of centres)."""
    c_p, r_p, c_q, r_q = sec3_circles(z_s, s, v0_abs)
    n = c_q - c_p
    d = np.array([-n[1], n[0]]) / np.hypot(*n)
    # A point of the radical line: equal power with respect to both circles.
    rhs = (c_q @ c_q - r_q ** 2) - (c_p @ c_p - r_p ** 2)
    x0 = n * rhs / (2 * (n @ n))
    # Points x0 + t d on circle p.
    b = d @ (x0 - c_p)
    c = (x0 - c_p) @ (x0 - c_p) - r_p ** 2
    ts = (-b + np.sqrt(b * b - c), -b - np.sqrt(b * b - c))
    return [complex(*(x0 + t * d)) for t in ts], np.hypot(*x0)


def test_load_impedances_lie_on_the_sec3_circles():
    """Sec. III geometry, independent of the quadratic: the circles' two intersections are the two
    load impedances, on a line through the origin, one inside and one outside |z_s|; the voltage
    divider v = v0 z_l / (z_s + z_l) of the outer one is the FPI's fixed point, of the inner one the
    low root that Newton-Raphson reaches from a nearby start."""
    z, s, v0 = fig2()
    (za, zb), offset = sec3_load_impedances(z, s, abs(v0))
    assert offset < 1e-12  # the paper's intercept beta = 0: the radical line passes through the origin
    c_p, r_p, c_q, r_q = sec3_circles(z, s, abs(v0))
    for zl in (za, zb):
        assert abs(np.hypot(zl.real - c_p[0], zl.imag - c_p[1]) - r_p) < 1e-12
        assert abs(np.hypot(zl.real - c_q[0], zl.imag - c_q[1]) - r_q) < 1e-12
    z_hi, z_lo = (za, zb) if abs(za) > abs(zb) else (zb, za)
    assert abs(z_lo) < abs(z) < abs(z_hi)
    assert abs(abs(z_lo) * abs(z_hi) - abs(z) ** 2) < 1e-12  # power of the origin: h^2 = |z_s|^2
    v_hi = v0 * z_hi / (z + z_hi)
    v_lo = v0 * z_lo / (z + z_lo)
    V, it, _ = two_bus_case(z, v0).solve(np.array([[s]]), tol=1e-14, max_iter=500)
    assert it[0] > 0 and abs(V[0, 0] - v_hi) < 1e-13
    hi, lo = O.two_bus_roots(z, s, v0)
    assert abs(hi - v_hi) < 1e-13 and abs(lo - v_lo) < 1e-13
    c = two_bus_case(z, v0)
    vnr, _, ok = O.nr_solve(c.ybus_sparse(), 0, v0, [1], [s], v_init=[v_lo * (1 + 1e-3)], tol=1e-13)
    assert ok and abs(vnr[0] - v_lo) < 1e-10
    # Eq. 11 with the geometric impedances: contraction at the outer solution only.
    assert abs(O.two_bus_contraction(z, s, hi) - abs(z) / abs(z_hi)) < 1e-12
    assert abs(z) / abs(z_lo) > 1.0


def test_critical_load_where_the_sec3_circles_touch():
    """Sec. III: the largest load in a fixed direction is where the two circles touch
    (r_p + r_q = distance of the centres); the single solution there has |z_l| = |z_s|.  Below it
    the oracle has two roots and its FPI converges, above it there is no root and the FPI never
    stops."""
    from scipy.optimize import brentq

    z, s0, v0 = fig2()

    def gap(lam):
        c_p, r_p, c_q, r_q = sec3_circles(z, lam * s0, abs(v0))
        return r_p + r_q - np.hypot(*(c_p - c_q))

    lam_max = min(abs(v0) ** 2 / (4 * z.real * s0.real), abs(v0) ** 2 / (4 * z.imag * s0.imag))
    lam = brentq(gap, 0.1, lam_max * (1 - 1e-12), xtol=1e-15, rtol=1e-15)
    c_p, r_p, c_q, r_q = sec3_circles(z, lam * s0, abs(v0))
    touch = c_p + (c_q - c_p) * r_p / (r_p + r_q)
    assert abs(np.hypot(*touch) - abs(z)) < 1e-7  # maximum power transfer: |z_l| = |z_s|
    assert O.two_bus_roots(z, lam * (1 - 1e-9) * s0, v0) is not None
    assert O.two_bus_roots(z, lam * (1 + 1e-9) * s0, v0) is None
    c = two_bus_case(z, v0)
    S = np.array([[0.98 * lam * s0], [1.02 * lam * s0]])
    V, it, _ = c.solve(S, tol=1e-12, max_iter=20000)
    assert it[0] > 0 and it[1] < 0
    zl = V[0, 0] * z / (v0 - V[0, 0])
    assert abs(zl) > abs(z)


def sec3_parabola(z_s: complex, v0_abs: float):
    """Coefficients (G, H, I, J, K, L) of Sec. III's conic f(p_l, q_l) = 0, the set of loads with a
    single (maximum power transfer) solution, read so that its discriminant H^2 - 4GI vanishes as
    the paper states: I = x_s^2, J = |v0|^2 x_s, L = -|v0|^4 / 4."""
    r, x, v2 = z_s.real, z_s.imag, v0_abs ** 2
    return r * r, -2 * r * x, x * x, v2 * x, v2 * r, -v2 * v2 / 4


def parabola_limit(coef, theta: float) -> float:
    """Largest |s| on the ray s = |s| e^{j theta} inside the parabola: the positive root of
    f(|s| cos theta, |s| sin theta) = 0."""
    G, H, I, J, K, L = coef
    c, s = np.cos(theta), np.sin(theta)
    a2, a1 = G * s * s + H * c * s + I * c * c, J * s + K * c
    if abs(a2) < 1e-15 * abs(a1):
        return -L / a1
    return (-a1 + np.sqrt(a1 * a1 - 4 * a2 * L)) / (2 * a2)


@pytest.mark.parametrize("theta", [0.15, 0.4, "z_s", 0.8, 1.2, 1.45])
def test_feasibility_boundary_is_the_sec3_parabola(theta):
    """Sec. III: the loads where the Eq. 6-7 circles touch form a parabola, which the Eq. 10 circle
    |s| = |v0|^2 / (4 |z_s|) touches in the direction of z_s and stays outside of elsewhere.  On every
    ray the oracle's roots exist up to that boundary and no further, and its FPI converges inside
    and never stops outside.  A slack voltage of 1.05 pu separates L = -|v0|^4 / 4 from the printed
    -|v0|^2 / 4."""
    from scipy.optimize import brentq

    z, _, _ = fig2()
    v0 = 1.05 + 0j
    th = float(np.angle(z)) if theta == "z_s" else theta
    coef = sec3_parabola(z, abs(v0))
    G, H, I, _, _, _ = coef
    assert abs(H * H - 4 * G * I) < 1e-15  # a parabola
    lam = parabola_limit(coef, th)
    u = np.exp(1j * th)

    def gap(m):
        c_p, r_p, c_q, r_q = sec3_circles(z, m * u, abs(v0))
        return r_p + r_q - np.hypot(*(c_p - c_q))

    m_max = min(abs(v0) ** 2 / (4 * z.real * u.real), abs(v0) ** 2 / (4 * z.imag * u.imag))
    assert abs(brentq(gap, 1e-3, m_max * (1 - 1e-12), xtol=1e-15, rtol=1e-15) - lam) < 1e-12
    eq10 = abs(v0) ** 2 / (4 * abs(z))
    if theta == "z_s":
        assert abs(lam - eq10) < 1e-14
    else:
        assert lam > eq10 * (1 + 1e-6)
    assert O.two_bus_roots(z, lam * (1 - 1e-9) * u, v0) is not None
    assert O.two_bus_roots(z, lam * (1 + 1e-9) * u, v0) is None
    V, it, _ = two_bus_case(z, v0).solve(np.array([[0.97 * lam * u], [1.03 * lam * u]]), tol=1e-12,
                                         max_iter=20000)
    assert it[0] > 0 and it[1] < 0
    assert abs(V[0, 0] - O.two_bus_roots(z, 0.97 * lam * u, v0)[0]) < 1e-9


def test_printed_parabola_coefficients_miss_the_tangency():
    """The coefficient table as printed (I = |v0|^2 x_s, J = x_s^2, L = -|v0|^2 / 4) is not a
    parabola and misses the circles' tangency, which is why the reading above exchanges I and J."""
    z, s0, v0 = fig2()
    r, x = z.real, z.imag
    printed = (r * r, -2 * r * x, abs(v0) ** 2 * x, x * x, abs(v0) ** 2 * r, -abs(v0) ** 2 / 4)
    assert abs(printed[1] ** 2 - 4 * printed[0] * printed[2]) > 0.1
    th = float(np.angle(s0))
    assert abs(parabola_limit(printed, th) / parabola_limit(sec3_parabola(z, abs(v0)), th) - 1) > 0.01


@pytest.mark.parametrize("scale", [0.5, 0.9, 0.99, 1.01, 1.5])
def test_feasibility_eq10(scale):
    """Eq. 10 is sufficient; the exact two-bus limit is the zero of the quadratic's discriminant."""
    z, s0, v0 = fig2()
    # Largest load in the direction of s0 with a real root: a^2 = 4|z|^2|s|^2.
    u = s0 / abs(s0)
    lim = None
    lo_, hi_ = 0.0, 10.0
    for _ in range(200):
        mid = 0.5 * (lo_ + hi_)
        if O.two_bus_roots(z, mid * u, v0) is None:
            hi_ = mid
        else:
            lo_ = mid
    lim = lo_
    s = scale * lim * u
    c = two_bus_case(z, v0)
    V, it, _ = c.solve(np.array([[s]]), tol=1e-12, max_iter=20000)
    if scale < 1.0:
        assert it[0] > 0
        assert abs(V[0, 0] - O.two_bus_roots(z, s, v0)[0]) < 1e-9
    else:
        assert it[0] < 0  # no solution: never converges
        assert not O.feasible_eq10(z, s, v0)
    if O.feasible_eq10(z, s, v0):
        assert it[0] > 0


@pytest.mark.parametrize("n_bus,seed", [(2, 1), (5, 2), (20, 3), (60, 4), (34, 1)])
def test_K_is_the_radial_path_sum(n_bus, seed):
    f = G.make_feeder(n_bus, seed)
    c = O.Case.from_feeder(f)
    Kp = O.path_sum_K(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    assert np.abs(c.K - Kp).max() <= 1e-12 * np.abs(Kp).max()
    # Shunt-free radial feeder: W = K Y_ds v_s = v_s for every bus.
    assert np.abs(c.W - f.v0).max() < 1e-13


def test_W_follows_a_complex_slack_voltage():
    f = G.make_feeder(30, 5)
    vs = 1.03 * np.exp(0.02j)
    c = O.Case(f.n_bus, f.from_bus, f.to_bus, f.z_pu, vs=vs)
    assert np.abs(c.W - vs).max() < 1e-13


def _config1(T=1440):
    f = G.make_feeder(34, 1)
    return f, O.Case.from_feeder(f), G.load_tensor(f, T, 1)


def test_fpi_agrees_with_newton_raphson_config1():
    f, c, S = _config1()
    V, it, _ = c.solve(S, tol=1e-13)
    assert (it > 0).all()
    Ysp = c.ybus_sparse()
    worst = 0.0
    for t in range(0, S.shape[0], 7):
        vnr, _, ok = O.nr_solve(Ysp, 0, f.v0, f.pq_bus, S[t], tol=1e-12)
        assert ok
        worst = max(worst, np.abs(vnr - V[t]).max())
    assert worst <= 1e-10


def test_fpi_agrees_with_newton_raphson_heavy_feeder():
    f = G.make_feeder(200, 2)
    c = O.Case.from_feeder(f)
    S = G.load_tensor(f, 4096, 2)[1100:1120]  # evening peak
    V, it, _ = c.solve(S, tol=1e-13)
    assert (it > 0).all()
    Ysp = c.ybus_sparse()
    for t in range(S.shape[0]):
        vnr, _, ok = O.nr_solve(Ysp, 0, f.v0, f.pq_bus, S[t], tol=1e-12)
        assert ok and np.abs(vnr - V[t]).max() <= 1e-10


def test_power_balance_residual_and_contraction_certificate():
    for nb, seed, sl in ((34, 1, slice(0, 1440, 5)), (200, 2, slice(1000, 1200)), (500, 3, slice(1100, 1130))):
        f = G.make_feeder(nb, seed)
        c = O.Case.from_feeder(f)
        S = G.load_tensor(f, 4096, seed)[sl]
        V, it, _ = c.solve(S, tol=1e-13)
        assert (it > 0).all()
        assert c.mismatch(S, V).max() <= 1e-10
        for t in range(0, S.shape[0], max(1, S.shape[0] // 10)):
            assert O.contraction_certificate(c.K, S[t], V[t]) < 1.0


def test_mismatch_is_the_power_balance_away_from_the_solution():
    """The oracle's mismatch (Eq. 1's power balance, S = load) pinned by branch currents written out
    by hand: at a wrong V it is the imbalance of each bus's drawn power, not a small number.

    Two buses: the power drawn at bus 1 is v conj((v0 - v)/z), so the imbalance is
    |v conj((v - v0)/z) + s|; zero at both roots of the two-bus quadratic (the low root is a
    power-flow solution too), and of the size of the perturbation elsewhere.  Three buses in a chain
    0 - 1 - 2: with branch currents I_01 = (v0 - v1)/z1 and I_12 = (v1 - v2)/z2, bus 1 draws
    v1 conj(I_01 - I_12) and bus 2 draws v2 conj(I_12); the mismatch is the larger imbalance."""
    z, s, v0 = fig2()
    c = two_bus_case(z, v0)
    hi, lo = O.two_bus_roots(z, s, v0)
    S = np.array([[s]])
    for v in (hi, lo):
        assert c.mismatch(S, np.array([[v]]))[0] < 1e-14
    for eps in (1e-6, 1e-6j, 1e-3 * (1 + 1j), -2e-2):
        v = hi + eps
        got = c.mismatch(S, np.array([[v]]))[0]
        want = power_balance(v, z, s, v0)
        assert want > 1e-7 and got == pytest.approx(want, rel=1e-10)
    z1, z2 = 0.02 + 0.04j, 0.05 + 0.03j
    s1, s2 = 0.8 + 0.3j, 0.6 + 0.25j
    vs = 1.02 + 0.01j
    c3 = O.Case(3, [0, 1], [1, 2], [z1, z2], slack=0, vs=vs)
    S3 = np.array([[s1, s2]])
    V3, it3, _ = c3.solve(S3, tol=1e-14, max_iter=500)
    assert it3[0] > 0

    def by_hand(v1, v2):
        i01, i12 = (vs - v1) / z1, (v1 - v2) / z2
        return max(abs(v1 * np.conj(i01 - i12) - s1), abs(v2 * np.conj(i12) - s2))

    assert by_hand(*V3[0]) < 1e-13 and c3.mismatch(S3, V3)[0] < 1e-13
    for d1, d2 in ((0.0, 1e-5), (3e-4j, 0.0), (1e-2, -1e-2j)):
        Vw = V3 + np.array([[d1, d2]])
        got = c3.mismatch(S3, Vw)[0]
        want = by_hand(*Vw[0])
        assert want > 1e-7 and got == pytest.approx(want, rel=1e-10)


def test_stopping_rule_counts_updates():
    """iters = number of updates applied; the returned V is that many steps from the start."""
    f, c, S = _config1(64)
    V, it, d = c.solve(S, tol=1e-10)
    for t in (0, 17, 63):
        k = int(it[t])
        Vk, itk, _ = c.solve(S[t:t + 1], tol=0.0, max_iter=k)
        assert np.array_equal(Vk[0], V[t]) and itk[0] == -k
        Vk1, _, dk1 = c.solve(S[t:t + 1], tol=0.0, max_iter=k - 1)
        assert np.abs(V[t] - Vk1[0]).max() == pytest.approx(d[t], rel=1e-12, abs=0)
        assert d[t] <= 1e-10 < np.abs(Vk1[0] - c.solve(S[t:t + 1], tol=0.0, max_iter=k - 2)[0][0]).max()


@pytest.mark.parametrize("n_bus,seed", [(3, 11), (4, 12)])
def test_tiny_feeders_brute_force(n_bus, seed):
    """All roots by NR from many starts; the FPI returns the one with the largest min |V|."""
    f = G.make_feeder(n_bus, seed)
    c = O.Case.from_feeder(f)
    rng = np.random.default_rng(seed)
    s_dir = rng.uniform(0.5, 3.0, n_bus - 1) + 1j * rng.uniform(0.2, 1.0, n_bus - 1)
    lo_, hi_ = 0.0, 1.0 / np.abs(c.K).max()
    while c.solve(hi_ * s_dir[None, :], tol=1e-9, max_iter=400)[1][0] > 0:
        hi_ *= 2
    for _ in range(30):  # loadability limit along s_dir (approximate: slow convergence near it)
        mid = 0.5 * (lo_ + hi_)
        lo_, hi_ = (mid, hi_) if c.solve(mid * s_dir[None, :], tol=1e-9, max_iter=400)[1][0] > 0 else (lo_, mid)
    s = 0.85 * lo_ * s_dir  # near the nose the low-voltage roots are within NR's reach
    V, it, _ = c.solve(s[None, :], tol=1e-13, max_iter=20000)
    assert it[0] > 0
    Ysp = c.ybus_sparse()
    roots = []
    for _ in range(300):
        v_init = rng.uniform(0.05, 1.1, n_bus - 1) * np.exp(1j * rng.uniform(-0.8, 0.3, n_bus - 1))
        v, _, ok = O.nr_solve(Ysp, 0, f.v0, f.pq_bus, s, v_init=v_init, tol=1e-11, max_iter=25)
        if ok and not any(np.abs(v - r).max() < 1e-7 for r in roots):
            roots.append(v)
    assert len(roots) >= 2  # the high root and at least one low-voltage root
    best = max(roots, key=lambda r: np.abs(r).min())
    assert np.abs(best - V[0]).max() < 1e-9


@pytest.mark.parametrize("mistake", ["K_sign", "no_conj", "no_W", "K_conj"])
def test_pins_catch_planted_mistakes(mistake):
    """A plausible mistake planted in the oracle's inputs fails the two-bus closed-form pin."""
    z, s, v0 = fig2()
    c = two_bus_case(z, v0)
    K, W, S = c.K.copy(), c.W.copy(), np.array([[s]])
    if mistake == "K_sign":
        K = -K
    elif mistake == "no_conj":
        S = np.conj(S)  # conj(S/V) would become S/conj(V)... i.e. the load current's conjugate dropped
    elif mistake == "no_W":
        W = np.zeros_like(W)
    elif mistake == "K_conj":
        K = np.conj(K)
    V, it, _ = O.fpi(K, W, S, tol=1e-13, max_iter=500)
    hi, _ = O.two_bus_roots(z, s, v0)
    assert not (it[0] > 0 and abs(V[0, 0] - hi) < 1e-6)
