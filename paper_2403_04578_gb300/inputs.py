"""Seeded synthetic inputs for the tensor power flow: radial feeders and load tensors.

This module only draws random numbers and shapes them into network data and load profiles.  It
holds none of the power-flow arithmetic (no admittance matrix, no inverse, no iteration), so both
the CUDA library and the CPU oracle can take their inputs from it without sharing any of the
method.

Recipe (stands in for the paper's k-ary-tree networks and copula load profiles, Sec. V, whose
data are not available):

* Feeder: ``n_bus`` buses, bus 0 is the slack at ``v0 = 1+0j`` pu (11 kV, 1 MVA base, so
  ``Z_base = 121 ohm``).  Bus ``i >= 1`` hangs off a uniformly drawn earlier bus whose depth is
  below ``max_depth`` (tree depth <= 12).  Lines: ``r ~ U(0.1, 0.6)`` ohm/km, ``x ~ U(0.05, 0.4)``
  ohm/km, length ``~ U(0.2, 1.5)`` km, no shunts.
* Loads: ``P = lam * base_i * shape(hour) * lognormal(0, 0.2)``, ``base_i ~ U(20, 150)`` kW,
  ``Q = P * tan(acos(pf_i))`` with ``pf_i ~ U(0.95, 0.99)`` lagging.  S is *consumption*
  (positive = load).  ``shape`` is a daily double peak (morning 8 h, evening 19 h) scaled to a
  maximum of 1.
* Load scale ``lam = min(1, drop_target / drop_lin)``: ``drop_lin`` is the largest first-order
  (linear, lossless) voltage drop ``sum_path (r_e P_e + x_e Q_e)`` of the peak column (shape 1,
  noise 1, largest scenario factor).  Without it the literal recipe has no power-flow solution
  at several hundred buses and up; the scale keeps the heaviest column near 0.90 pu.

Random streams are Philox keyed by ``(seed, purpose)``; load noise is drawn in fixed chunks of
``CHUNK`` columns, each with its own counter, so any chunk can be regenerated on its own.
"""
from __future__ import annotations

import dataclasses
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

Z_BASE_OHM = (11e3 ** 2) / 1e6  # 121 ohm
S_BASE_KW = 1000.0  # 1 MVA
CHUNK = 4096  # columns per independently seeded noise chunk
DROP_TARGET = 0.092  # linear drop of the peak column after scaling (peak column ~0.90 pu)

_TAG_TREE, _TAG_LOAD, _TAG_PV, _TAG_SCEN, _TAG_BATCH = 1, 2, 3, 4, 5


def _rng(seed: int, tag: int, chunk: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(tag)], counter=[0, int(chunk), 0, 0]))


@dataclasses.dataclass
class Feeder:
    """A radial feeder: branch list in per-unit plus the per-bus load parameters."""

    n_bus: int
    from_bus: np.ndarray  # int32 [n_branch], parent bus of each branch
    to_bus: np.ndarray  # int32 [n_branch], child bus of each branch
    z_pu: np.ndarray  # complex128 [n_branch], series impedance r + jx in pu
    depth: np.ndarray  # int32 [n_bus]
    base_kw: np.ndarray  # float64 [n_bus], 0 at the slack
    pf: np.ndarray  # float64 [n_bus]
    load_scale: float  # lam, already folded into load tensors, recorded for reports
    seed: int
    slack: int = 0
    v0: complex = 1.0 + 0.0j

    @property
    def n_branch(self) -> int:
        return int(self.from_bus.shape[0])

    @property
    def pq_bus(self) -> np.ndarray:
        """PQ buses in increasing bus order (every bus but the slack)."""
        return np.array([b for b in range(self.n_bus) if b != self.slack], dtype=np.int32)

    @property
    def n_pq(self) -> int:
        return self.n_bus - 1

    def pq_params(self):
        pq = self.pq_bus
        return self.base_kw[pq], self.pf[pq]


def daily_shape(hour: np.ndarray) -> np.ndarray:
    """Double-peak daily load shape, maximum 1 (morning peak 8 h, evening peak 19 h)."""
    h = np.asarray(hour, dtype=np.float64)

    def raw(x):
        return 0.3 + 0.5 * np.exp(-0.5 * ((x - 8.0) / 1.5) ** 2) + 0.7 * np.exp(-0.5 * ((x - 19.0) / 2.0) ** 2)

    grid = np.linspace(0.0, 24.0, 24 * 3600 + 1)
    return raw(h) / raw(grid).max()


def clear_sky(hour: np.ndarray) -> np.ndarray:
    """Clear-sky PV bell, 0 at night, 1 at solar noon (12 h)."""
    h = np.asarray(hour, dtype=np.float64)
    return np.maximum(0.0, np.sin(np.pi * (h - 6.0) / 12.0))


def _linear_drop(parent: np.ndarray, depth: np.ndarray, r: np.ndarray, x: np.ndarray,
                 p: np.ndarray, q: np.ndarray) -> float:
    """Largest first-order voltage drop sum_path (r_e P_e + x_e Q_e) for bus loads p, q (pu).

    ``r, x`` are indexed by the child bus of each branch.  This is the input recipe's load-scale
    heuristic (a lossless linear drop), not a power-flow solve.
    """
    n = parent.shape[0]
    order = np.argsort(depth, kind="stable")
    pe, qe = p.copy(), q.copy()
    for b in order[::-1]:  # children before parents: accumulate downstream load
        if b != 0:
            pe[parent[b]] += pe[b]
            qe[parent[b]] += qe[b]
    drop = np.zeros(n)
    for b in order:
        if b != 0:
            drop[b] = drop[parent[b]] + r[b] * pe[b] + x[b] * qe[b]
    return float(drop.max())


def make_feeder(n_bus: int, seed: int, max_depth: int = 12, peak_factor: float = 1.0,
                drop_target: float = DROP_TARGET) -> Feeder:
    """Grow a radial feeder of ``n_bus`` buses (bus 0 = slack) from ``seed``.

    ``peak_factor`` is the largest multiplier any column applies to the base loads (the largest
    scenario factor); the load scale is chosen for that column.
    """
    if n_bus < 2:
        raise ValueError("a feeder needs the slack and at least one PQ bus")
    rng = _rng(seed, _TAG_TREE)
    parent = np.zeros(n_bus, dtype=np.int64)
    depth = np.zeros(n_bus, dtype=np.int64)
    for i in range(1, n_bus):
        eligible = np.flatnonzero(depth[:i] < max_depth)
        p = int(eligible[rng.integers(eligible.shape[0])])
        parent[i] = p
        depth[i] = depth[p] + 1
    r_km = rng.uniform(0.1, 0.6, n_bus)
    x_km = rng.uniform(0.05, 0.4, n_bus)
    length = rng.uniform(0.2, 1.5, n_bus)
    base_kw = rng.uniform(20.0, 150.0, n_bus)
    pf = rng.uniform(0.95, 0.99, n_bus)
    base_kw[0] = 0.0
    pf[0] = 1.0
    r_pu = r_km * length / Z_BASE_OHM
    x_pu = x_km * length / Z_BASE_OHM
    p_pk = base_kw / S_BASE_KW * peak_factor
    q_pk = p_pk * np.tan(np.arccos(pf))
    drop = _linear_drop(parent, depth, r_pu, x_pu, p_pk, q_pk)
    lam = min(1.0, drop_target / drop) if drop > 0 else 1.0
    kids = np.arange(1, n_bus)
    return Feeder(
        n_bus=n_bus,
        from_bus=parent[kids].astype(np.int32),
        to_bus=kids.astype(np.int32),
        z_pu=(r_pu[kids] + 1j * x_pu[kids]).astype(np.complex128),
        depth=depth.astype(np.int32),
        base_kw=base_kw,
        pf=pf,
        load_scale=lam,
        seed=seed,
    )


def _noise_chunk(seed: int, chunk: int, n_cols: int, n_pq: int, tag: int = _TAG_LOAD) -> np.ndarray:
    rng = _rng(seed, tag, chunk)
    return np.exp(0.2 * rng.standard_normal((n_cols, n_pq)))


def load_tensor(feeder: Feeder, T: int, seed: int, step_minutes: float = 1.0, t0: int = 0,
                dtype=np.complex128, threads: int = 8, out: np.ndarray | None = None) -> np.ndarray:
    """Load tensor S[T][n_pq] (consumption, pu) for ``T`` consecutive steps starting at ``t0``.

    ``t0`` must be a multiple of ``CHUNK`` so that chunk seeding lines up with a full run.  ``out``
    (optional) is a C-contiguous [T][n_pq] array to fill, e.g. a view of pinned host memory.
    """
    if t0 % CHUNK:
        raise ValueError("t0 must be a multiple of CHUNK")
    base, pf = feeder.pq_params()
    p0 = feeder.load_scale * base / S_BASE_KW
    tanphi = np.tan(np.arccos(pf))
    if out is None:
        out = np.empty((T, feeder.n_pq), dtype=dtype)
    elif out.shape != (T, feeder.n_pq) or not out.flags.c_contiguous:
        raise ValueError("out must be C-contiguous with shape (T, n_pq)")
    n_chunks = (T + CHUNK - 1) // CHUNK

    def work(c):
        a, b = c * CHUNK, min(T, (c + 1) * CHUNK)
        hours = ((t0 + np.arange(a, b)) * step_minutes / 60.0) % 24.0
        noise = _noise_chunk(seed, t0 // CHUNK + c, CHUNK, feeder.n_pq)[: b - a]
        p = p0[None, :] * daily_shape(hours)[:, None] * noise
        out[a:b].real = p
        out[a:b].imag = p * tanphi[None, :]

    if n_chunks == 1 or threads <= 1:
        for c in range(n_chunks):
            work(c)
    else:
        with ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(work, range(n_chunks)))
    return out


def scenario_tensor(feeder: Feeder, n_scen: int, n_hours: int, seed: int,
                    factor_range=(0.5, 1.8), pv_fraction: float = 0.3, pv_kw_max: float = 8.0,
                    dtype=np.complex64, threads: int = 8) -> np.ndarray:
    """Scenario x time load tensor S[scenario, hour, n_pq] (consumption minus PV, pu).

    Each scenario scales the loads by a factor ~ U(factor_range); a fixed ``pv_fraction`` of the
    PQ buses inject ``U(0, pv_kw_max)`` kW (drawn per scenario and bus) times the clear-sky bell,
    with no reactive power.  The feeder should be made with ``peak_factor = factor_range[1]``.
    """
    base, pf = feeder.pq_params()
    n_pq = feeder.n_pq
    p0 = feeder.load_scale * base / S_BASE_KW
    tanphi = np.tan(np.arccos(pf))
    rs = _rng(seed, _TAG_SCEN)
    factor = rs.uniform(factor_range[0], factor_range[1], n_scen)
    rp = _rng(seed, _TAG_PV)
    has_pv = np.zeros(n_pq, dtype=bool)
    has_pv[rp.choice(n_pq, size=int(round(pv_fraction * n_pq)), replace=False)] = True
    pv_kw = rp.uniform(0.0, pv_kw_max, (n_scen, n_pq)) * has_pv[None, :]
    hours = np.arange(n_hours) % 24
    shape = daily_shape(hours)
    bell = clear_sky(hours)
    out = np.empty((n_scen, n_hours, n_pq), dtype=dtype)

    def work(s):
        rng = _rng(seed, _TAG_LOAD, s)
        noise = np.exp(0.2 * rng.standard_normal((n_hours, n_pq)))
        pl = p0[None, :] * shape[:, None] * noise * factor[s]
        ppv = pv_kw[s][None, :] / S_BASE_KW * bell[:, None]
        out[s].real = pl - ppv
        out[s].imag = pl * tanphi[None, :]

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        list(ex.map(work, range(n_scen)))
    return out


def batch_specs(n_feeders: int, seed0: int = 1000, n_range=(20, 2000), t_choices=(96, 288, 1440),
                seed: int = 7):
    """Bus counts (log-uniform in ``n_range``), column counts and seeds of a feeder batch."""
    rng = _rng(seed, _TAG_BATCH)
    n_bus = np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), n_feeders))
    n_bus = np.clip(np.round(n_bus).astype(np.int64), n_range[0], n_range[1])
    T = rng.choice(np.array(t_choices), n_feeders)
    return [(int(n_bus[i]), int(T[i]), seed0 + i) for i in range(n_feeders)]


def step_minutes_for(T: int) -> float:
    """A day split into ``T`` steps (96 -> 15 min, 288 -> 5 min, 1440 -> 1 min)."""
    return 1440.0 / T


def flat_start(T: int, n_pq: int) -> np.ndarray:
    return np.ones((T, n_pq), dtype=np.complex128)


# ---------------------------------------------------------------------------------------------
# The same recipes drawn directly on a CUDA device (torch), for workloads too large to build on
# the host.  The noise comes from torch's device generator seeded from (seed, purpose), so these
# tensors are reproducible for a given torch build but differ from the host recipes' draws; checks
# against the oracle read the sampled columns back from the device.
# ---------------------------------------------------------------------------------------------

def _torch_gen(device, seed: int, tag: int, sub: int = 0):
    import torch

    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1_000_003 + int(tag) * 7_919 + int(sub)) % (2 ** 63))
    return g


def load_tensor_device(feeder: Feeder, T: int, seed: int, device, step_minutes: float = 1.0,
                       dtype=None):
    """Load tensor S[T][n_pq] on ``device`` with the recipe of ``load_tensor`` (complex128 default)."""
    import torch

    dtype = dtype or torch.complex128
    real = torch.float64 if dtype == torch.complex128 else torch.float32
    base, pf = feeder.pq_params()
    p0 = torch.tensor(feeder.load_scale * base / S_BASE_KW, dtype=torch.float64, device=device)
    tanphi = torch.tensor(np.tan(np.arccos(pf)), dtype=torch.float64, device=device)
    hours = torch.tensor((np.arange(T) * step_minutes / 60.0) % 24.0, dtype=torch.float64)
    shape = torch.tensor(daily_shape(hours.numpy()), dtype=torch.float64, device=device)
    noise = torch.randn((T, feeder.n_pq), generator=_torch_gen(device, seed, _TAG_LOAD), device=device,
                        dtype=torch.float64).mul_(0.2).exp_()
    p = noise.mul_(p0[None, :]).mul_(shape[:, None])
    return torch.complex(p.to(real), (p * tanphi[None, :]).to(real)).to(dtype)


def scenario_tensor_device(feeder: Feeder, n_scen: int, n_hours: int, seed: int, device,
                           factor_range=(0.5, 1.8), pv_fraction: float = 0.3, pv_kw_max: float = 8.0):
    """Scenario x time load tensor S[scenario, hour, n_pq], complex64, with the recipe of
    ``scenario_tensor`` (scenario factors, PV buses and PV sizes are the host recipe's draws)."""
    import torch

    base, pf = feeder.pq_params()
    n_pq = feeder.n_pq
    p0 = torch.tensor(feeder.load_scale * base / S_BASE_KW, dtype=torch.float32, device=device)
    tanphi = torch.tensor(np.tan(np.arccos(pf)), dtype=torch.float32, device=device)
    rs = _rng(seed, _TAG_SCEN)
    factor = torch.tensor(rs.uniform(factor_range[0], factor_range[1], n_scen), dtype=torch.float32, device=device)
    rp = _rng(seed, _TAG_PV)
    has_pv = np.zeros(n_pq, dtype=bool)
    has_pv[rp.choice(n_pq, size=int(round(pv_fraction * n_pq)), replace=False)] = True
    pv_kw = torch.tensor(rp.uniform(0.0, pv_kw_max, (n_scen, n_pq)) * has_pv[None, :], dtype=torch.float32,
                         device=device)
    hours = np.arange(n_hours) % 24
    shape = torch.tensor(daily_shape(hours), dtype=torch.float32, device=device)
    bell = torch.tensor(clear_sky(hours), dtype=torch.float32, device=device)
    out = torch.empty((n_scen, n_hours, n_pq), dtype=torch.complex64, device=device)
    g = _torch_gen(device, seed, _TAG_LOAD)
    for s in range(n_scen):
        noise = torch.randn((n_hours, n_pq), generator=g, device=device, dtype=torch.float32).mul_(0.2).exp_()
        pl = noise.mul_(p0[None, :]).mul_(shape[:, None]).mul_(factor[s])
        ppv = pv_kw[s][None, :] / S_BASE_KW * bell[:, None]
        out[s] = torch.complex(pl - ppv, pl * tanphi[None, :])
    return out


# ---------------------------------------------------------------------------------------------
# Polyphase feeders (Eq. 1 with phases > 1): the radial recipe above with a phases x phases
# series impedance per branch and per-phase loads.
# ---------------------------------------------------------------------------------------------

_TAG_POLY = 6


@dataclasses.dataclass
class PolyFeeder:
    """A radial polyphase feeder: per branch a [phases][phases] impedance block (pu)."""

    n_bus: int
    phases: int
    from_bus: np.ndarray  # int32 [n_branch]
    to_bus: np.ndarray  # int32 [n_branch]
    z_blocks: np.ndarray  # complex128 [n_branch][phases][phases]
    base_kw: np.ndarray  # float64 [n_bus][phases], 0 at the slack
    pf: np.ndarray  # float64 [n_bus][phases]
    load_scale: float
    seed: int
    slack: int = 0

    @property
    def n_pq(self) -> int:
        return self.n_bus - 1

    @property
    def pq_bus(self) -> np.ndarray:
        return np.arange(1, self.n_bus, dtype=np.int32)

    @property
    def v0(self) -> np.ndarray:
        """Balanced source (1, a^2, a) for three phases, a = exp(j 2 pi / 3)."""
        return np.exp(-2j * np.pi * np.arange(self.phases) / self.phases)


def make_feeder_poly(n_bus: int, seed: int, phases: int = 3, mutual: float = 0.4, unbalance: float = 0.2,
                     max_depth: int = 12, load_factor: float = 0.8) -> PolyFeeder:
    """Polyphase version of ``make_feeder``: the same tree and line draws; each branch gets the
    self impedance z + z_m and the mutual impedance z_m = mutual * (0.2 r + j x) between phases
    (so its positive-sequence impedance is the single-phase z); each phase of each bus carries
    the single-phase base load times a share in [1 - unbalance, 1 + unbalance] (mean 1), scaled by
    ``load_factor`` times the single-phase feeder's load scale."""
    f = make_feeder(n_bus, seed, max_depth=max_depth)
    z = f.z_pu
    zm = mutual * (0.2 * z.real + 1j * z.imag)
    blocks = np.empty((z.shape[0], phases, phases), dtype=np.complex128)
    blocks[:] = zm[:, None, None]
    for p in range(phases):
        blocks[:, p, p] = z + zm
    rng = _rng(seed, _TAG_POLY)
    share = rng.uniform(1.0 - unbalance, 1.0 + unbalance, (n_bus, phases))
    share /= share.mean(axis=1, keepdims=True)
    base = f.base_kw[:, None] * share
    base[0] = 0.0
    pf = np.repeat(f.pf[:, None], phases, axis=1)
    return PolyFeeder(n_bus=n_bus, phases=phases, from_bus=f.from_bus, to_bus=f.to_bus, z_blocks=blocks,
                      base_kw=base, pf=pf, load_scale=f.load_scale * load_factor, seed=seed)


def load_tensor_poly(feeder: PolyFeeder, T: int, seed: int, step_minutes: float = 1.0) -> np.ndarray:
    """Loads S[T][n_pq][phases] (complex128, consumption), the recipe of ``load_tensor`` per phase."""
    ph = feeder.phases
    base = feeder.base_kw[1:]
    tanphi = np.tan(np.arccos(feeder.pf[1:]))
    hours = (np.arange(T) * step_minutes / 60.0) % 24.0
    rng = _rng(seed, _TAG_LOAD, 1 << 20)
    noise = np.exp(0.2 * rng.standard_normal((T, feeder.n_pq, ph)))
    p = feeder.load_scale * base[None] / S_BASE_KW * daily_shape(hours)[:, None, None] * noise
    return (p + 1j * p * tanphi[None]).astype(np.complex128)
