"""Oracle for the tensor power flow -- TEST INFRASTRUCTURE ONLY.

Plain, slow, double-precision CPU implementations used to check the CUDA library.  Only the
tests, the smoke check and the benchmark's CPU legs (the timed CPU baseline, the reference arm,
and the accuracy checks against this oracle that follow each timed region) may import this
module; the library never does, and the two share no code (inputs come from
``paper_2403_04578_gb300.inputs``, which holds no power-flow arithmetic).

Contents, each following the passage it cites:

* ``build()`` / ``lib()`` compile and load ``fpi.c`` (Eq. 1-3, Eq. 12, Algorithm 1).
* ``ybus``, ``precompute``, ``fpi``, ``mismatch`` -- thin ctypes wrappers over ``fpi.c``.
* ``fpi_zip``, ``mismatch_zip`` -- Eq. 3 with ZIP loads, column by column (per-column B, F and w),
  and the ZIP power balance (``fpi.c``).
* ``Case`` / ``PolyCase`` -- a feeder prepared for the oracle (Y, K, W and the bus bookkeeping);
  ``PolyCase`` builds Y from phases x phases branch blocks (Eq. 1 with phi > 1).
* ``nr_solve`` -- an independent sparse polar Newton-Raphson (the "NR (Sparse)" method the paper
  compares against in Sec. V), used to cross-check the fixed-point solution.
* ``two_bus_roots``, ``feasible_eq10``, ``two_bus_contraction`` -- the two-bus closed forms of
  Sec. III (Eq. 5-10) and the contraction ratio of Eq. 11.
* ``contraction_certificate`` -- the column-norm contraction factor of Eq. 9-11 evaluated at a
  solution.
* ``path_sum_K`` -- the bus-impedance path-sum of a radial feeder (follows from Eq. 1 and the
  Z_B remark after Eq. 11); pins the dense inverse.

Every function is pinned in ``tests/test_oracle_pins.py`` (dense FPI, NR, two-bus closed forms and
geometry), ``tests/test_oracle_zip.py`` (ZIP loads) and ``tests/test_oracle_poly.py`` (polyphase);
the learned start's reference network (``oracle/mlp.py``) in ``tests/test_oracle_mlp.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_c128p = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``fpi.c`` into ``oracle/_build/liboracle.so`` (gcc, OpenMP, no fast-math)."""
    src = os.path.join(_HERE, "fpi.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_build_ybus.argtypes = [ctypes.c_int, ctypes.c_int, _i32p, _i32p, _c128p, _c128p]
            L.orc_build_ybus.restype = ctypes.c_int
            L.orc_invert.argtypes = [ctypes.c_int, _c128p]
            L.orc_invert.restype = ctypes.c_int
            L.orc_precompute.argtypes = [ctypes.c_int, _c128p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         _i32p, _c128p, _c128p]
            L.orc_precompute.restype = ctypes.c_int
            L.orc_fpi.argtypes = [ctypes.c_int, _c128p, _c128p, ctypes.c_long, _c128p, ctypes.c_void_p,
                                  ctypes.c_double, ctypes.c_int, _c128p, _i32p, _f64p, ctypes.c_int]
            L.orc_fpi.restype = None
            L.orc_mismatch.argtypes = [ctypes.c_int, _c128p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, _i32p,
                                       ctypes.c_long, _c128p, _c128p, _f64p]
            L.orc_mismatch.restype = None
            L.orc_build_ybus_poly.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _i32p, _i32p, _c128p, _c128p]
            L.orc_build_ybus_poly.restype = ctypes.c_int
            L.orc_fpi_zip.argtypes = [ctypes.c_int, _c128p, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      _i32p, _f64p, ctypes.c_long, _c128p, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
                                      _c128p, _i32p, _f64p, ctypes.c_int]
            L.orc_fpi_zip.restype = None
            L.orc_mismatch_zip.argtypes = [ctypes.c_int, _c128p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, _i32p, _f64p, ctypes.c_long, _c128p, _c128p, _f64p]
            L.orc_mismatch_zip.restype = None
            _lib = L
        return _lib


def _cd(z: complex):
    return float(np.real(z)), float(np.imag(z))


def ybus(n_bus: int, from_bus, to_bus, z_pu) -> np.ndarray:
    """Dense nodal admittance matrix of Eq. 1 (no shunts)."""
    Y = np.zeros((n_bus, n_bus), dtype=np.complex128)
    rc = lib().orc_build_ybus(n_bus, len(from_bus), np.ascontiguousarray(from_bus, np.int32),
                              np.ascontiguousarray(to_bus, np.int32), np.ascontiguousarray(z_pu, np.complex128), Y)
    if rc:
        raise ValueError(f"bad branch data (code {rc})")
    return Y


def precompute(Y: np.ndarray, slack: int, vs: complex, pq) -> tuple[np.ndarray, np.ndarray]:
    """K = -Y_dd^{-1} and W = K Y_ds v_s (Eq. 3, constant power, Alg. 1's Z_B and W)."""
    pq = np.ascontiguousarray(pq, np.int32)
    n = pq.shape[0]
    K = np.zeros((n, n), dtype=np.complex128)
    W = np.zeros(n, dtype=np.complex128)
    if lib().orc_precompute(Y.shape[0], np.ascontiguousarray(Y), int(slack), *_cd(vs), n, pq, K, W):
        raise np.linalg.LinAlgError("Y_dd is singular")
    return K, W


def fpi(K: np.ndarray, W: np.ndarray, S: np.ndarray, V0: np.ndarray | None = None, tol: float = 1e-13,
        max_iter: int = 100, threads: int = 0):
    """Algorithm 1 per column: returns (V [T][n], iters [T], last_delta [T])."""
    S = np.ascontiguousarray(S, np.complex128)
    T, n = S.shape
    V = np.empty_like(S)
    iters = np.empty(T, dtype=np.int32)
    delta = np.empty(T, dtype=np.float64)
    v0p = None
    if V0 is not None:
        V0 = np.ascontiguousarray(V0, np.complex128)
        assert V0.shape == S.shape
        v0p = V0.ctypes.data
    lib().orc_fpi(n, np.ascontiguousarray(K, np.complex128), np.ascontiguousarray(W, np.complex128), T, S, v0p,
                  float(tol), int(max_iter), V, iters, delta, int(threads))
    return V, iters, delta


def mismatch(Y: np.ndarray, slack: int, vs: complex, pq, S: np.ndarray, V: np.ndarray) -> np.ndarray:
    """max_i |V_i conj((Y v)_i) + S_i| per column (power balance of Eq. 1, S = load)."""
    S = np.ascontiguousarray(S, np.complex128)
    V = np.ascontiguousarray(V, np.complex128)
    out = np.empty(S.shape[0], dtype=np.float64)
    pq = np.ascontiguousarray(pq, np.int32)
    lib().orc_mismatch(Y.shape[0], np.ascontiguousarray(Y), int(slack), *_cd(vs), pq.shape[0], pq, S.shape[0], S,
                       V, out)
    return out


def fpi_zip(Y: np.ndarray, slack: int, vs: complex, pq, alpha, S: np.ndarray, V0: np.ndarray | None = None,
            tol: float = 1e-13, max_iter: int = 100, threads: int = 0):
    """Eq. 3 with ZIP loads, column by column (alpha = [alpha_P, alpha_I, alpha_Z], each [n_pq]):
    F = -B^{-1} A and w = -B^{-1} c of each column's operating point, v <- F conj(v)^{-1} + w.
    Returns (V, iters, last_delta) like fpi."""
    S = np.ascontiguousarray(S, np.complex128)
    T, n = S.shape
    alpha = np.ascontiguousarray(alpha, np.float64).reshape(3, n)
    pq = np.ascontiguousarray(pq, np.int32)
    V = np.empty_like(S)
    iters = np.empty(T, dtype=np.int32)
    delta = np.empty(T, dtype=np.float64)
    v0p = None
    if V0 is not None:
        V0 = np.ascontiguousarray(V0, np.complex128)
        assert V0.shape == S.shape
        v0p = V0.ctypes.data
    lib().orc_fpi_zip(Y.shape[0], np.ascontiguousarray(Y), int(slack), *_cd(vs), n, pq, alpha, T, S, v0p, float(tol),
                      int(max_iter), V, iters, delta, int(threads))
    return V, iters, delta


def mismatch_zip(Y: np.ndarray, slack: int, vs: complex, pq, alpha, S: np.ndarray, V: np.ndarray) -> np.ndarray:
    """max_i |V_i| |(Y v)_i + i_d,i| per column with the ZIP demand current of Eq. 3."""
    S = np.ascontiguousarray(S, np.complex128)
    V = np.ascontiguousarray(V, np.complex128)
    pq = np.ascontiguousarray(pq, np.int32)
    alpha = np.ascontiguousarray(alpha, np.float64).reshape(3, pq.shape[0])
    out = np.empty(S.shape[0], dtype=np.float64)
    lib().orc_mismatch_zip(Y.shape[0], np.ascontiguousarray(Y), int(slack), *_cd(vs), pq.shape[0], pq, alpha,
                           S.shape[0], S, V, out)
    return out


class PolyCase:
    """A polyphase feeder for the oracle (Eq. 1 with phases > 1): nodes are (bus, phase), index
    b*phases + p; the demand unknowns are ordered bus-major over pq (i*phases + p), the slack
    bus's phases hold vs[0..phases).  K = -Y_dd^{-1} by Gauss-Jordan, W = K Y_ds v_s, and the
    fixed-point iteration of Algorithm 1 (orc_fpi) are the single-phase ones on this index space."""

    def __init__(self, n_bus, from_bus, to_bus, z_blocks, phases, slack=0, vs=None, pq=None, with_k=True):
        """with_k=False skips K and W (the O(n^3) inverse): the case then only evaluates mismatches."""
        self.n_bus, self.phases, self.slack = int(n_bus), int(phases), int(slack)
        ph = self.phases
        z = np.ascontiguousarray(z_blocks, np.complex128).reshape(len(from_bus), ph, ph)
        N = self.n_bus * ph
        self.Y = np.zeros((N, N), dtype=np.complex128)
        rc = lib().orc_build_ybus_poly(self.n_bus, len(from_bus), ph, np.ascontiguousarray(from_bus, np.int32),
                                       np.ascontiguousarray(to_bus, np.int32), z, self.Y)
        if rc:
            raise ValueError(f"bad branch data (code {rc})")
        pq = np.asarray(pq if pq is not None else [b for b in range(self.n_bus) if b != slack], np.int64)
        self.vs = np.asarray(vs if vs is not None else np.exp(-2j * np.pi * np.arange(ph) / ph), np.complex128)
        self.nodes = (pq[:, None] * ph + np.arange(ph)[None, :]).reshape(-1)
        self.snodes = self.slack * ph + np.arange(ph)
        if not with_k:
            self.K = self.W = None
            return
        Ydd = np.ascontiguousarray(self.Y[np.ix_(self.nodes, self.nodes)])
        self.K = Ydd.copy()
        if lib().orc_invert(self.K.shape[0], self.K):
            raise np.linalg.LinAlgError("Y_dd is singular")
        self.K = -self.K
        self.W = self.K @ (self.Y[np.ix_(self.nodes, self.snodes)] @ self.vs)

    def solve(self, S, V0=None, tol=1e-13, max_iter=100, threads=0):
        """S: [T][n_pq*phases] loads (bus-major)."""
        return fpi(self.K, self.W, S, V0, tol, max_iter, threads)

    def mismatch(self, S, V):
        """max over demand nodes of |V_i conj((Y v)_i) + S_i| per column."""
        S = np.atleast_2d(np.asarray(S, np.complex128))
        V = np.atleast_2d(np.asarray(V, np.complex128))
        full = np.empty((V.shape[0], self.Y.shape[0]), dtype=np.complex128)
        full[:, self.snodes] = self.vs
        full[:, self.nodes] = V
        acc = full @ self.Y.T
        return np.abs(V * np.conj(acc[:, self.nodes]) + S).max(axis=1)


class Case:
    """A feeder prepared for the oracle: Y, K, W and the bus bookkeeping."""

    def __init__(self, n_bus, from_bus, to_bus, z_pu, slack=0, vs=1.0 + 0j, pq=None):
        self.n_bus = int(n_bus)
        self.from_bus = np.asarray(from_bus, np.int32)
        self.to_bus = np.asarray(to_bus, np.int32)
        self.z_pu = np.asarray(z_pu, np.complex128)
        self.slack = int(slack)
        self.vs = complex(vs)
        self.pq = np.asarray(pq if pq is not None else [b for b in range(n_bus) if b != slack], np.int32)
        self.Y = ybus(self.n_bus, self.from_bus, self.to_bus, self.z_pu)
        self.K, self.W = precompute(self.Y, self.slack, self.vs, self.pq)

    @classmethod
    def from_feeder(cls, f):
        return cls(f.n_bus, f.from_bus, f.to_bus, f.z_pu, f.slack, f.v0, f.pq_bus)

    def solve(self, S, V0=None, tol=1e-13, max_iter=100, threads=0):
        return fpi(self.K, self.W, S, V0, tol, max_iter, threads)

    def mismatch(self, S, V):
        return mismatch(self.Y, self.slack, self.vs, self.pq, S, V)

    def solve_zip(self, S, alpha, V0=None, tol=1e-13, max_iter=100, threads=0):
        return fpi_zip(self.Y, self.slack, self.vs, self.pq, alpha, S, V0, tol, max_iter, threads)

    def mismatch_zip(self, S, alpha, V):
        return mismatch_zip(self.Y, self.slack, self.vs, self.pq, alpha, S, V)

    def ybus_sparse(self):
        return sp.csr_matrix(self.Y)


# ---------------------------------------------------------------------------------------------
# Independent check: sparse polar Newton-Raphson ("NR (Sparse)" of Sec. V).
# ---------------------------------------------------------------------------------------------

def nr_solve(Ysp, slack: int, vs: complex, pq, s_load, v_init=None, tol: float = 1e-12, max_iter: int = 40):
    """Polar Newton-Raphson on the PQ-bus power balance.  Returns (V_pq, iterations, converged).

    Unknowns are the angles and magnitudes of the PQ buses; the mismatch is
    V_i conj((Y V)_i) + S_i = 0 (the injection of a load bus is minus its load).  The Jacobian uses
    the standard complex-power derivatives dS/dVa = j diag(V) conj(diag(I) - Y diag(V)) and
    dS/dVm = diag(V) conj(Y diag(V/|V|)) + conj(diag(I)) diag(V/|V|), with I = Y V, and each step
    is one sparse LU solve.
    """
    Ysp = sp.csr_matrix(Ysp)
    n_bus = Ysp.shape[0]
    pq = np.asarray(pq)
    npq = pq.shape[0]
    V = np.ones(n_bus, dtype=np.complex128)
    V[slack] = vs
    V[pq] = 1.0 if v_init is None else np.asarray(v_init, np.complex128)
    Va, Vm = np.angle(V), np.abs(V)
    s_inj = -np.asarray(s_load, np.complex128)
    for it in range(max_iter + 1):
        I = Ysp @ V
        mis = V[pq] * np.conj(I[pq]) - s_inj
        F = np.r_[mis.real, mis.imag]
        if np.max(np.abs(F)) <= tol:
            return V[pq].copy(), it, True
        if it == max_iter or not np.all(np.isfinite(F)):
            break
        dV = sp.diags(V)
        dI = sp.diags(I)
        dVn = sp.diags(V / np.abs(V))
        dS_dVa = 1j * dV @ np.conj(dI - Ysp @ dV)
        dS_dVm = dV @ np.conj(Ysp @ dVn) + np.conj(dI) @ dVn
        A = sp.csr_matrix(dS_dVa)[pq][:, pq]
        B = sp.csr_matrix(dS_dVm)[pq][:, pq]
        J = sp.bmat([[A.real, B.real], [A.imag, B.imag]], format="csc")
        try:
            dx = spla.splu(J).solve(-F)
        except RuntimeError:
            break
        Va[pq] += dx[:npq]
        Vm[pq] += dx[npq:]
        V = Vm * np.exp(1j * Va)
    return V[pq].copy(), max_iter, False


# ---------------------------------------------------------------------------------------------
# Two-bus closed forms (Sec. III) and the contraction factor (Eq. 9-11).
# ---------------------------------------------------------------------------------------------

def two_bus_roots(z: complex, s: complex, v0: complex = 1.0):
    """Both solutions of the two-bus system (slack v0, series z, load s at bus 1).

    From v = v0 - z conj(s / v):  |v|^2 = v0 conj(v) - z conj(s), so u = |v|^2 solves
    u^2 - a u + |z|^2 |s|^2 = 0 with a = |v0|^2 - 2 Re(z conj(s)), and then
    v = conj((u + z conj(s)) / v0).  Returns (v_high, v_low), or None if a^2 < 4|z|^2|s|^2
    (no real root: the load is infeasible).
    """
    a = abs(v0) ** 2 - 2.0 * (z * np.conj(s)).real
    disc = a * a - 4.0 * abs(z) ** 2 * abs(s) ** 2
    if disc < 0:
        return None
    out = []
    for u in ((a + np.sqrt(disc)) / 2.0, (a - np.sqrt(disc)) / 2.0):
        out.append(complex(np.conj((u + z * np.conj(s)) / v0)))
    return out[0], out[1]


def feasible_eq10(z: complex, s: complex, v0: complex = 1.0) -> bool:
    """Eq. 10's sufficient condition for a two-bus solution: |v0|^2 >= 4 |s| |z|."""
    return abs(v0) ** 2 >= 4.0 * abs(s) * abs(z)


def two_bus_contraction(z: complex, s: complex, v: complex) -> float:
    """Eq. 11 for two buses: k = |z_s| / |z_l| with the load impedance |z_l| = |v|^2 / |s|."""
    return abs(z) * abs(s) / abs(v) ** 2


def contraction_certificate(K: np.ndarray, s: np.ndarray, v: np.ndarray) -> float:
    """Eq. 9-11 at a solution: k = || K diag(s ./ |v|^2) ||_1 (largest column sum of moduli).

    ``diag(1 ./ z_l)`` of Eq. 9 is ``diag(conj(s) ./ |v|^2)``; conjugation does not change the
    moduli, so the column norm uses |s_j| / |v_j|^2.
    """
    w = np.abs(s) / np.abs(v) ** 2
    return float(np.max(np.sum(np.abs(K), axis=0) * w))


def path_sum_K(n_bus: int, from_bus, to_bus, z_pu, slack: int = 0) -> np.ndarray:
    """K = -Y_dd^{-1} of a radial, shunt-free feeder from the path-sum of branch impedances.

    (Y_dd^{-1})_{ij} is the total impedance of the branches shared by the slack-to-i and
    slack-to-j paths.  Returned over the PQ buses in increasing bus order.
    """
    parent = -np.ones(n_bus, dtype=np.int64)
    zb = np.zeros(n_bus, dtype=np.complex128)
    for a, b, z in zip(from_bus, to_bus, z_pu):
        parent[b] = a
        zb[b] = z
    pq = [b for b in range(n_bus) if b != slack]
    paths = {}
    for b in pq:
        p, edges = b, []
        while p != slack:
            edges.append(p)
            p = parent[p]
            if p < 0:
                raise ValueError("not a tree rooted at the slack")
        paths[b] = set(edges)
    n = len(pq)
    K = np.zeros((n, n), dtype=np.complex128)
    for i, bi in enumerate(pq):
        for j, bj in enumerate(pq):
            K[i, j] = -sum(zb[e] for e in paths[bi] & paths[bj])
    return K
