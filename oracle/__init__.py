"""CPU FP64 oracle of the CT-MHD step: TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded C++ implementation of one RK2 + first-order-flux-correction
step of the paper's constrained-transport MHD method (Sec. 2), written from the paper's
equations in the paper's order (see ``mhd_oracle.cpp`` for the readings it takes). It shares no
code with the CUDA path. Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg of ``bench.py`` may import it; the product package never does.

Arrays use the layout of the product library: ``cons`` is ``(5, nz, ny, nx)`` (rho, rho*u_d,
e_tot) and ``b`` is ``(3, nz, ny, nx)`` with ``b[d][X]`` the normal field on the d-face of cell X
at index_d - 1/2, all float64, periodic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mhd_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

RECON = {"pc": 0, "plm_mc": 1, "plm_minmod": 2, "ppm": 3, "ppm_ep": 4}
RIEMANN = {"hll": 0, "hlld": 1, "llf": 2}
EMF = {"q26": 0, "fs18": 1, "b25a": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, so x86 and Arm agree)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int * 3),
        ("h", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("recon", ctypes.c_int),
        ("riemann", ctypes.c_int),
        ("emf", ctypes.c_int),
        ("fofc_criteria", ctypes.c_int),
        ("eta", ctypes.c_double),
    ]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        _lib.oracle_step.argtypes = [P(_Cfg), P(d), P(d), d, P(ctypes.c_longlong)]
        _lib.oracle_fluxes.argtypes = [P(_Cfg), P(d), P(d), P(d), P(d)]
        _lib.oracle_corner_emfs.argtypes = [P(_Cfg), P(d), P(d), P(d)]
        _lib.oracle_fluxes_jvp.argtypes = [P(_Cfg), P(d), P(d), P(d), P(d), P(d), P(d), P(d), P(d)]
        u8 = P(ctypes.c_ubyte)
        _lib.oracle_step_flags.argtypes = [P(_Cfg), P(d), P(d), d, u8, u8, P(ctypes.c_longlong)]
        _lib.oracle_prim.argtypes = [P(_Cfg), P(d), P(d), P(d)]
        _lib.oracle_recon.argtypes = [P(_Cfg), ctypes.c_int, P(d), ctypes.c_int, P(d), P(d)]
        _lib.oracle_riemann.argtypes = [ctypes.c_int, d, P(d), P(d), d, P(d)]
        _lib.oracle_max_dt.argtypes = [P(_Cfg), P(d), P(d), d]
        _lib.oracle_max_dt.restype = d
        _lib.oracle_divb.argtypes = [P(_Cfg), P(d), P(d), P(d)]
        _lib.oracle_steps_jvp.argtypes = [P(_Cfg), P(d), P(d), P(d), P(d), d, P(d), ctypes.c_int]
        _lib.oracle_count_ops.argtypes = [P(_Cfg), P(d), P(d), d, P(ctypes.c_longlong), P(ctypes.c_longlong),
                                          P(ctypes.c_longlong)]
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Config:
    """Box and scheme. ``shape`` is (nx, ny, nz); ``h`` the cell widths (dx, dy, dz)."""

    shape: tuple
    h: tuple
    gamma: float = 5.0 / 3.0
    recon: str = "plm_mc"
    riemann: str = "hll"
    emf: str = "q26"
    fofc_criteria: int = 3
    eta: float = 0.0

    def c(self) -> _Cfg:
        c = _Cfg()
        for d in range(3):
            c.n[d] = int(self.shape[d])
            c.h[d] = float(self.h[d])
        c.gamma = self.gamma
        c.recon = RECON[self.recon]
        c.riemann = RIEMANN[self.riemann]
        c.emf = EMF[self.emf]
        c.fofc_criteria = int(self.fofc_criteria)
        c.eta = float(self.eta)
        return c


def _check(cfg: Config, cons, b):
    nx, ny, nz = cfg.shape
    assert cons.shape == (5, nz, ny, nx) and b.shape == (3, nz, ny, nx)


def step(cfg: Config, cons: np.ndarray, b: np.ndarray, dt: float):
    """One full step; returns new (cons, b) and the flagged-cell counts of both stages."""
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64).copy()
    b = np.ascontiguousarray(b, dtype=np.float64).copy()
    counts = (ctypes.c_longlong * 2)()
    c = cfg.c()
    _L().oracle_step(ctypes.byref(c), _ptr(cons), _ptr(b), float(dt), counts)
    return cons, b, (int(counts[0]), int(counts[1]))


def step_user_flags(cfg: Config, cons, b, dt: float, flags1=None, flags2=None):
    """One step where the boolean arrays flags1/flags2 (nz, ny, nx) also invalidate cells after
    stage 1 / stage 2 (a user validity criterion)."""
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64).copy()
    b = np.ascontiguousarray(b, dtype=np.float64).copy()
    keep = []

    def u8(f):
        if f is None:
            return None
        a = np.ascontiguousarray(f, dtype=np.uint8)
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))

    counts = (ctypes.c_longlong * 2)()
    c = cfg.c()
    _L().oracle_step_flags(ctypes.byref(c), _ptr(cons), _ptr(b), float(dt), u8(flags1), u8(flags2), counts)
    return cons, b, (int(counts[0]), int(counts[1]))


def fluxes(cfg: Config, cons: np.ndarray, b: np.ndarray):
    """Face fluxes (3, 5, nz, ny, nx) and edge EMFs (3, nz, ny, nx) of one state."""
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    nx, ny, nz = cfg.shape
    F = np.zeros((3, 5, nz, ny, nx))
    E = np.zeros((3, nz, ny, nx))
    c = cfg.c()
    _L().oracle_fluxes(ctypes.byref(c), _ptr(cons), _ptr(b), _ptr(F), _ptr(E))
    return F, E


def fluxes_jvp(cfg: Config, cons, b, dcons, db):
    """Fluxes and EMFs of one state (as `fluxes`) and their directional derivative along
    (dcons, db), exact on the branches the values take: (F, E, dF, dE)."""
    _check(cfg, cons, b)
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (cons, b, dcons, db)]
    nx, ny, nz = cfg.shape
    F, dF = np.zeros((3, 5, nz, ny, nx)), np.zeros((3, 5, nz, ny, nx))
    E, dE = np.zeros((3, nz, ny, nx)), np.zeros((3, nz, ny, nx))
    c = cfg.c()
    _L().oracle_fluxes_jvp(ctypes.byref(c), *[_ptr(x) for x in arrs], _ptr(F), _ptr(E), _ptr(dF), _ptr(dE))
    return F, E, dF, dE


def corner_emfs(cfg: Config, cons: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The four corner EMFs of every edge, (3, 4, nz, ny, nx): [e][q] with q = 0 LB, 1 RB, 2 LT,
    3 RT (L/R the sides of the a-face, B/T of the c-face, a = e+1, c = e+2), as the EMF compute
    scheme (Q26, FS18 or B25a) forms them before the averaging of Eq. (ld04)."""
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    nx, ny, nz = cfg.shape
    C = np.zeros((3, 4, nz, ny, nx))
    c = cfg.c()
    _L().oracle_corner_emfs(ctypes.byref(c), _ptr(cons), _ptr(b), _ptr(C))
    return C


def prim(cfg: Config, cons: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Primitive variables (8, nz, ny, nx): rho, u0, u1, u2, p, cell-averaged b0, b1, b2."""
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    nx, ny, nz = cfg.shape
    P = np.zeros((8, nz, ny, nx))
    c = cfg.c()
    _L().oracle_prim(ctypes.byref(c), _ptr(cons), _ptr(b), _ptr(P))
    return P


def recon(cfg: Config, method: str, q: np.ndarray, d: int):
    """Reconstruct the periodic array q (nz, ny, nx) along d: (value at X-1/2, value at X+1/2)."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    qm = np.zeros_like(q)
    qp = np.zeros_like(q)
    c = cfg.c()
    _L().oracle_recon(ctypes.byref(c), RECON[method], _ptr(q), int(d), _ptr(qm), _ptr(qp))
    return qm, qp


def riemann(solver: str, gamma: float, WL, WR, bn: float):
    """One face problem in the face frame; W = (rho, u_n, u_t1, u_t2, p, b_t1, b_t2).

    Returns (flux[5] of rho, m_n, m_t1, m_t2, e_tot; alpha+; alpha-; u*)."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    out = np.zeros(8)
    _L().oracle_riemann(RIEMANN[solver], float(gamma), _ptr(WL), _ptr(WR), float(bn), _ptr(out))
    return out[:5].copy(), out[5], out[6], out[7]


def max_dt(cfg: Config, cons: np.ndarray, b: np.ndarray, cfl: float) -> float:
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    c = cfg.c()
    return float(_L().oracle_max_dt(ctypes.byref(c), _ptr(cons), _ptr(b), float(cfl)))


def divb(cfg: Config, b: np.ndarray):
    """(max |div b| over cells, max |b| over faces)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    md = ctypes.c_double()
    mb = ctypes.c_double()
    c = cfg.c()
    _L().oracle_divb(ctypes.byref(c), _ptr(b), ctypes.byref(md), ctypes.byref(mb))
    return md.value, mb.value


def steps_jvp(cfg: Config, cons, b, dcons, db, deta: float, dts):
    """Forward-mode directional derivative of len(dts) steps with frozen dts.

    Returns (cons, b, dcons, db): final state and its tangent."""
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64).copy()
    b = np.ascontiguousarray(b, dtype=np.float64).copy()
    dcons = np.ascontiguousarray(dcons, dtype=np.float64).copy()
    db = np.ascontiguousarray(db, dtype=np.float64).copy()
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    c = cfg.c()
    rc = _L().oracle_steps_jvp(
        ctypes.byref(c), _ptr(cons), _ptr(b), _ptr(dcons), _ptr(db), float(deta), _ptr(dts), len(dts)
    )
    assert rc == 0
    return cons, b, dcons, db


def run(cfg: Config, cons, b, nsteps: int, cfl: float = 0.3, dt: float | None = None):
    """Advance nsteps with dt from the CFL condition each step (or a fixed dt)."""
    dts = []
    counts = []
    for _ in range(nsteps):
        h = dt if dt is not None else max_dt(cfg, cons, b, cfl)
        cons, b, cnt = step(cfg, cons, b, h)
        dts.append(h)
        counts.append(cnt)
    return cons, b, dts, counts


PHASES = ["prim", "recon", "riemann", "edge", "joule", "update", "flag", "fo"]


def count_ops(cfg: Config, cons, b, dt: float, with_unused: bool = False):
    """FP64 operations (+, -, *, /, sqrt) of one step of the oracle, by phase; with_unused also
    returns the Riemann-phase operations a one-sided HLLD would not form."""
    _check(cfg, cons, b)
    cons = np.ascontiguousarray(cons, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    ops = (ctypes.c_longlong * 8)()
    counts = (ctypes.c_longlong * 2)()
    unused = ctypes.c_longlong(0)
    c = cfg.c()
    _L().oracle_count_ops(ctypes.byref(c), _ptr(cons), _ptr(b), float(dt), ops, counts, ctypes.byref(unused))
    res = {k: int(ops[i]) for i, k in enumerate(PHASES)}, (int(counts[0]), int(counts[1]))
    return res + (int(unused.value),) if with_unused else res
