"""Thin ctypes binding of libmhd.so (include/mhd.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels. PyTorch supplies device memory and
the stream. If the library is missing or cannot load, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmhd.so")

# scheme bits (include/mhd.h)
RECON = {"pc": 0, "plm_mc": 1, "plm_minmod": 2, "ppm": 3, "ppm_ep": 4}
RIEMANN = {"hll": 0 << 4, "hlld": 1 << 4, "llf": 2 << 4}
EMF = {"q26": 0 << 8, "fs18": 1 << 8, "b25a": 2 << 8}
AVG = {"ld04": 0 << 12, "b25b": 1 << 12}
FOFC_OFF = 1 << 16

OK, ERR_ARG, ERR_CUDA, ERR_NONFINITE, ERR_UNSUPPORTED, ERR_TIMEOUT = range(6)
KERNELS = ["prim", "face", "edge_bt", "edge_lr", "update", "flag", "fofc", "maxspeed", "divb", "extra"]
K_COUNT = 16
_NAMES = ["OK", "ARG", "CUDA", "NONFINITE", "UNSUPPORTED", "TIMEOUT"]


def scheme(recon="plm_mc", riemann="hll", emf="q26", avg="ld04", fofc=True) -> int:
    return RECON[recon] | RIEMANN[riemann] | EMF[emf] | AVG[avg] | (0 if fofc else FOFC_OFF)


class MHDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mhd error {_NAMES[code] if 0 <= code < 6 else code}: {msg}")
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("gamma", ctypes.c_double), ("fofc_criteria", ctypes.c_int),
    ]


class _State(ctypes.Structure):
    _fields_ = [("cons", ctypes.c_void_p), ("b0", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("b2", ctypes.c_void_p)]


class _BatchState(ctypes.Structure):
    _fields_ = [("cons", ctypes.c_void_p), ("b", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libmhd.so (raises if it is absent: build it with paper_2609_10816_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2609_10816_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    d = ctypes.c_double
    L.mhd_create.argtypes = [P(_Config), vp, P(vp)]
    L.mhd_create.restype = ctypes.c_int
    L.mhd_destroy.argtypes = [vp]
    L.mhd_destroy.restype = None
    L.mhd_step.argtypes = [vp, P(_State), d, ctypes.c_int, d]
    L.mhd_step.restype = ctypes.c_int
    L.mhd_max_dt.argtypes = [vp, P(_State), d, d, P(d)]
    L.mhd_max_dt.restype = ctypes.c_int
    L.mhd_divb.argtypes = [vp, P(_State), P(d), P(d)]
    L.mhd_divb.restype = ctypes.c_int
    L.mhd_stats.argtypes = [vp, P(ctypes.c_longlong), P(ctypes.c_longlong)]
    L.mhd_stats.restype = ctypes.c_int
    L.mhd_last_error.argtypes = [vp]
    L.mhd_last_error.restype = ctypes.c_char_p
    L.mhd_create_error.argtypes = []
    L.mhd_create_error.restype = ctypes.c_char_p
    L.mhd_step_adjoint.argtypes = [vp, P(_State), P(_State), d, ctypes.c_int, d, P(d)]
    L.mhd_step_adjoint.restype = ctypes.c_int
    L.mhd_step_cfl.argtypes = [vp, P(_State), d, ctypes.c_int, d]
    L.mhd_step_cfl.restype = ctypes.c_int
    L.mhd_last_dt.argtypes = [vp, P(d)]
    L.mhd_last_dt.restype = ctypes.c_int
    L.mhd_fp64_rate.argtypes = [ctypes.c_int, ctypes.c_longlong, vp, P(d)]
    L.mhd_fp64_rate.restype = ctypes.c_int
    L.mhd_math_check.argtypes = [vp, ctypes.c_longlong, P(d)]
    L.mhd_math_check.restype = ctypes.c_int
    L.mhd_adjoint_check.argtypes = [vp, ctypes.c_longlong, ctypes.c_int, ctypes.c_ulonglong, P(d)]
    L.mhd_adjoint_check.restype = ctypes.c_int
    L.mhd_profile.argtypes = [vp, ctypes.c_int]
    L.mhd_profile.restype = ctypes.c_int
    L.mhd_profile_read.argtypes = [vp, P(d), P(ctypes.c_longlong), ctypes.c_int]
    L.mhd_profile_read.restype = ctypes.c_int
    i = ctypes.c_int
    ll = ctypes.c_longlong
    L.mhd_batch_create.argtypes = [P(i), i, d, d, vp, P(vp)]
    L.mhd_batch_create.restype = i
    L.mhd_batch_destroy.argtypes = [vp]
    L.mhd_batch_destroy.restype = None
    L.mhd_batch_offsets.argtypes = [vp, P(ll)]
    L.mhd_batch_offsets.restype = i
    L.mhd_batch_step.argtypes = [vp, P(_BatchState), d, i, d]
    L.mhd_batch_step.restype = i
    L.mhd_batch_last_dt.argtypes = [vp, P(d)]
    L.mhd_batch_last_dt.restype = i
    L.mhd_batch_stats.argtypes = [vp, P(ll), P(ll)]
    L.mhd_batch_stats.restype = i
    L.mhd_batch_phase_ms.argtypes = [vp, P(d)]
    L.mhd_batch_phase_ms.restype = i
    L.mhd_batch_set_schedule.argtypes = [vp, i, i, i, i]
    L.mhd_batch_set_schedule.restype = i
    L.mhd_batch_tune.argtypes = [vp, P(_BatchState), d, i, d, P(i), P(i), P(i), P(i)]
    L.mhd_batch_tune.restype = i
    L.mhd_batch_set_launches.argtypes = [vp, i]
    L.mhd_batch_set_launches.restype = i
    L.mhd_batch_test_barrier.argtypes = [vp, i, ll]
    L.mhd_batch_test_barrier.restype = i
    L.mhd_batch_last_error.argtypes = [vp]
    L.mhd_batch_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


FP64_RATE_KINDS = {"dfma": 0, "dadd": 1, "dmul": 2, "ffma": 3, "int_mul": 4, "dfma_int_mul": 5,
                   "dfma_int_mul_2x128": 6, "dfma_16_lanes": 7, "dfma_8_lanes": 8}


def fp64_rate(kind: str = "dfma", iters: int = 1 << 14, stream: torch.cuda.Stream | None = None) -> float:
    """mhd_fp64_rate: instructions per second (per lane) of one FP64 (or FP32 FFMA) kind, or
    (kinds int_mul, dfma_int_mul, dfma_int_mul_2x128) operations per second of chains of the
    integer-pipe multiply, alone or beside DFMA chains."""
    s = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double()
    rc = lib().mhd_fp64_rate(FP64_RATE_KINDS[kind], int(iters), ctypes.c_void_p(s.cuda_stream), ctypes.byref(out))
    if rc != OK:
        raise MHDError(rc, "mhd_fp64_rate failed")
    return out.value


def _check_field(t: torch.Tensor, shape, name):
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {tuple(shape)}, got {tuple(t.shape)}")


class State:
    """Device state of one periodic box: cons (5, nz, ny, nx) and b (3, nz, ny, nx), float64."""

    def __init__(self, cons: torch.Tensor, b: torch.Tensor):
        self.cons = cons
        self.b = b

    def c(self) -> _State:
        return _State(self.cons.data_ptr(), self.b[0].data_ptr(), self.b[1].data_ptr(), self.b[2].data_ptr())


class Context:
    """mhd_create / mhd_destroy for one box size, on a torch CUDA stream."""

    def __init__(self, shape, h, gamma=5.0 / 3.0, stream: torch.cuda.Stream | None = None, fofc_criteria=3):
        L = lib()
        self.shape = tuple(int(n) for n in shape)
        self.h = tuple(float(x) for x in h)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = _Config(self.shape[0], self.shape[1], self.shape[2], self.h[0], self.h[1], self.h[2],
                      float(gamma), int(fofc_criteria))
        out = ctypes.c_void_p()
        rc = L.mhd_create(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(out))
        if rc != OK:
            raise MHDError(rc, L.mhd_create_error().decode())
        self._h = out

    def _err(self, rc):
        if rc != OK:
            raise MHDError(rc, lib().mhd_last_error(self._h).decode())

    def _state(self, st: State) -> _State:
        nx, ny, nz = self.shape
        _check_field(st.cons, (5, nz, ny, nx), "cons")
        _check_field(st.b, (3, nz, ny, nx), "b")
        return st.c()

    def step(self, st: State, dt: float, scheme_bits: int, eta: float = 0.0):
        s = self._state(st)
        self._err(lib().mhd_step(self._h, ctypes.byref(s), float(dt), int(scheme_bits), float(eta)))

    def max_dt(self, st: State, cfl: float, eta: float = 0.0) -> float:
        s = self._state(st)
        out = ctypes.c_double()
        self._err(lib().mhd_max_dt(self._h, ctypes.byref(s), float(cfl), float(eta), ctypes.byref(out)))
        return out.value

    def step_cfl(self, st: State, cfl: float, scheme_bits: int, eta: float = 0.0):
        """max_dt + step with dt kept on the device (no synchronisation)."""
        s = self._state(st)
        self._err(lib().mhd_step_cfl(self._h, ctypes.byref(s), float(cfl), int(scheme_bits), float(eta)))

    def last_dt(self) -> float:
        """dt of the last step_cfl (synchronises)."""
        out = ctypes.c_double()
        self._err(lib().mhd_last_dt(self._h, ctypes.byref(out)))
        return out.value

    def divb(self, st: State):
        s = self._state(st)
        md, mb = ctypes.c_double(), ctypes.c_double()
        self._err(lib().mhd_divb(self._h, ctypes.byref(s), ctypes.byref(md), ctypes.byref(mb)))
        return md.value, mb.value

    def stats(self):
        a, b = ctypes.c_longlong(), ctypes.c_longlong()
        self._err(lib().mhd_stats(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def step_adjoint(self, st: State, lam: State, dt: float, scheme_bits: int, eta: float = 0.0) -> float:
        """lam <- (dS^{n+1}/dS^n)^T lam for the step from st; returns the step's d/d(eta) term."""
        s = self._state(st)
        l = self._state(lam)
        out = ctypes.c_double(0.0)
        self._err(lib().mhd_step_adjoint(self._h, ctypes.byref(s), ctypes.byref(l), float(dt), int(scheme_bits),
                                         float(eta), ctypes.byref(out)))
        return out.value

    ADJ_CHECK_KINDS = ("equal", "nearby", "bn_zero", "field_along_n", "low_pressure", "large")

    def adjoint_check(self, scheme_bits: int, n: int = 1 << 20, seed: int = 1):
        """Largest relative gap between the reverse-mode and dual-number gradients of the face solve:
        (overall, {kind of face problem: largest gap})."""
        out = (ctypes.c_double * 7)()
        self._err(lib().mhd_adjoint_check(self._h, int(n), int(scheme_bits), int(seed), out))
        return out[0], dict(zip(self.ADJ_CHECK_KINDS, out[1:]))

    def math_check(self, n: int = 1 << 22):
        """(largest relative errors of the kernels' reciprocal, rsqrt and sqrt vs IEEE, bit
        mismatches of the integer halving, of the integer quadrupling, disagreements of the
        integer-pipe comparisons and sign operations with IEEE, bit mismatches of the integer-pipe
        multiply)."""
        out = (ctypes.c_double * 7)()
        self._err(lib().mhd_math_check(self._h, int(n), out))
        return tuple(out)

    def profile(self, enable: bool):
        self._err(lib().mhd_profile(self._h, 1 if enable else 0))

    def profile_read(self, reset: bool = False):
        """{kernel class: (total ms of timed launches, launches)}."""
        ms = (ctypes.c_double * K_COUNT)()
        n = (ctypes.c_longlong * K_COUNT)()
        self._err(lib().mhd_profile_read(self._h, ms, n, 1 if reset else 0))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNELS)}

    def close(self):
        if getattr(self, "_h", None):
            lib().mhd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def to_device(cons, b, device="cuda") -> State:
    return State(torch.as_tensor(cons, dtype=torch.float64).to(device).contiguous(),
                 torch.as_tensor(b, dtype=torch.float64).to(device).contiguous())


class Batch:
    """mhd_batch_*: many periodic patches of cell width h advanced together on the device."""

    def __init__(self, dims, h, gamma=5.0 / 3.0, stream: torch.cuda.Stream | None = None):
        L = lib()
        self.dims = [tuple(int(x) for x in d) for d in dims]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        flat = (ctypes.c_int * (3 * len(self.dims)))(*[x for d in self.dims for x in d])
        out = ctypes.c_void_p()
        rc = L.mhd_batch_create(flat, len(self.dims), float(h), float(gamma),
                                ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(out))
        if rc != OK:
            raise MHDError(rc, L.mhd_batch_last_error(None).decode())
        self._h = out
        offs = (ctypes.c_longlong * (len(self.dims) + 1))()
        self._err(L.mhd_batch_offsets(self._h, offs))
        self.offsets = list(offs)
        self.ncell = self.offsets[-1]

    def _err(self, rc):
        if rc != OK:
            raise MHDError(rc, lib().mhd_batch_last_error(self._h).decode())

    def empty_state(self, device="cuda"):
        return (torch.zeros(5 * self.ncell, dtype=torch.float64, device=device),
                torch.zeros(3 * self.ncell, dtype=torch.float64, device=device))

    def pack(self, patches, device="cuda"):
        """[(cons (5,nz,ny,nx), b (3,nz,ny,nx)) per patch] -> device (cons, b) in batch layout."""
        import numpy as np

        cons = np.concatenate([np.ascontiguousarray(c, dtype=np.float64).ravel() for c, _ in patches])
        b = np.concatenate([np.ascontiguousarray(bb, dtype=np.float64).ravel() for _, bb in patches])
        assert cons.size == 5 * self.ncell and b.size == 3 * self.ncell
        return torch.from_numpy(cons).to(device), torch.from_numpy(b).to(device)

    def unpack(self, cons, b, p):
        """Host numpy (cons, b) of patch p."""
        nx, ny, nz = self.dims[p]
        o, n = self.offsets[p], nx * ny * nz
        c = cons[5 * o:5 * (o + n)].reshape(5, nz, ny, nx).cpu().numpy()
        bb = b[3 * o:3 * (o + n)].reshape(3, nz, ny, nx).cpu().numpy()
        return c, bb

    def _st(self, cons, b):
        if cons.dtype != torch.float64 or b.dtype != torch.float64 or not cons.is_cuda or not b.is_cuda:
            raise TypeError("batch state must be float64 CUDA tensors")
        if cons.numel() != 5 * self.ncell or b.numel() != 3 * self.ncell:
            raise ValueError("batch state has the wrong size")
        return _BatchState(cons.data_ptr(), b.data_ptr())

    def step(self, cons, b, cfl, scheme_bits, eta=0.0):
        s = self._st(cons, b)
        self._err(lib().mhd_batch_step(self._h, ctypes.byref(s), float(cfl), int(scheme_bits), float(eta)))

    def last_dt(self):
        out = ctypes.c_double()
        self._err(lib().mhd_batch_last_dt(self._h, ctypes.byref(out)))
        return out.value

    def stats(self):
        a, c = ctypes.c_longlong(), ctypes.c_longlong()
        self._err(lib().mhd_batch_stats(self._h, ctypes.byref(a), ctypes.byref(c)))
        return a.value, c.value

    PHASES = ("prim", "face", "edge_bt", "edge_lr", "update_flag", "fo_fluxes")

    def phase_ms(self):
        """Device time of each phase of the last step's two stages, {stage: {phase: ms}}."""
        out = (ctypes.c_double * 12)()
        self._err(lib().mhd_batch_phase_ms(self._h, out))
        return {s: {ph: out[6 * s + j] for j, ph in enumerate(self.PHASES)} for s in (0, 1)}

    def set_schedule(self, seg=64, order=1, blocks_per_sm=0, use_graph=True):
        self._err(lib().mhd_batch_set_schedule(self._h, int(seg), int(order), int(blocks_per_sm), 1 if use_graph else 0))

    def set_launches(self, launches_per_stage: int):
        """1: one persistent launch per RK stage (the default); 3: face / edge-update-flag /
        first-order-correction launches."""
        self._err(lib().mhd_batch_set_launches(self._h, int(launches_per_stage)))

    def tune(self, cons, b, cfl, scheme_bits, eta=0.0):
        s = self._st(cons, b)
        seg, order, bps, nl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._err(lib().mhd_batch_tune(self._h, ctypes.byref(s), float(cfl), int(scheme_bits), float(eta),
                                       ctypes.byref(seg), ctypes.byref(order), ctypes.byref(bps), ctypes.byref(nl)))
        return {"seg": seg.value, "order": order.value, "blocks_per_sm": bps.value, "launches_per_stage": nl.value}

    def test_barrier(self, extra_blocks, spin_limit):
        self._err(lib().mhd_batch_test_barrier(self._h, int(extra_blocks), int(spin_limit)))

    def close(self):
        if getattr(self, "_h", None):
            lib().mhd_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
