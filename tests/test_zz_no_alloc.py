"""mhd_step_noalloc against mhd_step (GPU).

mhd_step_noalloc serves callers that cannot let the library allocate device memory (an
application whose own memory manager owns the device, loops that cannot afford cudaMalloc's
synchronisation): it runs the step with its scratch in a fixed device array
inside libmhd.so. This test calls it through the C ABI twice in a row on different boxes and
compares each result with mhd_step's, at the parity tolerance of the other GPU tests; the first
call sets flux-correction flags and counters in the shared array, so leftovers would show in the
second. It also checks that a box above the fixed limit is refused with a message.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2609_10816_gb300 import inputs, mhd
from tests.util import state_errors

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _noalloc():
    f = mhd.lib().mhd_step_noalloc
    f.argtypes = [ctypes.POINTER(mhd._Config), ctypes.POINTER(mhd._State), ctypes.c_double, ctypes.c_int,
                  ctypes.c_double, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _low_pressure_state(shape, seed=1):
    """Strong expansion over a near-vacuum pressure: the high-order step leaves cells invalid."""
    cons, b, info = inputs.random_smooth(shape, seed=seed, rough=0.0)
    rng = np.random.default_rng(seed)
    rho = cons[0]
    u = [cons[1 + d] / rho for d in range(3)]
    nx = shape[0]
    x = (np.arange(nx) + 0.5) / nx
    u[0] = u[0] + 3.0 * np.sin(2 * np.pi * x)[None, None, :] + 0.3 * rng.uniform(-1, 1, rho.shape)
    p = 1e-3 * np.ones_like(rho)
    return inputs.assemble(rho, u, p, b), b, info


def _cfg(shape, h):
    return mhd._Config(shape[0], shape[1], shape[2], h[0], h[1], h[2], 5.0 / 3.0, 3)


def test_noalloc_matches_mhd_step_on_two_calls_in_a_row(gpu_lib):
    f = _noalloc()
    stream = torch.cuda.current_stream()
    cases = []
    cons, b, info = _low_pressure_state((16, 6, 4))
    cases.append(((16, 6, 4), cons, b, info, mhd.scheme("ppm", "hlld", "q26"), 0.0, 0.6))
    cons, b, info = inputs.random_smooth((20, 12, 8), seed=17, rough=0.03)
    cases.append(((20, 12, 8), cons, b, info, mhd.scheme("plm_mc", "hll", "q26"), 2e-3, 0.3))
    for k, (shape, cons, b, info, sch, eta, cfl) in enumerate(cases):
        ctx = mhd.Context(shape, info["h"])
        ref = mhd.to_device(cons, b)
        dt = ctx.max_dt(ref, cfl, eta)
        ctx.step(ref, dt, sch, eta)
        flagged = ctx.stats()
        ctx.close()
        if k == 0:
            assert flagged[0] + flagged[1] > 0  # the first call exercises the flags and counters
        st = mhd.to_device(cons, b)
        rc = f(ctypes.byref(_cfg(shape, info["h"])), ctypes.byref(st.c()), dt, sch, eta,
               ctypes.c_void_p(stream.cuda_stream))
        assert rc == mhd.OK, mhd.lib().mhd_create_error()
        torch.cuda.synchronize()
        errs = state_errors(st.cons.cpu().numpy(), st.b.cpu().numpy(), ref.cons.cpu().numpy(), ref.b.cpu().numpy())
        assert all(v <= TOL for v in errs.values()), (k, errs)


def test_noalloc_refuses_boxes_above_its_fixed_scratch(gpu_lib):
    f = _noalloc()
    shape = (33, 32, 32)
    assert shape[0] * shape[1] * shape[2] > 32768
    st = mhd.State(torch.zeros((5, 32, 32, 33), dtype=torch.float64, device="cuda"),
                   torch.zeros((3, 32, 32, 33), dtype=torch.float64, device="cuda"))
    rc = f(ctypes.byref(_cfg(shape, (0.1, 0.1, 0.1))), ctypes.byref(st.c()), 1e-3, 0, 0.0, None)
    assert rc == mhd.ERR_ARG
    assert b"exceeds the fixed scratch" in mhd.lib().mhd_create_error()
