"""CUDA path (libmhd.so through the C ABI) against the CPU oracle, element by element.

Tolerance: relative L1 per stored field per step <= 1e-12 (denominator floored at N times the
field family's natural scale), the accuracy bar of the method's parity requirement, and element
by element max |gpu - oracle| <= 1e-11 of the field's mean magnitude (floored the same way); the
face field's divergence stays at rounding, max |div b| dx / max |b| <= 1e-13.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_10816_gb300 import inputs
from paper_2609_10816_gb300 import mhd
from tests.util import L1_TOL, parity_failures

pytestmark = pytest.mark.gpu

TOL = L1_TOL


def gpu_step(ctx, cons, b, dt, sch, eta=0.0):
    st = mhd.to_device(cons, b)
    ctx.step(st, dt, sch, eta)
    torch.cuda.synchronize()
    return st.cons.cpu().numpy(), st.b.cpu().numpy(), ctx.stats()


def assert_parity(cg, bg, co, bo, what=""):
    bad = parity_failures(cg, bg, co, bo)
    assert not bad, f"{what}: (relative L1, relative max) above the bars: {bad}"


COMBOS = [(r, s, e) for r in ("pc", "plm_mc", "plm_minmod", "ppm", "ppm_ep") for s in ("hll", "hlld", "llf")
          for e in ("q26", "fs18", "b25a")]


@pytest.mark.parametrize("recon,rs,emf", COMBOS)
@pytest.mark.parametrize("shape", [(8, 8, 8), (70, 9, 5)])
def test_one_step_all_schemes(gpu_lib, recon, rs, emf, shape):
    cons, b, info = inputs.random_smooth(shape, seed=11, rough=0.05)
    cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann=rs, emf=emf, eta=1e-3)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    co, bo, cnt = oracle.step(cfg, cons, b, dt)
    ctx = mhd.Context(shape, info["h"])
    cg, bg, cntg = gpu_step(ctx, cons, b, dt, mhd.scheme(recon, rs, emf), eta=1e-3)
    assert_parity(cg, bg, co, bo, what=f"{recon}/{rs}/{emf}/{shape}")
    assert cntg == cnt


@pytest.mark.parametrize("shape", [(42, 16, 12), (16, 8, 42), (24, 12, 8)])
def test_warp_patches_of_lines(gpu_lib, shape):
    """Sweeps whose warps walk 8 x 4 patches of lines (both line axes multiples of 8 and 4) beside
    sweeps that cannot (42 cells), with ragged segment tails along 42 cells and several patches per
    plane: one step against the oracle for each EMF compute scheme, flagged-cell counts equal."""
    cons, b, info = inputs.random_smooth(shape, seed=13, rough=0.05)
    for recon, rs, emf in (("ppm", "hlld", "q26"), ("ppm_ep", "hlld", "fs18"), ("plm_mc", "hll", "b25a"),
                           ("ppm", "llf", "q26")):
        cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann=rs, emf=emf, eta=1e-3)
        dt = oracle.max_dt(cfg, cons, b, 0.3)
        co, bo, cnt = oracle.step(cfg, cons, b, dt)
        ctx = mhd.Context(shape, info["h"])
        cg, bg, cntg = gpu_step(ctx, cons, b, dt, mhd.scheme(recon, rs, emf), eta=1e-3)
        assert_parity(cg, bg, co, bo, what=f"{recon}/{rs}/{emf}/{shape}")
        assert cntg == cnt


@pytest.mark.parametrize("shape", [(16, 1, 1), (1, 12, 3), (2, 5, 9), (130, 3, 2)])
def test_degenerate_and_ragged_boxes(gpu_lib, shape):
    cons, b, info = inputs.random_smooth(shape, seed=5, rough=0.02)
    for recon, rs, emf in (("ppm", "hlld", "q26"), ("plm_mc", "hll", "fs18"), ("ppm", "llf", "b25a"),
                           ("ppm_ep", "hlld", "q26")):
        cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann=rs, emf=emf)
        dt = oracle.max_dt(cfg, cons, b, 0.3)
        co, bo, _ = oracle.step(cfg, cons, b, dt)
        ctx = mhd.Context(shape, info["h"])
        cg, bg, _ = gpu_step(ctx, cons, b, dt, mhd.scheme(recon, rs, emf))
        assert_parity(cg, bg, co, bo, what=f"{recon}/{rs}/{emf}/{shape}")


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


@pytest.mark.parametrize("recon,emf", [("ppm", "q26"), ("ppm", "fs18"), ("ppm", "b25a"), ("ppm_ep", "q26")])
def test_flux_correction_against_oracle(gpu_lib, recon, emf):
    """Cells the high-order step leaves invalid take first-order fluxes: same flags and state."""
    shape = (16, 6, 4)
    cons, b, info = _low_pressure_state(shape)
    cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann="hlld", emf=emf, eta=1e-3)
    dt = oracle.max_dt(cfg, cons, b, 0.6)
    co, bo, cnt = oracle.step(cfg, cons, b, dt)
    assert cnt[0] + cnt[1] > 0
    ctx = mhd.Context(shape, info["h"])
    cg, bg, cntg = gpu_step(ctx, cons, b, dt, mhd.scheme(recon, "hlld", emf), eta=1e-3)
    assert cntg == cnt
    assert_parity(cg, bg, co, bo, what=f"fofc {emf}")


def test_fast_wave_32cubed_multistep(gpu_lib):
    """32^3 oblique fast eigenmode, PLM-MC + HLL + Q26 + LD04, CFL 0.3: 10 steps, every step."""
    shape = (32, 32, 32)
    cons, b, info = inputs.fast_wave(shape)
    cfg = oracle.Config(shape=shape, h=info["h"], recon="plm_mc", riemann="hll")
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    co, bo = cons, b
    sch = mhd.scheme("plm_mc", "hll")
    for _ in range(10):
        dt = oracle.max_dt(cfg, co, bo, 0.3)
        dtg = ctx.max_dt(st, 0.3)
        assert abs(dtg - dt) <= 1e-14 * dt
        co, bo, _ = oracle.step(cfg, co, bo, dt)
        ctx.step(st, dt, sch)
        torch.cuda.synchronize()
        assert_parity(st.cons.cpu().numpy(), st.b.cpu().numpy(), co, bo, what="fast wave")
    md, mb = ctx.divb(st)
    assert md * info["h"][0] / mb <= 1e-13


@pytest.mark.parametrize("emf", ["q26", "fs18", "b25a"])
def test_turbulence_32cubed_first_step_from_rest_field(gpu_lib, emf):
    """The turbulence recipe's initial state at 32^3 (Mach 5, mean field (0, 0, 0.5)): b_x = b_y = 0
    on every face, so every x and y face solve is HLLD's b_n = 0 case (no rotational waves, the
    star states' degenerate branch). First step from t = 0, PPM + HLLD, on the whole box."""
    shape = (32, 32, 32)
    cons, b, info = inputs.turbulence(shape, seed=2, v_rms=5.0)
    assert not b[0].any() and not b[1].any()
    cfg = oracle.Config(shape=shape, h=info["h"], recon="ppm", riemann="hlld", emf=emf)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    co, bo, cnt = oracle.step(cfg, cons, b, dt)
    ctx = mhd.Context(shape, info["h"])
    assert abs(ctx.max_dt(mhd.to_device(cons, b), 0.3) - dt) <= 1e-14 * dt
    cg, bg, cntg = gpu_step(ctx, cons, b, dt, mhd.scheme("ppm", "hlld", emf))
    assert cntg == cnt
    assert_parity(cg, bg, co, bo, what=f"turbulence t=0 {emf}")
    md, mb = ctx.divb(mhd.to_device(cg, bg))
    assert md * info["h"][0] / mb <= 1e-13


def test_resistive_step(gpu_lib):
    shape = (24, 20, 6)
    cons, b, info = inputs.random_smooth(shape, seed=7, rough=0.02)
    for recon, rs in (("plm_mc", "hlld"), ("ppm", "hll")):
        cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann=rs, eta=3e-3)
        dt = oracle.max_dt(cfg, cons, b, 0.3)
        co, bo, _ = oracle.step(cfg, cons, b, dt)
        ctx = mhd.Context(shape, info["h"])
        cg, bg, _ = gpu_step(ctx, cons, b, dt, mhd.scheme(recon, rs), eta=3e-3)
        assert_parity(cg, bg, co, bo, what=f"eta {recon}/{rs}")


def test_max_dt_and_divb(gpu_lib):
    shape = (20, 12, 7)
    cons, b, info = inputs.random_smooth(shape, seed=3, rough=0.1)
    cfg = oracle.Config(shape=shape, h=info["h"], eta=2e-2)
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    for eta in (0.0, 2e-2, 10.0):
        cfg.eta = eta
        assert abs(ctx.max_dt(st, 0.3, eta) - oracle.max_dt(cfg, cons, b, 0.3)) <= 1e-14 * oracle.max_dt(cfg, cons, b, 0.3)
    md, mb = ctx.divb(st)
    mdo, mbo = oracle.divb(cfg, b)
    assert mb == mbo
    assert abs(md - mdo) <= 1e-12 * mbo / min(info["h"])


@pytest.mark.parametrize("case", ["turbulence", "bulk_flow", "fast_cell_last", "non_cubic"])
def test_max_dt_early_exit_cases(gpu_lib, case):
    """The CFL reduction's per-cell early exit (a bound on squares for cubic cells) never drops the
    cell that sets dt: Mach-5 turbulence, a smooth state carried by a bulk flow far faster than its
    sound and Alfven speeds, one fast cell at the end of the cell order, non-cubic cells; dt equals
    the oracle's to 1e-14."""
    if case == "turbulence":
        shape = (24, 24, 24)
        cons, b, info = inputs.turbulence(shape)
    else:
        shape = (24, 20, 16)
        h = (0.05, 0.04, 0.03) if case == "non_cubic" else (0.05, 0.05, 0.05)
        cons, b, info = inputs.random_smooth(shape, seed=29, rough=0.05, h=h)
    cons = cons.copy()
    if case == "bulk_flow":  # u_x += 1e3 (kinetic energy added accordingly)
        rho = cons[0]
        mx = cons[1] + 1e3 * rho
        cons[4] = cons[4] + 0.5 * (mx**2 - cons[1] ** 2) / rho
        cons[1] = mx
    if case == "fast_cell_last":  # the last cell in memory order moves at 30x the others
        rho = cons[0, -1, -1, -1]
        mz = cons[3, -1, -1, -1] + 30.0 * rho
        cons[4, -1, -1, -1] += 0.5 * (mz**2 - cons[3, -1, -1, -1] ** 2) / rho
        cons[3, -1, -1, -1] = mz
    cfg = oracle.Config(shape=shape, h=info["h"])
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    ref = oracle.max_dt(cfg, cons, b, 0.3)
    assert abs(ctx.max_dt(st, 0.3) - ref) <= 1e-14 * ref
    ctx.step_cfl(st, 0.3, mhd.scheme("plm_mc", "hll", "q26"))
    assert abs(ctx.last_dt() - ref) <= 1e-14 * ref


def test_step_with_device_cfl_equals_host_cfl(gpu_lib):
    """step_cfl (CFL reduction, dt and dt/h kept on the device) gives bit for bit the state and the
    dt of max_dt + step, over several steps, ideal and resistive; and the oracle's step agrees."""
    shape = (18, 10, 7)
    cons, b, info = inputs.random_smooth(shape, seed=11, rough=0.05)
    ctx = mhd.Context(shape, info["h"])
    sch = mhd.scheme("ppm", "hlld", "q26")
    for eta in (0.0, 4e-3, 50.0):  # the last makes the resistive speed set dt
        st_h, st_d = mhd.to_device(cons, b), mhd.to_device(cons, b)
        for _ in range(3):
            dt = ctx.max_dt(st_h, 0.3, eta)
            ctx.step(st_h, dt, sch, eta)
            ctx.step_cfl(st_d, 0.3, sch, eta)
            assert ctx.last_dt() == dt
        torch.cuda.synchronize()
        assert torch.equal(st_h.cons, st_d.cons) and torch.equal(st_h.b, st_d.b)
    cfg = oracle.Config(shape=shape, h=info["h"], recon="ppm", riemann="hlld", eta=4e-3)
    co, bo, _ = oracle.step(cfg, cons, b, oracle.max_dt(cfg, cons, b, 0.3))
    st = mhd.to_device(cons, b)
    ctx.step_cfl(st, 0.3, sch, 4e-3)
    torch.cuda.synchronize()
    assert_parity(st.cons.cpu().numpy(), st.b.cpu().numpy(), co, bo, what="step_cfl")


@pytest.mark.parametrize("case", ["smooth", "flagged"])
def test_step_cfl_equals_max_dt_and_step(gpu_lib, case):
    """mhd_step_cfl (dt on the device): the state, dt and flag counts equal bitwise those of
    mhd_max_dt + mhd_step over three steps, with and without flux-corrected cells, and the first
    step agrees with the oracle."""
    shape = (20, 12, 8)
    h = (0.05, 0.05, 0.05)
    if case == "smooth":
        cons, b, _ = inputs.random_smooth(shape, seed=17, rough=0.05, h=h)
        cfl, eta = 0.3, 2e-3
    else:
        cons, b, _ = _low_pressure_state(shape)
        cfl, eta = 0.6, 0.0
    sch = mhd.scheme("ppm", "hlld", "q26")
    ctx = mhd.Context(shape, h)
    st_s, st_b = mhd.to_device(cons, b), mhd.to_device(cons, b)
    flagged = 0
    for k in range(3):
        dt = ctx.max_dt(st_s, cfl, eta)
        ctx.step(st_s, dt, sch, eta)
        cnt = ctx.stats()
        ctx.step_cfl(st_b, cfl, sch, eta)
        assert ctx.last_dt() == dt and ctx.stats() == cnt
        flagged += cnt[0] + cnt[1]
        torch.cuda.synchronize()
        assert torch.equal(st_s.cons, st_b.cons) and torch.equal(st_s.b, st_b.b), k
    assert case == "smooth" or flagged > 0
    cfg = oracle.Config(shape=shape, h=h, recon="ppm", riemann="hlld", eta=eta)
    co, bo, _ = oracle.step(cfg, cons, b, oracle.max_dt(cfg, cons, b, cfl))
    st = mhd.to_device(cons, b)
    ctx.step_cfl(st, cfl, sch, eta)
    torch.cuda.synchronize()
    assert_parity(st.cons.cpu().numpy(), st.b.cpu().numpy(), co, bo, what=f"step_cfl {case}")


def test_step_cfl_replays_its_own_graph(gpu_lib):
    """Repeated mhd_step_cfl calls on a small box replay a recorded graph (profiling off): state, dt
    and flag counts equal bitwise those of the eager steps (profiling on forces them), also when
    cfl changes between calls (a new recording) and around a call with other arrays."""
    shape = (18, 14, 10)
    h = (0.05, 0.05, 0.05)
    cons, b, _ = inputs.random_smooth(shape, seed=23, rough=0.05, h=h)
    sch = mhd.scheme("ppm", "hlld", "q26")
    eager, graphed = mhd.Context(shape, h), mhd.Context(shape, h)
    eager.profile(True)
    st_e, st_g, other = mhd.to_device(cons, b), mhd.to_device(cons, b), mhd.to_device(cons, b)
    cfls = [0.3, 0.3, 0.3, 0.3, 0.25, 0.25, 0.25, 0.3, 0.3]
    for k, cfl in enumerate(cfls):
        if k == 6:
            graphed.step_cfl(other, cfl, sch)  # other arrays in between (st_g's recording stays valid)
        eager.step_cfl(st_e, cfl, sch)
        graphed.step_cfl(st_g, cfl, sch)
        assert eager.last_dt() == graphed.last_dt() and eager.stats() == graphed.stats(), k
        torch.cuda.synchronize()
        assert torch.equal(st_e.cons, st_g.cons) and torch.equal(st_e.b, st_g.b), k


def test_step_cfl_sequence_in_a_cuda_graph(gpu_lib):
    """Four step_cfl calls recorded in one CUDA graph replay to the eager result bit for bit (the
    step needs no host round trip, so a sequence of steps can run as one graph launch)."""
    shape = (16, 12, 10)
    cons, b, info = inputs.random_smooth(shape, seed=13, rough=0.05)
    s = torch.cuda.Stream()
    ctx = mhd.Context(shape, info["h"], stream=s)
    sch = mhd.scheme("ppm", "hlld", "q26")
    st_e, st_g = mhd.to_device(cons, b), mhd.to_device(cons, b)
    torch.cuda.synchronize()
    assert ctx.last_dt() == 0.0  # no step_cfl yet
    for _ in range(4):
        ctx.step_cfl(st_e, 0.3, sch, 1e-3)
    dt_e = ctx.last_dt()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for _ in range(4):
            ctx.step_cfl(st_g, 0.3, sch, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(st_g.cons, mhd.to_device(cons, b).cons)  # capture ran nothing
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(st_e.cons, st_g.cons) and torch.equal(st_e.b, st_g.b)
    assert ctx.last_dt() == dt_e


def test_step_cfl_reports_a_non_finite_speed(gpu_lib):
    """A cell without a finite signal speed: step_cfl runs with dt = 0 and last_dt raises, as
    max_dt does."""
    shape = (8, 6, 5)
    cons, b, info = inputs.random_smooth(shape, seed=5, rough=0.05)
    cons = cons.copy()
    cons[4, 2, 3, 1] = np.inf  # infinite energy in one cell
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    ctx.step_cfl(st, 0.3, mhd.scheme("plm_mc", "hll", "q26"))
    with pytest.raises(RuntimeError):
        ctx.last_dt()
    with pytest.raises(RuntimeError):  # the host-side CFL step reports the same cell
        ctx.max_dt(mhd.to_device(cons, b), 0.3)


def test_fast_reciprocal_and_sqrt_against_ieee(gpu_lib):
    """The kernels' reciprocal / rsqrt / sqrt stay within a few ulp of CUDA's IEEE results."""
    ctx = mhd.Context((4, 4, 4), (1, 1, 1))
    er, es, eq, hbad, fbad, pbad, mbad = ctx.math_check(1 << 22)
    assert er <= 4 * 2.0**-53 and es <= 4 * 2.0**-53 and eq <= 4 * 2.0**-53, (er, es, eq)
    assert hbad == 0 and fbad == 0, (hbad, fbad)  # halving / quadrupling bit-exact
    assert pbad == 0, pbad  # sign tests, comparisons, min/max, |x|, sign copy / flip
    assert mbad == 0, mbad  # the integer-pipe multiply of the rate probe, bit for bit


def test_fp64_rate_probe(gpu_lib):
    """The FP64 rate probe: DFMA, DADD and DMUL each at 1-4 lanes per SM per clock at the GPU's
    clock (GB300's FP64 units), and the FP32 FMA many times faster."""
    import subprocess

    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    try:
        mhz = float(subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits",
                                    "-i", "0"], capture_output=True, text=True, timeout=30).stdout.split()[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        mhz = 2070.0
    rates = {k: mhd.fp64_rate(k, 1 << 13) for k in ("dfma", "dadd", "dmul", "ffma")}
    per_sm_clk = {k: v / nsm / (mhz * 1e6) for k, v in rates.items()}
    print("FP64 probe", {k: f"{v:.3e}/s ({per_sm_clk[k]:.2f}/SM/clk)" for k, v in rates.items()})
    for k in ("dfma", "dadd", "dmul"):
        assert 0.5 <= per_sm_clk[k] <= 4.5, per_sm_clk
    assert rates["ffma"] > 10 * rates["dfma"]
    # the integer-pipe multiply: a rate of the same order as the FP64 pipe's, alone and mixed
    mixed = {k: mhd.fp64_rate(k, 1 << 12) / nsm / (mhz * 1e6) for k in ("int_mul", "dfma_int_mul",
                                                                        "dfma_int_mul_2x128")}
    print("integer-pipe multiply", {k: f"{v:.2f}/SM/clk" for k, v in mixed.items()})
    assert all(0.2 <= v <= 8.0 for v in mixed.values()), mixed
    # DFMA on 16 and 8 lanes per warp: the active lanes' operations at no more than the full rate
    part = {k: mhd.fp64_rate(k, 1 << 12) / rates["dfma"] for k in ("dfma_16_lanes", "dfma_8_lanes")}
    print("DFMA on part of the warp, of the full-warp rate", {k: f"{v:.3f}" for k, v in part.items()})
    assert all(0.05 <= v <= 1.2 for v in part.values()), part
    with pytest.raises(mhd.MHDError):
        mhd.fp64_rate("dfma", 0)
    with pytest.raises(mhd.MHDError):
        lib = mhd.lib()
        import ctypes
        out = ctypes.c_double()
        rc = lib.mhd_fp64_rate(9, 1 << 10, None, ctypes.byref(out))
        if rc != mhd.OK:
            raise mhd.MHDError(rc, "kind 9")

