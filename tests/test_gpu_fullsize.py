"""Parity at the workloads' full sizes, in the launch configuration bench.py times (GPU).

A one-step update is local: through both stages, PPM + HLLD + Q26 + LD04 and flux correction
reach no further than ~16 cells. So a cell's result is reproduced by the oracle run on any
periodic sub-box that contains it with a 16-cell margin: the full-size GPU result is compared
with the oracle on the central 16^3 of 48^3 sub-boxes cut (periodically) around sample points.
Properties that hold at any size (div b at rounding, conservation) are checked on the whole box.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_10816_gb300 import inputs, mhd
from tests.util import MAX_TOL, field_scales, parity_failures, rel_l1, rel_max

pytestmark = pytest.mark.gpu

MARGIN = 16
INNER = 16


def _cut(cons, b, centre, widths):
    nz, ny, nx = cons.shape[1:]
    idx = [(centre[d] - widths[d] // 2 + np.arange(widths[d])) % (nx, ny, nz)[d] for d in range(3)]
    ix, iy, iz = idx
    c = cons[:, iz][:, :, iy][:, :, :, ix]
    bb = b[:, iz][:, :, iy][:, :, :, ix]
    return np.ascontiguousarray(c), np.ascontiguousarray(bb), idx


def _sampled_parity(cons, b, cg, bg, h, dt, scheme_kw, eta, centres, widths=(48, 48, 48), scales=None):
    """Oracle on sub-boxes around `centres` vs the GPU result cg/bg: central region only.
    Returns the worst relative L1 and asserts the element-wise bar on every compared cell."""
    if scales is None:
        scales = field_scales(cons, b)
    worst = 0.0
    for ctr in centres:
        sc, sb, idx = _cut(cons, b, ctr, widths)
        cfg = oracle.Config(shape=widths, h=h, eta=eta, **scheme_kw)
        oc, ob, _ = oracle.step(cfg, sc, sb, dt)
        gc, gb, _ = _cut(cg, bg, ctr, widths)
        sl = tuple(slice(MARGIN, w - MARGIN) if w > 2 * MARGIN else slice(None) for w in widths[::-1])
        for v in range(5):
            worst = max(worst, rel_l1(gc[v][sl], oc[v][sl], scales[0][v]))
            assert rel_max(gc[v][sl], oc[v][sl], scales[0][v]) <= MAX_TOL, (ctr, v)
        for d in range(3):
            worst = max(worst, rel_l1(gb[d][sl], ob[d][sl], scales[1][d]))
            assert rel_max(gb[d][sl], ob[d][sl], scales[1][d]) <= MAX_TOL, (ctr, "b", d)
    return worst


def _gpu_step(shape, h, cons, b, sch, eta, cfl=0.3):
    ctx = mhd.Context(shape, h)
    st = mhd.to_device(cons, b)
    dt = ctx.max_dt(st, cfl, eta)
    ctx.step(st, dt, sch, eta)
    torch.cuda.synchronize()
    md, mb = ctx.divb(st)
    out = st.cons.cpu().numpy(), st.b.cpu().numpy(), dt, md * min(h) / mb, ctx.stats()
    ctx.close()
    return out


def test_fast_wave_32cubed_100_steps_full(gpu_lib):
    """The 32^3 oblique fast eigenmode, PLM-MC + HLL + Q26 + LD04, CFL 0.3, all 100 steps."""
    shape = (32, 32, 32)
    cons, b, info = inputs.fast_wave(shape)
    cfg = oracle.Config(shape=shape, h=info["h"], recon="plm_mc", riemann="hll")
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    sch = mhd.scheme("plm_mc", "hll", "q26")
    co, bo = cons, b
    scales = field_scales(cons, b)
    for n in range(100):
        dt = ctx.max_dt(st, 0.3)
        ctx.step(st, dt, sch)
        co, bo, _ = oracle.step(cfg, co, bo, dt)
    torch.cuda.synchronize()
    cg, bg = st.cons.cpu().numpy(), st.b.cpu().numpy()
    bad = parity_failures(cg, bg, co, bo, scales)
    assert not bad, bad
    md, mb = ctx.divb(st)
    assert md * info["h"][0] / mb <= 1e-13


@pytest.mark.parametrize("emf", ["q26", "fs18", "b25a"])
def test_turbulence_256cubed_sampled(gpu_lib, emf):
    """256^3 Mach-5 turbulence, PPM + HLLD, each EMF compute scheme: one full-size GPU step
    (after two warm-up steps) against the oracle on four sampled sub-boxes."""
    n = 256
    cons, b, info = inputs.turbulence((n, n, n), seed=2, v_rms=5.0)
    sch = mhd.scheme("ppm", "hlld", emf)
    ctx = mhd.Context((n, n, n), info["h"])
    st = mhd.to_device(cons, b)
    for _ in range(2):
        ctx.step(st, ctx.max_dt(st, 0.3), sch)
    c0, b0 = st.cons.cpu().numpy(), st.b.cpu().numpy()
    dt = ctx.max_dt(st, 0.3)
    ctx.step(st, dt, sch)
    torch.cuda.synchronize()
    cg, bg = st.cons.cpu().numpy(), st.b.cpu().numpy()
    md, mb = ctx.divb(st)
    ctx.close()
    assert md * info["h"][0] / mb <= 1e-13
    for v in range(5):  # conservation over the whole box
        assert abs(cg[v].sum() - c0[v].sum()) <= 1e-12 * (np.abs(c0[v]).sum() + np.abs(c0[0]).sum())
    rng = np.random.default_rng(7)
    centres = [tuple(int(x) for x in rng.integers(0, n, 3)) for _ in range(4)]
    worst = _sampled_parity(c0, b0, cg, bg, info["h"], dt, dict(recon="ppm", riemann="hlld", emf=emf), 0.0, centres)
    assert worst <= 1e-12, worst


@pytest.mark.parametrize("recon,emf", [("ppm", "q26"), ("ppm", "fs18"), ("ppm", "b25a"), ("ppm_ep", "q26"),
                                      ("ppm_ep", "fs18"), ("ppm_ep", "b25a")])
def test_alfven_oblique_24cubed_full(gpu_lib, recon, emf):
    """The throughput workload's oblique Alfven wave (k ~ (1, 2, 3), theta = pi/4) at 24^3,
    PPM and the paper's PPM-EP with HLLD, each EMF compute scheme: 5 CFL steps against the oracle
    on the whole box."""
    shape = (24, 24, 24)
    cons, b, info = inputs.alfven_oblique(shape)
    cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann="hlld", emf=emf)
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    sch = mhd.scheme(recon, "hlld", emf)
    scales = field_scales(cons, b)
    co, bo = cons, b
    for _ in range(5):
        dt = ctx.max_dt(st, 0.3)
        ctx.step(st, dt, sch)
        co, bo, _ = oracle.step(cfg, co, bo, dt)
    torch.cuda.synchronize()
    cg, bg = st.cons.cpu().numpy(), st.b.cpu().numpy()
    bad = parity_failures(cg, bg, co, bo, scales)
    assert not bad, bad
    md, mb = ctx.divb(st)
    ctx.close()
    assert md * info["h"][0] / mb <= 1e-13


@pytest.mark.parametrize("recon,emf", [("ppm", "q26"), ("ppm_ep", "q26"), ("ppm_ep", "fs18"), ("ppm_ep", "b25a")])
def test_alfven_oblique_128cubed_sampled(gpu_lib, recon, emf):
    """The same wave at the throughput run's 128^3 with the paper's PPM-EP (and plain PPM): one
    full-size GPU step against the oracle on three sampled sub-boxes."""
    n = 128
    cons, b, info = inputs.alfven_oblique((n, n, n))
    sch = mhd.scheme(recon, "hlld", emf)
    cg, bg, dt, div, _ = _gpu_step((n, n, n), info["h"], cons, b, sch, 0.0)
    assert div <= 1e-13
    centres = [(0, 0, 0), (64, 32, 100), (17, 90, 45)]
    worst = _sampled_parity(cons, b, cg, bg, info["h"], dt, dict(recon=recon, riemann="hlld", emf=emf), 0.0,
                            centres)
    assert worst <= 1e-12, worst


def test_reconnection_512x512x4_sampled(gpu_lib):
    """512 x 512 x 4 double Harris sheet, eta = 1e-4, PLM-MC + HLLD + Q26 + LD04: one full-size
    step against the oracle on sub-boxes across both current sheets (all 4 cells in z)."""
    shape = (512, 512, 4)
    cons, b, info = inputs.harris_sheet(shape)
    sch = mhd.scheme("plm_mc", "hlld", "q26")
    cg, bg, dt, div, _ = _gpu_step(shape, info["h"], cons, b, sch, 1e-4)
    assert div <= 1e-13
    centres = [(256, 128, 2), (100, 384, 2), (400, 250, 2)]  # the sheets sit at y = +-1/4
    worst = _sampled_parity(cons, b, cg, bg, info["h"], dt, dict(recon="plm_mc", riemann="hlld", emf="q26"), 1e-4,
                            centres, widths=(48, 48, 4))
    assert worst <= 1e-12, worst


def test_reconnection_512x512x4_five_steps_sampled(gpu_lib):
    """Five full-size steps of the reconnection run (GPU dt sequence) against the oracle on two
    sub-boxes across the sheets, 192 x 192 x 4 each, compared on the central 32 x 32 x 4 (a margin
    of 80 cells covers five steps' reach of PLM + Q26 + flux correction)."""
    shape = (512, 512, 4)
    cons, b, info = inputs.harris_sheet(shape)
    sch = mhd.scheme("plm_mc", "hlld", "q26")
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    dts = []
    for _ in range(5):
        dts.append(ctx.max_dt(st, 0.3, 1e-4))
        ctx.step(st, dts[-1], sch, 1e-4)
    torch.cuda.synchronize()
    cg, bg = st.cons.cpu().numpy(), st.b.cpu().numpy()
    md, mb = ctx.divb(st)
    ctx.close()
    assert md * info["h"][0] / mb <= 1e-13
    scales = field_scales(cons, b)
    widths = (192, 192, 4)
    for ctr in [(256, 128, 2), (100, 384, 2)]:
        sc, sb, _ = _cut(cons, b, ctr, widths)
        cfg = oracle.Config(shape=widths, h=info["h"], recon="plm_mc", riemann="hlld", emf="q26", eta=1e-4)
        for dt in dts:
            sc, sb, _ = oracle.step(cfg, sc, sb, dt)
        gc, gb, _ = _cut(cg, bg, ctr, widths)
        sl = (slice(None), slice(80, 112), slice(80, 112))
        bad = parity_failures(gc[(slice(None),) + sl], gb[(slice(None),) + sl], sc[(slice(None),) + sl],
                              sb[(slice(None),) + sl], scales)
        assert not bad, (ctr, bad)


def test_batch_1024_patches_full(gpu_lib):
    """The 1024-patch batch (edges from {16, 24, 32, 48, 64}) with the autotuned schedule: one
    graph-replayed step; sampled patches equal single-box steps bitwise."""
    dims = [tuple(int(x) for x in d) for d in inputs.patch_dims(1024, seed=4)]
    rng = np.random.default_rng(4)
    h = 1.0 / 64
    pats = [inputs.random_patch(d, rng, h=h)[:2] for d in dims]
    bt = mhd.Batch(dims, h)
    cons, b = bt.pack(pats)
    sch = mhd.scheme("ppm", "hlld", "q26")
    bt.tune(cons, b, 0.3, sch)
    bt.step(cons, b, 0.3, sch)
    dt = bt.last_dt()
    pick = np.random.default_rng(11).choice(len(dims), 6, replace=False)
    for p in pick:
        c1, b1 = bt.unpack(cons, b, int(p))
        ctx = mhd.Context(dims[p], (h, h, h))
        st = mhd.to_device(*pats[p])
        ctx.step(st, dt, sch)
        torch.cuda.synchronize()
        assert np.array_equal(c1, st.cons.cpu().numpy()) and np.array_equal(b1, st.b.cpu().numpy()), p
        ctx.close()
    bt.close()
