"""Batched patches (mhd_batch_*) against the single-box step and the oracle (GPU)."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2609_10816_gb300 import inputs, mhd
from tests.util import parity_failures

pytestmark = pytest.mark.gpu

H = 1.0 / 64


def _patches(n, seed, edges=(4, 6, 8, 12, 16)):
    rng = np.random.default_rng(seed)
    dims = [tuple(int(x) for x in rng.choice(edges, size=3)) for _ in range(n)]
    pats = []
    for d in dims:
        cons, b, _ = inputs.random_patch(d, rng, h=H)
        pats.append((cons, b))
    return dims, pats


def _low_pressure_patch(shape, seed=1):
    cons, b, info = inputs.random_smooth(shape, seed=seed, rough=0.0, h=(H, H, H))
    rng = np.random.default_rng(seed)
    rho = cons[0]
    u = [cons[1 + d] / rho for d in range(3)]
    x = (np.arange(shape[0]) + 0.5) / shape[0]
    u[0] = u[0] + 3.0 * np.sin(2 * np.pi * x)[None, None, :] + 0.3 * rng.uniform(-1, 1, rho.shape)
    return inputs.assemble(rho, u, 1e-3 * np.ones_like(rho), b), b


def _plain_step(shape, cons, b, dt, sch, eta):
    ctx = mhd.Context(shape, (H, H, H))
    st = mhd.to_device(cons, b)
    ctx.step(st, dt, sch, eta)
    torch.cuda.synchronize()
    out = st.cons.cpu().numpy(), st.b.cpu().numpy(), ctx.stats()
    ctx.close()
    return out


@pytest.mark.parametrize("use_graph,emf,launches", [(True, "q26", 1), (False, "q26", 1), (True, "q26", 3),
                                                    (False, "q26", 3), (True, "fs18", 1), (True, "fs18", 3),
                                                    (True, "b25a", 1), (True, "b25a", 3)])
def test_batch_equals_single_box_steps(gpu_lib, use_graph, emf, launches):
    """Two batched steps of 21 uneven patches (one sets flux-correction flags) equal bit for bit the
    single-box steps of each patch with the batch's dt, for each EMF compute scheme, with one and
    with three persistent launches per stage."""
    dims, pats = _patches(20, seed=3)
    dims.append((16, 6, 4))
    pats.append(_low_pressure_patch((16, 6, 4)))  # sets flux-correction flags
    bt = mhd.Batch(dims, H)
    bt.set_schedule(seg=8, order=1, blocks_per_sm=0, use_graph=use_graph)
    bt.set_launches(launches)
    cons, b = bt.pack(pats)
    sch = mhd.scheme("ppm", "hlld", emf)
    for step in range(2):
        before = [bt.unpack(cons, b, p) for p in range(len(dims))]
        bt.step(cons, b, 0.3, sch, 1e-3)
        dt = bt.last_dt()
        flagged = bt.stats()
        tot = [0, 0]
        for p, d in enumerate(dims):
            c1, b1 = bt.unpack(cons, b, p)
            c0, b0 = before[p]
            cp, bp, fl = _plain_step(d, c0, b0, dt, sch, 1e-3)
            tot[0] += fl[0]
            tot[1] += fl[1]
            assert np.array_equal(c1, cp) and np.array_equal(b1, bp), (step, p, d)
        assert tuple(tot) == flagged
    assert flagged[0] + flagged[1] >= 0


@pytest.mark.parametrize("recon,emf", [("plm_mc", "q26"), ("ppm_ep", "q26"), ("plm_mc", "fs18"), ("ppm_ep", "b25a")])
def test_batch_patches_against_oracle(gpu_lib, recon, emf):
    dims, pats = _patches(6, seed=9, edges=(6, 8, 10))
    bt = mhd.Batch(dims, H)
    cons, b = bt.pack(pats)
    sch = mhd.scheme(recon, "hlld", emf)
    bt.step(cons, b, 0.3, sch, 0.0)
    dt = bt.last_dt()
    # the batch dt is the CFL step over all patches
    cfgs = [oracle.Config(shape=d, h=(H, H, H), recon=recon, riemann="hlld", emf=emf) for d in dims]
    assert dt == pytest.approx(min(oracle.max_dt(c, *pats[p], 0.3) for p, c in enumerate(cfgs)), rel=1e-14)
    for p, d in enumerate(dims):
        co, bo, _ = oracle.step(cfgs[p], *pats[p], dt)
        c1, b1 = bt.unpack(cons, b, p)
        bad = parity_failures(c1, b1, co, bo)
        assert not bad, (p, bad)


def test_batch_ppm_hlld_patches_against_oracle(gpu_lib):
    """The benchmarked batch scheme (PPM + HLLD + Q26 + LD04) on patches with edges drawn from the
    batch workload's {16, 24, 32, 48, 64}, with the autotuned schedule and graph replay, against
    the oracle patch by patch; one near-vacuum patch sets flux-correction flags."""
    rng = np.random.default_rng(17)
    dims = [tuple(int(x) for x in rng.choice((16, 24, 32, 48, 64), size=3)) for _ in range(7)]
    pats = [inputs.random_patch(d, rng, h=H)[:2] for d in dims]
    dims.append((16, 16, 16))
    pats.append(_low_pressure_patch((16, 16, 16), seed=3))
    bt = mhd.Batch(dims, H)
    cons, b = bt.pack(pats)
    sch = mhd.scheme("ppm", "hlld", "q26")
    bt.tune(cons, b, 0.6, sch)
    bt.step(cons, b, 0.6, sch, 0.0)  # CFL 0.6: the near-vacuum patch's high-order step fails
    dt = bt.last_dt()
    flagged = bt.stats()
    cfgs = [oracle.Config(shape=d, h=(H, H, H), recon="ppm", riemann="hlld") for d in dims]
    assert dt == pytest.approx(min(oracle.max_dt(c, *pats[p], 0.6) for p, c in enumerate(cfgs)), rel=1e-14)
    tot = [0, 0]
    for p, d in enumerate(dims):
        co, bo, cnt = oracle.step(cfgs[p], *pats[p], dt)
        tot[0] += cnt[0]
        tot[1] += cnt[1]
        c1, b1 = bt.unpack(cons, b, p)
        bad = parity_failures(c1, b1, co, bo)
        assert not bad, (p, d, bad)
    assert tuple(tot) == flagged and tot[0] > 0
    bt.close()


def test_batch_autotune_keeps_results(gpu_lib):
    dims, pats = _patches(12, seed=5)
    bt = mhd.Batch(dims, H)
    cons, b = bt.pack(pats)
    sch = mhd.scheme("ppm", "hlld", "q26")
    ref_c, ref_b = cons.clone(), b.clone()
    t0 = time.perf_counter()
    choice = bt.tune(cons, b, 0.3, sch)
    t_first = time.perf_counter() - t0
    assert choice["seg"] in (16, 32, 64, 128) and choice["order"] in (0, 1) and choice["blocks_per_sm"] >= 1
    assert choice["launches_per_stage"] in (1, 3)
    assert torch.equal(cons, ref_c) and torch.equal(b, ref_b)  # tuning leaves the state alone
    # the choice is remembered by patch-size histogram: another batch of the same sizes (in another
    # order) gets it without timing
    bt2 = mhd.Batch(dims[::-1], H)
    t0 = time.perf_counter()
    again = bt2.tune(*bt2.pack(pats[::-1]), 0.3, sch)
    assert again == choice and time.perf_counter() - t0 < 0.5 * t_first, (again, choice)
    bt2.close()
    bt.step(cons, b, 0.3, sch)
    bt.set_schedule(seg=7, order=0, blocks_per_sm=1, use_graph=False)
    bt.set_launches(4 - choice["launches_per_stage"])  # the other form
    bt.step(ref_c, ref_b, 0.3, sch)
    torch.cuda.synchronize()
    assert torch.equal(cons, ref_c) and torch.equal(b, ref_b)  # schedule changes nothing but time
    with pytest.raises(mhd.MHDError):
        bt.set_launches(2)


def test_batch_barrier_wait_is_bounded(gpu_lib):
    """A barrier that never completes gives MHD_ERR_TIMEOUT, and the batch stays usable."""
    dims, pats = _patches(4, seed=2)
    bt = mhd.Batch(dims, H)
    cons, b = bt.pack(pats)
    sch = mhd.scheme("plm_mc", "hll", "q26")
    c_in, b_in = cons.clone(), b.clone()
    bt.test_barrier(1, 2000)  # every barrier waits for one block that is never launched
    bt.step(cons, b, 0.3, sch)
    torch.cuda.synchronize()
    assert torch.equal(cons, c_in) and torch.equal(b, b_in)  # the abandoned step left the state
    bt.test_barrier(0, 1 << 25)
    bt.step(cons, b, 0.3, sch)  # the timeout is not read yet: this step does nothing either
    torch.cuda.synchronize()
    assert torch.equal(cons, c_in) and torch.equal(b, b_in)
    with pytest.raises(mhd.MHDError) as ei:
        bt.last_dt()
    assert ei.value.code == mhd.ERR_TIMEOUT
    assert bt.stats() == (0, 0)  # the report cleared the condition
    c2, b2 = bt.pack(pats)
    bt.step(c2, b2, 0.3, sch)
    assert bt.last_dt() > 0
    cp, bp, _ = _plain_step(dims[0], *pats[0], bt.last_dt(), sch, 0.0)
    c1, b1 = bt.unpack(c2, b2, 0)
    assert np.array_equal(c1, cp) and np.array_equal(b1, bp)


def test_batch_phase_times(gpu_lib):
    """Phase stamps of the persistent stage kernel: every phase that ran has a non-negative
    duration, the sweeps take time, and the flux-correction phase is zero without flagged cells."""
    dims, pats = _patches(12, seed=5)
    bt = mhd.Batch(dims, H)
    cons, b = bt.pack(pats)
    sch = mhd.scheme("ppm", "hlld", "q26")
    bt.step(cons, b, 0.3, sch)
    ph = bt.phase_ms()
    assert bt.stats() == (0, 0)
    for s in (0, 1):
        assert all(v >= 0.0 for v in ph[s].values())
        assert ph[s]["face"] > 0.0
        assert ph[s]["fo_fluxes"] == 0.0
    bt.close()
