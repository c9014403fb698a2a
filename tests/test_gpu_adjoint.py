"""Hand-written adjoint of the step (mhd_step_adjoint, MHDEvolve) against the oracle (GPU).

Reference: the oracle run on forward-mode dual numbers gives the exact directional derivative
J v of the same steps (same frozen dts, same branches); the adjoint must satisfy
<lam, J v> = <J^T lam, v> to ~1e-10 relative. Central finite differences (h = 1e-6) of the GPU
forward run check the assembled torch gradient, including d/d(eta).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2609_10816_gb300 import adjoint, inputs, mhd
from tests.util import shock_state as _shock_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("recon,rs,emf", [("ppm", "hlld", "q26"), ("plm_mc", "hll", "q26"), ("plm_minmod", "llf", "q26"),
                                         ("pc", "hlld", "q26"), ("ppm_ep", "hlld", "q26"), ("ppm", "hlld", "fs18"),
                                         ("plm_mc", "hlld", "fs18"), ("ppm_ep", "hll", "fs18"), ("pc", "llf", "fs18"),
                                         ("ppm", "hlld", "b25a"), ("plm_mc", "hll", "b25a"), ("ppm_ep", "hlld", "b25a"),
                                         ("pc", "llf", "b25a")])
@pytest.mark.parametrize("eta", [0.0, 3e-3])
# the second: windows wrap onto themselves; the third: the reverse face solve's warps on 8 x 4
# patches of an x-y plane
@pytest.mark.parametrize("shape", [(10, 8, 6), (7, 4, 2), (16, 8, 6)])
def test_one_step_adjoint_identity(gpu_lib, recon, rs, emf, eta, shape):
    """<lam, J v> from the oracle's dual numbers equals <J^T lam, v> from the adjoint step (the
    line sweeps of the PPM reverse and the point-wise reverse of the other reconstructions), for
    the Q26, FS18 and B25a EMF compute schemes."""
    cons, b, info = inputs.random_smooth(shape, seed=21, rough=0.02)
    cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann=rs, emf=emf, eta=eta)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    rng = np.random.default_rng(1)
    lc, lb = rng.normal(size=cons.shape), rng.normal(size=b.shape)
    vc, vb, veta = rng.normal(size=cons.shape) * 1e-2, rng.normal(size=b.shape) * 1e-3, 0.7
    _, _, tc, tb = oracle.steps_jvp(cfg, cons, b, vc, vb, veta, [dt])
    lhs = (lc * tc).sum() + (lb * tb).sum()
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    lam = mhd.to_device(lc, lb)
    deta = ctx.step_adjoint(st, lam, dt, mhd.scheme(recon, rs, emf), eta)
    torch.cuda.synchronize()
    rc, rb = lam.cons.cpu().numpy(), lam.b.cpu().numpy()
    rhs = (rc * vc).sum() + (rb * vb).sum() + deta * veta
    print(f"ADJ {recon} {rs} {emf} eta={eta}: lhs {lhs:.15e} rhs {rhs:.15e} rel {abs(lhs - rhs) / abs(lhs):.2e}")
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + abs((rc * vc).sum()) + abs((rb * vb).sum()) + 1e-300), (lhs, rhs)
    # the state is not modified by the adjoint
    assert np.array_equal(st.cons.cpu().numpy(), cons) and np.array_equal(st.b.cpu().numpy(), b)


# (shape, seed, velocity amplitude, pressure, CFL, reconstruction, EMF compute): a few cells
# flagged after stage 1; half the box flagged after stage 1 and a few cells after stage 2; a few
# cells after each stage with PLM; the second again with FS18 and B25a, and PLM with B25a
# (their first-order corners take the cell velocities, and B25a's the cell fields)
FOFC_CASES = [((10, 8, 6), 1, 0.3, 1e-2, 0.4, "ppm", "q26"), ((10, 8, 6), 4, 3.0, 1e-3, 0.3, "ppm", "q26"),
              ((10, 8, 6), 4, 0.6, 1e-2, 0.6, "plm_mc", "q26"), ((10, 8, 6), 4, 3.0, 1e-3, 0.3, "ppm", "fs18"),
              ((10, 8, 6), 4, 3.0, 1e-3, 0.3, "ppm", "b25a"), ((10, 8, 6), 3, 1.0, 1e-2, 0.6, "plm_mc", "b25a")]


@pytest.mark.parametrize("case", range(len(FOFC_CASES)))
@pytest.mark.parametrize("eta", [0.0, 3e-3])
def test_flux_corrected_step_adjoint_identity(gpu_lib, case, eta):
    """Steps in which flux correction (Sec. 2.5) replaces fluxes with first-order ones, in stage 1
    and in stage 2: <lam, J v> from the oracle's dual numbers (the same flagged cells, taken from
    the values) equals <J^T lam, v> from the adjoint, to ~1e-10 relative."""
    shape, seed, amp, p0, cfl, recon, emf = FOFC_CASES[case]
    cons, b, info = _shock_state(shape, seed, amp, p0)
    cfg = oracle.Config(shape=shape, h=info["h"], recon=recon, riemann="hlld", emf=emf, eta=eta)
    dt = oracle.max_dt(cfg, cons, b, cfl)
    _, _, cnt = oracle.step(cfg, cons, b, dt)
    assert cnt[0] > 0 and (case == 0 or cnt[1] > 0), cnt
    sch = mhd.scheme(recon, "hlld", emf)
    ctx = mhd.Context(shape, info["h"])
    st = mhd.to_device(cons, b)
    ctx.step(mhd.to_device(cons, b), dt, sch, eta)
    assert ctx.stats() == cnt  # the GPU step flags the same cells' count
    rng = np.random.default_rng(2 + case)
    lc, lb = rng.normal(size=cons.shape), rng.normal(size=b.shape)
    vc, vb, veta = rng.normal(size=cons.shape) * 1e-3, rng.normal(size=b.shape) * 1e-4, 0.7
    _, _, tc, tb = oracle.steps_jvp(cfg, cons, b, vc, vb, veta, [dt])
    lhs = (lc * tc).sum() + (lb * tb).sum()
    lam = mhd.to_device(lc, lb)
    deta = ctx.step_adjoint(st, lam, dt, sch, eta)
    torch.cuda.synchronize()
    rc, rb = lam.cons.cpu().numpy(), lam.b.cpu().numpy()
    rhs = (rc * vc).sum() + (rb * vb).sum() + deta * veta
    scale = abs(lhs) + abs((rc * vc).sum()) + abs((rb * vb).sum()) + abs(deta * veta)
    print(f"ADJ-FOFC {case} eta={eta} flags={cnt}: lhs {lhs:.15e} rhs {rhs:.15e} rel {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-10 * scale, (lhs, rhs)
    assert np.array_equal(st.cons.cpu().numpy(), cons) and np.array_equal(st.b.cpu().numpy(), b)


def test_multistep_gradient_through_flux_correction(gpu_lib):
    """Three steps of a state that flux correction acts on, through MHDEvolve (checkpoints every 2):
    the torch gradient of the final sum of b^2 in the initial state and eta against the oracle's
    exact directional derivative."""
    shape = (10, 8, 6)
    cons, b, info = _shock_state(shape, 1, 0.3, 1e-2)
    eta0 = 2e-3
    sch = mhd.scheme("ppm", "hlld", "q26")
    cfg = oracle.Config(shape=shape, h=info["h"], recon="ppm", riemann="hlld", eta=eta0)
    dts, c, bb, flagged = [], cons, b, 0
    for _ in range(3):
        dts.append(oracle.max_dt(cfg, c, bb, 0.4))
        c, bb, cnt = oracle.step(cfg, c, bb, dts[-1])
        flagged += cnt[0] + cnt[1]
    assert flagged > 0
    dev = "cuda"
    c0 = torch.tensor(cons, device=dev, requires_grad=True)
    b0 = torch.tensor(b, device=dev, requires_grad=True)
    eta = torch.tensor(eta0, dtype=torch.float64, requires_grad=True)
    ctx = mhd.Context(shape, info["h"])
    cf, bf = adjoint.evolve(c0, b0, eta, ctx, dts, sch, every=2)
    (bf * bf).sum().backward()
    gc, gb, ge = c0.grad.cpu().numpy(), b0.grad.cpu().numpy(), float(eta.grad)
    rng = np.random.default_rng(9)
    for _ in range(2):
        vc, vb, veta = rng.normal(size=cons.shape) * 1e-3, rng.normal(size=b.shape) * 1e-4, rng.normal()
        _, bfin, _, tbf = oracle.steps_jvp(cfg, cons, b, vc, vb, veta, dts)
        exact = 2.0 * (bfin * tbf).sum()
        got = (gc * vc).sum() + (gb * vb).sum() + ge * veta
        assert abs(got - exact) <= 1e-9 * (abs(exact) + abs((gc * vc).sum()) + abs((gb * vb).sum())), (got, exact)


def _initial(shape, u, rho, p, b):
    """Conserved state from an initial velocity (torch, differentiable), density, pressure, field."""
    bc = 0.5 * (b + torch.stack([torch.roll(b[d], -1, dims=2 - d) for d in range(3)]))
    m = rho * u
    e = p / (5.0 / 3.0 - 1.0) + 0.5 * rho * (u * u).sum(0) + 0.5 * (bc * bc).sum(0)
    return torch.cat([rho[None], m, e[None]], 0)


def test_multistep_gradient_wrt_velocity_and_eta(gpu_lib):
    """L = sum of b^2 after 6 steps (checkpoints every 2): torch gradient vs the oracle's exact
    directional derivative and vs central differences of the GPU forward run."""
    shape = (12, 10, 8)
    cons, b, info = inputs.turbulence(shape, seed=2, v_rms=2.0)
    eta0 = 1e-3
    sch = mhd.scheme("ppm", "hlld", "q26")
    cfg = oracle.Config(shape=shape, h=info["h"], recon="ppm", riemann="hlld", eta=eta0)
    dts, c, bb = [], cons, b
    for _ in range(6):
        dts.append(oracle.max_dt(cfg, c, bb, 0.3))
        c, bb, _ = oracle.step(cfg, c, bb, dts[-1])
    dev = "cuda"
    rho = torch.tensor(cons[0], device=dev)
    u0 = torch.tensor(cons[1:4] / cons[0], device=dev, requires_grad=True)
    p = torch.tensor(np.full(cons[0].shape, 1.0 / (5.0 / 3.0)), device=dev)
    bt = torch.tensor(b, device=dev)
    eta = torch.tensor(eta0, dtype=torch.float64, requires_grad=True)
    ctx = mhd.Context(shape, info["h"])

    def loss(u, e):
        c0 = _initial(shape, u, rho, p, bt).contiguous()
        cf, bf = adjoint.evolve(c0, bt, e, ctx, dts, sch, every=2)
        return (bf * bf).sum()

    L = loss(u0, eta)
    L.backward()
    gu, geta = u0.grad.cpu().numpy(), float(eta.grad)
    rng = np.random.default_rng(5)
    for trial in range(2):
        vu = rng.normal(size=u0.shape)
        veta = rng.normal()
        # exact directional derivative from the oracle on dual numbers
        u_np = cons[1:4] / cons[0]
        dm = cons[0] * vu
        de = cons[0] * (u_np * vu).sum(0)
        dc = np.concatenate([np.zeros_like(cons[:1]), dm, de[None]], 0)
        _, bfin, _, tbf = oracle.steps_jvp(cfg, cons, b, dc, np.zeros_like(b), veta, dts)
        exact = 2.0 * (bfin * tbf).sum()
        got = (gu * vu).sum() + geta * veta
        assert abs(got - exact) <= 1e-9 * abs(exact), (got, exact)
        # central differences of the GPU forward run
        h = 1e-6
        with torch.no_grad():
            vt = torch.tensor(vu, device=dev)
            lp = float(loss(u0 + h * vt, eta + h * veta))
            lm = float(loss(u0 - h * vt, eta - h * veta))
        fd = (lp - lm) / (2 * h)
        assert abs(got - fd) <= 1e-5 * abs(fd), (got, fd)


@pytest.mark.parametrize("rs", ["hll", "hlld", "llf"])
def test_reverse_sweep_of_face_solve_matches_dual_numbers(gpu_lib, rs):
    """The adjoint's reverse sweep through the Riemann solver against 15 forward-mode passes on
    hashed face problems (equal, nearby and unrelated states, zero normal field, field along the
    normal, near-vacuum pressure, large velocities and fields). The two compute the same branch
    derivatives in different orders, so they differ by rounding times the problem's condition:
    a wrong term would give differences of order one. Over 2^16 problems every kind stays within
    1e-10; over 2^20 the rare near-singular HLLD problems (a denominator such as
    rho (S - u)(S - S_M) - b_n^2 just above the degeneracy threshold) reach ~1e-8, so the bound
    there is 1e-6, and 1e-12 for the well-conditioned kinds."""
    ctx = mhd.Context((4, 4, 4), (0.25, 0.25, 0.25))
    sch = mhd.scheme("ppm", rs, "q26")
    err16, kinds16 = ctx.adjoint_check(sch, n=1 << 16, seed=3)
    err20, kinds20 = ctx.adjoint_check(sch, n=1 << 20, seed=3)
    ctx.close()
    print(f"VJP {rs}: 2^16 {err16:.1e}, 2^20 " + " ".join(f"{k}={v:.1e}" for k, v in kinds20.items()))
    assert err16 == max(kinds16.values()) and err20 == max(kinds20.values())
    assert err16 <= 1e-10, kinds16
    assert err20 <= 1e-6, kinds20
    for k in ("equal", "bn_zero", "large"):
        assert kinds20[k] <= 1e-12, (k, kinds20)
