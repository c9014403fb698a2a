"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each pin is chosen so that a plausible mistake in the oracle fails it: a wrong sign or index in
a flux or EMF breaks conservation, the divergence, the eigenmode's convergence or the symmetry
checks; a wrong Riemann fan breaks the exact-discontinuity cases; a wrong Ohmic or Joule term
breaks the resistive decay rate or the Joule-heating profile; a wrong flux-correction mask
breaks the forward-Euler special case.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2609_10816_gb300 import inputs
from tests.util import relerr_pert, shock_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = 5.0 / 3.0
ALL = [(r, s, e) for r in ("pc", "plm_mc", "plm_minmod", "ppm", "ppm_ep") for s in ("hll", "hlld", "llf")
       for e in ("q26", "fs18", "b25a")]


def cfg_for(shape, info, **kw):
    return oracle.Config(shape=shape, h=info["h"], **kw)


# ---------------------------------------------------------------------------------------
# Reconstruction (Sec. 2.2): hand-computed cases and exactness on linear data
# ---------------------------------------------------------------------------------------
def _golden_recon():
    rows = []
    with open(os.path.join(GOLDEN, "recon_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            m, vals, qm, qp = [x.strip() for x in line.split(";")]
            rows.append((m, [float(v) for v in vals.split()], float(qm), float(qp)))
    return rows


@pytest.mark.parametrize("method,vals,qm,qp", _golden_recon())
def test_recon_golden(method, vals, qm, qp):
    q = np.asarray(vals, float).reshape(1, 1, 7)
    cfg = oracle.Config(shape=(7, 1, 1), h=(1, 1, 1))
    m, p = oracle.recon(cfg, method, q, 0)
    assert m[0, 0, 3] == pytest.approx(qm, abs=1e-15)
    assert p[0, 0, 3] == pytest.approx(qp, abs=1e-15)


@pytest.mark.parametrize("method", ["plm_mc", "plm_minmod", "ppm", "ppm_ep"])
@pytest.mark.parametrize("d", [0, 1, 2])
def test_recon_exact_on_linear_data(method, d):
    n = 16
    shape = [3, 3, 3]
    shape[d] = n
    ramp = np.concatenate([np.arange(10.0), 10 - 1.7 * np.arange(1, 7)])  # periodic, linear inside
    q = np.broadcast_to(ramp.reshape([-1 if a == 2 - d else 1 for a in range(3)]),
                        (shape[2], shape[1], shape[0])).copy()
    cfg = oracle.Config(shape=tuple(shape), h=(1, 1, 1))
    m, p = oracle.recon(cfg, method, q, d)
    idx = [slice(None)] * 3
    idx[2 - d] = slice(3, 7)  # points whose stencil lies on the rising ramp
    assert np.allclose(m[tuple(idx)], q[tuple(idx)] - 0.5, atol=1e-14)
    assert np.allclose(p[tuple(idx)], q[tuple(idx)] + 0.5, atol=1e-14)


def _sine_cell_averages(n, phase=0.3):
    """Exact cell averages of sin(2 pi x + phase) on n cells of [0, 1), and the exact values at the
    cells' lower and upper faces."""
    xf = np.arange(n + 1) / n
    F = -np.cos(2 * np.pi * xf + phase) / (2 * np.pi)
    return (F[1:] - F[:-1]) * n, np.sin(2 * np.pi * xf[:-1] + phase), np.sin(2 * np.pi * xf[1:] + phase)


def test_ppm_ep_fourth_order_at_smooth_extrema():
    """PPM-EP's interface values are those of the fourth-order interpolant of cell averages
    wherever the data are smooth, extrema included: the largest face error on a sine falls 16x per
    doubling. Plain PPM clips the extrema (Sec. 3.1.5 traces its error floor to that) and its
    largest error falls only about 4x."""
    errs = {}
    for m in ("ppm", "ppm_ep"):
        errs[m] = []
        for n in (16, 32, 64, 128):
            q, lo, hi = _sine_cell_averages(n)
            cfg = oracle.Config(shape=(n, 1, 1), h=(1.0 / n, 1, 1))
            qm, qp = oracle.recon(cfg, m, q.reshape(1, 1, n), 0)
            errs[m].append(max(np.abs(qm.ravel() - lo).max(), np.abs(qp.ravel() - hi).max()))
    ep = np.array(errs["ppm_ep"])
    assert (ep[:-1] / ep[1:] > 15.0).all(), ep
    pp = np.array(errs["ppm"])
    assert (pp[-2:] / ep[-2:] > 500.0).all() and pp[-2] / pp[-1] < 6.0, (pp, ep)


# ---------------------------------------------------------------------------------------
# Riemann solvers (Sec. 2.2): closed forms, consistency and exact discontinuities
# ---------------------------------------------------------------------------------------
W_CASE = np.array([2.0, 0.5, 0.1, -0.2, 1.0, 0.4, -0.1])  # rho, u_n, u_t1, u_t2, p, b_t1, b_t2
BN_CASE = 0.3
F_CASE = np.array([1.0, 1.54, -0.02, -0.17, 1.467])  # Eq. (mhd:conservation-laws) by hand


@pytest.mark.parametrize("solver", ["hll", "hlld", "llf"])
def test_riemann_consistency(solver):
    F, ap, am, us = oracle.riemann(solver, G, W_CASE, W_CASE, BN_CASE)
    assert np.allclose(F, F_CASE, rtol=0, atol=1e-14)
    assert ap >= 0 and am >= 0
    assert us == pytest.approx(W_CASE[1], abs=1e-15)


def test_fast_speed_closed_forms():
    # static uniform state, c_s = 1 (p = 1/gamma, rho = 1), |b| = 2
    par = np.array([1.0, 0, 0, 0, 1 / G, 0, 0])  # b along the normal: c_f = max(c_s, c_A) = 2
    _, ap, am, _ = oracle.riemann("hll", G, par, par, 2.0)
    assert ap == pytest.approx(2.0, rel=1e-15) and am == pytest.approx(2.0, rel=1e-15)
    perp = np.array([1.0, 0, 0, 0, 1 / G, 2.0, 0])  # b normal to it: c_f = sqrt(c_s^2 + c_A^2)
    _, ap, am, _ = oracle.riemann("hlld", G, perp, perp, 0.0)
    assert ap == pytest.approx(np.sqrt(5.0), rel=1e-15)
    # oblique, theta = 60 deg: Eq. (waves:fast-speed)
    ob = np.array([1.0, 0, 0, 0, 1 / G, 2.0 * np.sin(np.pi / 3), 0])
    cf2 = 0.5 * (1 + 4 + np.sqrt(25 - 4 * 4 * 0.25))
    _, ap, _, _ = oracle.riemann("llf", G, ob, ob, 2.0 * np.cos(np.pi / 3))
    assert ap == pytest.approx(np.sqrt(cf2), rel=1e-14)


def test_hlld_resolves_stationary_contact_hll_does_not():
    WL = np.array([1.0, 0, 0, 0, 1.0, 0.3, 0.0])
    WR = np.array([2.0, 0, 0, 0, 1.0, 0.3, 0.0])
    F, *_ = oracle.riemann("hlld", G, WL, WR, 0.5)
    assert abs(F[0]) < 1e-15 and abs(F[4]) < 1e-15
    assert F[1] == pytest.approx(1.0 + 0.5 * (0.25 + 0.09) - 0.25, abs=1e-15)
    Fh, *_ = oracle.riemann("hll", G, WL, WR, 0.5)
    assert abs(Fh[0]) > 1e-2


def test_hlld_resolves_rotational_discontinuity():
    # stationary Alfvenic discontinuity: rho = 1, p = 1, bn = 1, u_n = c_An = 1, b_t rotates by
    # 90 deg and u_t jumps by delta b_t (jump conditions rho u_n du_t = bn db_t, u_n db_t = bn du_t)
    WL = np.array([1.0, 1.0, 0.0, 0.0, 1.0, 1.0, 0.0])
    WR = np.array([1.0, 1.0, -1.0, 1.0, 1.0, 0.0, 1.0])
    F, *_ = oracle.riemann("hlld", G, WL, WR, 1.0)
    exact = np.array([1.0, 2.0, -1.0, 0.0, 4.0])  # F_L = F_R
    assert np.allclose(F, exact, atol=1e-13)
    Fh, *_ = oracle.riemann("hll", G, WL, WR, 1.0)
    assert np.abs(Fh - exact).max() > 1e-2


def test_hlld_moving_rotational_discontinuity_double_star_region():
    # the same discontinuity moving at V = -0.2 (u_n = 0.8 on both sides): the face x/t = 0 lies
    # between the rotational wave and the contact, so the exact flux is the physical flux of the
    # right state, reached through HLLD's double-star state
    WL = np.array([1.0, 0.8, 0.0, 0.0, 1.0, 1.0, 0.0])
    WR = np.array([1.0, 0.8, -1.0, 1.0, 1.0, 0.0, 1.0])
    F, *_ = oracle.riemann("hlld", G, WL, WR, 1.0)
    FR, *_ = oracle.riemann("hlld", G, WR, WR, 1.0)  # = F(U_R) by the consistency pin
    assert np.allclose(F, FR, atol=1e-13)
    Fh, *_ = oracle.riemann("hll", G, WL, WR, 1.0)
    assert np.abs(Fh - FR).max() > 1e-2


@pytest.mark.parametrize("bn", [1.0, -1.0])
def test_hlld_exact_for_rotational_plus_contact(bn):
    # L | left-going rotational discontinuity | M | contact | R, with no fast waves: M has L's
    # density, rotated b_t and u_t = u_t,L + sgn(bn) db_t / sqrt(rho); R differs from M only in
    # density. HLLD's estimates are exact here (S_M = u_n, rho* = rho), so its double-star state
    # is M and the flux at x/t = 0 (between the waves at -0.7 and +0.3) is F(U_M).
    sg = np.sign(bn)
    WL = np.array([1.0, 0.3, 0.0, 0.0, 1.0, 1.0, 0.0])
    WM = np.array([1.0, 0.3, -1.0 * sg, 1.0 * sg, 1.0, 0.0, 1.0])
    WR = WM.copy()
    WR[0] = 2.0
    F, *_ = oracle.riemann("hlld", G, WL, WR, bn)
    FM, *_ = oracle.riemann("hlld", G, WM, WM, bn)
    assert np.allclose(F, FM, atol=1e-13)


def _hllc_toro(WL, WR, SL, SR, gam):
    """Textbook HLLC flux (Toro, Riemann Solvers and Numerical Methods, Sec. 10.4) for the Euler
    equations, W = (rho, u, v, w, p), with given outer wave speeds."""
    def cons_flux(W):
        r, u, v, w, p = W
        E = p / (gam - 1) + 0.5 * r * (u * u + v * v + w * w)
        U = np.array([r, r * u, r * v, r * w, E])
        F = np.array([r * u, r * u * u + p, r * u * v, r * u * w, u * (E + p)])
        return U, F
    UL, FL = cons_flux(WL)
    UR, FR = cons_flux(WR)
    rL, uL, pL = WL[0], WL[1], WL[4]
    rR, uR, pR = WR[0], WR[1], WR[4]
    Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))
    def star(W, U, S):
        r, u, v, w, p = W
        f = r * (S - u) / (S - Ss)
        return f * np.array([1.0, Ss, v, w, U[4] / r + (Ss - u) * (Ss + p / (r * (S - u)))])
    if SL >= 0:
        return FL
    if Ss >= 0:
        return FL + SL * (star(WL, UL, SL) - UL)
    if SR >= 0:
        return FR + SR * (star(WR, UR, SR) - UR)
    return FR


@pytest.mark.parametrize("seed", range(6))
def test_hlld_reduces_to_hllc_without_field(seed):
    rng = np.random.default_rng(seed)
    WL = np.array([rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1),
                   rng.uniform(0.5, 2), 0.0, 0.0])
    WR = np.array([rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1),
                   rng.uniform(0.5, 2), 0.0, 0.0])
    F, ap, am, _ = oracle.riemann("hlld", G, WL, WR, 0.0)
    assert ap > 0 and am > 0  # S_L = -alpha-, S_R = alpha+ straddle the face
    Fc = _hllc_toro(WL[:5], WR[:5], -am, ap, G)
    assert np.allclose(F, Fc, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", range(4))
def test_hlld_flux_continuous_as_contact_crosses_face(seed):
    # The fan is built from both sides; where S_M passes x/t = 0 the left- and right-built fluxes
    # must agree (integral consistency of the intermediate states), so the flux is continuous in
    # a Galilean boost V of both states along the normal.
    rng = np.random.default_rng(100 + seed)
    def w():
        return np.array([rng.uniform(0.5, 2), rng.uniform(-0.5, 0.5), rng.uniform(-1, 1), rng.uniform(-1, 1),
                         rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1)])
    WL, WR = w(), w()
    bn = rng.uniform(0.3, 1.0)
    Vs = np.linspace(-2.0, 2.0, 4001)
    Fs = []
    for V in Vs:
        a, b_ = WL.copy(), WR.copy()
        a[1] += V
        b_[1] += V
        Fs.append(oracle.riemann("hlld", G, a, b_, bn)[0])
    jumps = np.abs(np.diff(np.array(Fs), axis=0)).max(axis=0)
    assert (jumps <= 0.02).all(), jumps  # step dV = 1e-3; a side inconsistency jumps by O(1)


# ---------------------------------------------------------------------------------------
# Whole step: conservation, divergence, symmetry (every scheme combination, 8^3)
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("recon,rs,emf", ALL)
def test_conservation_and_divergence_all_schemes(recon, rs, emf):
    shape = (8, 8, 8)
    cons, b, info = inputs.random_smooth(shape, seed=21, rough=0.05)
    cfg = cfg_for(shape, info, recon=recon, riemann=rs, emf=emf, eta=1e-3)
    c, bb, dts, _ = oracle.run(cfg, cons, b, 3)
    for v in range(5):
        scale = np.abs(cons[v]).sum() + np.abs(cons[0]).sum()
        assert abs(c[v].sum() - cons[v].sum()) <= 1e-13 * scale
    md, mb = oracle.divb(cfg, bb)
    assert md * min(info["h"]) / mb <= 1e-13
    assert np.isfinite(c).all()


def _rotate(cons, b, h):
    """Cyclic relabelling of axes: new x0 = old x1, new x1 = old x2, new x2 = old x0."""
    rc = np.empty((5,) + cons.shape[1:][::1])
    rc = np.stack([cons[0].transpose(2, 0, 1), cons[2].transpose(2, 0, 1), cons[3].transpose(2, 0, 1),
                   cons[1].transpose(2, 0, 1), cons[4].transpose(2, 0, 1)])
    rb = np.stack([b[1].transpose(2, 0, 1), b[2].transpose(2, 0, 1), b[0].transpose(2, 0, 1)])
    return np.ascontiguousarray(rc), np.ascontiguousarray(rb), (h[1], h[2], h[0])


def _reflect(cons, b):
    """Point reflection x -> -x through the box centre."""
    rc = np.flip(cons, axis=(1, 2, 3)).copy()
    rc[1:4] *= -1
    rb = np.empty_like(b)
    for d in range(3):
        rb[d] = -np.roll(np.flip(b[d], axis=(0, 1, 2)), 1, axis=2 - d)
    return rc, rb


@pytest.mark.parametrize("recon,rs,emf", [("ppm", "hlld", "q26"), ("plm_mc", "hll", "fs18"),
                                          ("plm_minmod", "llf", "b25a"), ("ppm_ep", "hlld", "q26")])
def test_cyclic_permutation_symmetry(recon, rs, emf):
    shape = (6, 5, 4)
    h = (0.1, 0.12, 0.09)
    cons, b, info = inputs.random_smooth(shape, seed=4, rough=0.05, h=h)
    cfg = oracle.Config(shape=shape, h=h, recon=recon, riemann=rs, emf=emf, eta=2e-3)
    dt = 0.5 * oracle.max_dt(cfg, cons, b, 0.3)
    c1, b1, _ = oracle.step(cfg, cons, b, dt)
    rc, rb, rh = _rotate(cons, b, h)
    cfg_r = oracle.Config(shape=(shape[1], shape[2], shape[0]), h=rh, recon=recon, riemann=rs, emf=emf, eta=2e-3)
    c2, b2, _ = oracle.step(cfg_r, rc, rb, dt)
    ec, eb, _ = _rotate(c1, b1, h)
    assert np.abs(c2 - ec).max() <= 1e-13 * np.abs(ec).max()
    assert np.abs(b2 - eb).max() <= 1e-13 * np.abs(eb).max()


@pytest.mark.parametrize("recon,rs,emf", [("ppm", "hlld", "q26"), ("plm_mc", "hll", "b25a"),
                                          ("plm_mc", "llf", "fs18"), ("ppm_ep", "hlld", "q26"),
                                          ("ppm_ep", "hll", "fs18")])
def test_point_reflection_symmetry(recon, rs, emf):
    shape = (6, 6, 6)
    cons, b, info = inputs.random_smooth(shape, seed=9, rough=0.05)
    cfg = cfg_for(shape, info, recon=recon, riemann=rs, emf=emf, eta=1e-3)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    c1, b1, _ = oracle.step(cfg, cons, b, dt)
    rc, rb = _reflect(cons, b)
    c2, b2, _ = oracle.step(cfg, rc, rb, dt)
    ec, eb = _reflect(c1, b1)
    assert np.abs(c2 - ec).max() <= 1e-13 * np.abs(ec).max()
    assert np.abs(b2 - eb).max() <= 1e-13 * np.abs(eb).max()


# ---------------------------------------------------------------------------------------
# EMF compute schemes (Sec. 2.3.1): corner EMFs of Q26, FS18 and B25a
# ---------------------------------------------------------------------------------------
def _uniform_state(shape, rho, u, p, bvec):
    nx, ny, nz = shape
    cons = np.empty((5, nz, ny, nx))
    cons[0] = rho
    for d in range(3):
        cons[1 + d] = rho * u[d]
    cons[4] = p / (G - 1.0) + 0.5 * rho * float(np.dot(u, u)) + 0.5 * float(np.dot(bvec, bvec))
    b = np.empty((3, nz, ny, nx))
    for d in range(3):
        b[d] = bvec[d]
    return cons, b


@pytest.mark.parametrize("recon", ["pc", "plm_mc", "plm_minmod", "ppm"])
@pytest.mark.parametrize("rs", ["hll", "hlld", "llf"])
@pytest.mark.parametrize("emf", ["q26", "fs18", "b25a"])
def test_uniform_state_corner_and_edge_emf_is_minus_u_cross_b(recon, rs, emf):
    """For a uniform state every reconstruction returns the cell value, so each of the four
    corner estimates of every compute scheme (Eqs. q26, fs18 with fs18-average, b25a-*) and
    the averaged edge EMF of Eq. (ld04) must equal eps = -u x b, whatever the averaging weights
    and the speeds; a wrong weight, sign or component in any scheme breaks this."""
    shape = (5, 4, 3)
    u = np.array([0.3, -0.7, 0.45])
    bvec = np.array([0.8, 0.35, -0.6])
    cons, b = _uniform_state(shape, 1.3, u, 0.9, bvec)
    cfg = oracle.Config(shape=shape, h=(0.2, 0.25, 1.0 / 3.0), recon=recon, riemann=rs, emf=emf)
    eps = -np.cross(u, bvec)
    C = oracle.corner_emfs(cfg, cons, b)
    _, E = oracle.fluxes(cfg, cons, b)
    for e in range(3):
        assert np.abs(C[e] - eps[e]).max() <= 4e-16 * np.abs(eps).max(), (e, C[e].ravel()[:4], eps[e])
        assert np.abs(E[e] - eps[e]).max() <= 4e-16 * np.abs(eps).max(), (e, E[e].ravel()[:4], eps[e])


def _golden_corners():
    rows = []
    with open(os.path.join(GOLDEN, "corner_emf_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            case, emf, table, expect = [x.strip() for x in line.split(";")]
            vals = np.array([float(v) for v in table.split()]).reshape(6, 6)  # [j][i]
            exp = {int(k): float(v) for k, v in (t.split(":") for t in expect.split())}
            rows.append((case, emf, vals, exp))
    return rows


@pytest.mark.parametrize("case,emf,table,expect", _golden_corners())
def test_corner_emfs_hand_computed(case, emf, table, expect):
    """FS18 and B25a corner EMFs on a 6 x 6 x 1 stencil, each corner derived by hand in
    tests/golden/corner_emf_cases.txt from Eqs. (fs18-average), (fs18), (b25a-b-avg),
    (b25a-emf-centre) and (b25a-average) with PLM-minmod: both reconstruction orders, their
    mean, and the product with the reconstructed field."""
    shape = (6, 6, 1)
    cons = np.zeros((5, 1, 6, 6))
    b = np.zeros((3, 1, 6, 6))
    cons[0] = 1.0
    if case == "velocity":
        cons[1, 0] = table
        b[1] = 1.0
    else:
        cons[1] = 1.0
        b[1, 0] = table
    bcell = 0.5 * (b[1] + np.roll(b[1], -1, axis=1))
    cons[4] = 1.0 / (G - 1.0) + 0.5 * (cons[1] ** 2 + cons[2] ** 2 + cons[3] ** 2) / cons[0] + 0.5 * bcell**2
    cfg = oracle.Config(shape=shape, h=(1.0, 1.0, 1.0), recon="plm_minmod", riemann="hll", emf=emf)
    C = oracle.corner_emfs(cfg, cons, b)
    for q, v in expect.items():
        assert C[2, q, 0, 2, 2] == v, (case, emf, q, C[2, :, 0, 2, 2], v)


@pytest.mark.parametrize("emf", ["fs18", "b25a"])
def test_fast_wave_second_order_3d_diagonal_fs18_b25a(emf):
    """Sec. 3.1.5: every compute scheme converges at second order. The oblique-diagonal fast
    eigenmode of the 32^3 workload with PLM-MC + HLL at 16^3 and 32^3."""
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        cons, b, info = inputs.fast_wave(shape)
        cbg, bbg, _ = inputs.fast_wave(shape, amp=0.0)
        cfg = cfg_for(shape, info, recon="plm_mc", riemann="hll", emf=emf)
        c, bb = _one_period(cfg, cons, b, info["period"])
        errs.append(_relerr_pert(cons, b, c, bb, cbg, bbg))
    assert errs[0] / errs[1] > 3.0, errs


def test_oblique_alfven_wave_second_order_ppm_ep():
    """The throughput workload as the paper runs it (Sec. 3.6): PPM-EP + HLLD + Q26 on the oblique
    Alfven wave returns to its initial state after one period with a second-order error ratio
    from 16^3 to 32^3, below plain PPM's error at 32^3."""
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        cons, b, info = inputs.alfven_oblique(shape)
        cbg, bbg, _ = inputs.alfven_oblique(shape, amp=0.0)
        cfg = cfg_for(shape, info, recon="ppm_ep", riemann="hlld")
        c, bb = _one_period(cfg, cons, b, 2 * np.pi / info["omega"])
        errs.append(_relerr_pert(cons, b, c, bb, cbg, bbg))
    assert errs[0] / errs[1] > 3.0, errs


@pytest.mark.parametrize("emf", ["fs18", "b25a"])
def test_oblique_alfven_wave_second_order_ppm_hlld_fs18_b25a(emf):
    """Sec. 3.1.5 for the comparison schemes: the oblique linear Alfven wave of the throughput
    workload with PPM + HLLD returns to its initial state after one period, the error falling
    towards second order from 16^3 to 32^3."""
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        cons, b, info = inputs.alfven_oblique(shape)
        cbg, bbg, _ = inputs.alfven_oblique(shape, amp=0.0)
        cfg = cfg_for(shape, info, recon="ppm", riemann="hlld", emf=emf)
        c, bb = _one_period(cfg, cons, b, 2 * np.pi / info["omega"])
        errs.append(_relerr_pert(cons, b, c, bb, cbg, bbg))
    assert errs[0] / errs[1] > 3.0, errs


# ---------------------------------------------------------------------------------------
# Convergence against closed-form waves (Sec. 3.1, Eq. error:relative)
# ---------------------------------------------------------------------------------------
_relerr_pert = relerr_pert  # Eq. (error:relative), normalised by the perturbation


def _one_period(cfg, cons, b, T, cfl=0.3):
    t = 0.0
    while t < T - 1e-14:
        dt = min(oracle.max_dt(cfg, cons, b, cfl), T - t)
        cons, b, _ = oracle.step(cfg, cons, b, dt)
        t += dt
    return cons, b


@pytest.mark.parametrize("recon,rs", [("plm_mc", "hll"), ("ppm", "hlld")])
def test_fast_wave_second_order_1d(recon, rs):
    errs = []
    for n in (32, 64, 128):
        shape = (n, 1, 1)
        cons, b, info = inputs.fast_wave(shape, kvec=(1, 0, 0), bdir=(0, 1, 0))
        cbg, bbg, _ = inputs.fast_wave(shape, kvec=(1, 0, 0), bdir=(0, 1, 0), amp=0.0)
        cfg = cfg_for(shape, info, recon=recon, riemann=rs)
        c, bb = _one_period(cfg, cons, b, info["period"])
        errs.append(_relerr_pert(cons, b, c, bb, cbg, bbg))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert r2 > 3.3 and r2 > r1 * 0.95, errs  # -> 4 (second order)


def test_fast_wave_ppm_ep_without_the_clipping_floor():
    """Sec. 3.1.5 on the 1D fast eigenmode with HLLD, one period, N = 32 .. 256: PPM-EP converges
    cleanly at second order (the time integrator's), reaching the error of PLM at about 4x lower
    resolution, while plain PPM's convergence stalls as its limiter clips the wave's extrema."""
    errs = {}
    for recon in ("plm_mc", "ppm", "ppm_ep"):
        errs[recon] = []
        for n in (32, 64, 128, 256):
            shape = (n, 1, 1)
            cons, b, info = inputs.fast_wave(shape, kvec=(1, 0, 0), bdir=(0, 1, 0))
            cbg, bbg, _ = inputs.fast_wave(shape, kvec=(1, 0, 0), bdir=(0, 1, 0), amp=0.0)
            cfg = cfg_for(shape, info, recon=recon, riemann="hlld")
            c, bb = _one_period(cfg, cons, b, info["period"])
            errs[recon].append(_relerr_pert(cons, b, c, bb, cbg, bbg))
    ep, pl, pp = (np.array(errs[k]) for k in ("ppm_ep", "plm_mc", "ppm"))
    assert (ep[1:-1] / ep[2:] > 3.7).all(), ep          # -> 4
    assert ep[1] <= 1.5 * pl[3] and ep[0] <= 1.5 * pl[2], (ep, pl)  # PLM at 4x the cells
    assert pp[2] / pp[3] < 3.3 and (ep < pp).all(), (pp, ep)      # PPM stalls, PPM-EP does not


def test_fast_wave_second_order_3d_diagonal():
    """The oblique-diagonal eigenmode of the 32^3 workload, at 16^3 and 32^3."""
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        cons, b, info = inputs.fast_wave(shape)
        cbg, bbg, _ = inputs.fast_wave(shape, amp=0.0)
        cfg = cfg_for(shape, info, recon="plm_mc", riemann="hll")
        c, bb = _one_period(cfg, cons, b, info["period"])
        errs.append(_relerr_pert(cons, b, c, bb, cbg, bbg))
    assert errs[0] / errs[1] > 3.0, errs


def test_oblique_alfven_wave_second_order_ppm_hlld():
    """The throughput workload's oblique linear Alfven wave (k ~ (1, 2, 3), theta = pi/4),
    PPM + HLLD + Q26: after one period the exact state is the initial one; the error shrinks
    towards second order from 16^3 to 32^3 (5 and 11 cells per wavelength along x2)."""
    errs = []
    for n in (16, 32):
        shape = (n, n, n)
        cons, b, info = inputs.alfven_oblique(shape)
        cbg, bbg, _ = inputs.alfven_oblique(shape, amp=0.0)
        assert np.allclose(info["n_perp"] @ np.array([1, 2, 3]), 0) and abs(info["n_perp"][2]) == 0.0
        assert info["n_bg"] @ info["n_perp"] == pytest.approx(0.0, abs=1e-15)
        cfg = cfg_for(shape, info, recon="ppm", riemann="hlld")
        c, bb = _one_period(cfg, cons, b, 2 * np.pi / info["omega"])
        errs.append(_relerr_pert(cons, b, c, bb, cbg, bbg))
    assert errs[0] / errs[1] > 3.0, errs


def test_circular_alfven_exact_nonlinear():
    """Finite-amplitude circularly polarised Alfven wave: exact solution, second-order error."""
    errs = []
    for n in (32, 64):
        shape = (n, 1, 1)
        cons, b, info = inputs.circular_alfven(shape, amp=0.1)
        cfg = cfg_for(shape, info, recon="ppm", riemann="hlld")
        T = 2 * np.pi / info["omega"]
        c, bb = _one_period(cfg, cons, b, T)
        ex_c, ex_b, _ = inputs.circular_alfven(shape, amp=0.1, t=T)
        errs.append(np.abs(bb[1:] - ex_b[1:]).mean() / 0.1)
    assert errs[0] / errs[1] > 3.0, errs
    assert errs[1] < 2e-2


# ---------------------------------------------------------------------------------------
# Ohmic resistivity (Sec. 2.4, Sec. 4.7)
# ---------------------------------------------------------------------------------------
def _wave_energy(cons, b):
    rho = cons[0]
    uz = cons[3] / rho
    return 0.5 * (rho * uz**2).sum() + 0.5 * (b[2] ** 2).sum()


def test_resistive_alfven_decay_rate():
    """Decay rate of the linearly polarised Alfven wave: lambda = eta k^2 / 2 (Eq. alfven-decay)."""
    n = 64
    shape = (n, 1, 1)
    rates = {}
    for eta in (0.0, 1e-2, 3e-2):
        cons, b, info = inputs.alfven_wave(shape)
        cfg = cfg_for(shape, info, recon="ppm", riemann="hlld", eta=eta)
        T = 1.0
        e0 = _wave_energy(cons, b)
        c, bb = _one_period(cfg, cons, b, T)
        rates[eta] = -np.log(_wave_energy(c, bb) / e0) / (2 * T)
    k = 2 * np.pi
    for eta in (1e-2, 3e-2):
        lam = rates[eta] - rates[0.0]
        assert lam == pytest.approx(eta * k * k / 2, rel=0.03)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_joule_heating_profile(d):
    """One small step: the internal energy the resistive terms deposit is eta |j|^2 dt locally
    (Sec. 4.7), with j from both tangential field components, and not the local magnetic-energy
    loss. The field varies along axis d only: b_a = delta sin(k s), b_c = delta2 cos(k s)."""
    n = 64
    shape = [1, 1, 1]
    shape[d] = n
    shape = tuple(shape)
    a, c = (d + 1) % 3, (d + 2) % 3
    box = inputs.Box(shape)
    delta, delta2, k, eta = 1e-3, 0.7e-3, 2 * np.pi, 5e-2
    A = np.zeros((3,) + tuple(shape[::-1]))
    s_c = box.edge_coords(c)[d]
    A[c] = delta * np.cos(k * s_c) / k  # b_a = -dA_c/ds
    s_a = box.edge_coords(a)[d]
    A[a] = delta2 * np.sin(k * s_a) / k  # b_c = dA_a/ds
    b = inputs.curl_edges_to_faces(box, A)
    b[d] += 0.2
    rho = np.ones(tuple(shape[::-1]))
    cons = inputs.assemble(rho, [0 * rho] * 3, np.ones_like(rho), b)
    dt = 1e-4
    out = {}
    for e in (0.0, eta):
        cfg = oracle.Config(shape=shape, h=box.h, recon="plm_mc", riemann="hll", eta=e)
        cc, bb, _ = oracle.step(cfg, cons, b, dt)
        bc = inputs.face_to_cell(bb)
        kin = 0.5 * (cc[1] ** 2 + cc[2] ** 2 + cc[3] ** 2) / cc[0]
        out[e] = cc[4] - kin - 0.5 * (bc**2).sum(axis=0)
    deposit = ((out[eta] - out[0.0]) / dt).ravel()
    s = box.coords()[d].ravel()
    expect = eta * k * k * ((delta * np.cos(k * s)) ** 2 + (delta2 * np.sin(k * s)) ** 2)
    assert np.abs(deposit - expect).max() <= 0.02 * expect.max()
    wrong = eta * k * k * ((delta * np.sin(k * s)) ** 2 + (delta2 * np.cos(k * s)) ** 2)
    assert np.abs(deposit - wrong).max() > 0.3 * expect.max()


def test_eta_zero_is_ideal():
    shape = (6, 5, 4)
    cons, b, info = inputs.random_smooth(shape, seed=2, rough=0.05)
    cfg0 = cfg_for(shape, info, recon="ppm", riemann="hlld", eta=0.0)
    cfg1 = cfg_for(shape, info, recon="ppm", riemann="hlld", eta=1e-300)
    dt = oracle.max_dt(cfg0, cons, b, 0.3)
    c0, b0, _ = oracle.step(cfg0, cons, b, dt)
    c1, b1, _ = oracle.step(cfg1, cons, b, dt)
    assert np.array_equal(c0, c1) and np.array_equal(b0, b1)


# ---------------------------------------------------------------------------------------
# First-order flux correction (Sec. 2.5)
# ---------------------------------------------------------------------------------------
def _fo_euler(cfg, cons, b, dt):
    """Forward Euler with first-order (PC + LLF) fluxes: Eqs. (rk:increment-*) by numpy."""
    fo = oracle.Config(shape=cfg.shape, h=cfg.h, recon="pc", riemann="llf", emf=cfg.emf, eta=cfg.eta)
    F, E = oracle.fluxes(fo, cons, b)
    h = cfg.h
    c = cons.copy()
    for d in range(3):
        c += dt * (F[d] - np.roll(F[d], -1, axis=3 - d)) / h[d]
    bb = b.copy()
    for d in range(3):
        a, cc = (d + 1) % 3, (d + 2) % 3
        bb[d] += dt * ((E[cc] - np.roll(E[cc], -1, axis=2 - a)) / h[a] + (np.roll(E[a], -1, axis=2 - cc) - E[a]) / h[cc])
    return c, bb


@pytest.mark.parametrize("emf", ["q26", "fs18", "b25a"])
def test_fofc_all_flagged_is_forward_euler_first_order(emf):
    shape = (7, 6, 5)
    cons, b, info = inputs.random_smooth(shape, seed=8, rough=0.05)
    cfg = cfg_for(shape, info, recon="ppm", riemann="hlld", emf=emf, eta=1e-3, fofc_criteria=4)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    c, bb, cnt = oracle.step(cfg, cons, b, dt)
    assert cnt == (np.prod(shape), np.prod(shape))
    ce, be = _fo_euler(cfg, cons, b, dt)
    assert np.abs(c - ce).max() <= 1e-14 * np.abs(ce).max()
    assert np.abs(bb - be).max() <= 1e-14 * np.abs(be).max()


def _update(cfg, cons, b, F, E, dt):
    """S + D(F, E), Eqs. (rk:increment-state) and (rk:increment-bfield), by numpy."""
    h = cfg.h
    c = cons.copy()
    for d in range(3):
        c += dt * (F[d] - np.roll(F[d], -1, axis=3 - d)) / h[d]
    bb = b.copy()
    for d in range(3):
        a, cc = (d + 1) % 3, (d + 2) % 3
        bb[d] += dt * ((E[cc] - np.roll(E[cc], -1, axis=2 - a)) / h[a] + (np.roll(E[a], -1, axis=2 - cc) - E[a]) / h[cc])
    return c, bb


def _masks(shape, cell):
    """Faces and edges of one cell (Fig. fofc): d-faces at X and X+d, e-edges at X, X+a, X+c, X+a+c."""
    nx, ny, nz = shape
    fm = np.zeros((3, nz, ny, nx), bool)
    em = np.zeros((3, nz, ny, nx), bool)
    i, j, k = cell
    pos = np.array([i, j, k])
    for d in range(3):
        for s in (0, 1):
            p = pos.copy()
            p[d] = (p[d] + s) % shape[d]
            fm[d, p[2], p[1], p[0]] = True
        a, c = (d + 1) % 3, (d + 2) % 3
        for sa in (0, 1):
            for sc in (0, 1):
                p = pos.copy()
                p[a] = (p[a] + sa) % shape[a]
                p[c] = (p[c] + sc) % shape[c]
                em[d, p[2], p[1], p[0]] = True
    return fm, em


@pytest.mark.parametrize("stage", [0, 1])
@pytest.mark.parametrize("emf", ["q26", "fs18"])
def test_fofc_single_flagged_cell_matches_mixed_flux_update(stage, emf):
    """A cell invalidated after stage 1 (or 2) takes first-order fluxes on its 6 faces and 12
    edges; every other face and edge keeps its high-order (or RK-averaged) value (Sec. 2.5)."""
    shape = (7, 6, 5)
    cons, b, info = inputs.random_smooth(shape, seed=31, rough=0.03)
    cfg = cfg_for(shape, info, recon="ppm", riemann="hlld", emf=emf, eta=1e-3)
    fo = cfg_for(shape, info, recon="pc", riemann="llf", emf=emf, eta=1e-3)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    cell = (3, 2, 1)
    flags = np.zeros((shape[2], shape[1], shape[0]), bool)
    flags[cell[2], cell[1], cell[0]] = True
    f1, f2 = (flags, None) if stage == 0 else (None, flags)
    c, bb, cnt = oracle.step_user_flags(cfg, cons, b, dt, f1, f2)
    assert cnt == ((1, 0) if stage == 0 else (0, 1))
    fm, em = _masks(shape, cell)
    F0, E0 = oracle.fluxes(cfg, cons, b)
    Ff, Ef = oracle.fluxes(fo, cons, b)
    if stage == 0:
        F0 = np.where(fm[:, None], Ff, F0)
        E0 = np.where(em, Ef, E0)
    c1, b1 = _update(cfg, cons, b, F0, E0, dt)
    F1, E1 = oracle.fluxes(cfg, c1, b1)
    Fm, Em = 0.5 * (F0 + F1), 0.5 * (E0 + E1)
    if stage == 1:
        Fm = np.where(fm[:, None], Ff, Fm)
        Em = np.where(em, Ef, Em)
    ce, be = _update(cfg, cons, b, Fm, Em, dt)
    assert np.abs(c - ce).max() <= 1e-13 * np.abs(ce).max()
    assert np.abs(bb - be).max() <= 1e-13 * np.abs(be).max()


def _low_pressure_state(shape, seed=1):
    cons, b, info = inputs.random_smooth(shape, seed=seed, rough=0.0)
    rng = np.random.default_rng(seed)
    # a strongly compressive/expanding velocity field over a near-vacuum pressure region
    nz, ny, nx = cons.shape[1:]
    rho = cons[0]
    u = [cons[1 + d] / rho for d in range(3)]
    x = (np.arange(nx) + 0.5) / nx
    u[0] = u[0] + 3.0 * np.sin(2 * np.pi * x)[None, None, :] + 0.3 * rng.uniform(-1, 1, rho.shape)
    p = 1e-3 * np.ones_like(rho)
    return inputs.assemble(rho, u, p, b), b, info


def test_fofc_flags_conserve_and_keep_divergence():
    shape = (16, 6, 4)
    cons, b, info = _low_pressure_state(shape)
    cfg = cfg_for(shape, info, recon="ppm", riemann="hlld")
    dt = oracle.max_dt(cfg, cons, b, 0.6)
    c, bb, cnt = oracle.step(cfg, cons, b, dt)
    assert cnt[0] + cnt[1] > 0
    for v in range(5):
        assert abs(c[v].sum() - cons[v].sum()) <= 1e-13 * (np.abs(cons[v]).sum() + np.abs(cons[0]).sum())
    md, mb = oracle.divb(cfg, bb)
    assert md * min(info["h"]) / mb <= 1e-13
    # without correction the same step is different only around flagged cells
    cfg_off = cfg_for(shape, info, recon="ppm", riemann="hlld", fofc_criteria=0)
    c_off, b_off, _ = oracle.step(cfg_off, cons, b, dt)
    assert not np.array_equal(c, c_off)


def test_fofc_without_flags_is_plain_rk2():
    shape = (6, 6, 6)
    cons, b, info = inputs.random_smooth(shape, seed=12, rough=0.02)
    on = cfg_for(shape, info, recon="ppm", riemann="hlld")
    off = cfg_for(shape, info, recon="ppm", riemann="hlld", fofc_criteria=0)
    dt = oracle.max_dt(on, cons, b, 0.3)
    c1, b1, cnt = oracle.step(on, cons, b, dt)
    c2, b2, _ = oracle.step(off, cons, b, dt)
    assert cnt == (0, 0)
    assert np.array_equal(c1, c2) and np.array_equal(b1, b2)


# ---------------------------------------------------------------------------------------
# Time step (Sec. 2.4) and the dual-number derivative
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("emf", ["q26", "fs18", "b25a"])
def test_flux_jvp_matches_fluxes_and_central_difference(emf):
    """The dual-number directional derivative of the fluxes and EMFs returns the fluxes themselves
    and agrees with a central difference on a smooth state, for each EMF compute scheme (the
    reference the adjoint of each is checked against)."""
    shape = (6, 5, 4)
    cons, b, info = inputs.random_smooth(shape, seed=12, rough=0.0)
    cfg = cfg_for(shape, info, recon="ppm", riemann="hlld", eta=2e-3)
    cfg.emf = emf
    rng = np.random.default_rng(3)
    dc, db = rng.normal(size=cons.shape) * 1e-2, rng.normal(size=b.shape) * 1e-2
    F, E, dF, dE = oracle.fluxes_jvp(cfg, cons, b, dc, db)
    F0, E0 = oracle.fluxes(cfg, cons, b)
    assert np.array_equal(F, F0) and np.array_equal(E, E0)
    h = 1e-6
    Fp, Ep = oracle.fluxes(cfg, cons + h * dc, b + h * db)
    Fm, Em = oracle.fluxes(cfg, cons - h * dc, b - h * db)
    assert np.abs((Fp - Fm) / (2 * h) - dF).max() <= 1e-6 * np.abs(dF).max()
    assert np.abs((Ep - Em) / (2 * h) - dE).max() <= 1e-6 * np.abs(dE).max()


@pytest.mark.parametrize("seed,amp,p0,cfl,recon,emf", [(4, 3.0, 1e-3, 0.3, "ppm", "q26"),
                                                      (4, 3.0, 1e-3, 0.3, "ppm", "fs18"),
                                                      (4, 3.0, 1e-3, 0.3, "ppm", "b25a"),
                                                      (3, 1.0, 1e-2, 0.6, "plm_mc", "b25a")])
def test_dual_number_derivative_through_flux_correction(seed, amp, p0, cfl, recon, emf):
    """A step in which flux correction (Sec. 2.5) replaces fluxes in both stages: the dual-number
    derivative (the flagged cells held as the values give them) agrees with a central difference
    of the oracle's own step, whose perturbed runs flag as many cells in each stage. The step is
    1e-9: this near-vacuum state has limiter branch points within 1e-8..1e-5 of it, across which
    a difference quotient is no derivative (at 1e-7 up to 1% of the derivatives' scale differ;
    at 1e-9 none by more than 2e-7 of it)."""
    shape = (10, 8, 6)
    cons, b, info = shock_state(shape, seed, amp, p0)
    cfg = cfg_for(shape, info, recon=recon, riemann="hlld", emf=emf)
    dt = oracle.max_dt(cfg, cons, b, cfl)
    _, _, cnt = oracle.step(cfg, cons, b, dt)
    assert cnt[0] > 0 and cnt[1] > 0, cnt
    rng = np.random.default_rng(5)
    dcons = np.zeros_like(cons)
    dcons[1:4] = rng.normal(size=cons[1:4].shape) * cons[0]
    db = np.zeros_like(b)
    _, _, tc, tb = oracle.steps_jvp(cfg, cons, b, dcons, db, 0.0, [dt])
    eps = 1e-9
    out = []
    for s in (1, -1):
        c, bb, cs = oracle.step(cfg, cons + s * eps * dcons, b, dt)
        assert cs == cnt, (cs, cnt)
        out.append((c, bb))
    fd_c = (out[0][0] - out[1][0]) / (2 * eps)
    fd_b = (out[0][1] - out[1][1]) / (2 * eps)
    assert np.abs(tc - fd_c).max() <= 1e-5 * np.abs(fd_c).max()
    assert np.abs(tb - fd_b).max() <= 1e-5 * np.abs(fd_b).max()


def test_max_dt_closed_form():
    shape = (4, 4, 4)
    box = inputs.Box(shape)
    rho = np.ones((4, 4, 4))
    b = np.zeros((3, 4, 4, 4))
    b[0] = 1.0
    cons = inputs.assemble(rho, [0.5 * rho, 0 * rho, 0 * rho], rho / G, b)
    cfg = oracle.Config(shape=shape, h=box.h)
    h = box.h[0]
    # along x: |u| + c_f(theta=0) = 0.5 + 1; along y, z: c_f = sqrt(2)
    assert oracle.max_dt(cfg, cons, b, 0.3) == pytest.approx(0.3 * h / 1.5, rel=1e-15)
    cfg.eta = 1.0  # parabolic limit 2 eta / h dominates
    assert oracle.max_dt(cfg, cons, b, 0.3) == pytest.approx(0.3 * h / (2.0 / h), rel=1e-15)


@pytest.mark.parametrize("emf,recon", [("q26", "ppm"), ("fs18", "ppm"), ("b25a", "ppm"), ("b25a", "plm_mc")])
def test_dual_number_derivative_matches_central_difference(emf, recon):
    """Two steps' dual-number derivative (in the state and in eta) against a central difference of
    the oracle's own steps with the same dts, for each EMF compute scheme."""
    shape = (6, 5, 4)
    cons, b, info = inputs.random_smooth(shape, seed=14, rough=0.01)
    cfg = cfg_for(shape, info, recon=recon, riemann="hlld", eta=1e-2)
    cfg.emf = emf
    dts = [0.5 * oracle.max_dt(cfg, cons, b, 0.3)] * 2
    rng = np.random.default_rng(0)
    dcons = np.zeros_like(cons)
    dcons[1:4] = rng.normal(size=cons[1:4].shape)
    db = np.zeros_like(b)
    deta = 0.7
    _, _, tc, tb = oracle.steps_jvp(cfg, cons, b, dcons, db, deta, dts)
    eps = 1e-6
    out = []
    for s in (1, -1):
        cfg.eta = 1e-2 + s * eps * deta
        c, bb, _, _ = oracle.run(cfg, cons + s * eps * dcons, b, 2, dt=dts[0])
        out.append((c, bb))
    fd_c = (out[0][0] - out[1][0]) / (2 * eps)
    fd_b = (out[0][1] - out[1][1]) / (2 * eps)
    assert np.abs(tc - fd_c).max() <= 1e-6 * np.abs(fd_c).max()
    assert np.abs(tb - fd_b).max() <= 1e-6 * np.abs(fd_b).max()
