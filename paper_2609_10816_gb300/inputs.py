"""Seeded synthetic initial states for the CT-MHD step (numpy, float64, host arrays).

This module only builds inputs: it holds none of the update's arithmetic, and it is the one
module that both the CUDA path's callers and the CPU oracle's tests draw states from.

Layout: ``cons`` is ``(5, nz, ny, nx)`` = (rho, rho*u0, rho*u1, rho*u2, e_tot) at cell centres;
``b`` is ``(3, nz, ny, nx)`` with ``b[d]`` the normal field on the d-face at index_d - 1/2.
Face fields always come from the discrete curl of a periodic vector potential held on cell
edges (the paper's initialisation, footnote in Sec. 3.1), so the discrete divergence is zero to
rounding at t = 0. ``e_tot`` uses the cell average of the face field, so the pressure at t = 0 is
exactly the prescribed one.
"""
from __future__ import annotations

import numpy as np

GAMMA = 5.0 / 3.0


class Box:
    """Periodic box of shape (nx, ny, nz) over [lo, lo + L) per direction."""

    def __init__(self, shape, length=(1.0, 1.0, 1.0), lo=(0.0, 0.0, 0.0)):
        self.shape = tuple(int(n) for n in shape)
        self.L = tuple(float(x) for x in length)
        self.lo = tuple(float(x) for x in lo)
        self.h = tuple(self.L[d] / self.shape[d] for d in range(3))

    def coords(self, stagger=(0.5, 0.5, 0.5)):
        """Meshgrid (x0, x1, x2) arrays of shape (nz, ny, nx); stagger 0.5 = cell centre, 0 = lower face."""
        nx, ny, nz = self.shape
        ax = [self.lo[d] + (np.arange(self.shape[d]) + stagger[d]) * self.h[d] for d in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return x, y, z

    def edge_coords(self, e):
        """Coordinates of the e-edges: half-integer (lower) in the two directions other than e."""
        st = [0.0, 0.0, 0.0]
        st[e] = 0.5
        return self.coords(tuple(st))


def curl_edges_to_faces(box: Box, A):
    """Face field b = curl A with A (3, nz, ny, nx) on edges (A[e] at the e-edge lower corner)."""
    b = np.zeros_like(A)
    for d in range(3):
        a, c = (d + 1) % 3, (d + 2) % 3
        ax_a = 2 - a  # numpy axis of direction a in (nz, ny, nx)
        ax_c = 2 - c
        b[d] = (np.roll(A[c], -1, axis=ax_a) - A[c]) / box.h[a] - (np.roll(A[a], -1, axis=ax_c) - A[a]) / box.h[c]
    return b


def face_to_cell(b):
    """Cell average of each face component (used only to set e_tot consistently)."""
    bc = np.empty_like(b)
    for d in range(3):
        bc[d] = 0.5 * (b[d] + np.roll(b[d], -1, axis=2 - d))
    return bc


def assemble(rho, u, p, b, gamma=GAMMA):
    """Conserved cell state from primitive cell values and the face field."""
    bc = face_to_cell(b)
    cons = np.empty((5,) + rho.shape)
    cons[0] = rho
    for d in range(3):
        cons[1 + d] = rho * u[d]
    cons[4] = p / (gamma - 1.0) + 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) + 0.5 * (
        bc[0] ** 2 + bc[1] ** 2 + bc[2] ** 2
    )
    return cons


def _uniform_faces(box, b0):
    nx, ny, nz = box.shape
    b = np.zeros((3, nz, ny, nx))
    for d in range(3):
        b[d] = b0[d]
    return b


# ----------------------------------------------------------------------------------------
# Linear fast magnetosonic eigenmode (Sec. 3.1.3 geometry; oblique, along k)
# ----------------------------------------------------------------------------------------
def fast_wave(shape, kvec=(1, 1, 1), bdir=(1.0, 1.0, 0.0), rho0=1.0, p0=1.0 / GAMMA, b0=1.0,
              amp=1e-6, t=0.0, gamma=GAMMA, L=1.0):
    """Fast eigenmode A cos(k.x - w t) from the linearised 1-D MHD relations along n_k.

    Returns (cons, b, info) with info = {"omega", "cf", "period", "k"}."""
    box = Box(shape, (L, L, L))
    k = 2 * np.pi * np.asarray(kvec, float) / L
    kk = np.linalg.norm(k)
    nk = k / kk
    nb = np.asarray(bdir, float) / np.linalg.norm(bdir)
    cos_t = float(nb @ nk)
    perp = nb - cos_t * nk
    if np.linalg.norm(perp) < 1e-14:
        raise ValueError("field parallel to k: no fast mode distinct from sound")
    nperp = perp / np.linalg.norm(perp)
    bn = b0 * cos_t
    bt = b0 * float(nb @ nperp)
    cs2 = gamma * p0 / rho0
    ca2 = b0 * b0 / rho0
    can2 = bn * bn / rho0
    cf2 = 0.5 * (cs2 + ca2 + np.sqrt((cs2 + ca2) ** 2 - 4 * cs2 * can2))
    cf = np.sqrt(cf2)
    omega = cf * kk
    # amplitudes per unit A
    du_n = cf
    db_t = bt * cf * du_n / (cf2 - can2)
    du_t = -bn * db_t / (rho0 * cf)
    x, y, z = box.coords()
    phase = k[0] * x + k[1] * y + k[2] * z - omega * t
    A = amp * np.cos(phase)
    rho = rho0 * (1 + A)
    u = [du_n * A * nk[d] + du_t * A * nperp[d] for d in range(3)]
    p = p0 + cs2 * rho0 * A
    # field: uniform background on faces + perturbation db_t * A along n_perp from a potential
    Avec = np.zeros((3,) + x.shape)
    coef = np.cross(nperp, k) / kk**2 * (amp * db_t)
    for e in range(3):
        ex, ey, ez = box.edge_coords(e)
        ph = k[0] * ex + k[1] * ey + k[2] * ez - omega * t
        Avec[e] = coef[e] * np.sin(ph)
    b = _uniform_faces(box, b0 * nb) + curl_edges_to_faces(box, Avec)
    cons = assemble(rho, u, p, b, gamma)
    return cons, b, {"omega": omega, "cf": cf, "period": 2 * np.pi / omega, "k": k, "h": box.h}


# ----------------------------------------------------------------------------------------
# Linearly polarised Alfven wave (Sec. 3.1.1), optionally resistive decay reference
# ----------------------------------------------------------------------------------------
def alfven_wave(shape, kvec=(1, 0, 0), bdir=(1.0, 0.0, 0.0), pol=(0.0, 0.0, 1.0), rho0=1.0,
                p0=1.0 / GAMMA, b0=1.0, amp=1e-6, gamma=GAMMA, L=1.0):
    """Alfven eigenmode: u = -c_A A n_perp, b = b_bg + b0 A n_perp, A = amp cos(k.x)."""
    box = Box(shape, (L, L, L))
    k = 2 * np.pi * np.asarray(kvec, float) / L
    kk = np.linalg.norm(k)
    nk = k / kk
    nb = np.asarray(bdir, float) / np.linalg.norm(bdir)
    npol = np.asarray(pol, float) / np.linalg.norm(pol)
    assert abs(npol @ nk) < 1e-12
    ca = b0 / np.sqrt(rho0)
    x, y, z = box.coords()
    A = amp * np.cos(k[0] * x + k[1] * y + k[2] * z)
    rho = rho0 * np.ones_like(x)
    u = [-ca * A * npol[d] for d in range(3)]
    p = p0 * np.ones_like(x)
    Avec = np.zeros((3,) + x.shape)
    coef = np.cross(npol, k) / kk**2 * (amp * b0)
    for e in range(3):
        ex, ey, ez = box.edge_coords(e)
        Avec[e] = coef[e] * np.sin(k[0] * ex + k[1] * ey + k[2] * ez)
    b = _uniform_faces(box, b0 * nb) + curl_edges_to_faces(box, Avec)
    cos_t = float(nb @ nk)
    return assemble(rho, u, p, b, gamma), b, {"omega": ca * kk * cos_t, "k": kk, "h": box.h}


def alfven_oblique(shape, kvec=(1, 2, 3), theta=np.pi / 4, amp=1e-6, gamma=GAMMA):
    """The linearly polarised Alfven wave of the paper's throughput runs (Sec. 5.2 with the setup
    of Sec. 4.1.1 and the oblique geometry of Sec. 5.1): rho = b_bg = 1, p = 1/gamma, L = 1,
    k L / 2 pi = kvec, theta = angle(b_bg, k) = pi/4. The polarisation n_perp is orthogonal to
    n_k and to the x2 axis ((-2, 1, 0)/sqrt5 for k ~ (1, 2, 3)); b_bg lies in the plane of n_k
    and the x2 axis, turned from n_k by theta towards +x2, so that n_perp is also orthogonal to
    it (an Alfven mode)."""
    k = np.asarray(kvec, float)
    nk = k / np.linalg.norm(k)
    npol = np.cross((0.0, 0.0, 1.0), nk)
    npol /= np.linalg.norm(npol)
    e = np.cross(nk, npol)  # unit, orthogonal to n_k and n_perp, positive x2 component
    if e[2] < 0:
        e = -e
    nb = np.cos(theta) * nk + np.sin(theta) * e
    cons, b, info = alfven_wave(shape, kvec=kvec, bdir=nb, pol=npol, amp=amp, gamma=gamma)
    info.update(n_bg=nb, n_perp=npol)
    return cons, b, info


def circular_alfven(shape, rho0=1.0, p0=1.0 / GAMMA, b0=1.0, amp=0.1, t=0.0, gamma=GAMMA, L=1.0):
    """Circularly polarised Alfven wave along x0 (Sec. 3.1.2): exact at any amplitude."""
    box = Box(shape, (L, L, L))
    k = 2 * np.pi / L
    ca = b0 / np.sqrt(rho0)
    omega = ca * k
    x, y, z = box.coords()
    phi = omega * t - k * x
    rho = rho0 * np.ones_like(x)
    u = [np.zeros_like(x), -ca * amp * np.sin(phi), -ca * amp * np.cos(phi)]
    p = p0 * np.ones_like(x)
    # b1 = b0 amp sin(w t - k x), b2 = b0 amp cos(w t - k x), from A on edges
    Avec = np.zeros((3,) + x.shape)
    ex, ey, ez = box.edge_coords(1)  # A1 (on x1-edges) gives b2 = dA1/dx0
    Avec[1] = b0 * amp * (-np.sin(omega * t - k * ex)) / k
    ex, ey, ez = box.edge_coords(2)  # A2 gives b1 = -dA2/dx0
    Avec[2] = b0 * amp * (-np.cos(omega * t - k * ex)) / k
    b = _uniform_faces(box, (b0, 0.0, 0.0)) + curl_edges_to_faces(box, Avec)
    return assemble(rho, u, p, b, gamma), b, {"omega": omega, "h": box.h}


# ----------------------------------------------------------------------------------------
# Random periodic states
# ----------------------------------------------------------------------------------------
def _lowk_field(rng, shape, kmax=2, scale=1.0):
    """Smooth periodic scalar field: a few random Fourier modes, unit-ish amplitude."""
    nx, ny, nz = shape
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    z = (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    f = np.zeros((nz, ny, nx))
    for _ in range(6):
        kv = rng.integers(-kmax, kmax + 1, size=3)
        if not kv.any():
            continue
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.normal() * np.cos(2 * np.pi * (kv[0] * X + kv[1] * Y + kv[2] * Z) + ph)
    m = np.abs(f).max()
    return scale * f / (m if m > 0 else 1.0)


def random_smooth(shape, seed=0, gamma=GAMMA, h=None, rough=0.0):
    """Smooth random state: rho in [0.5, 2], |u| < 1, p ~ 1, b = curl of a random potential.

    ``rough`` > 0 adds cell-to-cell noise of that relative size (exercises every limiter and
    Riemann-solver branch)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    if h is None:
        h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    box = Box(shape, (h[0] * nx, h[1] * ny, h[2] * nz))
    rho = 1.25 + 0.75 * _lowk_field(rng, shape)
    u = [0.55 * _lowk_field(rng, shape) for _ in range(3)]
    p = 1.0 + 0.5 * _lowk_field(rng, shape)
    A = np.stack([0.05 * _lowk_field(rng, shape) for _ in range(3)])
    if rough > 0:
        rho = rho * (1 + rough * rng.uniform(-1, 1, rho.shape))
        u = [ui + rough * rng.uniform(-1, 1, ui.shape) for ui in u]
        p = p * (1 + rough * rng.uniform(-1, 1, p.shape))
        A = A + rough * 0.05 * rng.uniform(-1, 1, A.shape) * min(h)
    b = _uniform_faces(box, (0.3, -0.2, 0.4)) + curl_edges_to_faces(box, A)
    return assemble(rho, u, p, b, gamma), b, {"h": box.h}


def turbulence(shape, seed=2, v_rms=5.0, b0=(0.0, 0.0, 0.5), rho0=1.0, gamma=GAMMA, kmin=1, kmax=3):
    """Decaying-turbulence start: rho = 1, uniform b0, p = rho / gamma (c_s = 1), and a seeded
    solenoidal Gaussian velocity with shell spectrum E(k) ~ k^-2 (per-mode variance ~ k^-4) on
    kmin <= |k| L / 2 pi <= kmax, scaled to v_rms."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    box = Box(shape)
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    kz = np.fft.fftfreq(nz, 1.0 / nz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    K = np.sqrt(KX**2 + KY**2 + KZ**2)
    shell = (K >= kmin) & (K <= kmax)
    amp = np.zeros_like(K)
    amp[shell] = K[shell] ** -2.0  # sqrt of per-mode variance k^-4
    uk = [amp * (rng.normal(size=K.shape) + 1j * rng.normal(size=K.shape)) for _ in range(3)]
    K2 = np.where(K > 0, K**2, 1.0)
    kdotu = KX * uk[0] + KY * uk[1] + KZ * uk[2]
    uk = [uk[0] - KX * kdotu / K2, uk[1] - KY * kdotu / K2, uk[2] - KZ * kdotu / K2]
    u = [np.real(np.fft.ifftn(c)) for c in uk]
    rms = np.sqrt(np.mean(u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    u = [ui * (v_rms / rms) for ui in u]
    rho = rho0 * np.ones((nz, ny, nx))
    p = rho / gamma
    b = _uniform_faces(box, b0)
    return assemble(rho, u, p, b, gamma), b, {"h": box.h}


def harris_sheet(shape=(512, 512, 4), seed=3, width=0.05, p_inf=0.1, noise=1e-3, gamma=GAMMA):
    """Periodic double Harris sheet in pressure balance (beta = 0.2 far field) with seeded
    velocity noise; domain [-1/2, 1/2)^2 in (x0, x1) and nz cells of the same width in x2."""
    nx, ny, nz = shape
    hx = 1.0 / nx
    box = Box(shape, (1.0, 1.0, nz * hx), lo=(-0.5, -0.5, 0.0))

    def lncosh(s):
        s = np.abs(s)
        return s + np.log1p(np.exp(-2 * s)) - np.log(2.0)

    def F(y):
        return width * (lncosh((y + 0.25) / width) - lncosh((y - 0.25) / width))

    m = F(0.5) - F(-0.5)  # makes A_z periodic, so b0 = dA_z/dx1 = F' - m
    A = np.zeros((3, nz, ny, nx))
    ex, ey, ez = box.edge_coords(2)
    A[2] = F(ey) - m * ey
    b = curl_edges_to_faces(box, A)
    bc0 = face_to_cell(b)[0]
    p = p_inf + 0.5 * (1.0 - bc0**2)
    rng = np.random.default_rng(seed)
    rho = np.ones((nz, ny, nx))
    u = [noise * rng.normal(size=rho.shape) for _ in range(3)]
    return assemble(rho, u, p, b, gamma), b, {"h": box.h}


def patch_dims(npatch=1024, seed=4, edges=(16, 24, 32, 48, 64)):
    """Per-patch interior sizes (nx, ny, nz), each edge drawn uniformly from ``edges``."""
    rng = np.random.default_rng(seed)
    return rng.choice(np.asarray(edges), size=(npatch, 3))


def random_patch(shape, rng, gamma=GAMMA, h=None):
    """Smooth random patch state: rho = 1.25 + 0.75 s (s in [-1, 1]), |u| < 1 from low-k modes,
    p = 1, b = curl of a random low-k periodic potential; cell width h (default 1/n per axis)."""
    nx, ny, nz = shape
    box = Box(shape) if h is None else Box(shape, (h * nx, h * ny, h * nz))
    rho = 1.25 + 0.75 * _lowk_field(rng, shape)
    u = [0.55 * _lowk_field(rng, shape) for _ in range(3)]
    p = np.ones((nz, ny, nx))
    A = np.stack([0.1 * _lowk_field(rng, shape) for _ in range(3)])
    b = curl_edges_to_faces(box, A)
    return assemble(rho, u, p, b, gamma), b, {"h": box.h}
