"""Shared helpers for the tests (no method arithmetic)."""
import numpy as np

from paper_2609_10816_gb300 import inputs

# Parity bars of the CUDA path against the oracle, per stored field and step:
#   relative L1 sum|gpu - oracle| / max(sum|oracle|, N * scale) <= L1_TOL, and, element by element,
#   max|gpu - oracle| / max(mean|oracle|, scale) <= MAX_TOL, so that one wrong cell cannot hide in
#   the sum of a large box.
L1_TOL = 1e-12
MAX_TOL = 1e-11


# natural scales of each stored field family, used to floor relative-L1 denominators so that
# perturbation-sized fields (momentum of a 1e-6 wave) are not judged on roundoff alone
def field_scales(cons, b):
    rho = float(np.abs(cons[0]).mean())
    e = float(np.abs(cons[4]).mean())
    bmag = float(np.sqrt((b**2).sum(axis=0)).mean()) or 1.0
    # momentum scale: rho times a signal speed of order sqrt(e / rho)
    mom = rho * np.sqrt(max(e / max(rho, 1e-300), 1e-300))
    return [rho, mom, mom, mom, e], [bmag, bmag, bmag]


def rel_l1(got, ref, scale):
    """sum |got - ref| / max(sum |ref|, N * scale)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    den = max(float(np.abs(ref).sum()), ref.size * scale)
    return float(np.abs(got - ref).sum()) / den


def rel_max(got, ref, scale):
    """max |got - ref| / max(mean |ref|, scale): the element-wise companion of rel_l1."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    if ref.size == 0:
        return 0.0
    den = max(float(np.abs(ref).mean()), scale)
    return float(np.abs(got - ref).max()) / den


NAMES = ["rho", "m0", "m1", "m2", "e", "b0", "b1", "b2"]


def state_errors(cg, bg, co, bo, scales=None, norm=rel_l1):
    if scales is None:
        scales = field_scales(co, bo)
    sc, sb = scales
    errs = {}
    for v in range(5):
        errs[NAMES[v]] = norm(cg[v], co[v], sc[v])
    for d in range(3):
        errs[NAMES[5 + d]] = norm(bg[d], bo[d], sb[d])
    return errs


def parity_failures(cg, bg, co, bo, scales=None, l1_tol=L1_TOL, max_tol=MAX_TOL):
    """Fields that miss either bar: {name: (rel L1, rel max)}; empty when the states agree."""
    if scales is None:
        scales = field_scales(co, bo)
    l1 = state_errors(cg, bg, co, bo, scales)
    mx = state_errors(cg, bg, co, bo, scales, norm=rel_max)
    return {k: (l1[k], mx[k]) for k in l1 if not (l1[k] <= l1_tol and mx[k] <= max_tol)}


def relerr_pert(c0, b0, c1, b1, cbg, bbg):
    """Eq. (error:relative) between two states, normalised by the perturbation of the first from
    the background state (cbg, bbg): the root of the summed squares of the per-field L1 norms."""
    num = den = 0.0
    for s0, s1, sb in list(zip(c0, c1, cbg)) + list(zip(b0, b1, bbg)):
        n = s0.size
        num += (np.abs(s0 - s1).mean() * n) ** 2
        den += (np.abs(s0 - sb).mean() * n) ** 2
    return (num / den) ** 0.5


def shock_state(shape, seed, amp, p0):
    """A near-vacuum state under a strong expansion: the high-order step leaves cells invalid. The
    pressure varies smoothly: on a uniform pressure its recomputed cell values differ only by
    rounding, where the limiters' branches (and so their derivatives) follow rounding noise that
    two correct implementations need not share."""
    cons, b, info = inputs.random_smooth(shape, seed=seed, rough=0.0)
    rng = np.random.default_rng(seed)
    rho = cons[0]
    u = [cons[1 + d] / rho for d in range(3)]
    nx, ny, nz = shape
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) / nz, (np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx,
                          indexing="ij")
    u[0] = u[0] + amp * np.sin(2 * np.pi * x) + 0.1 * amp * rng.uniform(-1, 1, rho.shape)
    p = p0 * (1.0 + 0.3 * np.sin(2 * np.pi * x + 1.3) * np.cos(2 * np.pi * y - 0.4) + 0.2 * np.sin(2 * np.pi * z + 0.7))
    return inputs.assemble(rho, u, p, b), b, info
