"""Shared helpers for the tests (no method arithmetic)."""
import numpy as np

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


def state_errors(cg, bg, co, bo, scales=None):
    if scales is None:
        scales = field_scales(co, bo)
    sc, sb = scales
    errs = {}
    names = ["rho", "m0", "m1", "m2", "e"]
    for v in range(5):
        errs[names[v]] = rel_l1(cg[v], co[v], sc[v])
    for d in range(3):
        errs[f"b{d}"] = rel_l1(bg[d], bo[d], sb[d])
    return errs
