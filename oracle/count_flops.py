"""Algorithmic FP64 work per unit of the method, counted by the oracle (test infrastructure).

Runs one step of the oracle on a small sample of each benchmark workload with an op-counting
scalar (every +, -, *, / and sqrt counts one flop; comparisons do not) and prints the flops
per cell-update and per face / edge / cell of each phase. These figures are the roofline's
algorithmic numerators; they are data-dependent through the limiter and Riemann branches, so
they are taken on a sample drawn from the same recipe as the timed workload.

    python -m oracle.count_flops
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2609_10816_gb300 import inputs  # noqa: E402


def _ops(cons, b, h, **scheme):
    nx, ny, nz = cons.shape[3], cons.shape[2], cons.shape[1]
    cfg = oracle.Config(shape=(nx, ny, nz), h=h, **scheme)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    ops, flagged, unused = oracle.count_ops(cfg, cons, b, dt, with_unused=True)
    return ops, flagged, unused, nx * ny * nz


def summarise(name, ops, flagged, unused, N):
    face = ops["recon"] + ops["riemann"] + ops["joule"]
    return {
        "workload_sample": name,
        "cells": N,
        "flagged": flagged,
        "flops_per_cell_update": sum(ops.values()) / N,
        "flops_per_cell_update_one_sided_hlld": (sum(ops.values()) - unused) / N,
        # two stages per step; 3 faces and 3 edges per cell per stage
        "face_kernel_flops_per_face": face / (6 * N),
        "face_kernel_flops_per_face_one_sided_hlld": (face - unused) / (6 * N),
        "edge_flops_per_edge": ops["edge"] / (6 * N),
        "prim_flops_per_cell": ops["prim"] / (2 * N),
        "update_flops_per_cell": ops["update"] / (2 * N),
        "by_phase_per_cell_update": {k: v / N for k, v in ops.items()},
    }


def count(name, cons, b, h, **scheme):
    return summarise(name, *_ops(cons, b, h, **scheme))


def count_cuts(name, cons, b, h, edge, centres, **scheme):
    """Counts summed over periodic sub-boxes of `edge`^3 cells cut from a larger state around
    `centres` (each cut is treated as its own periodic box, so its wrap seams add a few faces
    with jumps)."""
    tot, fl, un, N = None, [0, 0], 0, 0
    nz, ny, nx = cons.shape[1:]
    for c in centres:
        idx = [(c[d] - edge // 2 + np.arange(edge)) % (nx, ny, nz)[d] for d in range(3)]
        cc = np.ascontiguousarray(cons[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]])
        bb = np.ascontiguousarray(b[:, idx[2]][:, :, idx[1]][:, :, :, idx[0]])
        ops, f, u, n = _ops(cc, bb, h, **scheme)
        tot = ops if tot is None else {k: tot[k] + ops[k] for k in ops}
        fl = [fl[0] + f[0], fl[1] + f[1]]
        un += u
        N += n
    return summarise(name, tot, tuple(fl), un, N)


def main():
    res = []
    cons, b, info = inputs.turbulence((256, 256, 256), seed=2, v_rms=5.0)
    rng = np.random.default_rng(7)
    centres = [tuple(int(x) for x in rng.integers(0, 256, 3)) for _ in range(4)]
    res.append(count_cuts("turbulence Mach 5: four 48^3 cuts of the timed 256^3 state, PPM+HLLD+Q26+LD04",
                          cons, b, info["h"], 48, centres, recon="ppm", riemann="hlld", emf="q26"))
    res.append(count_cuts("turbulence Mach 5: four 48^3 cuts of the timed 256^3 state, PPM-EP+HLLD+Q26+LD04",
                          cons, b, info["h"], 48, centres, recon="ppm_ep", riemann="hlld", emf="q26"))
    del cons, b
    cons, b, info = inputs.turbulence((32, 32, 32), seed=2, v_rms=5.0)
    res.append(count("turbulence Mach 5, the recipe at 32^3, PPM+HLLD+Q26+LD04", cons, b, info["h"],
                     recon="ppm", riemann="hlld", emf="q26"))
    cons, b, info = inputs.alfven_oblique((32, 32, 32))
    res.append(count("oblique Alfven wave 32^3, PPM-EP+HLLD+Q26+LD04", cons, b, info["h"],
                     recon="ppm_ep", riemann="hlld", emf="q26"))
    cons, b, info = inputs.fast_wave((32, 32, 32))
    res.append(count("fast eigenmode 32^3, PLM-MC+HLL+Q26+LD04", cons, b, info["h"],
                     recon="plm_mc", riemann="hll", emf="q26"))
    cons, b, info = inputs.harris_sheet((64, 64, 4))
    res.append(count("Harris sheet 64x64x4 sample, PLM-MC+HLLD+Q26+LD04, eta 1e-4", cons, b, info["h"],
                     recon="plm_mc", riemann="hlld", emf="q26", eta=1e-4))
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
