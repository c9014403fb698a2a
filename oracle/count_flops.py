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

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_2609_10816_gb300 import inputs  # noqa: E402


def count(name, cons, b, h, **scheme):
    nx = cons.shape[3]
    ny = cons.shape[2]
    nz = cons.shape[1]
    cfg = oracle.Config(shape=(nx, ny, nz), h=h, **scheme)
    dt = oracle.max_dt(cfg, cons, b, 0.3)
    ops, flagged = oracle.count_ops(cfg, cons, b, dt)
    N = nx * ny * nz
    out = {
        "workload_sample": name,
        "cells": N,
        "flagged": flagged,
        "flops_per_cell_update": sum(ops.values()) / N,
        # two stages per step; 3 faces and 3 edges per cell per stage
        "face_kernel_flops_per_face": (ops["recon"] + ops["riemann"] + ops["joule"]) / (6 * N),
        "edge_flops_per_edge": ops["edge"] / (6 * N),
        "prim_flops_per_cell": ops["prim"] / (2 * N),
        "update_flops_per_cell": ops["update"] / (2 * N),
        "by_phase_per_cell_update": {k: v / N for k, v in ops.items()},
    }
    return out


def main():
    res = []
    cons, b, info = inputs.turbulence((32, 32, 32), seed=2, v_rms=5.0)
    res.append(count("turbulence Mach 5, 32^3 sample, PPM+HLLD+Q26+LD04", cons, b, info["h"],
                     recon="ppm", riemann="hlld", emf="q26"))
    cons, b, info = inputs.fast_wave((32, 32, 32))
    res.append(count("fast eigenmode 32^3, PLM-MC+HLL+Q26+LD04", cons, b, info["h"],
                     recon="plm_mc", riemann="hll", emf="q26"))
    cons, b, info = inputs.harris_sheet((64, 64, 4))
    res.append(count("Harris sheet 64x64x4 sample, PLM-MC+HLLD+Q26+LD04, eta 1e-4", cons, b, info["h"],
                     recon="plm_mc", riemann="hlld", emf="q26", eta=1e-4))
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
