"""Writes cylinder_compression.json: the shape of Section 7's compression study on the
synthetic cylinder (workloads.cylinder), computed with the FP64 oracle only.

Section 7 (its Table 1 and rank map) reports, for the Tucker solution of the Mach-10
cylinder flow, the compression ratio C = (r1 r2 r3 + N (r1 + r2 + r3)) / N^3 averaged
over the cells at rounding accuracies eps = 1e-3, 1e-4, 1e-5, and where in the flow the
ranks grow.  The paper's mesh is not available and a full-size CPU solve is out of
reach, so this script takes a coarse stand-in: 16 x 12 cells, N = 40 on the same
velocity box, run towards its steady state with the oracle's implicit LU-SGS step at
20 x the explicit time step, then compresses every cell's tensor with the truncated
HOSVD (Section 4, the per-mode rule with eps) and records, per eps, the mean
compression ratio, the rank distribution, the mean largest rank by radial band, and the
error in T of the compressed state (a one-time rounding error, not the paper's solution
difference Delta T), and the map of each cell's largest rank (rows: theta from the
downstream axis, 0, to the stagnation line, pi; columns: wall to outer boundary).

With --staircase the same study runs on the lattice variant (cylinder_staircase, h = 0.5,
402 cells), which the Tucker format can take, into cylinder_staircase_compression.json.

With --N=64 either mesh runs at the paper's velocity grid (cylinder[_staircase]_N64_
compression.json; about 35 / 50 minutes on 8 cores).

Run: python tests/golden/make_cylinder_compression.py [--staircase] [--N=64]  (about 7 / 15
minutes on 8 cores without --N).
"""
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import tucker as tk  # noqa: E402
import workloads as W  # noqa: E402

SHAPE = dict(n_theta=16, n_r=12, N=40, dr1=0.1)
STAIRCASE = dict(h=0.5, N=40)   # the Tucker-ready lattice variant, 402 cells
STEPS, DT_FACTOR, EPS = 400, 20.0, (1e-3, 1e-4, 1e-5)


def temperature(o, f):
    """T of one cell's tensor through the oracle's own moments (Algorithm 2)."""
    _, a = o.shakhov_of(f)
    return a[4]


def main(staircase=False, N=None):
    if staircase:
        kw = dict(STAIRCASE, **({"N": N} if N else {}))
        wl = W.cylinder_staircase(**kw)
        tag = f"_N{N}" if N else ""
        out = os.path.join(HERE, f"cylinder_staircase{tag}_compression.json")
    else:
        kw = dict(SHAPE, **({"N": N} if N else {}))
        wl = W.cylinder(**kw)
        tag = f"_N{N}" if N else ""
        out = os.path.join(HERE, f"cylinder{tag}_compression.json")
    o = oracle.FullGridOracle(wl)
    dt = DT_FACTOR * o.dt()
    hist, t0 = [], time.time()
    for k in range(STEPS // 10):
        hist.append([10 * (k + 1), o.step_lusgs(10, dt)])
        print(f"step {10 * (k + 1)}: residual {hist[-1][1]:.3e} ({time.time() - t0:.0f} s)",
              flush=True)
    f = o.f()
    m = o.macro()
    N = wl.N[0]
    centre = np.array([wl.xyz[q].mean(axis=0) for q in wl.hex8])
    rad = np.hypot(centre[:, 0], centre[:, 1])
    if staircase:     # radial bands by distance from the axis
        bands = {"wall (r < 1.5)": rad < 1.5, "near wall (1.5-2.5)": (rad >= 1.5) & (rad < 2.5),
                 "middle (2.5-5)": (rad >= 2.5) & (rad < 5.0), "outer (r >= 5)": rad >= 5.0}
    else:
        j_r = wl.cell_ijk[:, 1]
        bands = {"wall (first cell)": j_r == 0, "near wall (cells 1-3)": (j_r >= 1) & (j_r <= 3),
                 "middle": (j_r >= 4) & (j_r <= 8), "outer (last 3 cells)": j_r >= kw["n_r"] - 3}
    res = {"workload": wl.name, "shape": kw,
           "velocity_box": [wl.lo[0], wl.hi[0]],
           "Kn": wl.Kn, "omega": wl.omega, "Tw": 5.0, "u_inf": wl.u0[0, 0],
           "implicit_steps": STEPS, "dt": dt, "residual_history": hist,
           "T_range": [float(m[:, 4].min()), float(m[:, 4].max())],
           "n_range": [float(m[:, 0].min()), float(m[:, 0].max())], "eps": {}}
    for eps in EPS:
        ranks, C, dT = [], [], []
        for c in range(wl.n_cell):
            t, _ = tk.hosvd(f[c], eps)
            r = tk.ranks(t)
            ranks.append(r)
            C.append(tk.compression(r, N))
            dT.append(abs(temperature(o, tk.full(t)) - m[c, 4]) / m[c, 4])
        ranks = np.array(ranks)
        rmax = ranks.max(axis=1)
        nx, ny = wl.cell_ijk[:, 0].max() + 1, wl.cell_ijk[:, 1].max() + 1
        rmap = np.zeros((nx, ny), dtype=int)    # removed lattice cells stay 0
        rmap[wl.cell_ijk[:, 0], wl.cell_ijk[:, 1]] = rmax
        res["eps"][f"{eps:g}"] = {
            "mean_compression": float(np.mean(C)),
            "rank_mean": float(ranks.mean()), "rank_max": int(ranks.max()),
            "max_rank_histogram": {int(v): int(np.sum(rmax == v)) for v in np.unique(rmax)},
            "mean_max_rank_by_band": {k: float(rmax[b].mean()) if b.any() else None
                                      for k, b in bands.items()},
            "T_rounding_error_rel_max": float(np.max(dT)),
            ("rank_map_x_by_y" if staircase else "rank_map_theta_by_radius"): rmap.tolist(),
        }
        print(eps, res["eps"][f"{eps:g}"]["mean_compression"], flush=True)
    with open(out, "w") as fp:
        json.dump(res, fp, indent=1)
    return res


if __name__ == "__main__":
    n_arg = [int(a.split("=")[1]) for a in sys.argv if a.startswith("--N=")]
    main(staircase="--staircase" in sys.argv, N=n_arg[0] if n_arg else None)
