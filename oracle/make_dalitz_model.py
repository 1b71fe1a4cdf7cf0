"""Writes the seeded Dalitz workload model to tests/golden/dalitz_model_<seed>.json.

Calls only the oracle and the seeded generators.  The draw (masses, widths, spins,
magnitudes rho and phases phi) comes from ``synth.dalitz_model_draw``; each coefficient
is then scaled so every resonance carries a comparable share of the rate:

    c_r = rho_r e^{i phi_r} / sqrt(G_rr / G_NR),   G_rr = dA sum_cells |A_r|^2,

with G_NR the grid area (the integral of |a_NR|^2 = 1).  The accept-reject envelope is
1.1 x the maximum of |A|^2 over the 512 x 512 cell centres and 10^5 uniform points
inside the region.

Usage:  python oracle/make_dalitz_model.py [seed]
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1311_1753_gb300 import synth  # noqa: E402


def main(seed: int = synth.SEED_DALITZ_MODEL):
    draw = synth.dalitz_model_draw(seed)
    kin = dict(M=synth.D0_MASS, m1=synth.PIC_MASS, m2=synth.PIC_MASS, m3=synth.PI0_MASS, R=1.5)
    d = oracle.Dalitz(kin["M"], kin["m1"], kin["m2"], kin["m3"], kin["R"])
    idx = []
    for r in draw:
        i = [d.param(r["m0"]), d.param(r["g0"]), d.param(0.0), d.param(0.0)]
        d.resonance(r["channel"], r["spin"], *i)
        idx.append(i)
    p = d.p
    area, ncells = d.norm(p, anr=0.0 + 0j)[1], None
    N_nr, ncells = d.norm(p, anr=1.0 + 0j)
    res = []
    for r, (dr, i) in enumerate(zip(draw, idx)):
        q = p.copy()
        q[i[2]] = 1.0
        G_rr, _ = d.norm(q, anr=0.0 + 0j)
        scale = dr["rho"] / math.sqrt(G_rr / N_nr)
        c = scale * complex(math.cos(dr["phi"]), math.sin(dr["phi"]))
        res.append(dict(channel=dr["channel"], spin=dr["spin"], m0=dr["m0"], g0=dr["g0"],
                        re=c.real, im=c.imag, G_rr=G_rr))
    for r, i in zip(res, idx):
        d.values[i[2]] = r["re"]
        d.values[i[3]] = r["im"]
    # envelope: max over cell centres and 1e5 random inside points
    x0, x1, y0, y1 = d.box()
    hx, hy = (x1 - x0) / d.nbx, (y1 - y0) / d.nby
    gx, gy = np.meshgrid(x0 + (np.arange(d.nbx) + 0.5) * hx, y0 + (np.arange(d.nby) + 0.5) * hy,
                         indexing="ij")
    gx, gy = gx.ravel(), gy.ravel()
    ins = d.inside(gx, gy)
    pmax = d.intensity(gx[ins], gy[ins]).max()
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    rx, ry = rng.uniform(x0, x1, 400000), rng.uniform(y0, y1, 400000)
    ins = d.inside(rx, ry)
    rx, ry = rx[ins][:100000], ry[ins][:100000]
    pmax = max(pmax, d.intensity(rx, ry).max())
    N, cnt = d.norm()
    spec = dict(seed=seed, kin=kin, nbx=d.nbx, nby=d.nby, a_nr=[1.0, 0.0], resonances=res,
                envelope=1.1 * float(pmax), norm=N, ncells=cnt, grid_area=N_nr,
                note="written by oracle/make_dalitz_model.py; parameters are the workload's truth")
    out = os.path.join(ROOT, "tests", "golden", f"dalitz_model_{seed}.json")
    with open(out, "w") as fh:
        json.dump(spec, fh, indent=1)
    print("wrote", out, "ncells", cnt, "area", N_nr, "N", N, "envelope", spec["envelope"])


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else synth.SEED_DALITZ_MODEL)
