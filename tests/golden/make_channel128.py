"""Write tests/golden/channel128_oracle.json: the FP64 oracle's run of the 128x32x32 two-component
bottleneck channel (sigma 4/6 at equal mole fraction, total packing 0.25, slit of width 16 and length 64,
tau 1/1, body force 1e-6 along x, uniform start) over STEPS DD-TR steps with the flux plane x = 64.

It records, for the precision-form comparison of the library (FP64, FP32 and the shifted 16-bit
storage forms against the FP64 oracle):
  - the time-averaged plane flux of each species over the steps;
  - the mass of each species;
  - n and J of each species at sampled fluid nodes (fixed nodes in the bulk, at the walls, in the
    corners, at the slit's entrance, exit and edges, plus seeded random fluid nodes).

Only the oracle computes anything here (its OpenMP build, which gives the same bits as the
single-threaded one).  Run:  python tests/golden/make_channel128.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1202_3842_gb300 import inputs  # noqa: E402

STEPS = 1000
PLANE = 64
OUT = os.path.join(HERE, "channel128_oracle.json")
FIXED = [(64, 16, 16), (10, 16, 16), (64, 1, 16), (64, 16, 1), (64, 30, 30), (10, 1, 1), (10, 30, 1),
         (64, 8, 16), (64, 23, 16), (32, 12, 16), (31, 12, 16), (95, 20, 20), (96, 20, 20), (40, 8, 1),
         (80, 23, 30), (0, 16, 16), (127, 16, 16), (20, 5, 27)]


def sample_nodes(solid, shape):
    nx, ny, nz = shape
    idx = [x + nx * (y + ny * z) for (x, y, z) in FIXED]
    u = inputs.uniform01(64, 4242)
    for v in u:
        idx.append(int(v * nx * ny * nz))
    return [i for i in dict.fromkeys(idx) if not solid[i]]


def main():
    w = inputs.WORKLOADS["channel128"]()
    a = inputs.build_workload(w)
    M = len(w["sigma"])
    sim = oracle.Sim(w["shape"], w["periodic"], M, openmp=True)
    sim.set_geometry(a["solid"])
    for k in range(M):
        sim.set_species(k, w["sigma"][k], w["tau"][k])
        sim.set_potential(k, a["V"][k])
        sim.set_body_force(k, w["body"][k])
    for k in range(M):
        sim.init_density(k, a["n"][k])
    sim.set_flux_plane(0, PLANE)
    sim.step(STEPS)
    o = sim.observe()
    fs, cnt = sim.flux()
    nodes = sample_nodes(a["solid"], w["shape"])
    out = {
        "_about": __doc__.strip().splitlines()[0] + " Written by tests/golden/make_channel128.py (oracle only).",
        "workload": "channel128", "steps": STEPS, "flux_plane_x": PLANE,
        "flux_time_avg": [float(fs[k] / cnt) for k in range(M)],
        "mass": [float(o["n"][k].sum()) for k in range(M)],
        "max_n": [float(o["n"][k].max()) for k in range(M)],
        "nodes": nodes,
        "n": [[float(o["n"][k][i]) for i in nodes] for k in range(M)],
        "J": [[[float(o["J"][k][c][i]) for i in nodes] for c in range(3)] for k in range(M)],
    }
    sim.close()
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(OUT)


if __name__ == "__main__":
    main()
