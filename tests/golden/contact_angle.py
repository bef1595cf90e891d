"""Contact angles of the oracle's wetting reading (solid neighbours enter the
colour-gradient field with wall_rho): a 2D drop (96 x 1 x 48, R 14, A 1e-3,
tau 0.7) on the solid bottom layer, relaxed for 16 000 steps from three
starting caps, the angle taken from a least-squares circle through the
interface cells (rows z >= 3) against the wall plane z = 0.5.

Writes contact_angle.json beside this file. Runs the oracle only (about two
minutes on one core): python tests/golden/contact_angle.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O                       # noqa: E402
from paper_0912_4230_gb300 import workloads as W     # noqa: E402


def circle_angle(p, o):
    t, _ = o.free_surface_state()
    z, x = np.nonzero(t.reshape(p.nz, p.nx) == W.INTERFACE)
    keep = z >= 3
    x, z = x[keep].astype(float), z[keep].astype(float)
    D, E, F = np.linalg.lstsq(np.stack([x, z, np.ones_like(x)], axis=1), -(x * x + z * z),
                              rcond=None)[0]
    xc, zc = -D / 2, -E / 2
    R = np.sqrt(xc * xc + zc * zc - F)
    return float(np.degrees(np.arccos(np.clip(-(zc - 0.5) / R, -1.0, 1.0))))


def run(wall_rho, gap, steps=16000):
    p = W.drop(nx=96, ny=1, nz=48, R=14.0, gap=gap, u_drop=0.0, perturb=0.0, wall_rho=wall_rho,
               steps=steps)
    o = O.Oracle(p)
    o.step(steps)
    return circle_angle(p, o)


def main():
    starts = {"from_150deg": -2.0, "from_90deg": -7.0, "from_60deg": -12.0}
    out = {"wall_rho": [0.0, 0.3, 0.6, 1.0], "angles_deg": {}}
    for name, gap in starts.items():
        out["angles_deg"][name] = [round(run(w, gap), 1) for w in out["wall_rho"]]
    json.dump(out, open(os.path.join(HERE, "contact_angle.json"), "w"), indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
