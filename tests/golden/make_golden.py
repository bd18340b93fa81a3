"""Writes ``c1_rays.txt``: oracle line integrals (Algorithm 1, FP64) and the
closed-form ellipsoid integrals (8 x 8 sub-pixel mean) for 64 seeded rays
of the 64^3 / 32-view cone-beam workload on the Shepp-Logan-shaped
phantom (2 x 2 x 2 supersampled).

It calls only ``oracle`` and the seeded input generators in ``synth``.  The
file is a regression fixture: any change to the oracle's arithmetic that
moves these values must be justified by the paper passage it follows.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_rays.txt")


def select_rays(seed=2024, n=64):
    rng = np.random.default_rng(seed)
    views = rng.integers(0, 32, size=n)
    ius = rng.integers(0, 64, size=n)
    ivs = rng.integers(0, 64, size=n)
    return views, ius, ivs


def main():
    vg, g = synth.c1_geometry()
    ell = synth.ellipsoids_world(vg)
    vol = synth.voxelize(vg, ell, supersample=2)
    views, ius, ivs = select_rays()
    vals = oracle.rays(vol, vg, g, views, ius, ivs)
    sub = g.subset(views)
    # analytic integral of the same pixels: project the selected views and pick
    ana_all = oracle.ellipsoid_project(ell, sub, sub=8)
    ana = ana_all[np.arange(len(views)), ivs, ius]
    with open(OUT, "w") as f:
        f.write("# GJP forward (Algorithm 1, FP64 oracle) and analytic ellipsoid line integrals\n")
        f.write("# workload: 64^3 Shepp-Logan-shaped phantom (2x2x2 supersampled), h = 1,\n")
        f.write("# D_so = 256, D_sd = 512, 64x64 detector, 32 views over 360 degrees\n")
        f.write("# written by tests/golden/make_golden.py (oracle + synth only)\n")
        f.write("# view iu iv gjp analytic\n")
        for v, u, w, a, b in zip(views, ius, ivs, vals, ana):
            f.write(f"{int(v)} {int(u)} {int(w)} {a:.17g} {b:.17g}\n")


if __name__ == "__main__":
    main()
