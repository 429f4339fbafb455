"""Mean Halley iterations per index evaluation of the oracle (cold start at
every evaluation) on the cloaked render of the 512 x 512, 4 samples per
pixel grating workload, over a seeded subset of pixels.  The algorithmic
FLOP and MUFU counts per RK4 step of the render kernel's roofline are fixed
from this mean I: 4 evaluations of (45 + 30 I) FLOP and (2 + 4 I) MUFU
operations, plus 40 FLOP of state update.

    python oracle/mean_halley.py [--pixels N]
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_1012_5107_gb300 import inputs  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--pixels", type=int, default=2000)
    args = ap.parse_args()
    p = inputs.three_renders(inputs.config_main(precision=inputs.FP64))["cloak"]
    pix = inputs.pixel_subset(512, 512, args.pixels, seed=21)
    _, rec = orc.render_pixels(orc.Scene(p), pix, records=True)
    halley, evals, steps = int(rec["halley"].sum()), int(rec["evals"].sum()), int(rec["steps"].sum())
    print(f"pixels {args.pixels}  samples {rec.size}  steps {steps}  evals {evals}  halley {halley}  "
          f"mean I = {halley / evals:.4f}  evals per step = {evals / max(steps, 1):.3f}")


if __name__ == "__main__":
    main()
