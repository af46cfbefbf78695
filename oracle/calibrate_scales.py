"""Magnitude calibration of the synthetic workloads (test infrastructure).

Prints, for one configuration of paper_1003_0524_gb300.synthetic, the two
magnitude constants of its CONFIGS entry, computed with the FP64 oracle only:

  a_scale  multiplies the LAPW muffin-tin coefficients A so that the largest
           |Z^MT| and |Z^IPW| of a pair are of the same order;
  scale    multiplies every Coulomb matrix so that the largest |V^x_nn| of the
           workload is of order 1 Ha.

The oracle cost grows with the mesh and the band windows, so the run uses a
1x1x2 mesh and a reduced band window (V^x_nn grows about linearly with the
number of occupied bands; the printed scale is corrected for that).  The
values only set magnitudes; no result is compared against them.

    python oracle/calibrate_scales.py 3
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1003_0524_gb300 import synthetic as S  # noqa: E402


def main(cfg: int, nb: int = 8, no: int = 4) -> None:
    spec = S.CONFIGS[cfg]
    no_full = spec["no"] if isinstance(spec["no"], int) else spec["no"][2]
    s = S.make_system(cfg, mesh=(1, 1, 2), nb=nb, no=no, scale=1.0)
    o = O.Oracle(s)
    zm = max(np.abs(o.zmt(ik, iq)).max() for ik in range(s.n_k) for iq in range(s.n_k))
    zi = max(np.abs(o.zipw(ik, iq)).max() for ik in range(s.n_k) for iq in range(s.n_k))
    a_now = float(spec.get("a_scale", 1.0))
    vmax = max(np.abs(np.diag(o.vx(ik, q0term=False))).max() for ik in range(s.n_k))
    print(f"config {cfg}: max|Z^MT| = {zm:.3e} (a_scale {a_now}), max|Z^IPW| = {zi:.3e}")
    # Z^MT is bilinear in the coefficients A
    print(f"  a_scale giving max|Z^MT| = max|Z^IPW|: {a_now * (zi / zm) ** 0.5:.3g}")
    print(f"  max|V^x_nn| at scale 1 with {no} occupied: {vmax:.3e}")
    print(f"  scale for max|V^x_nn| ~ 1 Ha with {no_full} occupied: {no / (no_full * vmax):.3g}")


if __name__ == "__main__":
    main(int(sys.argv[1]), *(int(x) for x in sys.argv[2:]))
