"""Write the stored oracle values of the full-size parity tests.

For the two largest workloads (configs 3 and 4 at their full sizes, and the
inversion-symmetric variant of config 4, Sec. III.D) the FP64 oracle cannot
build V^x for a whole k in test time.  It computes exactly the
sub-block V^x(k)[S][S] for a few bands S of one sampled k (every q and every
occupied band of k - q in the sums, the q->0 term included), with the same
summation order as its full V^x.  This script calls only the oracle and the
seeded input generator and writes one text file per workload:

    python tests/golden/make_fullsize_samples.py          # all
    python tests/golden/make_fullsize_samples.py 4 4inv   # some

Each file records the seed, the k point, the bands and the values.
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# workload key: (config, inversion variant, k point, bands): first and last
# occupied band, first empty band, last band
SAMPLES = {"3": (3, False, 100, [0, 19, 20, 119]), "4": (4, False, 37, [0, 47, 48, 249]),
           "4inv": (4, True, 37, [0, 47, 48, 249])}


def path_for(key) -> str:
    return os.path.join(HERE, f"vx_fullsize_cfg{key}.txt")


def write(key) -> None:
    from oracle import oracle as O
    from paper_1003_0524_gb300 import synthetic as S
    t0 = time.time()
    cfg, inv, ik, bands = SAMPLES[str(key)]
    s = S.make_system(cfg, inversion=inv)
    o = O.Oracle(s)
    V = o.vx_sub(ik, bands)
    with open(path_for(key), "w") as f:
        f.write(f"# V^x(k)[S][S] of the FP64 oracle (with the q->0 term), workload {key}: {s.name}\n")
        f.write(f"# written by tests/golden/make_fullsize_samples.py ({time.time() - t0:.0f} s, "
                f"{O.num_threads()} threads)\n")
        f.write(f"seed {s.seed}\nk {ik}\nbands {' '.join(str(b) for b in bands)}\n")
        for i in range(len(bands)):
            for j in range(len(bands)):
                f.write(f"{i} {j} {V[i, j].real:.17e} {V[i, j].imag:.17e}\n")


def read(key):
    """(seed, k, bands, V) from a stored file."""
    import numpy as np
    seed = ik = None
    bands = []
    vals = {}
    with open(path_for(key)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == "seed":
                seed = int(tok[1])
            elif tok[0] == "k":
                ik = int(tok[1])
            elif tok[0] == "bands":
                bands = [int(x) for x in tok[1:]]
            else:
                vals[(int(tok[0]), int(tok[1]))] = float(tok[2]) + 1j * float(tok[3])
    V = np.zeros((len(bands), len(bands)), np.complex128)
    for (i, j), v in vals.items():
        V[i, j] = v
    return seed, ik, bands, V


if __name__ == "__main__":
    cfgs = sys.argv[1:] or sorted(SAMPLES)
    for c in cfgs:
        write(c)
        print(f"wrote {path_for(c)}")
