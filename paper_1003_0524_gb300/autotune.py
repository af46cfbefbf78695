"""Tile-shape autotuner of the exchange-matrix library.

The tensor-core kernels take two tile parameters that the library otherwise
picks by a closed formula: the band block of the Z^H Y tiles (tile_nb_zhy, a
multiple of 8 up to 64) and the band block of the interstitial tiles
(tile_nb_zipw, a multiple of 8 up to 64).  Their best values depend on the
band window, the occupied count and the aux size, not on the number of k
points: every (k, q) pair of a size class runs the same tile shapes.  The
tuner therefore times the candidates on a part of the workload that still
fills the GPU with tiles: the whole step when it takes well under a second,
else V^x of one k (its N_k pairs: 64 or 216 on the large workloads), reading
each kernel's device time from the build statistics of a graph-replayed
build.  (A reduced k mesh does not do: with a few pairs the kernels run a
fraction of a wave, and small band blocks win there that lose at full size.)
It stores the fastest per size class in a JSON file beside this module:

    python -m paper_1003_0524_gb300.autotune 1 2 3 4 4inv  # configs to tune

Context(..., tuning=True) looks up the nearest stored size class there; a
missing class leaves the library's formula in charge.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_FILE = os.path.join(HERE, "tuning.json")
NB_ZHY = (8, 16, 24, 32, 40, 48, 56, 64)
NB_ZIPW = (8, 16, 24, 32, 40, 48, 56, 64)


def size_class(sysm) -> dict:
    """What the tile choice depends on: band windows, occupied bands, aux and
    plane-wave sizes, the MT basis, and the real (inversion-symmetric) path."""
    return {"nb": int(max(sysm.n_bands)), "no": int(max(sysm.n_occ)),
            "naux": int(max(sysm.n_aux(q) for q in range(sysm.n_k))),
            "npw": int(max(g.shape[0] for g in sysm.Gk)), "n_mt": int(sysm.n_mt), "P": int(sysm.P),
            "inv": bool(getattr(sysm, "inversion", False))}


def lookup(sysm, path: str = TUNING_FILE):
    """The stored tiles of the nearest size class: the same MT basis, a band
    window within 8 bands and an aux size within 15 %; None if there is none.
    (The tuner's reduced mesh draws its own band windows and aux lists, so its
    maxima can differ a little from those of the full mesh.)"""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    key = size_class(sysm)
    best, dist = None, None
    for e in data.get("entries", []):
        k = e.get("key", {})
        if k.get("n_mt") != key["n_mt"] or k.get("P") != key["P"]:
            continue
        db, da = abs(k["nb"] - key["nb"]), abs(k["naux"] - key["naux"]) / key["naux"]
        if db > 8 or da > 0.15:
            continue
        # the real path (inversion symmetry) prefers its own entry, else takes
        # the complex one of the same band windows and aux size
        d = db + 50.0 * da + abs(k["no"] - key["no"]) + (100.0 if bool(k.get("inv", False)) != key["inv"] else 0.0)
        if dist is None or d < dist:
            best, dist = e, d
    return best


def _time(sysm, reps: int, one_k: bool, **tiles) -> dict:
    from . import hfx
    with hfx.Context(sysm, precision="sliced", **tiles) as c:
        c.load_system()
        run = (lambda: c.build_exchange(0, stats=True)[1]) if one_k else c.build_all
        for _ in range(2):          # direct run, then the graph capture
            run()
        sts = [run() for _ in range(reps)]
    return {k: min(st[k] for st in sts) for k in ("ms_zhy", "ms_zipw", "ms_total")}


def tune(cfg, reps: int = 3) -> dict:
    """Time every candidate of both tile parameters on config cfg (an index, or
    "<index>inv" for its inversion-symmetric variant); return the entry (not yet
    stored)."""
    from . import synthetic as S
    inv = str(cfg).endswith("inv")
    cfg = int(str(cfg)[:-3]) if inv else int(cfg)
    s = S.make_system(cfg, inversion=inv)
    one_k = cfg >= 3
    res_zhy = {nb: _time(s, reps, one_k, tile_nb_zhy=nb)["ms_zhy"] for nb in NB_ZHY}
    best_zhy = min(res_zhy, key=res_zhy.get)
    res_zipw = {nb: _time(s, reps, one_k, tile_nb_zhy=best_zhy, tile_nb_zipw=nb)["ms_zipw"] for nb in NB_ZIPW}
    best_zipw = min(res_zipw, key=res_zipw.get)
    import torch
    return {"key": size_class(s), "config": cfg, "timed": "V^x of k = 0" if one_k else "whole step",
            "tile_nb_zhy": best_zhy, "tile_nb_zipw": best_zipw,
            "ms_zhy": {str(k): v for k, v in res_zhy.items()}, "ms_zipw": {str(k): v for k, v in res_zipw.items()},
            "device": torch.cuda.get_device_name(), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}


def store(entries, path: str = TUNING_FILE) -> None:
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {"entries": []}
    keep = [e for e in data.get("entries", []) if all(e.get("key") != n["key"] for n in entries)]
    data["entries"] = keep + list(entries)
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


def main(argv) -> None:
    import argparse
    ap = argparse.ArgumentParser(description="time the tile candidates and store the fastest per size class")
    ap.add_argument("configs", nargs="*", default=["1", "2", "3", "4"],
                    help="config indices, or <index>inv for the inversion-symmetric variant")
    ap.add_argument("--out", default=TUNING_FILE, help="JSON file to update (default: beside this module)")
    args = ap.parse_args(argv)
    from . import build as B
    from . import hfx
    B.build()
    hfx.load()
    out = []
    for c in args.configs:
        e = tune(c)
        print(json.dumps(e), flush=True)
        out.append(e)
    store(out, args.out)


if __name__ == "__main__":
    main(sys.argv[1:])
