"""Benchmark: V^x build seconds per SCF step on one GB300.

Default workload (the largest configuration): a 10-atom corundum-like
rhombohedral cell (5.3 A axes, alpha 55.3 deg), 4x4x4 Gamma-centred k mesh
(64 k, 4096 (k,q) pairs), 250 bands, 48 occupied, MT product basis L <= 5 with
2 radial functions (720), 2300 interstitial plane waves per q (N_aux = 3020),
block-sparse transformed Coulomb matrix.  --config selects another workload.
One step = V^x(k) for every k of the mesh plus E_x, from device-resident wave
functions and transformed v(q) (the transform runs once per SCF cycle, in
warm-up).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (the comparison arm; it never touches the GPU).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "V^x build s/SCF step and TFLOP/s vs plain FP64 GPU, at max|ΔV^x|≤1e-8 Ha"
UNIT = "s/SCF step"
WORKLOADS = {
    0: "cubic 1-atom cell a=8 bohr, 2x2x2 k (64 k,q pairs), 8 bands, 4 occupied, N_aux~197, dense v(q)",
    1: "zincblende 2-atom cell a=10.3 bohr, 4x4x4 k (4096 k,q pairs), 40 bands, 8 occupied, N_aux~635, sparse v(q)",
    2: "zincblende 2-atom cell a=10.3 bohr, 4x4x4 k (4096 k,q pairs), 32-48 bands, 6-10 occupied per k, "
       "N_aux 670-830 per q, sparse v(q)",
    3: "ABO3 5-atom cubic cell a=7.4 bohr, 6x6x6 k (46656 k,q pairs), 120 bands, 20 occupied, N_aux=1475, sparse v(q)",
    4: "corundum-like 10-atom rhombohedral cell (5.3 A, 55.3 deg), 4x4x4 k (4096 k,q pairs), 250 bands, "
       "48 occupied, N_aux=3020, sparse v(q)",
}
# FFT grid (n^3 points) of the interstitial products in the algorithmic flop
# count of the paper's method, per workload
FFT_N = {0: 16, 1: 24, 2: 24, 3: 24, 4: 27}
DEFAULT_CONFIG = 4


def _profiled_traffic(kernel_file: str, profile: str):
    """DRAM bytes per launch recorded by an ncu capture under profiles/, or None
    when the kernel source changed since the capture."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", profile)).read()
        src = open(os.path.join(ROOT, "paper_1003_0524_gb300", "csrc", kernel_file), "rb").read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    h = re.search(r"source_sha256_prefix: ([0-9a-f]+)", text)
    if not m or not h or hashlib.sha256(src).hexdigest()[:len(h.group(1))] != h.group(1):
        return None
    return int(m.group(1))


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="hfx_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _fold(s, ik, iq):
    m = s.mesh
    jk = (ik // (m[1] * m[2]), (ik // m[2]) % m[1], ik % m[2])
    jq = (iq // (m[1] * m[2]), (iq // m[2]) % m[1], iq % m[2])
    jp = [(jk[x] - jq[x]) % m[x] for x in range(3)]
    return (jp[0] * m[1] + jp[1]) * m[2] + jp[2]


def oracle_flops(s, ik, nsel, qs):
    """Flops of the oracle's own loops for bands nsel of k and the q in qs:
    dense v Z and Z^H (v Z), the Gaunt-weighted MT sums and the two-step
    interstitial sums, each complex multiply-add counted as 8."""
    f = 0.0
    nl = 2 * (s.lmax + 1) ** 2
    for iq in qs:
        ikp = _fold(s, ik, iq)
        m = int(s.n_occ[ikp])
        naux = s.n_aux(iq)
        nipw = int(s.Gaux[iq].shape[0])
        npw = int(s.Gk[ikp].shape[0])
        f += 8.0 * m * nsel * (naux * naux + nsel * naux + nl * s.n_mt + nipw * npw)
    return f


def oracle_sample(s, sample):
    """Time the FP64 oracle on one sample: (k, bands or None, q list or None).
    Returns seconds, the oracle's flops of the sample, its result, threads."""
    from oracle import oracle as O
    o = O.Oracle(s)
    ik, bands, qs = sample
    nsel = int(s.n_bands[ik]) if bands is None else len(bands)
    qlist = list(range(s.n_k)) if qs is None else list(qs)
    t0 = time.perf_counter()
    if bands is None and qs is None:
        V = o.vx(ik)
    elif qs is None:
        V = o.vx_sub(ik, bands)
    else:
        V = o.vx_part(ik, list(range(nsel)) if bands is None else bands, qlist)
    dt = time.perf_counter() - t0
    return dt, oracle_flops(s, ik, nsel, qlist), V, O.num_threads()


def oracle_step_flops(s):
    return sum(oracle_flops(s, ik, int(s.n_bands[ik]), range(s.n_k)) for ik in range(s.n_k))


def reference_sample(cfg, s):
    """Per-step sample of the reference arm: about a second or two of the
    oracle on the host cores."""
    if cfg <= 2:
        return (0, None, None)
    return (0, [0], list(range(8)))


def baseline_sample(cfg, s):
    """Sample of the CPU baseline inside the GPU run (about 10-30 s of CPU work),
    also compared element by element with the GPU result."""
    if cfg <= 2:
        return [(0, None, None), (min(37, s.n_k - 1), None, None)]
    return [(0, [0, int(s.n_occ[0]) - 1, int(s.n_occ[0])], None)] if cfg == 3 else [(0, [0], None)]


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1003_0524_gb300 import synthetic as S
    s = S.make_system(args.config, inversion=args.inversion)
    smp = reference_sample(args.config, s)
    full = oracle_step_flops(s)
    for _ in range(args.warmup):
        oracle_sample(s, smp)
    times = []
    cores = 1
    for _ in range(args.steps):
        dt, fs, _, cores = oracle_sample(s, smp)
        times.append(dt * full / fs)
    v = statistics.mean(times)
    ik, bands, qs = smp
    what = (f"V^x(k={ik})" + (f" bands {bands}" if bands is not None else " all bands") +
            (f", q {qs[0]}..{qs[-1]} of {s.n_k}" if qs is not None else f", all {s.n_k} q"))
    sample = f"{what} per step, extrapolated to the whole step by the oracle's flop count (x{full / fs:.4g})"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(args, ws),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _workload(args):
    w = WORKLOADS[args.config]
    return w + ", inversion-symmetric variant (real path, Sec. III.D)" if getattr(args, "inversion", False) else w


def _config(args, ws):
    return {"workload": _workload(args), "config_index": args.config, "precision": args.precision,
            "inversion": bool(getattr(args, "inversion", False)),
            "l2": "inputs larger than L2 (per-step working set of tens to hundreds of GB)",
            "parallelism": "replicas" if ws > 1 else "1 GPU"}


def fft_flops(stats_pairs, n):
    """Interstitial products by FFT in the algorithmic count: m n (5 N log2 N + 6 N), N = n^3."""
    N = n ** 3
    return stats_pairs * (5.0 * N * math.log2(N) + 6.0 * N)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1003_0524_gb300 import build as B
    from paper_1003_0524_gb300 import hfx
    from paper_1003_0524_gb300 import synthetic as S

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    hfx.load()
    t_gen = time.perf_counter()
    s = S.make_system(args.config, inversion=args.inversion, **({"mesh": (args.mesh,) * 3} if args.mesh else {}))
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream().cuda_stream
    ctx = hfx.Context(s, precision=args.precision, stream=stream, device=local, tuning=True)
    tuned = ctx.tuned
    ctx.load_system()
    # the first build after set_coulomb also runs the once-per-SCF-cycle work
    # (multipole transform of every v(q), sparse check, slices of v_t, q->0
    # bracket) and the build plan; the second captures the launches as a graph
    first_ms = None
    for i in range(args.warmup):
        t0 = time.perf_counter()
        ctx.build_all()
        torch.cuda.synchronize()
        if i == 0:
            first_ms = (time.perf_counter() - t0) * 1e3
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.4)
    stats = []
    _barrier(ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        stats.append(ctx.build_all())
    e1.record()
    torch.cuda.synchronize()
    _barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ck = clocks.stop()
    ms = _max_over_ranks(ms, ws)

    def avg(key):
        return statistics.mean(st[key] for st in stats)

    st = stats[0]
    # pair count m n per (k, q), for the FFT term of the algorithmic count
    mn = sum(int(s.n_occ[_fold(s, ik, iq)]) * int(s.n_bands[ik]) for ik in range(s.n_k) for iq in range(s.n_k))
    fl_fft = fft_flops(mn, FFT_N.get(args.config, 24))
    if args.inversion:
        fl_fft *= 0.5   # real products: real-to-complex transforms, half the work
    useful_8d = st["useful_flops"] - st["flops_zipw"] + fl_fft
    V_ours = {ik: ctx.exchange(ik) for ik in range(s.n_k)}
    ex_ours = ctx.energy()

    # end to end through the ABI: pinned host inputs in, V^x and E_x out
    pinned = []
    h2d = 0
    for ik in range(s.n_k):
        c = torch.from_numpy(np.ascontiguousarray(s.c[ik])).pin_memory()
        A = torch.from_numpy(np.ascontiguousarray(s.A[ik])).pin_memory()
        G = torch.from_numpy(np.ascontiguousarray(s.Gk[ik], dtype=np.int32)).pin_memory()
        pinned.append((c.numpy(), A.numpy(), G.numpy()))
        h2d += c.numel() * 16 + A.numel() * 16 + G.numel() * 4
    d2h = sum(int(n) * int(n) * 16 for n in s.n_bands) + 8
    e2e_times = []
    for _ in range(max(1, args.e2e_steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ik in range(s.n_k):
            c, A, G = pinned[ik]
            hfx.hfx_set_kpoint(ctx.ctx, ik, int(s.n_bands[ik]), int(s.n_occ[ik]), G, c, A)
        ctx.build_all()
        out = [ctx.exchange(ik) for ik in range(s.n_k)]
        ex = ctx.energy()
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    # N replicas finish N steps in the slowest replica's time
    e2e = _max_over_ranks(statistics.mean(e2e_times), ws) / ws
    del out, ex
    # the step after the build: V^x in the LAPW basis of every k (Eq. APW trafo)
    lapw = None
    if not args.mesh:
        for ik in range(s.n_k):
            hfx.hfx_set_overlap(ctx.ctx, ik, S.overlap(s, ik))
        hfx.hfx_lapw_transform_all(ctx.ctx)
        lt = [hfx.hfx_lapw_transform_all(ctx.ctx) for _ in range(3)]
        ms_l = statistics.mean(x["ms_total"] for x in lt)
        lapw = {"ms": ms_l, "tflops_fp64": lt[0]["useful_flops"] / (ms_l * 1e-3) / 1e12, "launches": lt[0]["n_launches"],
                "what": "V_GG'(k) = (S c) V^x (c^H S) for every k, FP64 batched GEMMs; not in value"}
    ctx.close()   # the FP64 build below needs the device memory

    # plain FP64 GPU build (the comparison of the metric): every k of small
    # workloads; one sampled k (its N_k pairs) of the large ones, scaled by the
    # pair count
    fp64 = None
    if args.fp64_steps > 0 and args.precision != "fp64":
        c64 = hfx.Context(s, precision="fp64", stream=stream, device=local)
        c64.load_system()
        full = args.config <= 2 or args.mesh
        ks64 = list(range(s.n_k)) if full else [0]
        if full:
            c64.build_all()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(args.fp64_steps):
            if full:
                st64 = c64.build_all()
            else:
                V64s = {0: c64.build_exchange(0)}
        f1.record()
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        if full:
            V64 = {ik: c64.exchange(ik) for ik in ks64}
            d_ex = ex_ours - c64.energy()
            fl64 = st64["useful_flops"] - st64["flops_zipw"] + fl_fft
        else:
            V64 = V64s
            ms64 *= s.n_k          # one k of N_k, every k costs the same
            d_ex = None
            fl64 = useful_8d
        d64 = max(float(np.abs(V_ours[k] - V64[k]).max()) for k in V64)
        fp64 = {"ms_per_step": ms64, "speedup_split_over_fp64": ms64 / ms, "max_abs_dV_split_vs_fp64_gpu": d64,
                "fp64_useful_tflops": fl64 / (ms64 * 1e-3) / 1e12, "dE_x_split_vs_fp64_gpu": d_ex,
                "sample": "every k" if full else f"V^x(k=0) (its {s.n_k} pairs), time x{s.n_k}"}
        c64.close()

    extra = {}
    if lapw:
        extra["lapw_transform"] = lapw
    if args.extra_config2 and args.config != 2 and not args.mesh:
        extra["config2"] = measure_config2(args, stream, local)
    if args.extra_inversion and args.precision == "sliced" and not args.mesh and not args.inversion:
        extra["inversion"] = measure_inversion(args, stream, local, ms)

    line = None
    if rank == 0:
        peaks, peak_kind = _peaks()
        kernels = {
            # the Coulomb apply as executed: the upper triangle of v_t (Hermitian split)
            "apply": (avg("ms_apply"), st["flops_apply_exec"]),
            "zhy": (avg("ms_zhy"), st["flops_zhy"]),
            "zipw": (avg("ms_zipw"), st["flops_zipw"]),
        }
        dom = max(kernels, key=lambda k: kernels[k][0])
        names = {"apply": "gemm1_kernel", "zhy": "gemm2_kernel", "zipw": "zipw_tc_kernel"}
        sfx = f"config{args.config}" + ("_inversion" if args.inversion else "")
        files = {"apply": ("k_contract_tc.cu", f"gemm1_kernel_{sfx}.md"),
                 "zhy": ("k_contract_tc.cu", f"gemm2_kernel_{sfx}.md"),
                 "zipw": ("k_zipw_tc.cu", f"zipw_tc_kernel_{sfx}.md")}
        nlaunch_dom = st["n_batches"]
        if args.precision == "sliced":
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            # algorithmic flops of the kernel's step (the interstitial products by
            # their FFT count); every real multiply-add expands into 10 BF16 slice products
            alg = fl_fft if dom == "zipw" else kernels[dom][1]
            achieved = 10.0 * alg / (kernels[dom][0] * 1e-3) / 1e12
            roof = {"bound": "tensor", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": _profiled_traffic(*files[dom]),
                    "peak_source": f"bf16_tflops_sustained ({peak_kind})",
                    "count": "10 BF16 slice products per real multiply-add of the algorithmic flops",
                    "algorithmic_flops_per_launch": alg / nlaunch_dom, "launches_per_step": nlaunch_dom,
                    "useful_tflops": alg / (kernels[dom][0] * 1e-3) / 1e12,
                    "per_kernel_ms": {names[k]: kernels[k][0] for k in kernels},
                    "per_kernel_frac": {names[k]: 10.0 * (fl_fft if k == "zipw" else kernels[k][1]) /
                                        (kernels[k][0] * 1e-3) / 1e12 / peak for k in kernels if kernels[k][0] > 0},
                    "zipw_frac_direct_sum_count": 10.0 * kernels["zipw"][1] / (kernels["zipw"][0] * 1e-3) / 1e12 / peak
                    if kernels["zipw"][0] > 0 else None}
        else:
            # FP64 on the CUDA cores: nominal GB300 FP64 rate
            alg = kernels[dom][1]
            achieved = alg / (kernels[dom][0] * 1e-3) / 1e12
            peak = 1.25
            roof = {"bound": "alu", "kernel": {"zipw": "zipw_kernel<double>", "apply": "zgemm64_kernel",
                                               "zhy": "zgemm64_kernel"}[dom],
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None, "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"}
        roof["kernel_ms_per_step"] = kernels[dom][0]
        cpu = None
        if not args.no_cpu_baseline:
            dts, fss, cores, dvs, what = 0.0, 0.0, 1, [], []
            for smp in baseline_sample(args.config, s):
                dt, fs, Vref, cores = oracle_sample(s, smp)
                dts += dt
                fss += fs
                ik, bands = smp[0], smp[1]
                sel = list(range(int(s.n_bands[ik]))) if bands is None else bands
                dvs.append(float(np.abs(V_ours[ik][np.ix_(sel, sel)] - Vref).max()))
                what.append(f"V^x(k={ik})" + (f"[{bands}][{bands}]" if bands is not None else "") + f", all {s.n_k} q")
            full = oracle_step_flops(s)
            cpu = {"value": dts * full / fss, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "; ".join(what) + f" ({dts:.1f} s), extrapolated by the oracle's flop count "
                                               f"(x{full / fss:.4g})",
                   "max_abs_dV_vs_oracle_sampled": max(dvs)}
        value = ms * 1e-3 / ws if ws > 1 else ms * 1e-3
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.precision == "sliced" else "f64", "data": "synthetic",
            "config": _config(args, ws),
            "useful_tflops": useful_8d / (ms * 1e-3) / 1e12,
            "useful_tflops_direct_sum": st["useful_flops"] / (ms * 1e-3) / 1e12,
            "stage_ms": {"stage1": avg("ms_stage1"), "contract": avg("ms_contract"), "finish": avg("ms_finish"),
                         "zipw": avg("ms_zipw"), "apply": avg("ms_apply"), "zhy": avg("ms_zhy")},
            "batches": st["n_batches"], "graph_replayed": all(x["graph_replayed"] for x in stats),
            "tiles": {"nb_zhy": st["tile_nb_zhy"], "nb_zipw": st["tile_nb_zipw"],
                      "source": "autotuner (paper_1003_0524_gb300/tuning.json)" if tuned else "library formula"},
            "roofline": roof,
            "cpu_baseline": cpu,
            "fp64_gpu": fp64,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(sum(x["n_launches"] for x in stats)),
            "once_per_scf_cycle": {
                "first_build_ms": first_ms,
                "coulomb_setup_ms": (first_ms - ms) if first_ms is not None else None,
                "what": "wall time of the first build minus a timed step: the v(q) multipole transform, sparse "
                        "check, v_t slices and q->0 bracket run by the first build after set_coulomb, plus the "
                        "build plan (host tables, buffers); not in value"},
            "input_generation_s": t_gen,
            "extra": extra or None,
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_config2(args, stream, local):
    """The uneven workload (n(k) 32-48, n_occ(k) 6-10, N_IPW(q) 520-680) through
    the same graph-captured build: a few steps, one k against the oracle."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_1003_0524_gb300 import hfx
    from paper_1003_0524_gb300 import synthetic as S
    s = S.make_system(2)
    with hfx.Context(s, precision="sliced", stream=stream, device=local) as c:
        c.load_system()
        for _ in range(3):
            c.build_all()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 5
        e0.record()
        sts = [c.build_all() for _ in range(n)]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        V5 = c.exchange(5)
    ref = O.Oracle(s).vx(5)
    return {"workload": WORKLOADS[2], "ms_per_step": ms, "steps": n, "useful_tflops_direct_sum":
            sts[0]["useful_flops"] / (ms * 1e-3) / 1e12, "n_launches_per_step": sts[0]["n_launches"],
            "graph_replayed": all(x["graph_replayed"] for x in sts), "batches": sts[0]["n_batches"],
            "max_abs_dV_vs_oracle_k5": float(np.abs(V5 - ref).max())}


def measure_inversion(args, stream, local, ms_complex):
    """The inversion-symmetric variant of the workload (same cell sizes, band
    windows and aux sizes; five atom pairs on config 4) on the real path of
    Sec. III.D: a few graph-replayed steps, the dominant kernel's fraction of the
    tensor peak, and V^x(k = 0) against the plain FP64 GPU build of that k."""
    import numpy as np
    import torch

    from paper_1003_0524_gb300 import hfx
    from paper_1003_0524_gb300 import synthetic as S
    t0 = time.perf_counter()
    s = S.make_system(args.config, inversion=True)
    t_gen = time.perf_counter() - t0
    with hfx.Context(s, precision="sliced", stream=stream, device=local, tuning=True) as c:
        tuned = c.tuned
        c.load_system()
        for _ in range(3):
            c.build_all()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = 3
        e0.record()
        sts = [c.build_all() for _ in range(n)]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / n
        V0 = c.exchange(0)
        imag_max = max(float(np.abs(c.exchange(ik).imag).max()) for ik in range(s.n_k))
    st = sts[0]
    peaks, peak_kind = _peaks()
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    ms_apply = statistics.mean(x["ms_apply"] for x in sts)
    with hfx.Context(s, precision="fp64", stream=stream, device=local) as c64:
        c64.load_system()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        V64 = c64.build_exchange(0)
        f1.record()
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) * s.n_k
    return {"workload": WORKLOADS[args.config] + ", inversion-symmetric variant (real path, Sec. III.D)",
            "ms_per_step": ms, "steps": n, "speedup_over_complex_path": ms_complex / ms,
            "useful_tflops_real_count": st["useful_flops"] / (ms * 1e-3) / 1e12,
            "stage_ms": {k: statistics.mean(x[k] for x in sts) for k in ("ms_zipw", "ms_apply", "ms_zhy")},
            "gemm1_frac": 10.0 * st["flops_apply_exec"] / (ms_apply * 1e-3) / 1e12 / peak,
            "gemm1_frac_peak_source": f"bf16_tflops_sustained ({peak_kind})",
            "batches": st["n_batches"], "graph_replayed": all(x["graph_replayed"] for x in sts),
            "tiles": {"nb_zhy": st["tile_nb_zhy"], "nb_zipw": st["tile_nb_zipw"],
                      "source": "autotuner" if tuned else "library formula"},
            "fp64_gpu_ms_per_step": ms64, "fp64_sample": f"V^x(k=0) (its {s.n_k} pairs), time x{s.n_k}",
            "speedup_over_fp64_gpu": ms64 / ms,
            "max_abs_dV_vs_fp64_gpu_k0": float(np.abs(V0 - V64).max()), "max_abs_imag_V": imag_max,
            "input_generation_s": t_gen}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=DEFAULT_CONFIG)
    ap.add_argument("--precision", choices=["sliced", "fp64"], default="sliced")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-config2", dest="extra_config2", action="store_false")
    ap.add_argument("--no-extra-inversion", dest="extra_inversion", action="store_false")
    ap.add_argument("--inversion", action="store_true",
                    help="time the inversion-symmetric variant of the workload (real path) as the main line")
    ap.add_argument("--mesh", type=int, default=0, help="override the k mesh (N x N x N); profiling of small cases only")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
