"""Benchmark: V^x build seconds per SCF step on one GB300.

Workload: the 2-atom zincblende cell (a = 10.3 bohr), 4x4x4 Gamma-centred k
mesh (64 k, 4096 (k,q) pairs), 40 bands, 8 occupied, MT product basis L <= 4
with 3 radial functions (150), interstitial plane waves |q+G| <= 3.0 (~485),
N_aux ~ 635, block-sparse transformed Coulomb matrix.  One step = V^x(k) for
every k of the mesh plus E_x, from device-resident wave functions and
transformed v(q) (the transform runs once per SCF cycle, in warm-up).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (the comparison arm; it never touches the GPU).
"""
from __future__ import annotations

import argparse
import json
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
WORKLOAD = "zincblende 2-atom cell a=10.3 bohr, 4x4x4 k (4096 k,q pairs), 40 bands, 8 occupied, N_aux~635, sparse v(q)"


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


def cpu_oracle_sample(sysm, ks, reps=1):
    """Time the FP64 oracle for the given k points (all q each), on the host."""
    from oracle import oracle as O
    o = O.Oracle(sysm)
    V = {}
    t0 = time.perf_counter()
    for _ in range(reps):
        for ik in ks:
            V[ik] = o.vx(ik)
    dt = (time.perf_counter() - t0) / reps
    return dt, V, O.num_threads()


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from paper_1003_0524_gb300 import synthetic as S
    s = S.make_system(args.config)
    ks = [0]
    for _ in range(args.warmup):
        cpu_oracle_sample(s, ks)
    times = []
    cores = 1
    for _ in range(args.steps):
        dt, _, cores = cpu_oracle_sample(s, ks)
        times.append(dt * s.n_k / len(ks))
    v = statistics.mean(times)
    sample = f"V^x(k) for {len(ks)} of {s.n_k} k points (all {s.n_k} q each) per step, extrapolated x{s.n_k // len(ks)}"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "config_index": args.config},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    s = S.make_system(args.config, **({"mesh": (args.mesh,) * 3} if args.mesh else {}))
    stream = torch.cuda.current_stream().cuda_stream
    ctx = hfx.Context(s, precision=args.precision, stream=stream, device=local)
    ctx.load_system()
    # the first build after set_coulomb also runs the once-per-SCF-cycle work
    # (multipole transform of every v(q), sparse check, slices of v_t, q->0 bracket)
    first_ms = None
    for i in range(args.warmup):
        st0 = ctx.build_all()
        if i == 0:
            first_ms = st0["ms_total"]
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

    useful = stats[0]["useful_flops"]
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

    # plain FP64 GPU build of the same step (the comparison of the metric)
    fp64 = None
    if args.fp64_steps > 0 and args.precision != "fp64":
        c64 = hfx.Context(s, precision="fp64", stream=stream, device=local)
        c64.load_system()
        c64.build_all()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(args.fp64_steps):
            st64 = c64.build_all()
        f1.record()
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / args.fp64_steps
        V64 = {ik: c64.exchange(ik) for ik in range(s.n_k)}
        d64 = max(float(np.abs(V_ours[k] - V64[k]).max()) for k in V64)
        fp64 = {"ms_per_step": ms64, "speedup_split_over_fp64": ms64 / ms, "max_abs_dV_split_vs_fp64_gpu": d64,
                "fp64_useful_tflops": st64["useful_flops"] / (ms64 * 1e-3) / 1e12,
                "dE_x_split_vs_fp64_gpu": ex_ours - c64.energy()}
        c64.close()

    line = None
    if rank == 0:
        peaks, peak_kind = _peaks()
        kernels = {
            "apply": (avg("ms_apply"), stats[0]["flops_apply"]),
            "zhy": (avg("ms_zhy"), stats[0]["flops_zhy"]),
            "zipw": (avg("ms_zipw"), stats[0]["flops_zipw"]),
        }
        dom = max(kernels, key=lambda k: kernels[k][0])
        names = {"apply": "gemm1_kernel", "zhy": "gemm2_kernel", "zipw": "zipw_tc_kernel"}
        if args.precision == "sliced":
            # every real multiply-add of the method expands into 10 BF16 slice products
            achieved = 10.0 * kernels[dom][1] / (kernels[dom][0] * 1e-3) / 1e12
            peak = peaks.get("bf16_tflops_sustained", 1700.0)
            traffic = _profiled_traffic("k_zipw_tc.cu", "zipw_tc_kernel_config1.md") if dom == "zipw" else None
            roof = {"bound": "tensor", "kernel": names[dom], "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "peak_source": f"bf16_tflops_sustained ({peak_kind})",
                    "useful_tflops": kernels[dom][1] / (kernels[dom][0] * 1e-3) / 1e12,
                    "per_kernel_ms": {names[k]: kernels[k][0] for k in kernels}}
        else:
            # FP64 on the CUDA cores: GB300 FP64 rate from the measured FP64 build is ~1 TFLOP/s
            achieved = kernels[dom][1] / (kernels[dom][0] * 1e-3) / 1e12
            peak = 1.25
            roof = {"bound": "alu", "kernel": {"zipw": "zipw_kernel<double>", "apply": "zgemm64_kernel",
                                               "zhy": "zgemm64_kernel"}[dom],
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "traffic": None, "peak_source": "nominal GB300 FP64 1.25 TFLOP/s"}
        roof["kernel_ms_per_step"] = kernels[dom][0]
        cpu = None
        if not args.no_cpu_baseline:
            ks = [0, 37]
            dt, Vref, cores = cpu_oracle_sample(s, ks)
            dv = max(float(np.abs(V_ours[k] - Vref[k]).max()) for k in ks)
            cpu = {"value": dt * s.n_k / len(ks), "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"V^x(k) for k in {ks} (all {s.n_k} q each), extrapolated x{s.n_k // len(ks)}",
                   "max_abs_dV_vs_oracle_sampled_k": dv}
        value = ms * 1e-3 / ws if ws > 1 else ms * 1e-3
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.precision == "sliced" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "config_index": args.config, "precision": args.precision,
                       "l2": "inputs larger than L2 (per-step working set ~20 GB)", "parallelism": "replicas" if ws > 1 else "1 GPU"},
            "useful_tflops": useful / (ms * 1e-3) / 1e12,
            "stage_ms": {"stage1": avg("ms_stage1"), "contract": avg("ms_contract"), "finish": avg("ms_finish"),
                         "zipw": avg("ms_zipw"), "apply": avg("ms_apply"), "zhy": avg("ms_zhy")},
            "roofline": roof,
            "cpu_baseline": cpu,
            "fp64_gpu": fp64,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(sum(st["n_launches"] for st in stats)),
            "once_per_scf_cycle": {
                "first_build_ms": first_ms,
                "coulomb_setup_ms": (first_ms - ms) if first_ms is not None else None,
                "what": "first build minus a timed step: the v(q) multipole transform, sparse check, v_t slices "
                        "and q->0 bracket run by the first build after set_coulomb, plus the first-use allocation "
                        "of the scratch buffers; not in value"},
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--precision", choices=["sliced", "fp64"], default="sliced")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mesh", type=int, default=0, help="override the k mesh (N x N x N); profiling of small cases only")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
