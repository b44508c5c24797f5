"""Benchmark of the FMM apply on one GB300 (or N independent replicas under torchrun).

Workload: 262,144 points uniform on the unit sphere (sources = targets), kappa = 64,
eps = 1e-6, complex64 charges N(0,1), one right-hand side.  The headline `value` is the
mixed-precision apply in Mpoints*RHS/s (N_t * R / t_apply / 1e6) with inputs resident in
HBM; `fp64_path` is the all-float64 apply on the same workload; `e2e` is the same metric
through the public API with pinned host buffers and both copies inside the timed region.
Every timed apply is preceded by an L2 flush (a 512 MiB write) outside its event pair.

--impl reference times the CPU oracle (direct sum over all sources for a seeded subset of
targets) on the host cores; it is the baseline arm, not the target.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="sphere262k", points=262144, surface="unit sphere", kappa=64.0, eps=1e-6,
                nrhs=1, charges="complex64 N(0,1)")
ORACLE_TARGETS = 2000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64-path measurement")
    ap.add_argument("--points", type=int, default=262144, help="smaller sphere for profiling runs")
    ap.add_argument("--skip-oracle", action="store_true", help="skip the CPU oracle timing")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint and 64-RHS cube measurements")
    return ap.parse_args()


def dist_setup(ngpus):
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if ngpus > 0 else "gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    """Maximum of x over the ranks (NCCL on the GPUs, gloo on the host)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(ms_local, points_per_rank, world):
    """Whole-job rate of N independent replicas: every rank applies the same workload, the
    job takes the slowest rank's time, and the points of all ranks count.  Returns
    (max ms over ranks, Mpoints*RHS/s)."""
    ms = allmax(float(ms_local), world)
    return ms, world * points_per_rank / (ms * 1e-3) / 1e6


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def time_oracle(s, t, q, kappa, ntargets, seed):
    from oracle import direct
    idx = np.sort(np.random.default_rng(seed).choice(len(t), ntargets, replace=False))
    t0 = time.perf_counter()
    direct.direct(s, t[idx], q, kappa)
    return time.perf_counter() - t0


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_0911_4114_gb300 import workloads as wl
    s, t = wl.points("sphere262k")
    q = wl.charges(len(s), 0, wl.rng(1, salt=1)).astype(np.complex64).astype(np.complex128)
    for i in range(args.warmup):
        time_oracle(s, t, q, 64.0, 200, 100 + i)
    secs = [time_oracle(s, t, q, 64.0, ORACLE_TARGETS, 200 + i) for i in range(args.steps)]
    value = ORACLE_TARGETS / float(np.mean(secs)) / 1e6
    line = {"impl": "reference", "metric": "FMM apply Mpoints*RHS/s at stated rel. err; mixed vs FP64 on one GB300",
            "value": value, "unit": "Mpoints*RHS/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD, l2="n/a (host)"),
            "cpu_baseline": {"value": value, "unit": "Mpoints*RHS/s", "cores": oracle_threads(), "kind": "oracle",
                             "sample": f"float64 direct sum over all 262,144 sources for {ORACLE_TARGETS} seeded "
                                       f"targets per step (exact; the FMM approximates it)"},
            "e2e": {"value": value, "unit": "Mpoints*RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def count_launches(info):
    lf = info["lf"]
    n = 3  # permute in, near field, permute out
    if lf >= 2:
        n += 1 + 3 * (lf - 2) + (lf - 1) + 3 * (lf - 2) + 1
    return n


ALU_NOTE = "152 SMs x 128 FP32 lanes x median SM clock under load"


def stage_rooflines(info, stage_ms, n_src, n_tgt, fp32_peak, hbm):
    """Roofline entry of every stage with a defined unit of work (plan summary `info`, live
    stage times in ms); FP32-pipe operations against fp32_peak (Gop/s) for arithmetic-bound
    stages, algorithmic bytes against hbm (GB/s) for the re-quadratures."""
    levels = {int(l): v for l, v in info["levels"].items()}
    lev = levels.get(info["lf"], {})
    sample_bytes = {"fp32": 8.0, "df": 16.0, "fp64": 16.0}
    # FP32-pipe operations per (list entry, sample) of M2L: complex multiply-add in float32
    # (4 FMA) or four Dekker products into lazy double-float accumulators (48)
    m2l_ops = {"fp32": 4.0, "df": 48.0}

    def alu(kernel, ops, ms, unit_work):
        return dict(kernel=kernel, bound="alu", achieved=ops / (ms * 1e-3) / 1e9, peak=fp32_peak,
                    unit="Gop/s", unit_work=unit_work, peak_note=ALU_NOTE)

    def one(stage):
        ms = stage_ms[stage]
        if ms <= 0.0:
            return None
        if stage == "near_field" and info["near_precision"] == "fp32":
            if info["near_symmetric"]:
                # pairs of distinct boxes evaluated once (38 ops) plus the reverse product and
                # its share of the warp reduction (13 ops); pairs inside a box one way (38 ops)
                off = info["p2p_pairs"] - info["p2p_self_pairs"]
                ops = 38.0 * info["p2p_self_pairs"] + (38.0 + 13.0) * off / 2
                return alu("k_p2p_mixed_sym_warp", ops, ms,
                           "38 float32 ops per evaluated pair + 13 for the reverse direction")
            return alu("k_p2p_mixed_warp", 38.0 * info["p2p_pairs"], ms, "38 float32 ops per target-source pair")
        if stage in ("s2m", "l2t") and lev.get("precision") == "df":
            units = float(lev["K"]) / 2 * (n_tgt if stage == "l2t" else n_src)
            return alu("k_l2t_df_warp" if stage == "l2t" else "k_s2m_df", 156.0 * units, ms,
                       "156 float32 ops per (point, antipodal sample pair) in double-float")
        if stage == "m2l" and levels and all(v["precision"] in m2l_ops for v in levels.values()):
            ops = sum(m2l_ops[v["precision"]] * v["ilist_total"] * v["K"] for v in levels.values())
            return alu("k_m2l", ops, ms, "4 (float32) or 48 (double-float) float32 ops per list entry and sample")
        if stage in ("m2l", "m2m", "l2l"):
            tot = 0.0
            for l, v in levels.items():
                b = sample_bytes[v["precision"]]
                if stage == "m2l":
                    tot += (2.0 * v["nbox"] * v["K"] + 316.0 * v["K"]) * b
                elif l > 2:
                    up = levels[l - 1]
                    tot += v["nbox"] * v["K"] * b + up["nbox"] * up["K"] * sample_bytes[up["precision"]]
            return dict(kernel={"m2l": "k_m2l", "m2m": "k_requad_spec_* (M2M)",
                                "l2l": "k_requad_spec_* (L2L)"}[stage],
                        bound="hbm", achieved=tot / (ms * 1e-3) / 1e9, peak=hbm, unit="GB/s",
                        unit_work="algorithmic signature bytes (each read and written once)")
        return None

    out = {}
    for name in stage_ms:
        r = one(name)
        if r is not None:
            r["frac"] = r["achieved"] / r["peak"]
            r["stage_ms"] = stage_ms[name]
            out[name] = r
    return out


def main():
    args = parse()
    rank, world = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from oracle import direct
    from paper_0911_4114_gb300 import FmmPlan, workloads as wl
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    s, t = wl.points("sphere262k", n=args.points)
    kappa, eps = 64.0, 1e-6
    q_host = wl.charges(len(s), 0, wl.rng(1, salt=1)).astype(np.complex64)
    q = torch.as_tensor(q_host).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(plan, steps, warmup):
        out = torch.empty((len(t), 1), dtype=torch.complex64, device=dev)
        q2 = q.reshape(-1, 1)
        for _ in range(warmup):
            plan.apply(q2, out=out)
        torch.cuda.synchronize()
        barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            plan.apply(q2, out=out)
            b.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms = [a.elapsed_time(b) for a, b in ev]
        return allmax(float(np.mean(ms)), world), out

    plans = {}
    for precision in (("mixed",) if args.no_fp64 else ("mixed", "fp64")):
        t0 = time.perf_counter()
        plans[precision] = FmmPlan(s, t, kappa, eps, precision=precision)
        plans[precision].plan_seconds = time.perf_counter() - t0

    idx = np.sort(wl.rng(1, salt=2).choice(len(t), 1000, replace=False))
    ref = direct.direct(s, t[idx], q_host.astype(np.complex128), kappa)
    results = {}
    with ClockSampler(local) as clk:
        for precision, plan in plans.items():
            ms, out = timed(plan, args.steps, args.warmup)
            got = out[:, 0].cpu().numpy().astype(np.complex128)[idx]
            results[precision] = dict(ms=ms, rel_err=float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    clocks = clk.summary()

    # per-stage device times of the mixed apply (library events on the apply stream)
    mp = plans["mixed"]
    mp.set_timing(True)
    stage_ms = {k: 0.0 for k in ("permute_in", "near_field", "s2m", "m2m", "m2l", "l2l", "l2t", "permute_out")}
    nst = max(3, args.steps // 2)
    out = torch.empty((len(t), 1), dtype=torch.complex64, device=dev)
    for _ in range(nst):
        flush.fill_(1.0)
        mp.apply(q.reshape(-1, 1), out=out)
        for k, v in mp.info()["stage_ms"].items():
            stage_ms[k] += v / nst
    mp.set_timing(False)
    info = mp.info()

    # end to end through the public API: pinned host in, host out
    qh = torch.as_tensor(q_host).reshape(-1, 1).pin_memory()
    ph = torch.empty((len(t), 1), dtype=torch.complex64).pin_memory()
    qd = torch.empty_like(qh, device=dev)
    od = torch.empty((len(t), 1), dtype=torch.complex64, device=dev)
    for _ in range(args.warmup):
        qd.copy_(qh, non_blocking=True)
        mp.apply(qd, out=od)
        ph.copy_(od, non_blocking=True)
    torch.cuda.synchronize()
    barrier(world)
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        qd.copy_(qh, non_blocking=True)
        mp.apply(qd, out=od)
        ph.copy_(od, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e = allmax(float(np.mean(e2e_ms)), world)

    # adjoint of the same plan, and the 64-RHS cube (tensor-core near field), device-timed
    extras = None
    if not args.no_extras and args.points == 262144:
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
        wadj = torch.empty((len(s), 1), dtype=torch.complex64, device=dev)
        mp.apply_adjoint(q.reshape(-1, 1), out=wadj)
        for a, b in ev:
            flush.fill_(1.0)
            a.record(stream)
            mp.apply_adjoint(q.reshape(-1, 1), out=wadj)
            b.record(stream)
        torch.cuda.synchronize()
        adj_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        cs, ct = wl.points("cube512k_rhs64")
        cplan = FmmPlan(cs, ct, 40.0, 1e-5, precision="mixed", max_rhs=64)
        cq = torch.as_tensor(wl.charges(len(cs), 64, wl.rng(3, salt=1)).astype(np.complex64)).to(dev)
        cout = torch.empty((len(ct), 64), dtype=torch.complex64, device=dev)
        cplan.apply(cq, out=cout)
        for a, b in ev[:2]:
            a.record(stream)
            cplan.apply(cq, out=cout)
            b.record(stream)
        torch.cuda.synchronize()
        cms = float(np.mean([a.elapsed_time(b) for a, b in ev[:2]]))
        cplan.set_timing(True)
        cplan.apply(cq, out=cout)
        torch.cuda.synchronize()
        ci = cplan.info()
        cplan.set_timing(False)
        extras = {"adjoint": {"ms_per_step": adj_ms, "value": len(s) / (adj_ms * 1e-3) / 1e6,
                              "unit": "Mpoints*RHS/s"},
                  "cube512k_rhs64": {"ms_per_step": cms, "value": len(ct) * 64 / (cms * 1e-3) / 1e6,
                                     "unit": "Mpoints*RHS/s", "nrhs": 64, "kappa": 40.0, "eps": 1e-5,
                                     "lf": ci["lf"], "p2p_pairs": ci["p2p_pairs"],
                                     "near_field": "tensor-core GEMM form (mma.sync 3xTF32)",
                                     "pair_rhs_per_s": ci["p2p_pairs"] * 64 / (cms * 1e-3),
                                     "stage_ms": ci["stage_ms"],
                                     "levels": {str(l): v["precision"] for l, v in ci["levels"].items()}}}
        del cplan, cq, cout

    # CPU oracle on this host (rank 0 only), bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.skip_oracle:
        secs = time_oracle(s, t, q_host.astype(np.complex128), kappa, ORACLE_TARGETS, 300)
        cpu = {"value": ORACLE_TARGETS / secs / 1e6, "unit": "Mpoints*RHS/s", "cores": oracle_threads(),
               "kind": "oracle", "sample": f"float64 direct sum over all 262,144 sources for {ORACLE_TARGETS} "
                                           f"seeded targets ({secs:.1f} s)"}

    # rooflines per stage; the top-level entry is the dominant stage's
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_clock = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * sm_clock * 1e6 / 1e9          # FP32-pipe ops/s (Gop/s)
    hbm = peaks.get("hbm_gbs", 6800.0)
    roof_stages = stage_rooflines(info, stage_ms, len(s), len(t), fp32_peak, hbm)
    stage = max(stage_ms, key=stage_ms.get)
    roof = dict(roof_stages.get(stage) or {"kernel": stage, "bound": None, "achieved": None, "peak": None,
                                          "unit": None, "frac": None, "stage_ms": stage_ms[stage]})
    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
    # this workload at full size (profiles/sphere262k_launch_list.md); a kernel changed since its
    # capture has no entry
    traffic = {"k_p2p_mixed_sym_warp": 25.35e6}
    roof["traffic"] = traffic.get(roof.get("kernel")) if len(t) == 262144 else None
    roof["peak_source"] = "of measured" if peaks else "of fallback"

    nt = len(t)
    _, value = replica_rate(results["mixed"]["ms"], nt, world)
    fp64_value = replica_rate(results["fp64"]["ms"], nt, world)[1] if "fp64" in results else None
    _, e2e_value = replica_rate(e2e, nt, world)
    line = {"metric": "FMM apply Mpoints*RHS/s at stated rel. err; mixed vs FP64 on one GB300",
            "value": value, "unit": "Mpoints*RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": results["mixed"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(WORKLOAD, points=len(t), parallelism="replicas" if world > 1 else "single",
                           l2="flushed before every timed apply (512 MiB write)",
                           lf=info["lf"], levels={str(l): v for l, v in info["levels"].items()},
                           p2p_pairs=info["p2p_pairs"]),
            "rel_err": results["mixed"]["rel_err"],
            "fp64_path": ({"value": fp64_value,
                           "ms_per_step": results["fp64"]["ms"], "rel_err": results["fp64"]["rel_err"],
                           "lf": plans["fp64"].info()["lf"]} if "fp64" in results else None),
            "stage_ms": stage_ms, "plan_seconds": plans["mixed"].plan_seconds,
            "e2e": {"value": e2e_value, "unit": "Mpoints*RHS/s",
                    "h2d_bytes_per_step": int(qh.numel() * 8), "d2h_bytes_per_step": int(ph.numel() * 8)},
            "roofline": roof, "roofline_stages": {k: {kk: v[kk] for kk in ("kernel", "bound", "achieved", "unit", "frac")}
                                                  for k, v in roof_stages.items()},
            "cpu_baseline": cpu, "gpu_launches": count_launches(info) * args.steps,
            "clocks": clocks, "extras": extras}
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
