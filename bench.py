"""Benchmark of the FMM apply on one GB300 (or N independent replicas under torchrun).

Headline workload: 2,097,152 points uniform by area on the (1, 0.5, 0.25) ellipsoid
(sources = targets), kappa = 200, eps = 1e-4, complex64 charges N(0,1), one right-hand side,
mixed precision.  `value` is that apply in Mpoints*RHS/s (N_t * R / t_apply / 1e6) with
inputs resident in HBM; every timed apply is preceded by an L2 flush (a 512 MiB write)
outside its event pair.  Beside it, on the same points:
  fp64_path   the all-float64 apply at eps 1e-4;
  tight       the mixed apply at eps 1e-8 with complex128 charges, and the float64 apply there;
  rel_err     relative L2 error against the float64 direct sum on 1,000 seeded targets
              (the library's float64 direct sum, which the tests pin to the oracle), and
              against the oracle's direct sum on a 64-target subset;
  e2e         the headline metric through the public API, pinned host buffers, both copies
              inside the timed region.
`extras`: the 262,144-point sphere (kappa 64, eps 1e-6, mixed and float64), the adjoint of
the headline plan, the 524,288-point cube with 64 right-hand sides and 32 uneven problems in
one graph launch.

cpu_baseline / --impl reference: the oracle's float64 Fourier FMM at the same plan, timed
stage by stage on seeded samples of boxes and extrapolated by each stage's work (plan and
transfer tables excluded, as for the GPU); the baseline arm, not the target.
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

METRIC = "FMM apply Mpoints*RHS/s at stated rel. err; mixed vs FP64 on one GB300"
HEADLINE = dict(workload="ellipsoid2m", points=2097152, surface="(1, 0.5, 0.25) ellipsoid, uniform by area",
                kappa=200.0, eps=1e-4, nrhs=1, charges="complex64 N(0,1)", precision="mixed",
                plan_shape="tuned (buffer boxes and leaf level chosen by the plan's cost model)")
AUTO = dict(buffer=0)     # plan shape chosen by the library's cost model
TIGHT_EPS = 1e-8
REL_ERR_TARGETS = 1000
ORACLE_DIRECT_TARGETS = 64
STAGES = ("permute_in", "near_field", "s2m", "m2m", "m2l", "l2l", "l2t", "permute_out")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", type=int, default=2097152, help="smaller ellipsoid for profiling runs")
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64-path measurements")
    ap.add_argument("--no-tight", action="store_true", help="skip the eps = 1e-8 measurements")
    ap.add_argument("--skip-oracle", action="store_true", help="skip the CPU oracle timing")
    ap.add_argument("--no-extras", action="store_true", help="skip the extra workloads")
    ap.add_argument("--cube-only", type=int, default=0, metavar="N",
                    help="time only the 64-RHS cube workload on its first N points and print its line (profiling runs)")
    ap.add_argument("--adaptive-only", action="store_true",
                    help="time only the adaptive-tree comparisons and print their line (profiling runs)")
    ap.add_argument("--buffer", type=int, default=0, choices=[0, 1, 2],
                    help="plan shape of the measured plans: 0 tuned (default), 1 or 2 buffer boxes (profiling runs)")
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


# ----------------------------------------------------------------------------------------
# CPU oracle legs (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------------------
def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [1])
    except Exception:
        return os.cpu_count() or 1


def oracle_direct_sample(s, t, q, kappa, ntargets, seed):
    """The oracle's float64 direct sum over all sources for `ntargets` seeded targets."""
    from oracle import direct
    idx = np.sort(np.random.default_rng(seed).choice(len(t), ntargets, replace=False))
    t0 = time.perf_counter()
    vals = direct.direct(s, t[idx], q, kappa, block=8)
    return idx, vals, time.perf_counter() - t0


class OracleFmmSampler:
    """The oracle's Fourier FMM at the GPU run's plan, timed stage by stage on seeded samples
    of boxes and extrapolated to one whole apply by each stage's work.

    Work measures: near field, target-source pairs; S2M, sources; L2T, targets; M2M and L2L,
    child boxes; M2L, interaction-list entries.  The plan (tree, quadratures) and the transfer
    tables of the sampled boxes are built before timing, as the GPU apply excludes its plan.
    Signatures fed to the sampled stages are zeros of the right shapes (the arithmetic does not
    depend on their values)."""

    def __init__(self, s, t, q, kappa, eps, precision="mixed", leaf_boxes=12, level_boxes=3, seed=0,
                 buffer=1, depth=0):
        from oracle import fmm as ofmm
        self.ofmm = ofmm
        self.plan = ofmm.Plan(s, t, kappa, eps, precision=precision, buffer=buffer, depth=depth)
        self.q = np.asarray(q, dtype=np.complex128).reshape(len(s), -1)
        self.nt = len(t)
        tr = self.plan.tree
        lf = tr.depth
        g = np.random.default_rng(seed)
        nleaf = len(tr.levels[lf]["key"])
        busy = np.flatnonzero((tr.tgt_count > 0) | (tr.src_count > 0))
        self.leaf = np.sort(g.choice(busy, min(leaf_boxes, len(busy)), replace=False))
        self.level = {}
        for l in range(2, lf + 1):
            nb = len(tr.levels[l]["key"])
            self.level[l] = np.sort(g.choice(nb, min(level_boxes, nb), replace=False))
        # work of the samples and of the whole apply
        pairs = np.array([tr.tgt_count[b] * sum(int(tr.src_count[n]) for n in tr.nlist[b]) for b in range(nleaf)],
                         dtype=np.float64)
        self.work = {"near": (pairs[self.leaf].sum(), pairs.sum()),
                     "s2m": (tr.src_count[self.leaf].sum(), tr.src_count.sum()),
                     "l2t": (tr.tgt_count[self.leaf].sum(), tr.tgt_count.sum())}
        for l in range(2, lf + 1):
            ilen = np.array([len(x) for x in tr.ilist[l]], dtype=np.float64)
            self.work[("m2l", l)] = (ilen[self.level[l]].sum(), ilen.sum())
            nb = len(tr.levels[l]["key"])
            if l > 2:
                self.work[("m2m", l)] = (len(self.level[l]), nb)
                self.work[("l2l", l)] = (len(self.level[l]), nb)
        # transfer tables of the sampled M2L boxes (plan time)
        for l in range(2, lf + 1):
            for a in self.level[l]:
                for v in tr.vlist[l][a]:
                    self.plan.table(l, v)

    def time_once(self):
        """Seconds of one extrapolated apply, and the per-stage estimates."""
        p, tr, of = self.plan, self.plan.tree, self.ofmm
        lf = tr.depth
        R = self.q.shape[1]
        qs = self.q[tr.src_perm]
        zeros = {l: np.zeros((len(tr.levels[l]["key"]), R, p.levels[l].K), dtype=np.complex128)
                 for l in range(2, lf + 1)}
        est = {}

        def clock(key, fn):
            t0 = time.perf_counter()
            fn()
            dt = time.perf_counter() - t0
            done, total = self.work[key]
            est[key] = dt * (total / done) if done > 0 else 0.0

        clock("near", lambda: of.p2p(p, qs, boxes=self.leaf))
        if lf >= 2:
            clock("s2m", lambda: of.s2m(p, qs, boxes=self.leaf))
            for l in range(lf, 2, -1):
                clock(("m2m", l), lambda l=l: of.m2m(p, zeros[l], l, boxes=self.level[l]))
            for l in range(2, lf + 1):
                clock(("m2l", l), lambda l=l: of.m2l(p, zeros[l], l, boxes=self.level[l]))
            for l in range(2, lf):
                clock(("l2l", l + 1), lambda l=l: of.l2l(p, zeros[l], zeros[l + 1], l, boxes=self.level[l + 1]))
            clock("l2t", lambda: of.l2t(p, zeros[lf], R, boxes=self.leaf))
        return float(sum(est.values())), est

    def sample_text(self):
        lf = self.plan.tree.depth
        return (f"oracle float64 Fourier FMM (buffer boxes {self.plan.buffer}, L_f = {lf}), timed on "
                f"{len(self.leaf)} seeded leaf "
                f"boxes (near field, S2M, L2T) and {max(len(v) for v in self.level.values()) if self.level else 0} "
                f"boxes per level (M2M, M2L, L2L), extrapolated per stage by pairs / points / boxes / list "
                f"entries; plan and transfer tables excluded")


def headline_points(n=None):
    from paper_0911_4114_gb300 import workloads as wl
    s, t = wl.points("ellipsoid2m", n=n)
    q = wl.charges(len(s), 0, wl.rng(2, salt=1)).astype(np.complex64)
    return s, t, q


def run_reference(args, rank, world):
    if rank != 0:
        return
    s, t, q = headline_points(args.points if args.points != 2097152 else None)
    smp = OracleFmmSampler(s, t, q.astype(np.complex128), HEADLINE["kappa"], HEADLINE["eps"],
                           leaf_boxes=4, level_boxes=1)
    for _ in range(args.warmup):
        smp.time_once()
    secs = [smp.time_once()[0] for _ in range(args.steps)]
    value = len(t) / float(np.mean(secs)) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpoints*RHS/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(secs)), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(HEADLINE, points=len(t), l2="n/a (host)",
                           plan_shape=f"oracle plan, {smp.plan.buffer} buffer box(es), L_f = {smp.plan.lf}"),
            "cpu_baseline": {"value": value, "unit": "Mpoints*RHS/s", "cores": oracle_threads(), "kind": "oracle",
                             "sample": smp.sample_text()},
            "e2e": {"value": value, "unit": "Mpoints*RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
# roofline arithmetic
# ----------------------------------------------------------------------------------------
ALU_NOTE = "152 SMs x 128 FP32 lanes x median SM clock under load"
FP64_NOTE = "152 SMs x 2 FP64 FMA per clock (4 flops) x median SM clock under load"


def count_launches(info):
    """Kernel launches of one apply (permutes, near field, the far-field stages)."""
    lf = info["lf"]
    n = 3  # permute in, near field, permute out
    if lf >= 2:
        n += 1 + 3 * (lf - 2) + (lf - 1) + 3 * (lf - 2) + 1
    return n


def stage_rooflines(info, stage_ms, n_src, n_tgt, fp32_peak, hbm, fp64_peak=None):
    """Roofline entry of every stage with a defined unit of work (plan summary `info`, live
    stage times in ms); FP32-pipe operations against fp32_peak (Gop/s) for arithmetic-bound
    stages, float64 flops against fp64_peak (Gflop/s) for the float64 plane-wave tables,
    algorithmic bytes against hbm (GB/s) for the re-quadratures."""
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
        if stage in ("s2m", "l2t") and lev.get("precision") == "fp64" and info.get("leaf_tables") and fp64_peak:
            # table-driven float64 plane waves: 4 FMA (8 flops) per (point, antipodal pair, RHS)
            units = float(lev["K"]) / 2 * (n_tgt if stage == "l2t" else n_src) * info.get("nrhs", 1)
            return dict(kernel="k_l2t_tab" if stage == "l2t" else "k_s2m_tab", bound="alu",
                        achieved=8.0 * units / (ms * 1e-3) / 1e9, peak=fp64_peak, unit="Gflop/s",
                        unit_work="8 float64 flops (4 FMA) per (point, antipodal sample pair, RHS)",
                        peak_note=FP64_NOTE)
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


# ----------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------
class Timer:
    """Device-timed applies on one stream with an L2 flush before each."""

    def __init__(self, dev, world):
        import torch
        self.torch = torch
        self.dev = dev
        self.world = world
        self.flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.stream = torch.cuda.current_stream(dev)

    def run(self, fn, steps, warmup):
        torch = self.torch
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier(self.world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            self.flush.fill_(1.0)
            a.record(self.stream)
            fn()
            b.record(self.stream)
        torch.cuda.synchronize()
        barrier(self.world)
        return allmax(float(np.mean([a.elapsed_time(b) for a, b in ev])), self.world)

    def stages(self, plan, fn, reps):
        plan.set_timing(True)
        acc = {k: 0.0 for k in STAGES}
        for _ in range(reps):
            self.flush.fill_(1.0)
            fn()
            self.torch.cuda.synchronize()
            for k, v in plan.info()["stage_ms"].items():
                acc[k] += v / reps
        plan.set_timing(False)
        return acc


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_direct_reference(s, t_sub, q, kappa, dev):
    """Float64 direct sum at a subset of targets by the library's float64 near-field kernel:
    a one-box float64 plan (occupancy bound = all sources) has no far field."""
    import torch
    from paper_0911_4114_gb300 import FmmPlan
    plan = FmmPlan(s, t_sub, kappa, 1e-6, precision="fp64", max_leaf=max(len(s), len(t_sub)))
    assert plan.info()["lf"] < 2
    out = plan.apply(torch.as_tensor(q.astype(np.complex128)).reshape(-1, 1).to(dev))
    torch.cuda.synchronize()
    return out[:, 0].cpu().numpy()


def cube_run(timer, dev, n=524288):
    """The cube workload with 64 right-hand sides (kappa 40, eps 1e-5, tuned plan): time per
    apply, stage times and the tensor-pipe roofline of its tcgen05 near field.  n < 524,288
    takes the first n points of the same cloud (profiling runs)."""
    import torch
    from paper_0911_4114_gb300 import FmmPlan, workloads as wl
    cs, ct = wl.points("cube512k_rhs64", n=n)
    cplan = FmmPlan(cs, ct, 40.0, 1e-5, precision="mixed", max_rhs=64, **AUTO)
    cq = torch.as_tensor(wl.charges(len(cs), 64, wl.rng(3, salt=1)).astype(np.complex64)).to(dev)
    cout = torch.empty((len(ct), 64), dtype=torch.complex64, device=dev)
    cms = timer.run(lambda: cplan.apply(cq, out=cout), 2, 1)
    ci = cplan.info()
    cst = timer.stages(cplan, lambda: cplan.apply(cq, out=cout), 1)
    res = {"ms_per_step": cms, "value": len(ct) * 64 / (cms * 1e-3) / 1e6, "unit": "Mpoints*RHS/s",
           "points": len(ct), "nrhs": 64, "kappa": 40.0, "eps": 1e-5, "lf": ci["lf"], "buffer": ci["buffer"],
           "p2p_pairs": ci["p2p_pairs"], "stage_ms": cst,
           "levels": {str(l): v["precision"] for l, v in ci["levels"].items()}}
    tiles = ci.get("near_mma_tiles", 0)
    if tiles and cst.get("near_field", 0.0) > 0.0:
        # tensor-pipe roofline of the tcgen05 near field: the MMAs it issues (12 of 128 x 128 x 8
        # per chunk-tile pair and 64-RHS pass) against the TF32 peak, and the algorithmic complex
        # multiply-adds (8 flops per pair and RHS) against the same peak
        try:
            bf16 = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
            src = "of measured"
        except (OSError, KeyError):
            bf16, src = 1900.0, "of fallback"
        tf32 = bf16 * 1.1 / 2.25
        sec = cst["near_field"] * 1e-3
        issued = tiles * 12 * 2.0 * 128 * 128 * 8
        algo = ci["p2p_pairs"] * 64 * 8.0
        res["near_field_roofline"] = {
            "kernel": "k_p2p_tc5", "bound": "tensor", "unit": "TFLOP/s", "peak": tf32,
            "peak_note": "TF32: measured bf16 GEMM peak x nominal TF32/bf16 ratio 1.1/2.25", "peak_source": src,
            "achieved": issued / sec / 1e12, "frac": issued / sec / 1e12 / tf32,
            "unit_work": "12 tcgen05.mma kind::tf32 M128 N128 K8 (three split products) per (128-target chunk, "
                         "16-source tile, 64-RHS pass)",
            "algorithmic": {"achieved": algo / sec / 1e12, "frac": algo / sec / 1e12 / tf32,
                            "unit_work": "8 flops per near-field pair and right-hand side"}}
    del cplan, cq, cout
    return res


def adaptive_run(timer, dev, steps):
    """Adaptive octree (HFMM_FLAG_ADAPTIVE, max_leaf 64) against the uniform tree, both with the
    tuned plan shape, mixed policy, eps 1e-4, one right-hand side: the clustered cloud
    (1,048,576 points in 16 dense small cubes plus 10% uniform, kappa 72.5) and the headline
    ellipsoid.  Time per apply, stage times, leaves per level, near-field pairs, boxes, and the
    error against the float64 direct sum on 500 seeded targets."""
    import torch
    from paper_0911_4114_gb300 import FmmPlan, workloads as wl
    out = {}
    for name, kappa in (("clusters1m", 72.5), ("ellipsoid2m", 200.0)):
        s, t = wl.points(name)
        qh = wl.charges(len(s), 0, wl.rng(6, salt=1)).astype(np.complex64)
        q = torch.as_tensor(qh).reshape(-1, 1).to(dev)
        o = torch.empty((len(t), 1), dtype=torch.complex64, device=dev)
        idx = np.sort(np.random.default_rng(20260105).choice(len(t), 500, replace=False))
        ref = gpu_direct_reference(s, t[idx], qh.astype(np.complex128), kappa, dev)
        res = {"points": len(t), "kappa": kappa, "eps": 1e-4, "unit": "Mpoints*RHS/s"}
        for tree in ("uniform", "adaptive"):
            p = FmmPlan(s, t, kappa, 1e-4, precision="mixed", max_leaf=64, adaptive=tree == "adaptive", **AUTO)
            ms = timer.run(lambda: p.apply(q, out=o), max(3, steps // 2), 2)
            err = rel(o[:, 0].cpu().numpy().astype(np.complex128)[idx], ref)
            i = p.info()
            res[tree] = {"ms_per_step": ms, "value": len(t) / (ms * 1e-3) / 1e6, "rel_err": err, "lf": i["lf"],
                         "buffer": i["buffer"], "p2p_pairs": i["p2p_pairs"], "nbox": i["nbox"],
                         "leaves": {str(l): n for l, n in enumerate(i["level_nleaf"]) if n},
                         "stage_ms": timer.stages(p, lambda: p.apply(q, out=o), 1)}
            del p
        out[name] = res
    return out


def extras_run(timer, dev, steps):
    """Device-timed extra workloads: the sphere, the 64-RHS cube and the 32-problem batch."""
    import torch
    from paper_0911_4114_gb300 import FmmBatch, FmmPlan, workloads as wl
    out = {}
    # 262,144 points on the unit sphere, kappa 64, eps 1e-6, mixed and float64
    s, t = wl.points("sphere262k")
    q = torch.as_tensor(wl.charges(len(s), 0, wl.rng(1, salt=1)).astype(np.complex64)).reshape(-1, 1).to(dev)
    o = torch.empty((len(t), 1), dtype=torch.complex64, device=dev)
    sph = {}
    for prec in ("mixed", "fp64"):
        p = FmmPlan(s, t, 64.0, 1e-6, precision=prec, **AUTO)
        ms = timer.run(lambda: p.apply(q, out=o), max(3, steps // 2), 2)
        sph[prec] = {"ms_per_step": ms, "value": len(t) / (ms * 1e-3) / 1e6}
        if prec == "mixed":
            sph["stage_ms"] = timer.stages(p, lambda: p.apply(q, out=o), 3)
            sph["lf"] = p.info()["lf"]
            sph["buffer"] = p.info()["buffer"]
        del p
    out["sphere262k"] = dict(sph, unit="Mpoints*RHS/s", kappa=64.0, eps=1e-6, charges="complex64")
    # 524,288 points in the unit cube, 64 right-hand sides, kappa 40, eps 1e-5
    out["cube512k_rhs64"] = cube_run(timer, dev)
    # 32 uneven cube problems, 4 RHS each, one graph launch per apply
    g = wl.rng(5)
    sizes = np.exp(g.uniform(np.log(8192), np.log(131072), 32)).astype(int)
    kappas = g.uniform(10.0, 60.0, 32)
    probs = [(wl.cube(int(n), g), float(k)) for n, k in zip(sizes, kappas)]
    batch = FmmBatch([(x, x, k, 1e-5) for x, k in probs], precision="mixed", max_rhs=4, **AUTO)
    qs = [torch.as_tensor(wl.charges(len(x), 4, g).astype(np.complex64)).to(dev) for x, _ in probs]
    outs = [torch.empty((len(x), 4), dtype=torch.complex64, device=dev) for x, _ in probs]
    bms = timer.run(lambda: batch.apply(qs, outs), max(3, steps // 2), 2)
    npts = int(sum(len(x) for x, _ in probs))
    out["batch32_rhs4"] = {"ms_per_step": bms, "value": npts * 4 / (bms * 1e-3) / 1e6, "unit": "Mpoints*RHS/s",
                           "problems": 32, "points_total": npts, "nrhs": 4, "eps": 1e-5,
                           "launch": "one cudaGraphLaunch per apply (hfmm_apply_batch replay)"}
    del batch
    # adaptive against uniform trees
    out["adaptive_tree"] = adaptive_run(timer, dev, steps)
    return out


def main():
    args = parse()
    rank, world = dist_setup(args.gpus)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_0911_4114_gb300 import FmmPlan
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    AUTO["buffer"] = args.buffer
    if args.cube_only:
        if rank == 0:
            print(json.dumps(dict(cube_run(Timer(dev, world), dev, args.cube_only), workload="cube_rhs64")))
        return
    if args.adaptive_only:
        if rank == 0:
            print(json.dumps(dict(adaptive_run(Timer(dev, world), dev, args.steps), workload="adaptive_tree")))
        return
    s, t, q_host = headline_points(args.points if args.points != 2097152 else None)
    kappa, eps = HEADLINE["kappa"], HEADLINE["eps"]
    AUTO["buffer"] = args.buffer
    nt = len(t)
    timer = Timer(dev, world)
    q64 = torch.as_tensor(q_host).reshape(-1, 1).to(dev)
    q128 = q64.to(torch.complex128)
    o64 = torch.empty((nt, 1), dtype=torch.complex64, device=dev)
    o128 = torch.empty((nt, 1), dtype=torch.complex128, device=dev)

    t0 = time.perf_counter()
    mp = FmmPlan(s, t, kappa, eps, precision="mixed", **AUTO)
    plan_seconds = time.perf_counter() - t0
    info = mp.info()

    results = {}
    with ClockSampler(local) as clk:
        results["mixed"] = timer.run(lambda: mp.apply(q64, out=o64), args.steps, args.warmup)
        head_out = o64[:, 0].cpu().numpy().astype(np.complex128)
    clocks = clk.summary()
    stage_ms = timer.stages(mp, lambda: mp.apply(q64, out=o64), max(3, args.steps // 4))

    # end to end through the public API: pinned host in, host out
    qh = torch.as_tensor(q_host).reshape(-1, 1).pin_memory()
    ph = torch.empty((nt, 1), dtype=torch.complex64).pin_memory()
    qd = torch.empty_like(qh, device=dev)

    def e2e_step():
        qd.copy_(qh, non_blocking=True)
        mp.apply(qd, out=o64)
        ph.copy_(o64, non_blocking=True)
    e2e_ms = timer.run(e2e_step, args.steps, args.warmup)

    # adjoint of the headline plan
    adj_out = torch.empty((len(s), 1), dtype=torch.complex64, device=dev)
    adj_ms = timer.run(lambda: mp.apply_adjoint(q64, out=adj_out), max(3, args.steps // 4), 1)
    del mp

    # accuracy: float64 direct sum on seeded targets
    idx = np.sort(np.random.default_rng(20260102).choice(nt, min(REL_ERR_TARGETS, nt), replace=False))
    ref = gpu_direct_reference(s, t[idx], q_host, kappa, dev)
    errs = {"mixed": rel(head_out[idx], ref)}

    fp64 = None
    if not args.no_fp64:
        p = FmmPlan(s, t, kappa, eps, precision="fp64", **AUTO)
        ms = timer.run(lambda: p.apply(q64, out=o64), 2, 1)
        errs["fp64"] = rel(o64[:, 0].cpu().numpy().astype(np.complex128)[idx], ref)
        fp64 = {"value": nt / (ms * 1e-3) / 1e6, "ms_per_step": ms, "rel_err": errs["fp64"], "lf": p.info()["lf"],
                "buffer": p.info()["buffer"],
                "stage_ms": timer.stages(p, lambda: p.apply(q64, out=o64), 1)}
        del p

    tight = None
    if not args.no_tight:
        tight = {"eps": TIGHT_EPS, "charges": "complex128 (the complex64 values)"}
        for prec in (("mixed",) if args.no_fp64 else ("mixed", "fp64")):
            p = FmmPlan(s, t, kappa, TIGHT_EPS, precision=prec, **AUTO)
            ms = timer.run(lambda: p.apply(q128, out=o128), 1 if prec == "fp64" else 2, 1)
            got = o128[:, 0].cpu().numpy()[idx]
            tight[prec] = {"value": nt / (ms * 1e-3) / 1e6, "ms_per_step": ms, "rel_err": rel(got, ref),
                           "lf": p.info()["lf"], "buffer": p.info()["buffer"]}
            if prec == "mixed":
                tight[prec]["stage_ms"] = timer.stages(p, lambda: p.apply(q128, out=o128), 1)
            del p

    extras = {"adjoint": {"ms_per_step": adj_ms, "value": len(s) / (adj_ms * 1e-3) / 1e6,
                          "unit": "Mpoints*RHS/s", "workload": "ellipsoid2m, eps 1e-4, mixed"}}
    if not args.no_extras and args.points == 2097152:
        extras.update(extras_run(timer, dev, args.steps))

    # CPU oracle on this host (rank 0 only): FMM at the same plan on a sample, direct-sum sample
    cpu = None
    if rank == 0 and world == 1 and not args.skip_oracle:
        oidx, ovals, osecs = oracle_direct_sample(s, t, q_host.astype(np.complex128), kappa,
                                                  ORACLE_DIRECT_TARGETS, 20260103)
        errs["mixed_vs_oracle_direct"] = rel(head_out[oidx], ovals)
        smp = OracleFmmSampler(s, t, q_host.astype(np.complex128), kappa, eps, buffer=info["buffer"],
                               depth=info["lf"])   # the GPU run's plan shape
        fmm_secs, parts = smp.time_once()
        cpu = {"value": nt / fmm_secs / 1e6, "unit": "Mpoints*RHS/s", "cores": oracle_threads(), "kind": "oracle",
               "sample": smp.sample_text(), "seconds_per_apply_extrapolated": fmm_secs,
               "direct_sum": {"value": ORACLE_DIRECT_TARGETS / osecs / 1e6, "unit": "Mpoints*RHS/s",
                              "sample": f"oracle float64 direct sum over all {len(s):,} sources for "
                                        f"{ORACLE_DIRECT_TARGETS} seeded targets ({osecs:.1f} s)"}}

    # rooflines per stage; the top-level entry is the dominant stage's
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    sm_clock = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * sm_clock * 1e6 / 1e9          # FP32-pipe ops/s (Gop/s)
    fp64_peak = 152 * 4 * sm_clock * 1e6 / 1e9            # float64 flops/s (Gflop/s)
    hbm = peaks.get("hbm_gbs", 6800.0)
    info_r = dict(info, nrhs=1)
    roof_stages = stage_rooflines(info_r, stage_ms, len(s), nt, fp32_peak, hbm, fp64_peak)
    stage = max(stage_ms, key=stage_ms.get)
    roof = dict(roof_stages.get(stage) or {"kernel": stage, "bound": None, "achieved": None, "peak": None,
                                          "unit": None, "frac": None, "stage_ms": stage_ms[stage]})
    # DRAM bytes per launch come from an ncu capture of the current build; none is read here
    roof["traffic"] = None
    roof["peak_source"] = "of measured" if peaks else "of fallback"

    _, value = replica_rate(results["mixed"], nt, world)
    _, e2e_value = replica_rate(e2e_ms, nt, world)
    line = {"metric": METRIC, "value": value, "unit": "Mpoints*RHS/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": results["mixed"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+df+f64", "data": "synthetic",
            "config": dict(HEADLINE, points=nt, parallelism="replicas" if world > 1 else "single",
                           l2="flushed before every timed apply (512 MiB write)",
                           lf=info["lf"], buffer=info["buffer"],
                           levels={str(l): v for l, v in info["levels"].items()},
                           p2p_pairs=info["p2p_pairs"],
                           predicted_ms={f"b{b}_L{l}": round(v, 2) for (b, l), v in info["predicted_ms"].items()}),
            "rel_err": errs["mixed"],
            "rel_err_ref": f"float64 direct sum at {len(idx)} seeded targets (library float64 kernel); "
                           f"mixed_vs_oracle_direct: oracle direct sum at {ORACLE_DIRECT_TARGETS} targets",
            "rel_errs": errs, "fp64_path": fp64, "tight": tight,
            "stage_ms": stage_ms, "plan_seconds": plan_seconds,
            "e2e": {"value": e2e_value, "unit": "Mpoints*RHS/s",
                    "h2d_bytes_per_step": int(qh.numel() * 8), "d2h_bytes_per_step": int(ph.numel() * 8)},
            "roofline": roof,
            "roofline_stages": {k: {kk: v[kk] for kk in ("kernel", "bound", "achieved", "unit", "frac")}
                                for k, v in roof_stages.items()},
            "cpu_baseline": cpu, "gpu_launches": count_launches(info) * args.steps,
            "clocks": clocks, "extras": extras}
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
