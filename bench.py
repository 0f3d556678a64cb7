#!/usr/bin/env python3
"""Benchmark of the MCMCMC step on one GB300.

Workload (default): Gaussian SK spin glass, N = 512, J_ij ~ N(0, 1/N) fp32,
64 disorder instances x 4096 independent chains (262,144 chains), K = 128
single-flip proposals per step, beta = 1 (T = T_c), observables recorded
every 100 steps.  One bench step = 100 Monte Carlo steps of every chain,
one persistent kernel launch over all instances.  The chains' state (spins +
fields, 671 MB) is larger than L2 and is streamed through on every launch.

Metric: candidate configurations per second (chains x K x MC steps / s);
MC steps per second (chain-steps / s) is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs the same workload with its own seeds (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N, INSTANCES, CHAINS, K, BETA, R = 512, 64, 4096, 128, 1.0, 100
WORKLOAD = (f"gaussian-sk N={N} J~N(0,1/N) fp32, {INSTANCES} instances x {CHAINS} chains, "
            f"MCMCMC K={K}, beta={BETA}, record every {R} steps; one bench step = {R} MC steps "
            f"of all chains in one persistent launch")
METRIC = "SK candidate configs/s (MCMCMC K=128, Gaussian N=512, 64x4096 chains)"
UNIT = "candidate configs/s"


def _env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples (every 50 ms) of the SM clock and the throttle
    reasons; stop() keeps the samples taken inside [mark_start(), stop()]."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(gpu_index), "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t0 = time.time()

    def mark_start(self):
        self.t0 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t1 = time.time()
        time.sleep(0.1)  # the sample that covers the region's end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        import datetime
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(p[2]), float(p[3]), p[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 - 0.05 <= r[0] <= t1 + 0.05]
        if not inside and rows:  # no sample inside a short region: the one nearest to it
            inside = [min(rows, key=lambda r: abs(r[0] - 0.5 * (self.t0 + t1)))]
        reasons = set()
        for r in inside:
            for n_, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(n_)
        return {"sm_mhz": statistics.median(r[1] for r in inside) if inside else None,
                "sm_max_mhz": max(r[2] for r in inside) if inside else None,
                "samples": len(inside), "region_s": round(t1 - self.t0, 3), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle timings (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_sample(couplings, chains_per_instance, steps, threads):
    """Runs the FP64 oracle on `chains_per_instance` chains of every instance
    for `steps` steps (records every R), on `threads` host threads."""
    import concurrent.futures as cf

    import oracle
    jobs = []
    for i, J in enumerate(couplings):
        for c0 in range(0, chains_per_instance, 16):
            jobs.append((i, J, c0, min(16, chains_per_instance - c0)))

    def one(job):
        i, J, c0, n = job
        oracle.run(J, K=K, beta=BETA, seed=1, stream=i, chain0=c0, chains=n, steps=steps,
                   record_every=R)

    oracle.lib()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, jobs))
    return time.perf_counter() - t0


def cpu_baseline(couplings):
    cores = _cores()
    per_inst = 512
    steps = R
    dt = _oracle_sample(couplings, per_inst, steps, cores)
    units = INSTANCES * per_inst * steps * K
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{per_inst} chains of each of the {INSTANCES} instances x {steps} steps "
                      f"(records included), FP64 C oracle, {cores} threads, {dt:.2f} s wall"}


def run_reference(args):
    rank, world, _ = _env()
    if rank != 0:
        return 0
    from paper_2102_05613_gb300 import inputs
    couplings = [inputs.couplings_gauss(N, i) for i in range(INSTANCES)]
    cores = _cores()
    per_inst = 32
    for _ in range(args.warmup):
        _oracle_sample(couplings, per_inst, R, cores)
    times = [_oracle_sample(couplings, per_inst, R, cores) for _ in range(args.steps)]
    T = sum(times)
    units = INSTANCES * per_inst * R * K * args.steps
    value = units / T
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "reference_sample":
                                            f"{per_inst} chains per instance per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{per_inst} chains of each of the {INSTANCES} instances x "
                                       f"{R} steps per bench step, {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# tensor-core field recompute (H = J s for all chains), config-3 sizes
# ---------------------------------------------------------------------------
RC_N, RC_CHAINS, RC_ITERS = 2048, 8192, 20


def recompute_report(stream, peaks, fp8_measured=None, own_mma=None):
    """Times mcmcmc_recompute on +-J (FP8 e4m3, check) and Gaussian (bf16 x3,
    resync) couplings with N = 2048 and 8192 chains, and states the error of
    each recompute format against the FP64 product on 64 chains."""
    import numpy as np
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    bf16_peak = peaks.get("bf16_tflops") or 1900.0
    out = {"N": RC_N, "chains": RC_CHAINS,
           "flops_per_recompute": 2.0 * RC_CHAINS * RC_N * RC_N}
    for kind, name in ((sk.SK_J_PM1, "pm1_fp8"), (sk.SK_J_GAUSS, "gauss_bf16x3")):
        J = inputs.couplings(RC_N, kind, 2048 + kind)
        inst = sk.Instance(J, stream=stream)
        # config 3's run: a recompute every 256 steps (the step kernel keeps
        # the spins' tensor-core operands, so the call converts nothing)
        run = sk.Run(inst, chains=RC_CHAINS, K=64, beta=2.0, seed=5, recompute_every=256)
        run.advance(256)
        mode = sk.SK_RECOMPUTE_CHECK if kind == sk.SK_J_PM1 else sk.SK_RECOMPUTE_RESYNC
        for _ in range(3):
            run.recompute(mode, terms=3)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(RC_ITERS)]
        for a, b in ev:
            a.record(stream)
            run.recompute(mode, terms=3, sync=False)
            b.record(stream)
        torch.cuda.synchronize()
        st, _ = run.recompute(mode, terms=3)
        ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        # executed flops: one product for FP8, three (one per bf16 term) for the split
        exec_flops = out["flops_per_recompute"] * (1 if kind == sk.SK_J_PM1 else 3)
        if kind == sk.SK_J_PM1:
            peak = fp8_measured or bf16_peak * 2.0
            src = ("measured this run: cuBLASLt e4m3 GEMM 8192^3" if fp8_measured
                   else "measured bf16 x 2 (nominal fp8/bf16 ratio)")
        else:
            peak, src = bf16_peak, "measured bf16 (MEASURED_PEAKS.json)"
        ent = {"ms": ms, "algorithmic_tflops": out["flops_per_recompute"] / ms / 1e9,
               "executed_tflops": exec_flops / ms / 1e9, "peak_tflops": peak, "peak_source": src,
               "frac_executed": exec_flops / ms / 1e9 / peak,
               "check": st}
        own = (own_mma or {}).get("own_mma_fp8_tflops" if kind == sk.SK_J_PM1 else "own_mma_bf16_tflops")
        if own:  # against the kernel's own MMA loop with nothing else to do
            ent["own_mma_tflops"] = own
            ent["frac_of_own_mma"] = exec_flops / ms / 1e9 / own
        # error of each format against the FP64 product on the first 64 chains
        spins, _ = run.state()
        ex = (J.astype(np.float64) @ spins[:64].T.astype(np.float64)).T
        errs = {}
        for terms in ((1,) if kind == sk.SK_J_PM1 else (1, 2, 3)):
            _, H = run.recompute(terms=terms, out=True)
            errs[f"terms={terms}" if kind == sk.SK_J_GAUSS else "fp8"] = float(
                np.abs(H[:64].astype(np.float64) - ex).max())
        ent["max_abs_error_vs_fp64"] = errs
        out[name] = ent
        run.close()
        inst.close()
    return out


# ---------------------------------------------------------------------------
# single-chain latency: +-J N = 64 (J seed 0), K = 8, beta = 1, 1e5 steps
# ---------------------------------------------------------------------------
def dependent_shuffles(G, wide, K=8):
    """Warp-collective rounds on one MCMCMC step's critical path with G lanes
    per chain (the few-chain variant): the broadcast of site a, the group
    minimum (one redux), the inclusive scan of the slot weights (64-bit +-J
    weights move as two shuffles issued together), the total's broadcast, the
    ballot(s) of the lanes past the draw and the broadcast of the chosen slot.
    Whole-warp chains with K <= 32 hold one slot per lane (slot d = lane + 1,
    two ballots: past the draw, positive weight) and their +-J scan covers the
    lanes that hold slots (8 for K <= 8, 32 for K <= 32); otherwise four slots
    per lane and a log2 G level scan.  The shuffles that hand out the next
    step's sites from the batch do not wait on the step and are not counted."""
    one_slot = G == 32 and K <= 32
    lanes = (8 if K <= 8 else 32) if (one_slot and wide) else G
    lg = int(math.log2(lanes))
    return {"shuffle_rounds": 1 + lg + 1 + 1, "redux": 1, "ballot": 2 if one_slot else 1,
            "shuffle_instructions": 1 + lg * (2 if wide else 1) + (2 if wide else 1) + 1}


def latency_report(stream):
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    J = inputs.couplings_pm1(64, 0)
    inst = sk.Instance(J, stream=stream)
    steps = 100_000
    run = sk.Run(inst, chains=1, K=8, beta=1.0, seed=1, record_every=1000, max_records=steps // 1000)
    run.advance(1000)
    run.reset()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    run.advance(steps)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    batch = sk.Batch([run])
    layout = batch.classes()[0]
    batch.close()
    run.close()
    inst.close()
    return {"workload": "+-J SK N=64, J seed 0, one chain, MCMCMC K=8, beta=1, 1e5 steps, Philox seed 1",
            "ns_per_step": 1e6 * ms / steps, "candidate_configs_per_s": 8 * steps / (ms / 1e3),
            "layout": {"lanes_per_chain": layout[1], "warps_per_cta": layout[3]},
            "dependent_collectives_per_step": dependent_shuffles(layout[1], True, 8)}


def _one_chain_ns(batch, stream, steps=20000):
    """Best of 3 timed launches of `steps` steps (CUDA events), ns per step."""
    import torch
    batch.advance(500)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        batch.advance(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, 1e6 * e0.elapsed_time(e1) / steps)
    return best


LATENCY_CLUSTERS = {64: (1, 2, 4), 512: (8, 16), 1024: ()}


def run_latency(args):
    """One-chain step times (the latency regime): config 1 and Gaussian
    instances of N = 1024 (the thermalisation runs) and N = 512 (whose columns
    of J fit a cluster's shared memory) at several K, and Metropolis; default
    layouts, autotuned ones and forced cluster-per-chain layouts, best of 3
    timed launches."""
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    out = {"config1": latency_report(stream)}
    # config 1 in the cluster layouts
    inst = sk.Instance(inputs.couplings_pm1(64, 0), stream=stream)
    for C in LATENCY_CLUSTERS[64]:
        run = sk.Run(inst, chains=1, K=8, beta=1.0, seed=1)
        b = sk.Batch([run])
        b.set_cluster(C)
        out["config1"][f"cluster{C}_ns_per_step"] = _one_chain_ns(b, stream)
        b.close()
        run.close()
    inst.close()
    for N in (1024, 512):
        key = f"gauss_n{N}_one_chain"
        out[key] = {}
        inst = sk.Instance(inputs.couplings_gauss(N, 0), stream=stream)
        for name, rule, Kt in (("metropolis", 1, 1), ("mcmcmc_k8", 0, 8), ("mcmcmc_k32", 0, 32),
                               ("mcmcmc_k128", 0, 128)):
            res = {}
            for mode in ("default", "autotuned") + tuple(f"cluster{C}" for C in LATENCY_CLUSTERS[N]):
                run = sk.Run(inst, chains=1, K=Kt, rule=rule, beta=TTT_BETA, seed=1)
                b = sk.Batch([run])
                if mode == "autotuned":
                    b.autotune(trial_steps=512)
                elif mode.startswith("cluster"):
                    b.set_cluster(int(mode[7:]))
                res[mode] = {"ns_per_step": _one_chain_ns(b, stream), "layout": b.classes()[0]}
                b.close()
                run.close()
            out[key][name] = res
        inst.close()
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# set-generation probabilities (App. D): every subset of n = 24 elements
# ---------------------------------------------------------------------------
def setgen_report(stream, n=24):
    import numpy as np
    import torch
    from paper_2102_05613_gb300 import sk
    rng = np.random.default_rng(0)
    P = rng.random((n, n))
    np.fill_diagonal(P, 0.0)
    P /= 1.5 * P.sum(axis=0, keepdims=True)
    out = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    res = {"workload": f"generation probabilities of all 2^{n} subsets, random P_gen, double precision"}
    for name, method in (("direct", sk.SK_SETGEN_DIRECT), ("cumulative", sk.SK_SETGEN_CUMULATIVE)):
        sk.set_generation(P, out=out, stream=stream, method=method)  # warm-up
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        sk.set_generation(P, out=out, stream=stream, method=method)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        res[name] = {"ms": ms, "subsets_per_s": (1 << n) / (ms / 1e3)}
    # terms of the direct recursion: for each mask M, |M| x |S minus M| parent
    # sums; the cumulative form does |M| per mask
    res["direct"]["terms_per_s"] = sum(math.comb(n, m) * m * (n - m) for m in range(1, n)) / (res["direct"]["ms"] / 1e3)
    res["cumulative"]["terms_per_s"] = sum(math.comb(n, m) * m for m in range(1, n)) / (res["cumulative"]["ms"] / 1e3)
    return res


# ---------------------------------------------------------------------------
# time to thermalise: MCMCMC vs K = 1 Metropolis (Gaussian N = 1024; beta = 1 by
# default, the paper's T = T_c; --ttt-beta for colder or hotter runs)
# ---------------------------------------------------------------------------
TTT_N, TTT_CHAINS, TTT_BETA = 1024, 4096, 1.0
# name, rule, K, steps, graph (the graphs of Fig. fig_sk: the 2^7 line, the
# binary tree of depth 7, the ternary of depth 5, the 16-ary of depth 3)
TTT_METHODS = [("metropolis", 1, 1, 1 << 23, {}),
               ("mcmcmc_k2", 0, 2, 1 << 23, {}), ("mcmcmc_k4", 0, 4, 1 << 22, {}),
               ("mcmcmc_k8", 0, 8, 1 << 22, {}), ("mcmcmc_k16", 0, 16, 1 << 21, {}),
               ("mcmcmc_k32", 0, 32, 1 << 21, {}), ("mcmcmc_k128", 0, 128, 1 << 20, {}),
               # the root distribution of the star (App. B.2 leaves p_r free): the centre
               # as the root with probability p_center, each leaf with (1 - p_center)/K
               ("mcmcmc_k32_pc0.5", 0, 32, 1 << 21, dict(p_center=0.5)),
               ("mcmcmc_k32_pc0.05", 0, 32, 1 << 21, dict(p_center=0.05)),
               ("mcmcmc_k128_pc0.5", 0, 128, 1 << 20, dict(p_center=0.5)),
               ("mcmcmc_k128_pc0.05", 0, 128, 1 << 20, dict(p_center=0.05)),
               ("line_128", 0, 1, 1 << 16, dict(graph=2, line_nodes=128)),
               ("tree2_d7", 0, 1, 1 << 15, dict(graph=1, arity=2, depth=7)),
               ("tree3_d5", 0, 1, 1 << 14, dict(graph=1, arity=3, depth=5)),
               ("tree16_d3", 0, 1, 1 << 13, dict(graph=1, arity=16, depth=3))]
# the default bench line: Metropolis against the star at every K of the sweep
TTT_LINE_METHODS = ("metropolis", "mcmcmc_k2", "mcmcmc_k4", "mcmcmc_k8", "mcmcmc_k16", "mcmcmc_k32",
                    "mcmcmc_k128")
TTT_EPS = (1e-2, 3e-3, 1e-3)


def ttt_measure(only, beta, scale, N=TTT_N):
    """e(t) = chain-mean E/N every T/2048 steps from a random start; e_inf and
    sigma_inf (one record's equilibrium fluctuation) from the last half of the
    K=128 run; t_therm(eps) = the first record after which
    |e - e_inf| <= eps + 3 sigma_inf holds for good; wall-clock = t_therm x
    the method's measured seconds per step (4096 chains, autotuned layout), and
    the same for 1 and 152 chains (few_chains)."""
    import numpy as np
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    stream = torch.cuda.current_stream()
    J = inputs.couplings_gauss(N, 0)
    inst = sk.Instance(J, stream=stream)
    curves = {}
    for name, rule, Kt, T, gkw in TTT_METHODS:
        if only and name not in only and name != "mcmcmc_k128":
            continue
        T *= scale
        R = T // 2048
        run = sk.Run(inst, chains=TTT_CHAINS, K=Kt, rule=rule, beta=beta, seed=7,
                     record_every=R, max_records=2048, **gkw)
        # each method runs with its own autotuned launch geometry (lanes per
        # chain, chains per CTA); tuning leaves the chains untouched
        batch = sk.Batch([run])
        batch.autotune(trial_steps=64)
        geometry = batch.classes()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        chunk = R * 128
        for _ in range(T // chunk):
            batch.advance(chunk)
        b.record(stream)
        torch.cuda.synchronize()
        batch.close()
        E, _, acc = run.observables()
        s_per_step = a.elapsed_time(b) / 1e3 / T
        curves[name] = dict(R=R, T=T, e=E.mean(axis=1) / N, per_chain=E / N,
                            s_per_step=s_per_step, acc=float(acc.mean()) / R, geometry=geometry,
                            nodes=Kt + 1 if not gkw.get("graph") else (gkw.get("line_nodes") or
                                                                       (gkw["arity"] ** (gkw["depth"] + 1) - 1) // (gkw["arity"] - 1)))
        run.close()
    # e_inf: mean of the last half of the K=128 run's records; sigma: the
    # equilibrium fluctuation of one record (its chain mean) over that half,
    # which is the noise the per-record criterion below has to tolerate
    ref = curves["mcmcmc_k128"]
    tail = ref["e"][1024:]
    e_inf = float(tail.mean())
    sig = float(tail.std(ddof=1))
    out = {"workload": f"gaussian-sk N={N} J seed 0, beta={beta}, {TTT_CHAINS} chains from "
                       f"a random start, records every T/2048 steps",
           "e_inf": e_inf, "sigma_inf": sig, "methods": {}}
    for name, c in curves.items():
        t = (np.arange(len(c["e"])) + 1) * c["R"]
        dev = np.abs(c["e"] - e_inf)
        m = {"steps_run": c["T"], "graph_nodes": c["nodes"], "s_per_step": c["s_per_step"],
             "launch_classes": c["geometry"],
             "chain_steps_per_s": TTT_CHAINS / c["s_per_step"], "acceptance": c["acc"],
             "e_final": float(c["e"][-1]), "t_therm_steps": {}, "t_therm_s": {}}
        for eps in TTT_EPS:
            ok = dev <= eps + 3 * sig
            bad = np.nonzero(~ok)[0]
            if len(bad) == 0:
                ts = int(t[0])
            elif bad[-1] + 1 < len(t):
                ts = int(t[bad[-1] + 1])
            else:
                ts = None  # not thermalised within the run
            m["t_therm_steps"][str(eps)] = ts
            m["t_therm_s"][str(eps)] = None if ts is None else ts * c["s_per_step"]
        out["methods"][name] = m
    sp, ss = {}, {}
    met = out["methods"].get("metropolis")
    for name, mm in out["methods"].items():
        if name == "metropolis" or met is None:
            continue
        sp[name], ss[name] = {}, {}
        for eps in TTT_EPS:
            a_, b_ = met["t_therm_s"][str(eps)], mm["t_therm_s"][str(eps)]
            sa, sb = met["t_therm_steps"][str(eps)], mm["t_therm_steps"][str(eps)]
            if b_ is None:
                sp[name][str(eps)] = ss[name][str(eps)] = None
            elif a_ is None:
                sp[name][str(eps)] = f">{met['steps_run'] * met['s_per_step'] / b_:.3g} (Metropolis not thermalised)"
                ss[name][str(eps)] = f">{met['steps_run'] / sb:.3g}"
            else:
                sp[name][str(eps)] = a_ / b_
                ss[name][str(eps)] = sa / sb
    out["wallclock_speedup_vs_metropolis"] = sp
    out["mc_step_ratio_vs_metropolis"] = ss
    out["few_chains"] = ttt_few_chains(inst, out["methods"], only, beta)
    # the best MCMCMC variant at each chain count and accuracy (wall-clock)
    best = {}
    for label, table in [(str(TTT_CHAINS), sp)] + [(c, v["wallclock_speedup_vs_metropolis"])
                                                    for c, v in out["few_chains"].items()]:
        best[label] = {}
        for eps in TTT_EPS:
            cand = [(v[str(eps)], n) for n, v in table.items() if isinstance(v.get(str(eps)), float)]
            best[label][str(eps)] = None if not cand else {"method": max(cand)[1], "speedup": max(cand)[0]}
    out["best_wallclock_speedup_vs_metropolis"] = best
    inst.close()
    return out


def run_ttt(args):
    import torch
    torch.cuda.set_device(0)
    only = set(args.ttt_methods.split(",")) if args.ttt_methods else None
    print(json.dumps(ttt_measure(only, args.ttt_beta, args.ttt_scale, args.ttt_n)), flush=True)
    return 0


TTT_FEW_CHAINS = (1, 152)


def run_cluster_one_chain(args):
    """One Gaussian N = 512 chain, K = 32, beta = 1, on clusters of
    --cluster-one-chain CTAs (the layout the autotuner picks for it): a warm-up
    launch, then 2000 steps in one launch, CUDA events."""
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    inst = sk.Instance(inputs.couplings_gauss(512, 0), stream=stream)
    run = sk.Run(inst, chains=1, K=32, beta=1.0, seed=1)
    b = sk.Batch([run])
    b.set_cluster(args.cluster_one_chain)
    b.advance(200)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    b.advance(2000)
    e1.record(stream)
    torch.cuda.synchronize()
    out = {"workload": "Gaussian SK N=512, one chain, K=32, beta=1", "ctas_per_cluster": args.cluster_one_chain,
           "ns_per_step": 1e6 * e0.elapsed_time(e1) / 2000, "launch_classes": b.classes()}
    b.close()
    run.close()
    inst.close()
    print(json.dumps(out), flush=True)
    return 0


def run_graph_one_chain(args):
    """The binary tree of depth 7 (Gaussian N = 1024, beta = 1), 500 steps in
    one launch: with one chain (8 warps per chain) the graph kernel's
    latency case, with --graph-chains C its throughput case (the layout given
    by --warps-per-cta / --lanes, else autotuned); the cases its ncu captures
    use."""
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    C = args.graph_chains
    inst = sk.Instance(inputs.couplings_gauss(TTT_N, 0), stream=stream)
    run = sk.Run(inst, chains=C, K=1, beta=TTT_BETA, seed=7, graph=sk.SK_GRAPH_TREE, arity=2, depth=7)
    if C == 1:
        batch = sk.Batch([run], warps_per_cta=16)  # 8 warps per chain, two chains' room per CTA
        batch.set_layout(lanes=256)
    elif args.warps_per_cta:
        batch = sk.Batch([run], warps_per_cta=args.warps_per_cta)
        batch.set_layout(lanes=args.lanes or 32)
    else:
        batch = sk.Batch([run])
        batch.autotune(trial_steps=20)
    if C > 1:
        batch.advance(20)  # warm-up launch (the one-chain case times its first launch)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    batch.advance(500)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    out = {"workload": f"binary tree depth 7 (255 nodes), Gaussian SK N=1024, {C} chain(s)",
           "us_per_step": 1e3 * ms / 500, "chain_steps_per_s": C * 500 / (ms / 1e3),
           "launch_classes": batch.classes()}
    batch.close()
    run.close()
    inst.close()
    print(json.dumps(out), flush=True)
    return 0


def ttt_few_chains(inst, methods, only, beta):
    """Time to thermalise when only a few chains run (one chain, or one per
    SM), where a Metropolis step cannot fill the GPU and the graph's nodes
    are what runs in parallel: seconds per step of each method at C chains
    (autotuned launch geometry, no records), times the steps to thermalise of
    the ensemble above (the ensemble mean relaxes the same way whatever the
    number of chains; only the time per step depends on it)."""
    import torch
    from paper_2102_05613_gb300 import sk
    stream = torch.cuda.current_stream()
    res = {}
    for C in TTT_FEW_CHAINS:
        per = {}
        for name, rule, Kt, _T, gkw in TTT_METHODS:
            if name not in methods or (only and name not in only and name != "mcmcmc_k128"):
                continue
            run = sk.Run(inst, chains=C, K=Kt, rule=rule, beta=beta, seed=11, **gkw)
            batch = sk.Batch([run])
            # trials long enough that the launch's fixed cost does not decide
            # between layouts a few per cent apart
            batch.autotune(trial_steps=32 if gkw.get("graph") else 512)
            geometry = batch.classes()

            def timed(T):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                batch.advance(T)
                b.record(stream)
                torch.cuda.synchronize()
                return a.elapsed_time(b) / 1e3

            timed(16)
            t64 = timed(64)
            T = int(min(1 << 20, max(64, 64 * 0.25 / max(t64, 1e-9))))  # ~0.25 s of steps
            s_per_step = timed(T) / T
            batch.close()
            run.close()
            m = methods[name]
            per[name] = {"s_per_step": s_per_step, "steps_timed": T, "launch_classes": geometry,
                         "t_therm_s": {e: (None if st_ is None else st_ * s_per_step)
                                       for e, st_ in m["t_therm_steps"].items()}}
        sp = {}
        met = per.get("metropolis")
        for name, mm in per.items():
            if name == "metropolis" or met is None:
                continue
            sp[name] = {e: (None if (mm["t_therm_s"][e] is None or met["t_therm_s"][e] is None)
                            else met["t_therm_s"][e] / mm["t_therm_s"][e]) for e in mm["t_therm_s"]}
        res[str(C)] = {"methods": per, "wallclock_speedup_vs_metropolis": sp}
    return res


# ---------------------------------------------------------------------------
# uneven batch: 256 instances of N in 128..4096 (half +-J, half Gaussian),
# 256..2048 chains, K in 16..256, beta in [0.5, 3]; autotuned, CUDA graphs
# ---------------------------------------------------------------------------
def run_uneven(args):
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    torch.cuda.set_device(0)
    st = torch.cuda.Stream()
    specs = inputs.uneven_batch(args.uneven_instances, seed=0)
    g = torch.Generator(device="cuda")
    insts, runs = [], []
    with torch.cuda.stream(st):
        for i, sp in enumerate(specs):
            N = sp["N"]
            g.manual_seed(sp["jseed"])
            if sp["kind"] == sk.SK_J_PM1:
                J = (2 * torch.randint(0, 2, (N, N), generator=g, device="cuda") - 1).to(torch.int8)
            else:
                J = torch.randn((N, N), generator=g, device="cuda") / math.sqrt(N)
            J = torch.triu(J, 1)
            J = (J + J.T).contiguous()
            insts.append(sk.Instance(J, stream=st))
            runs.append(sk.Run(insts[-1], chains=sp["chains"], K=sp["K"], beta=sp["beta"], seed=3,
                               stream_id=i, record_every=R, max_records=args.warmup + args.steps + 2))
    torch.cuda.synchronize()
    # --uneven-warps W: one CTA shape for every class (whole-warp chains, rows
    # through L1, W warps per CTA) instead of the autotuner's per-class choice,
    # the shape a single kernel for all classes would have to fix
    # --uneven-fused W: every run in one persistent launch of W-warp CTAs
    W = args.uneven_warps
    batch = sk.Batch(runs, warps_per_cta=W)
    t0 = time.perf_counter()
    if args.uneven_fused:
        batch.set_fused(args.uneven_fused)
    elif W:
        batch.set_layout(32, 2)
    else:
        batch.autotune(trial_steps=10)
    tune_s = time.perf_counter() - t0
    batch.capture(R)
    batch.replay(args.warmup)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(0)
    for a, b in ev:
        a.record(st)
        batch.replay(1)
        b.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    T = ev[0][0].elapsed_time(ev[-1][1]) / 1e3
    cand = sum(sp["chains"] * sp["K"] for sp in specs) * R * args.steps
    cs = sum(sp["chains"] for sp in specs) * R * args.steps
    out = {"config": "uneven batch", "workload": f"{len(specs)} SK instances, N uniform in 128..4096 (even: +-J "
           "int8, odd: Gaussian fp32), 256..2048 chains, K uniform in 16..256, beta uniform in "
           "[0.5, 3], MCMCMC; one CUDA graph = 100 steps of every chain (launches: see layout and "
           "classes)", "metric": UNIT, "value": cand / T, "mc_steps_per_s": cs / T,
           "ms_per_step": 1e3 * T / args.steps, "steps": args.steps, "warmup": args.warmup,
           "layout": (f"one persistent launch for every run: 32 lanes per chain, rows through L1, "
                      f"{args.uneven_fused} warps per CTA" if args.uneven_fused else
                      f"one shape for every class: 32 lanes per chain, rows through L1, {W} warps per CTA"
                      if W else "autotuned per class"),
           "autotune_s": tune_s, "classes": batch.classes(), "clocks": clk,
           "chains_total": sum(sp["chains"] for sp in specs)}
    batch.close()
    for r in runs:
        r.close()
    for x in insts:
        x.close()
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# serving: Poisson arrivals of sampling jobs into the request server
# ---------------------------------------------------------------------------
def _serve_once(rate, duration, pool, budget, quantum, seed):
    import numpy as np
    from paper_2102_05613_gb300 import inputs, sk
    srv = sk.Server(budget_bytes=budget, quantum_steps=quantum)
    for cid, (N, kind, J) in pool.items():
        srv.add_couplings(cid, J)
    jobs = inputs.poisson_jobs(rate, duration, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    ids = list(pool.keys())
    tickets = []
    t0 = time.perf_counter()
    for k, jb in enumerate(jobs):
        cid = ids[int(rng.integers(0, len(ids)))]
        N, kind, _ = pool[cid]
        delay = jb["t_arrive"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        rule = sk.SK_RULE_METROPOLIS if jb["K"] == 1 else sk.SK_RULE_MCMCMC
        tk = srv.submit(N=N, kind=kind, chains=jb["chains"], steps=jb["steps"], K=jb["K"], rule=rule,
                        beta=jb["beta"], seed=jb["seed"], stream_id=k & 0xFFFFFF, couplings_id=cid)
        tickets.append((tk, jb, N))
    submit_s = time.perf_counter() - t0
    srv.wait_all()
    st = [srv.poll(t) for t, _, _ in tickets]
    lat = np.array([x["t_done"] - x["t_submit"] for x in st if x["state"] == sk.SK_JOB_DONE])
    wait = np.array([x["t_admit"] - x["t_submit"] for x in st if x["state"] == sk.SK_JOB_DONE])
    done = [x for x in st if x["state"] == sk.SK_JOB_DONE]
    cand = sum(jb["chains"] * jb["steps"] * jb["K"] for (t, jb, N), x in zip(tickets, st)
               if x["state"] == sk.SK_JOB_DONE)
    offered = sum(jb["chains"] * jb["steps"] * jb["K"] for _, jb, _ in tickets)
    span = max(x["t_done"] for x in done) - min(x["t_submit"] for x in st) if done else float("nan")
    sstat = srv.stats()
    srv.close()
    return {"rate_per_s": rate, "arrival_window_s": duration, "jobs": len(jobs),
            "completed": len(done), "failed": len(st) - len(done),
            "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "queue_wait_p50_s": float(np.percentile(wait, 50)) if len(wait) else None,
            "throughput_candidates_per_s": cand / span, "span_s": span, "submit_s": submit_s,
            "offered_candidates_per_s": offered / duration,
            # saturated: the backlog outlives the arrival window by more than half of it
            "saturated": span > 1.5 * duration,
            "device_busy_s": sstat["busy_seconds"], "quanta": sstat["quanta"],
            "host_admit_s": sstat["admit_seconds"], "host_retire_s": sstat["retire_seconds"],
            "host_plan_s": sstat["plan_seconds"]}


def run_serve(args):
    import numpy as np
    import torch
    from paper_2102_05613_gb300 import inputs, sk
    torch.cuda.set_device(0)
    # 12 disorder instances, N log-uniform in [64, 8192], half +-J / half Gaussian,
    # registered once; each job samples one of them
    rng = np.random.Generator(np.random.PCG64(11))
    pool = {}
    for i in range(12):
        N = int(round(math.exp(rng.uniform(math.log(64), math.log(8192)))))
        kind = i % 2
        pool[i + 1] = (N, kind, inputs.couplings(N, kind, 7000 + i))
    budget = 100 << 30
    res = [_serve_once(args.serve_rate, args.serve_window, pool, budget, 256, seed=1),
           _serve_once(args.serve_low_rate, args.serve_window, pool, budget, 256, seed=2)]
    out = {"config": "serving", "workload": "Poisson arrivals of SK sampling jobs; each job: one of 12 "
           "registered instances (N log-uniform in [64, 8192], +-J or Gaussian), beta U[0.3, 3], K in "
           "{1 (Metropolis), 16, 64, 256}, steps log-uniform [1e3, 1e5], chains log-uniform [1, 4096]; "
           "server: 100 GiB budget, 256-step quanta", "runs": res}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------------------
# measured ceilings: L2 and shared-memory bandwidth (the library's probes,
# sk_peaks.h) and the FP8 tensor-core rate (a cuBLASLt FP8 GEMM, timed the
# way the driver times the bf16 one), each best of several launches
# ---------------------------------------------------------------------------
def measure_peaks(stream):
    import torch
    from paper_2102_05613_gb300 import sk
    out = {}
    out["l2_read_gbps"] = max(sk.peak_l2_read(48 << 20, passes=64, reps=3, stream=stream) for _ in range(3))
    out["smem_vec16_gbps"] = max(sk.peak_smem(sk.SK_PEAK_SMEM_VEC16, iters=1024, reps=3, stream=stream)
                                 for _ in range(3))
    out["smem_gather4_gbps"] = max(sk.peak_smem(sk.SK_PEAK_SMEM_GATHER4, iters=1024, reps=3, stream=stream)
                                   for _ in range(3))
    out["how"] = ("L2: 48 MiB resident working set, 16-byte ld.global.cg loads, 4 CTAs x 512 threads "
                  "per SM, 64 sweeps per launch; shared memory: 64 KiB per CTA, 2 CTAs x 1024 threads "
                  "per SM, 16 loads in flight per thread, conflict-free 16-byte loads (a warp reads 512 "
                  "contiguous bytes) and random 4-byte gathers (useful bytes); best of 3 x 3 launches, "
                  "CUDA events")
    try:
        M = 8192
        a = torch.randn(M, M, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(M, M, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out["fp8_tflops"] = 2.0 * M ** 3 / (best * 1e-3) / 1e12
        out["fp8_how"] = "torch._scaled_mm e4m3 8192^3 (cuBLASLt), best of 10, CUDA events"
        del a, b
    except Exception as e:  # noqa: BLE001 -- reported, and the nominal ratio is used instead
        out["fp8_tflops"] = None
        out["fp8_how"] = f"unavailable ({type(e).__name__}: {e})"
    # the recompute kernel's own MMA loop with its operand ring filled once (no
    # epilogue, no operand traffic): what its tcgen05 issue reaches at best
    out["own_mma_fp8_tflops"] = max(sk.peak_tensor(sk.SK_J_PM1, tiles=64, reps=3, stream=stream) for _ in range(3))
    out["own_mma_bf16_tflops"] = max(sk.peak_tensor(sk.SK_J_GAUSS, tiles=64, reps=3, stream=stream)
                                     for _ in range(3))
    out["own_mma_how"] = ("sk_peak_tensor: the recompute kernel, one CTA per SM, 64 tiles of 128 x 256 per CTA "
                          "(K = 2048 e4m3 / 1024 bf16) issued over a 4-stage ring loaded once; best of 3 x 3 "
                          "launches, CUDA events")
    return out


# ---------------------------------------------------------------------------
# BASELINE config 2 in full: beta in {0.5, 1, 2, 3} x K in {1 (Metropolis),
# 32, 128}, 64 instances x 4096 chains, 1e4 steps, records every 100
# ---------------------------------------------------------------------------
SWEEP_BETAS, SWEEP_KS, SWEEP_STEPS = (0.5, 1.0, 2.0, 3.0), (1, 32, 128), 10_000


def config2_sweep(stream, insts):
    import torch
    from paper_2102_05613_gb300 import sk
    res = []
    for Kc in SWEEP_KS:
        rule = sk.SK_RULE_METROPOLIS if Kc == 1 else sk.SK_RULE_MCMCMC
        geometry = None
        for beta in SWEEP_BETAS:
            runs = [sk.Run(inst, chains=CHAINS, K=Kc, rule=rule, beta=beta, seed=3, stream_id=i,
                           record_every=R, max_records=SWEEP_STEPS // R) for i, inst in enumerate(insts)]
            if geometry is None:
                batch = sk.Batch(runs)
                batch.autotune(trial_steps=10)
                geometry = batch.classes()
            else:  # the layout tuned at the first beta (it does not depend on beta)
                batch = sk.Batch(runs, warps_per_cta=geometry[0][3])
                batch.set_layout(geometry[0][1], 1 if (geometry[0][0] >> 5) & 3 == 1 else 2)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(SWEEP_STEPS // R):
                batch.advance(R)
            b.record(stream)
            torch.cuda.synchronize()
            s_ = a.elapsed_time(b) / 1e3
            E, _, acc = runs[0].observables()
            cs = len(insts) * CHAINS * SWEEP_STEPS
            res.append({"rule": "metropolis" if Kc == 1 else "mcmcmc", "K": Kc, "beta": beta,
                        "seconds": s_, "mc_steps_per_s": cs / s_, "candidate_configs_per_s": cs * Kc / s_,
                        "acceptance": float(acc[-10:].mean()) / R,
                        "e_final_instance0": float(E[-1].mean()) / N, "launch_classes": geometry})
            batch.close()
            for r_ in runs:
                r_.close()
    return {"workload": f"gaussian-sk N={N}, {len(insts)} instances x {CHAINS} chains, {SWEEP_STEPS} steps "
                        f"from the Philox random start, records every {R} steps; Metropolis is K = 1",
            "runs": res}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    global INSTANCES, CHAINS, WORKLOAD
    if (args.instances, args.chains) != (INSTANCES, CHAINS):
        WORKLOAD = WORKLOAD.replace(f"{INSTANCES} instances x {CHAINS} chains",
                                    f"{args.instances} instances x {args.chains} chains")
        INSTANCES, CHAINS = args.instances, args.chains
    rank, world, local = _env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2102_05613_gb300 import inputs, replicas, sk
    stream = torch.cuda.current_stream()
    seed_base = replicas.seed_base(rank)
    couplings = [inputs.couplings_gauss(N, seed_base + i) for i in range(INSTANCES)]
    cap = args.warmup + args.steps + args.e2e_steps + 2
    insts = [sk.Instance(J, stream=stream) for J in couplings]
    runs = [sk.Run(inst, chains=CHAINS, K=K, beta=BETA, seed=1 + rank, stream_id=i,
                   record_every=R, max_records=cap) for i, inst in enumerate(insts)]
    batch = sk.Batch(runs, warps_per_cta=args.warps_per_cta)
    if args.lanes or args.staging:
        batch.set_layout(args.lanes, args.staging)
    elif not args.warps_per_cta:
        batch.autotune(trial_steps=10)  # launch geometry only; the chains are untouched
    info = batch.info()
    info["classes"] = batch.classes()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    clocks = Clocks(local)  # sampling from before the warm-up; stop() keeps the timed region's samples
    for _ in range(args.warmup):
        batch.advance(R)
    barrier()
    c0 = [r.counters() for r in runs]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    clocks.mark_start()
    for s, e in ev:
        s.record(stream)
        batch.advance(R)
        e.record(stream)
    barrier()
    clk = clocks.stop()
    for r in runs:
        r.wait()
    c1 = [r.counters() for r in runs]
    total_ms = ev[0][0].elapsed_time(ev[-1][1])
    launch_ms = [s.elapsed_time(e) for s, e in ev]
    T = replicas.max_over_ranks(total_ms / 1e3, dist, device="cuda")
    chain_steps_rank = INSTANCES * CHAINS * R * args.steps
    value = world * chain_steps_rank * K / T
    mc_steps = world * chain_steps_rank / T

    # Roofline of the step kernel (the batched step is bound by the memory
    # level that holds J and the chains' state).  Algorithmic bytes of one
    # chain-step, from the kernel's counters (r = J rows the steps needed, f =
    # spins flipped per step):
    #   J rows               r N b_J          (from L2, through L1)
    #   proposal gathers     K (b_s + b_h)    (shared memory)
    #   field update         2 f N b_h        (shared-memory read-modify-write)
    # All three pass the SM's L1 / shared-memory data path: their sum against
    # the measured conflict-free shared-memory bandwidth is the headline
    # fraction; the J-row bytes against the measured L2 read bandwidth and the
    # lane-operation count against the ALU peak are reported beside it.
    flips = sum(b[0] - a[0] for a, b in zip(c0, c1))
    rows = sum(b[1] - a[1] for a, b in zip(c0, c1))
    cs = INSTANCES * CHAINS * R * args.steps
    rows_ps, flips_ps = rows / cs, flips / cs
    bJ, bs, bh = 4, 1, 4
    bytes_J = rows_ps * N * bJ
    bytes_gather = K * (bs + bh)
    bytes_update = 2 * flips_ps * N * bh
    bytes_ps = bytes_J + bytes_gather + bytes_update
    mean_launch_s = statistics.mean(launch_ms) / 1e3
    cs_launch = INSTANCES * CHAINS * R
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    mp = measure_peaks(stream) if rank == 0 else {}
    sm_clock = peaks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # DRAM bytes of one launch: ncu capture of the 16-instance case at the
    # profiled layout, scaled by the chains processed (the state streamed once
    # per launch grows in proportion); null for any other layout
    profiled = [268, 16, 3072, 24]
    traffic = (4 * 296.8e6 * INSTANCES / 64 if N == 512 and info["classes"]
               and list(info["classes"][0][:4]) == profiled else None)
    smem_peak = mp.get("smem_vec16_gbps")
    achieved = bytes_ps * cs_launch / mean_launch_s / 1e9
    roofline = {"bound": "smem", "achieved": achieved, "peak": smem_peak, "unit": "GB/s",
                "frac": (achieved / smem_peak) if smem_peak else None, "traffic": traffic,
                "peak_source": "measured this run: conflict-free 16-byte shared-memory loads (sk_peak_smem)",
                "kernel": "step_kernel", "mean_launch_ms": 1e3 * mean_launch_s,
                "chain_steps_per_launch": cs_launch,
                "bytes_per_chain_step": bytes_ps,
                "terms": {"J_rows_r_N_bJ": bytes_J, "gathers_K_bs_bh": bytes_gather,
                          "field_update_2fN_bh": bytes_update},
                "J_rows_per_chain_step": rows_ps, "flips_per_chain_step": flips_ps}
    l2_peak = mp.get("l2_read_gbps")
    l2_ach = bytes_J * cs_launch / mean_launch_s / 1e9
    roofline["l2"] = {"achieved": l2_ach, "peak": l2_peak, "unit": "GB/s",
                      "frac": (l2_ach / l2_peak) if l2_peak else None, "bytes_per_chain_step": bytes_J,
                      "peak_source": "measured this run: 48 MiB resident, ld.global.cg (sk_peak_l2_read)"}
    g4 = mp.get("smem_gather4_gbps")
    g_ach = bytes_gather * cs_launch / mean_launch_s / 1e9
    roofline["gathers_vs_random_gather_peak"] = {
        "achieved": g_ach, "peak": g4, "unit": "GB/s", "frac": (g_ach / g4) if g4 else None,
        "note": "the proposal gathers alone against random 4-byte shared-memory gathers"}
    # lane operations (MCMCMC): Philox (ceil(K/4) + 1/32) blocks x 84 (10 rounds
    # x 8 ops + 4 range reductions), candidate energies 4 K, min + weights
    # 4 (K + 1), prefix + choice 2 (K + 1), field update f N, against 152 SMs x
    # 128 lanes x the maximum SM clock
    ops_ps = (math.ceil(K / 4) + 1 / 32) * 84 + 4 * K + 6 * (K + 1) + flips_ps * N
    alu_peak = sms * 128 * sm_clock * 1e6 / 1e12
    alu_ach = ops_ps * cs_launch / mean_launch_s / 1e12
    roofline["alu"] = {"achieved": alu_ach, "peak": alu_peak, "unit": "Tops/s", "frac": alu_ach / alu_peak,
                       "ops_per_chain_step": ops_ps,
                       "peak_source": f"{sms} SMs x 128 lanes x {sm_clock:.0f} MHz"}

    # end to end through the C ABI from pinned host buffers: upload the 64
    # coupling matrices and the 262,144 start configurations, run 100 steps,
    # read the step's records back.  Two sets of instances and runs (the same
    # workload, the same launch geometry) on two streams take the steps in
    # turn, so that one step's input copies and device checks overlap the
    # other set's compute; every step's copies and its records' read-back are
    # inside the timed region.
    e2e = None
    if args.e2e_steps > 0:
        hJ = [torch.from_numpy(J).pin_memory() for J in couplings]
        hS = [torch.from_numpy(inputs.initial_spins(CHAINS, N, seed_base + 77 + i)).pin_memory()
              for i in range(INSTANCES)]
        st2 = torch.cuda.Stream()
        insts2 = [sk.Instance(J, stream=st2) for J in couplings]
        runs2 = [sk.Run(inst, chains=CHAINS, K=K, beta=BETA, seed=1 + rank, stream_id=i,
                        record_every=R, max_records=cap) for i, inst in enumerate(insts2)]
        cls0 = info["classes"][0]
        batch2 = sk.Batch(runs2, warps_per_cta=cls0[3])
        batch2.set_layout(cls0[1], 1 if (cls0[0] >> 5) & 3 == 1 else 2)
        sets = []
        for ii, rr, bb in ((insts, runs, batch), (insts2, runs2, batch2)):
            outs = [(torch.empty((1, CHAINS), dtype=torch.float64).pin_memory(),
                     torch.empty((1, CHAINS // 2), dtype=torch.float64).pin_memory(),
                     torch.empty((1, CHAINS), dtype=torch.int32).pin_memory()) for _ in rr]
            sets.append((ii, rr, bb, outs))

        def e2e_issue(x):
            # the batched entry points: every instance's (run's) copy and check
            # enqueued, one wait for all checks, then the new state and the steps
            sk.set_couplings_many(x[0], hJ)
            sk.reset_many(x[1], hS)
            x[2].advance(R)

        def e2e_read(x):
            sk.observables_many(x[1], 0, 1, x[3])

        for x in sets:  # untimed: first-use staging buffers of both sets
            e2e_issue(x)
            e2e_read(x)
        barrier()
        t0 = time.perf_counter()
        prev = None
        for i in range(args.e2e_steps):
            x = sets[i % 2]
            e2e_issue(x)
            if prev is not None:
                e2e_read(prev)
            prev = x
        e2e_read(prev)
        barrier()
        te = replicas.max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
        h2d = sum(x.numel() * x.element_size() for x in hJ + hS)
        d2h = sum(t.numel() * t.element_size() for o in sets[0][3] for t in o)
        e2e = {"value": world * INSTANCES * CHAINS * R * K * args.e2e_steps / te, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "steps": args.e2e_steps, "ms_per_step": 1e3 * te / args.e2e_steps,
               "pipelined": "two run sets on two streams take the steps in turn"}
        batch2.close()
        for r in runs2:
            r.close()
        for i_ in insts2:
            i_.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(couplings)
    rc = None
    if rank == 0 and not args.no_recompute:
        rc = recompute_report(stream, peaks, mp.get("fp8_tflops"), mp)
    lat = latency_report(stream) if rank == 0 else None
    sg = setgen_report(stream) if rank == 0 else None
    sweep = config2_sweep(stream, insts) if (rank == 0 and not args.no_sweep) else None

    batch.close()
    for r in runs:
        r.close()
    for i in insts:
        i.close()
    ttt = ttt_measure(set(TTT_LINE_METHODS), TTT_BETA, 1) if (rank == 0 and not args.no_ttt) else None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "N": N, "instances": INSTANCES, "chains": CHAINS,
                           "K": K, "beta": BETA, "mc_steps_per_bench_step": R,
                           "l2": f"state ({INSTANCES * CHAINS * N * 5 / 1e6:.0f} MB) larger than L2, "
                                 "streamed every launch",
                           "launch": info},
                "mc_steps_per_s": mc_steps,
                "gpu_launches": 2 * args.steps,
                "roofline": roofline, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
                "recompute": rc, "latency_config1": lat, "set_generation": sg,
                "peaks_measured": mp, "time_to_thermalise": ttt, "config2_sweep": sweep}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=12)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--config", choices=["default", "uneven"], default="default",
                    help="uneven: the 256-instance uneven batch in CUDA graphs instead of the bench line")
    ap.add_argument("--serve", action="store_true", help="the request-server measurement")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-low-rate", type=float, default=10.0)
    ap.add_argument("--serve-window", type=float, default=5.0)
    ap.add_argument("--ttt-methods", default="",
                    help="comma-separated subset of the --ttt methods (the K=128 reference always runs)")
    ap.add_argument("--ttt-beta", type=float, default=TTT_BETA,
                    help="inverse temperature of the --ttt comparison (1 = T_c, the paper's setting)")
    ap.add_argument("--uneven-warps", type=int, default=0,
                    help="--config uneven: one CTA shape for every class (this many warps, 32 lanes per "
                         "chain) instead of the autotuned per-class layouts")
    ap.add_argument("--uneven-instances", type=int, default=256,
                    help="--config uneven: instances (256 = BASELINE config 4; fewer for profiler captures)")
    ap.add_argument("--cluster-one-chain", type=int, default=0,
                    help="one Gaussian N=512 chain, K=32, on clusters of this many CTAs: 2000 steps in one "
                         "launch after a warm-up launch (the cluster kernel's profiler case)")
    ap.add_argument("--uneven-fused", type=int, default=0,
                    help="--config uneven: every run in one persistent launch of this many warps per CTA")
    ap.add_argument("--ttt-n", type=int, default=TTT_N,
                    help="spins of the --ttt instance (512: its columns of J fit a cluster's shared memory)")
    ap.add_argument("--ttt-scale", type=int, default=1,
                    help="multiplies every --ttt method's steps (colder runs relax more slowly)")
    ap.add_argument("--graph-chains", type=int, default=1,
                    help="chains of the --graph-one-chain case (1: the latency case)")
    ap.add_argument("--graph-one-chain", action="store_true",
                    help="the graph kernel's single-chain latency case (binary tree, depth 7)")
    ap.add_argument("--latency", action="store_true",
                    help="one-chain step times (config 1, Gaussian N=1024 at several K, Metropolis)")
    ap.add_argument("--ttt", action="store_true",
                    help="time-to-thermalise comparison instead of the throughput line")
    ap.add_argument("--no-recompute", action="store_true",
                    help="skip the tensor-core recompute measurement")
    ap.add_argument("--no-ttt", action="store_true",
                    help="skip the time-to-thermalise comparison in the bench line")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the beta x K sweep of the full workload in the bench line")
    ap.add_argument("--instances", type=int, default=INSTANCES,
                    help="smaller cases for profiling only; the bench line uses the default")
    ap.add_argument("--chains", type=int, default=CHAINS)
    ap.add_argument("--warps-per-cta", type=int, default=0,
                    help="warps per CTA (no autotuning); 0 = autotuned")
    ap.add_argument("--lanes", type=int, default=0, help="lanes per chain (no autotuning)")
    ap.add_argument("--staging", type=int, default=0,
                    help="1 TMA-staged rows, 2 rows through L1 (no autotuning)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.ttt:
        return run_ttt(args)
    if args.latency:
        return run_latency(args)
    if args.graph_one_chain:
        return run_graph_one_chain(args)
    if args.config == "uneven":
        return run_uneven(args)
    if args.cluster_one_chain:
        return run_cluster_one_chain(args)
    if args.serve:
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
