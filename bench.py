#!/usr/bin/env python
"""Benchmark: KBE time steps per second of the GB300 stepper.

One bench "step" is one full propagation of the workload: every KBE time
step T = k+1 .. N_t-1 (extrapolation, self-energy, retarded row, mixed,
lesser column, density matrix, self-consistency loop per step), for every
instance of the batch, starting from the bootstrapped state (the bootstrap is
set-up, outside the timed region, as in the paper's timings).

  value     = instances x (N_t - k - 1) / (device seconds of one propagation),
              summed over ranks (each rank propagates its own instances)
  e2e       = the same metric through the public C ABI with HOST buffers:
              upload eps(t), G^M, propagate, download the density matrix
  roofline  = the dominant kernel's algorithmic bytes / its device time
  cpu_baseline = the FP64 oracle on the host cores, on a bounded sample

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import kbe_workloads as wk  # noqa: E402

WORKLOADS = {
    "C1": dict(desc="Bethe lattice, Sigma=v^2 G (v=1), beta=5, N_t=256, h=0.025, order 5, "
                    "DLR Lambda=100 eps=1e-10, undriven, dense FP64",
               make=lambda seed: wk.c1_workload(seed=seed), n_inst=1),
    "C2": dict(desc="Bethe lattice, beta=5, N_t=4096, h=0.02, order 5, level quench eps0 0->1 at t=5, "
                    "HODLR leaf 64, SVD tol 1e-8, complex128",
               make=lambda seed: wk.c2_workload(seed=seed), n_inst=1),
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def batch_inputs(spec, n_inst, rank):
    ws = [spec["make"](seed=rank * n_inst + i) for i in range(n_inst)]
    w = ws[0]
    eps = np.concatenate([x["eps"] for x in ws])
    gm = np.concatenate([x["gm"] for x in ws])
    mp = np.concatenate([x["model_params"] for x in ws])
    return w, eps, gm, mp


def hodlr_bytes(phase, T, c, no, r, L, blocks, ranks_sr, ranks_sl):
    """Unique bytes a phase must move at step T in the HODLR form: the
    uncompressed rows [c, T], the compressed leaves below c, and the stored
    factors (U rows below c, V, rank columns) of every block, per orbital pair."""
    e = 16 * no * no
    direct = sum(s + 1 for s in range(c, T + 1)) * e
    leaves = (c // L) * (L * (L + 1) // 2) * e
    row = (T + 1) * e

    def factors(ranks):
        tot = 0
        for b in range(len(blocks["r0"])):
            r0, r1, c0, c1 = blocks["r0"][b], blocks["r1"][b], blocks["c0"][b], blocks["c1"][b]
            if r0 >= c:
                continue
            rows = min(r1, c) - r0
            tot += int(sum((rows + (c1 - c0)) * int(rk) for rk in ranks[b])) * 16
        return tot
    if phase in ("ret", "les"):
        return direct + leaves + factors(ranks_sr) + 2 * row
    if phase == "src":
        return direct + leaves + factors(ranks_sl) + 2 * row + (T + 1) * r * e
    if phase == "mixed":
        return row + (T + 1) * r * e
    return 0


def algorithmic_bytes(phase, T, no, r, nt_dense=True):
    """Unique bytes a phase must move at step T for one instance (FP64
    complex = 16 B per element; dense lower-triangular storage)."""
    e = 16 * no * no
    tri = (T + 1) * (T + 2) // 2
    row = (T + 1) * e
    if phase in ("ret", "les"):
        return tri * e + 2 * row            # Sigma^R triangle + row in/out
    if phase == "src":
        return tri * e + row + (T + 1) * r * e + row   # Sigma^< triangle, G^R row, Sigma^tv, q
    if phase == "mixed":
        return row + (T + 1) * r * e + r * r * e + 2 * r * e
    return 0


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(",") for ln in self.f if ln.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) >= 9:
                for i, nm in enumerate(names):
                    if r[5 + i].strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def oracle_sample(spec, seconds=15.0, seed=0):
    """Time the FP64 oracle stepping on the host for about `seconds`."""
    from oracle.kbe import from_workload
    w = spec["make"](seed=seed)
    o = from_workload(w)
    o.bootstrap()
    k, nt = w["wl"].k, w["wl"].nt
    t0 = time.perf_counter()
    steps = 0
    for T in range(k + 1, nt):
        o.step(T)
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return steps / dt, steps, dt, T


def run_reference(args, spec, wname):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_rep = []
    for rep in range(args.warmup + args.steps):
        v, steps, dt, Tlast = oracle_sample(spec, seconds=args.ref_seconds, seed=0)
        if rep >= args.warmup:
            per_rep.append((v, steps, dt, Tlast))
    val = statistics.median(p[0] for p in per_rep)
    steps, dt, Tlast = per_rep[0][1:]
    sample = (f"oracle (numpy FP64, dense) on {wname}: bootstrap, then time steps k+1..{Tlast} "
              f"({steps} steps, {dt:.1f} s) per rep; median of {args.steps} reps after {args.warmup} warm-up")
    line = {"impl": "reference", "metric": "KBE time steps/s", "value": val, "unit": "time steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "desc": spec["desc"]},
            "cpu_baseline": {"value": val, "unit": "time steps/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "time steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="C1", choices=sorted(WORKLOADS))
    ap.add_argument("--n-inst", type=int, default=None, help="instances per GPU (default: the workload's)")
    ap.add_argument("--ref-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, spec, args.workload)

    import torch
    import paper_2604_05319_gb300 as pk

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n_inst = args.n_inst or spec["n_inst"]
    w, eps, gm, mp = batch_inputs(spec, n_inst, rank)
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=wl.nao, n_inst=n_inst, rho_mode=wl.rho_mode,
                    max_iter=wl.max_iter, tol=wl.tol, svd_tol=wl.svd_tol, leaf=wl.leaf, r_max=64)
    mid, _ = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], gm, eps, mid, mp)
    st.bootstrap()
    nsteps = wl.nt - 1 - wl.k
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def propagate():
        pk.hkbe_rewind(st.h)
        st.step(nsteps)

    for _ in range(args.warmup):
        propagate()
    # profiling pass (untimed): per-phase device time and launches; in the
    # HODLR form the ranks are sampled every leaf of steps for the byte count
    pk.hkbe_reset_counters(st.h)
    pk.hkbe_set_profiling(st.h, True)
    pk.hkbe_rewind(st.h)
    hod = wl.svd_tol > 0
    seg_info = []
    its = []
    T = wl.k
    blocks = pk.hkbe_get_blocks(st.h) if hod else None
    while T < wl.nt - 1:
        nseg = min(wl.leaf if hod else nsteps, wl.nt - 1 - T)
        it_seg, _ = st.step(nseg)
        its.append(it_seg)
        if hod:
            nb = len(blocks["r0"])
            rs, c = pk.hkbe_get_ranks(st.h, 0, 2, nb, wl.nao)
            rl, _ = pk.hkbe_get_ranks(st.h, 0, 3, nb, wl.nao)
            seg_info.append((T + 1, T + nseg, c, rs, rl))
        T += nseg
    pk.hkbe_set_profiling(st.h, False)
    prof = st.timing()
    iters = np.concatenate(its)  # (nsteps, n_inst)
    # timed region
    sampler = ClockSampler(local)
    pk.hkbe_reset_counters(st.h)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        pk.hkbe_rewind(st.h)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        st.step(nsteps)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b) / 1e3)
    clocks = sampler.stop()
    launches = sum(v[1] for v in st.timing().values())
    if dist:
        dist.barrier()
    t_step = statistics.mean(times)
    # e2e through the public API with host buffers
    eps_h = np.ascontiguousarray(eps)
    gm_h = np.ascontiguousarray(gm)
    e2e_times = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pk.hkbe_set_hamiltonian(st.h, eps_h)
        pk.hkbe_set_matsubara(st.h, gm_h)
        pk.hkbe_rewind(st.h)
        st.step(nsteps)
        rho = st.density()
        e2e_times.append(time.perf_counter() - t0)
    t_e2e = statistics.mean(e2e_times)
    h2d = eps_h.nbytes + gm_h.nbytes
    d2h = rho.nbytes
    tt = torch.tensor([t_step, t_e2e], device="cuda", dtype=torch.float64)
    if dist:
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    t_step, t_e2e = tt.tolist()
    units = n_inst * nsteps * world
    value = units / t_step
    # roofline of the dominant kernel (from the profiling pass)
    dom = max(("ret", "les", "src", "mixed"), key=lambda p: prof[p][0])
    nb = 0
    if not hod:
        for s_idx, T in enumerate(range(wl.k + 1, wl.nt)):
            nb += int(iters[s_idx].sum()) * algorithmic_bytes(dom, T, wl.nao, len(w["tau"]))
    else:
        for (Ta, Tb, c, rs, rl) in seg_info:
            for T in range(Ta, Tb + 1):
                cT = min(c, max(0, (T - wl.k) // wl.leaf * wl.leaf))
                nb += int(iters[T - wl.k - 1].sum()) * hodlr_bytes(dom, T, cT, wl.nao, len(w["tau"]), wl.leaf,
                                                                 blocks, rs, rl)
    achieved = nb / (prof[dom][0] / 1e3) / 1e9
    peak, peak_kind = peaks()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, steps, dt, Tlast = oracle_sample(spec, seconds=15.0)
        cpu = {"value": v, "unit": "time steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{args.workload} instance 0: time steps k+1..{Tlast} ({steps} steps, {dt:.1f} s), "
                         f"numpy FP64 dense oracle, single thread"}
    if rank == 0:
        tot = sum(v[0] for v in prof.values())
        line = {
            "metric": "KBE time steps/s", "value": value, "unit": "time steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "n_inst_per_gpu": n_inst,
                       "storage": f"HODLR leaf {wl.leaf}, svd_tol {wl.svd_tol}" if hod else "dense",
                       "nt": wl.nt, "h": wl.h, "k": wl.k, "time_steps_per_propagation": nsteps,
                       "mean_iterations_per_time_step": float(iters.mean()),
                       "l2": "256 MB buffer written between timed propagations"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None},
            "phase_share": {k2: round(v[0] / tot, 4) for k2, v in prof.items() if v[0] > 0},
            "cpu_baseline": cpu,
            "e2e": {"value": units / t_e2e, "unit": "time steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line))
    st.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
