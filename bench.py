#!/usr/bin/env python
"""Benchmark: KBE time steps per second of the GB300 stepper, batched.

One bench "step" is one KBE time step T of the whole batch: extrapolation,
self-energy, retarded row, mixed, lesser source and column, density matrix,
the self-consistency loop, and the HODLR compression of that step, for every
instance.  The run bootstraps, propagates untimed to N_t - 1 - 2K, then
  e2e window   : K steps through the public C ABI with host buffers: eps(T)
                 of every instance uploaded from pinned memory, one step,
                 rho(T) of every instance downloaded into pinned memory;
  timed window : the last K steps (the most expensive ones), inputs resident
                 in HBM, CUDA events on the library's stream.
  value        = instances x K / seconds of the timed window (summed over ranks)
  roofline     = the dominant history kernel's algorithmic bytes / its device time
  cpu_baseline = the FP64 oracle on the host cores, on a bounded sample

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload C2-batch|C2|C1] [--n-inst B] [--precision mixed|fp64]
"""
from __future__ import annotations

import os

# The CPU baseline is the single-threaded oracle: keep numpy's BLAS on one
# thread (the GPU arm uses numpy only to build its inputs).
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import kbe_workloads as wk  # noqa: E402

def _batch_c2(n_inst, seed=0, nt=4096):
    """C2 (Bethe, quench eps0 0 -> 1 at t=5, N_t=4096, h=0.02, HODLR leaf 64,
    eps_SVD 1e-8) for a batch: instance 0 is C2 itself, instance i > 0 takes
    its quench amplitude from U[0.5, 1.5] (numpy default_rng(seed))."""
    w = wk.c2_workload(nt=nt, n_inst=n_inst)
    amp = np.concatenate([[1.0], np.random.default_rng(seed).uniform(0.5, 1.5, size=n_inst - 1)])
    w["eps"][:, 1:, 0, 0] *= amp[:, None]
    return w


def _batch_c4(n_inst, seed=0, nt=8192):
    """C4-shaped batch: Nambu Bethe DMFT with the Holstein-Migdal term (g=0.5,
    w0=0.6), beta=50, N_t=8192, h=0.01, pulse A(t) = A0 sin(t) exp(-(t-20)^2/50)
    with A0 = 0.3 for instance 0 and A0 ~ 0.3 U[0.5, 1.5] for the others,
    HODLR leaf 64, eps_SVD 1e-7.  Initial state: the normal non-interacting
    Bethe lattice (closed-form G^M), not the coupled superconducting
    equilibrium (no Matsubara solver here)."""
    w = wk.nambu_workload(nt=nt, h=0.01, k=5, beta=50.0, n_inst=n_inst, v=1.0, eps0=0.0, A0=0.3, Omega=1.0,
                          tc=20.0, width=50.0, g=0.5, w0=0.6, dlr_lambda=200.0, dlr_eps=1e-10)
    amp = np.concatenate([[1.0], np.random.default_rng(seed).uniform(0.5, 1.5, size=n_inst - 1)])
    w["drive_A"] = w["drive_A"] * amp[:, None]
    w["wl"].svd_tol = 1e-7
    return w


WORKLOADS = {
    "C4-batch": dict(desc="C4-shaped: Nambu Bethe-lattice DMFT, hybridisation with Peierls phases + Holstein-Migdal "
                          "(g=0.5, w0=0.6), beta=50, N_t=8192, h=0.01, order 5, DLR Lambda=200 eps=1e-10, pulse "
                          "A(t)=A0 sin(t) exp(-(t-20)^2/50) (A0=0.3 instance 0, 0.3 U[0.5,1.5] others), HODLR "
                          "leaf 64, eps_SVD 1e-7, normal non-interacting initial state",
                     make=_batch_c4, n_inst=76, precision="mixed"),
    "C2-batch": dict(desc="Bethe lattice (Sigma=v^2 G, v=1), beta=5, N_t=4096, h=0.02, order 5, DLR Lambda=100 "
                          "eps=1e-10, level quench 0 -> A at t=5 (A=1 for instance 0, U[0.5,1.5] for the others), "
                          "HODLR leaf 64, eps_SVD 1e-8, r_max 64",
                     make=_batch_c2, n_inst=304, precision="mixed"),
    "C2": dict(desc="C2: Bethe lattice, beta=5, N_t=4096, h=0.02, order 5, quench eps0 0->1 at t=5, "
                    "HODLR leaf 64, eps_SVD 1e-8, one instance",
               make=lambda n_inst, seed=0: wk.c2_workload(n_inst=n_inst), n_inst=1, precision="fp64"),
    "C3": dict(desc="C3-shaped: 2D Hubbard second Born on a 16 x 16 k-grid (256 coupled instances), J=1, "
                    "half filling, beta=10, N_t=2048, h=0.02, order 5, interaction quenched 0 -> U=2 at t=0 "
                    "(the free lattice as initial state), undriven, HODLR leaf 64, eps_SVD 1e-6",
               make=lambda n_inst, seed=0: wk.lattice_workload(L=16, nt=2048, h=0.02, k=5, beta=10.0, U=2.0,
                                                                t_quench=0.0, svd_tol=1e-6, leaf=64),
               n_inst=256, precision="mixed"),
    "C1": dict(desc="C1: Bethe lattice, beta=5, N_t=256, h=0.025, order 5, undriven, dense storage",
               make=lambda n_inst, seed=0: wk.c1_workload(seed=seed, n_inst=n_inst), n_inst=1, precision="fp64"),
}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def phase_bytes(phase, T, c, nfroz, no, r, L, k, es, blocks, ranks):
    """Algorithmic bytes one launch of `phase` moves at step T for one
    instance: every stored element it needs, read once.  es = bytes per
    element of the two-time storage (rows, leaves, factors, band: 16
    complex128, 8 complex64); chunk inverses, the row being solved (FP64
    buffer), projections and mixed components are complex128 in both forms.
      ret / les: Sigma^R uncompressed rows [c, T], leaf triangles below c,
                 built factor rows of U and V times rank, band (k per row),
                 frozen chunk inverses, the solved row (r/w) and its storage;
      src:       the same for Sigma^< plus the G^R row, Sigma^tv and q(t)."""
    n2 = no * no
    direct = sum(s + 1 for s in range(c, T + 1)) * n2 * es if c <= T else 0
    leaves = (c // L) * (L * (L + 1) // 2) * n2 * es
    fac = 0
    if blocks is not None:
        for b in range(len(blocks["r0"])):
            r0, r1, c0, c1 = (int(blocks[x][b]) for x in ("r0", "r1", "c0", "c1"))
            if r0 >= c:
                continue
            fac += ((min(r1, c) - r0) + (c1 - c0)) * int(np.sum(ranks[b])) * es
    band = c * k * n2 * es if blocks is not None else 0
    row = (T + 1) * n2
    if phase in ("ret", "les"):
        return int(direct + leaves + fac + band + nfroz * (32 * no) ** 2 * 16 + row * (32 + es))
    if phase == "src":
        return int(direct + leaves + fac + band + row * es + (T + 1) * r * n2 * 16 + row * 16)
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
    """Time the FP64 oracle stepping instance 0 of the workload on the host
    for about `seconds` (from the bootstrap: the early, cheapest steps).  For
    the lattice the sample is all k-points (they are coupled), on a grid of
    64 time steps; the rate is counted in instance time steps."""
    w = spec["make"](n_inst=1, seed=seed)
    if w["wl"].model == "lattice2b":
        from oracle.lattice import LatticeOracle
        wl = w["wl"]
        nts = 64
        o = LatticeOracle(w["L"], nts, wl.h, wl.k, wl.beta, w["eps"][:, :nts + 1], w["gm"], w["tau"], w["omega"],
                          w["drive_U"][0][:nts + 1], tol=wl.tol)
        o.bootstrap()
        t0 = time.perf_counter()
        steps, T = 0, wl.k
        for T in range(wl.k + 1, nts):
            o.step(T)
            steps += 1
            if time.perf_counter() - t0 > seconds:
                break
        dt = time.perf_counter() - t0
        return steps * len(o.orcs) / dt, steps, dt, T
    from oracle.kbe import from_workload
    o = from_workload(w)
    o.bootstrap()
    k, nt = w["wl"].k, w["wl"].nt
    t0 = time.perf_counter()
    steps, T = 0, k
    for T in range(k + 1, nt):
        o.step(T)
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return steps / dt, steps, dt, T


def rank_seed(rank):
    """Seed of a rank's instances: every rank propagates its own batch
    (weak scaling; the instances need no data-path communication)."""
    return 1000 * rank


def max_over_ranks(values, dist, device):
    """Wall times of the timed regions, reduced to their maximum over ranks
    (the job ends when its slowest rank does)."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


METRIC = "KBE time steps/s"
UNIT = "instance time steps/s"


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
    sample = (f"oracle (numpy FP64, dense, one thread) on instance 0 of {wname}: bootstrap, then time steps "
              f"k+1..{Tlast} ({steps} steps, {dt:.1f} s) per rep; median of {args.steps} reps after "
              f"{args.warmup} warm-up reps")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "desc": spec["desc"]},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=128, help="time steps per timed window")
    ap.add_argument("--warmup", type=int, default=3, help="minimum untimed time steps before the windows")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="C2-batch", choices=sorted(WORKLOADS))
    ap.add_argument("--n-inst", type=int, default=None, help="instances per GPU (default: the workload's)")
    ap.add_argument("--precision", default=None, choices=["mixed", "fp64"])
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
    if args.workload == "C3" and n_inst != 256:
        raise SystemExit("C3 has one instance per k-point of its 16 x 16 grid: --n-inst must be 256")
    prec_name = args.precision or spec["precision"]
    prec = pk.PREC_MIXED if prec_name == "mixed" else pk.PREC_FP64
    w = spec["make"](n_inst=n_inst, seed=rank_seed(rank))   # each rank its own instances
    wl = w["wl"]
    nt, k, no, r = wl.nt, wl.k, wl.nao, len(w["tau"])
    hod = wl.svd_tol > 0
    K = max(1, min(args.steps, (nt - 1 - k - args.warmup) // 2))
    T0 = nt - 1 - 2 * K                      # the untimed propagation ends here
    tol = 1e-7 if prec == pk.PREC_MIXED else wl.tol
    st = pk.Stepper(nt, wl.h, k, wl.beta, nao=no, n_inst=n_inst, rho_mode=wl.rho_mode,
                    max_iter=wl.max_iter, tol=tol, precision=prec, svd_tol=wl.svd_tol, leaf=wl.leaf, r_max=64)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    if "drive_U" in w:
        pk.hkbe_set_drive(st.h, w["drive_A"], w["drive_U"])
    st.bootstrap()
    # ---- untimed propagation (at least `warmup` time steps) ----
    t_prop0 = time.perf_counter()
    st.step(T0 - k)
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t_prop0
    resident = pk.hkbe_get_stats(st.h)
    # ---- e2e window: per step, eps(T) host -> device from pinned memory, one
    # time step, rho(T) device -> host into pinned memory, all through the C ABI
    n2 = no * no
    eps_pin = torch.empty((K, n_inst, n2 * 2), dtype=torch.float64).pin_memory()
    eps_pin.copy_(torch.from_numpy(np.ascontiguousarray(
        w["eps"][:, T0 + 2:T0 + 2 + K].transpose(1, 0, 2, 3)).view(np.float64).reshape(K, n_inst, n2 * 2)))
    rho_pin = torch.empty((K, n_inst, n2 * 2), dtype=torch.float64).pin_memory()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j in range(K):
        T = T0 + 1 + j
        pk.hkbe_set_hamiltonian_at(st.h, T, eps_pin[j].data_ptr())
        st.step(1)
        pk.hkbe_get_density_at(st.h, T, rho_pin[j].data_ptr())
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    h2d = n_inst * n2 * 16
    d2h = n_inst * n2 * 16
    # ---- device-timed window: the last K time steps, inputs resident ----
    blocks = pk.hkbe_get_blocks(st.h) if hod else None
    nb = len(blocks["r0"]) if hod else 0
    ranks0 = [pk.hkbe_get_ranks(st.h, i, X, nb, no)[0] for i in range(n_inst) for X in (2, 3)] if hod else None
    pk.hkbe_reset_counters(st.h)
    pk.hkbe_set_profiling(st.h, True)
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.cudart().cudaProfilerStart()   # a profiler started with --profile-from-start off sees this window only
    ev_a.record()
    iters, _ = st.step(K)
    ev_b.record()
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    clocks = sampler.stop()
    t_win = ev_a.elapsed_time(ev_b) / 1e3
    pk.hkbe_set_profiling(st.h, False)
    prof = st.timing()
    launches = sum(v[1] for v in prof.values())
    t_win, t_e2e = max_over_ranks([t_win, t_e2e], dist, "cuda")
    units = n_inst * K * world
    value = units / t_win
    # ---- roofline of the dominant history kernel over the window ----
    dom = max(("ret", "les", "src"), key=lambda p: prof[p][0])
    es = 8 if prec == pk.PREC_MIXED else 16
    nbytes = 0
    for j in range(K):
        T = T0 + K + 1 + j
        c = ((T - 1 - k) // wl.leaf) * wl.leaf if hod else 0          # first uncompressed row at step T
        nfroz = {"ret": max(0, (T - 2 * k) // 32), "les": max(0, T // 32), "src": 0}[dom]
        for i in range(n_inst):
            rk = ranks0[2 * i + (1 if dom == "src" else 0)] if hod else None
            nbytes += int(iters[j, i]) * phase_bytes(dom, T, c, nfroz, no, r, wl.leaf, k, es, blocks, rk)
    dom_s = prof[dom][0] / 1e3
    achieved = nbytes / dom_s / 1e9
    peak, peak_kind = peaks()
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, steps, dt, Tlast = oracle_sample(spec, seconds=15.0)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"instance 0 of {args.workload}: time steps k+1..{Tlast} ({steps} steps, {dt:.1f} s) "
                         f"from the bootstrap, numpy FP64 dense oracle, one thread (early steps, cheaper than "
                         f"the GPU's timed window at T > {T0 + K})"}
    if rank == 0:
        tot = sum(v[0] for v in prof.values())
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": T0 - k, "ms_per_step": t_win / K * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 storage, f32 bulk sums, f64 solves" if prec == pk.PREC_MIXED else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": spec["desc"], "n_inst_per_gpu": n_inst,
                       "precision": prec_name, "nt": nt, "h": wl.h, "k": k,
                       "timed_window": f"time steps {T0 + K + 1}..{nt - 1} (the last {K}); e2e window "
                                       f"{T0 + 1}..{T0 + K}",
                       "mean_iterations_per_time_step": float(np.mean(iters)),
                       "untimed_propagation_s": round(t_prop, 2),
                       "propagation_avg_steps_per_s": round(n_inst * (T0 - k) / t_prop, 1),
                       "device_bytes": int(resident),
                       "l2": f"inputs larger than L2: {resident / 1e9:.1f} GB of state resident"},
            "roofline": {"bound": "hbm", "kernel": {"ret": "k_ret2", "les": "k_les2", "src": "k_src_h"}[dom],
                         "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "bytes_model": "phase_bytes() per instance and corrector iteration, window ranks"},
            "phase_share": {k2: round(v[0] / tot, 4) for k2, v in prof.items() if v[0] > 0},
            "cpu_baseline": cpu,
            "e2e": {"value": units / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line))
    st.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
