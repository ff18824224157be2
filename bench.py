#!/usr/bin/env python
"""Benchmark: KBE time steps per second of the GB300 stepper, batched.

One bench "step" is one KBE time step T of the whole batch: extrapolation,
self-energy, retarded row, mixed, lesser source and column, density matrix,
the self-consistency loop, and the HODLR compression of that step, for every
instance.  Default workload: C4 (N_t = 8192, Nambu Holstein-Migdal, 128
instances), the configuration the metric is quoted on.

The timed window is K consecutive time steps starting at T_s, the first step
at or after N_t/4 after which a leaf is compressed (T_s - k a multiple of the
leaf), so every window holds its compressions at the rate of one per leaf of
steps or more (one per window when K < leaf: a conservative figure).  The
run bootstraps, propagates untimed to T_s - 1, saves a device snapshot, and
  e2e window    : the K steps through the public C ABI with host buffers: eps(T)
                  of every instance uploaded from pinned memory, one step,
                  rho(T) of every instance downloaded into pinned memory;
  device window : the same K steps again from the restored snapshot, inputs
                  resident in HBM, CUDA events on the library's stream;
  phase pass    : the same K steps once more with per-phase CUDA events (phase
                  shares, the dominant kernel's time for the roofline).
The plain FP64 form of the same batch then runs the same window (its own
handle; profiled pass only: its device state leaves no room for a snapshot).

  value        = instances x K / seconds of the device window (mixed form)
  roofline     = algorithmic bytes of the dominant history kernel per launch /
                 its mean launch time, against the measured HBM copy bandwidth
  cpu_baseline = the FP64 oracle stepping the same window, one core and every
                 core (one instance per process)

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload C4|C2-batch|C3|C1] [--n-inst B] [--no-fp64]
"""
from __future__ import annotations

import os

# The oracle baseline runs one thread per process (cores = processes).
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import multiprocessing as mp
import re
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
    "C4": dict(desc="C4: Nambu Bethe-lattice DMFT, hybridisation with Peierls phases + Holstein-Migdal "
                    "(g=0.5, w0=0.6), beta=50, N_t=8192, h=0.01, order 5, DLR Lambda=200 eps=1e-10, pulse "
                    "A(t)=A0 sin(t) exp(-(t-20)^2/50) (A0=0.3 instance 0, 0.3 U[0.5,1.5] others), HODLR "
                    "leaf 64, eps_SVD 1e-7, diagonal rho scheme, normal non-interacting initial state",
               make=lambda n_inst, seed=0, **kw: wk.c4_batch_workload(n_inst, seed, **kw), n_inst=128, precision="mixed",
               tol_fp64=1e-12, tol_mixed=1e-7),
    "C2-batch": dict(desc="Bethe lattice (Sigma=v^2 G, v=1), beta=5, N_t=4096, h=0.02, order 5, DLR Lambda=100 "
                          "eps=1e-10, level quench 0 -> A at t=5 (A=1 for instance 0, U[0.5,1.5] for the others), "
                          "HODLR leaf 64, eps_SVD 1e-8, r_max 64",
                     make=lambda n_inst, seed=0, **kw: wk.c2_batch_workload(n_inst, seed, **kw), n_inst=304,
                     precision="mixed", tol_fp64=1e-12, tol_mixed=1e-7),
    "C3": dict(desc="C3-shaped: 2D Hubbard second Born on a 16 x 16 k-grid (256 coupled instances), J=1, "
                    "half filling, beta=10, N_t=2048, h=0.02, order 5, interaction quenched 0 -> U=2 at t=0 "
                    "(the free lattice as initial state), undriven, HODLR leaf 64, eps_SVD 1e-6",
               make=lambda n_inst, seed=0: wk.lattice_workload(L=16, nt=2048, h=0.02, k=5, beta=10.0, U=2.0,
                                                                t_quench=0.0, svd_tol=1e-6, leaf=64),
               n_inst=256, precision="mixed", tol_fp64=1e-12, tol_mixed=1e-7),
    "C3-ysymm": dict(desc="C3 on the reflection-reduced k-set: the 16 x 9 k-points with m_y <= 8 (144 instances; "
                          "the mirror points enter the real-space sums through their instance), otherwise as C3",
                     make=lambda n_inst, seed=0: wk.lattice_workload(L=16, nt=2048, h=0.02, k=5, beta=10.0, U=2.0,
                                                                      t_quench=0.0, svd_tol=1e-6, leaf=64,
                                                                      ysymm=True),
                     n_inst=144, grid_points=256, precision="mixed", tol_fp64=1e-12, tol_mixed=1e-7),
    "C1": dict(desc="C1: Bethe lattice, beta=5, N_t=256, h=0.025, order 5, undriven, dense storage",
               make=lambda n_inst, seed=0: wk.c1_workload(seed=seed, n_inst=n_inst), n_inst=1,
               precision="fp64", tol_fp64=1e-12, tol_mixed=1e-7),
}
WORKLOADS["C4-batch"] = WORKLOADS["C4"]   # name used by earlier profiles
C5_DESC = ("C5: 64 independent instances, N_o = 1..4 (16 each: Bethe driven level, Nambu second Born with U "
           "quenched on and a Peierls drive, and for N_o = 3, 4 a driven level matrix on two bath levels), "
           "N_t ~ U[512, 4096] per instance, beta=5, h=0.02, order 5, DLR Lambda=100 eps=1e-10, HODLR leaf 64, "
           "eps_SVD 1e-7, complex64 form; one handle per N_o, the four stepped concurrently from four host "
           "threads on four CUDA streams")

METRIC = "KBE time steps/s"
UNIT = "instance time steps/s"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def window_start(nt, k, leaf, hodlr):
    """First step T >= N_t/4 after which a leaf is compressed (T - k is a
    multiple of the leaf); N_t/4 for dense storage."""
    T = max(nt // 4, k + 1)
    if hodlr:
        while (T - k) % leaf:
            T += 1
    return T


def history_elements(T, k, L, blocks, rank_of_block, hodlr):
    """H(T): stored elements (one orbital pair) of one two-time component that
    the history integrals of step T read.  HODLR: the paper's scheme, whose
    front is c = T - k (rows older than k + 1 steps are compressed at every
    step): built block factor rows times the pair's rank plus all factor
    columns, built leaf triangles, and the k + 1 uncompressed rows s = c..T
    (s + 1 elements each).  Dense storage: the lower triangle up to row T."""
    if not hodlr:
        return (T + 1) * (T + 2) // 2
    c = T - k
    fac = 0
    for b in range(len(blocks["r0"])):
        r0, r1, c0, c1 = (int(blocks[x][b]) for x in ("r0", "r1", "c0", "c1"))
        if r0 >= c:
            continue
        fac += (min(r1, c) - r0 + (c1 - c0)) * int(rank_of_block[b])
    leaves = 0
    for j in range(0, c, L):
        m = min(L, c - j)
        leaves += m * (m + 1) // 2
    direct = sum(s + 1 for s in range(c, T + 1))
    return fac + leaves + direct


def history_all_pairs(T, k, L, no, blocks, ranks, hodlr):
    """H(T) summed over the N_o^2 orbital pairs; ranks[b, p] is the rank of
    block b, pair p."""
    if not hodlr:
        return no * no * history_elements(T, k, L, None, None, False)
    return sum(history_elements(T, k, L, blocks, ranks[:, p], True) for p in range(no * no))


def phase_bytes(phase, T, k, no, r, L, es, blocks, ranks, hodlr):
    """Algorithmic bytes of one launch of `phase` at step T for one instance
    (one corrector iteration): every stored element it needs, read once.
    es = bytes per element of the two-time storage (16 complex128, 8 complex64).
      ret / les: Sigma^R history H_R(T) plus the row read and written;
      src:       Sigma^< history H_<(T), the G^R row, Sigma^tv rows (T+1) r
                 (complex128 in both forms) and q(t) written."""
    n2 = no * no
    H = history_all_pairs(T, k, L, no, blocks, ranks, hodlr)
    row = (T + 1) * n2
    if phase in ("ret", "les"):
        return int(H * es + 2 * row * es)
    if phase == "src":
        return int(H * es + row * es + (T + 1) * r * n2 * 16 + row * 16)
    return 0


def phase_flops(phase, T, k, no, L, blocks, ranks, hodlr):
    """Algorithmic real flops of one launch of `phase` (one instance): every
    history element read enters N_o complex multiply-adds (8 N_o flop)."""
    if phase not in ("ret", "les", "src"):
        return 0
    return int(8 * no * history_all_pairs(T, k, L, no, blocks, ranks, hodlr))


KERNEL_OF = {"ret": "k_ret2", "les": "k_les2", "src": "k_src_c"}
_SWEEP_SRC = ["kernels_sweep.cu", "bulk_copy.cuh", "hodlr_util.cuh", "dev_util.cuh", "common.cuh", "state.h"]
_SRC_SRC = ["kernels_hodlr.cu", "lattice.cuh", "hodlr_util.cuh", "dev_util.cuh", "common.cuh", "state.h"]
SOURCE_OF = {"ret": _SWEEP_SRC, "les": _SWEEP_SRC, "src": _SRC_SRC}


def code_digest(names):
    """sha256 of the kernel's translation unit (its .cu and local headers) with
    comments and white space removed: a change of code, not of comments,
    invalidates a traffic record taken on the old code."""
    h = hashlib.sha256()
    for nm in names:
        text = open(os.path.join(ROOT, "paper_2604_05319_gb300", "csrc", nm)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        lines = [" ".join(line.split()) for line in text.splitlines()]
        h.update(("\n".join(line for line in lines if line) + "\n").encode())
    return h.hexdigest()


def traffic_record(phase, n_inst, T):
    """DRAM bytes per launch of the phase's main kernel from a committed ncu
    summary (profiles/traffic_<kernel>.json: dram__bytes_read.sum +
    dram__bytes_write.sum of one capture, per instance, with the code digest
    of the kernel's sources it was taken on), scaled to n_inst instances and to
    step T in proportion to T.  None when there is no capture or the code has
    changed since."""
    kern = KERNEL_OF.get(phase)
    p = os.path.join(ROOT, "profiles", f"traffic_{kern}.json")
    if kern is None or not os.path.exists(p):
        return None
    rec = json.load(open(p))
    if code_digest(SOURCE_OF[phase]) != rec.get("code_sha256"):
        return None
    return float(rec["dram_bytes_per_instance"]) * n_inst * (T / float(rec["T"]))


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


# ---------------------------------------------------------------------------
# The oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_window_worker(job):
    """One process: the FP64 oracle for instance `inst` of the workload, sized
    to the window (N = T_s + steps + 1 time points), stepping T_s, T_s+1, ...
    Its history arrays are zero-filled rather than propagated from the
    bootstrap (a C4 oracle would need hours to reach T_s); a time step's
    arithmetic does not depend on the values it reads, and the iteration count
    is fixed to `iters` (tol 0), the GPU's mean count in that window.  Returns
    the seconds of every step."""
    wname, n_inst, seed, inst, T_s, steps, iters = job
    from oracle.kbe import KBEOracle
    from oracle.models import make_model
    spec = WORKLOADS[wname]
    w = spec["make"](n_inst=n_inst, seed=seed)
    wl = w["wl"]
    nt = T_s + steps + 1
    params = dict(wl.params)
    if "drive_A" in w:
        params.update({"A": w["drive_A"][inst][:nt + 1], "U": w["drive_U"][inst][:nt + 1]})
    o = KBEOracle(nt, wl.h, wl.k, wl.beta, w["eps"][inst][:nt + 1], w["gm"][inst], w["tau"], w["omega"],
                  make_model(wl.model, params), rho_mode=wl.rho_mode, tol=0.0, max_iter=int(iters))
    out = []
    for j in range(steps):
        t0 = time.perf_counter()
        o.step(T_s + j)
        out.append(time.perf_counter() - t0)
    return out


def oracle_window(wname, n_inst, seed, T_s, steps, iters, procs):
    """The oracle on `procs` host processes (one instance each, spawned), each
    stepping `steps` time steps from T_s.  Returns (instance steps per second
    over the slowest process, per-process step times)."""
    n = min(procs, n_inst)
    jobs = [(wname, n_inst, seed, i, T_s, steps, iters) for i in range(n)]
    if n == 1:
        res = [_oracle_window_worker(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.map(_oracle_window_worker, jobs)
    wall = max(sum(r) for r in res)
    return n * steps / wall, res


def run_reference(args, wname):
    """The oracle as it stands, on the GPU machine's host cores, on this arm's
    window: one process per core (one instance each); a bench step is one
    time step of every process; W warm-up steps, then K timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec = WORKLOADS[wname]
    w = spec["make"](n_inst=1, seed=0)
    wl = w["wl"]
    hod = wl.svd_tol > 0
    T_s = window_start(wl.nt, wl.k, wl.leaf, hod)
    procs = min(os.cpu_count() or 1, args.n_inst or spec["n_inst"])
    iters = args.ref_iters
    v, res = oracle_window(wname, args.n_inst or spec["n_inst"], 0, T_s, args.warmup + args.steps, iters, procs)
    timed = [r[args.warmup:] for r in res]
    wall = max(sum(r) for r in timed)
    val = len(timed) * args.steps / wall
    sample = (f"oracle (numpy FP64, dense) in {len(timed)} processes (one core and one instance each) "
              f"stepping time steps {T_s}..{T_s + args.warmup + args.steps - 1} of {wname}; "
              f"{args.warmup} warm-up steps, then {args.steps} timed; history arrays zero-filled (a time step's "
              f"arithmetic does not depend on the values), {iters} corrector iterations per step")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "desc": spec["desc"], "window_start": T_s},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": len(timed), "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arms
# ---------------------------------------------------------------------------

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


def make_stepper(pk, w, prec, tol):
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=wl.nao, n_inst=w["eps"].shape[0], rho_mode=wl.rho_mode,
                    max_iter=wl.max_iter, tol=tol, precision=prec, svd_tol=wl.svd_tol, leaf=wl.leaf, r_max=64)
    mid, mpar = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mpar)
    if "drive_U" in w:
        pk.hkbe_set_drive(st.h, w["drive_A"], w["drive_U"])
    st.bootstrap()
    return st


def roofline_of(pk, st, w, prof, iters, T_s, K, es, dom, n_inst):
    """Algorithmic bytes and flops of the dominant phase over the window
    (per-instance iteration counts, ranks at the window start)."""
    wl = w["wl"]
    hod = wl.svd_tol > 0
    no, r = wl.nao, len(w["tau"])
    blocks = pk.hkbe_get_blocks(st.h) if hod else None
    nb = len(blocks["r0"]) if hod else 0
    comp = 3 if dom == "src" else 2
    nbytes = nflops = 0
    for i in range(n_inst):
        rk = pk.hkbe_get_ranks(st.h, i, comp, nb, no)[0] if hod else None
        for j in range(K):
            T = T_s + j
            it = int(iters[j, i])
            nbytes += it * phase_bytes(dom, T, wl.k, no, r, wl.leaf, es, blocks, rk, hod)
            nflops += it * phase_flops(dom, T, wl.k, no, wl.leaf, blocks, rk, hod)
    # one launch of the phase (over all instances) per corrector iteration of
    # the step; a step iterates until its slowest instance has converged
    launches = int(np.sum(np.max(iters, axis=1)))
    t_dom = prof[dom][0] / 1e3
    return nbytes, nflops, t_dom, launches


def run_arm(pk, torch, spec, wname, n_inst, prec_name, K, seed, dist, local, snapshot, want_e2e):
    """One precision form on the window: returns a dict of measurements."""
    w = spec["make"](n_inst=n_inst, seed=seed)
    wl = w["wl"]
    prec = pk.PREC_MIXED if prec_name == "mixed" else pk.PREC_FP64
    tol = spec["tol_mixed"] if prec_name == "mixed" else spec["tol_fp64"]
    nt, k, no = wl.nt, wl.k, wl.nao
    hod = wl.svd_tol > 0
    T_s = window_start(nt, k, wl.leaf, hod)
    K = max(1, min(K, nt - T_s))
    st = make_stepper(pk, w, prec, tol)
    t0 = time.perf_counter()
    st.step(T_s - 1 - k)                       # untimed propagation to T_s - 1
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t0
    resident = pk.hkbe_get_stats(st.h)
    out = {"T_s": T_s, "K": K, "t_prop": t_prop, "resident": resident, "w": w}
    n2 = no * no
    if snapshot:
        pk.hkbe_snapshot_save(st.h)
    # ---- e2e window (public C ABI, host buffers, copies inside the timed region) ----
    if want_e2e:
        eps_pin = torch.empty((K, n_inst, n2 * 2), dtype=torch.float64).pin_memory()
        eps_pin.copy_(torch.from_numpy(np.ascontiguousarray(
            w["eps"][:, T_s + 1:T_s + 1 + K].transpose(1, 0, 2, 3)).view(np.float64).reshape(K, n_inst, n2 * 2)))
        rho_pin = torch.empty((K, n_inst, n2 * 2), dtype=torch.float64).pin_memory()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(K):
            T = T_s + j
            pk.hkbe_set_hamiltonian_at(st.h, T, eps_pin[j].data_ptr())
            st.step(1)
            pk.hkbe_get_density_at(st.h, T, rho_pin[j].data_ptr())
        torch.cuda.synchronize()
        out["t_e2e"] = time.perf_counter() - t0
        out["h2d"] = n_inst * n2 * 16
        out["d2h"] = n_inst * n2 * 16
        pk.hkbe_snapshot_restore(st.h)
    # ---- device window: same steps, inputs resident, no per-phase events ----
    if snapshot:
        pk.hkbe_reset_counters(st.h)
        sampler = ClockSampler(local)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        sampler.start()
        ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev_a.record()
        iters, _ = st.step(K)
        ev_b.record()
        torch.cuda.synchronize()
        out["clocks"] = sampler.stop()
        out["t_win"] = ev_a.elapsed_time(ev_b) / 1e3
        out["launches"] = sum(v[1] for v in st.timing().values())
        pk.hkbe_snapshot_restore(st.h)
    # ---- phase pass: per-phase CUDA events (profiled) ----
    pk.hkbe_reset_counters(st.h)
    pk.hkbe_set_profiling(st.h, True)
    sampler = None if snapshot else ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.cudart().cudaProfilerStart()   # ncu --profile-from-start off sees this pass only
    ev_a.record()
    iters, _ = st.step(K)
    ev_b.record()
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    pk.hkbe_set_profiling(st.h, False)
    t_prof = ev_a.elapsed_time(ev_b) / 1e3
    prof = st.timing()
    if not snapshot:
        out["clocks"] = sampler.stop()
        out["t_win"] = t_prof
        out["launches"] = sum(v[1] for v in prof.values())
    out["t_prof"] = t_prof
    out["iters"] = iters
    out["prof"] = prof
    es = 8 if prec == pk.PREC_MIXED else 16
    dom = max(("ret", "les", "src"), key=lambda p: prof[p][0])
    nbytes, nflops, t_dom, nl = roofline_of(pk, st, w, prof, iters, T_s, K, es, dom, n_inst)
    out.update(dom=dom, dom_bytes=nbytes, dom_flops=nflops, t_dom=t_dom, dom_launches=nl)
    st.close()
    return out


def run_c5(args, pk, torch):
    """The uneven batch C5: every N_o group is one handle with per-instance
    N_t, the four handles step concurrently (host threads, one CUDA stream
    each).  Window: K steps from T_s (the first compression step at or after
    N_t,max/4); value = instance steps taken in the window / its wall time
    (the groups run on several streams, so the window is bracketed by device
    synchronisations and timed on the host)."""
    from concurrent.futures import ThreadPoolExecutor
    draws = wk.c5_draws()
    groups = [wk.c5_group_workload(no, draws) for no in (1, 2, 3, 4)]
    nt_max = max(g["wl"].nt for g in groups)
    k, L = groups[0]["wl"].k, groups[0]["wl"].leaf
    T_s = window_start(nt_max, k, L, True)
    K = args.steps
    steppers = []
    for g in groups:
        wl = g["wl"]
        s = torch.cuda.Stream()
        st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=wl.nao, n_inst=wl.n_inst, rho_mode=wl.rho_mode,
                        max_iter=wl.max_iter, tol=1e-7, precision=pk.PREC_MIXED, svd_tol=wl.svd_tol, leaf=wl.leaf,
                        r_max=64, stream=s.cuda_stream, nt_per_inst=g["nt_per_inst"])
        mid, mpar = pk.model_params_for(g)
        st.set_inputs(g["tau"], g["omega"], g["gm"], g["eps"], mid, mpar)
        if "drive_U" in g:
            pk.hkbe_set_drive(st.h, g["drive_A"], g["drive_U"])
        st.bootstrap()
        steppers.append((st, s, g))
    pool = ThreadPoolExecutor(4)

    def advance(to):
        def one(item):
            st, s, g = item
            cur = pk.hkbe_current_step(st.h)
            n = min(to, g["wl"].nt - 1) - cur
            return st.step(n)[0] if n > 0 else None
        return list(pool.map(one, steppers))
    t0 = time.perf_counter()
    advance(T_s - 1)
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = advance(T_s - 1 + K)
    torch.cuda.synchronize()
    t_win = time.perf_counter() - t0
    done = sum(int(np.sum(it > 0)) for it in its if it is not None)
    total_steps = sum(int(np.sum(g["nt_per_inst"] - 1 - k)) for g in groups)
    line = {"metric": METRIC, "value": done / t_win, "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": T_s - 1 - k,
            "ms_per_step": t_win / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64 storage, f32 bulk sums, f64 point solves and TSVD", "data": "synthetic",
            "config": {"workload": "C5", "desc": C5_DESC, "n_inst_per_gpu": 64,
                       "timed_window": f"time steps {T_s}..{T_s + K - 1} of every group (instances past their "
                                       f"N_t idle); host-timed between device synchronisations",
                       "instance_steps_in_window": done, "instances_active_at_window_end":
                           int(sum(np.sum(g["nt_per_inst"] - 1 >= T_s + K - 1) for g in groups)),
                       "untimed_propagation_s": round(t_prop, 2),
                       "nt_per_inst_total_steps": total_steps}}
    for st, s, g in steppers:
        st.close()
    print(json.dumps(line))


def run_scaling(args, pk, torch):
    """Scaling study (the paper's "Timing results"): one propagation of a
    small batch of the workload to N_t - 1; every `every` steps the per-step
    device time (CUDA events over 16 steps), the epsilon-ranks against block
    size (max over instances and orbital pairs, per component), and the stored
    elements of the compressed form against the dense lower triangle.  Fits
    the per-step time to T^p (the whole propagation then grows as N_t^(p+1);
    the paper's Dyson solver: T^(2+alpha) in total) and the rank to block
    size^q.  Prints one JSON record."""
    wname = "C4" if args.workload in ("C4", "C4-batch") else args.workload
    spec = WORKLOADS[wname]
    n_inst = args.n_inst or 4
    w = spec["make"](n_inst=n_inst, seed=0)
    wl = w["wl"]
    st = make_stepper(pk, w, pk.PREC_MIXED, spec["tol_mixed"])
    blocks = pk.hkbe_get_blocks(st.h)
    nb, no, k, L = len(blocks["r0"]), wl.nao, wl.k, wl.leaf
    size = (blocks["r1"] - blocks["r0"]).astype(int)
    every, probe = 512, 16
    rec = {"T": [], "ms_per_step": [], "ranks_by_size": [], "compressed_over_dense": []}
    ev_a, ev_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_all0 = time.perf_counter()
    for Tm in range(every, wl.nt - probe, every):
        st.step(Tm - pk.hkbe_current_step(st.h))
        ev_a.record()
        st.step(probe)
        ev_b.record()
        torch.cuda.synchronize()
        T = pk.hkbe_current_step(st.h)
        rk = np.array([pk.hkbe_get_stats(st.h, i, nb, no)[1] for i in range(n_inst)])  # [inst, 4, nblk, no2]
        front = pk.hkbe_get_ranks(st.h, 0, 0, nb, no)[1]
        by = {}
        for sz in sorted(set(size.tolist())):
            sel = size == sz
            by[int(sz)] = [int(rk[:, X][:, sel].max()) for X in range(4)]
        stored = 0
        for b in range(nb):
            if blocks["r0"][b] < front:
                stored += ((min(int(blocks["r1"][b]), front) - int(blocks["r0"][b])) +
                           int(blocks["c1"][b] - blocks["c0"][b])) * int(rk[0, 2, b].max())
        stored += (front // L) * L * (L + 1) // 2 + sum(s2 + 1 for s2 in range(front, T + 1))
        rec["T"].append(int(T))
        rec["ms_per_step"].append(ev_a.elapsed_time(ev_b) / probe)
        rec["ranks_by_size"].append(by)
        rec["compressed_over_dense"].append(stored / ((T + 1) * (T + 2) / 2))
    t_all = time.perf_counter() - t_all0
    Ts, ms = np.array(rec["T"], float), np.array(rec["ms_per_step"])
    half = Ts >= Ts.max() / 4
    p_fit = float(np.polyfit(np.log(Ts[half]), np.log(ms[half]), 1)[0])
    last = rec["ranks_by_size"][-1]
    szs = np.array([s2 for s2 in last if max(last[s2]) > 0], float)
    rks = np.array([max(last[int(s2)]) for s2 in szs], float)
    q_fit = float(np.polyfit(np.log(szs), np.log(rks), 1)[0]) if len(szs) > 1 else None
    out = {"study": "scaling", "workload": wname, "desc": spec["desc"], "n_inst": n_inst,
           "precision": "mixed", "every": every, "probe_steps": probe, "propagation_s": round(t_all, 1),
           "per_step_time_exponent": p_fit, "whole_run_exponent": p_fit + 1.0,
           "rank_vs_block_size_exponent": q_fit, **rec}
    st.close()
    print(json.dumps(out))


def run_matsubara_study(args, pk, torch):
    """Equilibrium Dyson solve on the device (hkbe_solve_matsubara) against
    the library's host solver (hkbe_matsubara_solve) on the initial states of
    C3 (16 x 16 lattice, U = 2, beta = 10; full and reflection-reduced k-set)
    and of the C4 batch (128 Nambu instances with the Holstein term, beta =
    50, DLR Lambda = 200): wall time of each (the device one includes its
    per-iteration convergence read-back), iterations, max |G_dev - G_host|."""
    out = {"study": "matsubara", "cases": []}

    def case(name, tau, om, beta, eps0, model, params, U, nao, n_inst):
        t0 = time.perf_counter()
        Gh, _, ith, _ = pk.hkbe_matsubara_solve(tau, om, beta, model, eps0, params, U_eq=U, mix=0.5, tol=1e-12,
                                                max_iter=2000)
        t_host = time.perf_counter() - t0
        st = pk.Stepper(16, 0.02, 5, beta, nao=nao, n_inst=n_inst, tol=1e-12, max_iter=80)
        eps = np.broadcast_to(eps0[:, None], (n_inst, 17, nao, nao)).astype(complex)
        st.set_inputs(tau, om, None, eps, model, params)
        pk.hkbe_solve_matsubara(st.h, n_inst, len(tau), nao, U_eq=U, mix=0.5, tol=1e-12, max_iter=2000)  # warm-up
        torch.cuda.synchronize()
        st.close()
        st = pk.Stepper(16, 0.02, 5, beta, nao=nao, n_inst=n_inst, tol=1e-12, max_iter=80)
        st.set_inputs(tau, om, None, eps, model, params)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Gd, itd, _ = pk.hkbe_solve_matsubara(st.h, n_inst, len(tau), nao, U_eq=U, mix=0.5, tol=1e-12, max_iter=2000)
        t_dev = time.perf_counter() - t0
        st.close()
        out["cases"].append({"case": name, "n_inst": n_inst, "r": len(tau), "host_s": round(t_host, 4),
                             "device_s": round(t_dev, 4), "speedup": round(t_host / t_dev, 1),
                             "iterations_host": ith, "iterations_device": itd,
                             "max_abs_diff": float(np.abs(Gd - Gh).max())})

    L = 16
    tau, om = wk.dlr_grid(100.0, 1e-10, 10.0)
    m = np.arange(L) * 2 * np.pi / L
    ek = (-2 * (np.cos(np.repeat(m, L)) + np.cos(np.tile(m, L))))[:, None, None].astype(complex)
    case("C3 16 x 16 lattice, U = 2", tau, om, 10.0, ek, pk.MODEL_LATTICE2B, np.array([[16.0]] * 256), 2.0, 1, 256)
    red = [x * L + y for x in range(L) for y in range(L // 2 + 1)]
    case("C3 reduced k-set (144)", tau, om, 10.0, ek[red], pk.MODEL_LATTICE2B, np.array([[16.0, 1.0]] * 144), 2.0,
         1, 144)
    tau, om = wk.dlr_grid(200.0, 1e-10, 50.0)
    case("C4 batch, Nambu + Holstein (g = 0.5, w0 = 0.6), beta = 50", tau, om, 50.0,
         np.zeros((128, 2, 2), complex), pk.MODEL_NAMBU, np.array([[1.0, 0.5, 0.6]] * 128), 0.0, 2, 128)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64, help="time steps per timed window")
    ap.add_argument("--warmup", type=int, default=3, help="untimed steps before the window (at least 3; the "
                                                          "propagation to the window start is longer)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="C4", choices=sorted(WORKLOADS) + ["C5"])
    ap.add_argument("--n-inst", type=int, default=None, help="instances per GPU (default: the workload's)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=2, help="oracle steps per process in cpu_baseline")
    ap.add_argument("--ref-iters", type=int, default=2, help="oracle corrector iterations per step")
    ap.add_argument("--study", default=None, choices=["scaling", "matsubara"],
                    help="a study instead of the bench line: rank/time scaling, or the equilibrium solve")
    args = ap.parse_args()
    assert args.warmup >= 3, "at least 3 warm-up steps"
    wname = "C4" if args.workload == "C4-batch" else args.workload
    if args.study:
        import torch
        import paper_2604_05319_gb300 as pk
        return (run_scaling if args.study == "scaling" else run_matsubara_study)(args, pk, torch)
    if wname == "C5":
        import torch
        import paper_2604_05319_gb300 as pk
        if args.impl == "reference":
            raise SystemExit("C5 has no reference arm; its oracle baseline is C4's")
        return run_c5(args, pk, torch)
    spec = WORKLOADS[wname]
    if args.impl == "reference":
        return run_reference(args, wname)

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
    if wname.startswith("C3") and n_inst != spec["n_inst"]:
        raise SystemExit(f"{wname} has one instance per k-point of its set: --n-inst must be {spec['n_inst']}")
    prec_name = spec["precision"]
    fp64_tf, fp32_tf = pk.hkbe_fma_peaks()
    main_arm = run_arm(pk, torch, spec, wname, n_inst, prec_name, args.steps, rank_seed(rank), dist, local,
                       snapshot=True, want_e2e=True)
    T_s, K = main_arm["T_s"], main_arm["K"]
    w = main_arm.pop("w")
    wl = w["wl"]
    fp64_arm = None
    if prec_name == "mixed" and not args.no_fp64:
        fp64_arm = run_arm(pk, torch, spec, wname, n_inst, "fp64", K, rank_seed(rank), dist, local,
                           snapshot=False, want_e2e=False)
        fp64_arm.pop("w")
    t_win, t_e2e = max_over_ranks([main_arm["t_win"], main_arm["t_e2e"]], dist, "cuda")
    units = n_inst * K * world
    value = units / t_win
    peak, peak_kind = peaks()
    dom = main_arm["dom"]
    achieved = main_arm["dom_bytes"] / main_arm["t_dom"] / 1e9
    traffic = traffic_record(dom, n_inst, T_s + K // 2)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        iters_mean = float(np.mean(main_arm["iters"]))
        it = max(1, int(round(iters_mean)))
        v1, _ = oracle_window(wname, n_inst, rank_seed(rank), T_s, args.cpu_steps, it, 1)
        procs = min(os.cpu_count() or 1, n_inst)
        vall, _ = oracle_window(wname, n_inst, rank_seed(rank), T_s, args.cpu_steps, it, procs)
        cpu = {"value": vall, "unit": UNIT, "cores": procs, "kind": "oracle", "one_core": v1,
               "nproc": os.cpu_count(),
               "sample": f"FP64 dense numpy oracle stepping time steps {T_s}..{T_s + args.cpu_steps - 1} of "
                         f"{wname} (the start of the GPU window), {it} corrector iterations per step (the GPU's "
                         f"mean in the window), history arrays zero-filled (a step's arithmetic does not depend "
                         f"on the values it reads); value: {procs} processes, one core and one instance each; "
                         f"one_core: one process"}
    if rank == 0:
        prof = main_arm["prof"]
        tot = sum(v[0] for v in prof.values())
        comp_steps = sum(1 for T in range(T_s, T_s + K) if wl.svd_tol > 0 and (T - wl.k) % wl.leaf == 0)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": T_s - 1 - wl.k, "ms_per_step": t_win / K * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("c64 storage, f32 bulk sums and TSVD, f64 point solves" if prec_name == "mixed" else "f64"),
            "data": "synthetic",
            "config": {"workload": wname, "desc": spec["desc"], "n_inst_per_gpu": n_inst,
                       "precision": prec_name, "nt": wl.nt, "h": wl.h, "k": wl.k,
                       "timed_window": f"time steps {T_s}..{T_s + K - 1} (first compression step at or after "
                                       f"N_t/4; {comp_steps} leaf compression(s) inside); e2e and the device "
                                       f"window run the same steps from one device snapshot",
                       "mean_iterations_per_time_step": float(np.mean(main_arm["iters"])),
                       "untimed_propagation_s": round(main_arm["t_prop"], 2),
                       "propagation_avg_steps_per_s": round(n_inst * (T_s - 1 - wl.k) / main_arm["t_prop"], 1),
                       "device_bytes": int(main_arm["resident"]),
                       "l2": f"inputs larger than L2: {main_arm['resident'] / 1e9:.1f} GB of state resident"},
            "roofline": {"bound": "hbm", "kernel": KERNEL_OF[dom], "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic,
                         "bytes_per_launch": main_arm["dom_bytes"] / max(1, main_arm["dom_launches"]),
                         "mean_launch_ms": main_arm["t_dom"] / max(1, main_arm["dom_launches"]) * 1e3,
                         "bytes_model": "Sigma history H(T) of the paper's scheme (factor rows x rank, leaf "
                                        "triangles, k+1 uncompressed rows) per instance and corrector iteration, "
                                        "ranks at the window start"},
            "phase_share": {k2: round(v[0] / tot, 4) for k2, v in prof.items() if v[0] > 0},
            "alu_peaks": {"fp64_tflops": fp64_tf, "fp32_tflops": fp32_tf, "how": "hkbe_fma_peaks, CUDA events"},
            "cpu_baseline": cpu,
            "e2e": {"value": units / t_e2e, "unit": UNIT, "h2d_bytes_per_step": main_arm["h2d"],
                    "d2h_bytes_per_step": main_arm["d2h"]},
            "gpu_launches": main_arm["launches"],
            "clocks": main_arm["clocks"],
        }
        if spec.get("grid_points"):   # reduced k-set: each step advances every point of the full grid
            line["config"]["grid_point_steps_per_s"] = spec["grid_points"] * K * world / t_win
        if fp64_arm is not None:
            f = fp64_arm
            fval = n_inst * f["K"] * world / f["t_win"]
            fprof = f["prof"]
            ftot = sum(v[0] for v in fprof.values())
            line["fp64"] = {
                "value": fval, "unit": UNIT, "ms_per_step": f["t_win"] / f["K"] * 1e3,
                "mixed_over_fp64": value / fval,
                "timed_window": f"time steps {f['T_s']}..{f['T_s'] + f['K'] - 1}, per-phase events on",
                "mean_iterations_per_time_step": float(np.mean(f["iters"])),
                "untimed_propagation_s": round(f["t_prop"], 2),
                "device_bytes": int(f["resident"]),
                "roofline": {"bound": "alu", "kernel": KERNEL_OF[f["dom"]],
                             "achieved": f["dom_flops"] / f["t_dom"] / 1e12, "peak": fp64_tf,
                             "peak_kind": "measured (hkbe_fma_peaks)", "unit": "TFLOP/s",
                             "frac": f["dom_flops"] / f["t_dom"] / 1e12 / fp64_tf,
                             "hbm_frac": f["dom_bytes"] / f["t_dom"] / 1e9 / peak},
                "phase_share": {k2: round(v[0] / ftot, 4) for k2, v in fprof.items() if v[0] > 0},
                "clocks": f["clocks"],
            }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
