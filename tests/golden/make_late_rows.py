"""Writes the late-time reference rows the full-size GPU parity tests compare
with, by running the FP64 oracle (and nothing else) on the workloads' own
seeded inputs.  Run from the repository root:

    python tests/golden/make_late_rows.py c2     # C2 instance 0, N_t = 4096
    python tests/golden/make_late_rows.py c4     # C4 parameters, N_t = 1024
    python tests/golden/make_late_rows.py c3     # C3's 16 x 16 lattice, N_t = 40

Each file holds, for a few steps T, sampled columns of the retarded row
G^R(T, t) and of the lesser column G^<(t, T) (every 8th t plus the last 64,
where the history is least compressed) and the mixed row G^tv(T, tau_i).
For the lattice (all 256 k-points coupled) the file holds every row of
eight sampled k-points and the lattice observables n, E_kin, j at every t.
The oracle runs with self-consistency tolerance 1e-13 (1e-14 for the
lattice; the FP64 parity setting).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import kbe_workloads as wk  # noqa: E402
from oracle.kbe import from_workload  # noqa: E402


def sample_cols(T):
    return np.unique(np.concatenate([np.arange(0, T + 1, 8), np.arange(max(0, T - 63), T + 1)]))


LATTICE_SAMPLE = (0, 17, 34, 51, 85, 136, 170, 255)


def run_lattice():
    from oracle.lattice import LatticeOracle
    w = wk.lattice_workload(L=16, nt=40, h=0.02, k=5, beta=10.0, U=2.0, t_quench=0.0)
    wl = w["wl"]
    o = LatticeOracle(w["L"], wl.nt, wl.h, wl.k, wl.beta, w["eps"], w["gm"], w["tau"], w["omega"],
                      w["drive_U"][0], tol=1e-14)
    o.run()
    n, ekin, j = o.observables(w["drive_A"][0])
    idx = np.tril_indices(wl.nt)
    out = {"k_sample": np.array(LATTICE_SAMPLE), "n": n, "ekin": ekin, "j": j}
    for q in LATTICE_SAMPLE:
        oq = o.orcs[q]
        out[f"gr_{q}"] = oq.GR[idx]
        out[f"gl_{q}"] = oq.GLs[idx]
        out[f"gtv_{q}"] = oq.GTV
    np.savez_compressed(os.path.join(HERE, "late_rows_c3.npz"), **out)


def run(name):
    if name == "c3":
        return run_lattice()
    if name == "c2":
        w = wk.c2_batch_workload(1)           # instance 0 of the C2 batch is C2 itself
        steps = (1024, 2048, 4095)
    elif name == "c4":
        w = wk.c4_batch_workload(1, nt=1024)  # instance 0 of the C4 batch, first 1024 steps
        steps = (512, 1023)
    else:
        raise SystemExit("workload: c2, c3 or c4")
    o = from_workload(w, tol=1e-13)
    t0 = time.time()
    o.bootstrap()
    out = {}
    for T in range(o.k + 1, o.nt):
        o.step(T)
        if T in steps:
            cols = sample_cols(T)
            out[f"cols_{T}"] = cols
            out[f"gr_{T}"] = o.GR[T, cols]
            out[f"gl_{T}"] = o.GLs[T, cols]
            out[f"gtv_{T}"] = o.GTV[T]
            print(f"{name}: T = {T} stored ({time.time() - t0:.0f} s)", flush=True)
    out["steps"] = np.array(steps)
    out["iters"] = o.iters
    np.savez_compressed(os.path.join(HERE, f"late_rows_{name}.npz"), **out)


if __name__ == "__main__":
    run(sys.argv[1])
