"""Full-size parity: late time steps of the bench's workloads against stored
FP64 oracle rows (tests/golden/late_rows_*.npz, written by
tests/golden/make_late_rows.py, which calls only the oracle).

  C2 instance 0 (Bethe, quench, N_t = 4096, HODLR leaf 64, eps_SVD 1e-8):
    rows at T = 1024, 2048, 4095, every level of the compression built;
  C4 parameters (Nambu, Holstein-Migdal, beta = 50, h = 0.01, pulse, diagonal
    rho, HODLR 1e-7) over N_t = 1024: rows at T = 512 and 1023.

Bars: the FP64 compressed form within 10 eps_SVD (absolute, |G| <= 1); the
complex64 form within 1e-6 of max |G| plus 10 eps_SVD.  The columns sampled
are every 8th t and the last 64 (least compressed).  The mixed form's error
is also printed per component (G^R, G^<, G^tv) and for the density matrix
rho(T) = xi i G^<(T, T), the observable of these models."""
import os

import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _run(w, prec, nt):
    wl = w["wl"]
    st = pk.Stepper(nt, wl.h, wl.k, wl.beta, nao=wl.nao, n_inst=1, rho_mode=wl.rho_mode, max_iter=wl.max_iter,
                    tol=1e-13 if prec == pk.PREC_FP64 else 1e-7, precision=prec, svd_tol=wl.svd_tol,
                    leaf=wl.leaf, r_max=64)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    if "drive_U" in w:
        pk.hkbe_set_drive(st.h, w["drive_A"], w["drive_U"])
    st.bootstrap()
    return st


def _compare(name, w, prec):
    g = np.load(os.path.join(GOLDEN, f"late_rows_{name}.npz"))
    steps = [int(T) for T in g["steps"]]
    wl = w["wl"]
    st = _run(w, prec, wl.nt)
    eps_svd = wl.svd_tol
    worst = 0.0
    report = []
    for T in steps:
        st.step(T - pk.hkbe_current_step(st.h))
        cols = g[f"cols_{T}"]
        gr, gl = st.row(0, T)
        gtv = st.tv(0, T)
        ref = max(np.abs(g[f"gr_{T}"]).max(), np.abs(g[f"gl_{T}"]).max(), 1.0)
        e = {"R": np.abs(gr[cols] - g[f"gr_{T}"]).max(), "<": np.abs(gl[cols] - g[f"gl_{T}"]).max(),
             "tv": np.abs(gtv - g[f"gtv_{T}"]).max(),
             "rho": np.abs(gl[T] - g[f"gl_{T}"][-1]).max()}    # rho(T) = xi i G^<(T,T): the same entry
        report.append((T, e))
        bound = 10 * eps_svd + (1e-6 * ref if prec == pk.PREC_MIXED else 0.0)
        worst = max(worst, max(e.values()) / bound)
    st.close()
    form = "complex64" if prec == pk.PREC_MIXED else "FP64"
    for T, e in report:
        print(f"{name} {form} T={T}: " + ", ".join(f"{k} {v:.2e}" for k, v in e.items()))
    assert worst < 1.0, report


@pytest.mark.parametrize("prec", [pk.PREC_FP64, pk.PREC_MIXED])
def test_c4_parameters_late_rows(prec):
    _compare("c4", wk.c4_batch_workload(1, nt=1024), prec)


@pytest.mark.parametrize("prec", [pk.PREC_FP64, pk.PREC_MIXED])
def test_c2_instance0_late_rows(prec):
    _compare("c2", wk.c2_batch_workload(1), prec)
