"""GPU parity of the Nambu model (Eq. Hybrid with Peierls phases, Eq.
Sigma2B, Eq. SigmaF) against the FP64 oracle, through the C ABI: a normal
Bethe-lattice state under an interaction quench and a vector-potential pulse
(both density-matrix schemes), a free Nambu level with pairing under a quench
(the Fock term and the anomalous components at work), the compressed form,
the mixed-precision form and a batch of instances with different U."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import from_workload

pytestmark = pytest.mark.gpu

BETA = 5.0
_CACHE = {}


def _case(name, rho_mode=0, n_inst=1):
    key = (name, rho_mode, n_inst)
    if key in _CACHE:
        return _CACHE[key]
    if name == "normal":
        w = wk.nambu_workload(nt=200, h=0.02, k=5, beta=BETA, v=1.0, eps0=0.2, U=1.0, t_quench=0.5,
                              A0=0.5, Omega=1.3, tc=2.0, width=0.5, rho_mode=rho_mode, n_inst=n_inst)
    else:
        w = wk.nambu_workload(nt=160, h=0.02, k=5, beta=BETA, v=0.0, eps0=0.1, pairing=0.3, U=0.8,
                              t_quench=0.3, A0=0.3, Omega=1.0, tc=1.5, width=0.5, rho_mode=rho_mode,
                              n_inst=n_inst)
    orc = []
    for i in range(n_inst):
        o = from_workload(w, inst=i, tol=1e-14)
        o.run()
        orc.append(o)
    _CACHE[key] = (w, orc)
    return _CACHE[key]


def _run(w, tol=1e-13, **kw):
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=2, n_inst=w["eps"].shape[0], rho_mode=wl.rho_mode,
                    tol=tol, max_iter=80, **kw)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    pk.hkbe_set_drive(st.h, w["drive_A"], w["drive_U"])
    st.run()
    return st


def _err(st, o, inst=0):
    GR, GL, GTV = st.dense(inst)
    n = GR.shape[0]
    idx = np.tril_indices(n)
    ref = max(np.abs(o.GR[:n, :n][idx]).max(), np.abs(o.GLs[:n, :n][idx]).max(), np.abs(o.GTV[:n]).max())
    err = max(np.abs(GR[idx] - o.GR[:n, :n][idx]).max(), np.abs(GL[idx] - o.GLs[:n, :n][idx]).max(),
              np.abs(GTV - o.GTV[:n]).max())
    return err, err / ref


@pytest.mark.parametrize("rho_mode", [0, 1])
def test_nambu_normal_quench_pulse_dense(rho_mode):
    w, (o,) = _case("normal", rho_mode)
    st = _run(w)
    assert _err(st, o)[1] < 1e-10
    GR, GL, _ = st.dense(0)
    assert np.abs(GR[..., 0, 1]).max() < 1e-13          # stays normal on the GPU as well


def test_nambu_pairing_fock_dense():
    w, (o,) = _case("pairing")
    st = _run(w)
    assert _err(st, o)[1] < 1e-10
    GR, GL, _ = st.dense(0)
    assert np.abs(GL[..., 0, 1]).max() > 1e-2           # anomalous components present


@pytest.mark.parametrize("svd_tol,bound", [(1e-10, 1e-9), (1e-8, 1e-7)])
def test_nambu_hodlr(svd_tol, bound):
    w, (o,) = _case("normal")
    st = _run(w, svd_tol=svd_tol, leaf=32, r_max=64)
    assert _err(st, o)[0] < bound


@pytest.mark.parametrize("svd_tol", [0.0, 1e-8])
def test_nambu_mixed(svd_tol):
    w, (o,) = _case("normal")
    kw = dict(svd_tol=svd_tol, leaf=32, r_max=64) if svd_tol else {}
    st = _run(w, tol=1e-7, precision=pk.PREC_MIXED, **kw)
    assert _err(st, o)[1] < 1e-6


def test_nambu_batch_distinct_u():
    w, orc = _case("pairing", n_inst=2)
    st = _run(w)
    for i, o in enumerate(orc):
        assert _err(st, o, i)[1] < 1e-10, i


@pytest.mark.parametrize("prec", [pk.PREC_FP64, pk.PREC_MIXED])
def test_nambu_holstein_migdal(prec):
    """The optional Holstein term (C4's g = 0.5, w0 = 0.6) on top of the
    hybridisation and a pulse: GPU vs oracle."""
    key = ("migdal",)
    if key not in _CACHE:
        w = wk.nambu_workload(nt=160, h=0.02, k=5, beta=BETA, v=1.0, eps0=0.1, A0=0.5, Omega=1.0, tc=1.5,
                              width=0.5, g=0.5, w0=0.6)
        o = from_workload(w, tol=1e-14)
        o.run()
        _CACHE[key] = (w, o)
    w, o = _CACHE[key]
    st = _run(w, tol=1e-13 if prec == pk.PREC_FP64 else 1e-7, precision=prec)
    assert _err(st, o)[1] < (1e-10 if prec == pk.PREC_FP64 else 1e-6)
