"""GPU parity of the 2D Hubbard second-Born lattice (Sec. 4.2, all k-points
coupled through the real-space self-energy) against the lockstep FP64 oracle,
through the C ABI: a 4 x 4 k-grid under an interaction quench and a Peierls
pulse along x, dense FP64, compressed and mixed forms, and the lattice
observables n, E_kin, j."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.lattice import LatticeOracle

pytestmark = pytest.mark.gpu

_CACHE = {}


def _case():
    if "w" not in _CACHE:
        w = wk.lattice_workload(L=4, nt=100, h=0.025, k=5, beta=10.0, U=2.0, t_quench=0.2, A0=0.5,
                                Omega=1.2, tc=1.0, width=0.4)
        wl = w["wl"]
        o = LatticeOracle(w["L"], wl.nt, wl.h, wl.k, wl.beta, w["eps"], w["gm"], w["tau"], w["omega"],
                          w["drive_U"][0], tol=1e-14)
        o.run()
        _CACHE["w"] = (w, o)
    return _CACHE["w"]


def _run(w, tol=1e-13, **kw):
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=1, n_inst=w["eps"].shape[0], tol=tol, max_iter=80, **kw)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    pk.hkbe_set_drive(st.h, w["drive_A"], w["drive_U"])
    st.run()
    return st


def _err(st, o):
    e, ref = 0.0, 0.0
    for q, oq in enumerate(o.orcs):
        GR, GL, GTV = st.dense(q)
        n = GR.shape[0]
        idx = np.tril_indices(n)
        ref = max(ref, np.abs(oq.GR[idx]).max(), np.abs(oq.GLs[idx]).max(), np.abs(oq.GTV).max())
        e = max(e, np.abs(GR[idx] - oq.GR[idx]).max(), np.abs(GL[idx] - oq.GLs[idx]).max(),
                np.abs(GTV - oq.GTV).max())
    return e, e / ref


def test_lattice_2b_dense_and_observables():
    w, o = _case()
    st = _run(w)
    assert _err(st, o)[1] < 1e-10
    n, ekin, j = o.observables(w["drive_A"][0])
    for t in (0, 10, 50, 99):
        ob = pk.hkbe_get_lattice_observables(st.h, t)
        assert np.allclose(ob, [n[t], ekin[t], j[t]], rtol=1e-10, atol=1e-12), (t, ob)
    assert np.abs(j).max() > 1e-3


def test_lattice_2b_hodlr():
    w, o = _case()
    st = _run(w, svd_tol=1e-10, leaf=32, r_max=64)
    assert _err(st, o)[0] < 1e-9


def test_lattice_2b_mixed():
    w, o = _case()
    st = _run(w, tol=1e-7, precision=pk.PREC_MIXED)
    assert _err(st, o)[1] < 1e-6
