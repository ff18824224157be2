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
_CASE = dict(L=4, nt=100, h=0.025, k=5, beta=10.0, U=2.0, t_quench=0.2, A0=0.5, Omega=1.2, tc=1.0, width=0.4)


def _case():
    if "w" not in _CACHE:
        w = wk.lattice_workload(**_CASE)
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


def _err(st, o, kset=None):
    """Max error over the instances; instance i holds the oracle's k-point
    kset[i] (default i)."""
    e, ref = 0.0, 0.0
    for i, q in enumerate(kset if kset is not None else range(len(o.orcs))):
        oq = o.orcs[q]
        GR, GL, GTV = st.dense(i)
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


def test_lattice_2b_reflection_reduced_set():
    """The reflection-reduced k-set (Sec. 4.2: the drive along x keeps
    k_y -> -k_y, so L(L/2+1) = 12 of the 16 k-points are propagated and the
    mirror points enter the real-space sums through their instance) against
    the full-grid oracle at its k-points: dense FP64 within 1e-10, compressed
    within 10 eps_SVD, complex64 within 1e-6; the lattice observables over the
    whole grid as for the full set."""
    w, o = _case()
    wr = wk.lattice_workload(**_CASE, ysymm=True)
    L = _CASE["L"]
    red = [x * L + y for x in range(L) for y in range(L // 2 + 1)]
    assert wr["eps"].shape[0] == len(red) == 12
    assert np.array_equal(wr["eps"], w["eps"][red])
    st = _run(wr)
    assert _err(st, o, red)[1] < 1e-10
    n, ekin, j = o.observables(w["drive_A"][0])
    for t in (0, 50, 99):
        ob = pk.hkbe_get_lattice_observables(st.h, t)
        assert np.allclose(ob, [n[t], ekin[t], j[t]], rtol=1e-10, atol=1e-12), (t, ob)
    st.close()
    st = _run(wr, svd_tol=1e-10, leaf=32, r_max=64)
    assert _err(st, o, red)[0] < 1e-9
    st.close()
    st = _run(wr, tol=1e-7, precision=pk.PREC_MIXED)
    assert _err(st, o, red)[1] < 1e-6
    st.close()


def test_lattice_reflection_argument_errors():
    """ysymm needs an even L and n_inst = L(L/2+1); ysymm is 0 or 1."""
    w = wk.lattice_workload(L=4, nt=20, h=0.025, k=5, beta=10.0, U=2.0)
    wl = w["wl"]
    for n_inst, mp in ((16, [4.0, 1.0]), (12, [4.0]), (12, [4.0, 2.0]), (6, [3.0, 1.0])):
        st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=1, n_inst=n_inst)
        with pytest.raises(pk.HKBEError):
            pk.hkbe_set_model(st.h, pk.MODEL_LATTICE2B, np.array([mp] * n_inst))
        st.close()


def test_lattice_16x16_c3_parameters():
    """C3's own grid and parameters (16 x 16 k, J = 1, U = 2 quenched on at
    t = 0, beta = 10, h = 0.02, undriven) on a short propagation: the L = 16
    path of the real-space self-energy (256 threads, one per k-point and
    real-space point) against stored oracle rows of eight k-points and the
    lattice observables at every t (tests/golden/late_rows_c3.npz, written by
    tests/golden/make_late_rows.py from the oracle alone); dense FP64 within
    1e-10, complex64 within 1e-6; the same for the reflection-reduced set of
    16 x 9 k-points (a sampled point with m_y > 8 is read from its mirror)."""
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "late_rows_c3.npz"))
    L = 16
    runs = [(False, pk.PREC_FP64, 1e-13, 1e-10), (False, pk.PREC_MIXED, 1e-7, 1e-6),
            (True, pk.PREC_FP64, 1e-13, 1e-10), (True, pk.PREC_MIXED, 1e-7, 1e-6)]
    for ysymm, prec, tol, bound in runs:
        w = wk.lattice_workload(L=L, nt=40, h=0.02, k=5, beta=10.0, U=2.0, t_quench=0.0, ysymm=ysymm)
        nt = w["wl"].nt
        idx = np.tril_indices(nt)
        st = _run(w, tol=tol, precision=prec)
        ref = max(np.abs(g[f"gr_{q}"]).max() for q in g["k_sample"])
        err = 0.0
        for q in g["k_sample"]:   # reduced set: (m_x, m_y) lives in instance m_x (L/2+1) + min(m_y, L - m_y)
            x, y = divmod(int(q), L)
            GR, GL, GTV = st.dense(x * (L // 2 + 1) + min(y, L - y) if ysymm else int(q))
            err = max(err, np.abs(GR[idx] - g[f"gr_{q}"]).max(), np.abs(GL[idx] - g[f"gl_{q}"]).max(),
                      np.abs(GTV - g[f"gtv_{q}"]).max())
        assert err < bound * ref, (prec, err)
        oerr = np.zeros(3)
        for t in range(nt):
            ob = pk.hkbe_get_lattice_observables(st.h, t)
            oerr = np.maximum(oerr, np.abs(np.asarray(ob) - [g["n"][t], g["ekin"][t], g["j"][t]]))
        print("16 x 16", "reduced" if ysymm else "full", "FP64" if prec == pk.PREC_FP64 else "complex64",
              "max error: G", err, "n, E_kin, j", oerr.tolist())
        assert (oerr < bound * np.maximum(1.0, np.abs([g["n"], g["ekin"], g["j"]]).max(axis=1))).all(), oerr
        st.close()
