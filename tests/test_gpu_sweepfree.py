"""GPU parity of the sweep-free variant (hkbe_set_scheme(HKBE_SCHEME_SWEEP_FREE),
dense FP64) against the oracle's sweep-free stepper (oracle/sweepfree.py),
element by element at 1e-10 relative: a level on two bath levels (N_o = 2,
non-commuting couplings, both density-matrix schemes), the self-consistent
Bethe lattice under a smooth drive (N_o = 1, k = 5, rows long enough for the
Gregory interior), and the driven Nambu model with second Born, Fock and
Holstein terms (N_o = 2); the variant's distance to the paper's scheme on the
GPU (it must be a different discretisation of the same equations); argument
errors."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import from_workload
from oracle.matsubara import MatsubaraOracle
from oracle.models import make_model
from oracle.sweepfree import SweepFreeOracle

pytestmark = pytest.mark.gpu

REL = 1e-10
BETA = 5.0
TAU, OM = wk.dlr_grid(100.0, 1e-12, BETA)
EPS2 = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.4]])


def _compare(st, o):
    GR, GL, GTV = st.dense(0)
    n = GR.shape[0]
    idx = np.tril_indices(n)
    ref = max(np.abs(o.GR[idx]).max(), np.abs(o.GLs[idx]).max(), np.abs(o.GTV).max())
    err = max(np.abs(GR[idx] - o.GR[idx]).max(), np.abs(GL[idx] - o.GLs[idx]).max(), np.abs(GTV - o.GTV).max())
    return err / ref


def _stepper(nt, h, k, no, rho_mode=0, beta=BETA):
    return pk.Stepper(nt, h, k, beta, nao=no, n_inst=1, rho_mode=rho_mode, tol=1e-13, max_iter=60)


@pytest.mark.parametrize("rho_mode", [0, 1])
def test_bath_two_orbitals(rho_mode):
    V = np.array([[0.5, 0.3j], [-0.2, 0.4]])
    eb = np.array([0.7, -0.9])
    H = np.block([[EPS2, V], [V.conj().T, np.diag(eb)]])
    E, U = np.linalg.eigh(H)
    gm = -np.einsum("xa,ia,ya->ixy", U[:2], wk._lehmann_kernel_unit(TAU / BETA, E * BETA), U[:2].conj())
    nt, h, k = 70, 0.05, 5
    eps = np.broadcast_to(EPS2, (nt + 1, 2, 2)).astype(complex)
    o = SweepFreeOracle(nt, h, k, BETA, eps, gm, TAU, OM, make_model("bath", {"V": V, "eb": eb}), tol=1e-14,
                        rho_mode=rho_mode).run()
    st = _stepper(nt, h, k, 2, rho_mode)
    params = np.concatenate([[len(eb)], eb, V.astype(complex).view(np.float64).ravel()])[None]
    st.set_inputs(TAU, OM, gm[None], eps[None], pk.MODEL_BATH, params)
    pk.hkbe_set_scheme(st.h, pk.SCHEME_SWEEP_FREE)
    st.run()
    assert _compare(st, o) < REL
    st.close()


def _bethe_driven():
    """Bethe lattice, k = 5, 120 steps of h = 0.05, driven level 0.3 sin(1.3 t)
    (smooth: a level quench on a grid point makes both schemes first order,
    the variant with a constant about 7 times larger)."""
    nt, h = 120, 0.05
    w = wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, dlr_eps=1e-12)
    n = np.arange(-1, nt)
    w["eps"][0, :, 0, 0] = 0.3 * np.sin(1.3 * np.maximum(n, 0) * h) * (n >= 0)
    w["gm"][0, :, 0, 0] = wk.semicircle_gm(w["tau"], BETA, 0.0)
    paper = from_workload(w, tol=1e-14)
    o = SweepFreeOracle(paper.nt, paper.h, paper.k, paper.beta, paper.eps, paper.gm, paper.tau, w["omega"],
                        paper.model, tol=1e-14).run()
    return w, o


def _gpu_run(w, scheme):
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=1, n_inst=1, tol=1e-13, max_iter=60)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"][:1], w["eps"][:1], mid, mp[:1] if mp is not None else None)
    pk.hkbe_set_scheme(st.h, scheme)
    st.run()
    return st


def test_bethe_driven_and_distance_to_paper_scheme():
    w, o = _bethe_driven()
    st = _gpu_run(w, pk.SCHEME_SWEEP_FREE)
    assert _compare(st, o) < REL
    sp = _gpu_run(w, pk.SCHEME_PAPER)
    GR, GL, _ = st.dense(0)
    GRp, GLp, _ = sp.dense(0)
    idx = np.tril_indices(GR.shape[0])
    dist = max(np.abs(GR[idx] - GRp[idx]).max(), np.abs(GL[idx] - GLp[idx]).max())
    print(f"sweep-free vs paper scheme on the GPU: {dist:.2e}")
    assert 1e-12 < dist < 1e-4
    st.close()
    sp.close()


def test_nambu_driven_second_born_holstein():
    """Driven Nambu impurity with second Born (U = 1), Fock and Holstein
    terms, started from its interacting equilibrium."""
    beta, nt, h, k = 5.0, 60, 0.04, 5
    em = np.array([[0.15, 0.0], [0.0, -0.15]])
    par = [1.0, 0.4, 0.8]
    t = np.arange(nt) * h
    A = np.concatenate([[0.0], 0.4 * np.sin(1.2 * t) * np.exp(-(t - 1.5) ** 2 / 0.5)])
    Uv = np.full(nt + 1, 1.0)
    # the interacting equilibrium as initial state (from a non-interacting one
    # the self-consistency of this driven case diverges in both schemes)
    Go, _, _, _ = MatsubaraOracle(TAU, OM, beta).solve("nambu", em[None], {"v": par[0], "U": 1.0, "g": par[1],
                                                                           "w0": par[2]}, tol=1e-13, mix=0.6)
    gm = Go[0]
    eps = np.broadcast_to(em, (nt + 1, 2, 2)).astype(complex)
    o = SweepFreeOracle(nt, h, k, beta, eps, gm, TAU, OM,
                        make_model("nambu", {"v": par[0], "A": A, "U": Uv, "g": par[1], "w0": par[2]}),
                        tol=1e-14).run()
    st = _stepper(nt, h, k, 2)
    st.set_inputs(TAU, OM, gm[None], eps[None], pk.MODEL_NAMBU, np.array([par]))
    pk.hkbe_set_drive(st.h, A[None], Uv[None])
    pk.hkbe_set_scheme(st.h, pk.SCHEME_SWEEP_FREE)
    st.run()
    assert _compare(st, o) < REL
    st.close()


def test_scheme_argument_errors(tmp_path):
    w = wk.c1_workload(seed=0, nt=30, h=0.05, k=5, dlr_eps=1e-12)
    wl = w["wl"]
    for kw in (dict(svd_tol=1e-8, leaf=32), dict(precision=pk.PREC_MIXED)):
        st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, **kw)
        with pytest.raises(pk.HKBEError):        # dense FP64 only
            pk.hkbe_set_scheme(st.h, pk.SCHEME_SWEEP_FREE)
        st.close()
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, tol=1e-13)
    with pytest.raises(pk.HKBEError):
        pk.hkbe_set_scheme(st.h, 7)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    pk.hkbe_set_scheme(st.h, pk.SCHEME_SWEEP_FREE)
    st.bootstrap()
    with pytest.raises(pk.HKBEError):            # after the bootstrap
        pk.hkbe_set_scheme(st.h, pk.SCHEME_PAPER)
    st.step(3)
    with pytest.raises(pk.HKBEError):            # checkpoints hold the paper's scheme only
        pk.hkbe_save(st.h, str(tmp_path / "x.ckp"))
    st.close()
