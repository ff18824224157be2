"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Bar (FP64 dense form): relative max-norm error <= 1e-10, i.e.
max |G_gpu - G_oracle| <= 1e-10 * max |G_oracle| over every stored element of
G^R, G^< and G^tv.  Both sides converge the self-consistency loop to 1e-14.
"""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import KBEOracle, from_workload
from oracle.models import make_model

pytestmark = pytest.mark.gpu

REL = 1e-10
BETA = 5.0
TAU, OM = wk.dlr_grid(100.0, 1e-12, BETA)


def _compare(st, o, inst=0):
    GR, GL, GTV = st.dense(inst)
    n = GR.shape[0]
    idx = np.tril_indices(n)
    ref = max(np.abs(o.GR[:n, :n][idx]).max(), np.abs(o.GLs[:n, :n][idx]).max(), np.abs(o.GTV[:n]).max())
    err = max(np.abs(GR[idx] - o.GR[:n, :n][idx]).max(), np.abs(GL[idx] - o.GLs[:n, :n][idx]).max(),
              np.abs(GTV - o.GTV[:n]).max())
    return err / ref


def _bath_params(V, eb):
    V = np.asarray(V, complex)
    return np.concatenate([[len(eb)], eb, V.view(np.float64).ravel()])


def _run_pair(nt, h, k, eps_d, model_name, model_params, gm, rho_mode=0, tau=TAU, om=OM, beta=BETA):
    no = eps_d.shape[-1]
    eps = np.broadcast_to(eps_d, (nt + 1, no, no)).astype(complex)
    o = KBEOracle(nt, h, k, beta, eps, gm, tau, om, make_model(model_name, model_params), tol=1e-14,
                  rho_mode=rho_mode)
    o.run()
    st = pk.Stepper(nt, h, k, beta, nao=no, n_inst=1, rho_mode=rho_mode, tol=1e-13, max_iter=60)
    mid = {"none": pk.MODEL_NONE, "bath": pk.MODEL_BATH}[model_name]
    mp = None if model_name == "none" else _bath_params(model_params["V"], model_params["eb"])[None]
    st.set_inputs(tau, om, gm[None], eps[None], mid, mp)
    st.run()
    return st, o


EPS2 = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.4]])


def test_sigma0_matrix_level():
    gm = wk.free_level_gm(TAU, BETA, EPS2)
    st, o = _run_pair(40, 0.05, 4, EPS2, "none", None, gm)
    assert _compare(st, o) < REL


@pytest.mark.parametrize("rho_mode", [0, 1])
def test_bath_two_orbitals(rho_mode):
    V = np.array([[0.5, 0.3j], [-0.2, 0.4]])
    eb = np.array([0.7, -0.9])
    H = np.block([[EPS2, V], [V.conj().T, np.diag(eb)]])
    E, U = np.linalg.eigh(H)
    gm = -np.einsum("xa,ia,a,ya->ixy", U[:2], wk._lehmann_kernel_unit(TAU / BETA, E * BETA), np.ones(4),
                    U[:2].conj())
    st, o = _run_pair(70, 0.05, 5, EPS2, "bath", {"V": V, "eb": eb}, gm, rho_mode=rho_mode)
    assert _compare(st, o) < REL


@pytest.mark.parametrize("no", [3, 4])
def test_bath_three_and_four_orbitals(no):
    rng = np.random.default_rng(no)
    A = rng.normal(size=(no, no)) + 1j * rng.normal(size=(no, no))
    eps_d = 0.3 * (A + A.conj().T)
    V = 0.3 * (rng.normal(size=(no, 2)) + 1j * rng.normal(size=(no, 2)))
    eb = np.array([0.5, -0.6])
    H = np.block([[eps_d, V], [V.conj().T, np.diag(eb)]])
    E, U = np.linalg.eigh(H)
    gm = -np.einsum("xa,ia,ya->ixy", U[:no], wk._lehmann_kernel_unit(TAU / BETA, E * BETA), U[:no].conj())
    st, o = _run_pair(45, 0.05, 3, eps_d, "bath", {"V": V, "eb": eb}, gm)
    assert _compare(st, o) < REL


@pytest.mark.parametrize("k,nt", [(1, 3), (2, 4), (5, 7), (5, 13), (3, 50)])
def test_minimal_and_ragged_lengths_bethe(k, nt):
    """nt = k + 2 (one step after the bootstrap), nt < 2k+1 (special Gregory
    rule), and lengths that are not multiples of the 32-point sweep chunk."""
    w = wk.bethe_workload(nt=nt, h=0.05, k=k, beta=BETA, seed=1, dlr_eps=1e-12)
    o = from_workload(w, tol=1e-14)
    o.run()
    st = pk.Stepper(nt, 0.05, k, BETA, tol=1e-13, max_iter=60)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.run()
    assert _compare(st, o) < REL


def test_bethe_c1_full_size_and_batch():
    """The C1 workload (Bethe, beta=5, N_t=256, h=0.025, order 5, DLR
    Lambda=100 / eps=1e-10) for three seeds stepped together in one batch."""
    seeds = [0, 1, 2]
    w = wk.c1_workload(seed=0, n_inst=3)
    w["eps"] = np.concatenate([wk.c1_workload(seed=s)["eps"] for s in seeds])
    w["gm"] = np.concatenate([wk.c1_workload(seed=s)["gm"] for s in seeds])
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, n_inst=3, tol=1e-13, max_iter=60)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.run()
    for inst, s in enumerate(seeds):
        ws = wk.c1_workload(seed=s)
        o = from_workload(ws, tol=1e-13)
        o.run()
        assert _compare(st, o, inst) < REL, s


def test_quench_c2_protocol_short():
    """C2's level quench (eps0: 0 -> 1 at t=5, h=0.02) on the first 300 steps."""
    w = wk.c2_workload(nt=300)
    o = from_workload(w, tol=1e-13)
    o.run()
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, tol=1e-13, max_iter=60)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.run()
    assert _compare(st, o) < REL


def test_range_and_order_errors():
    st = pk.Stepper(10, 0.05, 2, BETA)
    with pytest.raises(pk.HKBEError):
        st.step(1)          # before bootstrap / inputs
    w = wk.bethe_workload(nt=10, h=0.05, k=2, beta=BETA)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.bootstrap()
    st.step(7)
    with pytest.raises(pk.HKBEError) as e:
        st.step(1)
    assert e.value.code == -4
    with pytest.raises(pk.HKBEError):
        pk.hkbe_get_ret(st.h, 1, 0, 5, 6)


@pytest.mark.parametrize("no,prec", [(3, pk.PREC_FP64), (4, pk.PREC_FP64), (3, pk.PREC_MIXED), (4, pk.PREC_MIXED)])
def test_bath_three_and_four_orbitals_compressed(no, prec):
    """N_o = 3 and 4 in the compressed form (leaf 32, four leaves compressed,
    blocks on two levels), FP64 (eps_SVD 1e-10, bound 1e-9 absolute) and
    complex64 (eps_SVD 1e-8, bound 1e-6 of max |G| plus 10 eps_SVD), with a
    driven level matrix eps(t) = eps_d + 0.2 sin(1.3 t) (C5's larger groups)."""
    nt, h, k = 140, 0.05, 5
    rng = np.random.default_rng(no)
    A = rng.normal(size=(no, no)) + 1j * rng.normal(size=(no, no))
    eps_d = 0.3 * (A + A.conj().T)
    V = 0.3 * (rng.normal(size=(no, 2)) + 1j * rng.normal(size=(no, 2)))
    eb = np.array([0.5, -0.6])
    H = np.block([[eps_d, V], [V.conj().T, np.diag(eb)]])
    E, U = np.linalg.eigh(H)
    gm = -np.einsum("xa,ia,ya->ixy", U[:no], wk._lehmann_kernel_unit(TAU / BETA, E * BETA), U[:no].conj())
    tt = np.concatenate([[0.0], np.arange(nt) * h])
    eps = eps_d[None] + (0.2 * np.sin(1.3 * tt) * (np.arange(nt + 1) > 0))[:, None, None] * np.eye(no)[None]
    o = KBEOracle(nt, h, k, BETA, eps, gm, TAU, OM, make_model("bath", {"V": V, "eb": eb}), tol=1e-14)
    o.run()
    svd_tol = 1e-10 if prec == pk.PREC_FP64 else 1e-8
    st = pk.Stepper(nt, h, k, BETA, nao=no, n_inst=1, tol=1e-13 if prec == pk.PREC_FP64 else 1e-7, max_iter=60,
                    precision=prec, svd_tol=svd_tol, leaf=32, r_max=64)
    st.set_inputs(TAU, OM, gm[None], eps[None].astype(complex), pk.MODEL_BATH, _bath_params(V, eb)[None])
    st.run()
    GR, GL, GTV = st.dense(0)
    idx = np.tril_indices(nt)
    ref = max(np.abs(o.GR[idx]).max(), np.abs(o.GLs[idx]).max())
    err = max(np.abs(GR[idx] - o.GR[idx]).max(), np.abs(GL[idx] - o.GLs[idx]).max(), np.abs(GTV - o.GTV).max())
    assert pk.hkbe_get_ranks(st.h, 0, 2, len(pk.hkbe_get_blocks(st.h)["r0"]), no)[1] >= 96
    bound = 1e-9 if prec == pk.PREC_FP64 else 1e-6 * ref + 10 * svd_tol
    print(f"N_o = {no}, {'FP64' if prec == pk.PREC_FP64 else 'complex64'} compressed: max error {err:.2e}")
    assert err < bound, err
