"""GPU parity of the compressed (HODLR) form against the uncompressed FP64
oracle.  With a working tolerance the error must stay within 10 eps_SVD
(absolute; |G| <= 1).  With a negligible SVD tolerance (1e-15, ranks near the
block width) the compressed path must reproduce the dense result to its
rounding floor, 1e-9 absolute: a check of the block projections, leaves, band
corrections and the TSVD update machinery rather than of truncation."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import KBEOracle, from_workload
from oracle.models import make_model

pytestmark = pytest.mark.gpu
BETA = 5.0


def _max_err(st, o):
    GR, GL, GTV = st.dense(0)
    n = GR.shape[0]
    idx = np.tril_indices(n)
    parts = (np.abs(GR[idx] - o.GR[:n, :n][idx]).max(), np.abs(GL[idx] - o.GLs[:n, :n][idx]).max(),
             np.abs(GTV - o.GTV[:n]).max())
    print("HODLR error (R, <, tv):", [f"{p:.2e}" for p in parts])
    return max(parts)


_ORACLE = {}


def _bethe_oracle(nt, h, quench):
    key = (nt, h, quench)
    if key not in _ORACLE:
        w = wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, seed=4, quench=(0.0, 1.0, 3.0) if quench else None)
        o = from_workload(w, tol=1e-13)
        o.run()
        _ORACLE[key] = (w, o)
    return _ORACLE[key]


@pytest.mark.parametrize("leaf,svd_tol,bound", [(32, 1e-15, 1e-9), (64, 1e-15, 1e-9), (64, 1e-10, 1e-9),
                                                 (32, 1e-8, 1e-7), (64, 1e-8, 1e-7)])
def test_bethe_quench_hodlr(leaf, svd_tol, bound):
    nt, h = 320, 0.02
    w, o = _bethe_oracle(nt, h, True)
    # without truncation the ranks approach the block width: give them room
    st = pk.Stepper(nt, h, 5, BETA, tol=1e-13, max_iter=60, svd_tol=svd_tol, leaf=leaf,
                    r_max=128 if svd_tol < 1e-12 else 64)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.run()
    blocks = pk.hkbe_get_blocks(st.h)
    ranks, first = pk.hkbe_get_ranks(st.h, 0, 2, len(blocks["r0"]), 1)
    assert first > leaf and len(blocks["r0"]) >= 3       # several levels were compressed
    assert ranks.max() >= 1
    err = _max_err(st, o)
    assert err < bound, err


def test_bath_two_orbitals_hodlr():
    V = np.array([[0.5, 0.3j], [-0.2, 0.4]])
    eb = np.array([0.7, -0.9])
    eps2 = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.4]])
    H = np.block([[eps2, V], [V.conj().T, np.diag(eb)]])
    tau, om = wk.dlr_grid(100.0, 1e-12, BETA)
    E, U = np.linalg.eigh(H)
    gm = -np.einsum("xa,ia,ya->ixy", U[:2], wk._lehmann_kernel_unit(tau / BETA, E * BETA), U[:2].conj())
    nt, h, k = 200, 0.05, 4
    eps = np.broadcast_to(eps2, (nt + 1, 2, 2)).astype(complex)
    o = KBEOracle(nt, h, k, BETA, eps, gm, tau, om, make_model("bath", {"V": V, "eb": eb}), tol=1e-14)
    o.run()
    st = pk.Stepper(nt, h, k, BETA, nao=2, tol=1e-13, max_iter=60, svd_tol=1e-14, leaf=32, r_max=128)
    mp = np.concatenate([[2], eb, V.view(np.float64).ravel()])[None]
    st.set_inputs(tau, om, gm[None], eps[None], pk.MODEL_BATH, mp)
    st.run()
    assert _max_err(st, o) < 3e-10


def test_hodlr_rewind_reproduces():
    nt, h = 200, 0.02
    w = wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, seed=1)
    st = pk.Stepper(nt, h, 5, BETA, tol=1e-13, max_iter=60, svd_tol=1e-10, leaf=32, r_max=64)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.run()
    a = st.dense(0)
    pk.hkbe_rewind(st.h)
    st.step(nt - 1 - 5)
    b = st.dense(0)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-13


@pytest.mark.parametrize("prec", [pk.PREC_FP64, pk.PREC_MIXED])
def test_hodlr_batch_of_instances(prec):
    """Three instances (different eps0) stepped together in the compressed
    form: each must match its own oracle run and carry its own ranks."""
    nt, h, seeds = 320, 0.02, (1, 2, 3)
    ws = [wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, seed=s, quench=(0.0, 1.0, 3.0)) for s in seeds]
    for w, s in zip(ws, seeds):  # distinct quench amplitudes per instance
        w["eps"][0, 1:, 0, 0] *= 0.5 + 0.25 * s
    st = pk.Stepper(nt, h, 5, BETA, n_inst=3, tol=1e-13 if prec == pk.PREC_FP64 else 1e-7, max_iter=60,
                    svd_tol=1e-8, leaf=32, r_max=64, precision=prec)
    mid, _ = pk.model_params_for(ws[0])
    mp = np.concatenate([pk.model_params_for(w)[1] for w in ws])
    st.set_inputs(ws[0]["tau"], ws[0]["omega"], np.concatenate([w["gm"] for w in ws]),
                  np.concatenate([w["eps"] for w in ws]), mid, mp)
    st.run()
    nb = len(pk.hkbe_get_blocks(st.h)["r0"])
    for i, w in enumerate(ws):
        o = from_workload(w, tol=1e-13)
        o.run()
        GR, GL, GTV = st.dense(i)
        n = GR.shape[0]
        idx = np.tril_indices(n)
        err = max(np.abs(GR[idx] - o.GR[:n, :n][idx]).max(), np.abs(GL[idx] - o.GLs[:n, :n][idx]).max(),
                  np.abs(GTV - o.GTV[:n]).max())
        ranks, _ = pk.hkbe_get_ranks(st.h, i, 2, nb, 1)
        print("instance", i, "err", err, "max rank", ranks.max())
        assert err < (1e-7 if prec == pk.PREC_FP64 else 1e-6), (i, err)
