"""GPU parity of the mixed-precision form (complex64 storage of the two-time
and mixed components, FP64 point solves and accumulations) against the FP64
oracle.

Bar: relative max-norm error <= 1e-6 over every stored element of G^R, G^< and
G^tv (for the HODLR form with eps_SVD = 1e-8 the truncation adds at most
10 eps_SVD absolute, below the same bar since |G| <= 1).  The self-consistency
loop stops at 1e-7: complex64 rounding of the stored row bounds how far the
iteration difference can fall (one unit in the last place is 6e-8 of |G|).
"""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import KBEOracle, from_workload
from oracle.models import make_model

pytestmark = pytest.mark.gpu

REL = 1e-6
BETA = 5.0


def _rel_err(st, o, inst=0):
    GR, GL, GTV = st.dense(inst)
    n = GR.shape[0]
    idx = np.tril_indices(n)
    ref = max(np.abs(o.GR[:n, :n][idx]).max(), np.abs(o.GLs[:n, :n][idx]).max(), np.abs(o.GTV[:n]).max())
    parts = (np.abs(GR[idx] - o.GR[:n, :n][idx]).max(), np.abs(GL[idx] - o.GLs[:n, :n][idx]).max(),
             np.abs(GTV - o.GTV[:n]).max())
    print("mixed-form error (R, <, tv) / max|G|:", [f"{p / ref:.2e}" for p in parts])
    return max(parts) / ref


_ORACLE = {}


def _bethe(nt, h, quench, seed):
    key = (nt, h, quench, seed)
    if key not in _ORACLE:
        w = wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, seed=seed, quench=(0.0, 1.0, 3.0) if quench else None)
        o = from_workload(w, tol=1e-13)
        o.run()
        _ORACLE[key] = (w, o)
    return _ORACLE[key]


def _stepper(w, nt, h, **kw):
    st = pk.Stepper(nt, h, 5, BETA, tol=1e-7, max_iter=60, precision=pk.PREC_MIXED, **kw)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.run()
    return st


def test_mixed_dense_bethe_quench():
    nt, h = 300, 0.02
    w, o = _bethe(nt, h, True, 4)
    st = _stepper(w, nt, h)
    err = _rel_err(st, o)
    assert err < REL, err
    assert err > 1e-12  # the storage really is single precision


@pytest.mark.parametrize("leaf,svd_tol", [(32, 1e-8), (64, 1e-8)])
def test_mixed_hodlr_bethe_quench(leaf, svd_tol):
    nt, h = 320, 0.02
    w, o = _bethe(nt, h, True, 4)
    st = _stepper(w, nt, h, svd_tol=svd_tol, leaf=leaf, r_max=64)
    _, first = pk.hkbe_get_ranks(st.h, 0, 2, len(pk.hkbe_get_blocks(st.h)["r0"]), 1)
    assert first > leaf
    err = _rel_err(st, o)
    assert err < REL, err


def test_mixed_bath_two_orbitals_hodlr():
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
    st = pk.Stepper(nt, h, k, BETA, nao=2, tol=1e-7, max_iter=60, svd_tol=1e-9, leaf=32, r_max=64,
                    precision=pk.PREC_MIXED)
    mp = np.concatenate([[2], eb, V.view(np.float64).ravel()])[None]
    st.set_inputs(tau, om, gm[None], eps[None], pk.MODEL_BATH, mp)
    st.run()
    err = _rel_err(st, o)
    assert err < REL, err


def test_mixed_batch_of_instances_matches_single():
    nt, h = 128, 0.02
    ws = [wk.bethe_workload(nt=nt, h=h, k=5, beta=BETA, seed=s) for s in (1, 2, 3)]
    st = pk.Stepper(nt, h, 5, BETA, n_inst=3, tol=1e-7, max_iter=60, precision=pk.PREC_MIXED)
    mid, mp = pk.model_params_for(ws[0])
    mp = np.concatenate([pk.model_params_for(w)[1] for w in ws])
    st.set_inputs(ws[0]["tau"], ws[0]["omega"], np.concatenate([w["gm"] for w in ws]),
                  np.concatenate([w["eps"] for w in ws]), mid, mp)
    st.run()
    for i, w in enumerate(ws):
        o = from_workload(w, tol=1e-13)
        o.run()
        err = _rel_err(st, o, i)
        assert err < REL, (i, err)


def test_integer_fp64_to_fp32_rounding():
    """The complex64 form's FP64 -> FP32 conversion of G^tv (integer pipes,
    IEEE 754 fields): equal to round-to-nearest FP32 away from ties, ties away
    from zero, relative error at most 2^-24, sub-normal-range magnitudes to
    zero, sign kept."""
    rng = np.random.default_rng(5)
    x = rng.choice([-1.0, 1.0], 200000) * 10.0 ** rng.uniform(-37, 30, 200000)   # normal FP32 range
    y = pk.hkbe_f32_of(x)
    ref = x.astype(np.float32)
    assert np.array_equal(y, ref), np.flatnonzero(y != ref)[:5]
    assert (np.abs(y.astype(np.float64) - x) <= 2.0 ** -24 * np.abs(x)).all()
    one_tie = 1.0 + 2.0 ** -24          # halfway between 1 and 1 + 2^-23
    special = np.array([0.0, -0.0, 1.0, -2.5, one_tie, -one_tie, 1e-39, -1e-300, 3.0e38])
    ys = pk.hkbe_f32_of(special)
    assert ys[0] == 0 and np.signbit(ys[1]) and ys[2] == 1.0 and ys[3] == -2.5
    assert ys[4] == np.float32(1.0 + 2.0 ** -23) and ys[5] == -np.float32(1.0 + 2.0 ** -23)
    assert ys[6] == 0 and ys[7] == 0 and np.signbit(ys[7]) and ys[8] == np.float32(3.0e38)
