"""GPU parity from interacting equilibria prepared by the library's host
Matsubara solver: the mixed self-energies of the second Born, Holstein and
lattice models with U and g on the equilibrium branch (zero in every other
GPU test), against the oracle started from the same G^M."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import KBEOracle
from oracle.lattice import LatticeOracle
from oracle.models import make_model

pytestmark = pytest.mark.gpu


def _cmp(st, orcs):
    e, ref = 0.0, 0.0
    for q, o in enumerate(orcs):
        GR, GL, GTV = st.dense(q)
        n = GR.shape[0]
        idx = np.tril_indices(n)
        ref = max(ref, np.abs(o.GR[idx]).max(), np.abs(o.GLs[idx]).max(), np.abs(o.GTV).max())
        e = max(e, np.abs(GR[idx] - o.GR[idx]).max(), np.abs(GL[idx] - o.GLs[idx]).max(),
                np.abs(GTV - o.GTV).max())
    return e / ref


def test_nambu_from_interacting_equilibrium():
    beta, nt, h, k = 5.0, 80, 0.04, 5
    tau, om = wk.dlr_grid(100.0, 1e-12, beta)
    em = np.array([[0.15, 0.0], [0.0, -0.15]])
    G, e_eff, _, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_NAMBU, em[None], [[1.0, 0.4, 0.8]],
                                             U_eq=1.0, mix=0.6, tol=1e-13)
    eps = np.broadcast_to(e_eff[0], (nt + 1, 2, 2)).astype(complex)
    t = np.arange(nt) * h
    A = np.concatenate([[0.0], 0.4 * np.sin(1.2 * t) * np.exp(-(t - 1.5) ** 2 / 0.5)])
    U = np.full(nt + 1, 1.0)
    o = KBEOracle(nt, h, k, beta, eps, G[0], tau, om,
                  make_model("nambu", {"v": 1.0, "A": A, "U": U, "g": 0.4, "w0": 0.8}), tol=1e-14)
    o.run()
    st = pk.Stepper(nt, h, k, beta, nao=2, tol=1e-13, max_iter=80)
    st.set_inputs(tau, om, G, eps[None], pk.MODEL_NAMBU, np.array([[1.0, 0.4, 0.8]]))
    pk.hkbe_set_drive(st.h, A[None], U[None])
    st.run()
    assert _cmp(st, [o]) < 1e-10


def test_lattice_from_interacting_equilibrium():
    beta, L, U, nt, h, k = 4.0, 4, 1.5, 60, 0.03, 5
    tau, om = wk.dlr_grid(60.0, 1e-12, beta)
    m = np.arange(L) * 2 * np.pi / L
    ek = (-2 * (np.cos(np.repeat(m, L)) + np.cos(np.tile(m, L))))
    G, _, _, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_LATTICE2B, ek[:, None, None].astype(complex),
                                         [[L]] * (L * L), U_eq=U, mix=0.6, tol=1e-13)
    eps = np.broadcast_to(ek[:, None, None, None], (L * L, nt + 1, 1, 1)).astype(complex)
    Uv = np.full(nt + 1, U)
    o = LatticeOracle(L, nt, h, k, beta, eps, G, tau, om, Uv, tol=1e-14).run()
    st = pk.Stepper(nt, h, k, beta, nao=1, n_inst=L * L, tol=1e-13, max_iter=80)
    st.set_inputs(tau, om, G, eps, pk.MODEL_LATTICE2B, np.array([[float(L)]] * (L * L)))
    pk.hkbe_set_drive(st.h, np.zeros((L * L, nt + 1)), np.tile(Uv, (L * L, 1)))
    st.run()
    assert _cmp(st, o.orcs) < 1e-10
