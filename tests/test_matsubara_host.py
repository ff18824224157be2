"""The library's host Matsubara solver (hkbe_matsubara_solve, no GPU needed)
against closed forms and against the independent oracle solver (which picks
its Matsubara frequencies differently: the two agree to the DLR accuracy)."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.matsubara import MatsubaraOracle


@pytest.fixture(scope="module")
def grid5():
    beta = 5.0
    tau, om = wk.dlr_grid(100.0, 1e-12, beta)
    return beta, tau, om, MatsubaraOracle(tau, om, beta)


def test_bethe_semicircle(grid5):
    beta, tau, om, _ = grid5
    G, _, it, err = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_BETHE, np.array([[[0.3]]]), [[1.0]],
                                            mix=0.7, tol=1e-13)
    assert err < 1e-13
    assert np.abs(G[0, :, 0, 0] - wk.semicircle_gm(tau, beta, 0.3)).max() < 1e-10


def test_free_level_model_none(grid5):
    beta, tau, om, _ = grid5
    em = np.array([[0.1, 0.3], [0.3, -0.1]])
    G, _, _, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_NONE, em[None], tol=1e-13)
    assert np.abs(G[0] - wk.free_level_gm(tau, beta, em)).max() < 1e-9


@pytest.mark.parametrize("params,U", [([1.0], 1.2), ([1.0, 0.5, 0.6], 0.0), ([1.0, 0.5, 0.6], 1.0)])
def test_nambu_matches_oracle(grid5, params, U):
    beta, tau, om, mo = grid5
    em = np.array([[0.2, 0.0], [0.0, -0.2]])
    G, e, it, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_NAMBU, em[None], [params], U_eq=U,
                                          mix=0.6, tol=1e-13)
    pd = {"v": params[0], "U": U}
    if len(params) == 3:
        pd.update({"g": params[1], "w0": params[2]})
    Go, eo, ito, _ = mo.solve("nambu", em[None], pd, tol=1e-13, mix=0.6)
    assert np.abs(G - Go).max() < 1e-9
    assert np.abs(e - eo).max() < 1e-12


def test_nambu_fock_with_pairing_matches_oracle(grid5):
    beta, tau, om, mo = grid5
    em = np.array([[0.1, 0.3], [0.3, -0.1]])
    G, e, _, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_NAMBU, em[None], [[0.8]], U_eq=0.7,
                                         mix=0.5, tol=1e-13)
    Go, eo, _, _ = mo.solve("nambu", em[None], {"v": 0.8, "U": 0.7}, tol=1e-13, mix=0.5)
    assert abs(e[0, 0, 1] - 0.3) > 1e-3                  # the Fock shift acts
    assert np.abs(G - Go).max() < 1e-9 and np.abs(e - eo).max() < 1e-9


def test_lattice_matches_oracle():
    beta, L = 4.0, 4
    tau, om = wk.dlr_grid(60.0, 1e-12, beta)
    mo = MatsubaraOracle(tau, om, beta)
    m = np.arange(L) * 2 * np.pi / L
    ek = (-2 * (np.cos(np.repeat(m, L)) + np.cos(np.tile(m, L))))[:, None, None].astype(complex)
    G, _, _, _ = pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_LATTICE2B, ek, [[L]] * (L * L), U_eq=1.5,
                                         mix=0.6, tol=1e-13)
    Go, _, _, _ = mo.solve("lattice2b", ek, {"L": L, "U": 1.5}, tol=1e-13, mix=0.6)
    assert np.abs(G - Go).max() < 1e-9


def test_errors(grid5):
    beta, tau, om, _ = grid5
    with pytest.raises(pk.HKBEError):      # Nambu needs two orbitals
        pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_NAMBU, np.zeros((1, 1, 1)), [[1.0]])
    with pytest.raises(pk.HKBEError):      # n_inst must be L^2
        pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_LATTICE2B, np.zeros((3, 1, 1)), [[2.0]] * 3)
    with pytest.raises(pk.HKBEError):      # not converged in 2 iterations
        pk.hkbe_matsubara_solve(tau, om, beta, pk.MODEL_BETHE, np.array([[[0.3]]]), [[1.0]], max_iter=2,
                                tol=1e-14)
