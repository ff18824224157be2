"""Per-step host I/O through the C ABI: eps(t) supplied one time at a time
(hkbe_set_hamiltonian_at) must give the same propagation as the whole eps
array set up front, and hkbe_get_density_at must return the rows of
hkbe_get_density, in both storage forms."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("svd_tol,prec", [(0.0, pk.PREC_FP64), (1e-8, pk.PREC_MIXED)])
def test_eps_per_step_and_density_at(svd_tol, prec):
    nt, h, n_inst = 200, 0.02, 3
    w = wk.bethe_workload(nt=nt, h=h, k=5, beta=5.0, n_inst=n_inst, seed=7, quench=(0.0, 1.0, 1.0))
    w["eps"][:, 1:, 0, 0] *= np.array([0.5, 1.0, 1.5])[:, None]
    mid, mp = pk.model_params_for(w)
    kw = dict(n_inst=n_inst, tol=1e-12 if prec == pk.PREC_FP64 else 1e-7, max_iter=60,
              precision=prec, svd_tol=svd_tol, leaf=32, r_max=64)

    a = pk.Stepper(nt, h, 5, 5.0, **kw)
    a.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    a.run()

    b = pk.Stepper(nt, h, 5, 5.0, **kw)
    eps0 = w["eps"].copy()
    eps0[:, 7:] = 0.0                   # times after the start square arrive step by step
    b.set_inputs(w["tau"], w["omega"], w["gm"], eps0, mid, mp)
    b.bootstrap()
    rho_t = np.zeros((n_inst, 1, 1), np.complex128)
    seen = np.zeros((n_inst, nt, 1, 1), np.complex128)
    for T in range(6, nt):
        pk.hkbe_set_hamiltonian_at(b.h, T, w["eps"][:, T + 1])
        b.step(1)
        pk.hkbe_get_density_at(b.h, T, rho_t)
        seen[:, T] = rho_t
    ra, rb = a.density(), b.density()
    assert np.array_equal(ra, rb)
    assert np.array_equal(seen[:, 6:], rb[:, 6:])
    for t in (0, 3, 40, nt - 1):        # also from compressed leaves
        pk.hkbe_get_density_at(b.h, t, rho_t)
        assert np.array_equal(rho_t, rb[:, t])
    with pytest.raises(pk.HKBEError):
        pk.hkbe_set_hamiltonian_at(b.h, nt - 1, w["eps"][:, nt])   # already computed
    with pytest.raises(pk.HKBEError):
        pk.hkbe_get_density_at(b.h, nt, rho_t)
