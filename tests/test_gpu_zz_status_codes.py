"""Failure detection through status codes, with the failures made on the host
(no GPU fault): a forced non-convergence (one iteration, tolerance 0) returns
HKBE_ERR_NOCONV while keeping the state and advancing the step counter, and a
NaN in a host-supplied eps(t) or drive is refused with HKBE_ERR_NAN before it
reaches the device.  The file sorts after the parity files."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk

pytestmark = pytest.mark.gpu

NOCONV, NAN = -3, -6


def _setup(max_iter, tol):
    w = wk.bethe_workload(nt=40, h=0.05, k=3, beta=5.0, n_inst=2, seed=2)
    st = pk.Stepper(40, 0.05, 3, 5.0, n_inst=2, tol=tol, max_iter=max_iter)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    return w, st


def test_forced_nonconvergence_keeps_state():
    _, st = _setup(max_iter=1, tol=0.0)
    with pytest.raises(pk.HKBEError) as e:
        st.bootstrap(max_iter=1)
    assert e.value.code == NOCONV
    assert pk.hkbe_current_step(st.h) == 3                 # the start square is kept
    it, er, rc = pk.hkbe_step(st.h, 2, 5, check=False)
    assert rc == NOCONV and pk.hkbe_current_step(st.h) == 8
    assert (it == 1).all() and (er > 0).all() and np.isfinite(er).all()
    gr, gl = st.row(1, 8)
    assert np.isfinite(gr).all() and np.isfinite(gl).all()


def test_nan_inputs_are_refused_on_the_host():
    w, st = _setup(max_iter=50, tol=1e-12)
    bad = w["eps"].copy()
    bad[1, 7, 0, 0] = np.nan
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_set_hamiltonian(st.h, bad)
    assert e.value.code == NAN
    A = np.zeros((2, 41))
    A[0, 3] = np.inf
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_set_drive(st.h, A, None)
    assert e.value.code == NAN
    st.bootstrap()
    st.step(2)
    eps_t = np.zeros((2, 1, 1), np.complex128)
    eps_t[0, 0, 0] = complex(np.nan, 0)
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_set_hamiltonian_at(st.h, 10, eps_t)
    assert e.value.code == NAN
    st.step(3)                                              # the refused inputs changed nothing
    assert np.isfinite(st.row(0, 8)[0]).all()
