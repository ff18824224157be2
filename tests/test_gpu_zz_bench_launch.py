"""Parity in the bench's own launch configuration: the C2-batch handle at
full size (304 instances, N_t = 4096 allocated, HODLR leaf 64, eps_SVD 1e-8,
mixed form, self-consistency tolerance 1e-7, r_max 64), propagated over its
first 280 steps, which span the level quench at t = 5 (step 250) and four
compressed leaves.  A sampled instance with a quench amplitude other than 1 is
compared element by element with the FP64 oracle on the same inputs (bar: the
mixed form's 1e-6 relative).  Every instance is checked for properties that
hold at any size: the instances' inputs are equal before the quench, so their
rows agree there to the mixed form's rounding (each is within 1e-6 of the
same FP64 solution, so two are within 2e-6: complex64 storage does not make
them bitwise equal across instances, measured 2.3e-8); G^R(T, T) = -i; every
row is finite; instances with other amplitudes differ after the quench.
The file name keeps it after the other GPU parity files: it runs the
largest handle of the suite."""
import numpy as np
import pytest

import paper_2604_05319_gb300 as pk
from oracle.kbe import from_workload

pytestmark = pytest.mark.gpu

N_INST, NT_CHECK, SAMPLE, T_QUENCH = 304, 281, 303, 250


def test_c2_batch_full_size_first_steps():
    import kbe_workloads as wk                        # the bench's own inputs
    w = wk.c2_batch_workload(N_INST)                  # N_t = 4096
    wl = w["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=1, n_inst=N_INST, rho_mode=wl.rho_mode,
                    max_iter=wl.max_iter, tol=1e-7, precision=pk.PREC_MIXED, svd_tol=wl.svd_tol,
                    leaf=wl.leaf, r_max=64)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.bootstrap()
    st.step(NT_CHECK - 1 - wl.k)
    T = NT_CHECK - 1
    assert pk.hkbe_get_ranks(st.h, SAMPLE, 0, len(pk.hkbe_get_blocks(st.h)["r0"]), 1)[1] == 256

    ws = wk.c2_batch_workload(N_INST, nt=NT_CHECK)          # the same inputs on the first NT_CHECK steps
    assert np.array_equal(ws["eps"], w["eps"][:, :NT_CHECK + 1])
    assert np.all(ws["eps"][:, :T_QUENCH + 1] == ws["eps"][0, :T_QUENCH + 1])
    o = from_workload(ws, inst=SAMPLE, tol=1e-13)
    o.run()
    GR, GL, GTV = st.dense(SAMPLE)
    idx = np.tril_indices(NT_CHECK)
    ref = max(np.abs(o.GR[idx]).max(), np.abs(o.GLs[idx]).max(), np.abs(o.GTV).max())
    err = max(np.abs(GR[idx] - o.GR[idx]).max(), np.abs(GL[idx] - o.GLs[idx]).max(),
              np.abs(GTV - o.GTV).max()) / ref
    assert err < 1e-6, err

    before = T_QUENCH - 1
    r0 = st.row(0, before)
    for n in range(N_INST):
        gr, gl = st.row(n, before)
        assert np.abs(gr - r0[0]).max() < 2e-6 * ref and np.abs(gl - r0[1]).max() < 2e-6 * ref, n
        gr, gl = st.row(n, T)
        assert np.isfinite(gr).all() and np.isfinite(gl).all(), n
        assert abs(gr[T, 0, 0] + 1j) < 1e-12, n
    assert np.abs(st.row(0, T)[0] - GR[T]).max() > 1e-2    # amplitude 1 vs 0.54 after the quench
