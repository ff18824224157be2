"""Per-instance N_t (hkbe_create's nt_per_inst): a batch whose instances end
at different steps, stepped together, each compared with its own FP64 oracle
run of its own length, in the dense FP64 form (1e-10) and in the compressed
complex64 form (1e-6 relative).  After an instance's last step it takes no
part (zero iterations), its rows stay readable up to its end (the compressed
ones through the frozen compression front), reads past its end are refused
(HKBE_ERR_RANGE), and its density matrix reads as zero there."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.kbe import from_workload

pytestmark = pytest.mark.gpu
BETA = 5.0


@pytest.mark.parametrize("prec,svd_tol,bound", [(pk.PREC_FP64, 0.0, 1e-10), (pk.PREC_MIXED, 1e-8, 1e-6)])
def test_uneven_batch_against_per_instance_oracles(prec, svd_tol, bound):
    nt, h, k = 320, 0.02, 5
    nts = [121, 200, 320]
    ws = [wk.bethe_workload(nt=nt, h=h, k=k, beta=BETA, seed=s, quench=(0.0, 0.5 + 0.25 * s, 3.0))
          for s in (1, 2, 3)]
    st = pk.Stepper(nt, h, k, BETA, n_inst=3, tol=1e-13 if prec == pk.PREC_FP64 else 1e-7, max_iter=60,
                    svd_tol=svd_tol, leaf=32, r_max=64, precision=prec, nt_per_inst=nts)
    mid, _ = pk.model_params_for(ws[0])
    mp = np.concatenate([pk.model_params_for(w)[1] for w in ws])
    st.set_inputs(ws[0]["tau"], ws[0]["omega"], np.concatenate([w["gm"] for w in ws]),
                  np.concatenate([w["eps"] for w in ws]), mid, mp)
    st.bootstrap()
    iters, _ = st.step(nt - 1 - k)
    for i, n_i in enumerate(nts):
        assert (iters[n_i - 1 - k:, i] == 0).all() and (iters[:n_i - 1 - k, i] > 0).all(), i
        wi = wk.bethe_workload(nt=n_i, h=h, k=k, beta=BETA, seed=i + 1, quench=(0.0, 0.75 + 0.25 * i, 3.0))
        assert np.array_equal(wi["eps"][0], ws[i]["eps"][0, :n_i + 1])   # the same inputs, cut at N_t,i
        o = from_workload(wi, tol=1e-13)
        o.run()
        ref = max(np.abs(o.GR).max(), np.abs(o.GLs).max())
        err = 0.0
        for T in range(n_i):
            gr, gl = st.row(i, T)
            err = max(err, np.abs(gr - o.GR[T, :T + 1]).max(), np.abs(gl - o.GLs[T, :T + 1]).max())
        assert err < bound * ref, (i, err)
        if n_i < nt:
            with pytest.raises(pk.HKBEError) as e:
                st.row(i, n_i)
            assert e.value.code == pk.HKBE_ERR_RANGE
    rho = np.zeros((3, 1, 1), np.complex128)
    pk.hkbe_get_density_at(st.h, nt - 1, rho)
    assert rho[0, 0, 0] == 0 and rho[1, 0, 0] == 0 and abs(rho[2, 0, 0]) > 0
    if svd_tol > 0:                     # the finished instances froze their compression front
        nb = len(pk.hkbe_get_blocks(st.h)["r0"])
        fronts = [pk.hkbe_get_ranks(st.h, i, 0, nb, 1)[1] for i in range(3)]
        assert fronts[0] == 32 * ((nts[0] - 1 - k) // 32) and fronts[0] < fronts[1] < fronts[2]
    st.close()
