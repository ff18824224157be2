"""The allocation-free entry point hkbe_lesser_column_noalloc.

Callers that cannot allocate device memory (they cannot create a handle)
pass in buffers they own; the entry point keeps its scratch in a static
device array.  This test feeds it the state of a finished handle-based
propagation and checks, on two calls in a row that share the array, that it
reproduces the lesser column G^<(., T) which hkbe_step computed, within the
1e-10 relative bound used by the other parity tests; for two orbitals (the
Nambu model, whose scratch offsets and kernel variants differ) it compares
with hkbe_step and with the FP64 oracle directly, one call on a non-default
stream.  It also checks that sizes beyond the array are refused.  The file
name makes pytest collect it last.
"""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk

pytestmark = pytest.mark.gpu

BETA = 5.0


def _tri(A):
    """Lower-triangular rows A[T, 0..T] packed as in the handle layout."""
    return np.ascontiguousarray(np.concatenate([A[T, :T + 1] for T in range(A.shape[0])]))


def test_lesser_column_noalloc_matches_step():
    torch = pytest.importorskip("torch")
    nt, h, k = 64, 0.05, 5
    w = wk.bethe_workload(nt=nt, h=h, k=k, beta=BETA, seed=2)
    st = pk.Stepper(nt, h, k, BETA, tol=1e-13, max_iter=60)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    st.run()
    GR, GL, GTV = st.dense(0)
    st.close()
    # Bethe lattice: Sigma = v^2 G with v = 1
    e0, _, rev, q, _ = pk.hkbe_dlr_matrices(w["tau"], w["omega"], BETA)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_gr, d_sr, d_sl = dev(_tri(GR)), dev(_tri(GR)), dev(_tri(GL))
    d_gtv, d_stv = dev(GTV), dev(GTV)
    d_eps = dev(w["eps"][0])
    d_e0, d_rev, d_q = dev(e0), dev(rev), dev(q)
    d_gl = torch.zeros_like(d_sl)
    r = len(w["tau"])
    for T in (nt - 1, nt - 2):
        pk.hkbe_lesser_column_noalloc(nt, k, 1, r, h, T, d_gr.data_ptr(), d_sr.data_ptr(), d_sl.data_ptr(),
                                      d_gtv.data_ptr(), d_stv.data_ptr(), d_eps.data_ptr(), d_e0.data_ptr(),
                                      d_rev.data_ptr(), d_q.data_ptr(), d_gl.data_ptr())
        torch.cuda.synchronize()
        off = T * (T + 1) // 2
        out = d_gl[off:off + T + 1].cpu().numpy()
        ref = GL[T, :T + 1]
        assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max(), T


def test_lesser_column_noalloc_two_orbitals_on_a_stream():
    """Nambu model at U = 0, undriven (Sigma = v^2 s_z G s_z, Eq. Hybrid with
    A = 0): the column from the entry point against hkbe_step's and the
    oracle's, the second call queued on a non-default CUDA stream."""
    torch = pytest.importorskip("torch")
    from oracle.kbe import from_workload
    nt, h, k = 48, 0.05, 5
    w = wk.nambu_workload(nt=nt, h=h, k=k, beta=BETA, eps0=0.2, v=1.0, A0=0.0, U=0.0)
    st = pk.Stepper(nt, h, k, BETA, nao=2, tol=1e-13, max_iter=60)
    mid, mp = pk.model_params_for(w)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    pk.hkbe_set_drive(st.h, w["drive_A"], w["drive_U"])
    st.run()
    GR, GL, GTV = st.dense(0)
    st.close()
    o = from_workload(w, tol=1e-13)
    o.run()
    sz = np.array([1.0, -1.0])
    sig = lambda G: G * np.multiply.outer(sz, sz)              # noqa: E731  v^2 s_i s_j G_ij, v = 1
    e0, _, rev, q, _ = pk.hkbe_dlr_matrices(w["tau"], w["omega"], BETA)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_gr, d_sr, d_sl = dev(_tri(GR)), dev(_tri(sig(GR))), dev(_tri(sig(GL)))
    d_gtv, d_stv = dev(GTV), dev(sig(GTV))
    d_eps = dev(w["eps"][0])
    d_e0, d_rev, d_q = dev(e0), dev(rev), dev(q)
    d_gl = torch.zeros_like(d_sl)
    r = len(w["tau"])
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for T, stream in ((nt - 1, None), (nt - 3, side)):
        pk.hkbe_lesser_column_noalloc(nt, k, 2, r, h, T, d_gr.data_ptr(), d_sr.data_ptr(), d_sl.data_ptr(),
                                      d_gtv.data_ptr(), d_stv.data_ptr(), d_eps.data_ptr(), d_e0.data_ptr(),
                                      d_rev.data_ptr(), d_q.data_ptr(), d_gl.data_ptr(),
                                      stream=None if stream is None else stream.cuda_stream)
        (stream or torch.cuda.current_stream()).synchronize()
        off = T * (T + 1) // 2
        out = d_gl[off:off + T + 1].cpu().numpy()
        for ref in (GL[T, :T + 1], o.GLs[T, :T + 1]):
            assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max(), T


def test_lesser_column_noalloc_rejects_oversize():
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_lesser_column_noalloc(70000, 5, 1, 30, 0.01, 10, *([1] * 10))
    assert e.value.code == -1
    assert "static array" in str(e.value)
