"""Checkpoint files (hkbe_save / hkbe_load, the paper's checkpoint files of
Sec. 3.6), a caller-supplied start square (hkbe_set_initial_slices) and
hkbe_get_observables, through the C ABI.  A loaded handle continues the saved
run bit for bit, in the dense FP64 and the compressed mixed forms, and
rewinds to the same bootstrap.  A start square read back from a bootstrapped
handle and given to a fresh one propagates the same way.  A damaged file is
refused with HKBE_ERR_IO."""
import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk

pytestmark = pytest.mark.gpu

NT, H, K, NI = 160, 0.02, 5, 2
CASES = [(0.0, pk.PREC_FP64), (1e-8, pk.PREC_MIXED)]


def _workload():
    w = wk.bethe_workload(nt=NT, h=H, k=K, beta=5.0, n_inst=NI, seed=11, quench=(0.0, 1.0, 1.0))
    w["eps"][:, 1:, 0, 0] *= np.array([0.7, 1.3])[:, None]
    return w


def _stepper(w, svd_tol, prec):
    mid, mp = pk.model_params_for(w)
    st = pk.Stepper(NT, H, K, 5.0, n_inst=NI, tol=1e-12 if prec == pk.PREC_FP64 else 1e-7, max_iter=60,
                    precision=prec, svd_tol=svd_tol, leaf=32, r_max=64)
    st.set_inputs(w["tau"], w["omega"], w["gm"], w["eps"], mid, mp)
    return st


def _wrap(handle, like):
    st = pk.Stepper.__new__(pk.Stepper)
    st.p, st.nao, st.n_inst, st.nt, st.r, st.h = like.p, like.nao, like.n_inst, like.nt, like.r, handle
    return st


def _rows(st, T1):
    return [(*st.row(n, T), st.tv(n, T)) for n in range(st.n_inst) for T in range(T1 + 1)]


def _max_diff(a, b):
    return max(float(np.abs(x - y).max()) for ra, rb in zip(a, b) for x, y in zip(ra, rb))


def _ranks(st):
    nblk = len(pk.hkbe_get_blocks(st.h)["r0"])
    return [pk.hkbe_get_ranks(st.h, n, c, nblk, 1) for n in range(NI) for c in range(4)]


@pytest.mark.parametrize("svd_tol,prec", CASES)
def test_save_load_continues_bit_for_bit(tmp_path, svd_tol, prec):
    w = _workload()
    a = _stepper(w, svd_tol, prec)
    a.bootstrap()
    a.step(90)                                   # T = 95: rows below 64 are compressed (leaf 32)
    path = str(tmp_path / "run.ckp")
    pk.hkbe_save(a.h, path)
    b = _wrap(pk.hkbe_load(path), a)
    assert pk.hkbe_current_step(b.h) == 95
    assert pk.hkbe_get_stats(b.h) == pk.hkbe_get_stats(a.h)
    a.step(NT - 1 - 95)
    b.step(NT - 1 - 95)
    ra = _rows(a, NT - 1)
    assert _max_diff(ra, _rows(b, NT - 1)) == 0.0
    assert np.array_equal(a.density(), b.density())
    if svd_tol:
        assert all(np.array_equal(x[0], y[0]) and x[1] == y[1] for x, y in zip(_ranks(a), _ranks(b)))
    pk.hkbe_rewind(b.h)                          # the bootstrap snapshot is part of the file
    b.step(NT - 1 - K)
    assert _max_diff(ra, _rows(b, NT - 1)) <= (1e-13 if prec == pk.PREC_FP64 else 1e-9)
    b.close()


@pytest.mark.parametrize("svd_tol,prec", CASES)
def test_initial_slices_reproduce_the_bootstrap(svd_tol, prec):
    w = _workload()
    a = _stepper(w, svd_tol, prec)
    a.bootstrap()
    nsq = (K + 1) * (K + 2) // 2
    gr = np.zeros((NI, nsq, 1, 1), np.complex128)
    gl = np.zeros_like(gr)
    gtv = np.zeros((NI, K + 1, a.r, 1, 1), np.complex128)
    for n in range(NI):
        o = 0
        for t in range(K + 1):
            gr[n, o:o + t + 1], gl[n, o:o + t + 1] = a.row(n, t)
            gtv[n, t] = a.tv(n, t)
            o += t + 1
    b = _stepper(w, svd_tol, prec)
    pk.hkbe_set_initial_slices(b.h, gr, gl, gtv)
    assert pk.hkbe_current_step(b.h) == K
    with pytest.raises(pk.HKBEError):
        b.bootstrap()
    with pytest.raises(pk.HKBEError):
        pk.hkbe_set_initial_slices(b.h, gr, gl, gtv)
    a.step(100)
    b.step(100)
    d = _max_diff(_rows(a, K + 100), _rows(b, K + 100))
    assert d <= (1e-12 if prec == pk.PREC_FP64 else 1e-6), d
    c = _stepper(w, svd_tol, prec)
    bad = gtv.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(pk.HKBEError):
        pk.hkbe_set_initial_slices(c.h, gr, gl, bad)


def test_get_observables():
    w = _workload()
    a = _stepper(w, 0.0, pk.PREC_FP64)
    a.bootstrap()
    a.step(10)
    rho, ek, cu = pk.hkbe_get_observables(a.h, 12, NI, 1)
    ref = np.zeros((NI, 1, 1), np.complex128)
    pk.hkbe_get_density_at(a.h, 12, ref)
    assert np.array_equal(rho, ref) and ek is None and cu is None
    with pytest.raises(pk.HKBEError):           # E_kin and j exist for the lattice model only
        pk.hkbe_get_observables(a.h, 12, NI, 1, lattice=True)
    with pytest.raises(pk.HKBEError):
        pk.hkbe_get_observables(a.h, 16, NI, 1)
    lw = wk.lattice_workload(L=2, nt=30, h=0.025, k=5, beta=10.0, U=2.0, t_quench=0.2, A0=0.5, Omega=1.2,
                             tc=0.3, width=0.2)
    wl = lw["wl"]
    st = pk.Stepper(wl.nt, wl.h, wl.k, wl.beta, nao=1, n_inst=4, tol=1e-13, max_iter=80)
    mid, mp = pk.model_params_for(lw)
    st.set_inputs(lw["tau"], lw["omega"], lw["gm"], lw["eps"], mid, mp)
    pk.hkbe_set_drive(st.h, lw["drive_A"], lw["drive_U"])
    st.run()
    ref = np.zeros((4, 1, 1), np.complex128)
    for t in (0, 12, wl.nt - 1):
        rho, ek, cu = pk.hkbe_get_observables(st.h, t, 4, 1, lattice=True)
        ob = pk.hkbe_get_lattice_observables(st.h, t)
        pk.hkbe_get_density_at(st.h, t, ref)
        assert ek == ob[1] and cu == ob[2] and np.array_equal(rho, ref)


def test_damaged_checkpoint_is_refused(tmp_path):
    w = _workload()
    a = _stepper(w, 1e-8, pk.PREC_MIXED)
    a.bootstrap()
    a.step(40)
    path = tmp_path / "run.ckp"
    pk.hkbe_save(a.h, str(path))
    data = path.read_bytes()
    (tmp_path / "short.ckp").write_bytes(data[:len(data) // 2])
    (tmp_path / "long.ckp").write_bytes(data + b"\0")
    for name in ("short.ckp", "long.ckp"):
        with pytest.raises(pk.HKBEError) as e:
            pk.hkbe_load(str(tmp_path / name))
        assert e.value.code == pk.HKBE_ERR_IO
    b = pk.hkbe_load(str(path))                  # the intact file still loads
    assert pk.hkbe_current_step(b) == 45
    pk.hkbe_destroy(b)
