"""CPU checks of the C ABI: the library loads, exports every symbol the
header declares, and its host-side set-up numerics (Appendix A weights, DLR
matrices) agree with the oracle's independent constructions.  No device work."""
import os
import re

import numpy as np
import pytest

import kbe_workloads as wk
import paper_2604_05319_gb300 as pk
from oracle.dlr import DLROracle, kernel
from oracle.weights import Weights

HDR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "hkbe.h")


def declared_symbols():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hkbe_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = pk.load()
    syms = declared_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(L, s), s


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_weights_match_oracle(k):
    a, om, D, I0 = pk.hkbe_weights(k)
    W = Weights(k)
    assert np.abs(a - W.a).max() < 1e-14
    assert np.abs(om - W.omega).max() < 1e-14
    assert np.abs(D - W.D).max() < 1e-12
    for n in range(k + 1):
        assert np.abs(I0[n] - W.I(0, n)).max() < 1e-13
    for n in range(0, 4 * k + 4):
        assert np.abs(pk.hkbe_rule(k, n) - W.rule(n)).max() < 1e-13


@pytest.mark.parametrize("beta,lam", [(5.0, 100.0), (50.0, 200.0)])
def test_dlr_matrices_agree_on_dlr_functions(beta, lam):
    t, o = wk.dlr_grid(lam, 1e-10, beta)
    e0, eb, rev, q, phi = pk.hkbe_dlr_matrices(t, o, beta)
    d = DLROracle(t, o, beta)
    rng = np.random.default_rng(1)
    for _ in range(10):
        w1, w2 = rng.uniform(-0.9 * lam / beta, 0.9 * lam / beta, 2)
        f = kernel(t, [w1], beta)[:, 0]
        g = kernel(t, [w2], beta)[:, 0]
        # evaluation at 0, beta and on the reversed grid
        assert abs(e0 @ f - kernel([0.0], [w1], beta)[0, 0]) < 1e-12
        assert abs(eb @ f - kernel([beta], [w1], beta)[0, 0]) < 1e-12
        assert np.abs(rev @ f - kernel(beta - t, [w1], beta)[:, 0]).max() < 1e-9   # 10 eps_dlr
        # product integral against the closed form
        s = w1 + w2
        ex = -np.expm1(-beta * s) / s / ((1 + np.exp(-beta * w1)) * (1 + np.exp(-beta * w2)))
        assert abs(f @ q @ g - ex) < 1e-10 * beta
        assert np.abs(np.einsum("a,aci,c->i", f, phi, g)
                      - np.einsum("a,aci,c->i", f, d.phi(), g)).max() < 1e-12


def test_create_rejects_bad_arguments_without_gpu():
    # argument validation happens before any device call
    for bad in [dict(k=0), dict(k=6), dict(nao=5), dict(nt=3, k=3), dict(n_inst=0)]:
        p = dict(nt=16, k=2, nao=1, xi=-1, n_inst=1, rho_mode=0, precision=0, max_iter=10,
                 h=0.1, beta=1.0, tol=1e-10)
        p.update(bad)
        with pytest.raises(pk.HKBEError) as e:
            pk.hkbe_create(pk.hkbe_params(**p))
        assert e.value.code == -1


def test_create_rejects_split_precision_and_bad_nt_per_inst_without_gpu():
    """Precision modes 2 and 3 (split-operand tensor-core forms) are refused
    with the reason; a per-instance N_t outside k+2..nt is refused."""
    base = dict(nt=16, k=2, nao=1, xi=-1, n_inst=3, rho_mode=0, precision=0, max_iter=10, h=0.1, beta=1.0,
                tol=1e-10)
    for prec in (pk.PREC_TF32X3, pk.PREC_BF16X3):
        with pytest.raises(pk.HKBEError) as e:
            pk.hkbe_create(pk.hkbe_params(**dict(base, precision=prec)))
        assert e.value.code == pk.HKBE_ERR_ARG and "matrix-vector" in str(e.value)
    for bad in ([16, 16, 17], [16, 3, 16]):
        with pytest.raises(pk.HKBEError) as e:
            pk.hkbe_create(pk.hkbe_params(**base), nt_per_inst=bad)
        assert e.value.code == pk.HKBE_ERR_ARG and "nt_per_inst" in str(e.value)
    with pytest.raises(ValueError):
        pk.hkbe_create(pk.hkbe_params(**base), nt_per_inst=[16, 16])


def _fnv_words(data):
    """FNV-1a 64 over little-endian 64-bit words, the last one zero-padded
    (the checkpoint trailer's definition in include/hkbe.h)."""
    import struct
    h = 14695981039346656037
    data = bytes(data) + b"\0" * (-len(data) % 8)
    for (w,) in struct.iter_unpack("<Q", data):
        h = ((h ^ w) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def test_checkpoint_load_refuses_bad_files_without_gpu(tmp_path):
    """hkbe_load checks the file's magic, version and header before any
    device call; hkbe_save and hkbe_load reject null arguments."""
    import ctypes as C
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_load(str(tmp_path / "missing.ckp"))
    assert e.value.code == pk.HKBE_ERR_IO
    (tmp_path / "junk.ckp").write_bytes(b"not a checkpoint file at all")
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_load(str(tmp_path / "junk.ckp"))
    assert e.value.code == pk.HKBE_ERR_IO and "magic" in str(e.value)
    p = pk.hkbe_params(nt=16, k=2, nao=1, xi=-1, n_inst=1, rho_mode=0, precision=0, max_iter=10,
                       h=0.1, beta=1.0, tol=1e-10)
    head = b"HKBECKP1" + (2).to_bytes(4, "little") + C.sizeof(p).to_bytes(4, "little") + bytes(p)
    (tmp_path / "short.ckp").write_bytes(head[:-3])
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_load(str(tmp_path / "short.ckp"))
    assert e.value.code == pk.HKBE_ERR_IO
    # scalars cur, have_dlr, have_gm, have_eps, have_model, self_consistent, model, r, cdir,
    # nfrozR, nfrozL, pad: a grid of r = 200 nodes is out of range
    sc = np.array([-1, 1, 0, 0, 0, 1, 1, 200, 0, 0, 0, 0], np.int32).tobytes()
    body = head + sc
    (tmp_path / "badhead.ckp").write_bytes(body + _fnv_words(body).to_bytes(8, "little"))
    with pytest.raises(pk.HKBEError) as e:      # the checksum passes; the header is refused
        pk.hkbe_load(str(tmp_path / "badhead.ckp"))
    assert e.value.code == pk.HKBE_ERR_IO and "inconsistent" in str(e.value)
    flipped = bytearray(body)
    flipped[40] ^= 0x10                          # one bit of the parameters
    (tmp_path / "flipped.ckp").write_bytes(bytes(flipped) + _fnv_words(body).to_bytes(8, "little"))
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_load(str(tmp_path / "flipped.ckp"))
    assert e.value.code == pk.HKBE_ERR_IO and "checksum" in str(e.value)
    # a version-1 file (before the checksum trailer and the per-instance N_t) gets the version error
    (tmp_path / "v1.ckp").write_bytes(b"HKBECKP1" + (1).to_bytes(4, "little") + head[12:] + sc)
    with pytest.raises(pk.HKBEError) as e:
        pk.hkbe_load(str(tmp_path / "v1.ckp"))
    assert e.value.code == pk.HKBE_ERR_IO and "version" in str(e.value)
    assert pk.load().hkbe_save(None, b"x") == -1
    assert pk.load().hkbe_load(None, None, None) == -1
