"""Python binding of libhkbe, the GB300 Kadanoff-Baym time stepper.

The functions mirror the C ABI of ``include/hkbe.h`` one to one (same names,
same argument order); they only marshal numpy arrays to host pointers and turn
negative status codes into ``HKBEError``.  All computation happens in the CUDA
library; there is no Python fallback: importing works without a GPU (for the
host-only utilities), but any stepping call needs the CUDA library and a GPU
and raises otherwise.

``Stepper`` is a thin convenience wrapper owning a handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

HKBE_OK = 0
HKBE_ERR_ARG, HKBE_ERR_CUDA, HKBE_ERR_NOCONV, HKBE_ERR_RANGE, HKBE_ERR_RANK = -1, -2, -3, -4, -5
HKBE_ERR_NAN, HKBE_ERR_NOMEM, HKBE_ERR_IO = -6, -7, -8
ERRORS = {-1: "HKBE_ERR_ARG", -2: "HKBE_ERR_CUDA", -3: "HKBE_ERR_NOCONV", -4: "HKBE_ERR_RANGE",
          -5: "HKBE_ERR_RANK", -6: "HKBE_ERR_NAN", -7: "HKBE_ERR_NOMEM", -8: "HKBE_ERR_IO"}
MODEL_NONE, MODEL_BETHE, MODEL_BATH, MODEL_NAMBU, MODEL_LATTICE2B = 0, 1, 2, 3, 4
PREC_FP64 = 0
PREC_MIXED = 1
PREC_TF32X3 = 2   # rejected by hkbe_create (no dense contraction on this path)
PREC_BF16X3 = 3   # rejected by hkbe_create


class HKBEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class hkbe_params(C.Structure):
    _fields_ = [("nt", C.c_int32), ("k", C.c_int32), ("nao", C.c_int32), ("xi", C.c_int32),
                ("n_inst", C.c_int32), ("rho_mode", C.c_int32), ("precision", C.c_int32),
                ("max_iter", C.c_int32), ("h", C.c_double), ("beta", C.c_double), ("tol", C.c_double),
                ("svd_tol", C.c_double), ("leaf", C.c_int32), ("r_max", C.c_int32)]


_lib = None
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)


def lib_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhkbe.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libhkbe.so is not built; run __graft_entry__.build()")
    L = C.CDLL(_build.LIB)
    H = C.c_void_p
    sig = {
        "hkbe_create": ([C.POINTER(hkbe_params), _I, C.c_void_p, C.POINTER(H)], C.c_int),
        "hkbe_destroy": ([H], C.c_int),
        "hkbe_last_error": ([H], C.c_char_p),
        "hkbe_set_dlr": ([H, C.c_int, _D, _D], C.c_int),
        "hkbe_set_matsubara": ([H, _D], C.c_int),
        "hkbe_set_hamiltonian": ([H, _D], C.c_int),
        "hkbe_set_hamiltonian_at": ([H, C.c_int, C.c_void_p], C.c_int),
        "hkbe_get_density_at": ([H, C.c_int, C.c_void_p], C.c_int),
        "hkbe_set_model": ([H, C.c_int, _D, C.c_int], C.c_int),
        "hkbe_set_drive": ([H, _D, _D], C.c_int),
        "hkbe_get_lattice_observables": ([H, C.c_int, _D], C.c_int),
        "hkbe_matsubara_solve": ([C.c_int, _D, _D, C.c_double, C.c_int, C.c_int, C.c_int, _D, _D, C.c_int,
                                  C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, _D, _D,
                                  _I, _D], C.c_int),
        "hkbe_solve_matsubara": ([H, C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, C.c_int, _D, _I, _D],
                                 C.c_int),
        "hkbe_set_scheme": ([H, C.c_int], C.c_int),
        "hkbe_bootstrap": ([H, C.c_int, C.c_double, _I, _D], C.c_int),
        "hkbe_set_initial_slices": ([H, _D, _D, _D], C.c_int),
        "hkbe_get_observables": ([H, C.c_int, _D, _D, _D], C.c_int),
        "hkbe_save": ([H, C.c_char_p], C.c_int),
        "hkbe_load": ([C.c_char_p, C.c_void_p, C.POINTER(H)], C.c_int),
        "hkbe_step": ([H, C.c_int, _I, _D], C.c_int),
        "hkbe_current_step": ([H, _I], C.c_int),
        "hkbe_get_ret": ([H, C.c_int, C.c_int, C.c_int, _D], C.c_int),
        "hkbe_get_les": ([H, C.c_int, C.c_int, C.c_int, _D], C.c_int),
        "hkbe_get_tv": ([H, C.c_int, C.c_int, _D], C.c_int),
        "hkbe_get_row": ([H, C.c_int, C.c_int, _D, _D], C.c_int),
        "hkbe_get_density": ([H, _D], C.c_int),
        "hkbe_get_stats": ([H, C.c_int, _I, C.POINTER(C.c_size_t)], C.c_int),
        "hkbe_rewind": ([H], C.c_int),
        "hkbe_snapshot_save": ([H], C.c_int),
        "hkbe_snapshot_restore": ([H], C.c_int),
        "hkbe_snapshot_free": ([H], C.c_int),
        "hkbe_fma_peaks": ([_D, _D], C.c_int),
        "hkbe_f32_of": ([C.c_int, _D, C.c_void_p], C.c_int),
        "hkbe_get_blocks": ([H, _I, _I, _I, _I, _I, _I], C.c_int),
        "hkbe_get_ranks": ([H, C.c_int, C.c_int, _I, _I], C.c_int),
        "hkbe_set_profiling": ([H, C.c_int], C.c_int),
        "hkbe_get_timing": ([H, C.c_int, _D, C.POINTER(C.c_int64)], C.c_int),
        "hkbe_reset_counters": ([H], C.c_int),
        "hkbe_weights": ([C.c_int, _D, _D, _D, _D], C.c_int),
        "hkbe_rule": ([C.c_int, C.c_int, _D], C.c_int),
        "hkbe_hodlr_partition": ([C.c_int, C.c_int, _I, _I, _I, _I, _I, _I], C.c_int),
        "hkbe_dlr_matrices": ([C.c_int, _D, _D, C.c_double, C.c_int, _D, _D, _D, _D, _D], C.c_int),
        "hkbe_lesser_column_noalloc": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int]
                                       + [C.c_void_p] * 6 + [C.c_void_p] * 3
                                       + [C.c_void_p, C.c_void_p, C.c_char_p, C.c_size_t], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _ip(a):
    if a is None:
        return None
    return a.ctypes.data_as(_I)


def _cplx(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128).reshape(shape))
    return a.view(np.float64)


def _check(rc, h=None):
    if rc != HKBE_OK:
        msg = load().hkbe_last_error(h).decode()
        raise HKBEError(rc, msg)


# ---- one-to-one wrappers of the C ABI -------------------------------------

def hkbe_create(params: hkbe_params, stream=None, nt_per_inst=None):
    """nt_per_inst: None (every instance runs params.nt steps) or one N_t per instance."""
    h = C.c_void_p()
    ntp = None
    if nt_per_inst is not None:
        ntp = np.ascontiguousarray(nt_per_inst, dtype=np.int32)
        if ntp.shape != (params.n_inst,):
            raise ValueError("nt_per_inst needs one entry per instance")
    _check(load().hkbe_create(C.byref(params), None if ntp is None else _ip(ntp), stream, C.byref(h)), None)
    return h


def hkbe_destroy(h):
    load().hkbe_destroy(h)


def hkbe_set_dlr(h, tau, omega):
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    _check(load().hkbe_set_dlr(h, len(tau), _dp(tau), _dp(om)), h)


def hkbe_set_matsubara(h, gm):
    g = _cplx(gm, np.shape(gm))
    _check(load().hkbe_set_matsubara(h, _dp(g)), h)


def hkbe_set_hamiltonian(h, eps):
    e = _cplx(eps, np.shape(eps))
    _check(load().hkbe_set_hamiltonian(h, _dp(e)), h)


def hkbe_set_model(h, model, params):
    p = np.ascontiguousarray(np.atleast_2d(np.asarray(params, dtype=np.float64))) if params is not None else None
    npar = 0 if p is None else p.shape[1]
    _check(load().hkbe_set_model(h, int(model), _dp(p), int(npar)), h)


def hkbe_bootstrap(h, n_inst, max_iter, tol):
    it = np.zeros(n_inst, np.int32)
    er = np.zeros(n_inst)
    rc = load().hkbe_bootstrap(h, int(max_iter), float(tol), _ip(it), _dp(er))
    _check(rc, h)
    return it, er


def hkbe_set_initial_slices(h, gr, gl, gtv):
    """Rows 0..k instead of the bootstrap: gr, gl complex
    [n_inst, (k+1)(k+2)/2, nao, nao] (G^R(t, s) and G^<(s, t), packed row by
    row for t = 0..k, s = 0..t), gtv complex [n_inst, k+1, r, nao, nao]."""
    a, b, c = (_cplx(x, np.shape(x)) for x in (gr, gl, gtv))
    _check(load().hkbe_set_initial_slices(h, _dp(a), _dp(b), _dp(c)), h)


def hkbe_get_observables(h, t, n_inst, nao, lattice=False):
    """(rho [n_inst, nao, nao], E_kin, j) at time t; E_kin and j only when
    `lattice` (a LATTICE2B handle), else None."""
    rho = np.zeros((n_inst, nao, nao), np.complex128)
    ek = np.zeros(1) if lattice else None
    cu = np.zeros(1) if lattice else None
    _check(load().hkbe_get_observables(h, int(t), _dp(rho.view(np.float64)), _dp(ek), _dp(cu)), h)
    return rho, (float(ek[0]) if lattice else None), (float(cu[0]) if lattice else None)


def hkbe_save(h, path):
    _check(load().hkbe_save(h, os.fsencode(path)), h)


def hkbe_load(path, stream=None):
    h = C.c_void_p()
    _check(load().hkbe_load(os.fsencode(path), stream, C.byref(h)), None)
    return h


def hkbe_step(h, n_inst, n_steps, check=True):
    it = np.zeros(max(1, n_inst * n_steps), np.int32)
    er = np.zeros(max(1, n_inst * n_steps))
    rc = load().hkbe_step(h, int(n_steps), _ip(it), _dp(er))
    if check:
        _check(rc, h)
    return it[:n_inst * n_steps].reshape(n_steps, n_inst), er[:n_inst * n_steps].reshape(n_steps, n_inst), rc


def hkbe_current_step(h):
    t = np.zeros(1, np.int32)
    _check(load().hkbe_current_step(h, _ip(t)), h)
    return int(t[0])


def hkbe_get_ret(h, nao, inst, t, tp):
    out = np.zeros((nao, nao), np.complex128)
    _check(load().hkbe_get_ret(h, inst, t, tp, _dp(out.view(np.float64))), h)
    return out


def hkbe_get_les(h, nao, inst, t, tp):
    out = np.zeros((nao, nao), np.complex128)
    _check(load().hkbe_get_les(h, inst, t, tp, _dp(out.view(np.float64))), h)
    return out


def hkbe_get_tv(h, nao, r, inst, t):
    out = np.zeros((r, nao, nao), np.complex128)
    _check(load().hkbe_get_tv(h, inst, t, _dp(out.view(np.float64))), h)
    return out


def hkbe_get_row(h, nao, inst, T):
    gr = np.zeros((T + 1, nao, nao), np.complex128)
    gl = np.zeros((T + 1, nao, nao), np.complex128)
    _check(load().hkbe_get_row(h, inst, T, _dp(gr.view(np.float64)), _dp(gl.view(np.float64))), h)
    return gr, gl


def _ptr(a):
    """Address of a host buffer: a numpy array (kept alive by the caller) or an int."""
    if isinstance(a, int):
        return C.c_void_p(a)
    return C.c_void_p(a.ctypes.data)


def hkbe_set_drive(h, A=None, U=None):
    """Nambu drive: A[n_inst, nt+1], U[n_inst, nt+1] (None: zero)."""
    a = None if A is None else np.ascontiguousarray(np.asarray(A, dtype=np.float64))
    u = None if U is None else np.ascontiguousarray(np.asarray(U, dtype=np.float64))
    _check(load().hkbe_set_drive(h, _dp(a) if a is not None else None, _dp(u) if u is not None else None), h)


def hkbe_matsubara_solve(tau, omega, beta, model, eps, params=None, U_eq=0.0, eta=0.0, n_eta=0, mix=0.5,
                         tol=1e-12, max_iter=500):
    """Self-consistent equilibrium G^M on the DLR nodes (host, no handle).
    eps: complex [n_inst, nao, nao]; params: [n_inst, nparams] or None.
    Returns (G^M [n_inst, r, nao, nao], eps with the Fock shift, iterations,
    final difference); raises HKBEError on failure or non-convergence."""
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.complex128))
    n_inst, nao = e.shape[0], e.shape[-1]
    r = len(tau)
    p = None if params is None else np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(n_inst, -1))
    gm = np.zeros((n_inst, r, nao, nao), np.complex128)
    eo = np.zeros((n_inst, nao, nao), np.complex128)
    it = np.zeros(1, np.int32)
    er = np.zeros(1)
    rc = load().hkbe_matsubara_solve(r, _dp(tau), _dp(om), float(beta), int(model), n_inst, nao,
                                     _dp(e.view(np.float64)), _dp(p) if p is not None else None,
                                     0 if p is None else p.shape[1], float(U_eq), float(eta), int(n_eta),
                                     float(mix), float(tol), int(max_iter), _dp(gm.view(np.float64)),
                                     _dp(eo.view(np.float64)), _ip(it), _dp(er))
    if rc != 0:
        raise HKBEError(rc, f"hkbe_matsubara_solve failed (rc={rc}, iterations {int(it[0])}, diff {er[0]:.3e})")
    return gm, eo, int(it[0]), float(er[0])


def hkbe_solve_matsubara(h, n_inst, r, nao, U_eq=0.0, eta=0.0, n_eta=0, mix=0.5, tol=1e-12, max_iter=500):
    """Equilibrium G^M of the handle's model solved on the device and
    installed (replaces hkbe_set_matsubara).  Returns (G^M [n_inst, r, nao,
    nao], iterations, final difference); raises HKBEError on failure or
    non-convergence."""
    gm = np.zeros((n_inst, r, nao, nao), np.complex128)
    it = np.zeros(1, np.int32)
    er = np.zeros(1)
    _check(load().hkbe_solve_matsubara(h, float(U_eq), float(eta), int(n_eta), float(mix), float(tol), int(max_iter),
                                       _dp(gm.view(np.float64)), _ip(it), _dp(er)), h)
    return gm, int(it[0]), float(er[0])


def hkbe_f32_of(x):
    """The device's integer-pipe FP64 -> FP32 rounding applied to x (float64 array)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.zeros(x.size, np.float32)
    _check(load().hkbe_f32_of(int(x.size), _dp(x), y.ctypes.data))
    return y


SCHEME_PAPER, SCHEME_SWEEP_FREE = 0, 1


def hkbe_set_scheme(h, scheme):
    _check(load().hkbe_set_scheme(h, int(scheme)), h)


def hkbe_get_lattice_observables(h, t):
    """(n, E_kin, j) of a LATTICE2B handle at time t."""
    out = np.zeros(3)
    _check(load().hkbe_get_lattice_observables(h, int(t), _dp(out)), h)
    return out


def hkbe_set_hamiltonian_at(h, t, eps_t):
    """eps(t) of every instance: complex [n_inst, nao, nao] array, or the
    address of such a buffer of interleaved doubles (e.g. pinned memory)."""
    if not isinstance(eps_t, int):
        eps_t = _cplx(eps_t, np.shape(eps_t))
    _check(load().hkbe_set_hamiltonian_at(h, int(t), _ptr(eps_t)), h)


def hkbe_get_density_at(h, t, out):
    """rho(t) of every instance into `out` (complex [n_inst, nao, nao] numpy
    array, C-contiguous, or the address of such a buffer); returns out."""
    if not isinstance(out, int) and not (out.dtype == np.complex128 and out.flags.c_contiguous):
        raise ValueError("out must be a C-contiguous complex128 array")
    _check(load().hkbe_get_density_at(h, int(t), _ptr(out)), h)
    return out


def hkbe_get_density(h, n_inst, nao, T):
    out = np.zeros((n_inst, T + 1, nao, nao), np.complex128)
    _check(load().hkbe_get_density(h, _dp(out.view(np.float64))), h)
    return out


def hkbe_get_stats(h, inst=None, nblk=0, nao=1):
    """Device bytes; with inst given (HODLR handle), also the ranks
    [4 components][nblk][nao*nao] of that instance."""
    b = C.c_size_t()
    if inst is None:
        _check(load().hkbe_get_stats(h, 0, None, C.byref(b)), h)
        return int(b.value)
    r = np.zeros(max(1, 4 * nblk * nao * nao), np.int32)
    _check(load().hkbe_get_stats(h, int(inst), _ip(r), C.byref(b)), h)
    return int(b.value), r[:4 * nblk * nao * nao].reshape(4, nblk, nao * nao)


def hkbe_rewind(h):
    _check(load().hkbe_rewind(h), h)


def hkbe_snapshot_save(h):
    _check(load().hkbe_snapshot_save(h), h)


def hkbe_snapshot_restore(h):
    _check(load().hkbe_snapshot_restore(h), h)


def hkbe_snapshot_free(h):
    _check(load().hkbe_snapshot_free(h), h)


def hkbe_fma_peaks():
    """(FP64, FP32) fused multiply-add throughput of the current device, TFLOP/s."""
    a, b = np.zeros(1), np.zeros(1)
    _check(load().hkbe_fma_peaks(_dp(a), _dp(b)))
    return float(a[0]), float(b[0])


def hkbe_get_blocks(h):
    nb = np.zeros(1, np.int32)
    _check(load().hkbe_get_blocks(h, _ip(nb), None, None, None, None, None), h)
    n = int(nb[0])
    a = [np.zeros(n, np.int32) for _ in range(5)]
    _check(load().hkbe_get_blocks(h, _ip(nb), *[_ip(x) for x in a]), h)
    return dict(zip(["r0", "r1", "c0", "c1", "level"], a))


def hkbe_get_ranks(h, inst, comp, nblk, nao):
    out = np.zeros(max(1, nblk * nao * nao), np.int32)
    fd = np.zeros(1, np.int32)
    _check(load().hkbe_get_ranks(h, inst, comp, _ip(out), _ip(fd)), h)
    return out[:nblk * nao * nao].reshape(nblk, nao * nao), int(fd[0])


def hkbe_set_profiling(h, on):
    _check(load().hkbe_set_profiling(h, int(bool(on))), h)


PHASES = ["extrap", "sigma", "ret", "mixed", "vt", "src", "les", "rho", "boot", "ctrl", "compress", "chunkinv"]


def hkbe_get_timing(h, phase):
    ms = np.zeros(1)
    n = C.c_int64()
    _check(load().hkbe_get_timing(h, int(phase), _dp(ms), C.byref(n)), h)
    return float(ms[0]), int(n.value)


def hkbe_reset_counters(h):
    _check(load().hkbe_reset_counters(h), h)


def hkbe_weights(k):
    a = np.zeros(k + 1)
    om = np.zeros(k + 1)
    D = np.zeros((k + 1) * (k + 1))
    I0 = np.zeros((k + 1) * (k + 1))
    _check(load().hkbe_weights(k, _dp(a), _dp(om), _dp(D), _dp(I0)))
    return a, om, D.reshape(k + 1, k + 1), I0.reshape(k + 1, k + 1)


def hkbe_rule(k, n):
    w = np.zeros(max(n, k) + 1)
    _check(load().hkbe_rule(k, n, _dp(w)))
    return w


def hkbe_hodlr_partition(nt, leaf):
    """Blocks of the HODLR partition (host only): dict of r0, r1, c0, c1, level."""
    nb = np.zeros(1, np.int32)
    _check(load().hkbe_hodlr_partition(int(nt), int(leaf), _ip(nb), None, None, None, None, None))
    n = int(nb[0])
    a = [np.zeros(max(n, 1), np.int32) for _ in range(5)]
    _check(load().hkbe_hodlr_partition(int(nt), int(leaf), _ip(nb), *[_ip(x) for x in a]))
    return dict(zip(["r0", "r1", "c0", "c1", "level"], [x[:n] for x in a]))


def hkbe_dlr_matrices(tau, omega, beta, xi=-1):
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    r = len(tau)
    e0, eb = np.zeros(r), np.zeros(r)
    rev, q, phi = np.zeros(r * r), np.zeros(r * r), np.zeros(r * r * r)
    _check(load().hkbe_dlr_matrices(r, _dp(tau), _dp(om), float(beta), int(xi), _dp(e0), _dp(eb),
                                    _dp(rev), _dp(q), _dp(phi)))
    return e0, eb, rev.reshape(r, r), q.reshape(r, r), phi.reshape(r, r, r)


def hkbe_lesser_column_noalloc(nt, k, nao, r, h, T, d_gr, d_sr, d_sl, d_gtv, d_stv, d_eps,
                               d_e0, d_rev, d_q, d_gl, stream=None):
    """Device pointers (ints) in, G^<(., T) written into d_gl; no allocation."""
    buf = C.create_string_buffer(256)
    rc = load().hkbe_lesser_column_noalloc(nt, k, nao, r, float(h), T, d_gr, d_sr, d_sl, d_gtv, d_stv,
                                           d_eps, d_e0, d_rev, d_q, d_gl, stream, buf, 256)
    if rc != HKBE_OK:
        raise HKBEError(rc, buf.value.decode())


# ---- convenience wrapper -----------------------------------------------------

class Stepper:
    """Owns one handle; inputs are numpy arrays shaped as in include/hkbe.h."""

    def __init__(self, nt, h, k, beta, nao=1, n_inst=1, rho_mode=0, max_iter=50, tol=1e-12,
                 precision=PREC_FP64, svd_tol=0.0, leaf=64, r_max=64, stream=None, nt_per_inst=None):
        self.p = hkbe_params(nt=nt, k=k, nao=nao, xi=-1, n_inst=n_inst, rho_mode=rho_mode,
                             precision=precision, max_iter=max_iter, h=h, beta=beta, tol=tol,
                             svd_tol=svd_tol, leaf=leaf, r_max=r_max)
        self.nao, self.n_inst, self.nt = nao, n_inst, nt
        self.h = hkbe_create(self.p, stream, nt_per_inst)
        self.r = 0

    def close(self):
        if self.h:
            hkbe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_inputs(self, tau, omega, gm, eps, model, model_params):
        """gm None: no G^M is set (hkbe_solve_matsubara installs one)."""
        self.r = len(tau)
        hkbe_set_dlr(self.h, tau, omega)
        if gm is not None:
            hkbe_set_matsubara(self.h, gm)
        hkbe_set_hamiltonian(self.h, eps)
        hkbe_set_model(self.h, model, model_params)

    def bootstrap(self, max_iter=200, tol=None):
        return hkbe_bootstrap(self.h, self.n_inst, max_iter, self.p.tol if tol is None else tol)

    def step(self, n_steps=1):
        it, er, _ = hkbe_step(self.h, self.n_inst, n_steps)
        return it, er

    def run(self):
        self.bootstrap()
        T = hkbe_current_step(self.h)
        return self.step(self.nt - 1 - T)

    def timing(self):
        """{phase: (device ms, launches)} accumulated since the last reset."""
        return {name: hkbe_get_timing(self.h, i) for i, name in enumerate(PHASES)}

    def row(self, inst, T):
        return hkbe_get_row(self.h, self.nao, inst, T)

    def tv(self, inst, t):
        return hkbe_get_tv(self.h, self.nao, self.r, inst, t)

    def density(self):
        return hkbe_get_density(self.h, self.n_inst, self.nao, hkbe_current_step(self.h))

    def dense(self, inst=0):
        """All rows up to the current step as lower-triangular arrays
        GR[T, t] = G^R(T, t), GLs[T, t] = G^<(t, T) and GTV[T, i]."""
        T = hkbe_current_step(self.h)
        GR = np.zeros((T + 1, T + 1, self.nao, self.nao), np.complex128)
        GL = np.zeros_like(GR)
        GTV = np.zeros((T + 1, self.r, self.nao, self.nao), np.complex128)
        for t in range(T + 1):
            gr, gl = self.row(inst, t)
            GR[t, :t + 1] = gr
            GL[t, :t + 1] = gl
            GTV[t] = self.tv(inst, t)
        return GR, GL, GTV


def model_params_for(workload_dict):
    """Model id and parameter array of a workload from ``kbe_workloads``."""
    wl = workload_dict["wl"]
    if wl.model == "bethe":
        return MODEL_BETHE, np.asarray(workload_dict["model_params"], dtype=float)
    if wl.model == "none":
        return MODEL_NONE, None
    if wl.model == "nambu":
        return MODEL_NAMBU, np.asarray(workload_dict["model_params"], dtype=float)
    if wl.model == "lattice2b":
        return MODEL_LATTICE2B, np.asarray(workload_dict["model_params"], dtype=float)
    if wl.model == "bath":   # per instance [nb, eps_b[nb], V[nao][nb] as (re, im) pairs]
        return MODEL_BATH, np.asarray(workload_dict["model_params"], dtype=float)
    raise ValueError(wl.model)
