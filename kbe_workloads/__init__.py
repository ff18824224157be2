"""Seeded, synthetic inputs for the Kadanoff-Baym time stepper.

This module is shared by the FP64 CPU oracle, the tests and ``bench.py``.  It
holds only *inputs*: the imaginary-time grid (DLR nodes), the model
parameters drawn from seeds, the equilibrium Matsubara Green's function of the
models whose thermal state has a closed form, and the drive protocols.  It
contains none of the time-stepping arithmetic (weights, history integrals,
Volterra solves, self-energies); those live separately in ``oracle/`` and in
the CUDA library.

Conventions (Sec. 2 of the paper, Table 1): fermions (xi = -1), matrices are
N_o x N_o complex, G^M(tau) = -<T d(tau) d^dagger> on (0, beta).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

XI_FERMION = -1


# ---------------------------------------------------------------------------
# DLR imaginary-time grid (Sec. 2.5; the construction of Kaye et al., the
# paper's reference kaye22: interpolative decomposition of the Lehmann kernel).
# ---------------------------------------------------------------------------

def _cheb_panel(a: float, b: float, p: int) -> np.ndarray:
    """p Chebyshev points of the first kind mapped to (a, b)."""
    j = np.arange(p)
    x = np.cos((2 * j + 1) * np.pi / (2 * p))[::-1]
    return 0.5 * (a + b) + 0.5 * (b - a) * x


def _lehmann_kernel_unit(tau: np.ndarray, om: np.ndarray) -> np.ndarray:
    """Fermionic kernel K(tau, w) = exp(-tau w) / (1 + exp(-w)) at beta = 1."""
    t = tau[:, None]
    w = om[None, :]
    pos = w >= 0
    out = np.empty(np.broadcast_shapes(t.shape, w.shape))
    wp = np.where(pos, w, 0.0)
    wn = np.where(pos, 0.0, w)
    kp = np.exp(-t * wp) / (1.0 + np.exp(-wp))
    kn = np.exp((1.0 - t) * wn) / (1.0 + np.exp(wn))
    out[...] = np.where(pos, kp, kn)
    return out


def dlr_grid(lam: float, eps: float, beta: float, p: int = 24):
    """DLR real frequencies and imaginary-time nodes for cutoff ``lam`` and
    accuracy ``eps`` (Sec. 2.5).  Returns ``(tau_nodes, omega_nodes)``, both
    sorted, of equal length r = O(log(lam) log(1/eps)).

    Frequencies are chosen by column-pivoted QR of the kernel sampled on a
    fine composite Chebyshev grid, dyadically refined toward w = 0; the tau
    nodes by pivoted QR of the selected columns' rows (fine tau grid refined
    toward both ends of (0, beta)).  The result is a grid (input data): the
    oracle and the CUDA library each build their own interpolation and
    quadrature matrices from it.
    """
    from scipy.linalg import qr

    nlev = max(1, int(math.ceil(math.log2(max(lam, 2.0)))))
    # frequency panels: [0,1],[1,2],[2,4],...,[lam/2,lam] and mirror
    edges = [0.0, 1.0] + [2.0 ** j for j in range(1, nlev)] + [lam]
    edges = sorted(set(e for e in edges if e <= lam))
    wpos = np.concatenate([_cheb_panel(edges[i], edges[i + 1], p)
                           for i in range(len(edges) - 1)])
    wfine = np.concatenate([-wpos[::-1], wpos])
    # tau panels on (0, 1/2] refined toward 0, mirrored onto [1/2, 1)
    tedges = [0.0] + [2.0 ** (-j) for j in range(nlev + 1, 0, -1)]
    tl = np.concatenate([_cheb_panel(tedges[i], tedges[i + 1], p)
                         for i in range(len(tedges) - 1)])
    tfine = np.concatenate([tl, 1.0 - tl[::-1]])
    A = _lehmann_kernel_unit(tfine, wfine)
    _, R, piv = qr(A, mode="economic", pivoting=True)
    d = np.abs(np.diag(R))
    r = int(np.sum(d > eps * d[0]))
    om = wfine[piv[:r]]
    _, _, piv2 = qr(A[:, piv[:r]].T, mode="economic", pivoting=True)
    tau = tfine[piv2[:r]]
    return np.sort(tau) * beta, np.sort(om) / beta


# ---------------------------------------------------------------------------
# Equilibrium initial states that have closed forms (inputs, not solved here)
# ---------------------------------------------------------------------------

def fermi(e, beta):
    e = np.asarray(e, dtype=float)
    return 0.5 * (1.0 - np.tanh(0.5 * beta * e))


def semicircle_gm(tau: np.ndarray, beta: float, eps0: float, v: float = 1.0,
                  nquad: int = 4000) -> np.ndarray:
    """G^M(tau) of the Bethe lattice (semicircular DOS of half-bandwidth 2v
    centred on eps0): -int A(w) exp(-tau w) / (1 + exp(-beta w)) dw, by
    Gauss-Chebyshev quadrature of the second kind (exact weight sqrt(1-x^2))."""
    j = np.arange(1, nquad + 1)
    th = j * np.pi / (nquad + 1)
    x = np.cos(th)
    wq = np.pi / (nquad + 1) * np.sin(th) ** 2  # int_{-1}^{1} f sqrt(1-x^2)
    w = eps0 + 2.0 * v * x
    # A(w) dw = sqrt(4v^2-(w-eps0)^2)/(2 pi v^2) dw = (2/pi) sqrt(1-x^2) dx
    t = np.asarray(tau, dtype=float)[:, None]
    ker = _lehmann_kernel_unit(t[:, 0] / beta, w * beta)
    return -(2.0 / np.pi) * (ker * wq[None, :]).sum(axis=1)


def two_level_gm(tau, beta, ed, eb, V):
    """Impurity block G_dd^M(tau) of the two-site model H = [[ed, V], [V, eb]]
    (exact diagonalisation of the 2x2 single-particle Hamiltonian)."""
    H = np.array([[ed, V], [V, eb]], dtype=float)
    E, U = np.linalg.eigh(H)
    wgt = np.abs(U[0, :]) ** 2
    t = np.asarray(tau, dtype=float)
    ker = _lehmann_kernel_unit(t / beta, E * beta)
    return -(ker * wgt[None, :]).sum(axis=1)


def free_level_gm(tau, beta, eps_mat):
    """G^M(tau) of a non-interacting N_o-level system with Hermitian level
    matrix eps_mat: -U diag(K(tau, E)) U^dagger."""
    E, U = np.linalg.eigh(np.asarray(eps_mat, dtype=complex))
    t = np.asarray(tau, dtype=float)
    ker = _lehmann_kernel_unit(t / beta, E * beta)  # (ntau, No)
    return -np.einsum("ia,ta,ja->tij", U, ker, U.conj())


# ---------------------------------------------------------------------------
# Workload descriptions (the five configurations this project is measured on)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    model: str                 # "none" | "bethe" | "bath"
    nt: int
    h: float
    k: int
    beta: float
    nao: int = 1
    n_inst: int = 1
    dlr_lambda: float = 100.0
    dlr_eps: float = 1e-10
    svd_tol: float = 0.0       # 0 -> dense (uncompressed) storage
    leaf: int = 64
    rho_mode: int = 0          # 0 horizontal, 1 diagonal
    max_iter: int = 50
    tol: float = 1e-12
    seed: int = 0
    params: dict = field(default_factory=dict)


def bethe_eps0(seed: int, n: int = 1) -> np.ndarray:
    """On-site levels eps0 ~ U[-0.5, 0.5] drawn from numpy's default_rng(seed)."""
    return np.random.default_rng(seed).uniform(-0.5, 0.5, size=n)


def quench_eps(nt: int, h: float, eps_before: float, eps_after: float,
               t_quench: float) -> np.ndarray:
    """Level eps(t) on the grid t = n h (n = -1 is the equilibrium branch),
    switched from eps_before to eps_after for t >= t_quench."""
    n = np.arange(-1, nt)
    t = np.maximum(n, 0) * h
    e = np.where((n >= 0) & (t >= t_quench - 1e-12), eps_after, eps_before)
    return e.astype(float)


def bethe_workload(name="C1", nt=256, h=0.025, k=5, beta=5.0, seed=0,
                   n_inst=1, svd_tol=0.0, leaf=64, quench=None,
                   dlr_lambda=100.0, dlr_eps=1e-10, tol=1e-12, max_iter=50,
                   rho_mode=0):
    """Bethe-lattice workload (Sigma = v^2 G, v = 1).  Returns a dict of
    arrays with everything both implementations need: DLR grid, eps(t) per
    instance (index 0 is the equilibrium branch), G^M on the DLR nodes."""
    tau, om = dlr_grid(dlr_lambda, dlr_eps, beta)
    eps0 = bethe_eps0(seed, n_inst)
    eps = np.zeros((n_inst, nt + 1, 1, 1), dtype=complex)
    gm = np.zeros((n_inst, len(tau), 1, 1), dtype=complex)
    for i in range(n_inst):
        if quench is None:
            eps[i, :, 0, 0] = eps0[i]
            gm[i, :, 0, 0] = semicircle_gm(tau, beta, eps0[i])
        else:
            e_before, e_after, tq = quench
            eps[i, :, 0, 0] = quench_eps(nt, h, e_before, e_after, tq)
            gm[i, :, 0, 0] = semicircle_gm(tau, beta, e_before)
    wl = Workload(name=name, model="bethe", nt=nt, h=h, k=k, beta=beta,
                  nao=1, n_inst=n_inst, dlr_lambda=dlr_lambda, dlr_eps=dlr_eps,
                  svd_tol=svd_tol, leaf=leaf, tol=tol, max_iter=max_iter,
                  seed=seed, rho_mode=rho_mode, params={"v": 1.0})
    return {"wl": wl, "tau": tau, "omega": om, "eps": eps, "gm": gm,
            "model_params": np.array([[1.0]] * n_inst)}


def c1_workload(seed=0, **kw):
    """Plain FP64 Bethe lattice, beta=5, N_t=256, h=0.025, order 5, DLR
    (Lambda=100, eps=1e-10), undriven, eps0 ~ U[-0.5,0.5] from ``seed``."""
    return bethe_workload(name="C1", nt=kw.pop("nt", 256), h=kw.pop("h", 0.025),
                          k=kw.pop("k", 5), beta=5.0, seed=seed, **kw)


def c2_workload(seed=0, **kw):
    """Bethe lattice with HODLR (leaf 64, SVD tol 1e-8), N_t=4096, h=0.02,
    beta=5, level quench eps0: 0 -> 1 at t = 5."""
    return bethe_workload(name="C2", nt=kw.pop("nt", 4096), h=kw.pop("h", 0.02),
                          k=kw.pop("k", 5), beta=5.0, seed=seed,
                          svd_tol=kw.pop("svd_tol", 1e-8), leaf=kw.pop("leaf", 64),
                          quench=(0.0, 1.0, 5.0), **kw)


def nambu_drive(nt, h, A0=0.0, Omega=1.0, tc=2.0, width=1.0, U=0.0, U_eq=0.0, t_quench=0.0):
    """Drive arrays on the grid (index 0 the equilibrium branch, index t+1
    time t = n h): vector potential A(t) = A0 sin(Omega t) exp(-(t-tc)^2/width)
    (A = 0 on the equilibrium branch) and interaction U(t) = U for
    t >= t_quench, U_eq before and on the equilibrium branch."""
    t = np.arange(nt) * h
    A = np.concatenate([[0.0], A0 * np.sin(Omega * t) * np.exp(-(t - tc) ** 2 / width)])
    Uv = np.concatenate([[U_eq], np.where(t >= t_quench - 1e-12, U, U_eq)])
    return A, Uv


def nambu_workload(nt=200, h=0.02, k=5, beta=5.0, n_inst=1, v=1.0, eps0=0.0, pairing=0.0,
                   U=0.0, t_quench=0.0, A0=0.0, Omega=1.0, tc=2.0, width=1.0,
                   dlr_lambda=100.0, dlr_eps=1e-10, tol=1e-12, max_iter=50, rho_mode=0, seed=0,
                   g=0.0, w0=0.6):
    """Nambu (2 x 2) Bethe-lattice DMFT impurity (Sec. 4.1): level matrix
    eps = [[eps0, pairing], [pairing, -eps0]], hopping scale v, Peierls drive
    A(t) and an interaction quench U_eq = 0 -> U at t_quench (so the initial
    state is non-interacting and its G^M is known in closed form):
      v != 0, pairing = 0: G^M = diag(semicircle(eps0), semicircle(-eps0));
      v = 0:               G^M of the free 2 x 2 level (any pairing).
    Per instance i > 0 the interaction is U * (1 + 0.25 i) (distinct instances).
    g, w0: optional Holstein coupling and phonon frequency (model parameters
    [v, g, w0]; with g != 0 the closed-form G^M is only a start, not the
    coupled equilibrium)."""
    if v != 0.0 and pairing != 0.0:
        raise ValueError("closed-form initial state needs pairing = 0 when v != 0")
    tau, om = dlr_grid(dlr_lambda, dlr_eps, beta)
    em = np.array([[eps0, pairing], [pairing, -eps0]], dtype=complex)
    eps = np.broadcast_to(em, (n_inst, nt + 1, 2, 2)).astype(complex).copy()
    if v != 0.0:
        g0 = np.zeros((len(tau), 2, 2), complex)
        g0[:, 0, 0] = semicircle_gm(tau, beta, eps0, v)
        g0[:, 1, 1] = semicircle_gm(tau, beta, -eps0, v)
    else:
        g0 = free_level_gm(tau, beta, em)
    gm = np.broadcast_to(g0, (n_inst,) + g0.shape).astype(complex).copy()
    As, Us = [], []
    for i in range(n_inst):
        A, Uv = nambu_drive(nt, h, A0, Omega, tc, width, U * (1.0 + 0.25 * i), 0.0, t_quench)
        As.append(A)
        Us.append(Uv)
    wl = Workload(name="nambu", model="nambu", nt=nt, h=h, k=k, beta=beta, nao=2, n_inst=n_inst,
                  dlr_lambda=dlr_lambda, dlr_eps=dlr_eps, svd_tol=0.0, leaf=64, tol=tol,
                  max_iter=max_iter, seed=seed, rho_mode=rho_mode,
                  params={"v": v, "g": g, "w0": w0} if g else {"v": v})
    mp = np.array([[v, g, w0]] * n_inst) if g else np.array([[v]] * n_inst)
    return {"wl": wl, "tau": tau, "omega": om, "eps": eps, "gm": gm,
            "model_params": mp, "drive_A": np.array(As), "drive_U": np.array(Us)}


def lattice_workload(L=4, nt=120, h=0.02, k=5, beta=10.0, U=2.0, t_quench=0.0, A0=0.0, Omega=1.0,
                     tc=1.0, width=0.5, A_step=0.0, dlr_lambda=100.0, dlr_eps=1e-10, tol=1e-12,
                     max_iter=50, rho_mode=0, svd_tol=0.0, leaf=64, ysymm=False):
    """2D Hubbard model on an L x L k-grid (Sec. 4.2), J = 1, half filling
    (Hartree absorbed, mu~ = 0), one instance per k = 2 pi (m_x, m_y)/L
    (instance m_x L + m_y).  Peierls drive along x: eps_k(t) =
    -2 (cos(k_x - A(t)) + cos k_y), with A(t) = A_step for t > 0 plus a
    pulse A0 sin(Omega t) exp(-(t-tc)^2/width); A = 0 on the equilibrium
    branch.  The interaction is quenched 0 -> U at t_quench, so the initial
    state is the free lattice, G^M_k known in closed form.  ysymm: only the
    k-points with m_y <= L/2 (instance m_x (L/2+1) + m_y), the reflection-
    reduced set of L(L/2+1) points (the drive along x keeps k_y -> -k_y)."""
    if ysymm and L % 2:
        raise ValueError("the reflection-reduced k-set needs an even L")
    tau, om = dlr_grid(dlr_lambda, dlr_eps, beta)
    m = np.arange(L) * 2 * np.pi / L
    ny = L // 2 + 1 if ysymm else L
    kx = np.repeat(m, ny)
    ky = np.tile(m[:ny], L)
    t = np.arange(nt) * h
    A = np.concatenate([[0.0], A_step * (t > 0) + A0 * np.sin(Omega * t) * np.exp(-(t - tc) ** 2 / width)])
    Uv = np.concatenate([[0.0], np.where(t >= t_quench - 1e-12, U, 0.0)])
    nk = L * ny
    eps = np.zeros((nk, nt + 1, 1, 1), complex)
    gm = np.zeros((nk, len(tau), 1, 1), complex)
    for q in range(nk):
        eps[q, :, 0, 0] = -2 * (np.cos(kx[q] - A) + np.cos(ky[q]))
        gm[q] = free_level_gm(tau, beta, np.array([[eps[q, 0, 0, 0].real]]))
    wl = Workload(name="lattice", model="lattice2b", nt=nt, h=h, k=k, beta=beta, nao=1, n_inst=nk,
                  dlr_lambda=dlr_lambda, dlr_eps=dlr_eps, svd_tol=svd_tol, leaf=leaf, tol=tol,
                  max_iter=max_iter, rho_mode=rho_mode, params={"L": L, "ysymm": bool(ysymm)})
    mpar = [float(L), 1.0] if ysymm else [float(L)]
    return {"wl": wl, "tau": tau, "omega": om, "eps": eps, "gm": gm, "L": L, "kx": kx, "ky": ky,
            "model_params": np.array([mpar] * nk), "drive_A": np.tile(A, (nk, 1)),
            "drive_U": np.tile(Uv, (nk, 1))}


# ---------------------------------------------------------------------------
# Batched workloads of the benchmark (many independent instances of one
# configuration; each instance is an input set, nothing is solved here)
# ---------------------------------------------------------------------------

def c2_batch_workload(n_inst, seed=0, nt=4096):
    """C2 for a batch: Bethe, quench eps0 0 -> A at t = 5, N_t = 4096,
    h = 0.02, HODLR leaf 64, eps_SVD 1e-8; instance 0 has A = 1 (C2 itself),
    instance i > 0 takes A ~ U[0.5, 1.5] from numpy default_rng(seed)."""
    w = c2_workload(nt=nt, n_inst=n_inst)
    amp = np.concatenate([[1.0], np.random.default_rng(seed).uniform(0.5, 1.5, size=n_inst - 1)])
    w["eps"][:, 1:, 0, 0] *= amp[:, None]
    return w


def c4_batch_workload(n_inst, seed=0, nt=8192, rho_mode=1):
    """C4-shaped batch: Nambu Bethe-lattice DMFT with the Holstein-Migdal term
    (g = 0.5, w0 = 0.6), beta = 50, N_t = 8192, h = 0.01, order 5, DLR
    Lambda = 200, eps = 1e-10, pulse A(t) = A0 sin(t) exp(-(t-20)^2/50), HODLR
    leaf 64, eps_SVD 1e-7, diagonal density-matrix scheme (driven).  Instance
    0 has A0 = 0.3; instance i > 0 takes A0 = 0.3 U[0.5, 1.5] from numpy
    default_rng(seed).  Initial state: the normal non-interacting Bethe
    lattice (closed-form G^M); the coupling is on from t = 0."""
    w = nambu_workload(nt=nt, h=0.01, k=5, beta=50.0, n_inst=n_inst, v=1.0, eps0=0.0, A0=0.3, Omega=1.0,
                       tc=20.0, width=50.0, g=0.5, w0=0.6, dlr_lambda=200.0, dlr_eps=1e-10, rho_mode=rho_mode)
    amp = np.concatenate([[1.0], np.random.default_rng(seed).uniform(0.5, 1.5, size=n_inst - 1)])
    w["drive_A"] = w["drive_A"] * amp[:, None]
    w["wl"].svd_tol = 1e-7
    return w


def bath_gm(tau, beta, eps0, V, eb):
    """G^M of the impurity block of the quadratic problem
    H = [[eps0, V], [V^dagger, diag(eb)]] (exact diagonalisation)."""
    H = np.block([[np.asarray(eps0, complex), np.asarray(V, complex)],
                  [np.asarray(V, complex).conj().T, np.diag(np.asarray(eb, float)).astype(complex)]])
    no = np.asarray(eps0).shape[0]
    return free_level_gm(tau, beta, H)[:, :no, :no]


C5_BATH_LEVELS = np.array([0.7, -0.9])


def c5_draws(n_inst=64, seed=0, nt_lo=512, nt_hi=4096):
    """Per-instance draws of the uneven batch C5 from numpy default_rng(seed):
    orbital count N_o in {1, 2, 3, 4} (equal shares), N_t ~ U[nt_lo, nt_hi]
    (integer), level entries ~ U[-0.5, 0.5] (Hermitian), drive amplitude
    A0 ~ U[0.1, 0.5], frequency Omega ~ U[0.5, 1.5], interaction U ~ U[0.5, 2]
    (Nambu instances), bath couplings ~ U[-0.5, 0.5] (N_o = 3, 4)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        no = 1 + i % 4
        e = rng.uniform(-0.5, 0.5, size=(no, no)) + 1j * rng.uniform(-0.5, 0.5, size=(no, no))
        out.append(dict(nao=no, nt=int(rng.integers(nt_lo, nt_hi + 1)), eps0=0.5 * (e + e.conj().T),
                        A0=float(rng.uniform(0.1, 0.5)), Omega=float(rng.uniform(0.5, 1.5)),
                        U=float(rng.uniform(0.5, 2.0)), V=rng.uniform(-0.5, 0.5, size=(no, 2))))
    return out


def c5_group_workload(nao, draws, h=0.02, k=5, beta=5.0, svd_tol=1e-7, leaf=64):
    """The instances of C5 with N_o = nao as one batch (one handle): inputs
    up to the group's longest N_t, and per-instance N_t in "nt_per_inst".
      N_o = 1: Bethe lattice (Sigma = v^2 G, v = 1), level eps0 + A0 sin(Omega t);
      N_o = 2: Nambu DMFT, level diag(e, -e) (e the drawn diagonal), second Born
               with U quenched on at t = 0, Peierls drive A0 sin(Omega t);
      N_o = 3, 4: the level matrix coupled to two bath levels (0.7, -0.9) by
               the drawn V (fixed Sigma = V g_b V^dagger), level
               eps0 + A0 sin(Omega t) times the identity.
    Initial states: the non-interacting equilibria (closed forms)."""
    ds = [d for d in draws if d["nao"] == nao]
    n = len(ds)
    nt = max(d["nt"] for d in ds)
    tau, om = dlr_grid(100.0, 1e-10, beta)
    r = len(tau)
    tt = np.concatenate([[0.0], np.arange(nt) * h])      # index 0: the equilibrium branch
    eps = np.zeros((n, nt + 1, nao, nao), complex)
    gm = np.zeros((n, r, nao, nao), complex)
    extra = {}
    if nao == 1:
        for i, d in enumerate(ds):
            e0 = d["eps0"][0, 0].real
            eps[i, :, 0, 0] = e0 + d["A0"] * np.sin(d["Omega"] * tt) * (np.arange(nt + 1) > 0)
            gm[i, :, 0, 0] = semicircle_gm(tau, beta, e0)
        model, mp = "bethe", np.ones((n, 1))
    elif nao == 2:
        As, Us = [], []
        for i, d in enumerate(ds):
            e0 = d["eps0"][0, 0].real
            eps[i] = np.diag([e0, -e0])
            gm[i, :, 0, 0] = semicircle_gm(tau, beta, e0)
            gm[i, :, 1, 1] = semicircle_gm(tau, beta, -e0)
            A = np.concatenate([[0.0], d["A0"] * np.sin(d["Omega"] * tt[1:])])
            As.append(A)
            Us.append(np.concatenate([[0.0], np.full(nt, d["U"])]))
        model, mp = "nambu", np.ones((n, 1))
        extra = {"drive_A": np.array(As), "drive_U": np.array(Us)}
    else:
        mp = []
        for i, d in enumerate(ds):
            drive = d["A0"] * np.sin(d["Omega"] * tt) * (np.arange(nt + 1) > 0)
            eps[i] = d["eps0"][None] + drive[:, None, None] * np.eye(nao)[None]
            gm[i] = bath_gm(tau, beta, d["eps0"], d["V"], C5_BATH_LEVELS)
            Vc = np.asarray(d["V"], complex)
            mp.append(np.concatenate([[2.0], C5_BATH_LEVELS, np.stack([Vc.real, Vc.imag], -1).ravel()]))
        model, mp = "bath", np.array(mp)
    wl = Workload(name=f"C5-no{nao}", model=model, nt=nt, h=h, k=k, beta=beta, nao=nao, n_inst=n,
                  svd_tol=svd_tol, leaf=leaf, rho_mode=1, params={"v": 1.0} if model != "bath" else
                  {"V": None, "eb": C5_BATH_LEVELS})
    return dict({"wl": wl, "tau": tau, "omega": om, "eps": eps, "gm": gm, "model_params": mp,
                 "nt_per_inst": np.array([d["nt"] for d in ds], np.int32)}, **extra)
