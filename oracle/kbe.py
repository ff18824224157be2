"""Oracle: dense, uncompressed FP64 Kadanoff-Baym stepper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Storage (Sec. 2.1): lower-triangular arrays indexed [T, t] for
  GR[T, t]  = G^R(T, t),   t <= T
  GLs[T, t] = G^<(t, T),   t <= T   (G^<_{t1 t2} = G^<(t2, t1))
and the same for Sigma; mixed GTV[T, i] = G^tv(T, tau_i) on the DLR nodes;
eps[t + 1] = eps(t), eps[0] is the equilibrium-branch value eps(0_|).
Every element is an N_o x N_o complex matrix.

The discrete equations (Eqs. KBER, KBET, KBEL with Appendix A):

Retarded row at step T > k (Eq. KBER, unknown y_s = G^R(T, T-s), y_0 = -i):
    (i/h) sum_j a_j y_{s-j} = y_s eps(T-s) + h sum_l w^(s)_l y_l SR(T-l, T-s)
  for s > k, and for the start block s = 1..k, solved together,
    (i/h) sum_l D_sl y_l = y_s eps(T-s) + h sum_l I_{0,s,l} y_l SR_x(T-l, T-s).
Mixed at step T (Eq. KBET):
    (i/h) sum_j a_j G^tv(T-j) = eps(T) G^tv(T) + h sum_l w^(T)_l SR(T,l) G^tv(l)
                               + int Sigma^tv(T, tb) G^M(tb - tau) dtb.
Lesser column x_t = G^<(t, T), t = 0..T (Eq. KBEL, solved in t):
    x_0 = -[G^tv(T, 0+)]^dagger,
    (i/h) sum_j a_j x_{t-j} = eps(t) x_t + h sum_l w^(t)_l SR(t,l) x_l + q_t,
    q_t = h sum_l w^(T)_l Sigma^<(t,l) G^A(l,T) - i int Sigma^tv(t,tau) G^vt(tau,T),
  start block t = 1..k with D and I_{0,t,.}.
Density matrix (Sec. 3.3): horizontal takes x_T; diagonal integrates
    d rho/dT = xi i (D - D^dagger),  D = d_t G^<(t,T)|_{t=T} from the KBEL
  right-hand side, with the BDF weights, and sets G^<(T,T) = -i xi rho(T).

SR_x is the smooth continuation across the diagonal, SR_x(a,b) = -[SR(b,a)]^dagger
for a < b (the anti-Hermitian symmetry of Sigma^> - Sigma^<, Sec. 2.1).

Bootstrap (T <= k) solves the (k+1) x (k+1) start square with the polynomial
weights D and I (Appendix A), by global iteration with Sigma (Sec. 3.3):
mixed rows 1..k together; retarded columns n = 0..k in increasing n with the
left equation (derivative in the first argument), entries above the diagonal
taken by continuation from the columns already solved; every lesser column m
solves the full start block t = 1..k and keeps t <= m.
"""
from __future__ import annotations

import numpy as np

from .dlr import DLROracle
from .weights import Weights


def _dag(x):
    return np.conj(np.swapaxes(x, -1, -2))


class KBEOracle:
    """The dense FP64 stepper of the discrete scheme above, for one instance
    (Eqs. KBER, KBET, KBEL; weights of Appendix A; DLR thermal leg of Sec. 2.5)."""

    def __init__(self, nt, h, k, beta, eps, gm, tau, omega, model, xi=-1,
                 rho_mode=0, tol=1e-12, max_iter=50, boot_tol=None,
                 boot_max_iter=200):
        self.nt = int(nt)
        self.h = float(h)
        self.k = int(k)
        self.beta = float(beta)
        self.xi = int(xi)
        self.eps = np.array(eps, dtype=complex)          # (nt+1, No, No), own copy (a Fock term updates it)
        self.no = self.eps.shape[-1]
        self.tau = np.asarray(tau, dtype=float)
        self.r = len(self.tau)
        self.gm = np.asarray(gm, dtype=complex)          # (r, No, No)
        self.model = model
        self.rho_mode = int(rho_mode)
        self.tol = float(tol)
        self.max_iter = int(max_iter)
        self.boot_tol = float(boot_tol if boot_tol is not None else tol)
        self.boot_max_iter = int(boot_max_iter)
        self.W = Weights(self.k)
        dl = DLROracle(self.tau, omega, beta, xi)
        self.e0 = dl.eval_row(0.0)
        self.ebeta = dl.eval_row(self.beta)
        self.Rev = dl.rev()
        self.Q = dl.Q()
        self.Wconv = dl.conv_tensor(self.gm)             # (r, r, No, No)
        No, N = self.no, self.nt
        shp = (N, N, No, No)
        self.GR = np.zeros(shp, complex)
        self.GLs = np.zeros(shp, complex)
        self.SR = np.zeros(shp, complex)
        self.SLs = np.zeros(shp, complex)
        self.GTV = np.zeros((N, self.r, No, No), complex)
        self.STV = np.zeros((N, self.r, No, No), complex)
        self.iters = np.zeros(N, int)
        self.errs = np.zeros(N)
        self.I1 = np.eye(No, dtype=complex)

    # ---- accessors ---------------------------------------------------------
    def ep(self, t):
        """eps(t) (index t + 1; t = -1 is the equilibrium branch, Sec. 3.2)."""
        return self.eps[t + 1]

    def sR_x(self, a, b):
        """Sigma^R(a, b), continued above the diagonal."""
        return self.SR[a, b] if a >= b else -_dag(self.SR[b, a])

    def sL(self, t, l):
        """Sigma^<(t, l) anywhere (anti-Hermitian symmetry, Eq. GLantiHerm)."""
        return self.SLs[l, t] if t <= l else -_dag(self.SLs[t, l])

    def conv(self, t):
        """int_0^beta Sigma^tv(t, tb) G^M(tb - tau_i) dtb for every node i."""
        return np.einsum("axy,aiyz->ixz", self.STV[t], self.Wconv)

    def gtv_at0(self, T):
        """G^tv(T, 0+) from the DLR expansion on the nodes (Sec. 2.5)."""
        return np.einsum("c,cxy->xy", self.e0, self.GTV[T])

    def gvt(self, T):
        """G^vt(tau_b, T) = -xi [G^tv(T, beta - tau_b)]^dagger on the nodes."""
        rev = np.einsum("bc,cxy->bxy", self.Rev, self.GTV[T])
        return -self.xi * _dag(rev)

    def rho(self, t):
        """rho(t) = xi i G^<(t, t) (Sec. 3.3)."""
        return self.xi * 1j * self.GLs[t, t]

    # ---- initial guess (green_from_H, Sec. 3.3) -----------------------------
    def hf_guess(self):
        """Mean-field start square (green_from_H, Sec. 3.3): G^R, G^< and G^tv of
        the levels eps(0_|) with rho = -G^M(beta^-), G^tv seeded from G^M."""
        k, h = self.k, self.h
        e_eq = self.eps[0]
        E, U = np.linalg.eigh(0.5 * (e_eq + _dag(e_eq)))
        rhoM = -np.einsum("c,cxy->xy", self.ebeta, self.gm)
        g0 = 1j * self.xi * np.einsum("bc,cxy->bxy", self.Rev, self.gm)

        def ex(f):
            return (U * f[None, :]) @ _dag(U)
        for t in range(k + 1):
            for tp in range(t + 1):
                self.GR[t, tp] = -1j * ex(np.exp(-1j * E * (t - tp) * h))
            for tp in range(t + 1):   # GLs[t, tp] = G^<(tp, t)
                self.GLs[t, tp] = 1j * ex(np.exp(-1j * E * tp * h)) @ rhoM @ ex(np.exp(1j * E * t * h))
            # G^tv(t, tau) = e^{-i eps t} G^tv(0, tau), started from the exact
            # G^tv(0, tau) = i xi G^M(beta - tau) (the same as the mean-field form
            # -xi i rho e^{eps tau} when G^M is that of eps; far better when not)
            self.GTV[t] = np.einsum("xy,iyz->ixz", ex(np.exp(-1j * E * t * h)), g0)

    # ---- bootstrap -------------------------------------------------------
    def _boot_mixed(self):
        """Mixed rows 1..k of the start square together (Eq. KBET with D and
        I_{0,m,.} of Appendix A), G^tv(0, tau) = i xi G^M(beta - tau)."""
        k, h, No, W = self.k, self.h, self.no, self.W
        g0 = 1j * self.xi * np.einsum("bc,cxy->bxy", self.Rev, self.gm)  # G^tv(0, tau)
        self.GTV[0] = g0
        E = np.zeros((k * No, k * No), complex)
        B = np.zeros((k * No, self.r * No), complex)
        for m in range(1, k + 1):
            Im = W.I(0, m)
            C = self.conv(m)                       # (r, No, No)
            rhs = np.concatenate([C[i] for i in range(self.r)], axis=1)
            c0 = (1j / h) * W.D[m, 0] * self.I1 - h * Im[0] * self.sR_x(m, 0)
            rhs = rhs - c0 @ np.concatenate([g0[i] for i in range(self.r)], axis=1)
            B[(m - 1) * No:m * No] = rhs
            for l in range(1, k + 1):
                blk = (1j / h) * W.D[m, l] * self.I1 - h * Im[l] * self.sR_x(m, l)
                if l == m:
                    blk = blk - self.ep(m)
                E[(m - 1) * No:m * No, (l - 1) * No:l * No] = blk
        X = np.linalg.solve(E, B)
        for m in range(1, k + 1):
            for i in range(self.r):
                self.GTV[m, i] = X[(m - 1) * No:m * No, i * No:(i + 1) * No]

    def _boot_ret(self):
        """Retarded columns n = 0..k of the start square (Eq. KBER in its first
        argument, D and I_{n,m,.} of Appendix A), G^R(n, n) = -i."""
        k, h, No, W = self.k, self.h, self.no, self.W
        for n in range(k + 1):
            self.GR[n, n] = -1j * self.I1
        for n in range(k):
            def gx(l):
                return self.GR[l, n] if l >= n else -_dag(self.GR[n, l])
            nu = k - n
            E = np.zeros((nu * No, nu * No), complex)
            B = np.zeros((nu * No, No), complex)
            for mi, m in enumerate(range(n + 1, k + 1)):
                Inm = W.I(n, m)
                acc = np.zeros((No, No), complex)
                for l in range(k + 1):
                    blk = (1j / h) * W.D[m, l] * self.I1 - h * Inm[l] * self.sR_x(m, l)
                    if l == m:
                        blk = blk - self.ep(m)
                    if l <= n:
                        acc -= blk @ gx(l)
                    else:
                        li = l - n - 1
                        E[mi * No:(mi + 1) * No, li * No:(li + 1) * No] = blk
                B[mi * No:(mi + 1) * No] = acc
            X = np.linalg.solve(E, B)
            for mi, m in enumerate(range(n + 1, k + 1)):
                self.GR[m, n] = X[mi * No:(mi + 1) * No]

    def _boot_les(self):
        """Lesser columns m = 0..k of the start square.  Column m solves the
        start block (the equations t = 1..k with D and I_{0,t,.}) for all
        x(t) = G^<(t, m), t = 1..k, and keeps the entries t <= m; the entries
        t > m are the lower triangle, owned by the columns t (anti-Hermitian
        symmetry)."""
        k, h, No, W = self.k, self.h, self.no, self.W
        E = np.zeros((k * No, k * No), complex)
        for t in range(1, k + 1):
            It = W.I(0, t)
            for l in range(1, k + 1):
                blk = (1j / h) * W.D[t, l] * self.I1 - h * It[l] * self.sR_x(t, l)
                if l == t:
                    blk = blk - self.ep(t)
                E[(t - 1) * No:t * No, (l - 1) * No:l * No] = blk
        for m in range(k + 1):
            x0 = -_dag(self.gtv_at0(m))
            self.GLs[m, 0] = x0
            if m == 0:
                continue
            Im = W.I(0, m)
            v = np.einsum("ab,bxy->axy", self.Q, self.gvt(m))

            def gA(l):   # G^A(l, m) continued: [G^R(m,l)]^dag, l<=m; -G^R(l,m), l>m
                return _dag(self.GR[m, l]) if l <= m else -self.GR[l, m]
            B = np.zeros((k * No, No), complex)
            for t in range(1, k + 1):
                q = np.zeros((No, No), complex)
                for l in range(k + 1):
                    q += h * Im[l] * self.sL(t, l) @ gA(l)
                q += -1j * np.einsum("axy,ayz->xz", self.STV[t], v)
                c0 = (1j / h) * W.D[t, 0] * self.I1 - h * W.I(0, t)[0] * self.sR_x(t, 0)
                B[(t - 1) * No:t * No] = q - c0 @ x0
            X = np.linalg.solve(E, B)
            for t in range(1, m + 1):
                self.GLs[m, t] = X[(t - 1) * No:t * No]

    def bootstrap(self):
        """Start square T <= k by global iteration with Sigma (Sec. 3.3,
        dyson_start): mean-field guess, then mixed, retarded and lesser parts
        until the change is below boot_tol."""
        k = self.k
        self.hf_guess()
        err = np.inf
        it = 0
        for it in range(1, self.boot_max_iter + 1):
            old = (self.GR[:k + 1, :k + 1].copy(), self.GLs[:k + 1, :k + 1].copy(),
                   self.GTV[:k + 1].copy())
            for t in range(k + 1):
                self.model.eval_step(self, t)
            self._boot_mixed()
            self._boot_ret()
            self._boot_les()
            err = max(np.abs(self.GR[:k + 1, :k + 1] - old[0]).max(),
                      np.abs(self.GLs[:k + 1, :k + 1] - old[1]).max(),
                      np.abs(self.GTV[:k + 1] - old[2]).max())
            if err < self.boot_tol or not self.model.self_consistent and it >= 2:
                break
        for t in range(k + 1):
            self.model.eval_step(self, t)
        self.iters[:k + 1] = it
        self.errs[:k + 1] = err
        return it, err

    # ---- time step T > k ---------------------------------------------------
    def extrapolate(self, T):
        """Guess of step T (Sec. 3.4): polynomial extrapolation of degree k with
        weights e_l = (-1)^l C(k+1, l+1) along lines of constant time
        difference, and of G^tv(T) in T; G^R(T, T) = -i."""
        k = self.k
        e = self.W.extrap()
        for tp in range(T + 1):
            if tp == T:
                self.GR[T, T] = -1j * self.I1
            elif tp >= k + 1:
                self.GR[T, tp] = sum(e[l] * self.GR[T - 1 - l, tp - 1 - l] for l in range(k + 1))
            elif tp == 0:
                self.GR[T, 0] = sum(e[l] * self.GR[T - 1 - l, 0] for l in range(k + 1))
            else:
                self.GR[T, tp] = self.GR[T - 1, tp - 1]
        for t in range(T + 1):
            if t >= k + 1:
                self.GLs[T, t] = sum(e[l] * self.GLs[T - 1 - l, t - 1 - l] for l in range(k + 1))
            elif t == 0:
                self.GLs[T, 0] = sum(e[l] * self.GLs[T - 1 - l, 0] for l in range(k + 1))
            else:
                self.GLs[T, t] = self.GLs[T - 1, t - 1]
        self.GTV[T] = sum(e[l] * self.GTV[T - 1 - l] for l in range(k + 1))

    def solve_ret(self, T):
        """Row G^R(T, .) from Eq. KBER in the second argument: start block
        s = 1..k, then BDF + Gregory (Appendix A) point solves for s > k."""
        k, h, No, W = self.k, self.h, self.no, self.W
        y = self._ret_start_block(T)
        a = W.a
        for s in range(k + 1, T + 1):
            w = W.rule(s)
            Ks = self.SR[T - np.arange(s + 1), T - s]          # SR(T-l, T-s), l=0..s
            rhs = -(1j / h) * np.einsum("j,jxy->xy", a[1:], y[s - 1:s - k - 1:-1] if s - k - 1 >= 0 else y[s - 1::-1][:k])
            rhs = rhs + h * np.einsum("l,lxy,lyz->xz", w[:s], y[:s], Ks[:s])
            M = (1j * a[0] / h) * self.I1 - self.ep(T - s) - h * w[s] * Ks[s]
            y[s] = np.linalg.solve(M.T, rhs.T).T
        for s in range(T + 1):
            self.GR[T, T - s] = y[s]

    def _ret_start_block(self, T):
        """y_s = G^R(T, T-s) for s = 0..k (y_0 = -i, the start block of
        Eq. KBER solved together); entries s > k left zero."""
        k, h, No, W = self.k, self.h, self.no, self.W
        y = np.zeros((T + 1, No, No), complex)
        y[0] = -1j * self.I1

        def K(l, s):
            return self.sR_x(T - l, T - s)
        # start block s = 1..k: sum_l y_l C[l, s] = b_s
        C = np.zeros((k * No, k * No), complex)
        Bm = np.zeros((No, k * No), complex)
        for s in range(1, k + 1):
            Is = W.I(0, s)
            c0 = (1j / h) * W.D[s, 0] * self.I1 - h * Is[0] * K(0, s)
            Bm[:, (s - 1) * No:s * No] = -y[0] @ c0
            for l in range(1, k + 1):
                blk = (1j / h) * W.D[s, l] * self.I1 - h * Is[l] * K(l, s)
                if l == s:
                    blk = blk - self.ep(T - s)
                C[(l - 1) * No:l * No, (s - 1) * No:s * No] = blk
        Ys = np.linalg.solve(C.T, Bm.T).T
        for s in range(1, k + 1):
            y[s] = Ys[:, (s - 1) * No:s * No]
        return y

    def solve_mixed(self, T):
        """G^tv(T, tau_i) from Eq. KBET: BDF + Gregory point solve with the DLR
        convolution of Sigma^tv with G^M (Sec. 2.5)."""
        k, h, W = self.k, self.h, self.W
        a = W.a
        w = W.rule(T)
        M = (1j * a[0] / h) * self.I1 - self.ep(T) - h * w[T] * self.SR[T, T]
        rhs = -(1j / h) * np.einsum("j,jixy->ixy", a[1:], self.GTV[T - 1:T - k - 1:-1] if T - k - 1 >= 0 else self.GTV[T - 1::-1][:k])
        rhs = rhs + h * np.einsum("l,lxy,liyz->ixz", w[:T], self.SR[T, :T], self.GTV[:T])
        rhs = rhs + self.conv(T)
        self.GTV[T] = np.linalg.solve(M[None], rhs)

    def lesser_source(self, T):
        """Source q_t of the lesser column (Eq. KBEL): h sum_l w^(T)_l
        Sigma^<(t, l) G^A(l, T) - i int Sigma^tv(t, tau) G^vt(tau, T) dtau."""
        h = self.h
        w = self.W.rule(T)
        GA = _dag(self.GR[T, :T + 1])                          # G^A(l, T), l = 0..T
        v = np.einsum("ab,bxy->axy", self.Q, self.gvt(T))
        A = self.SLs[:T + 1, :T + 1]                          # A[l, t] = Sigma^<(t, l), t <= l
        idx = np.arange(T + 1)
        upper = (idx[:, None] <= idx[None, :])[:, :, None, None]
        F = np.where(upper, A.transpose(1, 0, 2, 3), -_dag(A))  # F[t, l] = Sigma^<(t, l)
        q = h * np.einsum("l,tlxy,lyz->txz", w[:T + 1], F, GA)
        q += -1j * np.einsum("taxy,ayz->txz", self.STV[:T + 1], v)
        return q

    def solve_les(self, T):
        """Column G^<(., T) from Eq. KBEL in the first argument: x_0 =
        -[G^tv(T, 0+)]^dagger, start block t = 1..k, BDF + Gregory for t > k;
        the last entry from the density-matrix scheme (Sec. 3.3)."""
        k, h, No, W = self.k, self.h, self.no, self.W
        a = W.a
        q = self.lesser_source(T)
        x = np.zeros((T + 1, No, No), complex)
        x[0] = -_dag(self.gtv_at0(T))
        E = np.zeros((k * No, k * No), complex)
        B = np.zeros((k * No, No), complex)
        for t in range(1, k + 1):
            It = W.I(0, t)
            acc = q[t].copy()
            for l in range(k + 1):
                blk = (1j / h) * W.D[t, l] * self.I1 - h * It[l] * self.sR_x(t, l)
                if l == t:
                    blk = blk - self.ep(t)
                if l == 0:
                    acc -= blk @ x[0]
                else:
                    E[(t - 1) * No:t * No, (l - 1) * No:l * No] = blk
            B[(t - 1) * No:t * No] = acc
        X = np.linalg.solve(E, B)
        for t in range(1, k + 1):
            x[t] = X[(t - 1) * No:t * No]
        last = T if self.rho_mode == 0 else T - 1
        for t in range(k + 1, last + 1):
            w = W.rule(t)
            rhs = -(1j / h) * np.einsum("j,jxy->xy", a[1:], x[t - 1:t - k - 1:-1] if t - k - 1 >= 0 else x[t - 1::-1][:k])
            rhs = rhs + h * np.einsum("l,lxy,lyz->xz", w[:t], self.SR[t, :t], x[:t]) + q[t]
            M = (1j * a[0] / h) * self.I1 - self.ep(t) - h * w[t] * self.SR[t, t]
            x[t] = np.linalg.solve(M, rhs)
        if self.rho_mode == 1:
            x[T] = self._rho_diagonal(T, x, q)
        self.GLs[T, :T + 1] = x

    def _rho_diagonal(self, T, x, q):
        """Diagonal integration of rho (Sec. 3.3):
        (a_0/h) rho + i (A rho - rho A^dag) = -(1/h) sum_{j>=1} a_j rho(T-j) + xi (r0 + r0^dag),
        A = eps(T) + h w_T Sigma^R(T,T), r0 = h sum_{l<T} w_l Sigma^R(T,l) x_l + q_T."""
        h, k, No, xi = self.h, self.k, self.no, self.xi
        a = self.W.a
        w = self.W.rule(T)
        A = self.ep(T) + h * w[T] * self.SR[T, T]
        r0 = h * np.einsum("l,lxy,lyz->xz", w[:T], self.SR[T, :T], x[:T]) + q[T]
        rhs = -(1.0 / h) * sum(a[j] * self.rho(T - j) for j in range(1, k + 1)) + xi * (r0 + _dag(r0))
        L = np.zeros((No * No, No * No), complex)
        for p in range(No * No):
            Eb = np.zeros((No, No), complex)
            Eb.flat[p] = 1.0
            L[:, p] = ((a[0] / h) * Eb + 1j * (A @ Eb - Eb @ _dag(A))).ravel()
        rho = np.linalg.solve(L, rhs.ravel()).reshape(No, No)
        return -1j * xi * rho

    def step(self, T):
        """Time step T > k (Sec. 3.4): extrapolate, then Sigma, retarded, mixed
        and lesser parts until max |G^(i) - G^(i-1)| < tol or max_iter."""
        self.extrapolate(T)
        err = np.inf
        it = 0
        for it in range(1, self.max_iter + 1):
            old = (self.GR[T, :T + 1].copy(), self.GLs[T, :T + 1].copy(), self.GTV[T].copy())
            self.model.eval_step(self, T)
            self.solve_ret(T)
            self.solve_mixed(T)
            self.solve_les(T)
            err = max(np.abs(self.GR[T, :T + 1] - old[0]).max(),
                      np.abs(self.GLs[T, :T + 1] - old[1]).max(),
                      np.abs(self.GTV[T] - old[2]).max())
            if err < self.tol or (not self.model.self_consistent and it >= 2):
                break
        self.iters[T] = it
        self.errs[T] = err
        return it, err

    def run(self, nt=None):
        """Bootstrap and step to nt - 1 (Sec. 3.3, 3.4)."""
        nt = self.nt if nt is None else nt
        self.bootstrap()
        for T in range(self.k + 1, nt):
            self.step(T)
        return self


def from_workload(w, inst=0, **kw):
    """Build an oracle for instance ``inst`` of a workload dict from
    ``kbe_workloads``."""
    from .models import make_model
    wl = w["wl"]
    params = dict(wl.params)
    if "drive_A" in w:   # per-instance drive arrays (Nambu model)
        params.update({"A": w["drive_A"][inst], "U": w["drive_U"][inst]})
    params.update(kw.pop("model_params", {}))
    model = make_model(wl.model, params)
    return KBEOracle(wl.nt, wl.h, wl.k, wl.beta, w["eps"][inst], w["gm"][inst],
                     w["tau"], w["omega"], model, rho_mode=kw.pop("rho_mode", wl.rho_mode),
                     tol=kw.pop("tol", wl.tol), max_iter=kw.pop("max_iter", wl.max_iter), **kw)
