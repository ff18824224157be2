"""Pin P6: the stepped FP64 oracle against a direct solve of the whole discrete
system on tiny grids (N_t <= 12, k = 1, 2).

The discrete scheme (Eqs. KBER, KBET, KBEL with the Appendix A weights and the
readings of the start square, the start blocks and the k < n < 2k+1 rule) is
written here once more, independently of the stepper's loops: every equation
of every time step is assembled into one global system whose unknowns are all
stored entries G^R(T, t), G^tv(T, tau_i), G^<(t, T) (plus the entries t > m
that the start-square lesser column m solves and discards).  Because the
lesser source and boundary value hold daggers of unknowns (G^A = [G^R]^dagger,
x_0 = -[G^tv(T, 0+)]^dagger, G^vt from G^tv), the system is linear over the
reals; it is solved as one dense real system.

  Sigma = 0 and the fixed bath (Sigma = V g_b V^dagger, closed form): one solve.
  Bethe lattice (Sigma = v^2 G): global fixed-point iteration of that solve
  with Sigma from the previous iterate, a different algorithm from the
  stepper's per-step loop, converging to the same discrete solution.

The integration rule is rebuilt here from the I_{m,n} weights and the Gregory
end weights (both pinned in test_oracle_weights.py), not taken from
Weights.rule, so a mis-indexed rule in the stepper fails this pin.  The
stepped oracle must agree to 1e-13; planted mistakes in CPU copies of the
stepper (a mis-indexed k < n < 2k+1 rule, a transposed continuation of
Sigma^R in the start block) fail it.
"""
import numpy as np
import pytest

import kbe_workloads as wk
from oracle.dlr import DLROracle
from oracle.kbe import KBEOracle, _dag
from oracle.models import make_model
from oracle.weights import Weights

BETA = 5.0
XI = -1
TAU, OM = wk.dlr_grid(40.0, 1e-10, BETA)


def _rule(W, k, n):
    """w^(n)_l for int_0^n, n > k: for k < n < 2k+1 the order-k polynomial
    over 0..n-k plus the same rule shifted onto n-k..n; for n >= 2k+1 the
    Gregory omega at both ends and 1 inside (Appendix A).  (n <= k never
    reaches a rule: those equations use the start weights I_{0,n}.)"""
    assert n > k
    w = np.zeros(n + 1)
    if n < 2 * k + 1:
        w[:k + 1] += W.I(0, n - k)
        w[n - k:n + 1] += W.I(0, k)
        return w
    w[:] = 1.0
    w[:k + 1] = W.omega
    w[n - k:] = W.omega[::-1]
    return w


class RealSystem:
    """Equations sum_j A_j X_j B_j (or A_j X_j^dagger B_j) = rhs over
    N_o x N_o complex block unknowns X_j, as one real linear system."""

    def __init__(self, no):
        self.no = no
        self.keys = {}
        self.rows = []
        n2 = no * no
        self.P = np.zeros((n2, n2))
        for i in range(no):
            for j in range(no):
                self.P[i * no + j, j * no + i] = 1.0   # vec(X^T) = P vec(X), row-major

    def key(self, k):
        if k not in self.keys:
            self.keys[k] = len(self.keys)
        return k

    def eq(self, terms, rhs):
        for t in terms:
            self.key(t[1])
        self.rows.append((terms, rhs))

    def solve(self):
        no, n2 = self.no, self.no * self.no
        nu = len(self.keys)
        assert len(self.rows) == nu, (len(self.rows), nu)   # one equation per unknown
        M = np.zeros((2 * n2 * nu, 2 * n2 * nu))
        b = np.zeros(2 * n2 * nu)
        for r, (terms, rhs) in enumerate(self.rows):
            r0 = 2 * n2 * r
            for A, key, B, cj in terms:
                K = np.kron(A, B.T)                         # vec(A X B) = (A kron B^T) vec(X)
                c = 2 * n2 * self.keys[key]
                if not cj:
                    M[r0:r0 + n2, c:c + n2] += K.real
                    M[r0:r0 + n2, c + n2:c + 2 * n2] -= K.imag
                    M[r0 + n2:r0 + 2 * n2, c:c + n2] += K.imag
                    M[r0 + n2:r0 + 2 * n2, c + n2:c + 2 * n2] += K.real
                else:                                       # vec(A X^dag B) = K P conj(vec X)
                    KP = K @ self.P
                    M[r0:r0 + n2, c:c + n2] += KP.real
                    M[r0:r0 + n2, c + n2:c + 2 * n2] += KP.imag
                    M[r0 + n2:r0 + 2 * n2, c:c + n2] += KP.imag
                    M[r0 + n2:r0 + 2 * n2, c + n2:c + 2 * n2] -= KP.real
            v = np.asarray(rhs, dtype=complex).reshape(n2)
            b[r0:r0 + n2] = v.real
            b[r0 + n2:r0 + 2 * n2] = v.imag
        z = np.linalg.solve(M, b)
        out = {}
        for key, i in self.keys.items():
            c = 2 * n2 * i
            out[key] = (z[c:c + n2] + 1j * z[c + n2:c + 2 * n2]).reshape(no, no)
        return out


def global_solve(N, k, h, eps, gm, sigma):
    """Every stored entry of the discrete scheme for N time points, for the
    self-energy given by sigma = (SR[T, t], SLs[T, t] = Sigma^<(t, T),
    STV[T, i]) on the lower triangle.  Returns GR, GLs, GTV arrays."""
    SR, SLs, STV = sigma
    no = eps.shape[-1]
    r = len(TAU)
    I1 = np.eye(no, dtype=complex)
    Z = np.zeros((no, no), complex)
    W = Weights(k)
    a = W.a
    dl = DLROracle(TAU, OM, BETA, XI)
    e0, Rev, Q, Wc = dl.eval_row(0.0), dl.rev(), dl.Q(), dl.conv_tensor(gm)
    ep = lambda t: eps[t + 1]                                   # noqa: E731

    def sRx(p, q):     # Sigma^R(p, q), continued above the diagonal
        return SR[p, q] if p >= q else -_dag(SR[q, p])

    def sL(t, l):      # Sigma^<(t, l) anywhere
        return SLs[l, t] if t <= l else -_dag(SLs[t, l])

    S = RealSystem(no)
    R = lambda T, t: ("R", T, t)                                # noqa: E731
    M_ = lambda T, i: ("M", T, i)                               # noqa: E731
    Lk = lambda t, T: ("L", t, T) if t <= T else ("X", t, T)    # noqa: E731
    # ---- retarded ----
    for n in range(N):
        S.eq([(I1, R(n, n), I1, False)], -1j * I1)
    for n in range(min(k, N)):                    # start square: columns n, rows m = n+1..k
        for m in range(n + 1, min(k, N - 1) + 1):
            Inm = W.I(n, m)
            terms = []
            for l in range(k + 1):
                blk = (1j / h) * W.D[m, l] * I1 - h * Inm[l] * sRx(m, l)
                if l == m:
                    blk = blk - ep(m)
                if l >= n:
                    terms.append((blk, R(l, n), I1, False))
                else:
                    terms.append((-blk, R(n, l), I1, True))
            S.eq(terms, Z)
    for T in range(k + 1, N):                     # rows T > k, y_s = G^R(T, T-s)
        for s in range(1, T + 1):
            terms = []
            if s <= k:
                Is = W.I(0, s)
                for l in range(k + 1):
                    C = (1j / h) * W.D[s, l] * I1 - h * Is[l] * sRx(T - l, T - s)
                    terms.append((I1, R(T, T - l), C, False))
                terms.append((I1, R(T, T - s), -ep(T - s), False))
            else:
                w = _rule(W, k, s)
                for j in range(k + 1):
                    terms.append((I1, R(T, T - (s - j)), (1j / h) * a[j] * I1, False))
                terms.append((I1, R(T, T - s), -ep(T - s), False))
                for l in range(s + 1):
                    terms.append((I1, R(T, T - l), -h * w[l] * SR[T - l, T - s], False))
            S.eq(terms, Z)
    # ---- mixed ----
    g0 = 1j * XI * np.einsum("bc,cxy->bxy", Rev, gm)
    conv = lambda T: np.einsum("axy,aiyz->ixz", STV[T], Wc)    # noqa: E731
    for i in range(r):
        S.eq([(I1, M_(0, i), I1, False)], g0[i])
    for m in range(1, min(k, N - 1) + 1):
        Im = W.I(0, m)
        cv = conv(m)
        for i in range(r):
            terms = []
            for l in range(k + 1):
                blk = (1j / h) * W.D[m, l] * I1 - h * Im[l] * sRx(m, l)
                if l == m:
                    blk = blk - ep(m)
                terms.append((blk, M_(l, i), I1, False))
            S.eq(terms, cv[i])
    for T in range(k + 1, N):
        w = _rule(W, k, T)
        cv = conv(T)
        for i in range(r):
            terms = [((1j / h) * a[j] * I1, M_(T - j, i), I1, False) for j in range(k + 1)]
            terms.append((-ep(T), M_(T, i), I1, False))
            for l in range(T + 1):
                terms.append((-h * w[l] * SR[T, l], M_(l, i), I1, False))
            S.eq(terms, cv[i])
    # ---- lesser, column by column ----
    # G^vt(tau_b, T) = -xi [sum_c Rev[b, c] G^tv(T, tau_c)]^dagger, v_a = sum_b Q[a, b] G^vt(tau_b, T):
    # -i sum_a Sigma^tv(t, tau_a) v_a = sum_c coefv[c] (t) G^tv(T, tau_c)^dagger with
    # coefv[c](t) = i xi sum_a sum_b Q[a, b] Rev[b, c] Sigma^tv(t, tau_a)
    QR = Q @ Rev
    for T in range(N):
        # boundary value x_0 = -[G^tv(T, 0+)]^dagger
        S.eq([(I1, Lk(0, T), I1, False)] + [(e0[c] * I1, M_(T, c), I1, True) for c in range(r)], Z)
        if T == 0:
            continue

        def minus_q(t):
            """-q_t as terms (moved to the left-hand side)."""
            terms = []
            if T <= k:
                wts = W.I(0, T)
                for l in range(k + 1):
                    A = -h * wts[l] * sL(t, l)
                    if l <= T:
                        terms.append((A, R(T, l), I1, True))
                    else:
                        terms.append((-A, R(l, T), I1, False))
            else:
                wts = _rule(W, k, T)
                for l in range(T + 1):
                    terms.append((-h * wts[l] * sL(t, l), R(T, l), I1, True))
            for c in range(r):
                coef = 1j * XI * np.einsum("a,axy->xy", QR[:, c], STV[t])
                terms.append((-coef, M_(T, c), I1, True))
            return terms
        for t in range(1, k + 1):                 # start block t = 1..k
            It = W.I(0, t)
            terms = []
            for l in range(k + 1):
                blk = (1j / h) * W.D[t, l] * I1 - h * It[l] * sRx(t, l)
                if l == t:
                    blk = blk - ep(t)
                terms.append((blk, Lk(l, T), I1, False))
            S.eq(terms + minus_q(t), Z)
        for t in range(k + 1, T + 1):
            w = _rule(W, k, t)
            terms = [((1j / h) * a[j] * I1, Lk(t - j, T), I1, False) for j in range(k + 1)]
            terms.append((-ep(t), Lk(t, T), I1, False))
            for l in range(t + 1):
                terms.append((-h * w[l] * SR[t, l], Lk(l, T), I1, False))
            S.eq(terms + minus_q(t), Z)
    sol = S.solve()
    GR = np.zeros((N, N, no, no), complex)
    GLs = np.zeros((N, N, no, no), complex)
    GTV = np.zeros((N, r, no, no), complex)
    for T in range(N):
        for t in range(T + 1):
            GR[T, t] = sol[R(T, t)]
            GLs[T, t] = sol[("L", t, T)]
        for i in range(r):
            GTV[T, i] = sol[M_(T, i)]
    return GR, GLs, GTV


def _bath_sigma(N, h, V, eb):
    """Sigma = V g_b V^dagger of free bath levels (Sec. 3.3 forms): g^R =
    -i e^{-i eb (t-t')}, g^< = i n_b e^{-i eb (t-t')}, g^tv = -xi i n_b
    e^{-i eb t} e^{eb tau}."""
    no = V.shape[0]
    nb = 0.5 * (1.0 - np.tanh(0.5 * BETA * eb))
    dress = lambda g: np.einsum("xb,b,yb->xy", V, g, V.conj())   # noqa: E731
    SR = np.zeros((N, N, no, no), complex)
    SLs = np.zeros((N, N, no, no), complex)
    STV = np.zeros((N, len(TAU), no, no), complex)
    for T in range(N):
        for t in range(T + 1):
            SR[T, t] = dress(-1j * np.exp(-1j * eb * (T - t) * h))
            SLs[T, t] = dress(1j * nb * np.exp(-1j * eb * (t - T) * h))     # Sigma^<(t, T)
        for i, tau in enumerate(TAU):
            STV[T, i] = dress(-XI * 1j * nb * np.exp(-1j * eb * T * h) * np.exp(eb * tau))
    return SR, SLs, STV


def _stepped(N, k, h, eps, gm, model, tol=1e-15):
    o = KBEOracle(N, h, k, BETA, eps, gm, TAU, OM, model, tol=tol, boot_tol=tol, max_iter=200,
                  boot_max_iter=400)
    o.run()
    return o


def _diff(o, G):
    idx = np.tril_indices(o.nt)
    return max(np.abs(o.GR[idx] - G[0][idx]).max(), np.abs(o.GLs[idx] - G[1][idx]).max(),
               np.abs(o.GTV - G[2]).max())


EPS2 = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.4]])
V2 = np.array([[0.5, 0.3j], [-0.2, 0.4]])
EB2 = np.array([0.7, -0.9])


def _bath_case(N, k, h):
    from _closed_forms import quadratic
    H = np.block([[EPS2, V2], [V2.conj().T, np.diag(EB2)]])
    GM = quadratic(H, BETA, np.arange(2) * h, TAU, slice(0, 2))[3]
    eps = np.broadcast_to(EPS2, (N + 1, 2, 2)).astype(complex)
    return eps, GM


@pytest.mark.parametrize("k,N", [(1, 9), (2, 12)])
def test_bath_stepped_equals_global_solve(k, N):
    h = 0.1
    eps, GM = _bath_case(N, k, h)
    G = global_solve(N, k, h, eps, GM, _bath_sigma(N, h, V2, EB2))
    o = _stepped(N, k, h, eps, GM, make_model("bath", {"V": V2, "eb": EB2}))
    assert _diff(o, G) < 1e-13


@pytest.mark.parametrize("k,N", [(1, 8), (2, 12)])
def test_sigma0_stepped_equals_global_solve(k, N):
    h = 0.1
    eps = np.broadcast_to(EPS2, (N + 1, 2, 2)).astype(complex).copy()
    eps[3:] += np.diag([0.2, -0.1])               # a level change inside the grid
    GM = wk.free_level_gm(TAU, BETA, EPS2)
    zero = (np.zeros((N, N, 2, 2), complex), np.zeros((N, N, 2, 2), complex),
            np.zeros((N, len(TAU), 2, 2), complex))
    G = global_solve(N, k, h, eps, GM, zero)
    o = _stepped(N, k, h, eps, GM, make_model("none"))
    assert _diff(o, G) < 1e-13


def _bethe_global(N, k, h, eps, gm, v=1.0, tol=1e-15):
    """Global fixed point of the whole system with Sigma = v^2 G."""
    no, r = 1, len(TAU)
    G = (np.zeros((N, N, no, no), complex), np.zeros((N, N, no, no), complex), np.zeros((N, r, no, no), complex))
    for it in range(200):
        Gn = global_solve(N, k, h, eps, gm, tuple(v * v * x for x in G))
        d = max(np.abs(x - y).max() for x, y in zip(Gn, G))
        G = Gn
        if d < tol:
            return G
    raise AssertionError("global fixed point did not converge")


@pytest.mark.parametrize("k,N", [(1, 8), (2, 11)])
def test_bethe_stepped_equals_global_fixed_point(k, N):
    h = 0.05
    e0 = 0.2
    eps = np.full((N + 1, 1, 1), e0, complex)
    eps[6:] = 0.7                                 # quench inside the grid
    gm = wk.semicircle_gm(TAU, BETA, e0)[:, None, None].astype(complex)
    G = _bethe_global(N, k, h, eps, gm)
    o = _stepped(N, k, h, eps, gm, make_model("bethe", {"v": 1.0}))
    assert _diff(o, G) < 1e-13


# ---- planted mistakes in CPU copies of the stepper fail P6 ----------------

class _BadRule(Weights):
    """The k < n < 2k+1 rule with its shifted part one point too early."""

    def rule(self, n):
        w = super().rule(n).copy()
        if self.k < n < 2 * self.k + 1:
            w = np.zeros(n + 1)
            w[:self.k + 1] += self.I(0, n - self.k)
            w[n - self.k - 1:n] += self.I(0, self.k)
        return w


class _BadContinuation(KBEOracle):
    """solve_ret with the start-block kernel continued with its arguments
    swapped (Sigma^R(T-s, T-l) where the scheme has Sigma^R(T-l, T-s))."""

    def sR_x(self, a, b):
        if getattr(self, "_swap", False):
            return super().sR_x(b, a)
        return super().sR_x(a, b)

    def solve_ret(self, T):
        self._swap = True
        try:        # only the start block reads the continuation
            super().solve_ret(T)
        finally:
            self._swap = False


def test_planted_mistakes_fail_p6():
    k, N, h = 2, 12, 0.1
    eps, GM = _bath_case(N, k, h)
    G = global_solve(N, k, h, eps, GM, _bath_sigma(N, h, V2, EB2))
    model = make_model("bath", {"V": V2, "eb": EB2})
    o = KBEOracle(N, h, k, BETA, eps, GM, TAU, OM, model, tol=1e-15, boot_tol=1e-15, max_iter=200)
    o.W = _BadRule(k)
    o.run()
    assert _diff(o, G) > 1e-8
    o = _BadContinuation(N, h, k, BETA, eps, GM, TAU, OM, model, tol=1e-15, boot_tol=1e-15, max_iter=200)
    o.run()
    assert _diff(o, G) > 1e-8
