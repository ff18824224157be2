"""Pins of the oracle's sweep-free variant (oracle/sweepfree.py): the retarded
row from the Dyson equation in its first argument beyond the start block, and
the lesser column in its resolvent (Duhamel) form.  The variant is a different
discretisation of the same equations, so it is pinned where the equations fix
the answer: closed forms of quadratic models (Sigma = 0, a level coupled to a
bath, exact diagonalisation), the Bethe lattice's J1 form (self-consistent
Sigma = v^2 G), each at the order k of the weights when h is halved, and its
distance to the paper's scheme, which must shrink at the same order.  Planted
mistakes (a dropped lesser source, a wrong end weight) must fail the pins."""
import numpy as np
import pytest

import kbe_workloads as wk
from oracle.kbe import from_workload
from oracle.models import make_model
from oracle.sweepfree import SweepFreeOracle

from _closed_forms import bethe, quadratic

BETA = 5.0
TAU, OM = wk.dlr_grid(100.0, 1e-12, BETA)
EPS2 = np.array([[0.3, 0.2 - 0.1j], [0.2 + 0.1j, -0.4]])
V = np.array([[0.5, 0.3j], [-0.2, 0.4]])
EB = np.array([0.7, -0.9])


def _quadratic_error(model, H, nt, h, k, rho_mode=0, cls=SweepFreeOracle):
    eps = np.broadcast_to(EPS2, (nt + 1, 2, 2)).astype(complex)
    ts = np.arange(nt) * h
    GR, GL, GTV, GM = quadratic(H, BETA, ts, TAU, slice(0, 2))
    o = cls(nt, h, k, BETA, eps, GM, TAU, OM, model, tol=1e-14, rho_mode=rho_mode).run()
    idx = np.tril_indices(nt)
    return max(np.abs(o.GR[idx] - GR[idx]).max(), np.abs(o.GLs[idx] - np.swapaxes(GL, 0, 1)[idx]).max(),
               np.abs(o.GTV - GTV).max())


def test_sigma0_matrix_level_closed_form():
    """Sigma = 0, a non-diagonal Hermitian 2 x 2 level: the left BDF row and the
    Duhamel column reproduce G^R = -i e^{-i eps (t-t')} and the free G^<."""
    e = [_quadratic_error(make_model("none"), EPS2, nt, h, 4) for nt, h in [(32, 0.1), (64, 0.05)]]
    assert e[1] < 2e-7 and e[0] / e[1] > 2 ** 3.5, e


@pytest.mark.parametrize("rho_mode", [0, 1])
def test_bath_matches_exact_diagonalisation(rho_mode):
    """Two orbitals on two bath levels with a non-commuting V: operator order in
    the left-equation history sum and in G^R q of the Duhamel column."""
    H = np.block([[EPS2, V], [V.conj().T, np.diag(EB)]])
    model = make_model("bath", {"V": V, "eb": EB})
    e = [_quadratic_error(model, H, nt, h, 4, rho_mode) for nt, h in [(32, 0.1), (64, 0.05)]]
    assert e[1] < 5e-6 and e[0] / e[1] > 2 ** 3.5, e


def _bethe_pair(nt, h):
    w = wk.c1_workload(seed=0, nt=nt, h=h, k=5, dlr_eps=1e-12)
    paper = from_workload(w, tol=1e-14).run()
    o = from_workload(w, tol=1e-14)
    sf = SweepFreeOracle(o.nt, o.h, o.k, o.beta, o.eps, o.gm, o.tau, w["omega"], o.model, tol=1e-14).run()
    return w, paper, sf


def test_bethe_closed_form_order5_and_distance_to_paper_scheme():
    """Self-consistent Bethe lattice (Sigma = v^2 G), k = 5: the J1 closed form
    at fifth order, and the distance to the paper's scheme shrinking at the
    same order (both discretise the same equations)."""
    errs, dist = [], []
    for nt, h in [(40, 0.1), (80, 0.05)]:
        w, paper, sf = _bethe_pair(nt, h)
        e0 = w["eps"][0, 1, 0, 0].real
        GR, GL = bethe(np.full(nt, e0), h, nt, BETA, e0)
        idx = np.tril_indices(nt)
        errs.append(max(np.abs(sf.GR[..., 0, 0][idx] - GR[idx]).max(), np.abs(sf.GLs[..., 0, 0][idx] - GL.T[idx]).max()))
        dist.append(max(np.abs(sf.GR[idx] - paper.GR[idx]).max(), np.abs(sf.GLs[idx] - paper.GLs[idx]).max()))
    assert errs[1] < 5e-7 and errs[0] / errs[1] > 2 ** 4.5, errs
    assert dist[1] < 5e-7 and dist[0] / dist[1] > 2 ** 4.5, dist
    assert dist[1] > 1e-12          # a different discretisation, not the same one


def test_pin_catches_dropped_lesser_source(monkeypatch):
    """The bath pin fails when q is left out of the Duhamel column."""
    H = np.block([[EPS2, V], [V.conj().T, np.diag(EB)]])
    model = make_model("bath", {"V": V, "eb": EB})
    monkeypatch.setattr(SweepFreeOracle, "lesser_source",
                        lambda self, T: np.zeros((T + 1, 2, 2), complex))
    assert _quadratic_error(model, H, 32, 0.1, 4) > 1e-3


def test_pin_catches_wrong_end_weight(monkeypatch):
    """The bath pin fails when the first Gregory end weight of the left
    equation's history sum is perturbed."""
    H = np.block([[EPS2, V], [V.conj().T, np.diag(EB)]])
    model = make_model("bath", {"V": V, "eb": EB})
    orig = SweepFreeOracle.solve_ret

    def bad(self, T):
        rule = self.W.rule

        def bent(n):
            w = rule(n).copy()
            if n > self.k:
                w[0] *= 1.1
            return w
        self.W.rule = bent
        try:
            orig(self, T)
        finally:
            self.W.rule = rule
    monkeypatch.setattr(SweepFreeOracle, "solve_ret", bad)
    assert _quadratic_error(model, H, 32, 0.1, 4) > 1e-4
