"""mm.map_solve, the torch.autograd.Function over the solver and its adjoint, on the CPU:
a stand-in plan with the library plan's solve / grad interface, computed by the oracle,
shows that the wrapper passes the map forward, sends dL/dm to the adjoint, returns
dL/dd and dL/dtheta to autograd, and skips what autograd does not need."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import adjoint
from oracle.pcg import dense_solve
from paper_1408_3048_gb300 import mm
from problems import oracle_problem, tiny_scan


class OraclePlan:
    """The Plan.solve / Plan.grad signatures, answered by the oracle (dense, tiny)."""

    def __init__(self, pr):
        self.pr = pr
        self.psds = np.array(pr.psds, dtype=np.float64)
        self.calls = []

    def solve(self, d, tol=1e-6, maxit=1000, kind=mm.MM_PREC_BD, solver=mm.MM_SOLVE_FP64, **kw):
        self.calls.append("solve")
        m = dense_solve(self.pr.dense_A(), self.pr.rhs(d.detach().numpy()))
        return torch.from_numpy(m), {"iters": 0}, mm.MM_OK

    def grad(self, d, m, g, tol=1e-10, maxit=10000, kind=mm.MM_PREC_BD, solver=mm.MM_SOLVE_FP64, want_d=True,
             want_psd=True):
        self.calls.append(("grad", want_d, want_psd))
        assert g.dtype == torch.float64
        dd, dp = adjoint.gradients(self.pr, d.numpy(), m.numpy(), g.numpy(), dense=True)
        return (torch.from_numpy(dd) if want_d else None), (dp if want_psd else None), {}


def test_map_solve_forward_and_backward():
    scan = tiny_scan(ncomp=3, psds=((1.0, 1.0, 1.3), (1.2, 0.6, 1.7)), lam=6)
    pr = oracle_problem(scan)
    plan = OraclePlan(pr)
    rng = np.random.default_rng(0)
    d = torch.from_numpy(rng.standard_normal(pr.nt)).requires_grad_(True)
    theta = torch.tensor(np.array(scan.psds), dtype=torch.float64, requires_grad=True)
    mref = torch.from_numpy(rng.standard_normal(pr.n))
    m = mm.map_solve(plan, d, theta)
    np.testing.assert_allclose(m.detach().numpy(), dense_solve(pr.dense_A(), pr.rhs(d.detach().numpy())))
    L = 0.5 * torch.sum((m - mref) ** 2)
    gd, gth = torch.autograd.grad(L, [d, theta])
    dd, dp = adjoint.gradients(pr, d.detach().numpy(), m.detach().numpy(), (m - mref).detach().numpy(), dense=True)
    np.testing.assert_allclose(gd.numpy(), dd, rtol=1e-12, atol=0)
    np.testing.assert_allclose(gth.numpy(), dp, rtol=1e-12, atol=0)
    assert plan.calls == ["solve", ("grad", True, True)]


def test_map_solve_skips_unneeded_gradients():
    scan = tiny_scan(ncomp=1, psds=((1.0, 1.0, 1.3),), lam=6)
    pr = oracle_problem(scan)
    plan = OraclePlan(pr)
    d = torch.from_numpy(np.random.default_rng(1).standard_normal(pr.nt)).requires_grad_(True)
    theta = torch.tensor(np.array(scan.psds), dtype=torch.float64)       # no gradient wanted
    (gd,) = torch.autograd.grad(mm.map_solve(plan, d, theta).sum(), [d])
    assert plan.calls[-1] == ("grad", True, False)
    # d/dd of sum(m) = N^-1 P A^-1 1: the adjoint with g = ones
    ref = pr.Ninv(pr.P(dense_solve(pr.dense_A(), np.ones(pr.n))))
    np.testing.assert_allclose(gd.numpy(), ref, rtol=1e-10, atol=1e-12)


def test_map_solve_rejects_theta_other_than_the_plans():
    scan = tiny_scan(ncomp=1, psds=((1.0, 1.0, 1.3),), lam=6)
    plan = OraclePlan(oracle_problem(scan))
    d = torch.zeros(plan.pr.nt, dtype=torch.float64)
    for bad in ([[1.0, 1.0, 1.4]], [[1.0, 1.0, 1.3], [1.0, 1.0, 1.3]]):
        with pytest.raises(ValueError):
            mm.map_solve(plan, d, torch.tensor(bad, dtype=torch.float64))
    assert plan.calls == []
