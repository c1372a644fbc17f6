"""The host logic of the flexible GMRES driver (paper_1901_08269_gb300/learned.py)
on a CPU stand-in for the context: a dense nonsymmetric matrix, checked
against a direct solve, with restarts and with a preconditioner that changes
at every step."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1901_08269_gb300 import learned  # noqa: E402


class DenseCtx:
    """apply / vec_dot / vec_axpby of a context, for a dense matrix A."""

    def __init__(self, A):
        self.A = torch.as_tensor(A)
        self.N = A.shape[0]

    def apply(self, x, y):
        y.copy_(self.A @ x)
        return y

    def vec_dot(self, a, b):
        return float(torch.dot(a, b))

    def vec_axpby(self, alpha, x, beta, y):
        y.copy_(alpha * x + beta * y)
        return y


def system(n=60, seed=0):
    r = np.random.default_rng(seed)
    A = np.eye(n) * 4.0 + r.standard_normal((n, n)) / np.sqrt(n)  # nonsymmetric, well conditioned
    b = r.standard_normal(n)
    return A, b


@pytest.mark.parametrize("m", [60, 7])  # no restart; restarts every 7 steps
def test_fgmres_matches_a_direct_solve(m):
    A, b = system()
    ctx = DenseCtx(A)
    x = torch.zeros(A.shape[0], dtype=torch.float64)
    its, rel = learned.fgmres(ctx, torch.as_tensor(b), x, lambda v, z: z.copy_(v), m=m, tol=1e-12, maxit=500)
    assert rel <= 1e-12 and its <= 500
    np.testing.assert_allclose(x.numpy(), np.linalg.solve(A, b), rtol=0, atol=1e-10)


def test_fgmres_with_a_preconditioner_that_changes_every_step():
    A, b = system(seed=1)
    ctx = DenseCtx(A)
    D = torch.as_tensor(np.diag(A).copy())
    step = [0]

    def prec(v, z):  # alternately Jacobi and a damped identity: not one linear map
        step[0] += 1
        z.copy_(v / D if step[0] % 2 else 0.3 * v)

    x = torch.zeros(A.shape[0], dtype=torch.float64)
    its, rel = learned.fgmres(ctx, torch.as_tensor(b), x, prec, m=20, tol=1e-11, maxit=500)
    assert rel <= 1e-11
    np.testing.assert_allclose(x.numpy(), np.linalg.solve(A, b), rtol=0, atol=1e-9)
