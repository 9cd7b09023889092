"""The likelihood-fit driver's host logic (Sec. 3's modified Newton), on objectives with
known maximisers (no GPU): paper_1105_5256_gb300.fit.fit only needs a callable returning
(value, gradient) in eta = (log kappa^2, log s) and an evaluation counter.

  * concave quadratic: the Newton step lands on the maximiser at once;
  * a non-quadratic concave objective with a flat direction: converges to the maximiser;
  * a start where the Hessian is indefinite: every accepted step increases the objective and
    stays inside the trust region (eigenvalues clamped negative, step halving).
"""
import numpy as np
import pytest

from paper_1105_5256_gb300.fit import fit


class Objective:
    def __init__(self, f, g):
        self.f, self.g = f, g
        self.evaluations = 0

    def __call__(self, eta):
        self.evaluations += 1
        eta = np.asarray(eta, dtype=np.float64)
        return float(self.f(eta)), np.asarray(self.g(eta), dtype=np.float64)


def test_concave_quadratic_is_solved_by_one_newton_step():
    star = np.array([np.log(0.3), np.log(2.5)])
    A = np.array([[3.0, 1.2], [1.2, 2.0]])
    obj = Objective(lambda e: -0.5 * (e - star) @ A @ (e - star), lambda e: -A @ (e - star))
    res = fit(obj, 0.5, 1.5, max_step=5.0)
    assert abs(np.log(res["kappa2"]) - star[0]) < 1e-8
    assert abs(np.log(res["scale"]) - star[1]) < 1e-8
    assert res["iterations"] <= 3


def test_non_quadratic_concave_objective_converges():
    star = np.array([0.4, -0.7])

    def f(e):
        d = e - star
        return -(d[0] ** 4) - 0.5 * d[1] ** 2 - 0.1 * (d[0] - d[1]) ** 2

    def g(e):
        d = e - star
        return np.array([-4 * d[0] ** 3 - 0.2 * (d[0] - d[1]), -d[1] + 0.2 * (d[0] - d[1])])

    res = fit(Objective(f, g), 3.0, 0.2, max_iter=60)
    assert abs(np.log(res["kappa2"]) - star[0]) < 1e-3
    assert abs(np.log(res["scale"]) - star[1]) < 1e-3


@pytest.mark.parametrize("start", [(20.0, 0.01), (1e-3, 50.0)])
def test_indefinite_start_takes_bounded_ascent_steps(start):
    star = np.array([0.2, 0.1])

    def f(e):
        return -np.log1p((e - star) @ (e - star))

    def g(e):
        d = e - star
        return -2 * d / (1 + d @ d)

    obj = Objective(f, g)
    res = fit(obj, *start, max_iter=80, max_step=1.0)
    path = np.array(res["path"])
    vals = path[:, 2]
    assert np.all(np.diff(vals) >= 0)
    steps = np.abs(np.diff(np.log(path[:, :2]), axis=0)).max(axis=1)
    assert np.all(steps <= 1.0 + 1e-12)
    assert abs(np.log(res["kappa2"]) - star[0]) < 1e-4
    assert abs(np.log(res["scale"]) - star[1]) < 1e-4
    assert res["evaluations"] == obj.evaluations
