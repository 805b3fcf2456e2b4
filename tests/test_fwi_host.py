"""The FWI drivers' host logic (Sec. 2.2 L-BFGS, Sec. 4.3 batchwise SGD),
pinned on closed-form problems: the secant condition of the two-loop
recursion, minimisers of an ill-conditioned quadratic and of the
Rosenbrock function, and the shot partition of the shuffled batches."""
import numpy as np
import pytest
import torch

from paper_2311_02293_gb300 import fwi


def test_two_loop_satisfies_the_newest_secant_condition():
    """The BFGS inverse-Hessian update satisfies H y_k = s_k for its newest
    pair whatever the older ones, so -two_loop(y_k) = s_k."""
    rng = np.random.default_rng(3)
    s_list, y_list = [], []
    for _ in range(6):
        s = torch.from_numpy(rng.standard_normal(30))
        y = s + 0.3 * torch.from_numpy(rng.standard_normal(30))
        assert float((s * y).sum()) > 0
        s_list.append(s)
        y_list.append(y)
    d = fwi.two_loop(y_list[-1], s_list, y_list)
    assert torch.allclose(-d, s_list[-1], rtol=1e-10, atol=1e-12)


def test_two_loop_without_pairs_is_steepest_descent():
    g = torch.tensor([1.0, -2.0, 3.0], dtype=torch.float64)
    assert torch.equal(fwi.two_loop(g, [], []), -g)


def test_two_loop_equals_the_explicit_bfgs_inverse_update():
    """-two_loop(g) = H g with H from H0 = gamma I (gamma = s.y / y.y of the
    newest pair) and H <- (I - r s y^T) H (I - r y s^T) + r s s^T per pair."""
    rng = np.random.default_rng(5)
    n = 8
    S, Y = [], []
    for _ in range(4):
        s = rng.standard_normal(n)
        S.append(s)
        Y.append(s + 0.3 * rng.standard_normal(n))
    H = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1]) * np.eye(n)
    for s, y in zip(S, Y):
        r = 1.0 / (y @ s)
        H = (np.eye(n) - r * np.outer(s, y)) @ H @ (np.eye(n) - r * np.outer(y, s)) + r * np.outer(s, s)
    g = rng.standard_normal(n)
    d = fwi.two_loop(torch.from_numpy(g), [torch.from_numpy(s) for s in S], [torch.from_numpy(y) for y in Y])
    assert np.abs(d.numpy() + H @ g).max() <= 1e-12 * np.abs(H @ g).max()


def test_lbfgs_minimises_an_ill_conditioned_quadratic():
    """Condition number 100 in 20 dimensions."""
    rng = np.random.default_rng(4)
    n = 20
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = torch.from_numpy(Q @ np.diag(np.logspace(0, 2, n)) @ Q.T)
    xs = torch.from_numpy(rng.standard_normal(n))

    def evaluate(x):
        r = x - xs
        return float(0.5 * r @ A @ r), A @ r

    x0 = torch.zeros(n, dtype=torch.float64)
    x, hist = fwi.minimize_lbfgs(evaluate, x0, niter=70, memory=10, first_step=0.1)
    assert float(torch.linalg.norm(x - xs)) <= 1e-6 * float(torch.linalg.norm(x0 - xs))
    assert all(b <= a for a, b in zip(hist.misfit, hist.misfit[1:]))


def test_lbfgs_reaches_the_rosenbrock_minimum():
    def evaluate(x):
        a, b = float(x[0]), float(x[1])
        f = (1 - a) ** 2 + 100 * (b - a * a) ** 2
        g = torch.tensor([-2 * (1 - a) - 400 * a * (b - a * a), 200 * (b - a * a)], dtype=torch.float64)
        return f, g

    x, hist = fwi.minimize_lbfgs(evaluate, torch.tensor([-1.2, 1.0], dtype=torch.float64), niter=200, memory=5,
                                 first_step=0.5, max_backtracks=30)
    assert torch.allclose(x, torch.tensor([1.0, 1.0], dtype=torch.float64), atol=1e-4)


def test_bounds_and_refused_trials():
    """Trials are projected onto the bounds; a refused trial halves the step."""
    calls = []

    def evaluate(x):
        calls.append(float(x[0]))
        if float(x[0]) > 2.5:
            raise RuntimeError("refused")
        return float((x[0] - 10.0) ** 2), 2 * (x - 10.0)

    x, _ = fwi.minimize_lbfgs(evaluate, torch.tensor([0.0], dtype=torch.float64), niter=5, first_step=8.0,
                              bounds=(0.0, 3.0), refused=(RuntimeError,))
    assert float(x[0]) <= 2.5 and max(calls) <= 3.0


@pytest.mark.parametrize("nshot,bs", [(400, 50), (23, 5), (7, 10)])
def test_shuffled_batches_partition_the_shots(nshot, bs):
    batches = fwi.shuffle_batches(nshot, bs, seed=1)
    allshots = np.concatenate(batches)
    assert sorted(allshots.tolist()) == list(range(nshot))
    assert [len(b) for b in batches] == [bs] * (nshot // bs) + ([nshot % bs] if nshot % bs else [])
    again = fwi.shuffle_batches(nshot, bs, seed=1)
    assert all(np.array_equal(a, b) for a, b in zip(batches, again))


@pytest.mark.parametrize("family", [1, 2])
def test_family_parameters_round_trip_and_bounds(family):
    vp = torch.tensor([[1500.0, 2500.0], [3000.0, 4500.0]], dtype=torch.float64)
    rho = torch.tensor([[1000.0, 2000.0], [2200.0, 2600.0]], dtype=torch.float64)
    m = fwi.family_parameters(vp, rho, family)
    assert m.shape == (2, 2, 2)
    v2, r2 = fwi.family_model(m, family)
    assert torch.allclose(v2, vp, rtol=1e-14) and torch.allclose(r2, rho, rtol=1e-14)
    if family == 2:
        assert torch.allclose(torch.exp(m[1]), vp * rho, rtol=1e-14)
    lo, hi = fwi.family_bounds((1400.0, 4600.0), (900.0, 2700.0), family, m)
    assert torch.all(lo <= m) and torch.all(m <= hi)
    ip_lo = 900.0 if family == 1 else 900.0 * 1400.0
    assert torch.allclose(lo[1], torch.full_like(lo[1], np.log(ip_lo)))
