"""Nonlinear FWI drivers over the library's misfit and gradient.

- ``lbfgs``: model updates m_k = m_{k-1} + alpha dm.  The descent direction
  dm = -H^-1 grad J comes from the limited-memory BFGS two-loop recursion
  (Nocedal 1980), and alpha from a backtracking line search on the
  sufficient-decrease (Armijo) condition (Nocedal & Wright 2006).  This is
  the paper's nonlinear FWI algorithm (Sec. 2.2).
- ``lbfgs_family``: the multiparameter form (Sec. 2.2, Sec. 3.7): the
  inversion parameters are the logarithms of family 1 (Vp, rho) or family 2
  (Vp, Ip = rho Vp), stacked into one vector for the same recursion, with
  bounds on Vp and rho mapped to bounds on those logarithms.
- ``shuffle_batches`` / ``sgd``: batchwise stochastic gradient descent.  The
  shots are randomly shuffled into batches of at most ``batchsize``, the last
  one taking the remainder, and each batch makes one steepest-descent update
  (Sec. 4.3, batchwise job scheduling).

Every misfit and gradient comes from ``smi.smi_fwi_gradient`` or
``smi.smi_fwi_gradient_family`` on the GPU.
The vectors of the recursion live on the model's device.  A trial model that
the library refuses (CFL or dispersion) counts as a failed line-search step.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class History:
    misfit: list = field(default_factory=list)   # J after every accepted update (J0 first)
    alpha: list = field(default_factory=list)    # accepted step lengths
    evaluations: int = 0                         # misfit + gradient evaluations


def _fwi_evaluator(rho, prob, srcs, recs, stf, dobs):
    """m -> (J, dJ/dm) through smi_fwi_gradient."""
    from . import smi

    def evaluate(vp):
        J, g = smi.smi_fwi_gradient(vp, rho, prob, srcs, recs, stf, dobs)
        return float(J.item()), g
    return evaluate


def two_loop(g, s_list, y_list):
    """-H g for the L-BFGS inverse-Hessian approximation built from the pairs
    (s_i, y_i), oldest first; H0 = (s.y / y.y) I of the newest pair."""
    q = g.clone()
    a = []
    for s, y in zip(reversed(s_list), reversed(y_list)):
        rho_i = 1.0 / float((y * s).sum())
        ai = rho_i * float((s * q).sum())
        q -= ai * y
        a.append((rho_i, ai))
    if s_list:
        s, y = s_list[-1], y_list[-1]
        q *= float((s * y).sum()) / float((y * y).sum())
    for (s, y), (rho_i, ai) in zip(zip(s_list, y_list), reversed(a)):
        bi = rho_i * float((y * q).sum())
        q += (ai - bi) * s
    return -q


def minimize_lbfgs(evaluate, m0, niter: int, memory: int = 5, first_step: float = 1.0, bounds: tuple | None = None,
                   c1: float = 1e-4, max_backtracks: int = 8, refused: tuple = ()):
    """L-BFGS on m -> (J, g) = evaluate(m).  first_step: the largest change
    of the first trial along the steepest-descent direction (and after a
    restart); other trials start from alpha = 1, halved until
    J(m + alpha d) <= J(m) + c1 alpha g.d.  bounds: (lo, hi) projection of
    every trial.  An exception in `refused` counts as a failed trial.
    Returns (m, History)."""
    hist = History()
    m = m0.clone()
    J, g = evaluate(m)
    hist.evaluations += 1
    hist.misfit.append(J)
    s_list, y_list = [], []
    for _ in range(niter):
        d = two_loop(g, s_list, y_list)
        slope = float((g * d).sum())
        if slope >= 0.0:                          # not a descent direction: restart
            s_list.clear()
            y_list.clear()
            d = -g
            slope = float((g * d).sum())
        alpha = 1.0 if s_list else first_step / max(float(d.abs().max()), 1e-30)
        accepted = False
        for _ in range(max_backtracks):
            trial = m + alpha * d
            if bounds is not None:
                trial = trial.clamp(bounds[0], bounds[1])
            try:
                Jt, gt = evaluate(trial)
                hist.evaluations += 1
            except refused:
                hist.evaluations += 1
                alpha *= 0.5
                continue
            if Jt <= J + c1 * alpha * slope:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            break
        s, y = trial - m, gt - g
        sy = float((s * y).sum())
        if sy > 1e-12 * float((s * s).sum()) ** 0.5 * float((y * y).sum()) ** 0.5:   # curvature condition
            s_list.append(s)
            y_list.append(y)
            if len(s_list) > memory:
                s_list.pop(0)
                y_list.pop(0)
        m, J, g = trial, Jt, gt
        hist.misfit.append(J)
        hist.alpha.append(alpha)
    return m, hist


def lbfgs(vp0, rho, prob, srcs, recs, stf, dobs, niter: int = 5, memory: int = 5, first_step: float = 50.0,
          bounds: tuple | None = None):
    """L-BFGS FWI of Vp (Sec. 2.2).  first_step: the largest model change
    (m/s) of the first trial step.  bounds: (vmin, vmax).  Returns
    (vp, History)."""
    from . import smi
    return minimize_lbfgs(_fwi_evaluator(rho, prob, srcs, recs, stf, dobs), vp0, niter, memory, first_step,
                          bounds, refused=(smi.SmiError,))


def family_parameters(vp, rho, family: int):
    """(log m1, log m2) stacked: family 1 (Vp, rho), family 2 (Vp, Ip = rho Vp)."""
    import torch
    return torch.stack([torch.log(vp), torch.log(rho if family == 1 else rho * vp)])


def family_model(m, family: int):
    """Inverse of family_parameters: (vp, rho)."""
    import torch
    vp = torch.exp(m[0]).contiguous()
    p2 = torch.exp(m[1])
    return vp, (p2 if family == 1 else p2 / vp).contiguous()


def family_bounds(vp_bounds, rho_bounds, family: int, like):
    """Bounds on the stacked log-parameters from bounds on Vp and rho (for
    family 2, Ip in [rho_min vp_min, rho_max vp_max])."""
    import torch
    lo2 = rho_bounds[0] if family == 1 else rho_bounds[0] * vp_bounds[0]
    hi2 = rho_bounds[1] if family == 1 else rho_bounds[1] * vp_bounds[1]
    one = torch.ones_like(like[0])
    lo = torch.stack([one * float(np.log(vp_bounds[0])), one * float(np.log(lo2))])
    hi = torch.stack([one * float(np.log(vp_bounds[1])), one * float(np.log(hi2))])
    return lo, hi


def _family_evaluator(prob, srcs, recs, stf, dobs, family: int):
    """m (stacked log-parameters) -> (J, dJ/dm) through smi_fwi_gradient_family
    with the log transform."""
    import torch
    from . import smi

    def evaluate(m):
        vp, rho = family_model(m, family)
        J, g1, g2 = smi.smi_fwi_gradient_family(vp, rho, prob, srcs, recs, stf, dobs, family=family, log=True)
        return float(J.item()), torch.stack([g1, g2])
    return evaluate


def lbfgs_family(vp0, rho0, prob, srcs, recs, stf, dobs, family: int = 2, niter: int = 5, memory: int = 5,
                 first_step: float = 0.02, vp_bounds: tuple | None = None, rho_bounds: tuple | None = None):
    """Multiparameter L-BFGS FWI in family 1 (Vp, rho) or 2 (Vp, Ip) on the
    logarithms of the parameters (Sec. 2.2, Sec. 3.7).  first_step: the
    largest change of a log-parameter in the first trial (0.02: about 2 %).
    vp_bounds, rho_bounds: (min, max), both or neither.  Returns
    (vp, rho, History)."""
    from . import smi
    m0 = family_parameters(vp0, rho0, family)
    bounds = None
    if vp_bounds is not None and rho_bounds is not None:
        bounds = family_bounds(vp_bounds, rho_bounds, family, m0)
    m, hist = minimize_lbfgs(_family_evaluator(prob, srcs, recs, stf, dobs, family), m0, niter, memory,
                             first_step, bounds, refused=(smi.SmiError,))
    vp, rho = family_model(m, family)
    return vp, rho, hist


def shuffle_batches(nshot: int, batchsize: int, seed: int = 0) -> list:
    """Random shuffle of the shot indices cut into batches of batchsize, the
    last batch taking the remainder."""
    order = np.random.default_rng(seed).permutation(nshot)
    return [order[k:k + batchsize] for k in range(0, nshot, batchsize)]


def sgd(vp0, rho, prob, srcs, recs, stf, dobs_list, batchsize: int, step: float = 20.0, seed: int = 0,
        bounds: tuple | None = None):
    """One epoch of batchwise SGD: for each shuffled batch, one steepest-
    descent update whose largest model change is `step` m/s.  dobs_list:
    observed data per shot (nt, nrec).  Returns (vp, History) with the
    misfit of every batch before its update."""
    hist = History()
    vp = vp0.clone()
    srcs = np.asarray(srcs)
    for batch in shuffle_batches(len(srcs), batchsize, seed):
        evaluate = _fwi_evaluator(rho, prob, srcs[batch], [recs[i] for i in batch], stf,
                                  [dobs_list[i] for i in batch])
        J, g = evaluate(vp)
        hist.evaluations += 1
        hist.misfit.append(J)
        vp = vp - (step / max(float(g.abs().max()), 1e-30)) * g
        if bounds is not None:
            vp = vp.clamp(bounds[0], bounds[1])
        hist.alpha.append(step)
    return vp, hist
