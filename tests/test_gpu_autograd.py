"""Differentiation through the library (GPU): the vector-Jacobian product of
the forward map (exact discrete adjoint with boundary-saving reconstruction)
against the FP64 oracle, against finite differences of the oracle's forward
map, and the torch.autograd.Function against the FWI-gradient entry point."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    from paper_2311_02293_gb300 import build
    build.build()
    from paper_2311_02293_gb300 import autograd, smi
    torch.cuda.init()
    return smi, autograd


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _probs(smi, w):
    return (smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb),
            O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm))


CASES = {
    "2d": lambda: S.tiny_2d(nz=40, nx=36, nt=130, nb=8, order=8, src=(8, 17), off_grid=True),
    "3d": lambda: S.tiny_3d(nz=24, nx=22, ny=20, nt=60, nb=6, off_grid=True),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_vjp_matches_oracle(mods, case):
    smi, _ = mods
    w = CASES[case]()
    gp, op = _probs(smi, w)
    rng = np.random.default_rng(11)
    g = rng.standard_normal((w.nt, len(w.recs[0]))).astype(np.float32)
    gv = smi.smi_forward_vjp(_dev(w.vp), _dev(w.rho), gp, w.srcs, w.recs, _dev(w.stf), _dev(g))
    seis = O.forward(op, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])
    # the oracle's gradient with residual seis - dobs = g
    _, ref, _ = O.gradient(op, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], seis - g.astype(np.float64))
    err = np.linalg.norm(gv.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-3


def test_vjp_dot_product_against_oracle_finite_differences(mods):
    """<(F(m+e dm) - F(m-e dm)) / 2e, g> (FP64 oracle) = <dm, J^T g> (GPU)."""
    smi, _ = mods
    w = CASES["2d"]()
    gp, op = _probs(smi, w)
    rng = np.random.default_rng(12)
    g = rng.standard_normal((w.nt, len(w.recs[0]))).astype(np.float32)
    vp = w.vp.astype(np.float64)
    dm = np.zeros_like(vp)
    dm[1:-1, 1:-1] = rng.standard_normal(dm[1:-1, 1:-1].shape)
    dm[vp >= vp.max()] = 0.0
    eps = 1e-3
    fp = O.forward(op, vp + eps * dm, w.rho, w.stf, w.srcs[0], w.recs[0])
    fm = O.forward(op, vp - eps * dm, w.rho, w.stf, w.srcs[0], w.recs[0])
    lhs = float(np.sum((fp - fm) / (2 * eps) * g))
    gv = smi.smi_forward_vjp(_dev(w.vp), _dev(w.rho), gp, w.srcs, w.recs, _dev(w.stf), _dev(g))
    rhs = float(np.sum(dm * gv.cpu().numpy().astype(np.float64)))
    assert abs(lhs - rhs) <= 1e-3 * abs(lhs)


def test_autograd_misfit_matches_fwi_gradient(mods):
    import torch
    smi, ag = mods
    w = S.layered_fault_2d(nz=50, nx=110, nt=260, nshot=2, order=4)
    w.srcs[:, 1] = [300.0, 900.0]
    gp = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    rho, stf = _dev(w.rho), _dev(w.stf)
    dobs = smi.smi_forward(_dev(w.vp_true), rho, gp, w.srcs, w.recs, stf, flat=True)
    vp = _dev(w.vp).requires_grad_(True)
    J = ag.misfit(vp, rho, gp, w.srcs, w.recs, stf, dobs)
    J.backward()
    J2, g2 = smi.smi_fwi_gradient(_dev(w.vp), rho, gp, w.srcs, w.recs, stf, dobs)
    assert abs(float(J.item()) - float(J2.item())) <= 1e-6 * float(J2.item())
    a, b = vp.grad.cpu().numpy(), g2.cpu().numpy()
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)


def test_autograd_gradient_descent_reduces_misfit(mods):
    """A few steepest-descent steps on the layered-fault stand-in lower J."""
    import torch
    smi, ag = mods
    w = S.layered_fault_2d(nz=50, nx=110, nt=260, nshot=2, order=4)
    w.srcs[:, 1] = [300.0, 900.0]
    gp = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    rho, stf = _dev(w.rho), _dev(w.stf)
    dobs = smi.smi_forward(_dev(w.vp_true), rho, gp, w.srcs, w.recs, stf, flat=True)
    vp = _dev(w.vp).requires_grad_(True)
    history = []
    for _ in range(4):
        J = ag.misfit(vp, rho, gp, w.srcs, w.recs, stf, dobs)
        history.append(float(J.item()))
        vp.grad = None
        J.backward()
        with torch.no_grad():
            step = 20.0 / vp.grad.abs().max()          # at most 20 m/s per cell
            vp -= step * vp.grad
    assert history[-1] < history[0]


@pytest.mark.parametrize("case", sorted(CASES))
def test_tape_reverse_pass_runs_no_forward_modelling(mods, case):
    """smi_forward_tape keeps the saved boundaries and the final state; the
    reverse pass from the tape takes no forward step (the call's stats count
    adjoint and reconstruction steps only) and equals smi_forward_vjp, which
    models the forward again; a tape serves one reverse pass."""
    import torch
    smi, _ = mods
    w = CASES[case]()
    gp, _ = _probs(smi, w)
    vp, rho, stf = _dev(w.vp), _dev(w.rho), _dev(w.stf)
    rng = np.random.default_rng(13)
    g = _dev(rng.standard_normal(w.nt * len(w.recs[0])).astype(np.float32))
    seis, tape = smi.smi_forward_tape(vp, rho, gp, w.srcs, w.recs, stf)
    ref_seis = smi.smi_forward(vp, rho, gp, w.srcs, w.recs, stf, flat=True)
    assert torch.equal(seis, ref_seis)
    gv = tape.vjp(g)
    st = smi.smi_last_stats()
    assert st["steps"][0] == 0 and st["steps"][1] == w.nt and st["steps"][2] == w.nt
    ref = smi.smi_forward_vjp(vp, rho, gp, w.srcs, w.recs, stf, g)
    assert float(torch.linalg.norm(gv - ref) / torch.linalg.norm(ref)) <= 1e-6
    with pytest.raises(smi.SmiError):
        tape.vjp(g)
    tape.free()


def test_autograd_backward_uses_the_tape(mods):
    """The autograd Function's gradient (tape reverse pass) equals the
    gradient of smi_fwi_gradient for the same misfit."""
    import torch
    smi, ag = mods
    w = CASES["3d"]()
    gp, op = _probs(smi, w)
    dobs = (0.7 * O.forward(op, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0])).astype(np.float32)
    vp = _dev(w.vp).requires_grad_(True)
    J = ag.misfit(vp, _dev(w.rho), gp, w.srcs, w.recs, _dev(w.stf), _dev(dobs).reshape(-1))
    J.backward()
    Jr, gr = smi.smi_fwi_gradient(vp.detach(), _dev(w.rho), gp, w.srcs, w.recs, _dev(w.stf), _dev(dobs))
    assert abs(float(J.item()) - float(Jr.item())) <= 1e-6 * abs(float(Jr.item()))
    assert float(torch.linalg.norm(vp.grad - gr) / torch.linalg.norm(gr)) <= 1e-5
