"""The FWI drivers on the GPU (Sec. 2.2 L-BFGS, Sec. 4.3 batchwise SGD):
updates of the layered-fault 2D stand-in's smoothed start model that lower
the misfit against data modelled in the true model."""
import numpy as np
import pytest

from paper_2311_02293_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2311_02293_gb300 import build
    build.build()
    from paper_2311_02293_gb300 import fwi, smi
    torch.cuda.init()
    w = S.layered_fault_2d(nz=60, nx=160, nt=500, nshot=4, order=8)
    w.srcs[:, 1] = [300.0, 800.0, 1300.0, 1700.0]
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(np.ascontiguousarray(getattr(w, k))).to(dev) for k in ("vp", "vp_true", "rho", "stf")}
    prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    dobs = [smi.smi_forward(t["vp_true"], t["rho"], prob, w.srcs[i:i + 1], w.recs[i:i + 1], t["stf"])[0]
            for i in range(len(w.srcs))]
    return fwi, w, t, prob, dobs


def test_lbfgs_lowers_the_misfit(env):
    fwi, w, t, prob, dobs = env
    """Six iterations from the smoothed start model (a strongly nonlinear
    problem: the misfit falls to about 0.77 of its start in this many)."""
    vp, hist = fwi.lbfgs(t["vp"], t["rho"], prob, w.srcs, w.recs, t["stf"], dobs, niter=6, first_step=100.0,
                         bounds=(float(w.vp.min()) * 0.9, float(w.vp.max()) * 1.1))
    print("L-BFGS misfit", hist.misfit, "evaluations", hist.evaluations)
    assert len(hist.misfit) == 7
    assert all(b < a for a, b in zip(hist.misfit, hist.misfit[1:]))
    assert hist.misfit[-1] <= 0.85 * hist.misfit[0]
    assert hist.alpha[1:] == [1.0] * 5                # quasi-Newton steps accepted at unit length


def test_sgd_epoch_lowers_the_misfit(env):
    import torch
    fwi, w, t, prob, dobs = env
    vp, hist = fwi.sgd(t["vp"], t["rho"], prob, w.srcs, w.recs, t["stf"], dobs, batchsize=3, step=15.0, seed=2)
    assert len(hist.misfit) == 2                      # batches of 3 and 1
    from paper_2311_02293_gb300 import smi
    J0 = float(smi.smi_fwi_gradient(t["vp"], t["rho"], prob, w.srcs, w.recs, t["stf"], dobs)[0].item())
    J1 = float(smi.smi_fwi_gradient(vp, t["rho"], prob, w.srcs, w.recs, t["stf"], dobs)[0].item())
    print("SGD epoch misfit", J0, "->", J1)
    assert J1 < J0


@pytest.mark.parametrize("family", [1, 2])
def test_multiparameter_lbfgs_lowers_the_misfit(env, family):
    """Vp and density together (Gardner density in the true and the start
    model), on the logarithms of family 1 (Vp, rho) or 2 (Vp, Ip), with the
    bounds mapped per family."""
    import torch
    fwi, w, t, prob, _ = env
    from paper_2311_02293_gb300 import smi
    rho_true = torch.from_numpy(S.gardner(w.vp_true)).cuda()
    rho0 = torch.from_numpy(S.gardner(w.vp)).cuda()
    dobs = [smi.smi_forward(t["vp_true"], rho_true, prob, w.srcs[i:i + 1], w.recs[i:i + 1], t["stf"])[0]
            for i in range(len(w.srcs))]
    vb = (float(w.vp.min()) * 0.9, float(w.vp.max()) * 1.1)
    rb = (float(rho0.min()) * 0.9, float(rho0.max()) * 1.1)
    vp, rho, hist = fwi.lbfgs_family(t["vp"], rho0, prob, w.srcs, w.recs, t["stf"], dobs, family=family,
                                     niter=6, first_step=0.03, vp_bounds=vb, rho_bounds=rb)
    print(f"family {family} misfit", hist.misfit, "evaluations", hist.evaluations)
    assert len(hist.misfit) == 7
    assert all(b < a for a, b in zip(hist.misfit, hist.misfit[1:]))
    assert hist.misfit[-1] <= 0.9 * hist.misfit[0]
    assert float(vp.min()) >= vb[0] * (1 - 1e-6) and float(vp.max()) <= vb[1] * (1 + 1e-6)
    assert float(rho.min()) > 0
