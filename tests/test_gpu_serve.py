"""Request server (continuous batching on one GPU): every result is the same
alone and in a concurrent mix, requests are admitted by device footprint,
over-budget requests fail cleanly, and latency statistics are reported."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2311_02293_gb300 import build
    build.build()
    from paper_2311_02293_gb300 import serve
    torch.cuda.init()
    dev = torch.device("cuda:0")
    reqs = serve.make_mix(10, scale=0.25, surveys=False)
    serve._prepare(reqs, dev)
    return serve, reqs, dev


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_mix_has_every_kind_and_both_dimensions(env):
    serve, reqs, dev = env
    assert {r.kind for r in reqs} >= {"gradient"} and any(r.w.ndim == 3 for r in reqs)
    assert len({(r.w.n, r.w.nt) for r in reqs}) > 3


def test_results_same_alone_and_in_mix(env):
    serve, reqs, dev = env
    alone, _ = serve.run_alone(reqs, dev)
    mix = serve.run_mix(reqs, dev, slots=4)
    assert mix["failed"] == 0
    for r, a, b in zip(reqs, alone, mix["outputs"]):
        assert _rel(b, a) <= 1e-6, r.kind
    # the mix overlapped: some request started before another finished
    res = sorted(mix["results"], key=lambda x: x["t_start"])
    assert any(res[k + 1]["t_start"] < res[k]["t_end"] for k in range(len(res) - 1))


def test_shots_of_one_survey_share_a_call(env):
    """Survey mix (two 2D surveys, one 3D survey): queued single-shot
    requests of one survey run as one shot-batched call with per-shot
    results; every request's output equals the same request run alone."""
    serve, _, dev = env
    reqs = serve.make_mix(14, seed=123, scale=0.25, surveys=True, n2d=2, n3d=1)
    serve._prepare(reqs, dev)
    alone, _ = serve.run_alone(reqs, dev)
    mix = serve.run_mix(reqs, dev, slots=2)
    assert mix["failed"] == 0
    assert mix["merged_calls"] >= 1 and mix["merged_requests"] >= 2 * mix["merged_calls"]
    worst = 0.0
    for r, a, b in zip(reqs, alone, mix["outputs"]):
        e = _rel(b, a)
        worst = max(worst, e)
        assert e <= 1e-6, r.kind
    print(f"survey mix: {mix['merged_calls']} merged calls carried {mix['merged_requests']} of {len(reqs)} "
          f"requests; largest difference from alone {worst:.1e}")


def test_an_invalid_request_fails_alone_in_a_merged_call(env):
    """Submission sizes a request without checking positions, so a request
    whose source lies outside the model can join a merged call: that call
    fails, the server runs the group's requests one by one, and only the
    invalid request reports the error."""
    serve, _, dev = env
    reqs = [r for r in serve.make_mix(16, seed=321, scale=0.25, surveys=True, n2d=1, n3d=1)
            if r.w.ndim == 2][:5]
    assert len(reqs) == 5
    serve._prepare(reqs, dev)
    alone, _ = serve.run_alone(reqs, dev)
    bad = reqs[2]
    bad.w.srcs = bad.w.srcs.copy()
    bad.w.srcs[0, 1] = 1e7                 # far outside the model
    mix = serve.run_mix(reqs, dev, slots=1)
    status = [r["status"] for r in mix["results"]]
    assert status[2] == -1, status
    assert all(st == 0 for k, st in enumerate(status) if k != 2), status
    assert mix["merged_calls"] >= 1
    for k in (0, 1, 3, 4):
        assert _rel(mix["outputs"][k], alone[k]) <= 1e-6


def test_per_shot_results_equal_single_shot_calls(env):
    """opts.per_shot: a 3-shot gradient call returns each shot's gradient
    and misfit, equal to the shot alone; the RTM images likewise."""
    import torch
    from paper_2311_02293_gb300 import synth as S
    serve, _, dev = env
    smi = serve.smi
    w = S.layered_fault_2d(nz=60, nx=150, nt=300, nshot=3, order=8)
    w.srcs[:, 1] = np.array([20.0, 70.0, 120.0]) * w.d[1]
    vp, rho, stf = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (w.vp, w.rho, w.stf))
    vpt = torch.from_numpy(w.vp_true).to(dev)
    p = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
    dobs = smi.smi_forward(vpt, rho, p, w.srcs, w.recs, stf, flat=True)
    ps = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, per_shot=True)
    J, g = smi.smi_fwi_gradient(vp, rho, ps, w.srcs, w.recs, stf, dobs)
    img = smi.smi_rtm(vp, rho, ps, w.srcs, w.recs, stf, dobs)
    assert g.shape == (3,) + tuple(w.vp.shape) and J.numel() == 3 and img.shape == g.shape
    n = w.nt * len(w.recs[0])
    Jsum, gsum = smi.smi_fwi_gradient(vp, rho, p, w.srcs, w.recs, stf, dobs)
    assert abs(float(J.sum()) - float(Jsum.item())) <= 1e-9 * float(Jsum.item())
    assert _rel(g.sum(0), gsum) <= 1e-6
    for s in range(3):
        one = w.subset([s])
        Js, gs = smi.smi_fwi_gradient(vp, rho, p, one.srcs, one.recs, stf, dobs[s * n:(s + 1) * n])
        assert abs(float(J[s]) - float(Js.item())) <= 1e-12 * float(Js.item())
        assert _rel(g[s], gs) <= 1e-6
        i1 = smi.smi_rtm(vp, rho, p, one.srcs, one.recs, stf, dobs[s * n:(s + 1) * n])
        assert _rel(img[s], i1) <= 1e-6


def test_budget_serialises_and_oversized_requests_fail(env):
    serve, reqs, dev = env
    small = [r for r in reqs if r.w.ndim == 2][:3]
    need = max(serve.smi.smi_query(r._dev[0], r._dev[1], r.prob, r.w.srcs, r.w.recs, r._stf,
                                   r.kind)[2] for r in small)
    mix = serve.run_mix(small, dev, slots=3, budget=int(need * 1.05))
    assert mix["failed"] == 0
    res = sorted(mix["results"], key=lambda x: x["t_start"])
    assert all(res[k + 1]["t_start"] >= res[k]["t_end"] - 1e-3 for k in range(len(res) - 1))
    tiny = serve.run_mix(small[:1], dev, slots=1, budget=1 << 20)
    assert tiny["failed"] == 1 and tiny["results"][0]["status"] == -4


def test_poisson_replay_reports_latency(env):
    serve, reqs, dev = env
    mix = serve.run_mix(reqs[:6], dev, slots=3, rate=20.0)
    assert mix["failed"] == 0
    assert 0 < mix["p50_s"] <= mix["p99_s"] and mix["requests_per_s"] > 0


def test_served_fp16_results_against_the_oracle(env):
    """One small request of each kind served with FP16 boundaries (the
    serving configuration) in one concurrent mix: each result's error against
    the FP64 oracle and against the plain FP32 method on the same GPU (direct
    call, FP32 boundaries).  Bars: seismograms 1e-4 (boundary storage does
    not enter the forward run); images and gradients 5e-3 against the oracle,
    the FP16 bar of the parity tests.  The measured values are printed."""
    import torch
    from oracle import oracle as O
    from paper_2311_02293_gb300 import synth as S
    serve, _, dev = env
    smi = serve.smi
    w2 = S.layered_fault_2d(nz=60, nx=150, nt=300, nshot=1, order=8)
    w3 = S.salt_3d(n=40, nt=160, nshot=1)
    w3.stf = S.ricker(w3.nt + 40, w3.dt, w3.fm)[40:].copy()
    cases = [("gradient", w2), ("forward", w3), ("rtm", w3)]
    reqs = []
    for kind, w in cases:
        prob = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb, shell_prec="f16")
        r = serve.Request(kind, w, prob)
        reqs.append(r)
    serve._prepare(reqs, dev)
    refs, plain = [], []
    for r in reqs:
        w = r.w
        op = O.Problem(w.n, w.d, w.nt, w.dt, order=w.order, nb=w.nb, fm=w.fm)
        vp_t = w.vp_true if w.vp_true is not None else w.vp
        d64 = O.forward(op, vp_t, w.rho, w.stf, w.srcs[0], w.recs[0])
        if r.kind != "forward":                 # observed data from the oracle, never from the GPU
            r.dobs = torch.from_numpy(d64.astype(np.float32).reshape(-1)).to(dev)
        p32 = smi.Problem(w.d, w.nt, w.dt, w.fm, order=w.order, nb=w.nb)
        vp, rho, _ = r._dev
        if r.kind == "forward":
            refs.append(O.forward(op, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0]).reshape(-1))
            plain.append(smi.smi_forward(vp, rho, p32, w.srcs, w.recs, r._stf, flat=True))
        elif r.kind == "rtm":
            refs.append(O.gradient(op, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], d64, mode="rtm")[1].reshape(-1))
            plain.append(smi.smi_rtm(vp, rho, p32, w.srcs, w.recs, r._stf, r.dobs).reshape(-1))
        else:
            refs.append(O.gradient(op, w.vp, w.rho, w.stf, w.srcs[0], w.recs[0], d64)[1].reshape(-1))
            plain.append(smi.smi_fwi_gradient(vp, rho, p32, w.srcs, w.recs, r._stf, r.dobs)[1].reshape(-1))
    mix = serve.run_mix(reqs, dev, slots=3)
    assert mix["failed"] == 0
    for r, out, ref, p in zip(reqs, mix["outputs"], refs, plain):
        e_ref = float(np.linalg.norm(out.double().cpu().numpy() - ref) / np.linalg.norm(ref))
        e_p = _rel(out, p)
        print(f"served FP16 {r.kind} ({r.w.ndim}D): vs oracle {e_ref:.2e}, vs plain FP32 {e_p:.2e}")
        assert e_ref <= (1e-4 if r.kind == "forward" else 5e-3)
