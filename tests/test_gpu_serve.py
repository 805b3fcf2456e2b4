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
    reqs = serve.make_mix(10, scale=0.25)
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
