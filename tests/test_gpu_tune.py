"""The parameter tuner (nufft_plan_tune): the chosen (gamma, eta, plan width)
is one of its candidates, is used by later plans with the same (N, precision,
tol), meets tol against the oracle's known truth, and is forgotten by
nufft_cache_clear."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()
    yield
    pkg.lib().nufft_cache_clear()


@pytest.mark.parametrize("prec,tol,N", [(pkg.FP32, 2e-5, 4000), (pkg.FP64, 3e-10, 1500)])
def test_tuned_parameters(prec, tol, N):
    x = synth.jittered_nodes(N, 0.45, seed=71)
    xt = torch.from_numpy(x).cuda()
    params, ms = pkg.plan_tune(xt, tol=tol, prec=prec, batch=4)
    assert ms > 0
    gammas = [30, 100, 300, 1000, 3000] if prec == pkg.FP32 else [100, 1000, 10000]
    assert params["gamma"] in gammas
    assert 0.4 * params["gamma"] ** -params["eta"] <= tol / 10
    assert 0.4 * params["gamma"] ** -(params["eta"] - 1) > tol / 10 or params["eta"] == 1
    plan = pkg.Plan(xt, tol=tol, prec=prec)
    info = plan.info()
    assert (info["gamma"], info["eta"], info["w_plan"]) == (params["gamma"], params["eta"], params["w_plan"])
    # known truth: c -> exact type-2 (oracle) -> inv5
    c = synth.cn01(N, seed=72)
    f = oracle.type2(x, c)
    dt = torch.complex64 if prec == pkg.FP32 else torch.complex128
    fr = f.astype(np.complex64).astype(complex) if prec == pkg.FP32 else f
    got = plan.inv5(torch.from_numpy(f).to(dt).cuda()).cpu().numpy().astype(complex)
    ref = oracle.inv5(x, fr)
    assert oracle.rel_l2(got, ref) <= tol
    plan.close()
    pkg.lib().nufft_cache_clear()
    assert pkg.Plan(xt, tol=tol, prec=prec).info()["gamma"] == (100.0 if prec == pkg.FP32 else 1000.0)
