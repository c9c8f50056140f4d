"""Large-N parity: the N = 2^20 workload with ill-conditioned clusters.

Nodes x_k = 2 pi (k + u_k)/N, u_k ~ U(-0.45, 0.45), then 1% of the even
indices get t_i = t_{i+1} - d_i/N with d_i ~ U(0.01, 0.05) (seed 2).  A dense
O(N^3) solve is out of reach, so parity uses what the oracle can compute at
this size:
  * sparse known truth: 64 nonzero coefficients (resp. node amplitudes), the
    inputs built by exact-phase direct sums over the support only, and the
    full recovered vector compared element by element;
  * the residual of dense CN(0,1) data at 1024 sampled nodes (resp. 1024
    sampled frequencies), by exact-phase direct sums over all N terms.
The clusters make L'(z_p) small for the paired nodes and the weights lose
accuracy to cancellation, so these plans use the refined method of Sec. V
(NUFFT_REFINE: one correction from a float64 residual).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402

N = 1 << 20
CDT = {pkg.FP32: torch.complex64, pkg.FP64: torch.complex128}
TOL = {pkg.FP32: 1e-5, pkg.FP64: 1e-10}


@pytest.fixture(scope="module")
def nodes():
    pkg.build()
    oracle.build()
    return synth.clustered_nodes(N, 0.45, 0.01, 0.01, 0.05, seed=2)


def _sparse_coeffs(seed, k=64):
    g = synth.rng(seed)
    idx = np.sort(g.choice(N, k, replace=False))
    vals = synth.cn01(k, generator=g)
    return idx, vals


@pytest.mark.parametrize("prec", [pkg.FP32, pkg.FP64])
def test_inv5_sparse_known_truth(nodes, prec):
    idx, vals = _sparse_coeffs(5)
    f = np.zeros(N, complex)
    for m, v in zip(idx, vals):
        f += oracle.type2(nodes, np.array([v]), m0=int(m))
    c = np.zeros(N, complex)
    c[idx] = vals
    plan = pkg.Plan(torch.from_numpy(nodes).cuda(), prec=prec | pkg.REFINE)
    S = plan.inv5(torch.from_numpy(f).to(CDT[prec]).cuda()).cpu().numpy().astype(complex)
    assert oracle.rel_l2(S, c) <= TOL[prec]


@pytest.mark.parametrize("prec", [pkg.FP32, pkg.FP64])
def test_inv4_sparse_known_truth(nodes, prec):
    idx, vals = _sparse_coeffs(6)
    A = oracle.type1(nodes[idx], vals, M=N)
    a = np.zeros(N, complex)
    a[idx] = vals
    plan = pkg.Plan(torch.from_numpy(nodes).cuda(), prec=prec | pkg.REFINE)
    got = plan.inv4(torch.from_numpy(A).to(CDT[prec]).cuda()).cpu().numpy().astype(complex)
    assert oracle.rel_l2(got, a) <= TOL[prec]


@pytest.mark.parametrize("prec", [pkg.FP32, pkg.FP64])
def test_dense_residual_at_sampled_points(nodes, prec):
    """||G S - f|| over 1024 sampled nodes relative to ||f|| there (type-5),
    and the same for type-4 at 1024 sampled frequencies; bounded by the
    tolerance (the residual is the backward error, at most the forward error
    times ||G|| ||S|| / ||f||, of order one here)."""
    f = synth.cn01(N, seed=7)
    plan = pkg.Plan(torch.from_numpy(nodes).cuda(), prec=prec | pkg.REFINE)
    fr = f.astype(np.complex64).astype(complex) if prec == pkg.FP32 else f
    S = plan.inv5(torch.from_numpy(f).to(CDT[prec]).cuda()).cpu().numpy().astype(complex)
    q = np.sort(synth.rng(8).choice(N, 1024, replace=False))
    assert oracle.rel_l2(oracle.type2(nodes[q], S), fr[q]) <= 10 * TOL[prec]
    a = plan.inv4(torch.from_numpy(f).to(CDT[prec]).cuda()).cpu().numpy().astype(complex)
    k = np.sort(synth.rng(9).choice(N, 1024, replace=False))
    Ak = oracle.type1_at(nodes, a, k)
    assert oracle.rel_l2(Ak, fr[k]) <= 10 * TOL[prec]
