"""The largest sizes: N = 2^26 (a 2^27-point transforms' grid, three-pass
FFT plans, and the plan's log-kernel spectrum on the streaming double-float
passes, beyond the few-vector kernel's 2^26 points).

Jittered nodes u ~ U(-0.45, 0.45) (seed 11), float32 path at tol 1e-5.
Dense data is out of the oracle's reach at this size (O(N^2) direct sums), so
known truth has 64 nonzero coefficients (resp. node amplitudes) at random
positions; the inputs are the oracle's exact-phase direct sums over that
support (2^32 terms each), and the full recovered vector is compared with
the truth, in rel-L2 and element by element.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402

N = 1 << 26
TOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    pkg.build()
    oracle.build()
    x = synth.jittered_nodes(N, 0.45, seed=11)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=pkg.FP32)
    return x, plan


def _check(got, truth):
    """rel-L2 within tol, and no element off by more than 30 tol times the
    RMS of the truth's nonzero entries (the scale of the signal: the RMS over
    all 2^26 entries, nearly all zero, says nothing about one entry)."""
    e = oracle.rel_l2(got, truth)
    rms_nz = np.linalg.norm(truth) / np.sqrt(np.count_nonzero(truth))
    assert e <= TOL, e
    assert np.abs(got - truth).max() <= 30 * TOL * rms_nz
    return e


def test_inv5_n2p26(setup):
    x, plan = setup
    g = synth.rng(12)
    ms = np.sort(g.choice(N, 64, replace=False))
    vals = synth.cn01(64, generator=g)
    f = oracle.type2_at(x, vals, ms)
    c = np.zeros(N, complex)
    c[ms] = vals
    got = plan.inv5(torch.from_numpy(f).to(torch.complex64).cuda()).cpu().numpy().astype(complex)
    print("N=2^26 inv5 rel-L2 %.3e" % _check(got, c))


def test_inv4_n2p26(setup):
    x, plan = setup
    g = synth.rng(13)
    idx = np.sort(g.choice(N, 64, replace=False))
    vals = synth.cn01(64, generator=g)
    A = oracle.type1(x[idx], vals, M=N)
    a = np.zeros(N, complex)
    a[idx] = vals
    got = plan.inv4(torch.from_numpy(A).to(torch.complex64).cuda()).cpu().numpy().astype(complex)
    print("N=2^26 inv4 rel-L2 %.3e" % _check(got, a))
