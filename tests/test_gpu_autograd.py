"""Gradients of the differentiable inverses (torch.autograd) on the GPU.

Checked against the dense-oracle gradient (LU solves and exact-phase sums,
itself pinned by finite differences in test_oracle_pins.py) and against
central finite differences of the float64 GPU path (h = 1e-6).
Loss: L = sum |inv(d, x) - c_target|^2 with c_target independent of the truth.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402
from paper_1604_06236_gb300 import autograd as ag  # noqa: E402

CDT = {pkg.FP32: torch.complex64, pkg.FP64: torch.complex128}
# relative L2 of the gradients against the oracle: float64 path near the
# method's own accuracy; float32 path ~ its 1e-6 solve error amplified by the
# derivative (factor up to 2 pi N in s')
TOL_GRAD = {pkg.FP32: 2e-4, pkg.FP64: 1e-8}


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _setup(N, B, seed, shared=True):
    x = synth.jittered_nodes(N, 0.45, seed=seed) if shared else np.stack(
        [synth.jittered_nodes(N, 0.45, seed=seed + i) for i in range(B)])
    d = synth.cn01((B, N), seed=seed + 100)
    ct = synth.cn01((B, N), seed=seed + 200)
    return x, d, ct


@pytest.mark.parametrize("kind", [5, 4])
@pytest.mark.parametrize("prec", [pkg.FP64, pkg.FP32])
def test_gradients_vs_dense_oracle(kind, prec):
    N, B = 256, 3
    x, d, ct = _setup(N, B, seed=41 + kind)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    dt = torch.from_numpy(d).to(CDT[prec]).cuda().requires_grad_(True)
    ctt = torch.from_numpy(ct).to(CDT[prec]).cuda()
    fn = ag.inv5 if kind == 5 else ag.inv4
    out = fn(dt, xt, prec=prec)
    loss = (out - ctt).abs().pow(2).sum()
    loss.backward()
    solve = oracle.inv5 if kind == 5 else oracle.inv4
    vjp = oracle.inv5_vjp if kind == 5 else oracle.inv4_vjp
    dr = d.astype(np.complex64).astype(np.complex128) if prec == pkg.FP32 else d
    gx_ref = np.zeros(N)
    for b in range(B):
        g_out = 2 * (solve(x, dr[b]) - ct[b].astype(np.complex64 if prec == pkg.FP32 else np.complex128))
        g_d, g_x = vjp(x, dr[b], g_out)
        assert _rel(dt.grad[b].cpu().numpy().astype(np.complex128), g_d) <= TOL_GRAD[prec]
        gx_ref += g_x
    assert _rel(xt.grad.cpu().numpy(), gx_ref) <= TOL_GRAD[prec]


@pytest.mark.parametrize("kind", [5, 4])
def test_per_instance_nodes(kind):
    N, B = 200, 2
    x, d, ct = _setup(N, B, seed=61 + kind, shared=False)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    dt = torch.from_numpy(d).cuda().requires_grad_(True)
    ctt = torch.from_numpy(ct).cuda()
    fn = ag.inv5 if kind == 5 else ag.inv4
    loss = (fn(dt, xt, prec=pkg.FP64) - ctt).abs().pow(2).sum()
    loss.backward()
    solve = oracle.inv5 if kind == 5 else oracle.inv4
    vjp = oracle.inv5_vjp if kind == 5 else oracle.inv4_vjp
    for b in range(B):
        g_d, g_x = vjp(x[b], d[b], 2 * (solve(x[b], d[b]) - ct[b]))
        assert _rel(dt.grad[b].cpu().numpy(), g_d) <= TOL_GRAD[pkg.FP64]
        assert _rel(xt.grad[b].cpu().numpy(), g_x) <= TOL_GRAD[pkg.FP64]


@pytest.mark.parametrize("kind", [5, 4])
def test_gradients_vs_finite_differences(kind):
    """Central differences (h = 1e-6) of the float64 GPU path on 8 node
    coordinates, 4 data coordinates and 2 random directions."""
    N, B = 512, 2
    x, d, ct = _setup(N, B, seed=81 + kind)
    fn = ag.inv5 if kind == 5 else ag.inv4
    ctt = torch.from_numpy(ct).cuda()

    def loss(xv, dv):
        with torch.no_grad():
            return float((fn(dv, xv, prec=pkg.FP64) - ctt).abs().pow(2).sum().item())

    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    dt = torch.from_numpy(d).cuda().requires_grad_(True)
    (fn(dt, xt, prec=pkg.FP64) - ctt).abs().pow(2).sum().backward()
    gx = xt.grad.cpu().numpy()
    gd = dt.grad.cpu().numpy()
    h = 1e-6
    x0 = torch.from_numpy(x).cuda()
    d0 = torch.from_numpy(d).cuda()
    g = synth.rng(7)
    scale = np.abs(gx).max()
    for q in g.choice(N, 8, replace=False):
        e = torch.zeros(N, dtype=torch.float64, device="cuda")
        e[q] = h
        fd = (loss(x0 + e, d0) - loss(x0 - e, d0)) / (2 * h)
        assert abs(fd - gx[q]) <= 1e-4 * scale, (q, fd, gx[q])
    for _ in range(4):
        b, q = int(g.integers(B)), int(g.integers(N))
        e = torch.zeros((B, N), dtype=torch.complex128, device="cuda")
        e[b, q] = h
        fdr = (loss(x0, d0 + e) - loss(x0, d0 - e)) / (2 * h)
        fdi = (loss(x0, d0 + 1j * e) - loss(x0, d0 - 1j * e)) / (2 * h)
        assert abs(complex(fdr, fdi) - gd[b, q]) <= 1e-4 * np.abs(gd).max()
    for _ in range(2):
        v = g.normal(size=N)
        v /= np.linalg.norm(v)
        vt = torch.from_numpy(v).cuda()
        fd = (loss(x0 + h * vt, d0) - loss(x0 - h * vt, d0)) / (2 * h)
        assert abs(fd - gx @ v) <= 1e-4 * np.linalg.norm(gx)


def test_full_size_finite_differences():
    """The N = 262144 differentiable workload (instances with their own nodes,
    seeds 4 + i), float64 path: central differences (h = 1e-6) on 8 node
    coordinates and 2 random directions per instance against autograd."""
    N, B = 262144, 2
    x = np.stack([synth.jittered_nodes(N, 0.45, seed=4 + i) for i in range(B)])
    f = synth.cn01((B, N), seed=50)
    ct = synth.cn01((B, N), seed=51)
    ctt = torch.from_numpy(ct).cuda()
    x0 = torch.from_numpy(x).cuda()
    f0 = torch.from_numpy(f).cuda()

    def loss(xv):
        with torch.no_grad():
            return float((ag.inv5(f0, xv, prec=pkg.FP64) - ctt).abs().pow(2).sum().item())

    xt = x0.clone().requires_grad_(True)
    (ag.inv5(f0, xt, prec=pkg.FP64) - ctt).abs().pow(2).sum().backward()
    gx = xt.grad.cpu().numpy()
    h = 1e-6
    g = synth.rng(12)
    for b in range(B):
        scale = np.abs(gx[b]).max()
        for q in g.choice(N, 8, replace=False):
            e = torch.zeros((B, N), dtype=torch.float64, device="cuda")
            e[b, q] = h
            fd = (loss(x0 + e) - loss(x0 - e)) / (2 * h)
            assert abs(fd - gx[b, q]) <= 1e-3 * scale, (b, q, fd, gx[b, q])
        for _ in range(2):
            v = np.zeros((B, N))
            v[b] = g.normal(size=N)
            v /= np.linalg.norm(v)
            vt = torch.from_numpy(v).cuda()
            fd = (loss(x0 + h * vt) - loss(x0 - h * vt)) / (2 * h)
            assert abs(fd - (gx * v).sum()) <= 1e-3 * np.linalg.norm(gx[b])


@pytest.mark.parametrize("kind", [5, 4])
def test_fp32_gradients_vs_dense_oracle_n1024(kind):
    """The differentiable workload's node law (u ~ U(-0.45, 0.45)) and data
    type (complex64) at the largest size the dense oracle handles quickly:
    gradients with respect to the data and the nodes against the oracle's LU
    and exact-phase gradient, for 2 instances with their own nodes."""
    N, B = 1024, 2
    x, d, ct = _setup(N, B, seed=91 + kind, shared=False)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    dt = torch.from_numpy(d).to(torch.complex64).cuda().requires_grad_(True)
    ctt = torch.from_numpy(ct).to(torch.complex64).cuda()
    fn = ag.inv5 if kind == 5 else ag.inv4
    (fn(dt, xt, prec=pkg.FP32) - ctt).abs().pow(2).sum().backward()
    solve = oracle.inv5 if kind == 5 else oracle.inv4
    vjp = oracle.inv5_vjp if kind == 5 else oracle.inv4_vjp
    dr = d.astype(np.complex64).astype(np.complex128)
    cr = ct.astype(np.complex64).astype(np.complex128)
    for b in range(B):
        g_d, g_x = vjp(x[b], dr[b], 2 * (solve(x[b], dr[b]) - cr[b]))
        assert _rel(dt.grad[b].cpu().numpy().astype(np.complex128), g_d) <= TOL_GRAD[pkg.FP32]
        assert _rel(xt.grad[b].cpu().numpy(), g_x) <= TOL_GRAD[pkg.FP32]


def test_full_size_fp32_gradients_vs_fp64():
    """The N = 262144 differentiable workload in its own precision: complex64
    samples, the float32-split path, instances with their own nodes (seeds
    4 + i, 4 of the 64), loss ||c_hat - c_target||^2.  Gradients with respect
    to the samples and the nodes against the float64 GPU path on the same
    (complex64-rounded) inputs, whose gradients the central-difference test
    above pins at this size."""
    N, B = 262144, 4
    x = np.stack([synth.jittered_nodes(N, 0.45, seed=4 + i) for i in range(B)])
    f = synth.cn01((B, N), seed=50).astype(np.complex64)
    ct = synth.cn01((B, N), seed=51).astype(np.complex64)
    grads = {}
    for prec, dt in ((pkg.FP32, torch.complex64), (pkg.FP64, torch.complex128)):
        xt = torch.from_numpy(x).cuda().requires_grad_(True)
        ft = torch.from_numpy(f).to(dt).cuda().requires_grad_(True)
        ctt = torch.from_numpy(ct).to(dt).cuda()
        (ag.inv5(ft, xt, prec=prec) - ctt).abs().pow(2).sum().backward()
        grads[prec] = (ft.grad.cpu().numpy().astype(np.complex128), xt.grad.cpu().numpy())
    gf32, gx32 = grads[pkg.FP32]
    gf64, gx64 = grads[pkg.FP64]
    for b in range(B):
        assert _rel(gf32[b], gf64[b]) <= TOL_GRAD[pkg.FP32], (b, _rel(gf32[b], gf64[b]))
        assert _rel(gx32[b], gx64[b]) <= TOL_GRAD[pkg.FP32], (b, _rel(gx32[b], gx64[b]))
