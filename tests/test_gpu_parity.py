"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle.

Tolerances (relative L2, the paper's error measure of Sec. VI):
  * float64 path: 1e-10 for the inverses (types 4, 5), 1e-12 for types 1, 2;
  * float32 path: 1e-5 for the inverses, 1e-6 for types 1, 2 (the float32
    rounding of the data is ~6e-8; spreading width 8 leaves ~4e-7);
  * plan quantities K_q, L'(z_p), w_p are always float64: 1e-10 for the
    float64 plan (gamma = 1000, eta = 4), 2e-6 for the float32 path's plan
    (gamma = 100, eta = 3: truncation ~0.4 gamma^-eta ~ 4e-7 in K, Sec. V;
    the weights add the width-12 kernel error through L'(z_p)).
Sizes span one to many CTA tiles and FFT passes, ragged tails, prime and
non-smooth N (Bluestein), and the N = 65536 workload in full.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402

FP32, FP64 = pkg.FP32, pkg.FP64
TOL_INV = {FP32: 1e-5, FP64: 1e-10}
TOL_FWD = {FP32: 1e-6, FP64: 1e-12}
TOL_PLAN = {FP32: 2e-6, FP64: 1e-10}
CDT = {FP32: torch.complex64, FP64: torch.complex128}


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    oracle.build()
    pkg.lib()


def _dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a)).to(CDT[prec]).cuda()


def _np(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def _close(got, ref, tol):
    """rel-L2 within tol, and no single element off by more than 30 tol times
    the reference's RMS value (a few wrong entries inside a passing rel-L2
    would break this)."""
    e = oracle.rel_l2(got, ref)
    rms = np.linalg.norm(ref) / np.sqrt(max(1, ref.size))
    m = np.abs(np.asarray(got) - ref).max() / rms if ref.size else 0.0
    return e <= tol and m <= 30 * tol


def _rounded(a, prec):
    """The input as the GPU sees it (complex64 rounding for FP32), in float64."""
    return a.astype(np.complex64).astype(np.complex128) if prec == FP32 else a


SIZES = [1, 2, 3, 17, 64, 255, 256, 1000, 1009, 4096]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("N", SIZES)
def test_plan_quantities(N, prec):
    x = synth.jittered_nodes(N, 0.45, seed=N)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    rho = plan.info()["rho"]
    K = _np(plan.export(0))
    D = _np(plan.export(1))
    w = _np(plan.export(2))
    assert oracle.rel_l2(K, oracle.kernel_samples(x, rho)) <= TOL_PLAN[prec]
    Do = oracle.deriv_samples(x)
    assert oracle.rel_l2(D, Do) <= TOL_PLAN[prec]
    assert oracle.rel_l2(w, oracle.weights(x, rho, Do)) <= TOL_PLAN[prec]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("N", SIZES)
def test_forward_transforms(N, prec):
    x = synth.jittered_nodes(N, 0.45, seed=N + 7)
    c = synth.cn01(N, seed=N + 8)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    cr = _rounded(c, prec)
    assert oracle.rel_l2(_np(plan.fwd2(_dev(c, prec))), oracle.type2(x, cr)) <= TOL_FWD[prec]
    assert oracle.rel_l2(_np(plan.fwd1(_dev(c, prec))), oracle.type1(x, cr)) <= TOL_FWD[prec]


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("N", SIZES)
def test_inverses_vs_lu(N, prec):
    """Element-by-element against Gaussian elimination on random data."""
    x = synth.jittered_nodes(N, 0.45, seed=N + 11)
    s = synth.cn01(N, seed=N + 12)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    sr = _rounded(s, prec)
    S_ref = oracle.inv5(x, sr)
    a_ref = oracle.inv4(x, sr)
    assert _close(_np(plan.inv5(_dev(s, prec))), S_ref, TOL_INV[prec])
    assert _close(_np(plan.inv4(_dev(s, prec))), a_ref, TOL_INV[prec])


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_cfg_n256_known_truth(prec):
    """N = 256, u ~ U(-0.3, 0.3), seed 0: c -> type-2 -> inv5 -> c and
    c -> type-1 -> inv4 -> c (exact-phase oracle sums make the inputs)."""
    N = 256
    g = synth.rng(0)
    x = synth.jittered_nodes(N, 0.3, generator=g)
    c = synth.cn01(N, generator=g)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    f = oracle.type2(x, c)
    A = oracle.type1(x, c)
    assert _close(_np(plan.inv5(_dev(f, prec))), c, TOL_INV[prec])
    assert _close(_np(plan.inv4(_dev(A, prec))), c, TOL_INV[prec])


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_equispaced_is_dft(prec):
    N = 512
    x = synth.equispaced_nodes(N)
    s = synth.cn01(N, seed=3)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    sr = _rounded(s, prec)
    assert oracle.rel_l2(_np(plan.inv5(_dev(s, prec))), np.fft.fft(sr) / N) <= TOL_INV[prec]
    assert oracle.rel_l2(_np(plan.inv4(_dev(s, prec))), np.fft.ifft(sr)) <= TOL_INV[prec]


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_batch_matches_single(prec):
    N = 3000
    x = synth.jittered_nodes(N, 0.4, seed=5)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    data = synth.cn01((5, N), seed=6)
    for op in ("inv5", "inv4", "fwd1", "fwd2"):
        fn = getattr(plan, op)
        batched = _np(fn(_dev(data, prec)))
        for b in range(5):
            single = _np(fn(_dev(data[b], prec)))
            np.testing.assert_array_equal(batched[b], single)


def test_node_order_is_free():
    """Permuting the nodes permutes the samples (inv5 input, inv4 output)."""
    N = 777
    x = synth.jittered_nodes(N, 0.45, seed=9)
    perm = synth.rng(10).permutation(N)
    s = synth.cn01(N, seed=11)
    p1 = pkg.Plan(torch.from_numpy(x).cuda(), prec=FP64)
    p2 = pkg.Plan(torch.from_numpy(x[perm]).cuda(), prec=FP64)
    S1 = _np(p1.inv5(_dev(s, FP64)))
    S2 = _np(p2.inv5(_dev(s[perm], FP64)))
    assert oracle.rel_l2(S2, S1) < 1e-12
    a1 = _np(p1.inv4(_dev(s, FP64)))
    a2 = _np(p2.inv4(_dev(s, FP64)))
    assert oracle.rel_l2(a2, a1[perm]) < 1e-12


def test_nodes_outside_one_period_wrap():
    N = 300
    x = synth.jittered_nodes(N, 0.45, seed=12)
    shift = 2 * np.pi * synth.rng(13).integers(-3, 4, size=N)
    s = synth.cn01(N, seed=14)
    p1 = pkg.Plan(torch.from_numpy(x).cuda(), prec=FP64)
    p2 = pkg.Plan(torch.from_numpy(x + shift).cuda(), prec=FP64)
    assert oracle.rel_l2(_np(p2.inv5(_dev(s, FP64))), _np(p1.inv5(_dev(s, FP64)))) < 1e-9


def test_duplicate_nodes_rejected():
    N = 100
    x = synth.jittered_nodes(N, 0.45, seed=15)
    x[40] = x[41] + 2 * np.pi   # the same node modulo 2 pi
    with pytest.raises(pkg.NufftError) as e:
        pkg.Plan(torch.from_numpy(x).cuda(), prec=FP64)
    assert e.value.status == "NUFFT_ERR_DUP_NODES"


def test_pinned_host_buffers_stream_ordered():
    """Pinned host buffers: the copies run on the library's copy streams and
    the calls return without waiting; after nufft_stream_check every output
    equals the device-buffer result, for pinned -> pinned, pinned -> device
    and device -> pinned, with calls queued back to back."""
    N = 4096
    x = torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=20)).cuda()
    f = synth.cn01((5, N), seed=21)
    A = synth.cn01((5, N), seed=22)
    plan = pkg.Plan(x, prec=FP32)
    ref5 = _np(plan.inv5(_dev(f, FP32)))
    ref4 = _np(plan.inv4(_dev(A, FP32)))
    fin = torch.from_numpy(f).to(torch.complex64).pin_memory()
    Ain = torch.from_numpy(A).to(torch.complex64).pin_memory()
    o5 = torch.empty_like(fin).pin_memory()
    o4 = torch.empty_like(Ain).pin_memory()
    d5 = torch.empty(5, N, dtype=torch.complex64, device="cuda")
    d4 = torch.empty_like(d5)
    o4b = torch.empty_like(Ain).pin_memory()
    plan.inv5(fin, out=o5)
    plan.inv4(Ain, out=o4)
    plan.inv5(fin, out=d5)
    plan.inv4(_dev(A, FP32), out=o4b)
    plan.inv4(Ain, out=d4)
    pkg.stream_check()
    for got, ref in ((o5, ref5), (o4, ref4), (d5, ref5), (o4b, ref4), (d4, ref4)):
        np.testing.assert_array_equal(_np(got), ref)


def test_deferred_duplicate_check():
    """NUFFT_DEFER_CHECK: the plan call returns without waiting; the
    duplicate-node condition surfaces in nufft_plan_check, and a plan of
    distinct nodes gives bit-identical results to a checked one."""
    N = 100
    x = synth.jittered_nodes(N, 0.45, seed=15)
    x[40] = x[41] + 2 * np.pi
    p = pkg.Plan(torch.from_numpy(x).cuda(), prec=FP64 | pkg.DEFER_CHECK)
    with pytest.raises(pkg.NufftError) as e:
        p.check()
    assert e.value.status == "NUFFT_ERR_DUP_NODES"
    p.close()
    N = 4096
    x = synth.jittered_nodes(N, 0.45, seed=18)
    f = synth.cn01((2, N), seed=19)
    for prec in (FP32, FP64):
        pd = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec | pkg.DEFER_CHECK)
        out_d = _np(pd.inv5(_dev(f, prec)))
        pd.check()
        pc = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
        pc.check()
        np.testing.assert_array_equal(out_d, _np(pc.inv5(_dev(f, prec))))


def test_host_buffers_match_device():
    N = 2048
    x = synth.jittered_nodes(N, 0.45, seed=16)
    f = synth.cn01((3, N), seed=17)
    plan_d = pkg.Plan(torch.from_numpy(x).cuda(), prec=FP32)
    plan_h = pkg.Plan(torch.from_numpy(x), prec=FP32)          # host nodes
    dev = _np(plan_d.inv5(_dev(f, FP32)))
    host_in = torch.from_numpy(f).to(torch.complex64).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    plan_h.inv5(host_in, out=host_out)       # pinned: copied on the library's copy streams
    pkg.stream_check()
    np.testing.assert_array_equal(host_out.numpy().astype(np.complex128), dev)
    pageable = torch.from_numpy(f).to(torch.complex64)
    np.testing.assert_array_equal(_np(plan_h.inv5(pageable)), dev)


def test_zero_batch_and_overlap():
    N = 64
    plan = pkg.Plan(torch.from_numpy(synth.jittered_nodes(N, 0.3, seed=1)).cuda(), prec=FP32)
    buf = torch.zeros(2, N, dtype=torch.complex64, device="cuda")
    L = pkg.lib()
    st = L.nufft_inv5(plan._h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()), 0, None)
    assert st == 0
    st = L.nufft_inv5(plan._h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf[1].data_ptr()), 2, None)
    assert st == 1   # overlapping input and output


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_n65536_known_truth(prec):
    """The N = 65536 workload: u ~ U(-0.45, 0.45), CN(0,1) coefficients, type-5
    and type-4 inputs from exact-phase oracle sums; full-vector comparison."""
    N = 65536
    g = synth.rng(1)
    x = synth.jittered_nodes(N, 0.45, generator=g)
    c = synth.cn01(N, generator=g)
    f = oracle.type2(x, c)
    A = oracle.type1(x, c)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    assert _close(_np(plan.inv5(_dev(f, prec))), c, TOL_INV[prec])
    assert _close(_np(plan.inv4(_dev(A, prec))), c, TOL_INV[prec])
    # batched right-hand sides as timed by the benchmark (more than one chunk
    # of the many-right-hand-side kernels, ragged)
    scales = [1, 1j, -1, 0.5, 2j, -0.25, 1 + 1j, 3, -2j, 0.125, 1 - 1j, -4, 0.75]
    fb = np.stack([sc * f for sc in scales])
    Sb = _np(plan.inv5(_dev(fb, prec)))
    for b, sc in enumerate(scales):
        assert oracle.rel_l2(Sb[b], sc * c) <= TOL_INV[prec]
    Ab = np.stack([sc * A for sc in scales[:11]])
    ab = _np(plan.inv4(_dev(Ab, prec)))
    for b, sc in enumerate(scales[:11]):
        assert oracle.rel_l2(ab[b], sc * c) <= TOL_INV[prec]


def test_n131072_known_truth_float32():
    """N = 131072: the scattering-store path without the fused pair (radix
    512 x 256 length-N passes) and the type-4 grid FFT that reads only the
    placed half of its 2^18-point grid; full-vector comparison with known
    truth from exact-phase direct sums."""
    N = 131072
    g = synth.rng(5)
    x = synth.jittered_nodes(N, 0.45, generator=g)
    c = synth.cn01(N, generator=g)
    f = oracle.type2(x, c)
    A = oracle.type1(x, c)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=FP32)
    fb = np.stack([f, -1j * f])
    Ab = np.stack([A, 2 * A])
    Sb = _np(plan.inv5(_dev(fb, FP32)))
    ab = _np(plan.inv4(_dev(Ab, FP32)))
    for b, sc in enumerate([1, -1j]):
        assert _close(Sb[b], sc * c, TOL_INV[FP32])
    for b, sc in enumerate([1, 2]):
        assert _close(ab[b], sc * c, TOL_INV[FP32])


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_refinement_on_clustered_nodes(prec):
    """Sec. V refinement on an ill-conditioned node set (1% of the nodes within
    0.01-0.05 grid spacings of a neighbour): the refined inverse meets the
    tolerance against LU and is no worse than the plain one."""
    N = 4096
    x = synth.clustered_nodes(N, 0.45, 0.01, 0.01, 0.05, seed=21)
    s = synth.cn01(N, seed=22)
    sr = _rounded(s, prec)
    S_ref = oracle.inv5(x, sr)
    a_ref = oracle.inv4(x, sr)
    plain = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    refined = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec | pkg.REFINE)
    for op, ref in (("inv5", S_ref), ("inv4", a_ref)):
        e0 = oracle.rel_l2(_np(getattr(plain, op)(_dev(s, prec))), ref)
        e1 = oracle.rel_l2(_np(getattr(refined, op)(_dev(s, prec))), ref)
        assert e1 <= TOL_INV[prec]
        assert e1 <= e0 * 1.01


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("N", [1, 17, 256, 1000, 1009, 4096])
def test_toeplitz_middle_stage_vs_lu(N, prec):
    """NUFFT_TOEPLITZ (the middle stage as S_m = c_m + rho^P c_{m+P}, c = L * A)
    against Gaussian elimination, element by element, at the default
    parameters."""
    x = synth.jittered_nodes(N, 0.45, seed=N + 31)
    s = synth.cn01(N, seed=N + 32)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec | pkg.TOEPLITZ)
    sr = _rounded(s, prec)
    assert oracle.rel_l2(_np(plan.inv5(_dev(s, prec))), oracle.inv5(x, sr)) <= TOL_INV[prec]
    assert oracle.rel_l2(_np(plan.inv4(_dev(s, prec))), oracle.inv4(x, sr)) <= TOL_INV[prec]


def test_toeplitz_avoids_rho_amplification():
    """float32 solves at a strong damping (gamma = 1e4, eta = 2): the scaled
    middle stage of Eqs. 37/30/31 loses accuracy with gamma, the convolution
    form keeps the float32 solve near its usual error."""
    N = 4096
    x = synth.jittered_nodes(N, 0.45, seed=41)
    s = synth.cn01(N, seed=42)
    sr = _rounded(s, FP32)
    ref5, ref4 = oracle.inv5(x, sr), oracle.inv4(x, sr)
    errs = {}
    for name, prec in (("scaled", FP32), ("toeplitz", FP32 | pkg.TOEPLITZ)):
        plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec, gamma=1e4, eta=2)
        errs[name] = max(oracle.rel_l2(_np(plan.inv5(_dev(s, FP32))), ref5),
                         oracle.rel_l2(_np(plan.inv4(_dev(s, FP32))), ref4))
    print(errs)
    assert errs["toeplitz"] <= TOL_INV[FP32]
    assert errs["toeplitz"] < errs["scaled"] / 3


@pytest.mark.parametrize("prec", [FP32, FP64, FP32 | pkg.REFINE])
def test_restored_plan_matches_plan(prec):
    """nufft_plan_restore from nufft_plan_save's K_q and L'(z_p): the node
    geometry, phases and weights are recomputed, the rest is taken over; every
    transform gives bit-identical results to the original plan, and a
    restored plan of duplicate nodes still reports them."""
    N = 3000
    x = torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=24)).cuda()
    p0 = pkg.Plan(x, prec=prec)
    K, D, prm = p0.save()
    p1 = pkg.Plan(x, prec=prec, saved=(K, D, prm))
    base = prec & 0xFF
    data = synth.cn01((3, N), seed=25)
    for op in ("inv5", "inv4", "fwd1", "fwd2"):
        a = _np(getattr(p0, op)(_dev(data, base)))
        b = _np(getattr(p1, op)(_dev(data, base)))
        np.testing.assert_array_equal(a, b)
    for which in (0, 1, 2):
        np.testing.assert_array_equal(_np(p0.export(which)), _np(p1.export(which)))
    xd = synth.jittered_nodes(100, 0.45, seed=15)
    pd = pkg.Plan(torch.from_numpy(xd).cuda(), prec=FP64)
    Kd, Dd, pr = pd.save()
    xd[40] = xd[41]
    with pytest.raises(pkg.NufftError) as e:
        pkg.Plan(torch.from_numpy(xd).cuda(), prec=FP64, saved=(Kd, Dd, pr))
    assert e.value.status == "NUFFT_ERR_DUP_NODES"


def _mixed_density_nodes(N, seed):
    """Half of the nodes packed into [0, 0.05) turns (about 5 per grid cell of
    the transforms' grid), the other half spread over [0.05, 1) (about 0.28
    per cell): the packed stretch overflows the node window of a spreading
    tile, the sparse one the grid window of an interpolation tile."""
    g = synth.rng(seed)
    t = np.concatenate([g.uniform(0.0, 0.05, N // 2), g.uniform(0.05, 1.0, N - N // 2)])
    return 2 * np.pi * g.permutation(t)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("nodes", ["jittered", "mixed"])
def test_many_right_hand_sides(prec, nodes):
    """20 right-hand sides (several chunks of the many-right-hand-side spread
    and interpolation kernels, the last one ragged): the forward transforms
    against exact-phase direct sums, element by element; on the jittered nodes
    also the inverses against Gaussian elimination."""
    N, B = 4096, 20
    x = synth.jittered_nodes(N, 0.45, seed=26) if nodes == "jittered" else _mixed_density_nodes(N, 27)
    data = synth.cn01((B, N), seed=28)
    plan = pkg.Plan(torch.from_numpy(x).cuda(), prec=prec)
    dr = _rounded(data, prec)
    A = _np(plan.fwd1(_dev(data, prec)))
    f = _np(plan.fwd2(_dev(data, prec)))
    for b in range(B):
        assert _close(A[b], oracle.type1(x, dr[b]), TOL_FWD[prec]), b
        assert _close(f[b], oracle.type2(x, dr[b]), TOL_FWD[prec]), b
    if nodes == "jittered":
        S = _np(plan.inv5(_dev(data, prec)))
        a = _np(plan.inv4(_dev(data, prec)))
        G = oracle.matrix(x)
        Sref = np.linalg.solve(G, dr.T).T
        aref = np.linalg.solve(G.conj().T, dr.T).T
        for b in range(B):
            assert _close(S[b], Sref[b], TOL_INV[prec]), b
            assert _close(a[b], aref[b], TOL_INV[prec]), b
