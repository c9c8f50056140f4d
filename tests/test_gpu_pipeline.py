"""Plans built on a second, higher-priority stream while the previous plan's
transforms run, with a step's type-5 and type-4 inverses on two further
streams side by side (the step schedule bench.py times), give the same
results, bit for bit, as the same calls made one after another on one
stream; and the results of that schedule stay within the FP32 tolerance of
the oracle's known truth on a sampled right-hand side."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1604_06236_gb300 as pkg  # noqa: E402


def _pipelined(xs, fs, As, outs, two=False):
    ss = torch.cuda.Stream()
    ps = torch.cuda.Stream(priority=-1)
    s4 = torch.cuda.Stream() if two else ss
    ss.wait_stream(torch.cuda.current_stream())
    ps.wait_stream(ss)
    s4.wait_stream(ss)

    def make(i):
        with torch.cuda.stream(ps):
            p = pkg.Plan(xs[i], prec=pkg.FP32 | pkg.DEFER_CHECK, stream=ps)
            e = torch.cuda.Event()
            e.record(ps)
        return p, e

    nxt = make(0)
    live = []
    for i in range(len(xs)):
        p, ready = nxt
        if i + 1 < len(xs):
            nxt = make(i + 1)
        ss.wait_event(ready)
        s4.wait_event(ready)
        p.inv5(fs[i], out=outs[i][0], stream=ss)
        p.inv4(As[i], out=outs[i][1], stream=s4)
        if two:
            d4 = torch.cuda.Event()
            d4.record(s4)
            ss.wait_event(d4)
        done = torch.cuda.Event()
        done.record(ss)
        live.append((p, done))
        while len(live) > 1:
            q, d = live.pop(0)
            ps.wait_event(d)
            q.check()
            q.close()
    for q, d in live:
        ps.wait_event(d)
        q.check()
        q.close()
    torch.cuda.current_stream().wait_stream(ss)
    torch.cuda.current_stream().wait_stream(ps)
    torch.cuda.current_stream().wait_stream(s4)
    torch.cuda.synchronize()


@pytest.mark.parametrize("two", [False, True], ids=["one_solve_stream", "inv5_inv4_side_by_side"])
@pytest.mark.parametrize("N,B,K", [(8192, 8, 5), (65536, 16, 4), (65536, 64, 3)])
def test_pipelined_plans_match_sequential(N, B, K, two):
    dev = torch.device("cuda", 0)
    xs = [torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=500 + i)).to(dev) for i in range(K)]
    fs = [torch.from_numpy(synth.cn01((B, N), seed=600 + i)).to(torch.complex64).to(dev) for i in range(K)]
    As = [torch.from_numpy(synth.cn01((B, N), seed=700 + i)).to(torch.complex64).to(dev) for i in range(K)]
    ref = []
    for i in range(K):
        p = pkg.Plan(xs[i], prec=pkg.FP32)
        ref.append((p.inv5(fs[i]).clone(), p.inv4(As[i]).clone()))
        p.close()
    torch.cuda.synchronize()
    outs = [(torch.empty_like(fs[i]), torch.empty_like(As[i])) for i in range(K)]
    _pipelined(xs, fs, As, outs, two)
    for i in range(K):
        assert torch.equal(outs[i][0], ref[i][0]), i
        assert torch.equal(outs[i][1], ref[i][1]), i


def test_pipelined_known_truth():
    """Right-hand side 0 of each kind built from known truth by the oracle's
    exact-phase direct sums at N = 8192; the pipelined schedule recovers the
    truth within the FP32 tolerance (1e-5 rel-L2) on every step."""
    import oracle
    oracle.build()
    dev = torch.device("cuda", 0)
    N, B, K = 8192, 4, 3
    xs_np = [synth.jittered_nodes(N, 0.45, seed=800 + i) for i in range(K)]
    xs = [torch.from_numpy(x).to(dev) for x in xs_np]
    c5 = [synth.cn01(N, seed=810 + i) for i in range(K)]
    a4 = [synth.cn01(N, seed=820 + i) for i in range(K)]
    fs, As = [], []
    for i in range(K):
        f = synth.cn01((B, N), seed=830 + i)
        A = synth.cn01((B, N), seed=840 + i)
        f[0] = oracle.type2(xs_np[i], c5[i])
        A[0] = oracle.type1(xs_np[i], a4[i])
        fs.append(torch.from_numpy(f).to(torch.complex64).to(dev))
        As.append(torch.from_numpy(A).to(torch.complex64).to(dev))
    outs = [(torch.empty_like(fs[i]), torch.empty_like(As[i])) for i in range(K)]
    _pipelined(xs, fs, As, outs, two=True)
    for i in range(K):
        s = outs[i][0][0].cpu().numpy().astype(np.complex128)
        a = outs[i][1][0].cpu().numpy().astype(np.complex128)
        e5 = np.linalg.norm(s - c5[i]) / np.linalg.norm(c5[i])
        e4 = np.linalg.norm(a - a4[i]) / np.linalg.norm(a4[i])
        assert e5 <= 1e-5 and e4 <= 1e-5, (i, e5, e4)


def test_transforms_replayed_from_cuda_graph():
    """inv5 and inv4 of a plan captured once in a CUDA graph and replayed on
    new data give the eager calls' results bit for bit: every launch of the
    FFT passes leaves its tile counters at zero for the next replay."""
    dev = torch.device("cuda", 0)
    N, B = 8192, 8
    p = pkg.Plan(torch.from_numpy(synth.jittered_nodes(N, 0.45, seed=900)).to(dev), prec=pkg.FP32)
    f_in = torch.zeros((B, N), dtype=torch.complex64, device=dev)
    A_in = torch.zeros_like(f_in)
    S_out = torch.empty_like(f_in)
    a_out = torch.empty_like(f_in)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        p.inv5(f_in, out=S_out, stream=s)   # first calls (one-time set-up) outside the capture
        p.inv4(A_in, out=a_out, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.inv5(f_in, out=S_out, stream=s)
        p.inv4(A_in, out=a_out, stream=s)
    torch.cuda.synchronize()
    for k in range(3):
        fk = torch.from_numpy(synth.cn01((B, N), seed=910 + k)).to(torch.complex64).to(dev)
        Ak = torch.from_numpy(synth.cn01((B, N), seed=920 + k)).to(torch.complex64).to(dev)
        f_in.copy_(fk)
        A_in.copy_(Ak)
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(S_out, p.inv5(fk)), k
        assert torch.equal(a_out, p.inv4(Ak)), k
    p.close()
