"""Slice-sharded Parareal, emulated on one GPU (the multi-GPU layout for a
single instance: each GPU owns a contiguous block of time slices).

Two virtual ranks, each with its own copies of the state, F and G arrays and
its own CUDA stream, run implicit-Euler-coarse Parareal (Eq. 7) on their block
of slices through the library's propagators: the fine propagation of all own
slices at once (fine_propagate with an active mask), the serial coarse sweep
one slice at a time (coarse_propagate), and the correction F + (G_new - G_old).
The one exchange per sweep -- the state at the block boundary, Nx doubles --
goes from rank r to rank r + 1 through pinned host memory (a device-to-host
copy on rank r's stream, an event, a host-to-device copy on rank r + 1's
stream), and the increment norm is the maximum of the ranks' partial maxima.
After k iterations the result must equal one parareal_solve launch of k
iterations bit for bit.  Test infrastructure: the library itself has no
slice-sharded driver (every run here has one GPU).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03848_b300 import binding, build

    build.build()
    return binding


def _sharded_ie_parareal(B, prob, cfg, iters, blocks):
    P, Nx = cfg["P"], cfg["Nx"]
    R = len(blocks)
    streams = [torch.cuda.Stream() for _ in range(R)]
    U = [torch.zeros(P + 1, Nx, dtype=torch.float64, device="cuda") for _ in range(R)]
    F = [torch.zeros(P, Nx, dtype=torch.float64, device="cuda") for _ in range(R)]
    G = [torch.zeros(P, Nx, dtype=torch.float64, device="cuda") for _ in range(R)]
    host = torch.empty(Nx, dtype=torch.float64).pin_memory()
    payoff = prob.serial_fine().view(P + 1, Nx)[0].clone()
    torch.cuda.synchronize()
    owner = {n: r for r, (a, b) in enumerate(blocks) for n in range(a, b)}

    def one_slice(fn, r, n, V):
        # propagate slice n of V (a (P+1) x Nx state) on rank r's stream
        inp = torch.zeros(P, Nx, dtype=torch.float64, device="cuda")
        inp[n] = V[n]
        act = torch.zeros(P, dtype=torch.uint8, device="cuda")
        act[n] = 1
        out = torch.zeros(P, Nx, dtype=torch.float64, device="cuda")
        fn(inp.view(-1), out.view(-1), act)
        return out[n]

    def send(r, n):
        # state at boundary n from rank r to rank r + 1 through host memory
        with torch.cuda.stream(streams[r]):
            host.copy_(U[r][n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record()
        ev.synchronize()
        with torch.cuda.stream(streams[r + 1]):
            U[r + 1][n].copy_(host, non_blocking=True)
            torch.cuda.current_stream().synchronize()

    def sweep(k):
        # serial over the slices, pipelined across the ranks; k < 0: initial sweep
        n0 = max(k, 0)
        for n in range(n0, P):
            r = owner[n]
            with torch.cuda.stream(streams[r]):
                g_new = one_slice(prob.coarse_propagate, r, n, U[r])
                if k < 0:
                    U[r][n + 1] = g_new
                else:
                    U[r][n + 1] = F[r][n] + (g_new - G[r][n])
                G[r][n] = g_new
            if n + 1 < P and owner[n + 1] != r:
                send(r, n + 1)

    with torch.cuda.stream(streams[0]):
        U[0][0] = payoff
    sweep(-1)
    norms = []
    for k in range(iters):
        torch.cuda.synchronize()
        old = [u.clone() for u in U]
        # fine propagation of each rank's own slices n >= k, the ranks side by side
        for r, (a, b) in enumerate(blocks):
            with torch.cuda.stream(streams[r]):
                act = torch.zeros(P, dtype=torch.uint8, device="cuda")
                act[max(a, k):b] = 1
                inp = U[r][:P].contiguous()
                out = F[r].clone()
                prob.fine_propagate(inp.view(-1), out.view(-1), act)
                F[r] = out
        for s in streams:
            s.synchronize()
        # slice k is exact since iteration k - 1: its owner already holds it
        sweep(k)
        torch.cuda.synchronize()
        # increment norm: each rank's maximum over its boundaries n + 1, then the max
        part = []
        for r, (a, b) in enumerate(blocks):
            ns = [n + 1 for n in range(max(a, k), b)]
            if ns:
                d = (U[r][ns] - old[r][ns]).norm(dim=1) / U[r][ns].norm(dim=1)
                part.append(float(d.max()))
        norms.append(max(part))
    # gather: boundary n + 1 from the owner of slice n
    out = torch.empty(P + 1, Nx, dtype=torch.float64, device="cuda")
    out[0] = U[0][0]
    for n in range(P):
        out[n + 1] = U[owner[n]][n + 1]
    return out, norms


@pytest.mark.parametrize("blocks", [[(0, 4), (4, 8)], [(0, 3), (3, 5), (5, 8)]])
def test_slice_sharded_ie_parareal_equals_one_launch(B, blocks):
    cfg = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=256, P=8, fine_steps=128, coarse_steps=1)
    prob = B.Problem(cfg)
    for iters in (1, 3):
        got, norms = _sharded_ie_parareal(B, prob, cfg, iters, blocks)
        ref, rn, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=0.0, max_iter=iters)
        assert stats[0]["iterations"] == iters
        assert torch.equal(got.view(-1), ref), float((got.view(-1) - ref).abs().max())
        np.testing.assert_allclose(norms, rn[0, :iters], rtol=1e-12)


@pytest.mark.parametrize("part", ["16,4,1", "8,4,2"])
def test_slice_sharded_ie_parareal_equals_one_launch_inner_rows(B, monkeypatch, part):
    # partitions with inner rows per thread: the sweep's implicit Euler step and
    # coarse_propagate finish the step the same way (a second sweep over the
    # inner rows), so the sharded solve still equals one launch bit for bit
    monkeypatch.setenv("BSP_PARTITION", part)
    cfg = dict(K=1.0, sigma=0.3, r=0.03, T=0.5, Smax=4.0, Nx=2000, P=6, fine_steps=16, coarse_steps=2)
    prob = B.Problem(cfg)
    m, nw, c = (int(v) for v in part.split(","))
    assert prob.partition(0) == dict(M=m, NW=nw, C=c)
    got, norms = _sharded_ie_parareal(B, prob, cfg, 2, [(0, 3), (3, 6)])
    ref, rn, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=0.0, max_iter=2)
    assert torch.equal(got.view(-1), ref), float((got.view(-1) - ref).abs().max())
    np.testing.assert_allclose(norms, rn[0, :2], rtol=1e-12)
