"""Parity at the full sizes of the benchmark workloads, in the launch
configurations bench.py times: sampled outputs against the oracle, and
properties that hold at any size.

* Benchmark workload (Nx = 1024, P = 32, 1024 Crank-Nicolson steps per slice,
  the built-in partition): the network-coarse solve with the BF16 table on the
  tensor cores needs k = P iterations and then equals the GPU serial fine
  solution bitwise (that serial fine solution is held to the oracle at this
  size in test_gpu_solver.py).
* Batched workload (4096 seeded instances, P = 64, 256 steps per slice,
  autotuned partitions): one fine propagation of every slice of the batch,
  sampled (instance, slice) outputs against the oracle; the implicit-Euler-coarse
  solve of the whole batch to 1e-6, sampled instances against the oracle's
  serial fine solution; the network-coarse solves (network-anchored IE to
  1e-6, and three iterations of the state-independent kind) of the whole batch
  with an FP64 table, one instance of every grid size against the oracle's
  Parareal.
* Large instance (Nx = 65536, P = 256, 4096 steps per slice, two slices per CTA
  on 16-CTA clusters): the first slice of GPU serial fine against the oracle;
  two implicit-Euler-coarse Parareal iterations leave the first three slices
  equal to GPU serial fine bitwise.
* Training workload (2->6x128, 65536 collocation points): every layer's BF16
  and TF32 tensor-core gradients against the oracle's FP64 gradient of the
  whole batch (computed in host threads from single-term chunks) and against
  the FP32 CUDA-core gradient of the same batch.

FP64 tolerance: max(1e-12, 2 kappa u N) as in test_gpu_solver.py (kappa the
mesh-ratio factor of the right-hand side, u = 2^-53, N the steps).
"""
import numpy as np
import pytest

from paper_2303_03848_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03848_b300 import binding, build

    build.build()
    return binding


def _kappa_tol(p, steps):
    h = 0.5 * p["T"] / (p["P"] * p["fine_steps"])
    j = p["Nx"] - 2
    kappa = 1.0 + h * (2.0 * p["sigma"] ** 2 * j * j + p["r"] * j + p["r"])
    return max(1e-12, 2.0 * kappa * 2.0 ** -53 * steps)


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_benchmark_network_solve_full_size_is_serial_fine(B):
    cfg = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=1024, P=32, fine_steps=1024, coarse_steps=1)
    prob = B.Problem(cfg)
    assert prob.partition(0) == dict(M=2, NW=4, C=4)
    net = B.PinnModel([2, 64, 64, 64, 64, 1], [0.0, 0.0], [4.0, 1.0], seed=0)
    U, norms, stats, rc = prob.parareal_solve(B.COARSE_PINN, model=net, prec=B.BF16, tol=1e-6, max_iter=32)
    Uf = prob.serial_fine()
    torch.cuda.synchronize()
    assert stats[0]["iterations"] == 32 and prob.device_status() == B.BS_OK
    assert torch.equal(U, Uf)


def test_batched_workload_full_size_sampled_against_oracle(B, orc):
    insts = synth.batched_instances(0, 4096, P=64, fine_steps=256, coarse_steps=1)
    prob = B.Problem(insts, tuned=True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    Uin = torch.rand(prob.total_slice, dtype=torch.float64, device="cuda", generator=gen)
    # one instance of every grid size, first and last slice; their inputs get the
    # exact Dirichlet nodes at tau_n (the other slices are independent of them)
    seen, picks = set(), []
    for i, p in enumerate(insts):
        if p["Nx"] not in seen:
            seen.add(p["Nx"])
            picks.append(i)
    assert len(picks) == 5
    for i in picks:
        p = insts[i]
        op = orc.params(**p)
        for n in (0, p["P"] - 1):
            o = prob.slice_off[i] + n * p["Nx"]
            Uin[o] = 0.0
            Uin[o + p["Nx"] - 1] = orc.right_bc(op, p["T"] * n / p["P"])
    Fo = prob.fine_propagate(Uin)
    torch.cuda.synchronize()
    assert prob.device_status() == B.BS_OK
    for i in picks:
        p = insts[i]
        op = orc.params(**p)
        for n in (0, p["P"] - 1):
            o = prob.slice_off[i] + n * p["Nx"]
            v_in = Uin[o:o + p["Nx"]].cpu().numpy()
            got = Fo[o:o + p["Nx"]].cpu().numpy()
            err = _rel(got, orc.fine(op, n, v_in))
            assert err <= _kappa_tol(p, p["fine_steps"]), (i, p["Nx"], n, err)
    # the implicit-Euler-coarse solve of the whole batch to 1e-6
    U, norms, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=1e-6, max_iter=64)
    assert rc == B.BS_OK and all(st["status"] == B.BS_OK for st in stats)
    for i in picks[:3]:  # Nx = 256 .. 1024 keeps the oracle's serial fine quick
        p = insts[i]
        op = orc.params(**p)
        o = prob.state_off[i]
        Ui = U[o:o + (p["P"] + 1) * p["Nx"]].cpu().numpy()
        assert orc.rel_error(op, Ui, orc.serial_fine(op)) <= 1e-6, (i, p["Nx"])


def _one_per_grid_size(insts):
    seen, picks = set(), []
    for i, p in enumerate(insts):
        if p["Nx"] not in seen:
            seen.add(p["Nx"])
            picks.append(i)
    return picks


def test_batched_network_coarse_full_size_sampled_against_oracle(B, orc):
    # the batched workload's network-coarse solves, every instance in one call
    # as bench.py runs them: a 5-input network on (S, tau, sigma, r, K) with an
    # FP64 table, network-anchored IE and state-independent kinds to 1e-6; one
    # instance of every grid size against the oracle's Parareal with the
    # oracle's own table (same iteration count, iterate within the calibrated
    # bound over the whole chain of fine steps)
    from concurrent.futures import ThreadPoolExecutor

    insts = synth.batched_instances(0, 4096, P=64, fine_steps=256, coarse_steps=1)
    prob = B.Problem(insts, tuned=True)
    widths = [5, 32, 32, 1]
    lo, hi = [0.0, 0.0, 0.1, 0.0, 0.5], [8.0, 2.0, 0.5, 0.08, 2.0]
    w = synth.xavier_params(widths, 11)
    net = B.PinnModel(widths, lo, hi, seed=11)
    net.set_weights(w)
    om = orc.MLP(widths, w, lo, hi)
    picks = _one_per_grid_size(insts)
    assert len(picks) == 5

    def oracle_solve(i, kind, max_iter):
        op = orc.params(**insts[i])
        return orc.parareal(op, kind, g=orc.pinn_table(op, om), tol=1e-6, max_iter=max_iter)

    for k_gpu, k_or, max_iter in ((B.COARSE_PINN_IE, orc.COARSE_PINN_IE, 64), (B.COARSE_PINN, orc.COARSE_PINN, 3)):
        U, norms, stats, rc = prob.parareal_solve(k_gpu, model=net, prec=B.FP64, tol=1e-6, max_iter=max_iter)
        torch.cuda.synchronize()
        assert prob.device_status() == B.BS_OK
        if k_gpu == B.COARSE_PINN_IE:
            assert rc == B.BS_OK and all(st["status"] == B.BS_OK for st in stats)
        with ThreadPoolExecutor(len(picks)) as ex:
            refs = list(ex.map(lambda i: oracle_solve(i, k_or, max_iter), picks))
        for i, (Ur, nr, st) in zip(picks, refs):
            p = insts[i]
            assert stats[i]["iterations"] == len(nr), (i, p["Nx"], stats[i], len(nr))
            np.testing.assert_allclose(norms[i, :len(nr)], nr, rtol=1e-6)
            o = prob.state_off[i]
            got = U[o:o + (p["P"] + 1) * p["Nx"]].cpu().numpy()
            assert _rel(got, Ur.ravel()) <= _kappa_tol(p, p["P"] * p["fine_steps"]), (i, p["Nx"])


def test_large_instance_full_size(B, orc):
    cfg = dict(K=1.0, sigma=0.3, r=0.03, T=2.0, Smax=8.0, Nx=65536, P=256, fine_steps=4096, coarse_steps=1)
    prob = B.Problem(cfg)
    assert prob.partition(0) == dict(M=32, NW=4, C=16) and prob.slices_per_cta(0) == 2
    Uf = prob.serial_fine()
    U2, norms, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=0.0, max_iter=2)
    torch.cuda.synchronize()
    assert prob.device_status() == B.BS_OK and stats[0]["iterations"] == 2
    Nx = cfg["Nx"]
    assert torch.equal(U2[:3 * Nx], Uf[:3 * Nx])
    op = orc.params(**cfg)
    first = orc.fine(op, 0, orc.payoff(op))
    assert _rel(Uf[Nx:2 * Nx].cpu().numpy(), first) <= _kappa_tol(cfg, cfg["fine_steps"])


def _oracle_loss_grad_threaded(orc, om, X, kind, prob, sok, chunk=2048):
    """The oracle's loss terms and gradient of a whole batch, from chunks of
    points that feed one loss term each, run in host threads (the oracle is C
    called through ctypes, which releases the GIL).  Each term of Eq. 11 is a
    mean over its own points, so the batch's term t and its gradient are the
    chunks' ones weighted by (chunk points / points of term t)."""
    import os
    from concurrent.futures import ThreadPoolExecutor

    jobs = []
    for t, kinds in ((0, (0,)), (1, (1, 2)), (2, (3,))):
        idx = np.nonzero(np.isin(kind, kinds))[0]
        for c in range(0, len(idx), chunk):
            jobs.append((t, idx[c:c + chunk], len(idx[c:c + chunk]) / len(idx)))

    def run(job):
        t, ix, _ = job
        return orc.pinn_loss_grad(om, X[ix], kind[ix], prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)

    with ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        res = list(ex.map(run, jobs))
    terms, grad = np.zeros(3), np.zeros(om.params.size)
    for (t, _, wgt), (t3, g) in zip(jobs, res):
        terms[t] += wgt * t3[t]
        grad += wgt * g
    return terms, grad


def test_training_step_full_size_matches_oracle_and_fp32_path(B, orc):
    # the 2->6x128 training workload at its full batch (65536 points): every
    # layer's BF16 and TF32 tensor-core gradients against the oracle's FP64
    # gradient of the whole batch and against the FP32 CUDA-core gradient of
    # the same batch, with the per-layer bounds of the BF16 and TF32 tests
    widths = [2] + [128] * 6 + [1]
    nb = 65536 // 32
    X, kind = synth.collocation(0, 65536 - 2 * nb, nb, nb, 4.0, 1.0)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    m = B.PinnModel(widths, [0.0, 0.0], [4.0, 1.0], seed=0)
    l16, g16 = m.loss_grad(Xd, kd, prob, 0.0, prec=B.BF16)
    l32, g32 = m.loss_grad(Xd, kd, prob, 0.0, prec=B.FP32)
    lt, gt = m.loss_grad(Xd, kd, prob, 0.0, prec=B.TF32)
    assert m.device_status() == B.BS_OK
    l16, g16, l32, g32, lt, gt = (v.cpu().numpy() for v in (l16, g16, l32, g32, lt, gt))
    om = orc.MLP(widths, synth.xavier_params(widths, 0), [0.0, 0.0], [4.0, 1.0])
    l64, g64 = _oracle_loss_grad_threaded(orc, om, X, kind, prob, 0.0)
    for c in range(3):
        assert abs(l16[c] - l64[c]) <= 5e-2 * abs(l64[c]), (c, l16[c], l64[c])
        assert abs(l32[c] - l64[c]) <= 1e-4 * abs(l64[c]), (c, l32[c], l64[c])
        assert abs(lt[c] - l64[c]) <= 2e-2 * abs(l64[c]), (c, lt[c], l64[c])
    off = 0
    for l in range(1, len(widths)):
        for n in (widths[l] * widths[l - 1], widths[l]):
            a, b, ref, tf = g16[off:off + n], g32[off:off + n], g64[off:off + n], gt[off:off + n]
            assert _rel(a, ref) <= 2e-2, (l, n, _rel(a, ref))
            assert _rel(a, b) <= 2e-2, (l, n, _rel(a, b))
            assert _rel(tf, ref) <= 5e-3, (l, n, _rel(tf, ref))
            off += n
    assert _rel(g32, g64) <= 1e-4


def test_training_batch_above_the_default_chunk(B, monkeypatch):
    # 600k points: two chunks at the default 2^19, one pass when the chunk is
    # raised above the batch; the loss terms agree to FP64 summation order and
    # the gradient to the order of its FP32 partial sums
    widths = [2, 64, 64, 64, 1]
    n = 600_000
    nb = n // 32
    X, kind = synth.collocation(3, n - 2 * nb, nb, nb, 4.0, 1.0)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    m = B.PinnModel(widths, [0.0, 0.0], [4.0, 1.0], seed=5)
    monkeypatch.delenv("BSP_TRAIN_CHUNK", raising=False)
    l2, g2 = m.loss_grad(Xd, kd, prob, 0.0, prec=B.BF16)
    monkeypatch.setenv("BSP_TRAIN_CHUNK", str(1 << 20))
    l1, g1 = m.loss_grad(Xd, kd, prob, 0.0, prec=B.BF16)
    assert m.device_status() == B.BS_OK
    l1, g1, l2, g2 = (v.cpu().numpy() for v in (l1, g1, l2, g2))
    np.testing.assert_allclose(l2, l1, rtol=1e-12)
    assert _rel(g2, g1) <= 1e-5
