"""Failure detection without a GPU fault, and checkpoint / resume of training.

A bounded device wait on a barrier that nothing completes must give up after
its limit and report BS_TIMEOUT through the status word, leaving the context
usable; the same wait on a completed barrier reports BS_OK.  A network's
training state (weights, Adam moments, step) saved to a file and loaded into
another handle continues training as the original does."""
import time

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


def test_bounded_wait_expires_and_the_context_stays_usable(B):
    B.wait_probe(True, 1 << 20)  # first launch: module load out of the timing
    t0 = time.perf_counter()
    assert B.wait_probe(False, 4_000_000) == B.BS_TIMEOUT  # about 2 ms at 2 GHz
    assert time.perf_counter() - t0 < 5.0
    assert B.wait_probe(True, 4_000_000) == B.BS_OK
    # the device still runs ordinary work after the timed-out wait
    prob = B.Problem(B.params(Nx=64, P=2, fine_steps=8))
    U = torch.zeros(prob.total_slice, dtype=torch.float64, device="cuda")
    out = torch.empty_like(U)
    prob.fine_propagate(U, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    assert prob.device_status() == B.BS_OK


@pytest.mark.parametrize("prec_name", ["FP64", "BF16"])
def test_checkpoint_resume_continues_training(B, tmp_path, prec_name):
    prec = getattr(B, prec_name)
    widths, lo, hi = [2, 64, 64, 64, 1], [0.0, 0.0], [4.0, 1.0]
    X, kind = synth.collocation(5, 900, 64, 64, 4.0, 1.0)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    a = B.PinnModel(widths, lo, hi, seed=1)
    for _ in range(3):
        a.train_step(Xd, kd, prob, lr=1e-3, prec=prec)
    saved = a.get_state()
    a.save(tmp_path / "a.ckpt")
    for _ in range(2):
        a.train_step(Xd, kd, prob, lr=1e-3, prec=prec)
    wa = a.get_weights()
    b = B.PinnModel(widths, lo, hi, seed=2)  # other weights until the load
    b.load(tmp_path / "a.ckpt")
    restored = b.get_state()
    for x, y in zip(saved[:3], restored[:3]):
        assert np.array_equal(x, y)
    assert restored[3] == saved[3] == 3
    for _ in range(2):
        b.train_step(Xd, kd, prob, lr=1e-3, prec=prec)
    # the gradient's FP64 atomic sums may add in another order: agree to rounding
    assert np.abs(b.get_weights() - wa).max() <= 1e-12 * max(np.abs(wa).max(), 1.0)
    with pytest.raises(ValueError):
        B.PinnModel([2, 32, 1], lo, hi).load(tmp_path / "a.ckpt")


def test_every_output_element_is_written(B):
    # poisoned outputs: NaN before the call, every element finite after it, for
    # each entry point that writes a device array (a missed tile, row or
    # instance would stay NaN)
    insts = synth.batched_instances(3, 7, P=5, fine_steps=9, coarse_steps=1, Nx_choices=(33, 256, 300, 1025))
    prob = B.Problem(insts)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    Uin = torch.rand(prob.total_slice, dtype=torch.float64, device="cuda", generator=gen)
    nan = float("nan")
    for f in (prob.fine_propagate, prob.coarse_propagate):
        out = torch.full_like(Uin, nan)
        f(Uin, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
    Us = torch.full((prob.total_state,), nan, dtype=torch.float64, device="cuda")
    prob.serial_fine(Us)
    torch.cuda.synchronize()
    assert torch.isfinite(Us).all()
    net5 = B.PinnModel([5, 32, 32, 1], [0.0, 0.0, 0.1, 0.0, 0.5], [8.0, 2.0, 0.5, 0.08, 2.0], seed=3)
    for kind, model, prec in ((B.COARSE_IE, None, B.FP64), (B.COARSE_PINN, net5, B.BF16)):
        Uo = torch.full((prob.total_state,), nan, dtype=torch.float64, device="cuda")
        prob.parareal_solve(kind, model=model, prec=prec, tol=1e-8, U_out=Uo)
        assert torch.isfinite(Uo).all()
    net = B.PinnModel([2, 64, 64, 1], [0.0, 0.0], [4.0, 1.0], seed=3)
    for n in (1, 127, 129, 1000):
        X = torch.rand(n, 2, dtype=torch.float64, device="cuda", generator=gen) * torch.tensor([4.0, 1.0], device="cuda")
        for prec in (B.FP64, B.FP32, B.TF32, B.BF16):
            u = torch.full((n,), nan, dtype=torch.float64, device="cuda")
            net.eval(X, prec=prec, out=u)
            torch.cuda.synchronize()
            assert torch.isfinite(u).all(), (n, prec)
    X, kind = synth.collocation(2, 300, 32, 32, 4.0, 1.0)
    prob1 = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    for prec in (B.FP64, B.FP32, B.BF16):
        g = torch.full((net.n_params,), nan, dtype=torch.float64, device="cuda")
        net.train_step(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob1, lr=1e-3, prec=prec,
                       grad_out=g)
        torch.cuda.synchronize()
        assert torch.isfinite(g).all(), prec
    assert prob.device_status() == B.BS_OK and net.device_status() == B.BS_OK


def test_misaligned_device_pointers_are_rejected_before_any_launch(B):
    # device arrays must start on 16-byte boundaries (the kernels read them with
    # 16-byte and TMA accesses): an 8-byte offset gives BS_EINVAL and leaves the
    # output as it was
    L = B.lib()
    prob = B.Problem(B.params(Nx=64, P=2, fine_steps=4))
    U = torch.zeros(prob.total_slice + 2, dtype=torch.float64, device="cuda")
    out = torch.full((prob.total_slice + 2,), float("nan"), dtype=torch.float64, device="cuda")
    for f in (L.fine_propagate, L.coarse_propagate):
        assert f(prob._h, U.data_ptr() + 8, out.data_ptr(), None, None) == B.BS_EINVAL
        assert f(prob._h, U.data_ptr(), out.data_ptr() + 8, None, None) == B.BS_EINVAL
    assert L.serial_fine(prob._h, out.data_ptr() + 8, None) == B.BS_EINVAL
    assert L.parareal_solve(prob._h, B.COARSE_IE, None, B.FP64, 1e-8, 2, out.data_ptr() + 8, None, None,
                            None) == B.BS_EINVAL
    net = B.PinnModel([2, 32, 1], [0.0, 0.0], [4.0, 1.0], seed=0)
    X = torch.zeros(17, 2, dtype=torch.float64, device="cuda")
    u = torch.full((18,), float("nan"), dtype=torch.float64, device="cuda")
    assert L.pinn_eval(net._h, B.BF16, X.data_ptr() + 8, 8, u.data_ptr(), None, None) == B.BS_EINVAL
    assert L.pinn_eval(net._h, B.BF16, X.data_ptr(), 8, u.data_ptr() + 8, None, None) == B.BS_EINVAL
    torch.cuda.synchronize()
    assert torch.isnan(out).all() and torch.isnan(u).all()
