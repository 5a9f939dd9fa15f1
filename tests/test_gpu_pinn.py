"""GPU parity of the network path (evaluation, derivatives, loss, adjoint
gradient, Adam) against the oracle, through the C ABI.  BF16 and TF32
evaluation of the w x w hidden layers runs on the tensor cores (tcgen05).

Tolerances (relative to the largest magnitude of the compared quantity):
  FP64: 1e-12 for u, 1e-10 for derivatives and gradients (the GPU sums in a
        different order; second derivatives and long dot products lose a few
        more digits);
  FP32: 2e-5 for u and derivatives, 1e-4 for loss terms and gradients
        (unit roundoff 6e-8 amplified by 4-8 layers of width <= 256);
  TF32: 1e-2 and BF16: 4e-2 for u (operands rounded to 10 / 7 mantissa bits,
        FP32 accumulation); BF16 gradients 1e-1 (operands of both passes rounded);
        TF32 gradients 5e-3 and loss terms 2e-2 (the residual term cancels
        u_tau against the S-derivative terms).
"""
import numpy as np
import pytest

from paper_2303_03848_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_EVAL = {0: 1e-12, 1: 2e-5, 2: 1e-2, 3: 4e-2}
# (loss terms, whole gradient) relative to the largest magnitude
TOL_TRAIN = {0: (1e-12, 1e-10), 1: (1e-4, 1e-4), 2: (2e-2, 5e-3), 3: (5e-2, 1e-1)}


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03848_b300 import binding, build

    build.build()
    return binding


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


ARCHS = {
    "2-4x64": [2, 64, 64, 64, 64, 1],
    "2-6x128": [2] + [128] * 6 + [1],
    "5-6x128": [5] + [128] * 6 + [1],
    "2-8x256": [2] + [256] * 8 + [1],
}
LO5 = [0.0, 0.0, 0.1, 0.0, 0.5]
HI5 = [8.0, 2.0, 0.5, 0.08, 2.0]


def _box(widths):
    d = widths[0]
    return ([0.0, 0.0], [4.0, 1.0]) if d == 2 else (LO5, HI5)


def _points(widths, n, seed):
    lo, hi = _box(widths)
    u = synth.uniform(seed, n * widths[0]).reshape(n, widths[0])
    return np.asarray(lo) + (np.asarray(hi) - np.asarray(lo)) * u


def _model(B, orc, widths, seed):
    lo, hi = _box(widths)
    m = B.PinnModel(widths, lo, hi, seed=seed)
    w = synth.xavier_params(widths, seed)
    w[np.arange(w.size) % 7 == 1] += 0.05
    m.set_weights(w)
    return m, orc.MLP(widths, w, lo, hi)


def test_pinn_create_initialisation_matches_generator(B):
    widths = ARCHS["2-4x64"]
    m = B.PinnModel(widths, [0.0, 0.0], [4.0, 1.0], seed=1234)
    np.testing.assert_array_equal(m.get_weights(), synth.xavier_params(widths, 1234))


@pytest.mark.parametrize("arch", list(ARCHS))
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_eval_matches_oracle(B, orc, arch, prec):
    widths = ARCHS[arch]
    if prec == 0 and arch == "2-8x256":
        n = 300
    else:
        n = 1000 + 37  # several CTAs and a ragged tail
    m, om = _model(B, orc, widths, 5)
    X = _points(widths, n, 9)
    ref = orc.mlp_eval(om, X, with_derivs=False)
    u = m.eval(torch.tensor(X, device="cuda"), prec=prec).cpu().numpy()
    assert m.device_status() == B.BS_OK
    assert _rel(u, ref) <= TOL_EVAL[prec]


@pytest.mark.parametrize("arch", ["2-4x64", "2-6x128", "5-6x128"])
@pytest.mark.parametrize("prec", [0, 1])
def test_eval_derivatives_match_oracle(B, orc, arch, prec):
    widths = ARCHS[arch]
    m, om = _model(B, orc, widths, 6)
    X = _points(widths, 517, 10)
    ru, rd = orc.mlp_eval(om, X)
    u, d = m.eval(torch.tensor(X, device="cuda"), prec=prec, derivs=True)
    u, d = u.cpu().numpy(), d.cpu().numpy()
    tol_u = TOL_EVAL[prec]
    tol_d = 1e-10 if prec == 0 else 2e-5
    assert _rel(u, ru) <= tol_u
    for c in range(3):
        assert _rel(d[:, c], rd[:, c]) <= tol_d, c


def test_eval_empty_batch_is_noop(B, orc):
    m, _ = _model(B, orc, ARCHS["2-4x64"], 1)
    X = torch.empty(0, 2, dtype=torch.float64, device="cuda")
    assert m.eval(X).numel() == 0


def _loss_case(widths, n_int, n_b, n_e, seed):
    if widths[0] == 2:
        X, kind = synth.collocation(seed, n_int, n_b, n_e, 4.0, 1.0)
        prob = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
        return X, kind, prob, 0.0
    X, kind = synth.collocation_parametric(seed, n_int, n_b, n_e, 4.0, 2.0)
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=2.0, Smax=8.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    return X, kind, prob, 4.0


@pytest.mark.parametrize("arch", ["2-4x64", "2-6x128", "5-6x128"])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_loss_and_gradient_match_oracle(B, orc, arch, prec):
    widths = ARCHS[arch]
    m, om = _model(B, orc, widths, 8)
    X, kind, prob, sok = _loss_case(widths, 1500, 128, 128, 4)
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=prec)
    l3, g = l3.cpu().numpy(), g.cpu().numpy()
    tol_l, tol_g = TOL_TRAIN[prec]
    for c in range(3):
        assert abs(l3[c] - terms[c]) <= tol_l * max(abs(terms[c]), 1e-300), (c, l3[c], terms[c])
    assert _rel(g, grad) <= tol_g


def _data_case(widths, seed, share=0.4):
    # PINN collocation points with a share turned into kind-4 data points, values y
    X, kind, prob, sok = _loss_case(widths, 1500, 128, 128, seed)
    rng = np.random.default_rng(seed)
    kind = kind.copy()
    kind[rng.random(kind.size) < share] = 4
    return X, kind, rng.normal(size=kind.size), prob, sok


@pytest.mark.parametrize("arch", ["2-4x64", "2-6x128"])
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_data_points_loss_and_gradient_match_oracle(B, orc, arch, prec):
    # kind-4 data points (squared misfit to a given value, in the mean of term 0)
    # among the PINN points, through pinn_loss_grad_data; the per-precision bounds
    # of the PINN loss (BF16 runs on the tensor cores for both networks)
    widths = ARCHS[arch]
    m, om = _model(B, orc, widths, 8)
    X, kind, y, prob, sok = _data_case(widths, 31)
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok, y=y)
    l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=prec,
                        y=torch.tensor(y, device="cuda"))
    assert m.device_status() == B.BS_OK
    l3, g = l3.cpu().numpy(), g.cpu().numpy()
    tol_l, tol_g = TOL_TRAIN[prec]
    for c in range(3):
        assert abs(l3[c] - terms[c]) <= tol_l * max(abs(terms[c]), 1e-300), (c, l3[c], terms[c])
    assert _rel(g, grad) <= tol_g


def test_data_only_tensor_core_gradient_every_layer_and_chunks(B, orc, monkeypatch):
    # a batch of data points only (no PDE terms) on the tensor cores: every
    # parameter block against the oracle (the per-block bound of the PINN
    # tests), and chunks of 1024 points equal to one pass (the values follow
    # their points into every chunk)
    widths = ARCHS["2-6x128"]
    m, om = _model(B, orc, widths, 45)
    X, kind, y, prob, sok = _data_case(widths, 47, share=1.0)
    Xd, kd, yd = (torch.tensor(v, device="cuda") for v in (X, kind, y))
    monkeypatch.delenv("BSP_TRAIN_CHUNK", raising=False)
    l_one, g_one = m.loss_grad(Xd, kd, prob, sok, prec=B.BF16, y=yd)
    monkeypatch.setenv("BSP_TRAIN_CHUNK", "1024")
    l_ch, g_ch = m.loss_grad(Xd, kd, prob, sok, prec=B.BF16, y=yd)
    assert m.device_status() == B.BS_OK
    l_one, g_one, l_ch, g_ch = (v.cpu().numpy() for v in (l_one, g_one, l_ch, g_ch))
    np.testing.assert_allclose(l_ch, l_one, rtol=1e-12)
    assert _rel(g_ch, g_one) <= 1e-5
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok, y=y)
    assert terms[1] == 0.0 and terms[2] == 0.0 and l_one[1] == 0.0 and l_one[2] == 0.0
    assert abs(l_one[0] - terms[0]) <= 5e-2 * terms[0]
    for name, a, b in _param_blocks(widths):
        err = np.abs(g_one[a:b] - grad[a:b]).max() / max(np.abs(grad[a:b]).max(), 1e-300)
        assert err <= 2e-2, (name, err)


def test_train_step_is_adam_on_the_gradient(B, orc):
    widths = ARCHS["2-4x64"]
    m, om = _model(B, orc, widths, 12)
    X, kind, prob, sok = _loss_case(widths, 700, 64, 64, 6)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    th = om.params.copy()
    m1, m2 = np.zeros_like(th), np.zeros_like(th)
    for t in (1, 2):
        terms, grad = orc.pinn_loss_grad(orc.MLP(widths, th, om.lo, om.hi), X, kind, 1.0, 0.2, 0.05, 4.0)
        loss = m.train_step(Xd, kd, prob, lr=1e-3, prec=B.FP64, want_loss=True)
        np.testing.assert_allclose(loss, terms, rtol=1e-12)
        orc.adam(th, m1, m2, grad, t, 1e-3)
        # Adam divides by sqrt(v): a gradient entry that is ~0 makes that
        # parameter's step sensitive to its rounding, so compare absolutely
        assert np.abs(m.get_weights() - th).max() <= 1e-12


def test_training_reduces_loss_fp32(B, orc):
    widths = ARCHS["2-4x64"]
    m = B.PinnModel(widths, [0.0, 0.0], [4.0, 1.0], seed=0)
    X, kind = synth.collocation(0, 2048, 128, 128, 4.0, 1.0)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    first = sum(m.train_step(Xd, kd, prob, lr=1e-3, prec=B.FP32, want_loss=True))
    for _ in range(200):
        m.train_step(Xd, kd, prob, lr=1e-3, prec=B.FP32)
    last = sum(m.train_step(Xd, kd, prob, lr=1e-3, prec=B.FP32, want_loss=True))
    assert last < 0.2 * first


@pytest.mark.parametrize("w,n_hidden,d_in", [(32, 1, 2), (32, 3, 2), (64, 4, 2), (128, 6, 5), (256, 3, 2), (256, 2, 5)])
@pytest.mark.parametrize("prec", [2, 3])
def test_tensor_core_eval_shapes_and_ragged_tiles(B, orc, w, n_hidden, d_in, prec):
    # tiles of 128 points: 1, 127, 128, 129 and a few thousand points
    widths = [d_in] + [w] * n_hidden + [1]
    m, om = _model(B, orc, widths, 21)
    for n in (1, 127, 128, 129, 2500):
        X = _points(widths, n, 30 + n)
        ref = orc.mlp_eval(om, X, with_derivs=False)
        u = m.eval(torch.tensor(X, device="cuda"), prec=prec).cpu().numpy()
        assert m.device_status() == B.BS_OK
        assert _rel(u, ref) <= TOL_EVAL[prec], (n, _rel(u, ref))


@pytest.mark.parametrize("arch", ["2-4x64", "2-6x128", "5-6x128"])
def test_tf32_tensor_core_eval_is_tf32_accurate(B, orc, arch):
    # the TF32 path keeps 10 explicit mantissa bits of both operands (BF16: 7),
    # so on the same network its error against the oracle is several times
    # smaller than BF16's (measured about 8-10x): a path that rounded to BF16 or
    # lost a layer would not pass
    widths = ARCHS[arch]
    m, om = _model(B, orc, widths, 5)
    X = _points(widths, 20000, 9)
    ref = orc.mlp_eval(om, X, with_derivs=False)
    Xd = torch.tensor(X, device="cuda")
    e_tf = _rel(m.eval(Xd, prec=B.TF32).cpu().numpy(), ref)
    e_bf = _rel(m.eval(Xd, prec=B.BF16).cpu().numpy(), ref)
    assert m.device_status() == B.BS_OK
    assert e_tf <= TOL_EVAL[2] and e_tf < 0.3 * e_bf, (e_tf, e_bf)


def _param_blocks(widths):
    out, off = [], 0
    for l in range(1, len(widths)):
        nw = widths[l] * widths[l - 1]
        out.append((f"W{l}", off, off + nw))
        off += nw
        out.append((f"b{l}", off, off + widths[l]))
        off += widths[l]
    return out


@pytest.mark.parametrize(
    "widths",
    [[2, 32, 32, 1], [2, 64, 64, 64, 64, 1], [5, 96, 96, 96, 1], [2] + [128] * 6 + [1], [5] + [128] * 6 + [1]],
    ids=["2-2x32", "2-4x64", "5-3x96", "2-6x128", "5-6x128"],
)
def test_tensor_core_gradient_every_layer(B, orc, widths):
    # each weight matrix and bias vector of the BF16 tensor-core gradient on its
    # own against the FP64 oracle, so that a lost stream, layer or bias term
    # cannot hide under the whole-vector bound.  Bound: BF16 operands round to
    # 8 significant bits (unit roundoff 2^-8 ~ 3.9e-3); every gradient entry is a
    # sum of products of two rounded operands whose inputs passed through up to
    # six rounded layers; 2e-2 ~ 5 roundoffs (measured worst case 7e-3).
    m, om = _model(B, orc, widths, 8)
    for n_int in (1500, 6000):
        X, kind, prob, sok = _loss_case(widths, n_int, 128, 128, 4 + n_int)
        terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
        l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=B.BF16)
        g = g.cpu().numpy()
        assert m.device_status() == B.BS_OK
        for name, a, b in _param_blocks(widths):
            err = np.abs(g[a:b] - grad[a:b]).max() / max(np.abs(grad[a:b]).max(), 1e-300)
            assert err <= 2e-2, (n_int, name, err)
        # the residual term cancels (u_tau against the S-derivative terms): the
        # per-term bound of the other BF16 loss tests
        for c in range(3):
            assert abs(l3[c].item() - terms[c]) <= 5e-2 * abs(terms[c]), (c, l3[c].item(), terms[c])


def _saturated_fraction(widths, w, X, lo, hi):
    # share of hidden neurons (over all points and hidden layers) with |tanh z| > 0.95, t' < 0.1
    h = 2.0 * (X - np.asarray(lo)) / (np.asarray(hi) - np.asarray(lo)) - 1.0
    off, sat, tot = 0, 0, 0
    for l in range(1, len(widths) - 1):
        W = w[off:off + widths[l] * widths[l - 1]].reshape(widths[l], widths[l - 1])
        off += widths[l] * widths[l - 1]
        b = w[off:off + widths[l]]
        off += widths[l]
        h = np.tanh(h @ W.T + b)
        sat += int((np.abs(h) > 0.95).sum())
        tot += h.size
    return sat / tot


@pytest.mark.parametrize("widths", [[2, 64, 64, 64, 1], [2] + [128] * 4 + [1]], ids=["2-3x64", "2-4x128"])
def test_tensor_core_gradient_saturated_network(B, orc, widths):
    # the Xavier weights times 3 push 12-17 % of the hidden neurons into
    # saturation (t' < 0.1), where t' = 1 - t^2 loses relative accuracy if t
    # itself is rounded; the adjoint recomputes t from the stored pre-activation.
    # Bound: the BF16 operands' error grows with the weights' scale (measured
    # 2.4e-2 worst block at scale 3, the same with FP32 activations); 5e-2.
    lo, hi = _box(widths)
    w = 3.0 * synth.xavier_params(widths, 3)
    m = B.PinnModel(widths, lo, hi, seed=3)
    m.set_weights(w)
    om = orc.MLP(widths, w, lo, hi)
    X, kind, prob, sok = _loss_case(widths, 3000, 128, 128, 21)
    assert _saturated_fraction(widths, w, X, lo, hi) >= 0.1
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=B.BF16)
    g = g.cpu().numpy()
    assert m.device_status() == B.BS_OK
    for name, a, b in _param_blocks(widths):
        err = np.abs(g[a:b] - grad[a:b]).max() / max(np.abs(grad[a:b]).max(), 1e-300)
        assert err <= 5e-2, (name, err)


@pytest.mark.parametrize("widths", [[2, 48, 48, 1], [2, 256, 256, 1], [5, 40, 24, 1]], ids=["2-2x48", "2-2x256", "5-40-24"])
def test_bf16_training_outside_the_tensor_core_shapes(B, orc, widths):
    # BF16 loss and gradient for networks the tensor-core training does not take
    # (width not in 32..128 by 32, or unequal widths): CUDA cores with BF16-rounded
    # operands, the BF16 bounds of the other tests
    m, om = _model(B, orc, widths, 9)
    X, kind, prob, sok = _loss_case(widths, 700, 64, 64, 13)
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=B.BF16)
    l3, g = l3.cpu().numpy(), g.cpu().numpy()
    for c in range(3):
        assert abs(l3[c] - terms[c]) <= 5e-2 * abs(terms[c]), (c, l3[c], terms[c])
    assert _rel(g, grad) <= 1e-1
    for name, a, b in _param_blocks(widths):
        assert np.abs(g[a:b] - grad[a:b]).max() / max(np.abs(grad[a:b]).max(), 1e-300) <= 2e-2, name


@pytest.mark.parametrize("widths", [[2, 7, 1], [2, 50, 50, 1], [5, 40, 24, 1], [2, 200, 130, 1]],
                         ids=["2-7", "2-2x50", "5-40-24", "2-200-130"])
@pytest.mark.parametrize("prec", [0, 1])
def test_cuda_core_paths_on_uneven_widths(B, orc, widths, prec):
    # the CUDA-core evaluation and training tile the layers in blocks of 16 RN
    # neurons: widths that fill no block exactly, unequal widths and a batch
    # that is no multiple of the 16-point tile, against the oracle
    m, om = _model(B, orc, widths, 12)
    X, kind, prob, sok = _loss_case(widths, 701, 61, 67, 17)
    Xd = torch.tensor(X, device="cuda")
    ru, rd = orc.mlp_eval(om, X)
    u, d = m.eval(Xd, prec=prec, derivs=True)
    assert _rel(u.cpu().numpy(), ru) <= TOL_EVAL[prec]
    for c in range(3):
        assert _rel(d.cpu().numpy()[:, c], rd[:, c]) <= (1e-10 if prec == 0 else 2e-5), c
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    l3, g = m.loss_grad(Xd, torch.tensor(kind, device="cuda"), prob, sok, prec=prec)
    l3, g = l3.cpu().numpy(), g.cpu().numpy()
    tol_l, tol_g = (1e-12, 1e-10) if prec == 0 else (1e-4, 1e-4)
    for c in range(3):
        assert abs(l3[c] - terms[c]) <= tol_l * abs(terms[c]), (c, l3[c], terms[c])
    assert _rel(g, grad) <= tol_g
    assert m.device_status() == B.BS_OK


@pytest.mark.parametrize("arch", ["2-4x64", "5-6x128"])
def test_tensor_core_training_in_chunks(B, orc, arch, monkeypatch):
    # a batch run as chunks of 1024 points (4 chunks, the last one ragged) gives
    # the one-pass result up to the order of the FP32 partial sums, and the oracle's
    widths = ARCHS[arch]
    m, om = _model(B, orc, widths, 41)
    X, kind, prob, sok = _loss_case(widths, 3000, 128, 128, 43)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    monkeypatch.delenv("BSP_TRAIN_CHUNK", raising=False)
    l_one, g_one = m.loss_grad(Xd, kd, prob, sok, prec=B.BF16)
    monkeypatch.setenv("BSP_TRAIN_CHUNK", "1024")
    l_ch, g_ch = m.loss_grad(Xd, kd, prob, sok, prec=B.BF16)
    assert m.device_status() == B.BS_OK
    l_one, g_one, l_ch, g_ch = (v.cpu().numpy() for v in (l_one, g_one, l_ch, g_ch))
    np.testing.assert_allclose(l_ch, l_one, rtol=1e-12)
    assert _rel(g_ch, g_one) <= 1e-5
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    for name, a, b in _param_blocks(widths):
        err = np.abs(g_ch[a:b] - grad[a:b]).max() / max(np.abs(grad[a:b]).max(), 1e-300)
        assert err <= 2e-2, (name, err)


@pytest.mark.parametrize("arch", ["2-4x64", "2-6x128", "5-6x128"])
def test_tensor_core_training_ragged_batches(B, orc, arch):
    # BF16 loss and gradient through the tensor-core forward, adjoint and weight
    # gradient: batches that leave a partial 32-point tile, a partial 64-point
    # chunk and an N that is not a multiple of 4 (element-wise loads)
    widths = ARCHS[arch]
    m, om = _model(B, orc, widths, 31)
    for n_int, n_b, n_e in ((1, 0, 0), (25, 3, 3), (27, 3, 3), (1501, 128, 128)):
        X, kind, prob, sok = _loss_case(widths, n_int, n_b, n_e, 17 + n_int)
        terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
        l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=B.BF16)
        l3, g = l3.cpu().numpy(), g.cpu().numpy()
        assert m.device_status() == B.BS_OK
        for c in range(3):
            assert abs(l3[c] - terms[c]) <= 5e-2 * max(abs(terms[c]), 1e-300), (len(kind), c, l3[c], terms[c])
        assert _rel(g, grad) <= 1e-1, (len(kind), _rel(g, grad))


TF32_SHAPES = {
    "2-2x32": [2, 32, 32, 1],
    "2-4x64": [2, 64, 64, 64, 64, 1],
    "5-3x96": [5, 96, 96, 96, 1],
    "2-6x128": [2] + [128] * 6 + [1],
    "5-6x128": [5] + [128] * 6 + [1],
}


def _block_errors(g, grad, widths):
    return {name: np.abs(g[a:b] - grad[a:b]).max() / max(np.abs(grad[a:b]).max(), 1e-300)
            for name, a, b in _param_blocks(widths)}


@pytest.mark.parametrize("shape", list(TF32_SHAPES))
def test_tf32_tensor_core_gradient_every_layer(B, orc, shape):
    # each weight matrix and bias vector of the TF32 tensor-core gradient
    # (tcgen05 kind::tf32 in the forward, the adjoint and the weight-gradient
    # GEMM over rows) on its own against the FP64 oracle.  Bound: TF32 operands
    # keep 11 significant bits (unit roundoff 2^-11 ~ 4.9e-4) and the forward's
    # tanh has a relative error of the same size; 5e-3 ~ 10 roundoffs (measured
    # worst 7.6e-4).  The same blocks in BF16 must be more than 3x farther off,
    # so a path that rounds to BF16 cannot pass.
    widths = TF32_SHAPES[shape]
    m, om = _model(B, orc, widths, 8)
    for n_int in (1500, 6000):
        X, kind, prob, sok = _loss_case(widths, n_int, 128, 128, 4 + n_int)
        terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
        Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
        l3, g = m.loss_grad(Xd, kd, prob, sok, prec=B.TF32)
        _, gb = m.loss_grad(Xd, kd, prob, sok, prec=B.BF16)
        assert m.device_status() == B.BS_OK
        e_tf = _block_errors(g.cpu().numpy(), grad, widths)
        e_bf = _block_errors(gb.cpu().numpy(), grad, widths)
        for name, err in e_tf.items():
            assert err <= 5e-3, (n_int, name, err)
        assert max(e_tf.values()) < 0.3 * max(e_bf.values()), (max(e_tf.values()), max(e_bf.values()))
        for c in range(3):
            assert abs(l3[c].item() - terms[c]) <= 2e-2 * abs(terms[c]), (c, l3[c].item(), terms[c])


@pytest.mark.parametrize("arch", ["2-4x64", "5-6x128"])
def test_tf32_training_ragged_batches(B, orc, arch):
    # batches of 1, 31, 33 and 1757 points: the padded rows of a partial
    # 32-point tile, of the last 32-row block of the weight gradient and of a
    # CTA's last row range must contribute nothing; the workspace grows between
    # the calls
    widths = ARCHS[arch]
    m, om = _model(B, orc, widths, 31)
    for n_int, n_b, n_e in ((1, 0, 0), (25, 3, 3), (27, 3, 3), (1501, 128, 128)):
        X, kind, prob, sok = _loss_case(widths, n_int, n_b, n_e, 17 + n_int)
        terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
        l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=B.TF32)
        l3, g = l3.cpu().numpy(), g.cpu().numpy()
        assert m.device_status() == B.BS_OK
        for c in range(3):
            assert abs(l3[c] - terms[c]) <= 2e-2 * max(abs(terms[c]), 1e-300), (len(kind), c, l3[c], terms[c])
        for name, err in _block_errors(g, grad, widths).items():
            assert err <= 5e-3, (len(kind), name, err)


@pytest.mark.parametrize("widths", [[2, 64, 64, 64, 1], [2] + [128] * 4 + [1]], ids=["2-3x64", "2-4x128"])
def test_tf32_tensor_core_gradient_saturated_network(B, orc, widths):
    # the saturated network of the BF16 test (12-17 % of the hidden neurons
    # with t' < 0.1): TF32 keeps its per-block bound there (the adjoint reads
    # the stored FP32 t, z_1, z_2, z_3; t' = 1 - t^2 from the FP32 t)
    lo, hi = _box(widths)
    w = 3.0 * synth.xavier_params(widths, 3)
    m = B.PinnModel(widths, lo, hi, seed=3)
    m.set_weights(w)
    om = orc.MLP(widths, w, lo, hi)
    X, kind, prob, sok = _loss_case(widths, 3000, 128, 128, 21)
    assert _saturated_fraction(widths, w, X, lo, hi) >= 0.1
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=B.TF32)
    assert m.device_status() == B.BS_OK
    for name, err in _block_errors(g.cpu().numpy(), grad, widths).items():
        assert err <= 1e-2, (name, err)


@pytest.mark.parametrize("widths", [[2, 48, 48, 1], [2, 256, 256, 1], [5, 40, 24, 1], [2, 64, 1]],
                         ids=["2-2x48", "2-2x256", "5-40-24", "2-1x64"])
def test_tf32_training_outside_the_tensor_core_shapes(B, orc, widths):
    # TF32 loss and gradient for networks the tensor-core training does not take
    # (width not in 32..128 by 32, unequal widths, a single hidden layer): CUDA
    # cores with TF32-rounded operands, the TF32 bounds
    m, om = _model(B, orc, widths, 9)
    X, kind, prob, sok = _loss_case(widths, 700, 64, 64, 13)
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    l3, g = m.loss_grad(torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda"), prob, sok, prec=B.TF32)
    l3, g = l3.cpu().numpy(), g.cpu().numpy()
    assert m.device_status() == B.BS_OK
    for c in range(3):
        assert abs(l3[c] - terms[c]) <= 2e-2 * abs(terms[c]), (c, l3[c], terms[c])
    for name, err in _block_errors(g, grad, widths).items():
        assert err <= 5e-3, (name, err)


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_autograd_function_gradient_matches_oracle_and_differences(B, orc, prec):
    # binding.pinn_loss: the total loss of Eq. 11 as a torch autograd function
    # of the flat parameter vector; .backward() gives the device adjoint
    widths = ARCHS["2-4x64"]
    m, om = _model(B, orc, widths, 41)
    X, kind, prob, sok = _loss_case(widths, 700, 64, 64, 9)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    theta = torch.tensor(om.params, device="cuda", requires_grad=True)
    loss = B.pinn_loss(theta, m, Xd, kd, prob, sok, prec=prec)
    loss.backward()
    terms, grad = orc.pinn_loss_grad(om, X, kind, prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    g = theta.grad.cpu().numpy()
    if prec == 0:
        assert abs(loss.item() - sum(terms)) <= 1e-12 * sum(terms)
        assert _rel(g, grad) <= 1e-10
        # central differences of the device forward in a few coordinates
        rng = np.random.default_rng(3)
        for q in rng.choice(om.params.size, 6, replace=False):
            h = 1e-6 * max(1.0, abs(om.params[q]))
            tp, tm = theta.detach().clone(), theta.detach().clone()
            tp[q] += h
            tm[q] -= h
            fd = (B.pinn_loss(tp, m, Xd, kd, prob, sok, prec=0).item() -
                  B.pinn_loss(tm, m, Xd, kd, prob, sok, prec=0).item()) / (2 * h)
            assert abs(fd - g[q]) <= 1e-6 * max(np.abs(g).max(), 1e-300), (q, fd, g[q])
    else:
        assert _rel(g, grad) <= TOL_TRAIN[prec][1]


def test_autograd_function_drives_a_torch_optimizer(B):
    widths = ARCHS["2-4x64"]
    m = B.PinnModel(widths, [0.0, 0.0], [4.0, 1.0], seed=5)
    X, kind = synth.collocation(2, 1024, 64, 64, 4.0, 1.0)
    Xd, kd = torch.tensor(X, device="cuda"), torch.tensor(kind, device="cuda")
    prob = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=5, P=1, fine_steps=1, coarse_steps=1)
    theta = torch.tensor(synth.xavier_params(widths, 5), device="cuda", requires_grad=True)
    opt = torch.optim.Adam([theta], lr=1e-3)
    first = None
    for _ in range(30):
        opt.zero_grad()
        loss = B.pinn_loss(theta, m, Xd, kd, prob, prec=B.FP32)
        loss.backward()
        opt.step()
        first = loss.item() if first is None else first
    assert loss.item() < first


def _c_loss_grad(B, m, X, kind, prob, sok, prec):
    # straight through the C ABI (the binding would refuse these kinds on the host)
    import ctypes

    loss3 = torch.empty(3, dtype=torch.float64, device="cuda")
    grad = torch.empty(m.n_params, dtype=torch.float64, device="cuda")
    pp = B._to_struct(prob)
    rc = B.lib().pinn_loss_grad(m._h, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(kind.data_ptr()), X.shape[0],
                                ctypes.byref(pp), sok, prec, ctypes.c_void_p(loss3.data_ptr()),
                                ctypes.c_void_p(grad.data_ptr()), B._stream())
    return rc, loss3.cpu().numpy(), grad.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_invalid_kinds_are_left_out_and_reported(B, orc, prec):
    # kinds outside 0..3, and data points in a call without values, are counted
    # nowhere and contribute nothing; the network's status word says BS_EINVAL
    widths = ARCHS["2-4x64"]
    X, kind, prob, sok = _loss_case(widths, 700, 64, 64, 3)
    kb = kind.copy()
    kb[np.arange(kind.size) % 11 == 5] = 7
    kb[np.arange(kind.size) % 13 == 6] = 4
    kb[np.arange(kind.size) % 17 == 8] = -3
    keep = (kb >= 0) & (kb <= 3)
    m_bad, _ = _model(B, orc, widths, 8)
    rc, l_bad, g_bad = _c_loss_grad(B, m_bad, torch.tensor(X, device="cuda"), torch.tensor(kb, device="cuda"), prob,
                                    sok, prec)
    assert rc == B.BS_OK and m_bad.device_status() == B.BS_EINVAL
    m_ok, om = _model(B, orc, widths, 8)
    terms, grad = orc.pinn_loss_grad(om, X[keep], kind[keep], prob["K"], prob["sigma"], prob["r"], prob["Smax"], sok)
    tol_l, tol_g = TOL_TRAIN[prec]
    for c in range(3):
        assert abs(l_bad[c] - terms[c]) <= tol_l * abs(terms[c]), (c, l_bad[c], terms[c])
    assert _rel(g_bad, grad) <= tol_g
    assert m_ok.device_status() == B.BS_OK


def test_data_only_network_as_coarse_propagator(B):
    # Section 4's data-only network: trained on the serial fine solution at the
    # grid points (kind-4 data points, no PDE terms), then used as the coarse
    # propagator.  The data loss falls, the trained table is closer to serial
    # fine than the untrained one, and network-anchored Parareal reaches its
    # tolerance in fewer than P iterations with the iterate within it of serial
    # fine.  The autograd wrapper takes the data values too.
    cfg = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=64, P=8, fine_steps=64, coarse_steps=1)
    prob = B.Problem(cfg)
    Uf = prob.serial_fine()
    S = torch.linspace(0.0, cfg["Smax"], cfg["Nx"], dtype=torch.float64, device="cuda")
    tau = torch.linspace(0.0, cfg["T"], cfg["P"] + 1, dtype=torch.float64, device="cuda")
    Xg = torch.stack([S.repeat(cfg["P"] + 1), tau.repeat_interleave(cfg["Nx"])], dim=1).contiguous()
    kd = torch.full((Xg.shape[0],), 4, dtype=torch.int8, device="cuda")
    widths = [2, 32, 32, 1]
    dnet = B.PinnModel(widths, [0.0, 0.0], [cfg["Smax"], cfg["T"]], seed=0)
    fresh = B.PinnModel(widths, [0.0, 0.0], [cfg["Smax"], cfg["T"]], seed=0)

    def table_err(m):
        g = m.eval(Xg, prec=B.FP64).view(cfg["P"] + 1, cfg["Nx"])[1:]
        f = Uf.view(cfg["P"] + 1, cfg["Nx"])[1:]
        return float(((g - f).norm(dim=1) / f.norm(dim=1)).max())

    first = dnet.train_step(Xg, kd, cfg, lr=3e-3, prec=B.BF16, want_loss=True, y=Uf)
    for _ in range(600):
        dnet.train_step(Xg, kd, cfg, lr=3e-3, prec=B.BF16, y=Uf)
    last = dnet.train_step(Xg, kd, cfg, lr=3e-3, prec=B.BF16, want_loss=True, y=Uf)
    assert first[1] == 0.0 and first[2] == 0.0 and last[0] < 0.05 * first[0], (first, last)
    assert table_err(dnet) < 0.5 * table_err(fresh)
    U, norms, stats, rc = prob.parareal_solve(B.COARSE_PINN_IE, model=dnet, prec=B.BF16, tol=1e-6)
    assert rc == B.BS_OK and stats[0]["iterations"] < cfg["P"], stats
    f = Uf.view(cfg["P"] + 1, cfg["Nx"])[1:]
    err = float(((U.view(cfg["P"] + 1, cfg["Nx"])[1:] - f).norm(dim=1) / f.norm(dim=1)).max())
    assert err < 1e-5
    theta = torch.tensor(dnet.get_weights(), dtype=torch.float64, requires_grad=True)
    loss = B.pinn_loss(theta, dnet, Xg, kd, cfg, prec=B.FP64, y=Uf)
    loss.backward()
    l3, g = dnet.loss_grad(Xg, kd, cfg, prec=B.FP64, y=Uf)
    assert abs(float(loss.detach()) - float(l3.sum())) <= 1e-12 * abs(float(l3.sum()))
    np.testing.assert_allclose(theta.grad.numpy(), g.cpu().numpy(), rtol=0, atol=1e-12 * float(g.abs().max()))
