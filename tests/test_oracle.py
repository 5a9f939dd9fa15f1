"""Pins of the oracle against things other than itself (CPU only).

Each test checks the FP64 oracle against a fact the paper or mathematics fixes:
published prices, closed forms, convergence orders, dense linear algebra from
numpy, automatic differentiation and Adam from PyTorch, finite differences and
the Parareal invariants of Section 3.1.
"""
import os

import numpy as np
import pytest
import torch

from paper_2303_03848_b300 import synth

from _longdouble import cn_longdouble as _cn_longdouble

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _norm_cdf(x):
    from scipy.stats import norm

    return norm.cdf(x)


# ---------------------------------------------------------------- closed form

def test_bs_call_published_prices(orc):
    rows = []
    with open(os.path.join(GOLDEN, "bs_call_prices.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            S, K, r, s, tau, price, tol, _ = line.split()
            rows.append(tuple(map(float, (S, K, r, s, tau, price, tol))))
    assert len(rows) == 3
    for S, K, r, s, tau, price, tol in rows:
        assert abs(orc.bs_call(S, K, r, s, tau) - price) <= tol


def test_bs_call_matches_scipy_and_parity(orc):
    # scipy's normal CDF is an independent library routine; put-call parity and
    # the limits are identities of the closed form
    for S, K, r, s, tau in [(0.7, 1.0, 0.03, 0.3, 2.0), (3.0, 1.0, 0.05, 0.2, 0.25), (1.2, 0.8, 0.0, 0.45, 1.5)]:
        d1 = (np.log(S / K) + (r + 0.5 * s * s) * tau) / (s * np.sqrt(tau))
        d2 = d1 - s * np.sqrt(tau)
        ref = S * _norm_cdf(d1) - K * np.exp(-r * tau) * _norm_cdf(d2)
        c = orc.bs_call(S, K, r, s, tau)
        assert abs(c - ref) < 1e-13
        put = K * np.exp(-r * tau) * _norm_cdf(-d2) - S * _norm_cdf(-d1)
        assert abs((c - put) - (S - K * np.exp(-r * tau))) < 1e-13
    assert orc.bs_call(2.0, 1.0, 0.05, 0.2, 0.0) == 1.0
    assert orc.bs_call(0.0, 1.0, 0.05, 0.2, 1.0) == 0.0


# ---------------------------------------------------------------- tridiagonal

def test_thomas_matches_dense_solve(orc):
    rng_u = synth.uniform(7, 200)
    k = 0
    for n in range(1, 9):
        lo = rng_u[k:k + n] - 0.5
        up = rng_u[k + n:k + 2 * n] - 0.5
        di = 2.0 + rng_u[k + 2 * n:k + 3 * n]
        rhs = rng_u[k + 3 * n:k + 4 * n]
        k += 4 * n
        A = np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
        x = orc.thomas(lo, di, up, rhs)
        np.testing.assert_allclose(x, np.linalg.solve(A, rhs), rtol=1e-14, atol=1e-15)


def test_thomas_zero_pivot_raises(orc):
    with pytest.raises(ArithmeticError):
        orc.thomas([0.0, 1.0], [0.0, 1.0], [1.0, 0.0], [1.0, 1.0])


def _dense_L(p):
    """Eq. 10 in tau as a dense matrix on the interior, built from the stencil written in S."""
    Nx = p.Nx
    n = Nx - 2
    dS = p.Smax / (Nx - 1)
    L = np.zeros((n, n))
    for i in range(n):
        S = (i + 1) * dS
        diff = 0.5 * p.sigma ** 2 * S ** 2 / dS ** 2
        conv = p.r * S / (2 * dS)
        if i > 0:
            L[i, i - 1] = diff - conv
        L[i, i] = -2 * diff - p.r
        if i < n - 1:
            L[i, i + 1] = diff + conv
    cN = 0.5 * p.sigma ** 2 * ((Nx - 2) * dS) ** 2 / dS ** 2 + p.r * (Nx - 2) * dS / (2 * dS)
    return L, cN


def test_cn_and_ie_steps_match_dense_formulas(orc):
    p = orc.params(Nx=9, sigma=0.3, r=0.04, Smax=3.0, K=1.2)
    L, cN = _dense_L(p)
    n = p.Nx - 2
    V = synth.random_states(3, 1, p.Nx)[0]
    V[0] = 0.0
    dt, tau_new = 0.01, 0.37
    V[-1] = orc.right_bc(p, tau_new - dt)
    Bn = orc.right_bc(p, tau_new)
    I = np.eye(n)
    b = np.zeros(n)
    b[-1] = cN * 0.5 * dt * (V[-1] + Bn)
    cn_ref = np.linalg.solve(I - 0.5 * dt * L, (I + 0.5 * dt * L) @ V[1:-1] + b)
    out = orc.cn_step(p, dt, tau_new, V)
    np.testing.assert_allclose(out[1:-1], cn_ref, rtol=1e-12, atol=1e-14)
    assert out[0] == 0.0 and out[-1] == Bn
    b2 = np.zeros(n)
    b2[-1] = cN * dt * Bn
    ie_ref = np.linalg.solve(I - dt * L, V[1:-1] + b2)
    out = orc.ie_step(p, dt, tau_new, V)
    np.testing.assert_allclose(out[1:-1], ie_ref, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- convergence

def _nodes_value(orc, p, S_probe):
    U = orc.serial_fine(p)
    dS = p.Smax / (p.Nx - 1)
    idx = [int(round(s / dS)) for s in S_probe]
    return U[-1][idx]


def test_cn_matches_closed_form_and_is_second_order(orc):
    # error against the exact price at nodes away from the kink, halving dS and dtau together
    S_probe = [0.5, 1.5, 2.0, 2.5]
    exact = np.array([orc.bs_call(s, 1.0, 0.05, 0.2, 1.0) for s in S_probe])
    errs = []
    for m in (6, 7, 8):
        Nx = 2 ** m + 1
        p = orc.params(Nx=Nx, P=4, fine_steps=2 ** (m - 3), Smax=4.0)
        errs.append(np.abs(_nodes_value(orc, p, S_probe) - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.8 and 3.3 < r2 < 4.8, errs
    assert errs[-1] < 2e-5


def test_cn_self_convergence_in_time(orc):
    # fixed grid, dtau halved: Richardson ratio of successive differences -> 4
    p = [orc.params(Nx=129, P=2, fine_steps=m, Smax=4.0) for m in (8, 16, 32, 64)]
    v = [_nodes_value(orc, q, [0.5, 2.0, 3.0]) for q in p]
    d1 = np.abs(v[0] - v[1]).max()
    d2 = np.abs(v[1] - v[2]).max()
    d3 = np.abs(v[2] - v[3]).max()
    assert 3.5 < d1 / d2 < 4.5 and 3.5 < d2 / d3 < 4.5


def test_ie_first_order_in_time(orc):
    p = [orc.params(Nx=129, P=1, coarse_steps=m, Smax=4.0) for m in (16, 32, 64, 128)]
    v = []
    for q in p:
        V = orc.payoff(q)
        v.append(orc.coarse_ie(q, 0, V)[[16, 64, 96]])
    d1 = np.abs(v[0] - v[1]).max()
    d2 = np.abs(v[1] - v[2]).max()
    d3 = np.abs(v[2] - v[3]).max()
    assert 1.8 < d1 / d2 < 2.2 and 1.8 < d2 / d3 < 2.2


# ---------------------------------------------------------------- Parareal

def test_parareal_k_equals_P_is_serial_fine_bitwise(orc):
    p = orc.params(Nx=64, P=6, fine_steps=16)
    Uf = orc.serial_fine(p)
    U, norms, st = orc.parareal(p, orc.COARSE_IE, tol=0.0)
    assert st == 0 and len(norms) == p.P
    assert np.array_equal(U, Uf)


def test_parareal_first_k_slices_exact(orc):
    p = orc.params(Nx=64, P=6, fine_steps=16)
    Uf = orc.serial_fine(p)
    for k in range(1, p.P):
        U, norms, st = orc.parareal(p, orc.COARSE_IE, tol=0.0, max_iter=k)
        assert st == 1 and len(norms) == k
        assert np.array_equal(U[: k + 1], Uf[: k + 1])
        if k + 1 <= p.P:
            assert not np.array_equal(U[k + 1:], Uf[k + 1:])


def test_parareal_ie_converges_fast(orc):
    # config-1 problem: IE coarse converges geometrically; error vs serial fine tracks the increment
    p = orc.params()
    Uf = orc.serial_fine(p)
    U, norms, st = orc.parareal(p, orc.COARSE_IE, tol=1e-6)
    assert st == 0 and len(norms) <= 6
    assert orc.rel_error(p, U, Uf) < 1e-6
    assert np.all(np.diff(norms) < 0)


def test_parareal_with_exact_coarse_table(orc):
    # coarse table = exact fine trajectory.  State-independent kind: U^0 = g is
    # exact and one iteration reproduces it bitwise (increment exactly 0).
    # Increment kind: U^0_{n+1} = U^0_n + g_{n+1} - g_n equals g up to rounding,
    # so the first increment is at rounding level and the result is exact after it.
    p = orc.params(Nx=64, P=5, fine_steps=8)
    Uf = orc.serial_fine(p)
    U, norms, st = orc.parareal(p, orc.COARSE_PINN, g=Uf, tol=1e-300)
    assert norms[0] == 0.0 and st == 0 and len(norms) == 1
    assert np.array_equal(U, Uf)
    U, norms, st = orc.parareal(p, orc.COARSE_PINN_INCR, g=Uf, tol=1e-14)
    assert norms[0] < 1e-15 and st == 0 and len(norms) == 1
    np.testing.assert_allclose(U, Uf, rtol=0, atol=1e-14)


def test_parareal_pinn_kind_reduces_to_fine_shift(orc):
    # G independent of U: U^{k+1}_{n+1} = F(U^k_n) exactly (G_new - G_old = 0)
    p = orc.params(Nx=48, P=4, fine_steps=8)
    g = np.tile(orc.payoff(p), (p.P + 1, 1)) * 0.9
    for n in range(p.P + 1):
        g[n, 0] = 0.0
        g[n, -1] = orc.right_bc(p, p.T * n / p.P)
    U1, _, _ = orc.parareal(p, orc.COARSE_PINN, g=g, tol=0.0, max_iter=1)
    U0 = g.copy()
    U0[0] = orc.payoff(p)
    for n in range(p.P):
        np.testing.assert_array_equal(U1[n + 1], orc.fine(p, n, U0[n]))


def _ie_parareal_by_hand(orc, p, iters):
    """Eq. 7 composed from the oracle's F and IE propagators, k iterations."""
    P = p.P
    U = np.empty((P + 1, p.Nx))
    U[0] = orc.payoff(p)
    Gold = np.empty((P, p.Nx))
    for n in range(P):
        Gold[n] = orc.coarse_ie(p, n, U[n])
        U[n + 1] = Gold[n]
    for k in range(iters):
        F = {n: orc.fine(p, n, U[n]) for n in range(k, P)}
        Unew = U.copy()
        for n in range(k, P):
            Gnew = orc.coarse_ie(p, n, Unew[n])
            Unew[n + 1] = F[n] + (Gnew - Gold[n])
            Gold[n] = Gnew
        U = Unew
    return U


def test_parareal_ie_iterations_compose_by_hand(orc):
    # Eq. 7 with G = implicit Euler, one and two iterations, built by hand from
    # the oracle's propagators: bitwise the oracle's Parareal
    p = orc.params(Nx=40, P=5, fine_steps=6)
    for iters in (1, 2):
        U, norms, st = orc.parareal(p, orc.COARSE_IE, tol=0.0, max_iter=iters)
        assert st == 1 and len(norms) == iters
        np.testing.assert_array_equal(U, _ie_parareal_by_hand(orc, p, iters))


def _smooth_table(orc, p, U, eps):
    """U perturbed by eps x a smooth bump in S and tau, Dirichlet nodes exact."""
    S = np.linspace(0.0, p.Smax, p.Nx)
    g = U.copy()
    for n in range(p.P + 1):
        g[n] += eps * np.sin(np.pi * S / p.Smax) * (1.0 + n / p.P) * p.Smax
        g[n, 0] = 0.0
        g[n, -1] = orc.right_bc(p, p.T * n / p.P)
    return g


def test_parareal_network_ie_one_iteration_by_hand(orc):
    # G(V) = IE(V) + (g_{n+1} - IE(g_n)) at the interior nodes, IE's Dirichlet
    # values at the ends: the initial sweep and one iteration composed by hand
    p = orc.params(Nx=40, P=5, fine_steps=6)
    g = _smooth_table(orc, p, orc.serial_fine(p), 3e-2)

    def G(n, V):
        out = orc.coarse_ie(p, n, V)
        gi = orc.coarse_ie(p, n, g[n])
        out[1:-1] = out[1:-1] + (g[n + 1, 1:-1] - gi[1:-1])
        return out

    U = np.empty((p.P + 1, p.Nx))
    U[0] = orc.payoff(p)
    Gold = [None] * p.P
    for n in range(p.P):
        Gold[n] = G(n, U[n])
        U[n + 1] = Gold[n]
    Unew = U.copy()
    for n in range(p.P):
        Unew[n + 1] = orc.fine(p, n, U[n]) + (G(n, Unew[n]) - Gold[n])
    U1, norms, st = orc.parareal(p, orc.COARSE_PINN_IE, g=g, tol=0.0, max_iter=1)
    np.testing.assert_array_equal(U1, Unew)


def test_parareal_network_ie_reduces_to_ie_on_the_ie_trajectory(orc):
    # with the table equal to the implicit Euler trajectory from the payoff the
    # correction g_{n+1} - IE(g_n) is exactly 0, so the kind is IE-coarse
    # Parareal bit for bit, iteration by iteration
    p = orc.params(Nx=64, P=6, fine_steps=16)
    g = np.empty((p.P + 1, p.Nx))
    g[0] = orc.payoff(p)
    for n in range(p.P):
        g[n + 1] = orc.coarse_ie(p, n, g[n])
    for iters in (1, 3):
        Ua, na, _ = orc.parareal(p, orc.COARSE_IE, tol=0.0, max_iter=iters)
        Ub, nb, _ = orc.parareal(p, orc.COARSE_PINN_IE, g=g, tol=0.0, max_iter=iters)
        np.testing.assert_array_equal(Ua, Ub)
        np.testing.assert_array_equal(na, nb)


def test_parareal_network_ie_invariants_and_convergence(orc):
    p = orc.params(Nx=64, P=6, fine_steps=16)
    Uf = orc.serial_fine(p)
    # exact table: G(F-trajectory) reproduces it up to rounding, so the first
    # increment is at rounding level
    U, norms, st = orc.parareal(p, orc.COARSE_PINN_IE, g=Uf, tol=1e-13)
    assert st == 0 and len(norms) == 1 and norms[0] < 1e-14
    np.testing.assert_allclose(U, Uf, rtol=0, atol=1e-14)
    # Section 3.1 invariants: slices 0..k exact after k iterations, k = P is serial fine
    g = _smooth_table(orc, p, Uf, 1e-2)
    for k in range(1, p.P + 1):
        U, norms, st = orc.parareal(p, orc.COARSE_PINN_IE, g=g, tol=0.0, max_iter=k)
        assert np.array_equal(U[: k + 1], Uf[: k + 1])
    assert np.array_equal(U, Uf)
    # the error recursion is IE-coarse Parareal's (the correction cancels in
    # G_new - G_old), so a table closer to the fine solution than IE's own
    # trajectory needs no more iterations than IE coarse
    p1 = orc.params()
    Uf1 = orc.serial_fine(p1)
    _, n_ie, _ = orc.parareal(p1, orc.COARSE_IE, tol=1e-10)
    for eps in (1e-3, 1e-5):
        U, n_pi, st = orc.parareal(p1, orc.COARSE_PINN_IE, g=_smooth_table(orc, p1, Uf1, eps), tol=1e-10)
        assert st == 0 and len(n_pi) <= len(n_ie)
        assert orc.rel_error(p1, U, Uf1) < 1e-9


def test_speedup_bound(orc):
    assert orc.speedup_bound(16, 3, 0.0) == pytest.approx(16.0 / 3.0, rel=1e-15)
    # eq. 8 with c_c = c_f and K = P gives 1 / (2 + 1) ... = 1/3
    assert orc.speedup_bound(4, 4, 1.0) == pytest.approx(1.0 / 3.0, rel=1e-15)


# ---------------------------------------------------------------- network

def _torch_mlp(widths, params, lo, hi, X):
    """Reference network in PyTorch FP64 (library layers + autograd)."""
    x = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    lo_t = torch.tensor(lo, dtype=torch.float64)
    hi_t = torch.tensor(hi, dtype=torch.float64)
    h = 2.0 * (x - lo_t) / (hi_t - lo_t) - 1.0
    off = 0
    P = torch.tensor(params, dtype=torch.float64)
    for l in range(1, len(widths)):
        wi, wo = widths[l - 1], widths[l]
        W = P[off:off + wo * wi].reshape(wo, wi)
        b = P[off + wo * wi:off + wo * wi + wo]
        off += wo * wi + wo
        h = torch.nn.functional.linear(h, W, b)
        if l < len(widths) - 1:
            h = torch.tanh(h)
    u = h[:, 0]
    g = torch.autograd.grad(u.sum(), x, create_graph=True)[0]
    uS, uT = g[:, 0], g[:, 1]
    uSS = torch.autograd.grad(uS.sum(), x)[0][:, 0]
    return u.detach().numpy(), uS.detach().numpy(), uSS.numpy(), uT.detach().numpy()


@pytest.mark.parametrize("widths", [[2, 16, 16, 1], [2, 8, 8, 8, 1], [5, 12, 12, 1]])
def test_mlp_forward_and_derivatives_match_autograd(orc, widths):
    d_in = widths[0]
    params = synth.xavier_params(widths, 11)
    params[np.arange(params.size) % 7 == 3] += 0.1  # non-zero biases too
    lo = np.array([0.0, 0.0, 0.1, 0.0, 0.5][:d_in])
    hi = np.array([4.0, 1.0, 0.5, 0.08, 2.0][:d_in])
    u01 = synth.uniform(5, 40 * d_in).reshape(40, d_in)
    X = lo + (hi - lo) * u01
    m = orc.MLP(widths, params, lo, hi)
    u, d = orc.mlp_eval(m, X)
    ru, ruS, ruSS, ruT = _torch_mlp(widths, params, lo, hi, X)
    np.testing.assert_allclose(u, ru, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(d[:, 0], ruS, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(d[:, 1], ruSS, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(d[:, 2], ruT, rtol=1e-12, atol=1e-13)


def test_mlp_derivatives_match_finite_differences(orc):
    widths = [2, 10, 10, 1]
    params = synth.xavier_params(widths, 2)
    lo, hi = np.array([0.0, 0.0]), np.array([4.0, 1.0])
    m = orc.MLP(widths, params, lo, hi)
    X = np.array([[0.7, 0.2], [2.1, 0.8], [3.3, 0.5]])
    u, d = orc.mlp_eval(m, X)
    h = 1e-5
    up = orc.mlp_eval(m, X + [h, 0], False)
    um = orc.mlp_eval(m, X - [h, 0], False)
    np.testing.assert_allclose(d[:, 0], (up - um) / (2 * h), rtol=1e-8)
    h2 = 1e-4
    up = orc.mlp_eval(m, X + [h2, 0], False)
    um = orc.mlp_eval(m, X - [h2, 0], False)
    np.testing.assert_allclose(d[:, 1], (up - 2 * u + um) / h2 ** 2, rtol=1e-5, atol=1e-7)
    tp = orc.mlp_eval(m, X + [0, h], False)
    tm = orc.mlp_eval(m, X - [0, h], False)
    np.testing.assert_allclose(d[:, 2], (tp - tm) / (2 * h), rtol=1e-8)


def test_pinn_table_boundary_nodes(orc):
    p = orc.params(Nx=17, P=3)
    widths = [2, 6, 1]
    m = orc.MLP(widths, synth.xavier_params(widths, 4), [0.0, 0.0], [4.0, 1.0])
    g = orc.pinn_table(p, m)
    dS = p.Smax / (p.Nx - 1)
    for n in range(p.P + 1):
        tau = p.T * n / p.P
        assert g[n, 0] == 0.0 and g[n, -1] == orc.right_bc(p, tau)
        X = np.stack([np.arange(1, p.Nx - 1) * dS, np.full(p.Nx - 2, tau)], axis=1)
        np.testing.assert_array_equal(g[n, 1:-1], orc.mlp_eval(m, X, False))


def _torch_loss(widths, params, lo, hi, X, kind, K, sigma, r, Smax, smax_over_K=0.0, y=None):
    """Eqs. 11-14 with PyTorch autograd (the paper's route), FP64; kind-4 points
    (with values y) add their squared misfit to the mean of term 0."""
    x = torch.tensor(X, dtype=torch.float64, requires_grad=True)
    P = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    lo_t = torch.tensor(lo, dtype=torch.float64)
    hi_t = torch.tensor(hi, dtype=torch.float64)
    h = 2.0 * (x - lo_t) / (hi_t - lo_t) - 1.0
    off = 0
    for l in range(1, len(widths)):
        wi, wo = widths[l - 1], widths[l]
        W = P[off:off + wo * wi].reshape(wo, wi)
        b = P[off + wo * wi:off + wo * wi + wo]
        off += wo * wi + wo
        h = torch.nn.functional.linear(h, W, b)
        if l < len(widths) - 1:
            h = torch.tanh(h)
    u = h[:, 0]
    g = torch.autograd.grad(u.sum(), x, create_graph=True)[0]
    uS, uT = g[:, 0], g[:, 1]
    uSS = torch.autograd.grad(uS.sum(), x, create_graph=True)[0][:, 0]
    kind = torch.tensor(kind)
    S = x[:, 0].detach()
    if X.shape[1] >= 5:
        sig, rr, KK = x[:, 2].detach(), x[:, 3].detach(), x[:, 4].detach()
        Sm = smax_over_K * KK if smax_over_K > 0 else torch.full_like(KK, Smax)
    else:
        sig = torch.full_like(S, sigma)
        rr = torch.full_like(S, r)
        KK = torch.full_like(S, K)
        Sm = torch.full_like(S, Smax)
    tau = x[:, 1].detach()
    f = uT - 0.5 * sig ** 2 * S ** 2 * uSS - rr * S * uS + rr * u
    tgt = torch.where(kind == 1, torch.zeros_like(S),
                      torch.where(kind == 2, Sm - KK * torch.exp(-rr * tau), torch.clamp(S - KK, min=0.0)))
    r0 = f[kind == 0] ** 2
    if y is not None:
        r0 = torch.cat([r0, (u - torch.tensor(y, dtype=torch.float64))[kind == 4] ** 2])
    mf = r0.mean()
    mb = ((u - tgt)[(kind == 1) | (kind == 2)] ** 2).mean()
    me = ((u - tgt)[kind == 3] ** 2).mean()
    total = mf + mb + me
    grad = torch.autograd.grad(total, P)[0]
    return np.array([mf.item(), mb.item(), me.item()]), grad.numpy()


def test_loss_and_gradient_match_autograd(orc):
    widths = [2, 12, 12, 1]
    params = synth.xavier_params(widths, 9)
    lo, hi = np.array([0.0, 0.0]), np.array([4.0, 1.0])
    X, kind = synth.collocation(21, 60, 16, 12, 4.0, 1.0)
    m = orc.MLP(widths, params, lo, hi)
    terms, grad = orc.pinn_loss_grad(m, X, kind, 1.0, 0.2, 0.05, 4.0)
    rt, rg = _torch_loss(widths, params, lo, hi, X, kind, 1.0, 0.2, 0.05, 4.0)
    np.testing.assert_allclose(terms, rt, rtol=1e-12)
    np.testing.assert_allclose(grad, rg, rtol=1e-10, atol=1e-13)


def test_data_points_loss_and_gradient_match_autograd(orc):
    # kind 4: squared misfit to a given value, in term 0 with the residual points
    # (a mixed batch) or alone (a data-only batch, no PDE terms)
    widths = [2, 12, 12, 1]
    params = synth.xavier_params(widths, 19)
    lo, hi = np.array([0.0, 0.0]), np.array([4.0, 1.0])
    m = orc.MLP(widths, params, lo, hi)
    X, kind = synth.collocation(23, 60, 16, 12, 4.0, 1.0)
    rng = np.random.default_rng(5)
    kind = kind.copy()
    kind[rng.random(kind.size) < 0.3] = 4
    y = rng.normal(size=kind.size)
    for kk in (kind, np.full_like(kind, 4)):
        terms, grad = orc.pinn_loss_grad(m, X, kk, 1.0, 0.2, 0.05, 4.0, y=y)
        rt, rg = _torch_loss(widths, params, lo, hi, X, kk, 1.0, 0.2, 0.05, 4.0, y=y)
        rt = np.nan_to_num(rt)  # an empty term's mean is NaN in torch, 0 in the oracle
        np.testing.assert_allclose(terms, rt, rtol=1e-12)
        np.testing.assert_allclose(grad, rg, rtol=1e-10, atol=1e-13)


def test_loss_rejects_invalid_kinds(orc):
    # kinds outside 0..3, and data points (kind 4) without their values, are
    # input errors of the loss definition, not a fifth term
    widths = [2, 8, 1]
    m = orc.MLP(widths, synth.xavier_params(widths, 1), [0.0, 0.0], [4.0, 1.0])
    X, kind = synth.collocation(3, 20, 4, 4, 4.0, 1.0)
    for bad in (5, -1):
        kb = kind.copy()
        kb[2] = bad
        with pytest.raises(ValueError):
            orc.pinn_loss_grad(m, X, kb, 1.0, 0.2, 0.05, 4.0)
    kb = kind.copy()
    kb[2] = 4
    with pytest.raises(ValueError):
        orc.pinn_loss_grad(m, X, kb, 1.0, 0.2, 0.05, 4.0)
    orc.pinn_loss_grad(m, X, kb, 1.0, 0.2, 0.05, 4.0, y=np.zeros(len(kb)))


def test_parametric_loss_gradient_matches_autograd(orc):
    widths = [5, 10, 10, 1]
    params = synth.xavier_params(widths, 13)
    lo = np.array([0.0, 0.0, 0.1, 0.0, 0.5])
    hi = np.array([8.0, 2.0, 0.5, 0.08, 2.0])
    X, kind = synth.collocation_parametric(3, 50, 10, 10, 4.0, 2.0)
    m = orc.MLP(widths, params, lo, hi)
    terms, grad = orc.pinn_loss_grad(m, X, kind, 0.0, 0.0, 0.0, 0.0, smax_over_K=4.0)
    rt, rg = _torch_loss(widths, params, lo, hi, X, kind, 0, 0, 0, 0, smax_over_K=4.0)
    np.testing.assert_allclose(terms, rt, rtol=1e-12)
    np.testing.assert_allclose(grad, rg, rtol=1e-10, atol=1e-13)


def test_loss_gradient_matches_central_differences(orc):
    widths = [2, 6, 6, 1]
    params = synth.xavier_params(widths, 17)
    lo, hi = np.array([0.0, 0.0]), np.array([4.0, 1.0])
    X, kind = synth.collocation(5, 30, 8, 8, 4.0, 1.0)
    m = orc.MLP(widths, params, lo, hi)
    _, grad = orc.pinn_loss_grad(m, X, kind, 1.0, 0.2, 0.05, 4.0)
    h = 1e-6
    idx = [0, 5, 13, 20, 40, 55, params.size - 1]
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fp = orc.pinn_loss_grad(orc.MLP(widths, pp, lo, hi), X, kind, 1.0, 0.2, 0.05, 4.0, with_grad=False).sum()
        fm = orc.pinn_loss_grad(orc.MLP(widths, pm, lo, hi), X, kind, 1.0, 0.2, 0.05, 4.0, with_grad=False).sum()
        assert abs((fp - fm) / (2 * h) - grad[i]) <= 1e-6 * max(1.0, abs(grad[i]))


def test_adam_matches_torch_and_hand_step(orc):
    # hand-computed first step on f(theta) = theta^2 from theta = 1, lr = 0.1:
    # m = 0.2, v = 0.004, m^ = 2, v^ = 4 -> theta = 1 - 0.1 * 2 / (2 + 1e-8)
    th, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    orc.adam(th, m, v, np.array([2.0]), 1, 0.1)
    assert th[0] == pytest.approx(1.0 - 0.2 / (2.0 + 1e-8), rel=1e-15)
    # 5 steps against torch.optim.Adam on a quadratic with 3 parameters
    theta0 = np.array([1.0, -2.0, 0.5])
    w = torch.tensor(theta0.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    th, m, v = theta0.copy(), np.zeros(3), np.zeros(3)
    A = np.array([1.0, 3.0, 0.2])
    for t in range(1, 6):
        opt.zero_grad()
        loss = (torch.tensor(A) * w * w).sum()
        loss.backward()
        g = 2 * A * th
        opt.step()
        orc.adam(th, m, v, g, t, 0.05)
    np.testing.assert_allclose(th, w.detach().numpy(), rtol=1e-14, atol=1e-15)


def test_oracle_rounding_within_calibrated_bound(orc):
    # noisy state at mesh ratio h sigma^2 j^2 ~ 6e3: the oracle's own distance to
    # a long-double recomputation stays within 2 kappa u N (N = 6 CN steps), the
    # bound the GPU parity tests use for such stress cases, and exceeds 1e-12
    K = 1.7
    p = orc.params(K=K, sigma=0.37, r=0.01, T=1.6, Smax=4 * K, Nx=1025, P=3, fine_steps=6)
    S = synth.random_states(111, 1, p.Nx, scale=p.Smax)[0]
    S[0], S[-1] = 0.0, orc.right_bc(p, 0.0)
    ref = _cn_longdouble(p, 0, S)
    err = float(np.abs(orc.fine(p, 0, S) - ref).max() / np.abs(ref).max())
    h = 0.5 * p.T / (p.P * p.fine_steps)
    j = p.Nx - 2
    kappa = 1 + h * (2 * p.sigma ** 2 * j * j + p.r * j + p.r)
    assert 1e-12 < err <= 2 * kappa * 2.0 ** -53 * p.fine_steps
