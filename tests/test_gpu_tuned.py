"""Partition choice: every compiled partition of a grid (forced with
BSP_PARTITION) matches the oracle, and bs_problem_init_tuned times the
candidates, keeps one per grid size and gives the same answers.  Tolerances as
in test_gpu_solver.py (calibrated FP64 bound, at least 1e-12 relative).
"""
import numpy as np
import pytest

from paper_2303_03848_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
RTOL = 1e-12
# partitions (M rows per thread, NW warps per CTA, C CTAs per grid) tried per grid
SHAPES = [(m, nw, c) for c in (1, 2, 4, 8, 16) for nw in (1, 2, 4, 8) for m in (2, 4, 8, 16, 32)]


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03848_b300 import binding, build

    build.build()
    return binding


def _tol(p, kind):
    steps = p["fine_steps"] if kind == "fine" else p["coarse_steps"]
    dt = p["T"] / (p["P"] * steps)
    h = 0.5 * dt if kind == "fine" else dt
    j = p["Nx"] - 2
    kappa = 1.0 + h * (2.0 * p["sigma"] ** 2 * j * j + p["r"] * j + p["r"])
    return max(RTOL, 2.0 * kappa * 2.0 ** -53 * steps)


def _close(a, b, rtol):
    a, b = np.asarray(a), np.asarray(b)
    err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
    assert err <= rtol, f"relative error {err:.3e} > {rtol:.1e}"


def _slices(orc, p, seed):
    op = orc.params(**p)
    S = synth.random_states(seed, p["P"], p["Nx"], scale=p["Smax"])
    for n in range(p["P"]):
        S[n, 0] = 0.0
        S[n, -1] = orc.right_bc(op, p["T"] * n / p["P"])
    return S


def _check_against_oracle(B, orc, prob, insts, parts):
    Uin = torch.tensor(np.concatenate([s.ravel() for s in parts]), device="cuda")
    F = prob.fine_propagate(Uin).cpu().numpy()
    G = prob.coarse_propagate(Uin).cpu().numpy()
    assert prob.device_status() == B.BS_OK
    for i, p in enumerate(insts):
        op = orc.params(**p)
        o = prob.slice_off[i]
        for n in range(p["P"]):
            sl = slice(o + n * p["Nx"], o + (n + 1) * p["Nx"])
            _close(F[sl], orc.fine(op, n, parts[i][n]), _tol(p, "fine"))
            _close(G[sl], orc.coarse_ie(op, n, parts[i][n]), _tol(p, "coarse"))


@pytest.mark.parametrize("Nx", [256, 1000, 2049, 40000])
def test_every_partition_matches_oracle(B, orc, monkeypatch, Nx):
    p = dict(K=1.0, sigma=0.25, r=0.04, T=1.0, Smax=4.0, Nx=Nx, P=2, fine_steps=6, coarse_steps=2)
    parts = [_slices(orc, p, 70 + Nx)]
    tried = 0
    for m, nw, c in SHAPES:
        R = m * nw * 32 * c
        if R < Nx - 1 or 2 * (R - (Nx - 1)) > R:
            continue
        monkeypatch.setenv("BSP_PARTITION", f"{m},{nw},{c}")
        try:
            prob = B.Problem(p)
        except B.BsError as e:
            assert e.code == B.BS_EUNSUPPORTED  # not a compiled class
            continue
        assert prob.partition(0) == dict(M=m, NW=nw, C=c)
        _check_against_oracle(B, orc, prob, [p], parts)
        tried += 1
    assert tried >= (2 if Nx > 32768 else 3)  # 40000 points: 32 rows x 4 warps x 16 CTAs, 32 x 8 x 8


def test_forced_partition_too_small_is_rejected(B, monkeypatch):
    monkeypatch.setenv("BSP_PARTITION", "2,1,1")
    with pytest.raises(B.BsError) as e:
        B.Problem(dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=1024, P=2, fine_steps=4, coarse_steps=1))
    assert e.value.code == B.BS_EUNSUPPORTED


def test_tuned_init_keeps_one_partition_per_grid_and_matches_oracle(B, orc):
    insts = [dict(K=0.8 + 0.1 * i, sigma=0.15 + 0.03 * i, r=0.01 * i, T=0.5 + 0.25 * i, Smax=4.0 * (0.8 + 0.1 * i),
                  Nx=Nx, P=3, fine_steps=8, coarse_steps=1)
             for i, Nx in enumerate((256, 1024, 256, 513, 1024, 513))]
    prob = B.Problem(insts, tuned=True)
    rep = prob.tuning
    assert {r["Nx"] for r in rep} == {256, 513, 1024}
    for Nx in (256, 513, 1024):
        mine = [r for r in rep if r["Nx"] == Nx]
        chosen = [r for r in mine if r["chosen"]]
        assert len(chosen) == 1 and all(r["ms"] > 0.0 for r in mine)
        best = min(mine, key=lambda r: r["ms"])
        assert chosen[0] == best
        for r in mine:
            R = r["M"] * r["NW"] * 32 * r["C"]
            assert R >= Nx - 1 and 2 * (R - (Nx - 1)) <= R
        for i, p in enumerate(insts):
            if p["Nx"] == Nx:
                assert prob.partition(i) == dict(M=best["M"], NW=best["NW"], C=best["C"])
    parts = [_slices(orc, p, 90 + i) for i, p in enumerate(insts)]
    _check_against_oracle(B, orc, prob, insts, parts)


def test_tuned_parareal_matches_oracle(B, orc):
    p = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=256, P=8, fine_steps=128, coarse_steps=1)
    prob = B.Problem([p], tuned=True)
    U, norms, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=1e-10)
    Ur, nr, st = orc.parareal(orc.params(**p), orc.COARSE_IE, tol=1e-10)
    assert rc == B.BS_OK and stats[0]["iterations"] == len(nr)
    np.testing.assert_allclose(norms[0, :len(nr)], nr, rtol=1e-6)
    steps = p["fine_steps"] * p["P"]
    j = p["Nx"] - 2
    kappa = 1.0 + 0.5 * p["T"] / steps * (2.0 * p["sigma"] ** 2 * j * j + p["r"] * j + p["r"])
    _close(U.cpu().numpy(), Ur.ravel(), max(RTOL, 2.0 * kappa * 2.0 ** -53 * steps))


@pytest.mark.parametrize("part", ["32,8,8", "32,4,16", "16,4,8"])
def test_three_table_partitions_parareal_match_oracle(B, orc, monkeypatch, part):
    # clusters of 8 or more CTAs keep three coefficient tables and finish each
    # step with a second sweep over the inner rows: implicit-Euler Parareal on
    # such a grid against the oracle's, iterates and increment norms
    monkeypatch.setenv("BSP_PARTITION", part)
    Nx = {"32,8,8": 40000, "32,4,16": 40000, "16,4,8": 12000}[part]
    p = dict(K=1.0, sigma=0.3, r=0.03, T=0.5, Smax=8.0, Nx=Nx, P=4, fine_steps=8, coarse_steps=1)
    prob = B.Problem(p)
    m, nw, c = (int(v) for v in part.split(","))
    assert prob.partition(0) == dict(M=m, NW=nw, C=c)
    U, norms, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=1e-9)
    assert prob.device_status() == B.BS_OK
    Ur, nr, st = orc.parareal(orc.params(**p), orc.COARSE_IE, tol=1e-9)
    assert rc == B.BS_OK and stats[0]["iterations"] == len(nr)
    np.testing.assert_allclose(norms[0, :len(nr)], nr, rtol=1e-6)
    steps = p["fine_steps"] * p["P"]
    j = p["Nx"] - 2
    kappa = 1.0 + 0.5 * p["T"] / steps * (2.0 * p["sigma"] ** 2 * j * j + p["r"] * j + p["r"])
    _close(U.cpu().numpy(), Ur.ravel(), max(RTOL, 2.0 * kappa * 2.0 ** -53 * steps))


# two slices per CTA (slice pairs sharing the coefficient tables; one-CTA grids
# step on a named barrier per slice, clusters on mbarriers): same per-slice
# arithmetic as one slice per CTA, so the results agree bit for bit; odd slice
# counts leave one group of the last pair idle
PAIR_CASES = [((16, 2, 1), 1000), ((32, 1, 1), 1000), ((32, 2, 1), 2000), ((16, 4, 1), 2000), ((32, 4, 1), 4000),
              ((16, 4, 2), 4000), ((32, 4, 2), 6000), ((16, 4, 4), 6000), ((32, 4, 4), 12000),
              ((16, 4, 8), 12000), ((32, 4, 8), 30000), ((16, 4, 16), 30000), ((32, 4, 16), 65536)]


@pytest.mark.parametrize("shape,Nx", PAIR_CASES)
def test_slice_pairs_equal_single_slices_and_match_oracle(B, orc, monkeypatch, shape, Nx):
    m, nw, c = shape
    p = dict(K=1.0, sigma=0.3, r=0.03, T=0.5, Smax=8.0, Nx=Nx, P=3, fine_steps=4, coarse_steps=1)
    parts = [_slices(orc, p, 7 + Nx)]
    Uin = torch.tensor(parts[0].ravel(), device="cuda")
    out = {}
    for s2 in (1, 2):
        monkeypatch.setenv("BSP_PARTITION", f"{m},{nw},{c},{s2}")
        prob = B.Problem(p)
        out[s2] = prob.fine_propagate(Uin)
        assert prob.device_status() == B.BS_OK
    assert torch.equal(out[1], out[2])
    F = out[2].cpu().numpy().reshape(p["P"], Nx)
    op = orc.params(**p)
    for n in range(p["P"]):
        _close(F[n], orc.fine(op, n, parts[0][n]), _tol(p, "fine"))


@pytest.mark.parametrize("P", [4, 5])
def test_slice_pairs_parareal_network_and_ie_bitwise(B, monkeypatch, P):
    p = dict(K=1.0, sigma=0.3, r=0.03, T=0.5, Smax=8.0, Nx=4000, P=P, fine_steps=8, coarse_steps=1)
    net = B.PinnModel([2, 32, 32, 1], [0.0, 0.0], [8.0, 0.5], seed=2)
    res = {}
    for s2 in (1, 2):
        monkeypatch.setenv("BSP_PARTITION", f"16,4,2,{s2}")
        prob = B.Problem(p)
        Un, nn, sn, rn = prob.parareal_solve(B.COARSE_PINN, model=net, prec=B.FP64, tol=0.0)
        Ui, ni, si, ri = prob.parareal_solve(B.COARSE_IE, tol=0.0)
        assert rn == B.BS_OK and ri == B.BS_OK and prob.device_status() == B.BS_OK
        res[s2] = (Un, nn, Ui, ni, prob.serial_fine())
    for a, b in zip(res[1], res[2]):
        if isinstance(a, torch.Tensor):
            assert torch.equal(a, b)
        else:
            np.testing.assert_array_equal(a, b)
    assert torch.equal(res[2][0], res[2][4])  # k = P reproduces serial fine


@pytest.mark.parametrize("shape", [(32, 4, 1), (16, 2, 1)])
@pytest.mark.parametrize("P", [4, 5])
def test_counter_fed_slice_pairs_parareal_bitwise(B, orc, monkeypatch, shape, P):
    # one-CTA grids in a Parareal solve take their task groups from a counter and
    # start them at slice k, so with odd k the pairs are (k, k+1), ...: the
    # iterates, norms and iteration counts equal one slice per CTA bit for bit,
    # and the implicit-Euler solve matches the oracle's
    m, nw, c = shape
    Nx = {(32, 4, 1): 4000, (16, 2, 1): 1000}[shape]
    insts = [dict(K=0.8 + 0.2 * i, sigma=0.25 + 0.05 * i, r=0.02 + 0.01 * i, T=0.5, Smax=4.0 * (0.8 + 0.2 * i),
                  Nx=Nx, P=P, fine_steps=6, coarse_steps=1) for i in range(3)]
    net = B.PinnModel([2, 32, 32, 1], [0.0, 0.0], [4.0, 0.5], seed=3)
    res = {}
    for s2 in (1, 2):
        monkeypatch.setenv("BSP_PARTITION", f"{m},{nw},{c},{s2}")
        prob = B.Problem(insts)
        assert prob.slices_per_cta(0) == s2
        Ui, ni, si, ri = prob.parareal_solve(B.COARSE_IE, tol=1e-9)
        Ua, na, sa, ra = prob.parareal_solve(B.COARSE_PINN_IE, model=net, prec=B.FP64, tol=0.0)
        assert ri == B.BS_OK and ra == B.BS_OK and prob.device_status() == B.BS_OK
        res[s2] = (Ui, ni, [x["iterations"] for x in si], Ua, na, prob.serial_fine())
    for a, b in zip(res[1], res[2]):
        if isinstance(a, torch.Tensor):
            assert torch.equal(a, b)
        else:
            np.testing.assert_array_equal(np.asarray(a), np.asarray(b))
    assert torch.equal(res[2][3], res[2][5])  # tol 0: k = P reproduces serial fine
    U = res[2][0].cpu().numpy()
    off = 0
    for i, p in enumerate(insts):
        Ur, nr, st = orc.parareal(orc.params(**p), orc.COARSE_IE, tol=1e-9)
        assert res[2][2][i] == len(nr)
        np.testing.assert_allclose(res[2][1][i, :len(nr)], nr, rtol=1e-6)
        steps = p["fine_steps"] * P
        kappa = 1.0 + 0.5 * p["T"] / steps * (2.0 * p["sigma"] ** 2 * (Nx - 2) ** 2 + p["r"] * (Nx - 2) + p["r"])
        _close(U[off:off + (P + 1) * Nx], Ur.ravel(), max(RTOL, 2.0 * kappa * 2.0 ** -53 * steps))
        off += (P + 1) * Nx


def test_converged_batch_skips_the_remaining_iterations(B):
    # once the stop-rule kernel counts no instance still iterating, the later
    # launches return at once: a solve allowed 64 iterations equals one allowed
    # just past the slowest instance's count, statistics included
    insts = synth.batched_instances(5, 6, P=16, fine_steps=32, coarse_steps=1, Nx_choices=(256, 1024))
    prob = B.Problem(insts, tuned=True)
    U1, n1, s1, r1 = prob.parareal_solve(B.COARSE_IE, tol=1e-6, max_iter=16)
    kmax = max(x["iterations"] for x in s1)
    assert r1 == B.BS_OK and kmax < 16  # the oracle takes 5 or 6 iterations on these instances
    U2, n2, s2, r2 = prob.parareal_solve(B.COARSE_IE, tol=1e-6, max_iter=kmax)
    assert r2 == B.BS_OK and torch.equal(U1, U2)
    assert [x["iterations"] for x in s1] == [x["iterations"] for x in s2]
    np.testing.assert_array_equal(n1[:, :kmax], n2[:, :kmax])
    assert np.isnan(n1[:, kmax:]).all()


def test_slice_pair_rule_follows_the_slice_count(B, monkeypatch):
    # a 30000-point grid takes a clustered partition with 16 or 32 rows per
    # thread (16 CTAs for 8 slices, 8 CTAs for 40); pairs once the slices can
    # keep every cluster busy twice over, and on request
    monkeypatch.delenv("BSP_PARTITION", raising=False)
    base = dict(K=1.0, sigma=0.3, r=0.03, T=0.5, Smax=8.0, Nx=30000, fine_steps=2, coarse_steps=1)
    few, many = B.Problem(dict(base, P=8)), B.Problem(dict(base, P=40))
    assert few.partition(0) == dict(M=16, NW=4, C=16) and many.partition(0) == dict(M=32, NW=4, C=8)
    assert few.slices_per_cta(0) == 1 and many.slices_per_cta(0) == 2
    monkeypatch.setenv("BSP_S2", "1")
    assert B.Problem(dict(base, P=40)).slices_per_cta(0) == 1
    monkeypatch.setenv("BSP_S2", "2")
    assert B.Problem(dict(base, P=8)).slices_per_cta(0) == 2


def test_slice_pairs_with_mixed_slice_counts(B, orc, monkeypatch):
    # instances of one class with P = 3, 5, 8: pairs partly or wholly past an
    # instance's last slice are skipped, the rest match single slices bitwise
    insts = [dict(K=0.9 + 0.1 * i, sigma=0.2 + 0.05 * i, r=0.02 * i, T=0.5, Smax=8.0, Nx=4000, P=P, fine_steps=3,
                  coarse_steps=1) for i, P in enumerate((3, 5, 8))]
    parts = [_slices(orc, p, 50 + i) for i, p in enumerate(insts)]
    Uin = torch.tensor(np.concatenate([s.ravel() for s in parts]), device="cuda")
    out = {}
    for s2 in (1, 2):
        monkeypatch.setenv("BSP_PARTITION", f"16,4,2,{s2}")
        prob = B.Problem(insts)
        out[s2] = (prob.fine_propagate(Uin), prob.parareal_solve(B.COARSE_IE, tol=1e-9)[0])
        assert prob.device_status() == B.BS_OK
    assert torch.equal(out[1][0], out[2][0]) and torch.equal(out[1][1], out[2][1])
    F = out[2][0].cpu().numpy()
    off = 0
    for i, p in enumerate(insts):
        op = orc.params(**p)
        for n in range(p["P"]):
            _close(F[off + n * p["Nx"]:off + (n + 1) * p["Nx"]], orc.fine(op, n, parts[i][n]), _tol(p, "fine"))
        off += p["P"] * p["Nx"]


def test_tuner_times_slice_pairs_where_supported(B, orc):
    insts = [dict(K=1.0, sigma=0.25, r=0.03, T=0.5, Smax=8.0, Nx=4000, P=40, fine_steps=4, coarse_steps=1)
             for _ in range(2)]
    prob = B.Problem(insts, tuned=True)
    rep = prob.tuning
    assert {r["S2"] for r in rep} == {1, 2}
    pairs = [r for r in rep if r["S2"] == 2]
    assert all(r["M"] >= 16 for r in pairs)
    chosen = [r for r in rep if r["chosen"]]
    assert len(chosen) == 1 and chosen[0] == min(rep, key=lambda r: r["ms"])
    assert prob.slices_per_cta(0) == chosen[0]["S2"]
    parts = [_slices(orc, p, 60 + i) for i, p in enumerate(insts)]
    _check_against_oracle(B, orc, prob, insts, parts)


def test_tuning_cache_round_trip(B, tmp_path):
    # the tuner's choices saved per device, grid size and slice count, then a
    # second set-up from the file without timing: same partitions, same results
    insts = synth.batched_instances(2, 40, P=8, fine_steps=16, coarse_steps=1, Nx_choices=(256, 1024))
    path = str(tmp_path / "tuning.json")
    a = B.Problem(insts, tuned=True, tuning_cache=path)
    assert a.tuning_source == "timed"
    b = B.Problem(insts, tuned=True, tuning_cache=path)
    assert b.tuning_source == "cache"
    for i in range(len(insts)):
        assert a.partition(i) == b.partition(i) and a.slices_per_cta(i) == b.slices_per_cta(i)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4)
    U = torch.rand(a.total_slice, dtype=torch.float64, device="cuda", generator=gen)
    assert torch.equal(a.fine_propagate(U), b.fine_propagate(U))
    # another slice count is another key: timed again
    c = B.Problem(synth.batched_instances(2, 3, P=8, fine_steps=16, coarse_steps=1, Nx_choices=(256,)), tuned=True,
                  tuning_cache=path)
    assert c.tuning_source == "timed"
