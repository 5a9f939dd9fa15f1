"""A whole Parareal solve captured in a CUDA graph replays to the same bits as
the direct call (numerical and network coarse propagators, one and several
instances), and replays are repeatable."""
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


def test_graph_replay_equals_direct_solve_ie(B):
    insts = [dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=256, P=8, fine_steps=128, coarse_steps=1),
             dict(K=1.5, sigma=0.3, r=0.02, T=0.5, Smax=6.0, Nx=512, P=8, fine_steps=64, coarse_steps=1)]
    prob = B.Problem(insts)
    U, norms, stats, rc = prob.parareal_solve(B.COARSE_IE, tol=1e-10)
    assert rc == B.BS_OK
    g = B.SolveGraph(prob, B.COARSE_IE, tol=1e-10)
    g.U.zero_()
    Ug = g.replay().clone()
    torch.cuda.synchronize()
    assert torch.equal(Ug, U)
    assert torch.equal(g.replay(), Ug)
    assert prob.device_status() == B.BS_OK


def test_graph_replay_equals_direct_solve_network(B):
    p = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=256, P=8, fine_steps=32, coarse_steps=1)
    prob = B.Problem(p)
    m = B.PinnModel([2, 64, 64, 1], [0.0, 0.0], [4.0, 1.0], seed=3)
    for prec in (B.FP64, B.BF16):
        U, norms, stats, rc = prob.parareal_solve(B.COARSE_PINN, model=m, prec=prec, tol=1e-8)
        g = B.SolveGraph(prob, B.COARSE_PINN, model=m, prec=prec, tol=1e-8)
        g.U.zero_()
        assert torch.equal(g.replay(), U)
        # reading (A): k = P iterations reproduce serial fine
        assert stats[0]["iterations"] <= p["P"]
    Uf = prob.serial_fine()
    if stats[0]["iterations"] == p["P"]:
        assert torch.equal(U, Uf)
