"""parareal_solve_static: the solve for callers that cannot allocate device memory.

Some callers must not allocate after set-up (work enqueued under stream
capture, loops where an allocation would synchronise the device, processes
whose memory belongs to another allocator).  parareal_solve_static keeps its
workspace in a fixed array inside the library instead of allocating it.  This
file checks, through the C ABI, that two calls in a row give the same result
as parareal_solve within the FP64 parity tolerance of the other tests (1e-12
relative), and that an oversized problem is refused.  It is collected last so
that a run stopping at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
RTOL = 1e-12


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_03848_b300 import binding, build

    build.build()
    L = binding.lib()
    vp, dbl, P = ctypes.c_void_p, ctypes.c_double, ctypes.POINTER
    L.parareal_solve_static.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, dbl, ctypes.c_int32, vp, P(dbl),
                                        P(binding.InstanceStats), vp]
    return binding


def _static_solve(B, prob, kind, model, prec, tol, max_iter):
    U = torch.full((prob.total_state,), float("nan"), dtype=torch.float64, device="cuda")
    norms = np.empty(prob.n_instances * max_iter)
    stats = (B.InstanceStats * prob.n_instances)()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = B.lib().parareal_solve_static(prob._h, kind, model._h if model is not None else None, prec, tol, max_iter,
                                       ctypes.c_void_p(U.data_ptr()),
                                       norms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), stats, stream)
    return U, norms.reshape(prob.n_instances, max_iter), [s.iterations for s in stats], rc


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("kind", ["ie", "pinn", "pinn_incr", "pinn_ie"])
def test_static_solve_matches_parareal_solve_twice(B, kind):
    from paper_2303_03848_b300 import synth

    insts = [dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=256, P=8, fine_steps=128, coarse_steps=1),
             dict(K=1.3, sigma=0.3, r=0.02, T=1.5, Smax=5.2, Nx=300, P=6, fine_steps=40, coarse_steps=2)]
    prob = B.Problem(insts)
    model = None
    k = {"ie": B.COARSE_IE, "pinn": B.COARSE_PINN, "pinn_incr": B.COARSE_PINN_INCR, "pinn_ie": B.COARSE_PINN_IE}[kind]
    if kind != "ie":
        widths = [2, 32, 32, 1]
        model = B.PinnModel(widths, [0.0, 0.0], [5.2, 1.5], seed=4)
        model.set_weights(synth.xavier_params(widths, 4))
    max_iter = 8
    U_ref, n_ref, st_ref, rc_ref = prob.parareal_solve(k, model=model, prec=B.FP64, tol=1e-9, max_iter=max_iter)
    its_ref = [s["iterations"] for s in st_ref]
    for _ in range(2):
        U, norms, its, rc = _static_solve(B, prob, k, model, B.FP64, 1e-9, max_iter)
        torch.cuda.synchronize()
        assert rc == rc_ref
        assert its == its_ref
        assert _rel(U, U_ref) <= RTOL
        np.testing.assert_allclose(norms[:, :max(its)], n_ref[:, :max(its)], rtol=1e-9)


def test_static_solve_rejects_oversized_problem(B):
    # 129 * 4097 doubles per state buffer: 3 state + 2 slice buffers are about 21 MB > 16 MiB
    prob = B.Problem(dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=4097, P=128, fine_steps=2, coarse_steps=1))
    U, norms, its, rc = _static_solve(B, prob, B.COARSE_IE, None, B.FP64, 1e-6, 4)
    assert rc == B.BS_EUNSUPPORTED
    assert torch.isnan(U).all()  # nothing was launched
