"""The C-ABI library loads, exports what the header declares, and rejects bad
arguments on the host before touching the GPU (CPU only: no compute calls)."""
import ctypes

import numpy as np
import pytest

from paper_2303_03848_b300 import binding as B
from paper_2303_03848_b300 import build as BUILD


@pytest.fixture(scope="module")
def L():
    BUILD.build()
    return B.lib()


def test_exports_every_declared_symbol(L):
    names = B.header_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n


def test_status_strings_and_version(L):
    assert B.status_string(B.BS_OK) == "ok"
    assert "not converged" in B.status_string(B.BS_NOT_CONVERGED)
    assert B.status_string(999) == "unknown status"
    assert B.version().startswith("bsparareal")


@pytest.mark.parametrize("bad", [
    dict(Nx=4), dict(P=0), dict(fine_steps=0), dict(coarse_steps=0), dict(K=0.0), dict(sigma=-0.1), dict(r=-0.01),
    dict(T=0.0), dict(Smax=0.5), dict(Smax=float("nan")), dict(K=float("inf")),
])
def test_problem_init_rejects_bad_parameters(L, bad):
    p = B.params()
    p.update(bad)
    for tuned in (False, True):
        with pytest.raises(B.BsError) as e:
            B.Problem(p, tuned=tuned)
        assert e.value.code == B.BS_EINVAL


def test_problem_init_rejects_oversized_grid(L):
    with pytest.raises(B.BsError) as e:
        B.Problem(B.params(Nx=65538))
    assert e.value.code == B.BS_EUNSUPPORTED


def test_null_arguments_rejected(L):
    h = ctypes.c_void_p()
    assert L.bs_problem_init(None, 1, ctypes.byref(h)) == B.BS_EINVAL
    p = B.BsParams(1.0, 0.2, 0.05, 1.0, 4.0, 256, 8, 128, 1)
    assert L.bs_problem_init(ctypes.byref(p), 0, ctypes.byref(h)) == B.BS_EINVAL
    assert L.fine_propagate(None, None, None, None, None) == B.BS_EINVAL
    assert L.serial_fine(None, None, None) == B.BS_EINVAL
    assert L.parareal_solve(None, 0, None, 0, 1e-6, 4, None, None, None, None) == B.BS_EINVAL
    assert L.pinn_eval(None, 0, None, 1, None, None, None) == B.BS_EINVAL
    assert L.bs_problem_device_status(None, None) == B.BS_EINVAL
    assert L.bs_problem_slices_per_cta(None, 0, None) == B.BS_EINVAL
    assert L.bs_problem_init_tuned(None, 1, ctypes.byref(h), None, 0, None) == B.BS_EINVAL
    assert L.bs_problem_init_tuned(ctypes.byref(p), 1, ctypes.byref(h), None, 4, None) == B.BS_EINVAL
    assert L.bs_problem_init_partitioned(None, 1, None, 0, ctypes.byref(h)) == B.BS_EINVAL
    tun = (B.Tuning * 1)(B.Tuning(512, 2, 4, 1, 1, 0.0, 1))
    assert L.bs_problem_init_partitioned(ctypes.byref(p), 1, tun, 1, ctypes.byref(h)) == B.BS_EINVAL  # no Nx=256
    tun[0] = B.Tuning(256, 3, 4, 1, 1, 0.0, 1)
    assert L.bs_problem_init_partitioned(ctypes.byref(p), 1, tun, 1, ctypes.byref(h)) == B.BS_EUNSUPPORTED
    s = ctypes.c_int32()
    assert L.bs_wait_probe(0, 0, ctypes.byref(s)) == B.BS_EINVAL  # limit out of range
    assert L.bs_wait_probe(0, 1 << 35, ctypes.byref(s)) == B.BS_EINVAL
    assert L.bs_wait_probe(0, 1000, None) == B.BS_EINVAL
    pp = B.BsParams(1.0, 0.2, 0.05, 1.0, 4.0, 5, 1, 1, 1)
    assert L.pinn_loss_grad_data(None, None, None, None, 1, ctypes.byref(pp), 0.0, 0, None, None, None) == B.BS_EINVAL
    assert L.pinn_train_step_data(None, None, None, None, 1, ctypes.byref(pp), 0.0, 0, 1e-3, None, None,
                                  None) == B.BS_EINVAL
    assert L.pinn_get_state(None, None, None, None, None) == B.BS_EINVAL
    assert L.pinn_set_state(None, None, None, None, 0) == B.BS_EINVAL
    L.bs_problem_destroy(None)
    L.pinn_destroy(None)


def test_checkpoint_file_round_trip(tmp_path):
    # the network checkpoint format: header and three FP64 arrays, exact
    rng = np.random.default_rng(3)
    widths, lo, hi = [5, 16, 16, 1], [0.0, 0.0, 0.1, 0.0, 0.5], [8.0, 2.0, 0.5, 0.08, 2.0]
    n = 5 * 16 + 16 + 16 * 16 + 16 + 16 + 1
    th, m1, m2 = rng.standard_normal(n), rng.standard_normal(n), rng.random(n)
    path = tmp_path / "net.ckpt"
    B.write_checkpoint(path, widths, lo, hi, 17, th, m1, m2)
    c = B.read_checkpoint(path)
    assert c["widths"] == widths and c["lo"] == lo and c["hi"] == hi and c["step"] == 17
    for k, a in (("theta", th), ("mom1", m1), ("mom2", m2)):
        assert np.array_equal(c[k], a)
    raw = path.read_bytes()
    (tmp_path / "cut").write_bytes(raw[:-8])
    with pytest.raises(ValueError):
        B.read_checkpoint(tmp_path / "cut")
    (tmp_path / "magic").write_bytes(b"X" + raw[1:])
    with pytest.raises(ValueError):
        B.read_checkpoint(tmp_path / "magic")
    with pytest.raises(ValueError):
        B.write_checkpoint(path, widths, lo, hi, 0, th, m1[:-1], m2)


@pytest.mark.parametrize("widths", [[3, 8, 1], [2, 8, 2], [2, 300, 1], [2, 0, 1]])
def test_pinn_create_rejects_bad_widths(L, widths):
    with pytest.raises(B.BsError) as e:
        B.PinnModel(widths, [0.0] * widths[0], [1.0] * widths[0])
    assert e.value.code == B.BS_EINVAL


def test_pinn_create_rejects_empty_box(L):
    with pytest.raises(B.BsError) as e:
        B.PinnModel([2, 8, 1], [0.0, 1.0], [4.0, 1.0])
    assert e.value.code == B.BS_EINVAL


def test_struct_layout_matches_header(L):
    # bs_params: 5 doubles then 4 int32 = 56 bytes; bs_instance_stats: 16 bytes
    assert ctypes.sizeof(B.BsParams) == 56
    assert ctypes.sizeof(B.InstanceStats) == 16
    assert ctypes.sizeof(B.Tuning) == 28
    assert B.BsParams.Nx.offset == 40


def test_splitmix_generator_matches_published_vectors():
    # SplitMix64 reference outputs for state 1234567 (first five draws), from the
    # generator's published definition (Steele, Lea, Flood 2014; also the seeding
    # generator of xoshiro): 6457827717110365317, 3203168211198807973,
    # 9817491932198370423, 4593380528125082431, 16408922859458223821
    from paper_2303_03848_b300 import synth

    out = synth.splitmix64(1234567, np.arange(5, dtype=np.uint64))
    assert [int(v) for v in out] == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                                     4593380528125082431, 16408922859458223821]


def test_training_batch_checks_run_before_any_launch():
    # lengths and kinds are checked on the host by the binding before the C ABI
    # is called (the library cannot see device lengths): CPU tensors suffice
    torch = pytest.importorskip("torch")
    X = torch.zeros(10, 2, dtype=torch.float64)
    kind = torch.zeros(10, dtype=torch.int8)
    y = torch.zeros(10, dtype=torch.float64)
    B.check_loss_inputs(X, kind)
    B.check_loss_inputs(X, kind, y)
    with pytest.raises(ValueError, match="kind must hold"):
        B.check_loss_inputs(X, kind[:9])
    with pytest.raises(ValueError, match="y must hold"):
        B.check_loss_inputs(X, kind, y[:9])
    k4 = kind.clone()
    k4[3] = 4
    B.check_loss_inputs(X, k4, y)  # a data point with its value
    with pytest.raises(ValueError, match="0..3"):
        B.check_loss_inputs(X, k4)  # a data point without values
    for bad in (5, -1, 7):
        kb = kind.clone()
        kb[7] = bad
        with pytest.raises(ValueError, match="kind values"):
            B.check_loss_inputs(X, kb, y)
    # a checked tensor modified in place is checked again
    kind[2] = 9
    with pytest.raises(ValueError):
        B.check_loss_inputs(X, kind)
