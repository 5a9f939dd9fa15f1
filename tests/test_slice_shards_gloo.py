"""Slice-sharded Parareal across processes on the CPU: world_size 2 and 3 gloo
ranks (rendezvous on 127.0.0.1), each owning a contiguous block of time slices
of one instance, run implicit-Euler-coarse Parareal (Eq. 7) with the oracle's
propagators.  Per iteration the fine propagation runs on every rank's own
slices at once; the serial coarse sweep is pipelined across the ranks with one
point-to-point message per rank boundary (the Nx-double state there, sent with
torch.distributed send/recv); the increment norm is an allreduce(max).  The
gathered result must equal the oracle's single-process Parareal bit for bit,
and the norms likewise.  No GPU.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _blocks(P, ws):
    cuts = [round(i * P / ws) for i in range(ws + 1)]
    return [(cuts[i], cuts[i + 1]) for i in range(ws)]


def _rank(rank, ws, port, cfg, iters, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import oracle as orc

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    p = orc.params(**cfg)
    P, Nx = cfg["P"], cfg["Nx"]
    a, b = _blocks(P, ws)[rank]
    U = np.zeros((P + 1, Nx))
    F = np.zeros((P, Nx))
    G = np.zeros((P, Nx))

    def recv_start(n):
        t = torch.empty(Nx, dtype=torch.float64)
        dist.recv(t, src=rank - 1)
        U[n] = t.numpy()

    def send_end(n):
        dist.send(torch.from_numpy(U[n].copy()), dst=rank + 1)

    def sweep(k):
        n0 = max(k, 0)
        if n0 >= b:
            return  # nothing of this block changes any more
        if n0 < a and rank > 0:
            recv_start(a)
        for n in range(max(n0, a), b):
            g_new = orc.coarse_ie(p, n, U[n])
            U[n + 1] = g_new if k < 0 else F[n] + (g_new - G[n])
            G[n] = g_new
        if rank < ws - 1:
            send_end(b)

    if rank == 0:
        U[0] = orc.payoff(p)
    sweep(-1)
    norms = []
    for k in range(iters):
        old = U.copy()
        for n in range(max(a, k), b):
            F[n] = orc.fine(p, n, U[n])
        sweep(k)
        e = 0.0
        for n in range(max(a, k), b):
            d = np.sqrt(np.sum((U[n + 1] - old[n + 1]) ** 2)) / np.sqrt(np.sum(U[n + 1] ** 2))
            e = max(e, d)
        t = torch.tensor([e], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        norms.append(float(t))
    # gather on rank 0: boundaries a+1 .. b of every rank (blocks of unequal size)
    if rank == 0:
        full = U.copy()
        for src, (lo, hi) in enumerate(_blocks(P, ws)):
            if src > 0:
                t = torch.empty((hi - lo, Nx), dtype=torch.float64)
                dist.recv(t, src=src)
                full[lo + 1:hi + 1] = t.numpy()
        out.put((full, norms))
    else:
        dist.send(torch.from_numpy(U[a + 1:b + 1].copy()), dst=0)
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_slice_sharded_parareal_across_gloo_ranks_equals_one_process(orc, ws):
    cfg = dict(K=1.0, sigma=0.2, r=0.05, T=1.0, Smax=4.0, Nx=64, P=7, fine_steps=16, coarse_steps=1)
    iters = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, cfg, iters, q)) for r in range(ws)]
    for pr in procs:
        pr.start()
    full, norms = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    U, rn, st = orc.parareal(orc.params(**cfg), orc.COARSE_IE, tol=0.0, max_iter=iters)
    np.testing.assert_array_equal(full, U)
    np.testing.assert_allclose(norms, rn, rtol=1e-15)
