"""The phi-slab decomposition of the step (tests/slabs.py) reproduces the
undecomposed oracle bit for bit: in-process with 2 and 4 slabs, and as two
gloo ranks that exchange their ghost planes with send/recv and reduce the
per-direction CFL minima with an all-reduce."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
from tests import slabs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _base():
    return O.default_params(n1=20, n2=16, n3=8, gam=13.0 / 9.0, r_out=40.0)


def _reference(steps):
    g = O.Grid(_base())
    g.init_torus(pert_amp=0.04, seed=5)
    P0, U0, t0, dt0 = g.get_state()
    for _ in range(steps):
        assert g.step() == 0
    return (P0, U0, t0, dt0), g.get_state()


@pytest.mark.parametrize("R", [2, 4])
def test_slabs_reproduce_the_undecomposed_step(R):
    (P0, U0, t0, dt0), (Pr, Ur, tr, dtr) = _reference(4)
    slabs = S.make_slabs(_base(), P0, U0, t0, dt0, R)
    for _ in range(4):
        assert S.step_slabs(slabs) == 0
    P, U, t, dt = S.gather(slabs)
    assert t == tr and dt == dtr
    assert np.array_equal(P, Pr)
    assert np.array_equal(U, Ur)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, steps, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from tests import slabs as S2
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    base = _base()
    g = O.Grid(base)
    g.init_torus(pert_amp=0.04, seed=5)
    P0, U0, t0, dt0 = g.get_state()
    Ps, Us = S2.split_state(P0, U0, world)[rank]
    mine = O.Grid(S2.slab_params(base, rank, world))
    mine.set_state(Ps, Us, t0, dt0)
    n3 = mine.shape[2]
    left, right = (rank - 1) % world, (rank + 1) % world

    def exchange(which):
        send_lo = torch.from_numpy(np.stack([mine.xplane(which, g_) for g_ in range(S2.NG)]))
        send_hi = torch.from_numpy(np.stack([mine.xplane(which, n3 - S2.NG + g_) for g_ in range(S2.NG)]))
        recv_lo, recv_hi = torch.empty_like(send_lo), torch.empty_like(send_hi)
        ops = [dist.P2POp(dist.isend, send_hi, right), dist.P2POp(dist.isend, send_lo, left),
               dist.P2POp(dist.irecv, recv_lo, left), dist.P2POp(dist.irecv, recv_hi, right)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for g_ in range(S2.NG):
            mine.set_xplane(which, -S2.NG + g_, recv_lo[g_].numpy())
            mine.set_xplane(which, n3 + g_, recv_hi[g_].numpy())

    exchange(0)
    for _ in range(steps):
        _, st = mine.stage0()
        assert st == 0
        d = torch.from_numpy(mine.last_dtd().copy())
        exchange(1)
        assert mine.stage1() == 0
        exchange(0)
        dist.all_reduce(d, op=dist.ReduceOp.MIN)
        mine.set_dt(O.combine_dt(d.numpy()))
    P, U, t, dt = mine.get_state()
    gathered = [None] * world
    dist.all_gather_object(gathered, (P, U, t, dt))
    dist.destroy_process_group()
    if rank == 0:
        out.put(gathered)


def test_two_gloo_ranks_reproduce_the_undecomposed_step():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, 3, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, (Pr, Ur, tr, dtr) = _reference(3)
    P = np.concatenate([g[0] for g in gathered], axis=3)
    U = np.concatenate([g[1] for g in gathered], axis=3)
    assert gathered[0][2] == tr and gathered[0][3] == dtr
    assert np.array_equal(P, Pr) and np.array_equal(U, Ur)
