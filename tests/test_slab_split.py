"""The single-mesh path sharded by slabs (the multi-GPU partition of the rhs:
contiguous element layers along z per rank, one face-trace exchange with the
two neighbouring ranks per rhs), emulated on CPU ranks with the oracle.

Each of two gloo ranks owns half of the element layers; it sends the trace
planes on its two boundary faces (the k = 0 nodes of its first layer to the
rank below, the k = N nodes of its last layer to the rank above, periodic),
receives its neighbours' planes, and evaluates the oracle's rhs on its slab
extended by one ghost layer on each side whose nodes carry the received
traces (only the ghost's face nodes enter the slab's surface fluxes). The
gathered slab results equal the one-rank rhs bitwise. This covers the
exchange's host logic; no GPU collective is built (one GPU per box)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

D, N, NE = 3, 2, (3, 2, 4)
NP, P, NV = N + 1, (N + 1) ** 3, 5


def _state():
    from paper_2108_06476_gb300 import workloads as W
    return W.random_state(D, N, NE, seed=41)


def _layers(u):
    """u as [ez][ey][ex][v][node]"""
    return u.reshape(NE[2], NE[1], NE[0], NV, P)


def _plane(layer, k):
    """the nodes with z index k of every element of a layer: [ey][ex][v][j][i]"""
    return layer.reshape(NE[1], NE[0], NV, NP, NP, NP)[:, :, :, k].copy()


def _ghost(plane, k):
    """a ghost layer whose nodes carry the received trace plane at z index k
    (the other node planes repeat it, so the ghost state stays physical)"""
    g = np.empty((NE[1], NE[0], NV, NP, NP, NP))
    g[:] = plane[:, :, :, None]
    g[:, :, :, k] = plane
    return g.reshape(NE[1], NE[0], NV, P)


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2108_06476_gb300 import workloads as W
        lay = _layers(_state())
        per = NE[2] // world
        own = lay[rank * per:(rank + 1) * per]
        below, above = (rank - 1) % world, (rank + 1) % world
        # exchange: my first layer's k = 0 plane goes below (the face that rank
        # shares with me has my nodes as its right trace), my last layer's k = N
        # plane goes above; I receive the matching planes
        send_down = torch.from_numpy(_plane(own[0], 0))
        send_up = torch.from_numpy(_plane(own[-1], N))
        from_above = torch.empty_like(send_down)
        from_below = torch.empty_like(send_up)
        ops = [dist.P2POp(dist.isend, send_down, below), dist.P2POp(dist.isend, send_up, above),
               dist.P2POp(dist.irecv, from_above, above), dist.P2POp(dist.irecv, from_below, below)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        ghost_lo = _ghost(from_below.numpy(), N)
        ghost_hi = _ghost(from_above.numpy(), 0)
        ext = np.concatenate([ghost_lo[None], own, ghost_hi[None]]).reshape(-1)
        # the slab with its ghost layers as a mesh of per + 2 layers of the same
        # element width (the oracle wraps the ghosts onto each other; only the
        # owned layers are kept)
        h = 2.0 / NE[2]
        dom = np.array([-1.0, 1.0, -1.0, 1.0, 0.0, h * (per + 2)])
        n_ext = (NE[0], NE[1], per + 2)
        du = oracle.rhs(D, N, n_ext, dom, ext).reshape(per + 2, NE[1], NE[0], NV, P)[1:-1]
        parts = [torch.empty(per, NE[1], NE[0], NV, P, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(np.ascontiguousarray(du)))
        if rank == 0:
            np.save(out_path, torch.cat(parts).numpy())
        del W
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_slab_split_equals_one_rank_rhs(orc, tmp_path):
    from paper_2108_06476_gb300 import workloads as W
    out = str(tmp_path / "slabs.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out).reshape(-1)
    ref = orc.rhs(D, N, NE, W.box(D), _state())
    assert np.array_equal(got, ref)
