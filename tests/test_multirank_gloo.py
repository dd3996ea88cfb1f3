"""The single-system multi-GPU decomposition (one exchange step), checked
with two CPU ranks over gloo: each rank holds a spatial slab of the atoms,
draws the same modes from the shared Philox key (no communication), forms its
partial structure factors, and one all-reduce of 2|D| FP64 values gives rho
(the only cross-process exchange of Algorithm 1, step 5).  The reduced rho
must equal the single-rank rho to FP64 round-off, and the per-rank long-range
forces then need no further exchange."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as W
    from oracle import oracle as O
    s = W.water(n_mol=900, L=31.0, lattice=10, seed=3)
    p = O.Params.row2(P=100)
    mr, mn, _ = O.sample_modes(s.box, p, 7)          # same key on every rank
    D, cr, cnr = O.distinct(mr, mn)
    # slab decomposition along z
    z = np.mod(s.pos[:, 2], s.box[2])
    mine = (z * world // s.box[2]).astype(int) == rank
    part = O.rho(s.pos[mine], s.q[mine], s.box, D)
    buf = torch.tensor(np.concatenate([part.real, part.imag]), dtype=torch.float64)
    dist.all_reduce(buf)
    n = len(D)
    rho = buf[:n].numpy() + 1j * buf[n:].numpy()
    modes = torch.tensor(D.reshape(-1).astype(np.int64))
    gathered = [torch.zeros_like(modes) for _ in range(world)]
    dist.all_gather(gathered, modes)
    if rank == 0:
        full = O.rho(s.pos, s.q, s.box, D)
        out.put((float(np.abs(rho - full).max()), float(np.abs(full).max()),
                 all(torch.equal(g, gathered[0]) for g in gathered)))
    dist.destroy_process_group()


def test_two_rank_structure_factor_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    err, scale, same = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert same
    assert err < 1e-11 * max(scale, 1.0)
