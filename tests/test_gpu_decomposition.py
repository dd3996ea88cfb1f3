"""Single-system decomposition over ranks (sec. 3.2; Algorithm 1 steps 4-6),
run as two processes on the GPU with a gloo process group (the pool's boxes
have one GPU; both ranks share it, and no kernel of one waits on the other).

Each rank draws the modes itself from the shared Philox key (rbsog_modes),
computes the partial structure factors of its slab of atoms
(rbsog_structure_factor), the partials are summed by one all-reduce of 2 nD
doubles, and each rank computes the long-range forces on its own atoms and
the estimators from the summed rho (rbsog_longrange_force), with no further
exchange.  Rank 0 checks that the sampled modes are those of the oracle (bit
for bit) and identical on both ranks, and that rho, the forces on every atom
and the estimators equal the oracle's for the whole system (FP64 build:
1e-12; FP32 build: rho 2e-6 of sum |q|, forces 1e-5 relative RMS, estimators
1e-6)."""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, prec):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import workloads as W
    from oracle import oracle as O
    from paper_2602_23582_gb300 import rbsog as R

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    dev = torch.device("cuda:0")
    s = W.water(n_mol=1500, L=36.0, lattice=12, seed=12)
    L = s.box
    p = R.rbsog_default_params(10.0, precision=prec, P=100)
    step, rng_id = 5, 7
    md = R.rbsog_modes(p, L, rng_id, step)                      # the same on every rank
    D, cr, cnr, (Sr, Snr) = md["D"], md["cr"], md["cnr"], md["S"]
    # this rank's slab: atoms with wrapped z in [rank L/world, (rank + 1) L/world)
    z = np.mod(s.pos[:, 2], L[2])
    mine = np.nonzero((z >= rank * L[2] / world) & (z < (rank + 1) * L[2] / world))[0]
    r = torch.tensor(s.pos[mine], device=dev)
    q = torch.tensor(s.q[mine], device=dev)
    m = torch.tensor(D, device=dev)
    nD = len(D)
    rho = torch.zeros(2 * nD, dtype=torch.float64, device=dev)
    work = torch.zeros(R.rbsog_structure_factor_workspace(max(len(mine), 1), nD), dtype=torch.uint8, device=dev)
    R.rbsog_structure_factor(r, q, L, m, rho, work, precision=prec)
    # the one exchange of the long-range part: sum rho over the ranks
    rho_h = rho.cpu()
    dist.all_reduce(rho_h, op=dist.ReduceOp.SUM)
    rho_tot = rho_h.to(dev)
    F = torch.zeros((len(mine), 3), dtype=torch.float64, device=dev)
    w2 = torch.zeros(R.rbsog_longrange_force_workspace(nD), dtype=torch.uint8, device=dev)
    U, Wnr = R.rbsog_longrange_force(r, q, L, m, torch.tensor(cr, device=dev), torch.tensor(cnr, device=dev),
                                     rho_tot, p.P, Sr, Snr, p.ke, F, w2, precision=prec)
    # gather to rank 0 (for checking only)
    out = [None] * world
    dist.all_gather_object(out, dict(idx=mine, F=F.cpu().numpy(), D=D, cr=cr, cnr=cnr, U=U, Wnr=Wnr,
                                     rho=rho_h.numpy()))
    dist.destroy_process_group()
    if rank != 0:
        return
    for o in out[1:]:
        assert np.array_equal(o["D"], D) and np.array_equal(o["cr"], cr) and np.array_equal(o["cnr"], cnr)
    op = O.Params.row2(P=100, seed=int(p.seed), sysid=rng_id)
    mr, mn, _ = O.sample_modes(L, op, step)
    Do, cro, cnro = O.distinct(mr, mn)
    assert np.array_equal(D, Do) and np.array_equal(cr, cro) and np.array_equal(cnr, cnro)
    w, sg, wt, st = O.sog_terms(p.b, p.sigma, p.omega, p.M)
    Hr, Hnr, *_ = O.normalizers(L, wt, st)
    assert abs(Sr - Hr.sum()) < 1e-13 * Hr.sum() and abs(Snr - Hnr.sum()) < 1e-13 * Hnr.sum()
    Fo, Uo, Wro, Wnro, rho_o = O.rb_longrange(s.pos, s.q, L, p.P, Do, cro, cnro, Hr.sum(), Hnr.sum(), ke=p.ke)
    Fg = np.zeros_like(Fo)
    for o in out:
        Fg[o["idx"]] = o["F"]
    g = out[0]["rho"]
    scale = float(np.abs(s.q).sum())
    tol_rho, tol_f, tol_e = (1e-12, 1e-12, 1e-12) if prec == R.RBSOG_FP64 else (2e-6, 1e-5, 1e-6)
    assert np.abs((g[0::2] + 1j * g[1::2]) - rho_o).max() < tol_rho * scale
    assert np.linalg.norm(Fg - Fo) / np.linalg.norm(Fo) < tol_f
    assert abs(U - Uo) <= tol_e * abs(Uo)
    assert np.linalg.norm(Wnr - Wnro) <= tol_e * np.linalg.norm(Wnro)


@pytest.mark.parametrize("prec", [0, 1])
def test_two_rank_slab_decomposition_matches_oracle(prec):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(2, _free_port(), prec), nprocs=2, join=True)
