"""Served path on the GPU: a pool of slots loaded and emptied at run time, and
the request loop on top of it.  Every system must come out bit-identical to
the same system run alone in a plain context with the same cell size and
Philox key (its counter starts at 0 on admission and advances only with its
own steps), whatever else shares the launches."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23582_gb300 import rbsog as R  # noqa: E402


def _systems():
    s = [W.electrolyte(n_ions=600, L=31.0, seed=11), W.water(n_mol=1500, L=36.0, lattice=12, seed=12),
         W.random_charges(n=777, box=(32.0, 35.0, 38.0), seed=13, min_dist=2.4, lj=True),
         W.electrolyte(n_ions=900, L=33.0, seed=14)]
    for k, x in enumerate(s):
        x.rng_id = 200 + k
    return s


def _alone(s, prec, nsteps):
    ctx = R.Context([s], R.rbsog_default_params(10.0, precision=prec, cell_sub=2))
    res = ctx.run(nsteps)
    r, v = ctx.positions(), ctx.velocities()
    ctx.close()
    return r, v, res[0]


def _caps(n=4):
    return [R.slot_caps(max_atoms=5000, max_box=(40.0, 40.0, 40.0), max_types=4) for _ in range(n)]


@pytest.mark.parametrize("prec", [R.RBSOG_FP32, R.RBSOG_FP64])
def test_pool_matches_plain_contexts(prec):
    systems = _systems()[:3]
    pool = R.Pool(_caps(4), R.rbsog_default_params(10.0, precision=prec))
    for slot, s in zip((0, 2, 3), systems):          # slot 1 stays empty
        pool.load(slot, s, index=s.rng_id)
    pool.prime()
    pool.run(5)
    state, steps, err = pool.state()
    assert list(state) == [1, 0, 1, 1] and list(steps[[0, 2, 3]]) == [5, 5, 5] and not err.any()
    for slot, s in zip((0, 2, 3), systems):
        r, v, res = pool.unload(slot)
        ra, va, resa = _alone(s, prec, 5)
        assert np.array_equal(r, ra), (prec, slot)
        assert np.array_equal(v, va), (prec, slot)
        assert np.array_equal(res["pressure"], resa["pressure"]), (prec, slot)
        assert res["coul"] == resa["coul"] and res["step"] == 5
    pool.close()


def test_pool_step_limits_and_slot_reuse():
    a, b, c = _systems()[:3]
    pool = R.Pool(_caps(2), R.rbsog_default_params(10.0))
    pool.load(0, a, nsteps=3, index=a.rng_id)
    pool.load(1, b, nsteps=6, index=b.rng_id)
    pool.prime()
    pool.run(6)                                       # a stops (frozen) after its 3 steps
    state, steps, _ = pool.state()
    assert list(state) == [2, 2] and list(steps) == [3, 6]
    ra, _, _ = pool.unload(0)
    assert np.array_equal(ra, _alone(a, R.RBSOG_FP32, 3)[0])
    pool.load(0, c, nsteps=2, index=c.rng_id)         # reuse the slot while b is finished
    pool.prime()
    pool.run(2)
    rc, _, resc = pool.unload(0)
    assert np.array_equal(rc, _alone(c, R.RBSOG_FP32, 2)[0]) and resc["step"] == 2
    rb, _, _ = pool.unload(1)
    assert np.array_equal(rb, _alone(b, R.RBSOG_FP32, 6)[0])
    pool.close()


def test_pool_rejects_what_does_not_fit():
    pool = R.Pool([R.slot_caps(max_atoms=700, max_box=35.0)], R.rbsog_default_params(10.0))
    big = W.electrolyte(n_ions=900, L=33.0, seed=14)
    with pytest.raises(R.RbsogError):
        pool.load(0, big)
    wide = W.electrolyte(n_ions=600, L=45.0, seed=15)   # box beyond the slot's cell grid
    with pytest.raises(R.RbsogError):
        pool.load(0, wide)
    pool.close()


def test_server_continuous_batching_matches_alone():
    systems = _systems()
    nsteps = [7, 3, 5, 4]
    srv = R.Server(_caps(2), R.rbsog_default_params(10.0), hbm_fraction=0.5)
    assert srv.slots == 2
    tickets = [srv.submit(systems[k], nsteps[k], rng_id=systems[k].rng_id) for k in range(3)]
    running, queued = srv.pump(2)                     # two admitted, one waits
    assert running == 2 and queued == 1
    tickets.append(srv.submit(systems[3], nsteps[3], rng_id=systems[3].rng_id))   # arrives mid-run
    for _ in range(40):
        running, queued = srv.pump(2)
        if running == 0 and queued == 0:
            break
    srv.pump(0)                                       # retire the last ones
    for k, t in enumerate(tickets):
        out = srv.result(t)
        assert out is not None, k
        r, v, res = out
        assert res["status"] == 0, k
        ra, va, resa = _alone(systems[k], R.RBSOG_FP32, nsteps[k])
        assert np.array_equal(r, ra), k
        assert np.array_equal(v, va), k
        assert np.array_equal(res["pressure"], resa["pressure"]), k
        assert res["step"] == nsteps[k]
    st = srv.stats()
    assert st["steps"] > 0 and st["p99_ms"] >= st["p50_ms"] > 0 and st["atom_steps_per_s"] > 0
    assert st["failed"] == 0
    srv.close()
