"""Runtime pieces around the step: the launch-shape autotuner and the
bounded wait of a request loop (RBSOG_ETIMEOUT)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23582_gb300 import rbsog as R  # noqa: E402
from oracle import oracle as O  # noqa: E402


def test_autotune_times_every_shape_and_picks_the_fastest():
    s = W.water(n_mol=3000, L=44.7, lattice=15, seed=3)
    p = R.rbsog_default_params(10.0, precision=R.RBSOG_FP32, thermo_every=0)
    best, cands = R.rbsog_autotune(p, [s], nsteps=5)
    timed = [(a, b, t) for a, b, t in cands if t is not None]
    assert len(cands) == 8 and len(timed) == 8          # 44.7 A holds cells of r_c and of r_c / 2
    a, b, t = min(timed, key=lambda x: x[2])
    assert (best.cell_sub, best.cluster_cols) == (a, b)
    # the tuned shape gives the oracle's forces and pressure (FP32 bars)
    ctx = R.Context([s], best)
    F, res = ctx.step(4)
    ctx.close()
    ref = O.force_eval(s, O.Params.row2(P=best.P, seed=int(best.seed), sysid=0), 4)
    assert np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) < 1e-5
    assert np.linalg.norm(res[0]["virial"] - ref["W"]) / np.linalg.norm(ref["W"]) < 1e-6


@pytest.mark.parametrize("cols", [1, 2, 3, 4])
def test_every_cluster_shape_matches_oracle(cols):
    s = W.water(n_mol=1200, L=33.0, lattice=11, seed=2)
    p = R.rbsog_default_params(10.0, precision=R.RBSOG_FP32, cluster_cols=cols, cell_sub=1 if cols % 2 else 2)
    ctx = R.Context([s], p)
    F, res = ctx.step(6)
    ctx.close()
    ref = O.force_eval(s, O.Params.row2(P=p.P, seed=int(p.seed), sysid=0), 6)
    assert np.linalg.norm(F - ref["F"]) / np.linalg.norm(ref["F"]) < 1e-5
    assert np.linalg.norm(res[0]["virial"] - ref["W"]) / np.linalg.norm(ref["W"]) < 1e-6


def test_bounded_wait_times_out_then_completes():
    # 20 FP64 steps of the 30,000-site water box take about 0.1 s: a 1 ms
    # wait gives up (the steps keep running), a long one sees them finish
    s = W.water()
    p = R.rbsog_default_params(10.0, precision=R.RBSOG_FP64, thermo_every=0)
    ctx = R.Context([s], p)
    R.rbsog_run(ctx.ctx, 1)                            # graph built, flags clean
    R.rbsog_run_async(ctx.ctx, 20)
    assert R.rbsog_sync_timeout(ctx.ctx, 1.0) == -6    # RBSOG_ETIMEOUT
    assert "still run" in R.lib().rbsog_last_error(ctx.ctx).decode()
    assert R.rbsog_sync_timeout(ctx.ctx, 120000.0) == R.RBSOG_OK
    res = ctx.run(0)[0]
    assert res["step"] == 21 and np.all(np.isfinite(res["pressure"]))
    ctx.close()
