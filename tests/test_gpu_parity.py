"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
identical seeded inputs and identical Philox counters.

Bars (from the contract of this build):
* cell membership and sampled mode indices: bit-exact;
* FP64 build: forces, virial/pressure (and each of its parts) and energies
  within 1e-12 relative;
* FP32 build (FP32 math, FP64 accumulation): forces within 1e-5 relative RMS,
  pressure tensor (Frobenius) and energies within 1e-6 relative;
* batched path: each system bit-identical alone and in a mix.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23582_gb300 import rbsog as R  # noqa: E402


def _ctx(systems, prec, **kw):
    p = R.rbsog_default_params(kw.pop("rc", 10.0), precision=prec, **kw)
    return R.Context(systems, p), p


def _oracle_params(p, sysid=0):
    # the binding keys system k with rng_id = k unless the system sets one
    return O.Params(rc=p.rc, b=p.b, sigma=p.sigma, omega=p.omega, ke=p.ke, M=p.M, ME=p.M_energy,
                    P=p.P, kind=p.sampler, seed=int(p.seed), sysid=sysid)


# FP64 build bar (forces, pressure tensor and its parts, energies), relative
TOL64 = 1e-12


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


SYSTEMS = {
    "electrolyte": lambda: W.electrolyte(n_ions=1000, L=30.0, seed=1),
    "water_small": lambda: W.water(n_mol=1200, L=33.0, lattice=11, seed=2),
    "ragged": lambda: W.random_charges(n=1333, box=(31.0, 34.5, 40.25), seed=5, min_dist=1.6, lj=True),
    # a few atoms per cell: with cells of r_c/2, pairs of cells of one x-row
    # become one list-build item
    "sparse_rows": lambda: W.random_charges(n=400, box=(80.0, 30.0, 31.0), seed=7, min_dist=2.0, lj=True),
}


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("sub", [1, 2])
def test_cells_bit_exact(name, sub):
    s = SYSTEMS[name]()
    ctx, p = _ctx([s], R.RBSOG_FP64, cell_sub=sub)
    nc, cell = ctx.cells(0)
    onc, ocell = O.cell_bin(s.pos, s.box, p.rc, sub)
    assert np.array_equal(nc, onc)
    assert np.array_equal(cell, ocell)
    ctx.close()


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("box", [(30.0, 30.0, 30.0), (31.0, 44.0, 66.88), (110.85, 110.85, 110.85)])
def test_modes_bit_exact(kind, box):
    s = W.random_charges(n=64, box=box, seed=3, min_dist=1.5)
    ctx, p = _ctx([s], R.RBSOG_FP64, sampler=kind, P=100)
    op = _oracle_params(p)
    for step in (1, 2, 17):
        ctx.step(step)
        g = ctx.modes(0)
        mr, mn, _ = O.sample_modes(s.box, op, step)
        assert np.array_equal(g["mr"], mr), (kind, box, step)
        assert np.array_equal(g["mnr"], mn), (kind, box, step)
        D, cr, cnr = O.distinct(mr, mn)
        assert np.array_equal(g["D"], D) and np.array_equal(g["cr"], cr) and np.array_equal(g["cnr"], cnr)
        w, sg, wt, st = O.sog_terms(p.b, p.sigma, p.omega, p.M)
        Hr, Hnr, *_ = O.normalizers(s.box, wt, st)
        assert abs(g["Sr"] - Hr.sum()) < 1e-13 * Hr.sum()
        assert abs(g["Snr"] - Hnr.sum()) < 1e-13 * Hnr.sum()
    ctx.close()


def _compare_eval(s, prec, step=5, **kw):
    ctx, p = _ctx([s], prec, **kw)
    F, res = ctx.step(step)
    ref = O.force_eval(s, _oracle_params(p), step)
    r = res[0]
    ctx.close()
    return F, r, ref


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("sub", [1, 2])
def test_eval_fp64_matches_oracle(name, sub):
    s = SYSTEMS[name]()
    F, r, ref = _compare_eval(s, R.RBSOG_FP64, cell_sub=sub)
    assert _rel(F, ref["F"]) < TOL64
    assert _rel(r["virial"], ref["W"]) < TOL64
    assert _rel(r["virial_coul_short"], ref["W_parts"][0]) < TOL64
    assert _rel(r["virial_long_r"], ref["W_parts"][1]) < TOL64
    assert _rel(r["virial_long_nr"], ref["W_parts"][2]) < TOL64
    assert _rel(r["virial_lj"], ref["W_parts"][3]) < TOL64
    assert _rel(r["virial_bonded"], ref["W_parts"][4]) < TOL64 or np.abs(ref["W_parts"][4]).max() == 0
    for k in ("coul_short", "coul_long", "coul_self", "lj", "bond", "angle"):
        assert abs(r[k] - ref[k]) <= TOL64 * max(abs(ref[k]), 1.0), k
    # the total Coulomb energy is a sum of parts that cancel (the self energy
    # is ~100x the total): its rounding error is set by the parts' magnitudes
    parts = sum(abs(ref[k]) for k in ("coul_short", "coul_long", "coul_self", "coul_excl"))
    assert abs(r["coul"] - ref["coul"]) <= TOL64 * parts
    assert r["n_distinct_modes"] == int(ref["n_distinct"])


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("sub", [1, 2])
def test_eval_fp32_matches_oracle(name, sub):
    # cell_sub 2 (cells of r_c/2, a dozen atoms each) makes the list build
    # take runs of several cells of one x-row per work item
    s = SYSTEMS[name]()
    F, r, ref = _compare_eval(s, R.RBSOG_FP32, cell_sub=sub)
    V = float(np.prod(s.box))
    assert _rel(F, ref["F"]) < 1e-5
    P_gpu = r["virial"] / V
    P_ref = ref["W"] / V
    assert _rel(P_gpu, P_ref) < 1e-6
    assert abs(r["coul"] - ref["coul"]) <= 1e-6 * abs(ref["coul"])
    assert abs(r["lj"] - ref["lj"]) <= 1e-6 * max(abs(ref["lj"]), 1.0)


def test_eval_fp32_run_items_wrapping_stencil():
    # cells of r_c/2 with five cells along x: a list-build item of two cells
    # spans six stencil columns, so its first and last column are one cell;
    # every atom must still see each neighbour cell once
    s = W.random_charges(n=300, box=(27.0, 40.0, 33.0), seed=17, min_dist=2.0, lj=True)
    F, r, ref = _compare_eval(s, R.RBSOG_FP32, cell_sub=2)
    assert _rel(F, ref["F"]) < 1e-5
    assert _rel(r["virial"], ref["W"]) < 1e-6
    assert abs(r["coul"] - ref["coul"]) <= 1e-6 * abs(ref["coul"])


def _last_forces(ctx, n):
    # forces of the last evaluation, from the state record (header, r, p, F, ...)
    state = R.rbsog_get_state(ctx.ctx)
    return np.frombuffer(state, np.float64, 3 * n, 16 + 48 * n).reshape(n, 3)


@pytest.mark.parametrize("name", ["electrolyte", "water_small"])
def test_skin_lists_match_oracle_after_npt_steps(name):
    # lists kept over NPT steps while the displacement bound holds: the last
    # step's forces and virial equal the oracle's at its positions and box
    import copy
    s = SYSTEMS[name]()
    ctx, p = _ctx([s], R.RBSOG_FP32, skin=1.0, thermo_every=0)
    res = ctx.run(40)[0]
    F = _last_forces(ctx, s.n)
    s2 = copy.copy(s)
    s2.pos = ctx.positions()
    s2.box = np.array(res["box"])
    ctx.close()
    # the context's first evaluation builds, then NPT steps rebuild only now and then
    assert 2 <= res["list_builds"] <= 30, res["list_builds"]
    ref = O.force_eval(s2, _oracle_params(p), int(res["step"]))
    assert _rel(F, ref["F"]) < 1e-5
    assert _rel(res["virial"], ref["W"]) < 1e-6
    assert abs(res["coul"] - ref["coul"]) <= 1e-6 * abs(ref["coul"])


@pytest.mark.parametrize("prec", [R.RBSOG_FP64, R.RBSOG_FP32])
@pytest.mark.parametrize("name", ["electrolyte", "water_small"])
def test_step_forces_matches_oracle(prec, name):
    # the force-only evaluation (rbsog_step_forces, the evaluation of an NPT
    # step, no energies): forces and virial against the oracle, at two step
    # counters through the same captured graph
    s = SYSTEMS[name]()
    ctx, p = _ctx([s], prec)
    out = {k: ctx.step_forces(k) for k in (5, 9)}
    ctx.close()
    tol_f, tol_w = (TOL64, TOL64) if prec == R.RBSOG_FP64 else (1e-5, 1e-6)
    for k, (F, W) in out.items():
        ref = O.force_eval(s, _oracle_params(p), k)
        assert _rel(F, ref["F"]) < tol_f, k
        assert _rel(W[0], ref["W"]) < tol_w, k


def test_fp64_trajectory_independent_of_energy_steps():
    # FP64 build: forces and the total virial are formed by the same
    # operations with and without energies (the two kernel variants may
    # round them differently where the compiler fuses a multiply-add), so the
    # trajectory depends on thermo_every only at the level of FP64 rounding
    s = SYSTEMS["water_small"]()
    out = []
    for every in (1, 0):
        ctx, _ = _ctx([s], R.RBSOG_FP64, thermo_every=every)
        R.rbsog_run_async(ctx.ctx, 12)
        R.rbsog_sync(ctx.ctx)
        out.append((ctx.positions(), ctx.run(0)[0]["box"]))
        ctx.close()
    assert _rel(out[0][0], out[1][0]) < 1e-12
    assert _rel(out[0][1], out[1][1]) < 1e-12


def _state_after_steps(ctx, n):
    # step counter, positions, forces and result record of the last step,
    # from the state record (header, r, p, F, per-system records, results)
    st = R.rbsog_get_state(ctx.ctx)
    step = int(np.frombuffer(st, np.uint64, 1, 0)[0])
    r = np.frombuffer(st, np.float64, 3 * n, 16).reshape(n, 3)
    F = np.frombuffer(st, np.float64, 3 * n, 16 + 48 * n).reshape(n, 3)
    red = np.frombuffer(st, np.float64, 64, len(st) - 8 * 64)
    W = red[9:15][[0, 3, 4, 3, 1, 5, 4, 5, 2]].reshape(3, 3)
    return step, r.copy(), F.copy(), W, red[52:55].copy()


@pytest.mark.parametrize("name", ["electrolyte", "water_small", "ragged"])
@pytest.mark.parametrize("sub", [1, 2])
def test_force_only_steps_match_oracle(name, sub):
    # steps without energies (box held: these boxes are near the stencil's
    # minimum and the compressing ones would leave it): the FP32 pair kernel forms the virial from
    # its force sums (x_i F_i per unit, (x_j + o) F_j per tile) instead of
    # pair by pair; the last step's forces and virial against the oracle at
    # its positions, box and step
    import copy
    s = SYSTEMS[name]()
    ctx, p = _ctx([s], R.RBSOG_FP32, cell_sub=sub, thermo_every=0, coupling=R.RBSOG_COUPLE_FIXED)
    R.rbsog_run_async(ctx.ctx, 6)
    R.rbsog_sync(ctx.ctx)
    step, r, F, Wg, box = _state_after_steps(ctx, s.n)
    ctx.close()
    s2 = copy.copy(s)
    s2.pos = r
    s2.box = box
    ref = O.force_eval(s2, _oracle_params(p), step)
    assert _rel(F, ref["F"]) < 1e-5
    assert _rel(Wg, ref["W"]) < 1e-6


def test_skin_lists_rebuilt_after_host_changes():
    s = SYSTEMS["water_small"]()
    ctx, p = _ctx([s], R.RBSOG_FP32, skin=1.5, thermo_every=0)
    b0 = ctx.run(1)[0]["list_builds"]
    b1 = ctx.run(1)[0]["list_builds"]
    assert b1 == b0                                  # a small step keeps the lists
    ctx.set_positions(ctx.positions())               # positions from the host: rebuilt
    b2 = ctx.run(1)[0]["list_builds"]
    assert b2 == b1 + 1
    R.rbsog_set_box(ctx.ctx, 0, ctx.run(0)[0]["box"])   # box from the host: rebuilt
    b3 = ctx.run(1)[0]["list_builds"]
    assert b3 == b2 + 1
    ctx.close()


def test_skin_lists_alone_equals_mixed():
    systems = [W.electrolyte(n_ions=600, L=31.0, seed=11), W.water(n_mol=1500, L=36.0, lattice=12, seed=12)]
    for k, s in enumerate(systems):
        s.rng_id = 300 + k
    mix, _ = _ctx(systems, R.RBSOG_FP32, cell_sub=2, skin=1.5)
    rm = mix.run(25)
    pos_m = mix.positions()
    mix.close()
    off = 0
    for k, s in enumerate(systems):
        alone, _ = _ctx([s], R.RBSOG_FP32, cell_sub=2, skin=1.5)
        ra = alone.run(25)
        assert np.array_equal(alone.positions(), pos_m[off:off + s.n]), k
        assert np.array_equal(ra[0]["pressure"], rm[k]["pressure"]), k
        assert ra[0]["list_builds"] == rm[k]["list_builds"] < 26, k
        alone.close()
        off += s.n


@pytest.mark.parametrize("prec", [R.RBSOG_FP64, R.RBSOG_FP32])
def test_eval_large_molecules_match_oracle(prec):
    # 15-site anions (32 springs and 105 excluded pairs each): the molecule
    # terms run one warp per molecule, its per-atom sums in shared memory
    s = W.ionic_liquid(n_pairs=100, seed=5)
    F, r, ref = _compare_eval(s, prec)
    tol_f, tol_w = (TOL64, TOL64) if prec == R.RBSOG_FP64 else (1e-5, 1e-6)
    assert _rel(F, ref["F"]) < tol_f
    assert _rel(r["virial"], ref["W"]) < tol_w
    assert abs(r["bond"] - ref["bond"]) <= tol_w * max(abs(ref["bond"]), 1.0)
    parts = sum(abs(ref[k]) for k in ("coul_short", "coul_long", "coul_self", "coul_excl"))
    assert abs(r["coul"] - ref["coul"]) <= tol_w * (parts if prec == R.RBSOG_FP64 else abs(ref["coul"]))


def test_eval_fp32_full_water_box():
    # the benchmark workload (10,000 molecules, 30,000 sites) at full size
    s = W.water()
    ctx, p = _ctx([s], R.RBSOG_FP32)
    F, res = ctx.step(11)
    ref = O.force_eval(s, _oracle_params(p), 11)
    ctx.close()
    assert _rel(F, ref["F"]) < 1e-5
    assert _rel(res[0]["virial"], ref["W"]) < 1e-6
    assert abs(res[0]["coul"] - ref["coul"]) <= 1e-6 * abs(ref["coul"])


def _npt_fp64_vs_oracle(s, coupling, nsteps=5):
    # FP64 NPT steps through the C ABI against the oracle's integrator from
    # the same start, with the box masses the library sets for the coupling
    rng = np.random.default_rng(0)
    s.vel = rng.normal(size=s.pos.shape) * np.sqrt(O.KB * 300.0 * O.FTM2V / s.mass[:, None])
    ctx, p = _ctx([s], R.RBSOG_FP64, P=50, dt=1.0, coupling=coupling)
    op = _oracle_params(p)
    # oracle state after the priming evaluation at counter 0
    out0 = O.force_eval(s, op, 0)
    st = dict(r=s.pos.copy(), p=s.vel * s.mass[:, None], L=s.box.copy(), ph=np.zeros(3),
              F=out0["F"], W=out0["W"].reshape(-1).copy())
    # box mass per group: M_g = n_g^2 V ftm2v / (kappa L_g^2 omega^2)
    kap = p.compressibility * O.NKTV2P
    om = 2 * np.pi / p.tau_box
    V = np.prod(s.box)
    if coupling == R.RBSOG_COUPLE_ISO:
        Mbox = (9.0 * V * O.FTM2V / (kap * s.box[0] ** 2 * om ** 2), 0.0, 0.0)
    else:
        Mbox = (4.0 * V * O.FTM2V / (kap * s.box[0] ** 2 * om ** 2),
                1.0 * V * O.FTM2V / (kap * s.box[2] ** 2 * om ** 2), 0.0)
    ig = O.Integ(dt=p.dt, T=p.T, Pext_atm=p.P_ext, gamma=p.gamma, gamma_box=p.gamma_box,
                 coupling=coupling, Mbox=Mbox)
    res = ctx.run(nsteps)
    O.npt_run(s, op, ig, st, 0, nsteps)
    r_gpu = ctx.positions()
    v_gpu = ctx.velocities()
    ctx.close()
    return res[0], r_gpu, v_gpu * s.mass[:, None], st


def test_npt_fp64_trajectory_matches_oracle():
    s = W.electrolyte(n_ions=300, L=30.0, seed=9)
    res, r_gpu, p_gpu, st = _npt_fp64_vs_oracle(s, R.RBSOG_COUPLE_ISO)
    assert np.allclose(res["box"], st["L"], rtol=1e-13, atol=0)
    d = r_gpu - st["r"]
    d -= st["L"] * np.rint(d / st["L"])
    assert np.abs(d).max() < 1e-10
    assert _rel(p_gpu, st["p"]) < 1e-10


def test_npt_fp64_semi_isotropic_trajectory_matches_oracle():
    # coupling 1: x = y share one box momentum, z its own (sec. 4.3, the
    # membrane's setting); an anisotropic box so that the groups differ
    s = W.random_charges(n=400, box=(31.0, 31.0, 37.0), seed=19, min_dist=2.2, lj=True)
    res, r_gpu, p_gpu, st = _npt_fp64_vs_oracle(s, R.RBSOG_COUPLE_SEMI_ISO)
    L = np.asarray(res["box"])
    assert L[0] == L[1]
    assert np.allclose(L, st["L"], rtol=1e-13, atol=0)
    # the z edge moved differently from x and y
    assert abs(L[2] / L[0] - 37.0 / 31.0) > 1e-9
    d = r_gpu - st["r"]
    d -= st["L"] * np.rint(d / st["L"])
    assert np.abs(d).max() < 1e-10
    assert _rel(p_gpu, st["p"]) < 1e-10


def test_batched_alone_equals_mixed():
    systems = [W.electrolyte(n_ions=600, L=31.0, seed=11), W.water(n_mol=1500, L=36.0, lattice=12, seed=12),
               W.random_charges(n=777, box=(32.0, 35.0, 38.0), seed=13, min_dist=2.4, lj=True)]
    for k, s in enumerate(systems):
        s.rng_id = 100 + k
    # one cell size for every context: the pair sums run over the same cells in
    # the same order only when the cell grids agree
    for prec in (R.RBSOG_FP32, R.RBSOG_FP64):
        mix, p = _ctx(systems, prec, cell_sub=2)
        Fm, rm = mix.step(4)
        rr = mix.run(3)
        pos_m = mix.positions()
        mix.close()
        off = 0
        for k, s in enumerate(systems):
            alone, _ = _ctx([s], prec, cell_sub=2)
            Fa, ra = alone.step(4)
            assert np.array_equal(Fa, Fm[off:off + s.n]), (prec, k)
            for key in ("coul", "lj", "bond", "angle"):
                assert ra[0][key] == rm[k][key], (prec, k, key)
            assert np.array_equal(ra[0]["virial"], rm[k]["virial"]), (prec, k)
            ra2 = alone.run(3)
            assert np.array_equal(alone.positions(), pos_m[off:off + s.n]), (prec, k)
            assert np.array_equal(ra2[0]["pressure"], rr[k]["pressure"]), (prec, k)
            alone.close()
            off += s.n


def test_structure_factor_stateless():
    s = W.water(n_mol=3000, L=45.0, lattice=15, seed=21)
    rng = np.random.default_rng(2)
    m = rng.integers(-9, 10, size=(57, 3)).astype(np.int32)
    m[np.all(m == 0, axis=1)] = [1, 0, 0]
    ref = O.rho(s.pos, s.q, s.box, m)
    dev = torch.device("cuda:0")
    r = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, device=dev)
    mt = torch.tensor(m, device=dev)
    for prec, tol in ((R.RBSOG_FP64, TOL64), (R.RBSOG_FP32, 2e-6)):
        rho = torch.zeros(2 * len(m), dtype=torch.float64, device=dev)
        nb = R.rbsog_structure_factor_workspace(s.n, len(m))
        work = torch.zeros(nb, dtype=torch.uint8, device=dev)
        R.rbsog_structure_factor(r, q, s.box, mt, rho, work, precision=prec)
        torch.cuda.synchronize()
        g = rho.cpu().numpy()
        g = g[0::2] + 1j * g[1::2]
        scale = np.abs(s.q).sum()
        assert np.abs(g - ref).max() < tol * scale, prec


def test_box_too_small_is_rejected():
    # below 2.5 r_c even cells of r_c/2 cannot hold the 5 x 5 x 5 stencil
    s = W.random_charges(n=50, box=(24.0, 30.0, 30.0), seed=1)
    p = R.rbsog_default_params(10.0)
    with pytest.raises(R.RbsogError) as e:
        R.Context([s], p)
    assert e.value.status == -3


def test_checkpoint_resume_is_bit_identical():
    s = W.electrolyte(n_ions=500, L=30.0, seed=4)
    ctx, p = _ctx([s], R.RBSOG_FP32, P=64)
    ctx.run(3)
    state = R.rbsog_get_state(ctx.ctx)
    ctx.run(4)
    a = ctx.positions()
    R.rbsog_set_state(ctx.ctx, state)
    ctx.run(4)
    b = ctx.positions()
    ctx.close()
    assert np.array_equal(a, b)


def test_run_is_deterministic():
    s = W.water(n_mol=1200, L=33.0, lattice=11, seed=2)
    out = []
    for _ in range(2):
        ctx, p = _ctx([s], R.RBSOG_FP32)
        ctx.run(5)
        out.append(ctx.positions())
        ctx.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("prec,tol", [(R.RBSOG_FP64, TOL64), (R.RBSOG_FP32, 2e-6)])
@pytest.mark.parametrize("name", ["electrolyte", "ragged"])
def test_shared_proposal_estimator_matches_oracle(name, prec, tol):
    # sec. 3.2: the radial samples of one evaluation reweighted for P^F,nr
    s = SYSTEMS[name]()
    ctx, p = _ctx([s], prec)
    ctx.step(5)
    g = ctx.virial_nr_shared()[0]
    ctx.close()
    op = _oracle_params(p)
    mr, mn, _ = O.sample_modes(s.box, op, 5)
    D, cr, cnr = O.distinct(mr, mn)
    rh = O.rho(s.pos, s.q, s.box, D)
    w, sg, wt, st = O.sog_terms(p.b, p.sigma, p.omega, p.M)
    Hr, Hnr, *_ = O.normalizers(s.box, wt, st)
    ref = O.nr_shared(s.box, op, D, cr, rh, Hr.sum())
    assert np.allclose(g, g.T, rtol=0, atol=0)
    assert _rel(g, ref) < tol


@pytest.mark.parametrize("prec", [R.RBSOG_FP32, R.RBSOG_FP64])
def test_overfull_cell_is_reported_without_pair_work(prec):
    # 2,500 atoms inside one 10 A cell (beyond the 2,048 a cell takes): the
    # scan flags the system, the pair kernels skip it (instead of walking the
    # cell's atoms from every work item) and the first evaluation reports
    # RBSOG_EOVERFLOW
    s = W.random_charges(n=3000, box=(30.0, 30.0, 30.0), seed=3, min_dist=0.3)
    rng = np.random.default_rng(3)
    s.pos[:2500] = rng.uniform(0.5, 4.5, (2500, 3))
    with pytest.raises(R.RbsogError) as e:
        R.Context([s], R.rbsog_default_params(10.0, precision=prec, cell_sub=1))
    assert e.value.status == -8


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("P", [1, 4096])
def test_batch_size_extremes_match_oracle(kind, P):
    # the smallest batch and the largest the library takes (4096 modes per
    # chain; the i.i.d. sampler then holds up to 8192 distinct modes): modes
    # bit-exact, FP64 forces and virial parts within 1e-12
    s = W.random_charges(n=300, box=(30.0, 31.0, 32.0), seed=13, min_dist=2.0, lj=True)
    ctx, p = _ctx([s], R.RBSOG_FP64, sampler=kind, P=P)
    op = _oracle_params(p)
    F, res = ctx.step(3)
    g = ctx.modes(0)
    ctx.close()
    mr, mn, _ = O.sample_modes(s.box, op, 3)
    assert np.array_equal(g["mr"], mr) and np.array_equal(g["mnr"], mn)
    ref = O.force_eval(s, op, 3)
    r = res[0]
    assert r["n_distinct_modes"] == int(ref["n_distinct"])
    assert _rel(F, ref["F"]) < TOL64
    assert _rel(r["virial_long_r"], ref["W_parts"][1]) < TOL64
    assert _rel(r["virial_long_nr"], ref["W_parts"][2]) < TOL64
    assert abs(r["coul_long"] - ref["coul_long"]) <= TOL64 * abs(ref["coul_long"])


@pytest.mark.parametrize("prec", [R.RBSOG_FP64, R.RBSOG_FP32])
def test_degenerate_systems_match_oracle(prec):
    # the method's degenerate cases: no charge at all (rho = 0: every
    # long-range term and the short-range Coulomb part vanish, LJ alone
    # remains), and two atoms whose single pair lies inside r_c (most cells
    # empty, one cluster each)
    zero = W.random_charges(n=200, box=(30.0, 30.0, 30.0), seed=31, min_dist=2.2, lj=True)
    zero.q = np.zeros_like(zero.q)
    two = W.random_charges(n=2, box=(30.0, 31.0, 32.0), seed=32, min_dist=2.0, lj=True)
    two.pos = np.array([[10.0, 11.0, 12.0], [13.5, 12.0, 14.0]])
    two.q = np.array([0.7, -0.7])
    for s in (zero, two):
        ctx, p = _ctx([s], prec)
        F, res = ctx.step(4)
        ctx.close()
        ref = O.force_eval(s, _oracle_params(p), 4)
        r = res[0]
        tol = TOL64 if prec == R.RBSOG_FP64 else 1e-5
        assert _rel(F, ref["F"]) < tol
        assert _rel(r["virial"], ref["W"]) < (TOL64 if prec == R.RBSOG_FP64 else 1e-6)
        if s is zero:
            for k in ("coul_short", "coul_long", "coul_excl"):
                assert r[k] == 0.0, k
            assert np.all(r["virial_long_r"] == 0.0) and np.all(r["virial_long_nr"] == 0.0)
            assert abs(r["lj"] - ref["lj"]) <= 1e-6 * abs(ref["lj"])
