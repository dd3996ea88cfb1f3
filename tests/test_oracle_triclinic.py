"""Pins of the oracle's general-cell (triclinic) path.

For a cell h = [[Lx, xy, xz], [0, Ly, yz], [0, 0, Lz]] (cell vectors as
columns), k = 2 pi h^{-T} m (eq. Sr), the proposal m* = round(h^T u) with its
mass q(m*) (eq. proposal, App. D), the lattice sums H^r_l, H^nr_l (eqs. Sr,
Snr) and the estimators (eqs. P_approx_r, P_approx_nr, f_approx).

* q: for a diagonal h it equals the product of 1D erf differences; for a
  sheared h it sums to 1 over the lattice, is even in m, is converged in the
  number of quadrature nodes, and matches the frequencies of round(h^T u)
  drawn directly (chi-square);
* normalizers: Proposition 3.5 (real-space form) for a sheared h, and the
  continuum limit H^r_l -> 6 V w~_l;
* sampler: for a diagonal h every mode equals the orthorhombic sampler's;
  for a sheared h the exact start draws and the App. D chain follow P^r
  enumerated mode by mode, and acceptance stays above 75 %;
* estimators: unbiased against the all-modes sums (eqs. U_long, P_long,
  force_SOG) in a sheared cell;
* force evaluation and the fixed-cell integrator reduce to the orthorhombic
  ones for a diagonal h.
"""
import math

import numpy as np
import pytest
from scipy.special import erf, erfc

import workloads as W
from oracle import oracle as O

H_SHEAR = O.tilted_box((22.0, 23.0, 21.0), (5.0, -3.5, 4.0))


def _terms(p):
    return O.sog_terms(p.b, p.sigma, p.omega, p.M)


def _q_product(L, st0, m):
    # 1D masses of an axis-aligned Gaussian over the unit interval around m_a
    sig = 1.0 / (math.sqrt(2.0) * math.pi * st0)
    out = 1.0
    for a in range(3):
        lo, hi = (m[a] - 0.5) / L[a] / (math.sqrt(2) * sig), (m[a] + 0.5) / L[a] / (math.sqrt(2) * sig)
        if lo >= 0:
            v = 0.5 * (erfc(lo) - erfc(hi))
        elif hi <= 0:
            v = 0.5 * (erfc(-hi) - erfc(-lo))
        else:
            v = 0.5 * (erf(hi) - erf(lo))
        out *= v
    return out


def test_q_reduces_to_erf_product_for_a_diagonal_cell():
    p = O.Params.row2()
    st0 = _terms(p)[3][0]
    L = (20.0, 31.0, 66.88)
    h = np.diag(L)
    for m in [(0, 0, 1), (1, -2, 3), (3, 2, -5), (6, 0, 0), (0, 0, 12), (-4, 7, 9)]:
        a, b = O.tri_q(h, st0, m), _q_product(L, st0, m)
        assert abs(a / b - 1) < 1e-13, (m, a, b)


def test_q_is_a_normalised_even_converged_mass():
    p = O.Params.row2()
    st0 = _terms(p)[3][0]
    h = H_SHEAR
    R = 8
    tot = 0.0
    for mx in range(-R, R + 1):
        for my in range(-R - 4, R + 5):
            for mz in range(-R - 4, R + 5):
                tot += O.tri_q(h, st0, (mx, my, mz), 12)
    assert abs(tot - 1.0) < 1e-12, tot
    for m in [(1, 2, 3), (2, -3, 1), (0, 4, -2), (3, 3, 3)]:
        a = O.tri_q(h, st0, m)
        assert abs(O.tri_q(h, st0, [-x for x in m]) / a - 1) < 1e-13
        assert abs(O.tri_q(h, st0, m, 40) / a - 1) < 1e-13


def test_q_matches_direct_draws_of_the_proposal():
    # m* = round(h^T u), u_a ~ N(0, 1/(2 pi^2 s~0^2)), drawn with numpy
    p = O.Params.row2()
    st0 = _terms(p)[3][0]
    h = H_SHEAR
    rng = np.random.default_rng(5)
    n = 400_000
    u = rng.normal(0.0, 1.0 / (math.sqrt(2) * math.pi * st0), size=(n, 3))
    m = np.floor(u @ h + 0.5).astype(np.int64)        # (h^T u)_a = sum_b h_ba u_b
    keys, counts = np.unique(m, axis=0, return_counts=True)
    chi, dof = 0.0, 0
    for k, c in zip(keys, counts):
        e = n * O.tri_q(h, st0, k)
        if e < 50:
            continue
        chi += (c - e) ** 2 / e
        dof += 1
    assert dof > 20
    assert chi < dof + 5 * math.sqrt(2 * dof), (chi, dof)


def test_normalizers_of_a_sheared_cell_against_proposition_3_5():
    p = O.Params.row2()
    w, s, wt, st = _terms(p)
    c = O.TriCell(H_SHEAR, p)
    Hr, Hnr, mm = c.normalizers()
    # the real-space sums of Prop. 3.5 converge fast for the narrow Gaussians
    for ell in range(3):
        nmax = [int(math.ceil(st[ell] * math.sqrt(46) / 20.0)) + 3] * 3
        Pr, Pnr = O.normalizers_poisson(H_SHEAR, wt[ell:ell + 1], st[ell:ell + 1], nmax)
        assert abs(Pr[0] / Hr[ell] - 1) < 1e-11, ell
        assert abs(Pnr[0] / Hnr[ell] - 1) < 1e-11, ell


def test_normalizer_continuum_limit_of_a_sheared_cell():
    p = O.Params.row2(M=2)
    w, s, wt, st = _terms(p)
    h = O.tilted_box((160.0, 150.0, 170.0), (40.0, -30.0, 25.0))
    Hr, Hnr, _ = O.TriCell(h, p).normalizers()
    V = float(np.linalg.det(h))
    assert abs(Hr[0] / (6 * V * wt[0]) - 1) < 1e-12
    assert abs(Hnr[0] / (60 * V * wt[0]) - 1) < 1e-12


@pytest.mark.parametrize("L", [(30.0, 33.0, 27.0), (20.0, 20.0, 20.0)])
def test_sampler_reduces_to_the_orthorhombic_one(L):
    p = O.Params.row2(P=200)
    c = O.TriCell(np.diag(L), p)
    for step in range(25):
        a = c.sample_modes(step)
        b = O.sample_modes(L, p, step)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), step
        assert np.array_equal(a[2], b[2])


def _enumerated_bins(c, p, nbins=24):
    # P^r over the truncated lattice, modes sorted by |k|^2, cut into bins of
    # about equal probability; returns (mode -> bin, bin probabilities)
    Hr, Hnr, mm = c.normalizers()
    Sr = Hr.sum()
    modes, probs = [], []
    for mx in range(-mm[0], mm[0] + 1):
        for my in range(-mm[1], mm[1] + 1):
            for mz in range(-mm[2], mm[2] + 1):
                pr = c.targets((mx, my, mz))[0] / Sr
                if pr > 1e-14:
                    modes.append((mx, my, mz))
                    probs.append(pr)
    probs = np.array(probs)
    assert abs(probs.sum() - 1) < 1e-9
    order = np.argsort(-probs)
    cum = np.cumsum(probs[order])
    bins = np.minimum((cum / cum[-1] * nbins).astype(int), nbins - 1)
    where = {modes[i]: bins[k] for k, i in enumerate(order)}
    pb = np.bincount(bins, weights=probs[order], minlength=nbins)
    return where, pb


@pytest.fixture(scope="module")
def shear_laws():
    p = O.Params.row2(P=1000)
    c = O.TriCell(H_SHEAR, p)
    return c, _enumerated_bins(c, p)


def _chi2_bins(modes, where, pb):
    idx = np.array([where.get(tuple(int(x) for x in m), -1) for m in modes])
    assert np.all(idx >= 0)
    cnt = np.bincount(idx, minlength=len(pb))
    e = pb * len(modes)
    ok = e > 20
    return float((((cnt - e) ** 2)[ok] / e[ok]).sum()), int(ok.sum())


def test_exact_draws_follow_the_radial_law_in_a_sheared_cell(shear_laws):
    c, (where, pb) = shear_laws
    modes = [c.draw_r(step, i) for step in range(20) for i in range(500)]
    chi, dof = _chi2_bins(modes, where, pb)
    assert chi < dof + 5 * math.sqrt(2 * dof), (chi, dof)


def test_mh_chain_follows_the_radial_law_in_a_sheared_cell(shear_laws):
    c, (where, pb) = shear_laws
    modes, acc = [], np.zeros(2)
    for step in range(10):
        mr, mn, st = c.sample_modes(step)
        modes.extend(mr)
        acc += st
    chi, dof = _chi2_bins(modes, where, pb)
    assert chi / 2 < dof + 5 * math.sqrt(2 * dof), (chi, dof)
    assert acc[0] / 10000 > 0.75 and acc[1] / 10000 > 0.75


@pytest.fixture(scope="module")
def tiny_shear():
    s = W.random_charges(n=24, box=(20.0, 21.0, 22.0), seed=21, min_dist=2.0)
    return W.sheared(s, (4.0, -3.0, 3.5))


def test_estimators_unbiased_in_a_sheared_cell(tiny_shear):
    s = tiny_shear
    h = O.tilted_box(s.box, s.tilt)
    p = O.Params.row2(P=100)
    c = O.TriCell(h, p)
    Hr, Hnr, _ = c.normalizers()
    Fall, Uall, Wall, Wrad = O.kspace_all(s, p, h=h, radial=True)
    U, Wr, F = [], [], []
    for step in range(3000):
        mr, mn, _ = c.sample_modes(step)
        D, cr, cnr = O.distinct(mr, mn)
        f, u, wr, wnr, _ = O.rb_longrange_h(s.pos, s.q, h, p.P, D, cr, cnr, Hr.sum(), Hnr.sum())
        U.append(u)
        Wr.append(wr[0, 0])
        F.append(f.reshape(-1))
    U, Wr, F = np.array(U), np.array(Wr), np.array(F)

    def z(x, ref):
        return np.abs(x.mean(0) - ref) / (x.std(0, ddof=1) / np.sqrt(len(x)))
    assert z(U, Uall) < 4.0
    assert z(Wr, Wrad) < 4.0
    idx = np.argsort(-np.abs(Fall.reshape(-1)))[:12]
    assert np.all(z(F[:, idx], Fall.reshape(-1)[idx]) < 4.5)
    # trace identity with the same samples: tr W^{F,r*} = 3 U^{F*}
    mr, mn, _ = c.sample_modes(7)
    D, cr, cnr = O.distinct(mr, mn)
    f, u, wr, wnr, _ = O.rb_longrange_h(s.pos, s.q, h, p.P, D, cr, cnr, Hr.sum(), Hnr.sum())
    assert abs(np.trace(wr) - 3 * u) < 1e-12 * abs(u)


def test_force_eval_reduces_to_the_orthorhombic_one():
    s = W.water(n_mol=300, L=22.0, lattice=7, seed=2)
    p = O.Params.row2(P=100)
    c = O.TriCell(np.diag(s.box), p)
    a = O.force_eval_h(s, p, 5, c)
    b = O.force_eval(s, p, 5)
    assert np.array_equal(a["mr"], b["mr"]) and np.array_equal(a["mnr"], b["mnr"])
    assert np.abs(a["F"] - b["F"]).max() < 1e-12 * np.abs(b["F"]).max()
    assert np.abs(a["W"] - b["W"]).max() < 1e-12 * np.abs(b["W"]).max()
    for k in ("coul_short", "coul_long", "coul_excl", "lj", "bond", "angle"):
        assert abs(a[k] - b[k]) <= 1e-12 * max(1.0, abs(b[k])), k


def test_fixed_cell_integrator_reduces_to_the_orthorhombic_one():
    s = W.water(n_mol=200, L=20.5, lattice=6, seed=8)
    p = O.Params.row2(P=50)
    ig = O.Integ(dt=0.5, coupling=2, Mbox=(0.0, 0.0, 0.0))
    c = O.TriCell(np.diag(s.box), p)
    rng = np.random.default_rng(1)
    p0 = rng.normal(0, 0.02, (s.n, 3)) * s.mass[:, None]
    r0 = s.pos.copy()
    ev = O.force_eval(s, p, 0, pos=r0)
    st_a = dict(r=r0.copy(), p=p0.copy(), F=ev["F"].copy(), W=ev["W"].reshape(-1).copy())
    O.nvt_run_h(s, p, ig, c, st_a, 0, 4)
    st_b = dict(r=r0.copy(), p=p0.copy(), L=np.array(s.box, dtype=float), ph=np.zeros(3),
                F=ev["F"].copy(), W=ev["W"].reshape(-1).copy())
    O.npt_run(s, p, ig, st_b, 0, 4)
    assert np.abs(st_a["r"] - st_b["r"]).max() < 1e-10
    assert np.abs(st_a["p"] - st_b["p"]).max() < 1e-10 * np.abs(st_b["p"]).max()


def test_fixed_cell_integrator_keeps_atoms_in_a_sheared_cell():
    s = W.sheared(W.water(n_mol=200, L=21.0, lattice=6, seed=8), (3.0, -2.0, 2.5))
    h = O.tilted_box(s.box, s.tilt)
    p = O.Params.row2(P=50)
    c = O.TriCell(h, p)
    ig = O.Integ(dt=0.5, coupling=2)
    ev = O.force_eval_h(s, p, 0, c)
    st = dict(r=s.pos.copy(), p=np.zeros((s.n, 3)), F=ev["F"].copy(), W=ev["W"].reshape(-1).copy())
    en, K = O.nvt_run_h(s, p, ig, c, st, 0, 5)
    f = np.linalg.solve(h, st["r"].T).T
    assert f.min() >= 0.0 and f.max() < 1.0
    assert np.all(np.isfinite(st["F"])) and np.isfinite(en["coul"])
