"""Pins of the oracle's random-batch estimators (sec. 3.2, App. B).

* algebra: tr P^{F,r*} V = 3 U^{F*} with the same samples;
* unbiasedness (Prop. 3.6): the mean over many seeds of U^{F*}, P^{F,r*},
  P^{F,nr*} and F^{F*} equals the deterministic all-modes value (eqs.
  U_long, PcoulFr/P_long, force_SOG) within 3 standard errors, for i.i.d.
  draws (kind 1) and, for the radial, energy and force parts, for the
  paper's MH chain started from an exact draw (kind 0); the recalibrated
  non-radial part is unbiased on i.i.d. radial proposals (kind 2);
* variance O(1/P) (Prop. 3.6 / Theorem 3.7);
* exclusion correction: the minimum-image pair kernel of every
  intramolecular pair is removed, with forces = -grad;
* bonded forces = -grad of the bonded energy (finite differences).
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

NSEED = 10000


@pytest.fixture(scope="module")
def tiny():
    return W.random_charges(n=24, box=(20.0, 21.0, 22.0), seed=21, min_dist=2.0)


def _rb(sys, p, step):
    w, s, wt, st = O.sog_terms(p.b, p.sigma, p.omega, p.M)
    Hr, Hnr, *_ = O.normalizers(sys.box, wt, st)
    mr, mn, _ = O.sample_modes(sys.box, p, step)
    D, cr, cnr = O.distinct(mr, mn)
    return O.rb_longrange(sys.pos, sys.q, sys.box, p.P, D, cr, cnr, Hr.sum(), Hnr.sum(), p.ke)


def test_trace_identity_of_radial_estimator(tiny):
    p = O.Params.row2(P=100)
    F, U, Wr, Wnr, _ = _rb(tiny, p, 1)
    assert abs(np.trace(Wr) - 3 * U) < 1e-12 * abs(U)
    assert np.allclose(Wr, np.diag(np.diag(Wr)))


def _stats(sys, kind, P, nseed):
    p = O.Params.row2(P=P, kind=kind)
    U, Wr, Wnr, F = [], [], [], []
    for step in range(nseed):
        f, u, wr, wnr, _ = _rb(sys, p, step)
        U.append(u)
        Wr.append(wr[0, 0])
        Wnr.append(wnr.reshape(-1))
        F.append(f.reshape(-1))
    return np.array(U), np.array(Wr), np.array(Wnr), np.array(F)


def _within(x, ref, k=3.5):
    m = x.mean(0)
    se = x.std(0, ddof=1) / np.sqrt(len(x))
    z = np.abs(m - ref) / np.maximum(se, 1e-300)
    return z, np.all(z < k)


@pytest.fixture(scope="module")
def exact(tiny):
    p = O.Params.row2(P=100)
    Fall, Uall, Wall, Wrad = O.kspace_all(tiny, p, radial=True)
    return Fall, Uall, Wall, Wrad


@pytest.mark.parametrize("kind", [1, 0, 2])
def test_radial_energy_force_unbiased(tiny, exact, kind):
    Fall, Uall, Wall, Wrad = exact
    U, Wr, Wnr, F = _stats(tiny, kind, 100, NSEED)
    z, ok = _within(U, Uall)
    assert ok, ("U", z)
    z, ok = _within(Wr, Wrad)
    assert ok, ("Wr", z)
    # force: test the components with the largest long-range force
    idx = np.argsort(-np.abs(Fall.reshape(-1)))[:12]
    z, ok = _within(F[:, idx], Fall.reshape(-1)[idx], k=4.0)
    assert ok, ("F", z)


@pytest.mark.parametrize("kind", [1, 2])
def test_nonradial_unbiased_with_iid_proposals(tiny, exact, kind):
    Fall, Uall, Wall, Wrad = exact
    U, Wr, Wnr, F = _stats(tiny, kind, 100, NSEED)
    Wnr_ref = (Wall - Wrad * np.eye(3)).reshape(-1)
    z, ok = _within(Wnr[:, [0, 1, 2, 4, 5, 8]], Wnr_ref[[0, 1, 2, 4, 5, 8]], k=4.0)
    assert ok, z


def test_nonradial_bias_of_the_paper_chain_is_measured(tiny, exact):
    # the paper's construction (kind 0): report the bias of the diagonal nr
    # components in units of their standard error (not asserted to vanish)
    Fall, Uall, Wall, Wrad = exact
    U, Wr, Wnr, F = _stats(tiny, 0, 100, NSEED)
    Wnr_ref = (Wall - Wrad * np.eye(3)).reshape(-1)
    m = Wnr.mean(0)
    rel = (m - Wnr_ref)[[0, 4, 8]] / np.abs(Wnr_ref[[0, 4, 8]])
    assert np.all(np.abs(rel) < 0.5)


def test_variance_scales_as_one_over_P(tiny):
    v = {}
    for P in (25, 100, 400):
        U, Wr, Wnr, F = _stats(tiny, 1, P, 600)
        v[P] = Wr.var(ddof=1) * P
    r1, r2 = v[100] / v[25], v[400] / v[100]
    assert 0.7 < r1 < 1.4 and 0.7 < r2 < 1.4, v


def test_exclusion_term_removes_intramolecular_pairs():
    # the Fourier part holds each intramolecular pair's q_i q_j F(r) at the
    # minimum image (its periodic images stay: they are other copies); the
    # exclusion term removes exactly that, and its force is minus its
    # gradient (finite differences)
    s = W.water(n_mol=8, L=24.0, lattice=2, seed=3)
    p = O.Params.row2(M=10, ME=10)
    F, U, Wx = O.exclusions(s, p)
    w, sg, wt, st = O.sog_terms(p.b, p.sigma, p.omega, 10)
    ref_u = 0.0
    for i, j in s.excl:
        d = s.pos[i] - s.pos[j]
        d -= s.box * np.rint(d / s.box)
        r2 = d @ d
        ref_u -= p.ke * s.q[i] * s.q[j] * np.sum(w * np.exp(-r2 / sg ** 2))
    assert abs(U - ref_u) < 1e-12 * abs(ref_u)
    assert np.abs(F.sum(0)).max() < 1e-10
    # force = -grad of the exclusion energy
    eps = 1e-6
    for a in range(3):
        pp, pm = s.pos.copy(), s.pos.copy()
        pp[1, a] += eps
        pm[1, a] -= eps
        up = O.exclusions(s, p, pos=pp)[1]
        um = O.exclusions(s, p, pos=pm)[1]
        assert abs(-(up - um) / (2 * eps) - F[1, a]) < 1e-6 * (1 + abs(F[1, a]))


def test_bonded_forces_are_minus_gradient():
    s = W.water(n_mol=8, L=24.0, lattice=2, seed=3, jitter=0.1)
    rng = np.random.default_rng(1)
    pos = s.pos + rng.normal(0, 0.05, s.pos.shape)
    F, en, Wb = O.bonded(s, pos=pos)
    eps = 1e-6
    for i in (0, 1, 2, 4):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[i, a] += eps
            pm[i, a] -= eps
            g = -(O.bonded(s, pos=pp)[1].sum() - O.bonded(s, pos=pm)[1].sum()) / (2 * eps)
            assert abs(g - F[i, a]) < 1e-5 * (1 + abs(F[i, a]))
    # virial = -dU/deps
    E = np.eye(3)
    E[0, 1] += 1e-6
    up = O.bonded(s, pos=pos @ E.T, h=E @ np.diag(s.box))[1].sum()
    E[0, 1] -= 2e-6
    um = O.bonded(s, pos=pos @ E.T, h=E @ np.diag(s.box))[1].sum()
    assert abs(-(up - um) / 2e-6 - Wb[0, 1]) < 1e-5 * (1 + np.abs(Wb).max())


def _shared_stats(sys, kind, P, nseed):
    p = O.Params.row2(P=P, kind=kind)
    w, s, wt, st = O.sog_terms(p.b, p.sigma, p.omega, p.M)
    Hr, Hnr, *_ = O.normalizers(sys.box, wt, st)
    out = []
    for step in range(nseed):
        mr, mn, _ = O.sample_modes(sys.box, p, step)
        D, cr, cnr = O.distinct(mr, mn)
        rh = O.rho(sys.pos, sys.q, sys.box, D)
        out.append(O.nr_shared(sys.box, p, D, cr, rh, Hr.sum()).reshape(-1))
    return np.array(out)


@pytest.mark.parametrize("kind", [1, 0])
def test_shared_proposal_nonradial_unbiased(tiny, exact, kind):
    # sec. 3.2: the radial samples reused for P^F,nr with weights f_nr / P^r
    # estimate the same tensor (every radial state is P^r-distributed)
    Fall, Uall, Wall, Wrad = exact
    Wsh = _shared_stats(tiny, kind, 100, NSEED)
    Wnr_ref = (Wall - Wrad * np.eye(3)).reshape(-1)
    z, ok = _within(Wsh[:, [0, 1, 2, 4, 5, 8]], Wnr_ref[[0, 1, 2, 4, 5, 8]], k=4.0)
    assert ok, z


def test_shared_proposal_weight_is_the_target_ratio(tiny):
    # one mode, multiplicity 1: the estimator equals -ke S^r/(8 V P) (f_nr/f_r) |rho|^2 k k / k^4,
    # with f_r, f_nr the unnormalised targets of eqs. samplingP, samplingPnr (oracle targets())
    p = O.Params.row2(P=7)
    w, s, wt, st = O.sog_terms(p.b, p.sigma, p.omega, p.M)
    Hr, Hnr, *_ = O.normalizers(tiny.box, wt, st)
    D = np.array([[1, -2, 3]], np.int32)
    rh = O.rho(tiny.pos, tiny.q, tiny.box, D)
    Wsh = O.nr_shared(tiny.box, p, D, np.array([1], np.int32), rh, Hr.sum())
    fr, fnr, _ = O.targets(tiny.box, p, D[0])
    k = 2 * np.pi * D[0] / np.asarray(tiny.box)
    k2 = k @ k
    V = float(np.prod(tiny.box))
    ref = -p.ke * Hr.sum() / (8 * V * p.P) * (fnr / fr) * abs(rh[0]) ** 2 * np.outer(k, k) / k2 ** 2
    assert np.allclose(Wsh, ref, rtol=1e-12, atol=0)


def test_pressure_variance_does_not_grow_with_N():
    # Theorem 3.7 (Debye-Hueckel regime): the variance of the random-batch
    # pressure is bounded independently of N.  At fixed density, 8,000 and
    # 27,000 ions give the same spread of P^F,r* and P^F,nr* over counters
    # (the per-atom force noise, by contrast, grows with the box)
    sds = []
    for n, L in ((8000, 60.0), (27000, 90.0)):
        s = W.electrolyte(n_ions=n, L=L, seed=1)
        p = O.Params.row2(P=100)
        V = float(np.prod(s.box))
        r, nr = [], []
        for step in range(40):
            _, _, wr, wnr, _ = _rb(s, p, step)
            r.append(wr[0, 0] / V)
            nr.append(wnr[0, 0] / V)
        sds.append((np.std(r, ddof=1), np.std(nr, ddof=1)))
    for k in range(2):
        assert 0.6 < sds[1][k] / sds[0][k] < 1.7, sds


def test_exclusion_energy_against_real_space_image_sum():
    # Independent pin of the exclusion energy: for one neutral 3-site
    # molecule whose three pairs are all excluded, the all-modes Fourier
    # energy minus the self energy plus the exclusion term must equal the
    # plain real-space image sum of the SOG energy kernel F_E(r) = sum_l w_l
    # exp(-r^2/s_l^2) over every periodic image except the molecule's own
    # (n = 0) copy:
    #   U^F - U_self + U_excl = ke sum_{n != 0} [ 1/2 sum_i q_i^2 F_E(|n L|)
    #                                            + sum_{i<j} q_i q_j F_E(|r_ij + n L|) ]
    # (App. A: U^F holds the pair sum over all images and the i = j, n = 0
    # terms; U_self removes the latter, the exclusion the n = 0 pair terms).
    # M = 4 force Gaussians and M_E = 6 energy Gaussians, so that an
    # exclusion using the force set for the energy fails.
    pos = np.array([[10.0, 11.0, 9.5], [10.9, 11.5, 9.8], [9.3, 11.6, 10.2]])
    q = np.array([-0.8, 0.45, 0.35])
    L = np.array([20.0, 22.0, 24.0])
    s = W.random_charges(n=3, box=tuple(L), seed=1, min_dist=0.5)
    s.pos, s.q = pos.copy(), q.copy()
    s.mol = np.zeros(3, np.int32)
    s.excl = np.array([[0, 1], [0, 2], [1, 2]], np.int32)
    p = O.Params.row2(M=4, ME=6)
    w, sg, wt, st = O.sog_terms(p.b, p.sigma, p.omega, 6)
    _, UF, _ = O.kspace_all(s, p, terms=(w, sg, wt[:4], st[:4]))
    Us = O.self_energy(p, q)
    _, Ux, _ = O.exclusions(s, p)
    lhs = UF - Us + Ux

    def FE(r2):
        return np.exp(-r2[..., None] / sg ** 2) @ w

    nmax = np.ceil(7.0 * sg.max() / L).astype(int)
    g = [np.arange(-k, k + 1) for k in nmax]
    n = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    n = n[np.any(n != 0, axis=1)] * L
    rhs = 0.5 * np.sum(q ** 2) * FE(np.sum(n ** 2, 1)).sum()
    for i in range(3):
        for j in range(i + 1, 3):
            d = pos[i] - pos[j] + n
            rhs += q[i] * q[j] * FE(np.sum(d ** 2, 1)).sum()
    rhs *= p.ke
    assert abs(lhs - rhs) < 1e-9 * max(abs(rhs), 1.0), (lhs, rhs)
