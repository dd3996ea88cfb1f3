"""Pins of the oracle's Langevin NPT integrator (eq. Langevin_NPT with the
BAOAB splitting that is our reading of the paper's integrator).

* with gamma = 0, a fixed box and deterministic forces (uncharged water: LJ
  and bonded terms only) the splitting is velocity Verlet: the total energy
  is conserved and its fluctuation falls as dt^2;
* with the thermostat on, the mean kinetic temperature matches the target;
* with the barostat on, an ideal-gas-like dilute system follows
  <(K + W) / V - kB T / V> = P_ext (the stationarity condition of the box
  equation) and the box moves.
"""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


def _state(sys, T, seed, zero_com=True):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=sys.pos.shape) * np.sqrt(sys.mass[:, None] * O.KB * T * O.FTM2V)
    if zero_com:
        p -= p.sum(0) / sys.n
    return dict(r=sys.pos.copy(), p=p, L=sys.box.copy(), ph=np.zeros(3),
                F=np.zeros_like(sys.pos), W=np.zeros(9))


def _prime(sys, par, st):
    out = O.force_eval(sys, par, 0, pos=st["r"], L=st["L"])
    st["F"] = out["F"]
    st["W"] = out["W"].reshape(-1).copy()
    return out


def _total_energy(sys, st):
    ke = 0.5 * np.sum(st["p"] ** 2 / sys.mass[:, None]) / O.FTM2V
    e = st["en"]
    return ke + e["coul"] + e["lj"] + e["bond"] + e["angle"]


def test_nve_energy_error_scales_as_dt_squared():
    s = W.water(n_mol=27, L=30.0, lattice=3, seed=1)
    s.q[:] = 0.0
    par = O.Params.row2(P=10)
    amp = {}
    for dt in (0.25, 0.5):
        st = _state(s, 300.0, 2)
        _prime(s, par, st)
        ig = O.Integ(dt=dt, T=300.0, gamma=0.0, gamma_box=0.0, Mbox=(0.0, 0.0, 0.0))
        E = []
        nsteps = int(round(40 / dt))
        for n in range(nsteps):
            O.npt_run(s, par, ig, st, n, 1)
            E.append(_total_energy(s, st))
        E = np.array(E)
        amp[dt] = E.max() - E.min()
    ratio = amp[0.5] / amp[0.25]
    assert 3.0 < ratio < 5.0, amp


def test_thermostat_reaches_target_temperature():
    s = W.water(n_mol=27, L=30.0, lattice=3, seed=1)
    s.q[:] = 0.0
    par = O.Params.row2(P=10)
    st = _state(s, 100.0, 3)
    _prime(s, par, st)
    ig = O.Integ(dt=0.5, T=300.0, gamma=0.02, Mbox=(0.0, 0.0, 0.0))
    temps = []
    ndof = 3 * s.n
    for n in range(600):
        O.npt_run(s, par, ig, st, n, 1)
        if n >= 200:
            temps.append(np.trace(st["K"]) / (ndof * O.KB))
    temps = np.array(temps)
    # 400 correlated samples; a 10 K band is > 5 standard errors
    assert abs(temps.mean() - 300.0) < 10.0, temps.mean()


def test_barostat_moves_box_and_balances_pressure():
    # dilute LJ fluid of uncharged atoms: virial small, P_ins ~ N kB T / V
    s = W.random_charges(n=64, box=(40.0, 40.0, 40.0), seed=4, min_dist=3.0, lj=True)
    s.q[:] = 0.0
    par = O.Params.row2(P=10)
    st = _state(s, 300.0, 5)
    _prime(s, par, st)
    V0 = np.prod(s.box)
    # strong coupling so that a short run equilibrates the box
    Mb = 5.0
    ig = O.Integ(dt=2.0, T=300.0, Pext_atm=2000.0, gamma=0.02, gamma_box=0.01,
                 Mbox=(Mb, 0.0, 0.0))
    lhs = []
    for n in range(1500):
        O.npt_run(s, par, ig, st, n, 1)
        V = np.prod(st["L"])
        if n >= 500:
            lhs.append((np.trace(st["K"]) + np.trace(st["W"].reshape(3, 3))) / (3 * V) - O.KB * 300.0 / V)
    assert abs(np.prod(st["L"]) - V0) / V0 > 0.05
    p_mean = np.mean(lhs) * O.NKTV2P
    assert abs(p_mean - 2000.0) < 400.0, p_mean


def test_semi_isotropic_barostat_per_group():
    # coupling 1 (x = y coupled, z free; the membrane setting of sec. 4.3):
    # * x and y share one box momentum, so L_x = L_y exactly at every step;
    # * z moves on its own, so L_z / L_x changes;
    # * each group's box equation is stationary: the mean of its generalised
    #   force vanishes, i.e. <(K_aa + W_aa) / V - kB T / V> = P_ext averaged
    #   over the axes of the group, for the xy group and the z group apart;
    # * the box momentum of each group is Maxwell distributed at T with that
    #   group's own mass (equipartition, <p_g^2 / M_g> = kB T): a mass used in
    #   the drift that differs from the one in the noise breaks it.
    s = W.random_charges(n=64, box=(40.0, 40.0, 48.0), seed=4, min_dist=3.0, lj=True)
    s.q[:] = 0.0
    par = O.Params.row2(P=10)
    st = _state(s, 300.0, 5)
    _prime(s, par, st)
    Mxy, Mz = 8.0, 3.0
    ig = O.Integ(dt=2.0, T=300.0, Pext_atm=2000.0, gamma=0.02, gamma_box=0.05, coupling=1,
                 Mbox=(Mxy, Mz, 0.0))
    ratio0 = s.box[2] / s.box[0]
    bal_xy, bal_z, e_xy, e_z, ratios = [], [], [], [], []
    kT = O.KB * 300.0
    for n in range(3000):
        O.npt_run(s, par, ig, st, n, 1)
        L = st["L"]
        assert L[0] == L[1], (n, L)
        V = np.prod(L)
        K, Wv = st["K"], st["W"].reshape(3, 3)
        ratios.append(L[2] / L[0])
        if n >= 500:
            bal_xy.append((K[0, 0] + Wv[0, 0] + K[1, 1] + Wv[1, 1]) / (2 * V) - kT / V)
            bal_z.append((K[2, 2] + Wv[2, 2]) / V - kT / V)
            e_xy.append(st["ph"][0] ** 2 / Mxy / O.FTM2V)
            e_z.append(st["ph"][1] ** 2 / Mz / O.FTM2V)
    assert np.ptp(ratios) > 0.02 * ratio0
    for name, b in (("xy", bal_xy), ("z", bal_z)):
        p_mean = np.mean(b) * O.NKTV2P
        assert abs(p_mean - 2000.0) < 400.0, (name, p_mean)
    for name, e in (("xy", e_xy), ("z", e_z)):
        assert abs(np.mean(e) / kT - 1.0) < 0.2, (name, np.mean(e) / kT)
    assert st["ph"][2] == 0.0
