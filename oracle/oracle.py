"""ctypes front end of the FP64 CPU oracle (``rbsog_oracle.c``).

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code
with the CUDA path.  Every function forwards to the C routine of the same
name, which cites the passage of arXiv 2602.23582 it follows.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os

import numpy as np

from . import build as _build

_lib = None

# Table 2, row 2 of the paper (used "in all tests", sec. 4): (b, sigma at
# r_c = 9 A, omega).  sigma scales with r_c: F(lambda r; lambda sigma) = F(r; sigma)/lambda.
TABLE2_ROW2 = (1.62976708826776469, 3.270345668108471, 1.007806979343806)

# LAMMPS "real" unit constants (our reading: the paper is silent on units)
KE = 332.06371                   # kcal A / (mol e^2)
NKTV2P = 68568.415               # atm per kcal/(mol A^3)
KB = 0.0019872067                # kcal / (mol K)
FTM2V = 1.0 / 48.88821291 / 48.88821291   # (kcal/mol/A)/(g/mol) -> A/fs^2


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_U64 = C.POINTER(C.c_uint64)


class _Params(C.Structure):
    _fields_ = [("rc", C.c_double), ("b", C.c_double), ("sigma", C.c_double),
                ("omega", C.c_double), ("ke", C.c_double), ("M", C.c_int),
                ("ME", C.c_int), ("P", C.c_int), ("kind", C.c_int),
                ("seed", C.c_uint64), ("sysid", C.c_uint64), ("short_cells", C.c_int)]


class _System(C.Structure):
    _fields_ = [("N", C.c_int), ("q", _D), ("mass", _D), ("type", _I), ("mol", _I),
                ("ntypes", C.c_int), ("lj_eps", _D), ("lj_sig", _D),
                ("nb", C.c_int), ("bonds", _I), ("bk", _D), ("br0", _D),
                ("na", C.c_int), ("angles", _I), ("ak", _D), ("at0", _D),
                ("ne", C.c_int), ("excl", _I)]


class _Integ(C.Structure):
    _fields_ = [("dt", C.c_double), ("T", C.c_double), ("Pext_atm", C.c_double),
                ("gamma", C.c_double), ("gamma_box", C.c_double), ("coupling", C.c_int),
                ("Mbox", C.c_double * 3), ("kB", C.c_double), ("ftm2v", C.c_double),
                ("nktv2p", C.c_double)]


def _declare(L):
    L.orc_sog_terms.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _D, _D, _D, _D]
    L.orc_nr_shared.argtypes = [_D, C.c_int, C.c_int, _I, _I, _D, C.c_int, _D, _D, C.c_double, C.c_double, _D]
    L.orc_sog_solve.argtypes = [C.c_double, C.c_double, _D, _D, _D]
    L.orc_sog_solve.restype = C.c_int
    L.orc_bsa.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int]
    L.orc_bsa.restype = C.c_double
    L.orc_philox.argtypes = [_U64, _U64, _U64]
    L.orc_u01.argtypes = [C.c_uint64]
    L.orc_u01.restype = C.c_double
    L.orc_cell_bin.argtypes = [C.c_int, _D, _D, C.c_double, C.c_int, _I, _I]
    L.orc_short_range.argtypes = [C.c_int, _D, _D, _I, _I, _D, C.c_double, C.c_int, _D, _D,
                                  C.c_int, _D, _D, C.c_int, _D, _D, C.c_double, _D, _D, _D, _D]
    L.orc_short_range_cells.argtypes = L.orc_short_range.argtypes
    L.orc_short_range_cells.restype = C.c_int
    L.orc_set_threads.argtypes = [C.c_int]
    L.orc_set_threads.restype = None
    L.orc_kspace_all.argtypes = [C.c_int, _D, _D, _D, C.c_int, _D, _D, C.c_int, _D, _D, _I,
                                 C.c_double, _D, _D, _D, _D]
    L.orc_pf_realspace.argtypes = [C.c_int, _D, _D, _D, C.c_double, C.c_double, _I, C.c_double, _D]
    L.orc_normalizers.argtypes = [_D, C.c_int, _D, _D, _D, _D, _D, _D, _D]
    L.orc_normalizers_3d.argtypes = [_D, C.c_int, _D, _D, _I, _D, _D]
    L.orc_normalizers_poisson.argtypes = [_D, C.c_int, _D, _D, _I, _D, _D]
    L.orc_sample_modes.argtypes = [_D, C.c_int, _D, _D, C.c_int, C.c_uint64, C.c_uint64,
                                   C.c_uint64, C.c_int, _I, _I, _D]
    L.orc_targets.argtypes = [_D, C.c_int, _D, _D, _I, _D]
    L.orc_distinct.argtypes = [C.c_int, _I, C.c_int, _I, _I, _I, _I]
    L.orc_distinct.restype = C.c_int
    L.orc_rho.argtypes = [C.c_int, _D, _D, _D, C.c_int, _I, _D]
    L.orc_rb_longrange.argtypes = [C.c_int, _D, _D, _D, C.c_int, C.c_int, _I, _I, _I,
                                   C.c_double, C.c_double, C.c_double, _D, _D, _D, _D, _D]
    L.orc_self_energy.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _D, C.c_double]
    L.orc_self_energy.restype = C.c_double
    L.orc_exclusions.argtypes = [C.c_int, _I, _D, _D, _D, C.c_int, _D, _D, C.c_int, _D, _D,
                                 C.c_double, _D, _D, _D]
    L.orc_bonded.argtypes = [C.c_int, _I, _D, _D, C.c_int, _I, _D, _D, _D, _D, _D, _D, _D]
    L.orc_force_eval.argtypes = [C.POINTER(_Params), C.POINTER(_System), _D, _D, C.c_uint64,
                                 _D, _D, _D, _D, _I]
    L.orc_npt_run.argtypes = [C.POINTER(_Params), C.POINTER(_System), C.POINTER(_Integ),
                              _D, _D, _D, _D, _D, _D, C.c_uint64, C.c_int, _D, _D]
    L.orc_num_threads.restype = C.c_int
    L.orc_tri_q.argtypes = [_D, C.c_double, _I, C.c_int]
    L.orc_tri_q.restype = C.c_double
    L.orc_tri_create.argtypes = [_D, C.c_int, _D, _D]
    L.orc_tri_create.restype = C.c_void_p
    L.orc_tri_free.argtypes = [C.c_void_p]
    L.orc_tri_free.restype = None
    L.orc_tri_normalizers.argtypes = [C.c_void_p, _D, _D, _I]
    L.orc_tri_normalizers.restype = None
    L.orc_tri_targets.argtypes = [C.c_void_p, _I, _D]
    L.orc_tri_targets.restype = None
    L.orc_tri_sample_modes.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_uint64, C.c_uint64, _I, _I, _D]
    L.orc_tri_sample_modes.restype = None
    L.orc_tri_draw_r.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint64, _I]
    L.orc_tri_draw_r.restype = None
    L.orc_rho_h.argtypes = [C.c_int, _D, _D, _D, C.c_int, _I, _D]
    L.orc_rb_longrange_h.argtypes = L.orc_rb_longrange.argtypes
    L.orc_force_eval_h.argtypes = [C.POINTER(_Params), C.POINTER(_System), _D, _D, C.c_void_p, C.c_uint64,
                                   _D, _D, _D, _D, _I]
    L.orc_nvt_run_h.argtypes = [C.POINTER(_Params), C.POINTER(_System), C.POINTER(_Integ), C.c_void_p,
                                _D, _D, _D, _D, C.c_uint64, C.c_int, _D, _D]


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(_D)


def _pi(a):
    return a.ctypes.data_as(_I)


def num_threads() -> int:
    return lib().orc_num_threads()


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    """SOG split and random-batch settings (sec. 2.2, 3.1, 3.2)."""
    rc: float = 10.0
    b: float = TABLE2_ROW2[0]
    sigma: float = TABLE2_ROW2[1] * 10.0 / 9.0
    omega: float = TABLE2_ROW2[2]
    ke: float = KE
    M: int = 10            # Gaussians of the force/pressure split (M~ = M)
    ME: int = 10           # Gaussians of the energy split
    P: int = 100           # batch size
    kind: int = 0          # 0: paper MH + recalibration; 1: exact i.i.d. draws;
                           # 2: exact i.i.d. radial draws + recalibration chain
    seed: int = 1
    sysid: int = 0
    short_cells: int = 0   # 1: short range over cell lists (bit-identical; for the timed baseline)

    @classmethod
    def row2(cls, rc=10.0, **kw):
        return cls(rc=rc, sigma=TABLE2_ROW2[1] * rc / 9.0, **kw)

    def c(self):
        return _Params(self.rc, self.b, self.sigma, self.omega, self.ke, self.M, self.ME,
                       self.P, self.kind, self.seed, self.sysid, self.short_cells)


def sog_terms(b, sigma, omega, M):
    w, s, wt, st = (np.zeros(M) for _ in range(4))
    lib().orc_sog_terms(b, sigma, omega, M, _pd(w), _pd(s), _pd(wt), _pd(st))
    return w, s, wt, st


def sog_solve(b, rc):
    sg, om, res = C.c_double(), C.c_double(), np.zeros(2)
    rcode = lib().orc_sog_solve(b, rc, C.byref(sg), C.byref(om), _pd(res))
    if rcode != 0:
        raise RuntimeError("no solution")
    return sg.value, om.value, res


def bsa(beta, b, sigma, r, lmin, lmax):
    return lib().orc_bsa(beta, b, sigma, r, lmin, lmax)


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox(c.ctypes.data_as(_U64), k.ctypes.data_as(_U64), out.ctypes.data_as(_U64))
    return out


def u01(x):
    return lib().orc_u01(int(x))


def cell_bin(pos, L, rc, sub=1):
    pos, L = _d(pos), _d(L)
    n = pos.shape[0]
    nc = np.zeros(3, np.int32)
    cell = np.zeros(n, np.int32)
    lib().orc_cell_bin(n, _pd(pos), _pd(L), rc, sub, _pi(nc), _pi(cell))
    return nc, cell


def box_matrix(L):
    return np.diag(_d(L))


def short_range(sys, params: Params, h=None, pos=None):
    """Returns (F, U_coul^N, U_LJ, W_coul, W_LJ); W in kcal/mol (3x3)."""
    pos = _d(sys.pos if pos is None else pos)
    h = _d(box_matrix(sys.box) if h is None else h)
    MM = max(params.M, params.ME)
    w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, MM)
    F = np.zeros((sys.n, 3))
    en, Wc, Wl = np.zeros(2), np.zeros(9), np.zeros(9)
    lib().orc_short_range(sys.n, _pd(pos), _pd(_d(sys.q)), _pi(_i(sys.type)), _pi(_i(sys.mol)),
                          _pd(h), params.rc, params.M, _pd(wt), _pd(st), params.ME, _pd(w), _pd(s),
                          sys.ntypes, _pd(_d(sys.lj_eps)), _pd(_d(sys.lj_sig)), params.ke,
                          _pd(F), _pd(en), _pd(Wc), _pd(Wl))
    return F, en[0], en[1], Wc.reshape(3, 3), Wl.reshape(3, 3)


def short_range_cells(sys, params: Params, h=None, pos=None):
    """As short_range, over cell lists (bit-identical; None if the box holds
    fewer than 3 cells of r_c per axis or h is not diagonal)."""
    pos = _d(sys.pos if pos is None else pos)
    h = _d(box_matrix(sys.box) if h is None else h)
    MM = max(params.M, params.ME)
    w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, MM)
    F = np.zeros((sys.n, 3))
    en, Wc, Wl = np.zeros(2), np.zeros(9), np.zeros(9)
    rc = lib().orc_short_range_cells(sys.n, _pd(pos), _pd(_d(sys.q)), _pi(_i(sys.type)), _pi(_i(sys.mol)),
                                     _pd(h), params.rc, params.M, _pd(wt), _pd(st), params.ME, _pd(w), _pd(s),
                                     sys.ntypes, _pd(_d(sys.lj_eps)), _pd(_d(sys.lj_sig)), params.ke,
                                     _pd(F), _pd(en), _pd(Wc), _pd(Wl))
    if rc != 0:
        return None
    return F, en[0], en[1], Wc.reshape(3, 3), Wl.reshape(3, 3)


def set_threads(n: int):
    """OpenMP threads of the oracle's parallel sums (the timed baseline)."""
    lib().orc_set_threads(int(n))


def kspace_mmax(h, st0, eps=1e-17):
    """|m_a| bound so that e^{-s~0^2 k^2/4} < eps beyond it (orthorhombic-like cells)."""
    lens = np.linalg.norm(_d(h), axis=0)
    return np.array([int(math.ceil(2.0 * math.sqrt(math.log(1 / eps)) * Lh / (math.pi * st0)))
                     for Lh in lens], dtype=np.int32)


def kspace_all(sys, params: Params, h=None, pos=None, mmax=None, terms=None, radial=False):
    """Deterministic all-modes Fourier part: (F, U^F, W^F) (W = V P^F, kcal/mol).
    ``terms`` = (w, s, wt, st) overrides the Gaussians (their lengths give ME, M)."""
    pos = _d(sys.pos if pos is None else pos)
    h = _d(box_matrix(sys.box) if h is None else h)
    if terms is None:
        MM = max(params.M, params.ME)
        w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, MM)
        M, ME = params.M, params.ME
    else:
        w, s, wt, st = (_d(t) for t in terms)
        ME, M = len(w), len(wt)
    if mmax is None:
        mmax = kspace_mmax(h, float(np.min(st)))
    mmax = _i(mmax)
    F = np.zeros((sys.n, 3))
    U, W, Wr = np.zeros(1), np.zeros(9), np.zeros(1)
    lib().orc_kspace_all(sys.n, _pd(pos), _pd(_d(sys.q)), _pd(h), M, _pd(wt), _pd(st),
                         ME, _pd(w), _pd(s), _pi(mmax), params.ke, _pd(F), _pd(U), _pd(W), _pd(Wr))
    if radial:
        return F, U[0], W.reshape(3, 3), Wr[0]
    return F, U[0], W.reshape(3, 3)


def pf_realspace(sys, wtl, stl, nmax, ke=KE, h=None, pos=None):
    pos = _d(sys.pos if pos is None else pos)
    h = _d(box_matrix(sys.box) if h is None else h)
    W = np.zeros(9)
    lib().orc_pf_realspace(sys.n, _pd(pos), _pd(_d(sys.q)), _pd(h), wtl, stl,
                           _pi(_i(nmax)), ke, _pd(W))
    return W.reshape(3, 3)


def normalizers(L, wt, st):
    M = len(wt)
    Hr, Hnr = np.zeros(M), np.zeros(M)
    T0, T2, T4 = np.zeros(3 * M), np.zeros(3 * M), np.zeros(3 * M)
    lib().orc_normalizers(_pd(_d(L)), M, _pd(_d(wt)), _pd(_d(st)), _pd(Hr), _pd(Hnr),
                          _pd(T0), _pd(T2), _pd(T4))
    return Hr, Hnr, T0.reshape(M, 3), T2.reshape(M, 3), T4.reshape(M, 3)


def normalizers_3d(h, wt, st, mmax):
    M = len(wt)
    Hr, Hnr = np.zeros(M), np.zeros(M)
    lib().orc_normalizers_3d(_pd(_d(h)), M, _pd(_d(wt)), _pd(_d(st)), _pi(_i(mmax)), _pd(Hr), _pd(Hnr))
    return Hr, Hnr


def normalizers_poisson(h, wt, st, nmax):
    M = len(wt)
    Hr, Hnr = np.zeros(M), np.zeros(M)
    lib().orc_normalizers_poisson(_pd(_d(h)), M, _pd(_d(wt)), _pd(_d(st)), _pi(_i(nmax)),
                                  _pd(Hr), _pd(Hnr))
    return Hr, Hnr


def sample_modes(L, params: Params, step, sysid=None):
    """(m^r (P,3), m^nr (P,3), [accepted radial, accepted nr])."""
    w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, params.M)
    P = params.P
    mr, mnr, stats = np.zeros((P, 3), np.int32), np.zeros((P, 3), np.int32), np.zeros(2)
    lib().orc_sample_modes(_pd(_d(L)), params.M, _pd(wt), _pd(st), P, params.seed,
                           params.sysid if sysid is None else sysid, step, params.kind,
                           _pi(mr), _pi(mnr), _pd(stats))
    return mr, mnr, stats


def targets(L, params: Params, m):
    w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, params.M)
    out = np.zeros(3)
    lib().orc_targets(_pd(_d(L)), params.M, _pd(wt), _pd(st), _pi(_i(m)), _pd(out))
    return out


def distinct(mr, mnr):
    mr, mnr = _i(mr), _i(mnr)
    n = len(mr) + len(mnr)
    D, cr, cnr = np.zeros((n, 3), np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
    nd = lib().orc_distinct(len(mr), _pi(mr), len(mnr), _pi(mnr), _pi(D), _pi(cr), _pi(cnr))
    return D[:nd].copy(), cr[:nd].copy(), cnr[:nd].copy()


def rho(pos, q, L, D):
    pos, q, D = _d(pos), _d(q), _i(D)
    out = np.zeros(2 * len(D))
    lib().orc_rho(len(q), _pd(pos), _pd(q), _pd(_d(L)), len(D), _pi(D), _pd(out))
    return out[0::2] + 1j * out[1::2]


def rb_longrange(pos, q, L, P, D, cr, cnr, Sr, Snr, ke=KE):
    """(F, U^F*, W^{F,r*}, W^{F,nr*}, rho) with W = V P (kcal/mol)."""
    pos, q, D = _d(pos), _d(q), _i(D)
    n = len(q)
    F = np.zeros((n, 3))
    U, Wr, Wnr, rh = np.zeros(1), np.zeros(9), np.zeros(9), np.zeros(2 * len(D))
    lib().orc_rb_longrange(n, _pd(pos), _pd(q), _pd(_d(L)), P, len(D), _pi(D), _pi(_i(cr)),
                           _pi(_i(cnr)), Sr, Snr, ke, _pd(F), _pd(U), _pd(Wr), _pd(Wnr), _pd(rh))
    return F, U[0], Wr.reshape(3, 3), Wnr.reshape(3, 3), rh[0::2] + 1j * rh[1::2]


def nr_shared(L, params: Params, D, cr, rh, Sr):
    """V P^{F,nr} by the shared-proposal estimator (sec. 3.2): the radial
    samples (multiplicities cr over the distinct modes D, structure factors rh)
    reused for the non-radial part with weights f_nr / P^r."""
    w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, params.M)
    D = _i(D)
    rr = np.zeros(2 * len(D))
    rr[0::2], rr[1::2] = np.real(rh), np.imag(rh)
    out = np.zeros(9)
    lib().orc_nr_shared(_pd(_d(L)), params.P, len(D), _pi(D), _pi(_i(cr)), _pd(rr), params.M, _pd(wt), _pd(st),
                        Sr, params.ke, _pd(out))
    return out.reshape(3, 3)


def self_energy(params: Params, q):
    q = _d(q)
    return lib().orc_self_energy(params.b, params.sigma, params.omega, params.ME, len(q), _pd(q), params.ke)


def exclusions(sys, params: Params, pos=None, h=None):
    pos = _d(sys.pos if pos is None else pos)
    h = _d(box_matrix(sys.box) if h is None else h)
    MM = max(params.M, params.ME)
    w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, MM)
    F, U, W = np.zeros((sys.n, 3)), np.zeros(1), np.zeros(9)
    ex = _i(sys.excl)
    lib().orc_exclusions(len(ex), _pi(ex), _pd(pos), _pd(_d(sys.q)), _pd(h), params.M, _pd(wt),
                         _pd(st), params.ME, _pd(w), _pd(s), params.ke, _pd(F), _pd(U), _pd(W))
    return F, U[0], W.reshape(3, 3)


def bonded(sys, pos=None, h=None):
    pos = _d(sys.pos if pos is None else pos)
    h = _d(box_matrix(sys.box) if h is None else h)
    F, en, W = np.zeros((sys.n, 3)), np.zeros(2), np.zeros(9)
    b, a = _i(sys.bonds), _i(sys.angles)
    lib().orc_bonded(len(b), _pi(b), _pd(_d(sys.bond_k)), _pd(_d(sys.bond_r0)), len(a), _pi(a),
                     _pd(_d(sys.angle_k)), _pd(_d(sys.angle_t0)), _pd(pos), _pd(h), _pd(F),
                     _pd(en), _pd(W))
    return F, en, W.reshape(3, 3)


class _SysHold:
    """Keeps the numpy arrays behind a _System alive."""

    def __init__(self, sys):
        self.arrs = dict(q=_d(sys.q), mass=_d(sys.mass), type=_i(sys.type), mol=_i(sys.mol),
                         eps=_d(sys.lj_eps), sig=_d(sys.lj_sig), bonds=_i(sys.bonds),
                         bk=_d(sys.bond_k), br=_d(sys.bond_r0), angles=_i(sys.angles),
                         ak=_d(sys.angle_k), at=_d(sys.angle_t0), excl=_i(sys.excl))
        a = self.arrs
        self.c = _System(sys.n, _pd(a["q"]), _pd(a["mass"]), _pi(a["type"]), _pi(a["mol"]),
                         sys.ntypes, _pd(a["eps"]), _pd(a["sig"]),
                         len(a["bonds"]), _pi(a["bonds"]), _pd(a["bk"]), _pd(a["br"]),
                         len(a["angles"]), _pi(a["angles"]), _pd(a["ak"]), _pd(a["at"]),
                         len(a["excl"]), _pi(a["excl"]))


EN_KEYS = ("coul_short", "coul_long", "coul_self", "coul_excl", "lj", "bond", "angle",
           "coul", "n_distinct")


def force_eval(sys, params: Params, step, pos=None, L=None):
    """One force evaluation (Algorithm 1, steps 2-7).

    Returns dict: F (N,3) kcal/mol/A; energies (kcal/mol); W (3,3) total
    virial kcal/mol; W_parts (5,3,3) = short-range Coulomb, radial estimator,
    non-radial estimator, LJ, bonded + exclusions; P (3,3) atm (virial part);
    modes m^r, m^nr."""
    pos = _d(sys.pos if pos is None else pos)
    L = _d(sys.box if L is None else L)
    hold = _SysHold(sys)
    pc = params.c()
    F, en, W, Wp = np.zeros((sys.n, 3)), np.zeros(9), np.zeros(9), np.zeros(45)
    modes = np.zeros(6 * params.P, np.int32)
    lib().orc_force_eval(C.byref(pc), C.byref(hold.c), _pd(pos), _pd(L), step, _pd(F),
                         _pd(en), _pd(W), _pd(Wp), _pi(modes))
    V = float(np.prod(L))
    out = {k: en[i] for i, k in enumerate(EN_KEYS)}
    out.update(F=F, W=W.reshape(3, 3), W_parts=Wp.reshape(5, 3, 3),
               P=W.reshape(3, 3) / V * NKTV2P,
               mr=modes[:3 * params.P].reshape(-1, 3), mnr=modes[3 * params.P:].reshape(-1, 3))
    return out


@dataclasses.dataclass
class Integ:
    """Langevin NPT settings (eq. Langevin_NPT; constants are our reading)."""
    dt: float = 1.0
    T: float = 300.0
    Pext_atm: float = 1.0
    gamma: float = 1.0 / 100.0       # 1/fs, thermostat time 0.1 ps
    gamma_box: float = 1.0 / 500.0   # 1/fs, barostat time 0.5 ps
    coupling: int = 0
    Mbox: tuple = (0.0, 0.0, 0.0)

    def c(self):
        return _Integ(self.dt, self.T, self.Pext_atm, self.gamma, self.gamma_box, self.coupling,
                      (C.c_double * 3)(*self.Mbox), KB, FTM2V, NKTV2P)


def npt_run(sys, params: Params, integ: Integ, state: dict, step0: int, nsteps: int):
    """Advance ``state`` (dict with r, p, L, ph, F, W) in place by nsteps."""
    hold = _SysHold(sys)
    pc, ic = params.c(), integ.c()
    for k in ("r", "p", "L", "ph", "F", "W"):
        state[k] = _d(state[k])
    en, K = np.zeros(9), np.zeros(9)
    lib().orc_npt_run(C.byref(pc), C.byref(hold.c), C.byref(ic), _pd(state["r"]),
                      _pd(state["p"]), _pd(state["L"]), _pd(state["ph"]), _pd(state["F"]),
                      _pd(state["W"]), step0, nsteps, _pd(en), _pd(K))
    state["en"] = {k: en[i] for i, k in enumerate(EN_KEYS)}
    state["K"] = K.reshape(3, 3)
    return state


# ---------------------------------------------------------------------------
# a general (triclinic) cell h: upper triangular, cell vectors as columns
# ---------------------------------------------------------------------------

def tilted_box(L, tilt):
    """h for edge lengths L = (Lx, Ly, Lz) and LAMMPS tilts (xy, xz, yz)."""
    Lx, Ly, Lz = L
    xy, xz, yz = tilt
    return np.array([[Lx, xy, xz], [0.0, Ly, yz], [0.0, 0.0, Lz]])


def tri_q(h, st0, m, nq=20):
    """q(m*) of eq. proposal for a general h (nq Gauss-Legendre nodes per axis)."""
    return lib().orc_tri_q(_pd(_d(h)), float(st0), _pi(_i(m)), int(nq))


class TriCell:
    """Sums of the sampler for one cell h and SOG split (orc_tri_create)."""

    def __init__(self, h, params: Params):
        w, s, wt, st = sog_terms(params.b, params.sigma, params.omega, params.M)
        self.h = _d(h)
        self.params = params
        self.st = st
        self._p = lib().orc_tri_create(_pd(self.h), params.M, _pd(wt), _pd(st))
        if not self._p:
            raise ValueError("h must be upper triangular with 1 <= M <= the oracle's maximum")

    def __del__(self):
        if getattr(self, "_p", None):
            lib().orc_tri_free(self._p)
            self._p = None

    def normalizers(self):
        M = self.params.M
        Hr, Hnr, mm = np.zeros(M), np.zeros(M), np.zeros(3, np.int32)
        lib().orc_tri_normalizers(self._p, _pd(Hr), _pd(Hnr), _pi(mm))
        return Hr, Hnr, mm

    def targets(self, m):
        out = np.zeros(3)
        lib().orc_tri_targets(self._p, _pi(_i(m)), _pd(out))
        return out

    def draw_r(self, step, index, sysid=None):
        m = np.zeros(3, np.int32)
        lib().orc_tri_draw_r(self._p, self.params.seed, self.params.sysid if sysid is None else sysid,
                             step, index, _pi(m))
        return m

    def sample_modes(self, step, sysid=None):
        P = self.params.P
        mr, mnr, stats = np.zeros((P, 3), np.int32), np.zeros((P, 3), np.int32), np.zeros(2)
        lib().orc_tri_sample_modes(self._p, P, self.params.seed,
                                   self.params.sysid if sysid is None else sysid, step,
                                   _pi(mr), _pi(mnr), _pd(stats))
        return mr, mnr, stats


def rho_h(pos, q, h, D):
    pos, q, D = _d(pos), _d(q), _i(D)
    out = np.zeros(2 * len(D))
    lib().orc_rho_h(len(q), _pd(pos), _pd(q), _pd(_d(h)), len(D), _pi(D), _pd(out))
    return out[0::2] + 1j * out[1::2]


def rb_longrange_h(pos, q, h, P, D, cr, cnr, Sr, Snr, ke=KE):
    """rb_longrange for a general h: (F, U^F*, W^{F,r*}, W^{F,nr*}, rho)."""
    pos, q, D = _d(pos), _d(q), _i(D)
    F, out, Wr, Wnr = np.zeros((len(q), 3)), np.zeros(1), np.zeros(9), np.zeros(9)
    rho_ = np.zeros(2 * len(D))
    lib().orc_rb_longrange_h(len(q), _pd(pos), _pd(q), _pd(_d(h)), P, len(D), _pi(D), _pi(_i(cr)),
                             _pi(_i(cnr)), Sr, Snr, ke, _pd(F), _pd(out), _pd(Wr), _pd(Wnr), _pd(rho_))
    return F, out[0], Wr.reshape(3, 3), Wnr.reshape(3, 3), rho_[0::2] + 1j * rho_[1::2]


def force_eval_h(sys, params: Params, step, cell: TriCell, pos=None):
    """force_eval for the general cell of `cell` (the paper's sampler)."""
    pos = _d(sys.pos if pos is None else pos)
    hold = _SysHold(sys)
    pc = params.c()
    F, en, W, Wp = np.zeros((sys.n, 3)), np.zeros(9), np.zeros(9), np.zeros(45)
    modes = np.zeros(6 * params.P, np.int32)
    lib().orc_force_eval_h(C.byref(pc), C.byref(hold.c), _pd(pos), _pd(cell.h), cell._p, step, _pd(F),
                           _pd(en), _pd(W), _pd(Wp), _pi(modes))
    V = float(abs(np.linalg.det(cell.h)))
    out = {k: en[i] for i, k in enumerate(EN_KEYS)}
    out.update(F=F, W=W.reshape(3, 3), W_parts=Wp.reshape(5, 3, 3),
               P=W.reshape(3, 3) / V * NKTV2P,
               mr=modes[:3 * params.P].reshape(-1, 3), mnr=modes[3 * params.P:].reshape(-1, 3))
    return out


def nvt_run_h(sys, params: Params, integ: "Integ", cell: TriCell, state: dict, step0: int, nsteps: int):
    """Langevin steps step0+1 .. step0+nsteps in the fixed cell of `cell`.
    state: r, p, F, W (updated in place); returns (energies, K)."""
    hold = _SysHold(sys)
    pc, ic = params.c(), integ.c()
    en, K = np.zeros(9), np.zeros(9)
    for k in ("r", "p", "F", "W"):
        state[k] = np.ascontiguousarray(state[k], dtype=np.float64)
    lib().orc_nvt_run_h(C.byref(pc), C.byref(hold.c), C.byref(ic), cell._p, _pd(state["r"]), _pd(state["p"]),
                        _pd(state["F"]), _pd(state["W"]), step0, nsteps, _pd(en), _pd(K))
    return {k: en[i] for i, k in enumerate(EN_KEYS)}, K.reshape(3, 3)
