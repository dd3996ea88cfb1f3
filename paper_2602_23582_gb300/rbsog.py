"""Thin ctypes binding of ``include/rbsog.h`` (argument marshalling only).

Every computation runs in ``librbsog.so`` (hand-written sm_103a kernels).  If
the library is missing this module raises: there is no CPU fallback.

Functions keep the C names; ``Context`` is a small convenience holder that
keeps the host arrays of a ``rbsog_create`` call alive and converts results
to numpy.  Device buffers may be passed as torch CUDA tensors (their
``data_ptr()`` is forwarded) -- PyTorch serves as device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librbsog.so")

RBSOG_OK = 0
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "EBOX", -4: "ENONFINITE", -5: "EUNSUPPORTED",
          -6: "ETIMEOUT", -7: "ECUDA", -8: "EOVERFLOW"}
RBSOG_SAMPLER_PAPER, RBSOG_SAMPLER_IID, RBSOG_SAMPLER_IID_RECAL = 0, 1, 2
RBSOG_FP64, RBSOG_FP32 = 0, 1
RBSOG_COUPLE_ISO, RBSOG_COUPLE_SEMI_ISO, RBSOG_COUPLE_FIXED = 0, 1, 2
E_NAMES = ("coul_short", "coul_long", "coul_self", "coul_excl", "lj", "bond", "angle", "coul", "kinetic")

EXPORTS = ("rbsog_default_params", "rbsog_create", "rbsog_destroy", "rbsog_last_error", "rbsog_n_atoms",
           "rbsog_system_range", "rbsog_set_box", "rbsog_set_positions", "rbsog_get_positions",
           "rbsog_get_velocities", "rbsog_step", "rbsog_step_forces", "rbsog_run", "rbsog_get_state", "rbsog_set_state",
           "rbsog_debug_cells", "rbsog_debug_modes", "rbsog_debug_device_alloc_calls", "rbsog_virial_nr_shared", "rbsog_set_timing", "rbsog_get_timing",
           "rbsog_structure_factor_workspace", "rbsog_structure_factor", "rbsog_run_async",
           "rbsog_sync", "rbsog_stream", "rbsog_structure_factor_noalloc", "rbsog_trace_pair",
           "rbsog_trace_pair_times", "rbsog_set_thermo_every", "rbsog_pool_create", "rbsog_pool_load",
           "rbsog_pool_prime", "rbsog_pool_state", "rbsog_pool_unload", "rbsog_server_create",
           "rbsog_server_destroy", "rbsog_server_slots", "rbsog_server_context", "rbsog_server_submit",
           "rbsog_server_pump", "rbsog_server_result", "rbsog_server_stats", "rbsog_modes_capacity",
           "rbsog_modes", "rbsog_longrange_force_workspace", "rbsog_longrange_force", "rbsog_autotune",
           "rbsog_sync_timeout")


class RbsogError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"rbsog status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class rbsog_slot_caps(C.Structure):
    _fields_ = [("max_atoms", C.c_int), ("max_molecules", C.c_int), ("max_bonds", C.c_int),
                ("max_angles", C.c_int), ("max_excl", C.c_int), ("max_types", C.c_int),
                ("max_box", C.c_double * 3), ("max_density", C.c_double)]


class rbsog_params(C.Structure):
    _fields_ = [("rc", C.c_double), ("b", C.c_double), ("sigma", C.c_double), ("omega", C.c_double),
                ("M", C.c_int), ("M_energy", C.c_int), ("P", C.c_int), ("sampler", C.c_int),
                ("seed", C.c_uint64), ("precision", C.c_int), ("ke", C.c_double),
                ("dt", C.c_double), ("T", C.c_double), ("P_ext", C.c_double), ("gamma", C.c_double),
                ("gamma_box", C.c_double), ("tau_box", C.c_double), ("compressibility", C.c_double),
                ("coupling", C.c_int), ("cell_sub", C.c_int), ("thermo_every", C.c_int), ("skin", C.c_double),
                ("cluster_cols", C.c_int)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


class rbsog_system_desc(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("q", _D), ("mass", _D), ("type", _I), ("mol", _I),
                ("ntypes", C.c_int), ("lj_eps", _D), ("lj_sig", _D),
                ("n_bonds", C.c_int), ("bonds", _I), ("bond_k", _D), ("bond_r0", _D),
                ("n_angles", C.c_int), ("angles", _I), ("angle_k", _D), ("angle_t0", _D),
                ("n_excl", C.c_int), ("excl", _I), ("r0", _D), ("v0", _D), ("box", C.c_double * 3),
                ("rng_id", C.c_uint64), ("tilt", C.c_double * 3)]


class rbsog_result(C.Structure):
    _fields_ = [("energy", C.c_double * 9), ("virial", C.c_double * 9),
                ("virial_coul_short", C.c_double * 9), ("virial_long_r", C.c_double * 9),
                ("virial_long_nr", C.c_double * 9), ("virial_lj", C.c_double * 9),
                ("virial_bonded", C.c_double * 9), ("pressure", C.c_double * 9),
                ("box", C.c_double * 3), ("volume", C.c_double), ("n_distinct_modes", C.c_int),
                ("n_accept_r", C.c_int), ("n_accept_nr", C.c_int), ("step", C.c_uint64),
                ("list_builds", C.c_int), ("tilt", C.c_double * 3)]


_lib = None


def lib():
    """Load librbsog.so (building it first if a source is newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2602_23582_gb300/build.py")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.rbsog_default_params.argtypes = [C.POINTER(rbsog_params), C.c_double]
    L.rbsog_default_params.restype = None
    L.rbsog_create.argtypes = [C.POINTER(rbsog_params), C.c_int, C.POINTER(rbsog_system_desc), P, C.POINTER(P)]
    L.rbsog_destroy.argtypes = [P]
    L.rbsog_destroy.restype = None
    L.rbsog_last_error.argtypes = [P]
    L.rbsog_last_error.restype = C.c_char_p
    L.rbsog_n_atoms.argtypes = [P]
    L.rbsog_system_range.argtypes = [P, C.c_int, _I, _I]
    L.rbsog_debug_device_alloc_calls.argtypes = []
    L.rbsog_debug_device_alloc_calls.restype = C.c_ulonglong
    L.rbsog_set_box.argtypes = [P, C.c_int, _D, C.c_int]
    L.rbsog_set_positions.argtypes = [P, P, C.c_int]
    L.rbsog_get_positions.argtypes = [P, P, C.c_int]
    L.rbsog_get_velocities.argtypes = [P, P, C.c_int]
    L.rbsog_step.argtypes = [P, C.c_uint64, P, C.c_int, C.POINTER(rbsog_result)]
    L.rbsog_step_forces.argtypes = [P, C.c_uint64, P, C.c_int, P]
    L.rbsog_run.argtypes = [P, C.c_int, C.POINTER(rbsog_result)]
    L.rbsog_run_async.argtypes = [P, C.c_int]
    L.rbsog_sync.argtypes = [P]
    L.rbsog_stream.argtypes = [P]
    L.rbsog_stream.restype = C.c_void_p
    L.rbsog_get_state.argtypes = [P, P, C.POINTER(C.c_size_t)]
    L.rbsog_set_state.argtypes = [P, P, C.c_size_t]
    L.rbsog_debug_cells.argtypes = [P, C.c_int, _I, _I]
    L.rbsog_debug_modes.argtypes = [P, C.c_int, _I, _I, _I, _I, _I, _I, _D, _D]
    L.rbsog_virial_nr_shared.argtypes = [P, _D]
    L.rbsog_set_timing.argtypes = [P, C.c_int]
    L.rbsog_get_timing.argtypes = [P, C.c_int, C.c_char_p, _D, _I]
    L.rbsog_structure_factor_workspace.argtypes = [C.c_int, C.c_int]
    L.rbsog_structure_factor_workspace.restype = C.c_size_t
    L.rbsog_structure_factor.argtypes = [P, P, C.c_int, _D, P, C.c_int, P, P, C.c_int, P]
    L.rbsog_structure_factor_noalloc.argtypes = [P, P, C.c_int, _D, P, C.c_int, P, C.c_int, P]
    L.rbsog_trace_pair.argtypes = [P, C.c_int]
    L.rbsog_set_thermo_every.argtypes = [P, C.c_int]
    L.rbsog_pool_create.argtypes = [C.POINTER(rbsog_params), C.c_int, C.POINTER(rbsog_slot_caps), P, C.POINTER(P)]
    L.rbsog_pool_load.argtypes = [P, C.c_int, C.POINTER(rbsog_system_desc), C.c_int]
    L.rbsog_pool_prime.argtypes = [P]
    L.rbsog_pool_state.argtypes = [P, _I, C.POINTER(C.c_ulonglong), _I]
    L.rbsog_pool_unload.argtypes = [P, C.c_int, _D, _D, C.POINTER(rbsog_result)]
    L.rbsog_server_create.argtypes = [C.POINTER(rbsog_params), C.c_int, C.POINTER(rbsog_slot_caps), C.c_double,
                                      P, C.POINTER(P)]
    L.rbsog_server_destroy.argtypes = [P]
    L.rbsog_server_destroy.restype = None
    L.rbsog_server_slots.argtypes = [P]
    L.rbsog_server_context.argtypes = [P]
    L.rbsog_server_context.restype = P
    L.rbsog_server_submit.argtypes = [P, C.POINTER(rbsog_system_desc), C.c_int, C.POINTER(C.c_longlong)]
    L.rbsog_server_pump.argtypes = [P, C.c_int, _I, _I]
    L.rbsog_server_result.argtypes = [P, C.c_longlong, _I, _D, _D, C.POINTER(rbsog_result)]
    L.rbsog_server_stats.argtypes = [P, _D, _D, _D, C.POINTER(C.c_longlong), _I]
    L.rbsog_trace_pair_times.argtypes = [P, C.c_int, _D, _I]
    L.rbsog_sync_timeout.argtypes = [P, C.c_double]
    L.rbsog_autotune.argtypes = [C.POINTER(rbsog_params), C.c_int, C.POINTER(rbsog_system_desc), C.c_int, P,
                                 C.POINTER(rbsog_params), _D]
    L.rbsog_modes_capacity.argtypes = [C.POINTER(rbsog_params)]
    L.rbsog_modes.argtypes = [C.POINTER(rbsog_params), _D, C.c_uint64, C.c_uint64, _I, _I, _I, _I, _D, P]
    L.rbsog_longrange_force_workspace.argtypes = [C.c_int]
    L.rbsog_longrange_force_workspace.restype = C.c_size_t
    L.rbsog_longrange_force.argtypes = [P, P, C.c_int, _D, P, P, P, C.c_int, P, C.c_int, C.c_double, C.c_double,
                                        C.c_double, P, _D, P, C.c_int, P]
    _lib = L
    return L


def _check(status, ctx=None):
    if status != RBSOG_OK:
        msg = lib().rbsog_last_error(ctx).decode() if ctx else ""
        raise RbsogError(status, msg)


def _ptr(x):
    """Pointer of a numpy array (host) or a torch CUDA tensor (device)."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        return C.c_void_p(x.data_ptr()), int(bool(x.is_cuda))
    return x.ctypes.data_as(C.c_void_p), 0


def rbsog_default_params(rc=10.0, **kw) -> rbsog_params:
    p = rbsog_params()
    lib().rbsog_default_params(C.byref(p), rc)
    names = {f[0] for f in rbsog_params._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"rbsog_params has no field {k!r}")
        setattr(p, k, v)
    return p


def _desc(sys, hold, index):
    def d(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        hold.append(a)
        return a.ctypes.data_as(_D)

    def i(a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        hold.append(a)
        return a.ctypes.data_as(_I)
    v0 = getattr(sys, "vel", None)
    desc = rbsog_system_desc()
    desc.n_atoms = sys.n
    desc.q, desc.mass, desc.type, desc.mol = d(sys.q), d(sys.mass), i(sys.type), i(sys.mol)
    desc.ntypes = sys.ntypes
    desc.lj_eps, desc.lj_sig = d(sys.lj_eps), d(sys.lj_sig)
    desc.n_bonds = len(sys.bonds)
    desc.bonds, desc.bond_k, desc.bond_r0 = i(sys.bonds), d(sys.bond_k), d(sys.bond_r0)
    desc.n_angles = len(sys.angles)
    desc.angles, desc.angle_k, desc.angle_t0 = i(sys.angles), d(sys.angle_k), d(sys.angle_t0)
    desc.n_excl = len(sys.excl)
    desc.excl = i(sys.excl)
    desc.r0 = d(sys.pos)
    desc.v0 = d(v0) if v0 is not None else None
    tilt = getattr(sys, "tilt", (0.0, 0.0, 0.0))
    for a in range(3):
        desc.box[a] = float(sys.box[a])
        desc.tilt[a] = float(tilt[a])
    desc.rng_id = int(getattr(sys, "rng_id", index))
    return desc


def rbsog_create(params: rbsog_params, systems, stream=None):
    """Create a context over a list of systems (duck-typed: pos, q, mass,
    type, mol, box, lj_eps, lj_sig, bonds, bond_k, bond_r0, angles, angle_k,
    angle_t0, excl; optional vel, rng_id -- the Philox key word, default
    the system's index -- and tilt = (xy, xz, yz) of a triclinic cell).
    Returns the opaque context pointer."""
    hold = []
    arr = (rbsog_system_desc * len(systems))()
    for k, s in enumerate(systems):
        arr[k] = _desc(s, hold, k)
    ctx = C.c_void_p()
    st = C.c_void_p(stream) if stream else None
    status = lib().rbsog_create(C.byref(params), len(systems), arr, st, C.byref(ctx))
    if status != RBSOG_OK:
        raise RbsogError(status, "rbsog_create: " + lib().rbsog_last_error(None).decode())
    return ctx


def rbsog_destroy(ctx):
    lib().rbsog_destroy(ctx)


def rbsog_step(ctx, step, forces=None, results=None):
    p, dev = _ptr(forces)
    _check(lib().rbsog_step(ctx, step, p, dev, results), ctx)


def rbsog_step_forces(ctx, step, forces=None, virial=None):
    p, dev = _ptr(forces)
    v = None if virial is None else virial.ctypes.data_as(C.c_void_p)
    _check(lib().rbsog_step_forces(ctx, step, p, dev, v), ctx)


def rbsog_run(ctx, nsteps, results=None):
    _check(lib().rbsog_run(ctx, nsteps, results), ctx)


def rbsog_run_async(ctx, nsteps):
    _check(lib().rbsog_run_async(ctx, nsteps), ctx)


def rbsog_sync(ctx):
    _check(lib().rbsog_sync(ctx), ctx)


def rbsog_stream(ctx):
    return lib().rbsog_stream(ctx)


def rbsog_set_positions(ctx, r):
    p, dev = _ptr(r)
    _check(lib().rbsog_set_positions(ctx, p, dev), ctx)


def rbsog_get_positions(ctx, r):
    p, dev = _ptr(r)
    _check(lib().rbsog_get_positions(ctx, p, dev), ctx)


def rbsog_get_velocities(ctx, v):
    p, dev = _ptr(v)
    _check(lib().rbsog_get_velocities(ctx, p, dev), ctx)


def rbsog_set_box(ctx, s, box, rescale=False):
    b = (C.c_double * 3)(*[float(x) for x in box])
    _check(lib().rbsog_set_box(ctx, s, b, int(rescale)), ctx)


def rbsog_get_state(ctx) -> bytes:
    n = C.c_size_t()
    _check(lib().rbsog_get_state(ctx, None, C.byref(n)), ctx)
    buf = (C.c_char * n.value)()
    _check(lib().rbsog_get_state(ctx, buf, C.byref(n)), ctx)
    return bytes(buf)


def rbsog_set_state(ctx, state: bytes):
    buf = (C.c_char * len(state)).from_buffer_copy(state)
    _check(lib().rbsog_set_state(ctx, buf, len(state)), ctx)


def rbsog_debug_cells(ctx, s, n_atoms):
    nc = np.zeros(3, np.int32)
    cell = np.zeros(n_atoms, np.int32)
    _check(lib().rbsog_debug_cells(ctx, s, nc.ctypes.data_as(_I), cell.ctypes.data_as(_I)), ctx)
    return nc, cell


def rbsog_debug_modes(ctx, s, P, Dcap):
    mr, mnr = np.zeros((P, 3), np.int32), np.zeros((P, 3), np.int32)
    D, cr, cnr = np.zeros((Dcap, 3), np.int32), np.zeros(Dcap, np.int32), np.zeros(Dcap, np.int32)
    nD = C.c_int()
    S2 = np.zeros(2)
    rho = np.zeros(2 * Dcap)
    _check(lib().rbsog_debug_modes(ctx, s, mr.ctypes.data_as(_I), mnr.ctypes.data_as(_I),
                                   D.ctypes.data_as(_I), cr.ctypes.data_as(_I), cnr.ctypes.data_as(_I),
                                   C.byref(nD), S2.ctypes.data_as(_D), rho.ctypes.data_as(_D)), ctx)
    n = nD.value
    return dict(mr=mr, mnr=mnr, D=D[:n].copy(), cr=cr[:n].copy(), cnr=cnr[:n].copy(), Sr=S2[0],
                Snr=S2[1], rho=rho[0:2 * n:2] + 1j * rho[1:2 * n:2])


def rbsog_virial_nr_shared(ctx, n_systems):
    out = np.zeros((n_systems, 3, 3))
    _check(lib().rbsog_virial_nr_shared(ctx, out.ctypes.data_as(_D)), ctx)
    return out


def rbsog_set_timing(ctx, enable=True):
    _check(lib().rbsog_set_timing(ctx, int(enable)), ctx)


def rbsog_get_timing(ctx, max_n=64):
    names = C.create_string_buffer(32 * max_n)
    ms = np.zeros(max_n)
    n = C.c_int()
    _check(lib().rbsog_get_timing(ctx, max_n, names, ms.ctypes.data_as(_D), C.byref(n)), ctx)
    raw = names.raw
    return [(raw[32 * k:32 * k + 32].split(b"\0")[0].decode(), ms[k]) for k in range(n.value)]


def rbsog_structure_factor_workspace(n_atoms, nD):
    return lib().rbsog_structure_factor_workspace(n_atoms, nD)


def _check_tensor(name, t, dtype, numel_min=None, numel_eq=None):
    """Refuse a device buffer the kernels would read or write out of bounds
    (or misread): not a torch tensor, wrong dtype, not contiguous, a wrong
    number of elements.  The device is checked apart (_check_devices), after
    every buffer has passed these checks."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != dtype:
        raise ValueError(f"{name}: expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if numel_eq is not None and t.numel() != numel_eq:
        raise ValueError(f"{name}: expected {numel_eq} elements, got {t.numel()}")
    if numel_min is not None and t.numel() < numel_min:
        raise ValueError(f"{name}: needs at least {numel_min} elements, got {t.numel()}")


def _check_devices(**tensors):
    """Every buffer must be CUDA device memory, all on one device."""
    for name, t in tensors.items():
        if not t.is_cuda:
            raise ValueError(f"{name}: must be a CUDA tensor (device memory), got device {t.device}")
    devs = {t.device for t in tensors.values()}
    if len(devs) != 1:
        raise ValueError(f"{', '.join(tensors)} must be on one device, got {sorted(str(d) for d in devs)}")


def _check_sf_args(r, q, box, m, rho, precision):
    """Arguments of the stateless structure factor: r float64 (n, 3), q
    float64 (n,), m int32 (nD, 3), rho float64 (>= 2 nD), box three positive
    finite edges, precision RBSOG_FP64 or RBSOG_FP32.  Returns (n, nD); the
    caller checks the devices."""
    import torch
    if precision not in (RBSOG_FP64, RBSOG_FP32):
        raise ValueError(f"precision: expected RBSOG_FP64 or RBSOG_FP32, got {precision!r}")
    b = np.asarray(box, dtype=np.float64).reshape(-1)
    if b.size != 3 or not np.all(np.isfinite(b)) or not np.all(b > 0):
        raise ValueError(f"box: expected three positive finite edge lengths, got {box!r}")
    if not isinstance(q, torch.Tensor) or q.numel() < 1:
        raise ValueError("q: expected a non-empty torch tensor of charges")
    n = int(q.numel())
    if not isinstance(m, torch.Tensor) or m.numel() < 3 or m.numel() % 3:
        raise ValueError("m: expected a torch tensor of shape (nD, 3), nD >= 1")
    nD = int(m.numel()) // 3
    _check_tensor("r", r, torch.float64, numel_eq=3 * n)
    _check_tensor("q", q, torch.float64, numel_eq=n)
    _check_tensor("m", m, torch.int32, numel_eq=3 * nD)
    _check_tensor("rho", rho, torch.float64, numel_min=2 * nD)
    return n, nD


def rbsog_structure_factor(r, q, box, m, rho, work, precision=RBSOG_FP32, stream=None):
    """r (n, 3) float64, q (n,) float64, m (nD, 3) int32, rho (2 nD,) float64
    and work (>= rbsog_structure_factor_workspace(n, nD) bytes, any dtype):
    contiguous torch CUDA tensors of one device.  Bad arguments raise
    ValueError before the library is called."""
    import torch
    n, nD = _check_sf_args(r, q, box, m, rho, precision)
    if not isinstance(work, torch.Tensor) or not work.is_contiguous():
        raise ValueError("work: expected a contiguous torch tensor")
    need = rbsog_structure_factor_workspace(n, nD)
    if work.numel() * work.element_size() < need:
        raise ValueError(f"work: needs {need} bytes, got {work.numel() * work.element_size()}")
    _check_devices(r=r, q=q, m=m, rho=rho, work=work)
    b = (C.c_double * 3)(*[float(x) for x in box])
    st = C.c_void_p(stream) if stream else None
    status = lib().rbsog_structure_factor(C.c_void_p(r.data_ptr()), C.c_void_p(q.data_ptr()), n,
                                          b, C.c_void_p(m.data_ptr()), nD,
                                          C.c_void_p(rho.data_ptr()), C.c_void_p(work.data_ptr()),
                                          precision, st)
    if status != RBSOG_OK:
        raise RbsogError(status, "rbsog_structure_factor")


def rbsog_set_thermo_every(ctx, every):
    _check(lib().rbsog_set_thermo_every(ctx, int(every)), ctx)


def rbsog_trace_pair(ctx, nsteps):
    _check(lib().rbsog_trace_pair(ctx, int(nsteps)), ctx)


def rbsog_trace_pair_times(ctx, max_steps):
    ms = np.zeros(max(int(max_steps), 1))
    n = C.c_int(0)
    _check(lib().rbsog_trace_pair_times(ctx, int(max_steps), ms.ctypes.data_as(_D), C.byref(n)), ctx)
    return ms[:n.value]


def rbsog_structure_factor_noalloc(r, q, box, m, rho, precision=RBSOG_FP32, stream=None):
    """As rbsog_structure_factor, with the library's fixed scratch instead of a
    caller workspace (no device allocation; calls on one device must not
    overlap in time).  Bad arguments raise ValueError before the library is
    called."""
    n, nD = _check_sf_args(r, q, box, m, rho, precision)
    _check_devices(r=r, q=q, m=m, rho=rho)
    b = (C.c_double * 3)(*[float(x) for x in box])
    st = C.c_void_p(stream) if stream else None
    status = lib().rbsog_structure_factor_noalloc(C.c_void_p(r.data_ptr()), C.c_void_p(q.data_ptr()),
                                                  n, b, C.c_void_p(m.data_ptr()), nD,
                                                  C.c_void_p(rho.data_ptr()), precision, st)
    if status != RBSOG_OK:
        raise RbsogError(status, lib().rbsog_last_error(None).decode())


def rbsog_sync_timeout(ctx, timeout_ms):
    """RBSOG_OK once the enqueued steps have finished (flags checked as by
    rbsog_sync), RBSOG_ETIMEOUT (returned, not raised) while they still run
    after timeout_ms; other errors raise."""
    st = lib().rbsog_sync_timeout(ctx, float(timeout_ms))
    if st not in (RBSOG_OK, -6):
        _check(st, ctx)
    return st


def rbsog_autotune(params: rbsog_params, systems, nsteps=10, stream=None):
    """Launch-shape search (cell_sub x cluster_cols): returns (best params,
    list of (cell_sub, cluster_cols, ms per step or None))."""
    hold = []
    descs = (rbsog_system_desc * len(systems))(*[_desc(s, hold, k) for k, s in enumerate(systems)])
    best = rbsog_params()
    f32 = params.precision == RBSOG_FP32
    cands = [(sub, col if f32 else 0) for sub in (1, 2) for col in ((1, 2, 3, 4) if f32 else (0,))]
    times = np.zeros(len(cands))
    st = C.c_void_p(stream) if stream else None
    _check(lib().rbsog_autotune(C.byref(params), len(systems), descs, int(nsteps), st, C.byref(best),
                                times.ctypes.data_as(_D)))
    return best, [(a, b, float(t) if t >= 0 else None) for (a, b), t in zip(cands, times)]


def rbsog_modes(params: rbsog_params, box, rng_id, step, stream=None):
    """The distinct modes of one evaluation (host arrays): dict with D (nD, 3),
    cr, cnr (nD,) and S = (S^r, S^nr)."""
    cap = lib().rbsog_modes_capacity(C.byref(params))
    D = np.zeros((cap, 3), np.int32)
    cr, cnr = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
    nD, S = C.c_int(0), np.zeros(2)
    b = (C.c_double * 3)(*[float(x) for x in box])
    st = C.c_void_p(stream) if stream else None
    status = lib().rbsog_modes(C.byref(params), b, int(rng_id), int(step), D.ctypes.data_as(_I),
                               cr.ctypes.data_as(_I), cnr.ctypes.data_as(_I), C.byref(nD),
                               S.ctypes.data_as(_D), st)
    if status != RBSOG_OK:
        raise RbsogError(status, lib().rbsog_last_error(None).decode())
    n = nD.value
    return dict(D=D[:n].copy(), cr=cr[:n].copy(), cnr=cnr[:n].copy(), S=(float(S[0]), float(S[1])))


def rbsog_longrange_force_workspace(nD):
    return lib().rbsog_longrange_force_workspace(int(nD))


def rbsog_longrange_force(r, q, box, m, cr, cnr, rho, P, Sr, Snr, ke, F, work, precision=RBSOG_FP64,
                          estimators=True, stream=None):
    """Long-range forces on the atoms (r, q) from the whole system's rho
    (device tensors: r (n, 3) / q (n,) / rho (2 nD,) / F (n, 3) float64, m
    (nD, 3) / cr / cnr (nD,) int32, work uint8 of the workspace size); returns
    (U^F*, V P^F,nr* as a 3x3 array) when estimators is set."""
    import torch
    n, nD = int(q.numel()), int(m.numel()) // 3
    if n > 0:
        _check_tensor("r", r, torch.float64, numel_eq=3 * n)
        _check_tensor("q", q, torch.float64, numel_eq=n)
        _check_tensor("F", F, torch.float64, numel_eq=3 * n)
    _check_tensor("m", m, torch.int32, numel_eq=3 * nD)
    _check_tensor("cr", cr, torch.int32, numel_eq=nD)
    if cnr is not None:
        _check_tensor("cnr", cnr, torch.int32, numel_eq=nD)
    _check_tensor("rho", rho, torch.float64, numel_min=2 * nD)
    need = lib().rbsog_longrange_force_workspace(nD)
    if not isinstance(work, torch.Tensor) or work.numel() * work.element_size() < need:
        raise ValueError(f"work: needs {need} bytes")
    devs = dict(m=m, cr=cr, rho=rho, work=work)
    if n > 0:
        devs.update(r=r, q=q, F=F)
    if cnr is not None:
        devs["cnr"] = cnr
    _check_devices(**devs)
    b = (C.c_double * 3)(*[float(x) for x in box])
    est = np.zeros(7)
    vp = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
    st = C.c_void_p(stream) if stream else None
    status = lib().rbsog_longrange_force(vp(r) if n else None, vp(q) if n else None, n, b, vp(m), vp(cr), vp(cnr),
                                         nD, vp(rho), int(P), float(Sr), float(Snr), float(ke),
                                         vp(F) if n else None, est.ctypes.data_as(_D) if estimators else None,
                                         vp(work), precision, st)
    if status != RBSOG_OK:
        raise RbsogError(status, lib().rbsog_last_error(None).decode())
    if estimators:
        W = np.array([[est[1], est[4], est[5]], [est[4], est[2], est[6]], [est[5], est[6], est[3]]])
        return float(est[0]), W
    return None


def result_dict(r: rbsog_result) -> dict:
    """rbsog_result -> numpy/dict (energies by name, 3x3 tensors)."""
    def t(x):
        return np.array(x[:]).reshape(3, 3)
    out = {k: r.energy[i] for i, k in enumerate(E_NAMES)}
    out.update(virial=t(r.virial), virial_coul_short=t(r.virial_coul_short),
               virial_long_r=t(r.virial_long_r), virial_long_nr=t(r.virial_long_nr),
               virial_lj=t(r.virial_lj), virial_bonded=t(r.virial_bonded), pressure=t(r.pressure),
               box=np.array(r.box[:]), volume=r.volume, n_distinct_modes=r.n_distinct_modes,
               n_accept_r=r.n_accept_r, n_accept_nr=r.n_accept_nr, step=r.step, list_builds=r.list_builds,
               tilt=np.array(r.tilt[:]))
    return out


def slot_caps(max_atoms, max_box, max_molecules=None, max_bonds=None, max_angles=None, max_excl=None,
              max_types=4, max_density=0.12) -> rbsog_slot_caps:
    """Capacities of one slot; term limits default to generous multiples of the atoms."""
    c = rbsog_slot_caps()
    c.max_atoms = int(max_atoms)
    c.max_molecules = int(max_molecules if max_molecules is not None else max_atoms)
    c.max_bonds = int(max_bonds if max_bonds is not None else max_atoms)
    c.max_angles = int(max_angles if max_angles is not None else max_atoms)
    c.max_excl = int(max_excl if max_excl is not None else 2 * max_atoms)
    c.max_types = int(max_types)
    c.max_density = float(max_density)
    for a in range(3):
        c.max_box[a] = float(max_box[a] if hasattr(max_box, "__len__") else max_box)
    return c


class Pool:
    """A pool context: slots loaded and emptied at run time (served path)."""

    def __init__(self, caps, params: rbsog_params | None = None, stream=None, **kw):
        self.params = params if params is not None else rbsog_default_params(**kw)
        arr = (rbsog_slot_caps * len(caps))(*caps)
        self.ctx = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        _check(lib().rbsog_pool_create(C.byref(self.params), len(caps), arr, st, C.byref(self.ctx)))
        self.S = len(caps)
        self.systems = [None] * self.S

    def load(self, slot, system, nsteps=-1, index=None):
        hold = []
        d = _desc(system, hold, slot if index is None else index)
        _check(lib().rbsog_pool_load(self.ctx, int(slot), C.byref(d), int(nsteps)), self.ctx)
        self.systems[slot] = system

    def prime(self):
        _check(lib().rbsog_pool_prime(self.ctx), self.ctx)

    def run(self, nsteps):
        res = (rbsog_result * self.S)()
        _check(lib().rbsog_run(self.ctx, int(nsteps), res), self.ctx)
        return [result_dict(res[k]) for k in range(self.S)]

    def state(self):
        """(state per slot: 0 empty, 1 running, 2 finished, 3 failed; Philox counters; error codes)."""
        st = np.zeros(self.S, dtype=np.int32)
        err = np.zeros(self.S, dtype=np.int32)
        steps = (C.c_ulonglong * self.S)()
        _check(lib().rbsog_pool_state(self.ctx, st.ctypes.data_as(_I), steps, err.ctypes.data_as(_I)), self.ctx)
        return st, np.array(steps[:], dtype=np.uint64), err

    def unload(self, slot):
        n = self.systems[slot].n
        r = np.zeros((n, 3))
        v = np.zeros((n, 3))
        res = rbsog_result()
        _check(lib().rbsog_pool_unload(self.ctx, int(slot), r.ctypes.data_as(_D), v.ctypes.data_as(_D),
                                       C.byref(res)), self.ctx)
        self.systems[slot] = None
        return r, v, result_dict(res)

    def close(self):
        if self.ctx:
            rbsog_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop of the served path (continuous batching over a pool)."""

    def __init__(self, caps, params: rbsog_params | None = None, hbm_fraction=0.5, stream=None, **kw):
        self.params = params if params is not None else rbsog_default_params(**kw)
        arr = (rbsog_slot_caps * len(caps))(*caps)
        self.srv = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        status = lib().rbsog_server_create(C.byref(self.params), len(caps), arr, float(hbm_fraction), st,
                                           C.byref(self.srv))
        if status != RBSOG_OK:
            raise RbsogError(status, "rbsog_server_create: " + lib().rbsog_last_error(None).decode())
        self.sizes = {}

    @property
    def slots(self):
        return lib().rbsog_server_slots(self.srv)

    def submit(self, system, nsteps, rng_id=None):
        hold = []
        d = _desc(system, hold, 0)
        if rng_id is not None:
            d.rng_id = int(rng_id)
        t = C.c_longlong()
        _check(lib().rbsog_server_submit(self.srv, C.byref(d), int(nsteps), C.byref(t)))
        self.sizes[t.value] = system.n
        return t.value

    def pump(self, max_steps):
        run = C.c_int()
        que = C.c_int()
        status = lib().rbsog_server_pump(self.srv, int(max_steps), C.byref(run), C.byref(que))
        if status != RBSOG_OK:
            raise RbsogError(status, lib().rbsog_last_error(lib().rbsog_server_context(self.srv)).decode())
        return run.value, que.value

    def result(self, ticket):
        n = self.sizes[ticket]
        done = C.c_int()
        r = np.zeros((n, 3))
        v = np.zeros((n, 3))
        res = rbsog_result()
        status = lib().rbsog_server_result(self.srv, int(ticket), C.byref(done), r.ctypes.data_as(_D),
                                           v.ctypes.data_as(_D), C.byref(res))
        if not done.value:
            if status != RBSOG_OK:
                raise RbsogError(status, "rbsog_server_result")
            return None
        out = result_dict(res)
        out["status"] = status                  # RBSOG_OK, or why the system was stopped early
        return r, v, out

    def stats(self):
        p50, p99, thr = C.c_double(), C.c_double(), C.c_double()
        n = C.c_longlong()
        failed = C.c_int()
        _check(lib().rbsog_server_stats(self.srv, C.byref(p50), C.byref(p99), C.byref(thr), C.byref(n),
                                        C.byref(failed)))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "atom_steps_per_s": thr.value, "steps": n.value,
                "failed": failed.value}

    def close(self):
        if self.srv:
            lib().rbsog_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """Owner of one rbsog context (n systems)."""

    def __init__(self, systems, params: rbsog_params | None = None, stream=None, **kw):
        self.params = params if params is not None else rbsog_default_params(**kw)
        self.systems = list(systems)
        self.ctx = rbsog_create(self.params, self.systems, stream)
        self.n_atoms = lib().rbsog_n_atoms(self.ctx)
        self.S = len(self.systems)
        self.Dcap = 2 * self.params.P if self.params.sampler == RBSOG_SAMPLER_IID else self.params.P + 1

    def close(self):
        if self.ctx:
            rbsog_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, step, forces=None):
        res = (rbsog_result * self.S)()
        if forces is None:
            forces = np.zeros((self.n_atoms, 3))
        rbsog_step(self.ctx, step, forces, res)
        return forces, [result_dict(res[k]) for k in range(self.S)]

    def step_forces(self, step, forces=None):
        """Force-only evaluation: forces (N x 3) and per-system virial (S x 3 x 3)."""
        if forces is None:
            forces = np.zeros((self.n_atoms, 3))
        virial = np.zeros((self.S, 3, 3))
        rbsog_step_forces(self.ctx, step, forces, virial)
        return forces, virial

    def run(self, nsteps):
        res = (rbsog_result * self.S)()
        rbsog_run(self.ctx, nsteps, res)
        return [result_dict(res[k]) for k in range(self.S)]

    def positions(self):
        r = np.zeros((self.n_atoms, 3))
        rbsog_get_positions(self.ctx, r)
        return r

    def velocities(self):
        v = np.zeros((self.n_atoms, 3))
        rbsog_get_velocities(self.ctx, v)
        return v

    def set_positions(self, r):
        rbsog_set_positions(self.ctx, np.ascontiguousarray(r, dtype=np.float64))

    def cells(self, s=0):
        return rbsog_debug_cells(self.ctx, s, self.systems[s].n)

    def modes(self, s=0):
        return rbsog_debug_modes(self.ctx, s, self.params.P, self.Dcap)

    def virial_nr_shared(self):
        """V P^F,nr of the last evaluation by the shared-proposal estimator (S, 3, 3)."""
        return rbsog_virial_nr_shared(self.ctx, self.S)
