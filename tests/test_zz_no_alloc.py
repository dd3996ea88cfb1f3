"""The allocation-free structure factor (rbsog_structure_factor_noalloc)
against the workspace entry point rbsog_structure_factor: same results on
two calls in a row, no change in device memory use, and a clear refusal of
sizes beyond its fixed scratch.  The file name keeps it last in collection so
that it also runs after every other test; it passes alone as well."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2602_23582_gb300 import rbsog as R  # noqa: E402


def _inputs(n_mol=3000, L=45.0, nmodes=57, seed=21):
    s = W.water(n_mol=n_mol, L=L, lattice=15, seed=seed)
    rng = np.random.default_rng(2)
    m = rng.integers(-9, 10, size=(nmodes, 3)).astype(np.int32)
    m[np.all(m == 0, axis=1)] = [1, 0, 0]
    return s, m


@pytest.mark.parametrize("prec,tol", [(R.RBSOG_FP64, 1e-11), (R.RBSOG_FP32, 2e-6)])
def test_noalloc_matches_workspace_entry_point(prec, tol):
    s, m = _inputs()
    dev = torch.device("cuda:0")
    r = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, device=dev)
    mt = torch.tensor(m, device=dev)
    ref = torch.zeros(2 * len(m), dtype=torch.float64, device=dev)
    work = torch.zeros(R.rbsog_structure_factor_workspace(s.n, len(m)), dtype=torch.uint8, device=dev)
    R.rbsog_structure_factor(r, q, s.box, mt, ref, work, precision=prec)
    out = [torch.full((2 * len(m),), np.nan, dtype=torch.float64, device=dev) for _ in range(3)]
    R.rbsog_structure_factor_noalloc(r, q, s.box, mt, out[0], precision=prec)   # may set up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    calls0 = R.lib().rbsog_debug_device_alloc_calls()
    for k in (1, 2):                                   # two calls in a row
        R.rbsog_structure_factor_noalloc(r, q, s.box, mt, out[k], precision=prec)
    torch.cuda.synchronize()
    # the library made no cudaMalloc or cudaFree call (its own counter), and
    # neither torch's allocator nor the device's free memory moved
    assert R.lib().rbsog_debug_device_alloc_calls() == calls0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    scale = float(np.abs(s.q).sum())
    g_ref = ref.cpu().numpy()
    for k in range(3):
        g = out[k].cpu().numpy()
        assert np.all(np.isfinite(g))
        assert np.abs(g - g_ref).max() < tol * scale, (prec, k)


def test_noalloc_refuses_sizes_beyond_its_scratch():
    dev = torch.device("cuda:0")
    n, nD = 200_000, 4000      # needs well over 4 MiB of scratch
    assert R.rbsog_structure_factor_workspace(n, nD) > 4 << 20
    r = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    q = torch.zeros(n, dtype=torch.float64, device=dev)
    m = torch.ones((nD, 3), dtype=torch.int32, device=dev)
    rho = torch.zeros(2 * nD, dtype=torch.float64, device=dev)
    with pytest.raises(R.RbsogError) as e:
        R.rbsog_structure_factor_noalloc(r, q, (50.0, 50.0, 50.0), m, rho)
    assert e.value.status == -8
    assert "scratch" in str(e.value)


_CHILD = r'''
import ctypes as C, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import workloads as W
from paper_2602_23582_gb300 import rbsog as R

cu = C.CDLL("libcuda.so.1")
def ck(r, what):
    if r != 0:
        raise SystemExit(f"{what}: CUresult {r}")
ck(cu.cuInit(0), "cuInit")
dev = C.c_int()
ck(cu.cuDeviceGet(C.byref(dev), 0), "cuDeviceGet")

def new_ctx():
    # a context of the caller's own (not the device's primary context); made current
    ctx = C.c_void_p()
    if hasattr(cu, "cuCtxCreate_v4"):
        ck(cu.cuCtxCreate_v4(C.byref(ctx), None, C.c_uint(0), dev), "cuCtxCreate_v4")
    else:
        ck(cu.cuCtxCreate_v2(C.byref(ctx), C.c_uint(0), dev), "cuCtxCreate_v2")
    return ctx

s = W.water(n_mol=2000, L=40.0, lattice=13, seed=23)
rng = np.random.default_rng(4)
m = rng.integers(-8, 9, size=(41, 3)).astype(np.int32)
m[np.all(m == 0, axis=1)] = [0, 1, 0]
n, nD = s.n, len(m)
lib = R.lib()
box = (C.c_double * 3)(*s.box)

def dmem(nbytes):
    p = C.c_uint64()
    ck(cu.cuMemAlloc_v2(C.byref(p), C.c_size_t(nbytes)), "cuMemAlloc")
    return p

def run_in_current(prec, tol):
    # both entry points in the current context, on its NULL stream; the
    # allocation-free one twice in a row
    pos, q = np.ascontiguousarray(s.pos), np.ascontiguousarray(s.q)
    bufs = {k: dmem(v) for k, v in dict(r=pos.nbytes, q=q.nbytes, m=m.nbytes, ref=16 * nD, a=16 * nD,
                                         b=16 * nD, work=lib.rbsog_structure_factor_workspace(n, nD)).items()}
    for k, arr in (("r", pos), ("q", q), ("m", m)):
        ck(cu.cuMemcpyHtoD_v2(bufs[k], arr.ctypes.data_as(C.c_void_p), C.c_size_t(arr.nbytes)), "HtoD")
    vp = lambda k: C.c_void_p(bufs[k].value)
    st = lib.rbsog_structure_factor(vp("r"), vp("q"), n, box, vp("m"), nD, vp("ref"), vp("work"), prec, None)
    assert st == 0, st
    for k in ("a", "b"):
        st = lib.rbsog_structure_factor_noalloc(vp("r"), vp("q"), n, box, vp("m"), nD, vp(k), prec, None)
        assert st == 0, (st, lib.rbsog_last_error(None))
    ck(cu.cuCtxSynchronize(), "sync")
    out = {}
    for k in ("ref", "a", "b"):
        h = np.empty(2 * nD)
        ck(cu.cuMemcpyDtoH_v2(h.ctypes.data_as(C.c_void_p), bufs[k], C.c_size_t(h.nbytes)), "DtoH")
        out[k] = h
    for v in bufs.values():
        ck(cu.cuMemFree_v2(v), "free")
    scale = float(np.abs(s.q).sum())
    for k in ("a", "b"):
        err = np.abs(out[k] - out["ref"]).max() / scale
        assert np.all(np.isfinite(out[k])) and err < tol, (k, err)

for prec, tol in ((0, 1e-12), (1, 2e-6)):
    A = new_ctx()
    run_in_current(prec, tol)          # first call in A: looks up A's scratch
    B = new_ctx()                      # now B is current
    run_in_current(prec, tol)          # B's scratch, not A's cached address
    ck(cu.cuCtxDestroy_v2(B), "destroy B")
    ck(cu.cuCtxSetCurrent(A), "set A")
    run_in_current(prec, tol)          # back in A
    ck(cu.cuCtxDestroy_v2(A), "destroy A")
print("ok")
'''


def test_noalloc_from_contexts_the_caller_creates():
    # The scratch is a module global, so each CUDA context has its own copy.
    # A host program that manages its own driver contexts calls in from A,
    # then from B, then from A again (after B is destroyed): every call must
    # use the scratch of the context it runs in.  Buffers come from the
    # driver (cuMemAlloc), the calls go through the C ABI; a fresh process
    # keeps torch's context out of it.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CHILD, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
