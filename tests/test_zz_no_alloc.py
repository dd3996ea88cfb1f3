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
    for k in (1, 2):                                   # two calls in a row
        R.rbsog_structure_factor_noalloc(r, q, s.box, mt, out[k], precision=prec)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
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
