"""The Python binding refuses device buffers that the stateless kernels
would read or write out of bounds, or misread, before it calls the library:
wrong dtype, wrong element count, not contiguous, not on a CUDA device, a
bad box or precision, and (for the workspace call) a short workspace.  Runs
on CPU: every refusal happens in argument marshalling, so nothing is ever
launched; a call that reached the library without a GPU would fail with a
CUDA status instead of ValueError."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2602_23582_gb300 import rbsog as R  # noqa: E402


def _good(n=10, nD=4):
    return dict(r=torch.zeros((n, 3), dtype=torch.float64), q=torch.zeros(n, dtype=torch.float64),
                m=torch.ones((nD, 3), dtype=torch.int32), rho=torch.zeros(2 * nD, dtype=torch.float64))


def _call(noalloc, a, box=(30.0, 30.0, 30.0), precision=R.RBSOG_FP64, work=None):
    if noalloc:
        R.rbsog_structure_factor_noalloc(a["r"], a["q"], box, a["m"], a["rho"], precision=precision)
    else:
        if work is None:
            work = torch.zeros(R.rbsog_structure_factor_workspace(a["q"].numel(), a["m"].numel() // 3),
                               dtype=torch.uint8)
        R.rbsog_structure_factor(a["r"], a["q"], box, a["m"], a["rho"], work, precision=precision)


BAD = {
    "r float32": ("r", lambda a: a["r"].float(), "dtype"),
    "q float32": ("q", lambda a: a["q"].float(), "dtype"),
    "m int64 (torch default)": ("m", lambda a: a["m"].long(), "dtype"),
    "rho float32": ("rho", lambda a: a["rho"].float(), "dtype"),
    "r short": ("r", lambda a: a["r"][:-1], "elements"),
    "r not contiguous": ("r", lambda a: a["r"].t().contiguous().t(), "contiguous"),
    "rho short": ("rho", lambda a: a["rho"][:-1], "elements"),
    "m not (nD, 3)": ("m", lambda a: a["m"].reshape(-1)[:-1], "m:"),
}


@pytest.mark.parametrize("noalloc", [False, True])
@pytest.mark.parametrize("case", list(BAD))
def test_bad_buffer_is_refused_before_the_call(case, noalloc):
    key, mutate, word = BAD[case]
    a = _good()
    a[key] = mutate(a)
    with pytest.raises(ValueError) as e:
        _call(noalloc, a)
    assert word in str(e.value), str(e.value)


@pytest.mark.parametrize("noalloc", [False, True])
def test_host_buffers_are_refused(noalloc):
    # every check but the device passes: CPU tensors are host memory
    with pytest.raises(ValueError) as e:
        _call(noalloc, _good())
    assert "CUDA" in str(e.value)


@pytest.mark.parametrize("box", [(30.0, 30.0), (30.0, -1.0, 30.0), (30.0, np.nan, 30.0)])
def test_bad_box_is_refused(box):
    with pytest.raises(ValueError) as e:
        _call(True, _good(), box=box)
    assert "box" in str(e.value)


def test_bad_precision_is_refused():
    with pytest.raises(ValueError) as e:
        _call(False, _good(), precision=7)
    assert "precision" in str(e.value)


def test_short_workspace_is_refused():
    a = _good()
    need = R.rbsog_structure_factor_workspace(10, 4)
    with pytest.raises(ValueError) as e:
        _call(False, a, work=torch.zeros(need - 1, dtype=torch.uint8))
    assert "work" in str(e.value)
