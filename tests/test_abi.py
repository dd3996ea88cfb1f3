"""CPU checks of the C ABI: the library builds and loads, exports every
function include/rbsog.h declares, the ctypes structures match the header's
layout, the default parameters are Table 2 row 2, and without a GPU the
library fails loudly with a status code (there is no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2602_23582_gb300 import build as B
from paper_2602_23582_gb300 import rbsog as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbsog.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbsog_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    B.build()
    lib = R.lib()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) == set(R.EXPORTS)


def test_struct_layout_matches_header(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rbsog.h"\n'
                    'int main(){printf("%zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(rbsog_params), sizeof(rbsog_result),'
                    ' sizeof(rbsog_system_desc), offsetof(rbsog_system_desc, rng_id),'
                    ' offsetof(rbsog_result, step), sizeof(rbsog_slot_caps), offsetof(rbsog_slot_caps, max_box),'
                    ' offsetof(rbsog_params, thermo_every));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(R.rbsog_params)
    assert out[1] == ctypes.sizeof(R.rbsog_result)
    assert out[2] == ctypes.sizeof(R.rbsog_system_desc)
    assert out[3] == R.rbsog_system_desc.rng_id.offset
    assert out[4] == R.rbsog_result.step.offset
    assert out[5] == ctypes.sizeof(R.rbsog_slot_caps)
    assert out[6] == R.rbsog_slot_caps.max_box.offset
    assert R.rbsog_slot_caps.max_density.offset == R.rbsog_slot_caps.max_box.offset + 24
    assert out[7] == R.rbsog_params.thermo_every.offset


def test_default_params_are_table2_row2(table2):
    p = R.rbsog_default_params(10.0)
    row = table2[1]
    assert p.b == row["b"] and p.omega == row["omega"]
    assert abs(p.sigma - row["sigma"] * 10.0 / 9.0) < 1e-15 * p.sigma
    assert p.M == 10 and p.M_energy == 10 and p.P == 100 and p.sampler == 0


def test_without_gpu_create_fails_loudly():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    import workloads as W
    s = W.electrolyte(n_ions=100, L=30.0, seed=1)
    with pytest.raises(R.RbsogError) as e:
        R.Context([s], R.rbsog_default_params(10.0))
    assert e.value.status in (-7, -2)


def test_invalid_arguments_are_rejected_before_any_device_call():
    import workloads as W
    s = W.electrolyte(n_ions=100, L=30.0, seed=1)
    for bad in (dict(P=0), dict(M=0), dict(M=70), dict(sampler=7), dict(precision=3), dict(cell_sub=3),
                dict(skin=-1.0), dict(skin=float("nan")), dict(skin=11.0)):
        p = R.rbsog_default_params(10.0, **bad)
        with pytest.raises(R.RbsogError) as e:
            R.rbsog_create(p, [s])
        assert e.value.status == -1, bad
    small = W.random_charges(n=10, box=(25.0, 30.0, 30.0), seed=1)
    small.box[0] = -1.0
    with pytest.raises(R.RbsogError) as e:
        R.rbsog_create(R.rbsog_default_params(10.0), [small])
    assert e.value.status == -3
