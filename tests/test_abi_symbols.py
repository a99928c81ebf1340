"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function
declared in include/*.h; the Python binding wraps exactly those names; without a GPU its
constructors fail with RKL_ECUDA."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_](?:[\w ]*?[\s\*])(\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rkl_create", "rkl_destroy", "set_coeffs", "apply_F", "rkl2_superstep",
                     "be_pcg_solve", "rkl2_stage_count", "rkl_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1610_01265_gb300 import build as B
    from paper_1610_01265_gb300 import rklpcg, warmstart

    path = B.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(rklpcg.EXPORTED) | set(warmstart.EXPORTED) == declared_functions()


def test_host_only_calls_without_gpu():
    """Pure host entry points (no device work) answer without a GPU."""
    from paper_1610_01265_gb300 import rklpcg

    rklpcg.load()
    assert rklpcg.rkl2_stage_count(100.0) == 20
    assert rklpcg.rkl2_stage_count(10000.0, rklpcg.RKL_FORCE_ODD) == 201
    assert rklpcg.strerror(rklpcg.RKL_ENOTCONV).startswith("PCG")
    lib = rklpcg.load()
    assert lib.rkl2_stage_count(-1.0, 0) == rklpcg.RKL_EINVAL
    assert lib.rkl2_stage_count(float("nan"), 0) == rklpcg.RKL_EINVAL
    from paper_1610_01265_gb300 import warmstart

    assert warmstart.num_params() == sum(co * ci * 27 + co for ci, co in warmstart.LAYERS) == 60577


def test_no_gpu_fails_loudly():
    """Without a CUDA device the library reports RKL_ECUDA from its constructors: there is no
    CPU fallback behind the C ABI."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1610_01265_gb300 import rklpcg as R
    from paper_1610_01265_gb300 import synth
    from paper_1610_01265_gb300 import warmstart as W

    c = synth.conduction_case(8, 4, 8, 1)
    with pytest.raises(R.RklError) as e:
        R.Context(c["rf"], 4, 8)
    assert e.value.code == R.RKL_ECUDA
    with pytest.raises(R.RklError) as e:
        W.Net(1)
    assert e.value.code == R.RKL_ECUDA
