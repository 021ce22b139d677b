"""The product path has no CPU fallback: without the CUDA library the binding raises, and
device work on a machine without a GPU ends in an error status, never in a silent result."""
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_missing_library_raises():
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1909_13772_gb300 import lbm\n"
            "try:\n"
            "    lbm.lbm_create_blocks(lbm.make_params(), [((0, 0, 0), (4, 4, 4))])\n"
            "except ImportError as e:\n"
            "    print('raised', e)\n" % ROOT)
    env = dict(os.environ, LBM_LIBRARY=os.path.join(ROOT, "no-such-dir", "liblbm.so"))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.startswith("raised liblbm.so not found"), out.stdout + out.stderr


def test_device_work_without_a_gpu_is_an_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    sys.path.insert(0, ROOT)
    from paper_1909_13772_gb300 import inputs, lbm
    ctx = lbm.lbm_create_blocks(lbm.make_params(), [((0, 0, 0), (8, 8, 8))])  # host-only set-up works
    try:
        rho, u = inputs.rest((8, 8, 8))
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_init_macroscopic(ctx, 0, rho, u)
        assert e.value.status == 3  # LBM_ERR_CUDA
        with pytest.raises(lbm.LbmError):
            lbm.lbm_step(ctx, 1)
    finally:
        lbm.lbm_destroy(ctx)


def test_product_package_never_touches_the_oracle():
    """The oracle is test infrastructure: no module or source of the package imports, loads or
    names it (the tests, smoke() and the bench's CPU legs are the only users)."""
    import re
    pkg = os.path.join(ROOT, "paper_1909_13772_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for name in files:
            if name.endswith((".py", ".cu", ".cuh", ".cpp", ".hpp", ".h")):
                text = open(os.path.join(dirpath, name)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|lbm_oracle|liboracle", text, re.M), name
