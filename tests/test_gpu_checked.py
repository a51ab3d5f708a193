"""The checked build (device bounds checks, LJMD_CHECKS) stands in for a race and
bounds checker on the GPU: it runs every hot kernel through the scenarios of
checked_scenarios.py without a failed check, and its results equal the product
build's bit for bit (the checks do not touch the arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(which: str, out: str) -> None:
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_scenarios.py"), which, out],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, f"{which} run failed:\n{r.stdout[-2000:]}\n{r.stderr[-4000:]}"


def test_checked_build_passes_and_matches_product(tmp_path):
    a, b = str(tmp_path / "product.npz"), str(tmp_path / "checked.npz")
    _run("product", a)
    _run("checked", b)
    pa, pb = np.load(a), np.load(b)
    assert sorted(pa.files) == sorted(pb.files)
    for k in pa.files:
        np.testing.assert_array_equal(pa[k], pb[k], err_msg=k)
