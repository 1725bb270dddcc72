"""Tensor-core products whose strided operand is read along a unit-stride
free index (the transposing pack, chosen for long-K products, with the
output then written through its offset tables in the reordered row order).

At the sizes the oracle handles no product is long enough to take this
path, so a child process forces it for every tensor-core product
(CDFNS_ROWS_MIN_K=1) and reruns residual and sigma parity cases against the
oracle there.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = """
import sys
sys.path.insert(0, {root!r})
sys.path.insert(0, {here!r})
import test_gpu_parity as t
for tier in ("fp16", "tf32x3", "fp16x3"):
    t.test_ccsd_residual_matches_oracle(tier, 7, 45, 66)
t.test_sigma_matches_oracle("fp16", "fp16x3")
t.test_sigma_matches_oracle("tf32x3", None)
print("row-order parity ok")
"""


def test_reordered_rows_match_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, CDFNS_ROWS_MIN_K="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, here=HERE)], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "row-order parity ok" in r.stdout, (
        r.stdout[-2000:] + r.stderr[-4000:])
