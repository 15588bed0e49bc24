"""The heavy numeric kernel built with its row membership check compiled in
(SPG_CHECK_MEMBERSHIP=1): every product's row must be present in the item's
symbolic bitmap; a missing one is accumulated into a separate slot and
reported as an internal error instead of landing on a neighbour's rank.  The
product build leaves the check out (both passes walk the same segments with
the same code).  This test builds the checked variant in-tree and runs heavy
products through it in a child process (the binding loads one library per
process), against the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import paper_2408_14558_gb300 as g, oracle, synth
from parity import assert_full_parity, run_gpu
g.load_library(LIB)
assert g.load_library() is g.load_library(LIB)
rng = np.random.default_rng(5)
for vals in ("f64", "i64big"):
    A = synth.random_sparse(5000, 600, 0.01, rng, values=vals)
    B = synth.random_sparse(600, 500, 0.05, rng, values=vals)
    assert_full_parity(run_gpu(A, B, 3, 64, light_max=32, slab_rows=1024), oracle.spgemm(A, B), "checked " + vals)
R = synth.rmat_symmetric(13, 16, seed=1)
assert_full_parity(run_gpu(R, R, 4, 256, light_max=64, slab_rows=2048), oracle.spgemm(R, R), "checked rmat13")
print("membership-checked build: parity ok")
'''


def test_membership_checked_build_matches_oracle():
    from paper_2408_14558_gb300 import build
    lib = build.build(extra=["-DSPG_CHECK_MEMBERSHIP=1"],
                      lib=os.path.join(ROOT, "paper_2408_14558_gb300", "libspgemm1d_check.so"),
                      build_dir=os.path.join(ROOT, "paper_2408_14558_gb300", "_build_check"))
    code = f"ROOT = {ROOT!r}\nLIB = {lib!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "parity ok" in r.stdout
