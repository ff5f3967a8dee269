"""The index-checked build (libdgh_checked.so, -DDGH_CHECKED) in place of a
memory checker: every index that a stage kernel gathers through or pushes to
is tested against its array.  A child process runs a spread of configurations
under the checked library (single problems, a batch of uneven problems, a
recording shadow chain); dgh_sync must report no violation (DGH_EBOUNDS),
and every level must be bit-identical to the normal build.  No index is
corrupted on purpose: the checks guard the set-up code, not a planted fault."""
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from paper_1610_05023_b300 import build, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (hexes per axis, N, P, boundary codes, precision)
CASES = [
    (2, 1, 1, (0,) * 6, 0),
    (2, 2, 3, (0, 0, 0, 0, 0, 1), 0),
    (3, 3, 2, (0,) * 6, 0),
    (2, 4, 6, (0,) * 6, 0),
    (2, 5, 2, (1, 0, 0, 1, 0, 1), 0),
    (2, 6, 4, (0,) * 6, 0),
    (2, 3, 12, (0,) * 6, 0),
    (2, 4, 2, (0,) * 6, dgh.PREC_SPLIT_BF16),
    (2, 3, 2, (1, 0, 0, 1, 0, 1), dgh.PREC_SPLIT_TF32),
    (3, 4, 6, (0,) * 6, dgh.PREC_SPLIT_TF32),
    (2, 1, 1, (0,) * 6, dgh.PREC_SPLIT_TF32),
    (2, 2, 3, (0, 0, 0, 0, 0, 1), dgh.PREC_SPLIT_TF32),
]


def run_cases(steps=12):
    out = {}
    for i, (n, N, P, bc, prec) in enumerate(CASES):
        VX, EToV = W.kuhn_mesh(n, 1.0, 0.03, seed=70 + i)
        g = dgh.Solver(VX, EToV, N, P, bc=bc, precision=prec)
        g.init_gaussian([0.2, -0.1, 0.15], 0.3)
        g.step(steps)
        g.sync()                      # DghError(EBOUNDS) on a violation
        for lv in (3, 2, 1):
            out["c%d_l%d" % (i, lv)] = g.get_state(lv)
        g.close()
    # a batch of uneven problems (one union context per (N, P) group)
    probs = []
    for j, (n, N, P) in enumerate([(2, 3, 2), (3, 4, 2), (2, 3, 2)]):
        VX, EToV = W.kuhn_mesh(n, 1.0, 0.03, seed=80 + j)
        g = dgh.Solver(VX, EToV, N, P)
        g.add_point_source([0.1 * j, 0.0, 0.1], 3.0, 0.3)
        g.init_gaussian([0.0, 0.1, 0.0], 0.3, 0.0)
        probs.append(g)
    b = dgh.Batch(probs)
    b.step(steps)
    b.sync()
    for j in range(len(probs)):
        for lv in (3, 2, 1):
            out["b%d_l%d" % (j, lv)] = b.get_state(j, lv)
    b.close()
    # the closure's recording shadow chain (its own 2D, 1D and 0D launches)
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.03, seed=90)
    g = dgh.Solver(VX, EToV, 3, 4)
    g.closure_record(shadow_order=2, every=3, fraction=1.0, max_samples=1 << 18, seed=9)
    g.init_gaussian([0.2, -0.1, 0.15], 0.3)
    g.step(steps)
    g.sync()
    S = g.closure_samples()
    out["shadow_rows"] = S[np.lexsort(S.T[::-1])]
    g.close()
    return out


CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np
import paper_1610_05023_b300 as dgh
dgh.load_library(dgh.CHECKED_LIB_PATH)
assert dgh._lib.dgh_is_checked_build() == 1
sys.path.insert(0, {tests!r})
import test_checked_build_gpu as T
np.savez({path!r}, **T.run_cases())
print("checked ok")
"""


@pytest.mark.gpu
def test_checked_build_finds_no_violation_and_changes_no_result():
    build.build(checked=True)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "checked.npz")
        code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), path=path)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
        checked = dict(np.load(path))
    normal = run_cases()
    assert dgh._lib.dgh_is_checked_build() == 0
    assert set(checked) == set(normal)
    for k in normal:
        assert np.array_equal(checked[k], normal[k]), k
