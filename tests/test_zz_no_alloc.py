"""dgh_get_energy_noalloc: the energy for callers that cannot allocate device
memory (code under a framework whose memory pool owns every byte of the
device, or a latency-critical loop that cannot afford cudaMalloc's implicit
synchronisation).  Its scratch is a fixed static array of the library, so it
must agree with the regular, allocating dgh_get_energy -- here on two calls
in a row, with the solution advanced in between.  Both reductions do the same
FP64 arithmetic and differ by summation order only, so the bound is 1e-12:
a wrong partial-sum index would show.  Collected last on purpose."""
import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from paper_1610_05023_b300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def test_noalloc_energy_matches_allocating_energy_twice():
    import torch
    VX, EToV = W.kuhn_mesh(3, 1.0, 0.02, seed=31)
    stream = torch.cuda.Stream()
    g = dgh.Solver(VX, EToV, 3, 2, stream=stream)
    g.init_gaussian([0.1, -0.1, 0.05], 0.3)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for i in range(2):
        g.step(7)
        ref = g.energy()                                 # allocating path (context scratch)
        g.energy_noalloc(out.data_ptr() + 8 * i, stream)  # static scratch, device output
        stream.synchronize()
        got = float(out[i].item())
        assert ref > 0.0
        assert abs(got - ref) <= TOL * ref, (i, got, ref)
    assert out[0].item() != out[1].item()                # the second call saw the advanced solution
    g.close()


def test_noalloc_energy_rejects_null_output():
    VX, EToV = W.kuhn_mesh(1, 1.0, 0.0, seed=1)
    g = dgh.Solver(VX, EToV, 2, 0)
    with pytest.raises(dgh.DghError):
        g.energy_noalloc(0)
    g.close()
