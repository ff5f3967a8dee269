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


def test_noalloc_energy_on_another_stream_follows_the_steps():
    """A caller stream other than the solver's is ordered after the work
    already enqueued on the solver's stream: called right after an
    asynchronous step(40), with no synchronisation, it returns the energy of
    the advanced fields."""
    import torch
    VX, EToV = W.kuhn_mesh(6, 1.0, 0.02, seed=32)
    g = dgh.Solver(VX, EToV, 4, 3)
    g.init_gaussian([0.2, 0.1, -0.1], 0.2)
    e0 = g.energy()
    other = torch.cuda.Stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.step(40)                                           # asynchronous on the solver's stream
    g.energy_noalloc(out.data_ptr(), other)
    other.synchronize()
    got = float(out[0].item())
    ref = g.energy()                                     # synchronises the solver's stream
    assert ref != e0
    assert abs(got - ref) <= TOL * ref, (got, ref, e0)
    g.close()


def test_noalloc_energy_rejects_a_mesh_above_its_scratch_limit():
    """The static scratch holds 65,536 partial sums of 64 cells: a mesh of
    89^3 x 6 = 4,229,814 cells (N = 1, no HABC) is above the 4,194,304-cell
    limit, and the call returns DGH_EINVAL without touching the output; the
    allocating energy still works."""
    import torch
    VX, EToV = W.kuhn_mesh(89, 1.0, 0.0, seed=33)
    assert EToV.shape[0] > 4194304
    g = dgh.Solver(VX, EToV, 1, 0)
    g.init_gaussian([0.0, 0.0, 0.0], 0.3)
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(dgh.DghError) as e:
        g.energy_noalloc(out.data_ptr())
    assert e.value.code == dgh.DGH_EINVAL
    torch.cuda.synchronize()
    assert float(out[0].item()) == -1.0
    assert g.energy() > 0.0
    g.close()
