"""The allocation-free axis vote, sprot_axis_vote_noalloc (gpu).

Callers that cannot allocate device memory -- code under a host framework that owns the
device heap, a plug-in whose memory its host process budgets, a latency-critical path where an
allocation may block -- get the accumulator from this entry point, which takes its scratch
from a fixed device array instead of allocating. These tests call it through the C ABI and
check its grid against sprot_axis_vote's on several calls in a row (the array keeps the last
call's contents, so each call must clear what it needs), and that a problem too large for the
array is rejected before anything runs. The file is collected last so that a failure here
stops a run only after every other test has run."""
import ctypes as C

import numpy as np
import pytest

from paper_2502_06337_gb300 import synth

pytestmark = pytest.mark.gpu


def _grids(lib, prob, G):
    import torch

    from paper_2502_06337_gb300 import binding as B

    P = torch.from_numpy(prob.P).cuda()
    Q = torch.from_numpy(prob.Q).cuda()
    want = torch.zeros(G * G, dtype=torch.int32, device="cuda")
    B.axis_vote(P, Q, G, want)
    got = torch.full((G * G,), -1, dtype=torch.int32, device="cuda")
    st = lib.sprot_axis_vote_noalloc(P.data_ptr(), Q.data_ptr(), prob.n, G, got.data_ptr(), None)
    assert st == B.OK, B.status_text(st)
    torch.cuda.synchronize()
    return got.cpu().numpy(), want.cpu().numpy()


def test_noalloc_axis_vote_equals_the_allocating_one_on_consecutive_calls(lib):
    cases = [(synth.make_problem(200_000, (0.1,), 0.01, seed=41), 512),
             (synth.make_problem(30_000, (0.3, 0.2), 0.01, seed=42), 256),
             (synth.make_problem(1000, (0.5,), 0.01, seed=43), 64),
             (synth.make_problem(200_000, (0.1,), 0.01, seed=41), 512)]
    for prob, G in cases:
        got, want = _grids(lib, prob, G)
        assert np.array_equal(got, want)
        assert int(got.view(np.uint32).max()) > 0


def test_noalloc_rejects_a_plan_beyond_its_scratch(lib):
    from paper_2502_06337_gb300 import binding as B

    import torch

    # real buffers of the stated sizes, so that nothing could be read out of bounds even if the
    # size check were missing
    P = torch.zeros((1_000_000, 3), dtype=torch.float32, device="cuda")
    grid = torch.zeros(2048 * 2048, dtype=torch.int32, device="cuda")
    # 2048^2 grid, 10^6 pairs: 16 slices of 8 MB of partial counters, more than the 40 MB array
    assert lib.sprot_axis_vote_noalloc(P.data_ptr(), P.data_ptr(), 1_000_000, 2048, grid.data_ptr(),
                                       None) == B.E_INVAL
    assert lib.sprot_axis_vote_noalloc(None, None, 4, 16, None, None) == B.E_INVAL
    assert lib.sprot_axis_vote_noalloc(P.data_ptr(), P.data_ptr(), 4, 48, grid.data_ptr(), None) == B.E_INVAL
    assert int(grid.abs().sum()) == 0  # nothing ran
