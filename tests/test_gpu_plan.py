"""The axis vote's work split on the device (gpu: the plan reads the device's SM count; no
kernel runs). The split's invariants (bands of whole row pairs within the tile budget, slices of
at most 65535 circles) are checked without a GPU in tests/test_plan_host.py for devices of 1 to
4096 SMs; here the device's own plan must be the host plan for its SM count, for every grid
side and pair counts from one to 2^31 - 1, single and batched."""
import pytest

pytestmark = pytest.mark.gpu

SIDES = [16, 32, 64, 128, 256, 512, 1024, 2048]
COUNTS = [1, 2, 999, 65535, 65536, 300_001, 1_000_000, 5_000_000, 123_456_789, 2**31 - 1]


def test_device_plan_is_the_host_plan_for_its_sm_count(lib):
    import torch

    from paper_2502_06337_gb300 import binding as B

    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    for G in SIDES:
        for batched in (False, True):
            for n in COUNTS:
                dev = B.vote_plan(n, G, batched=batched)
                assert dev == B.vote_plan(n, G, batched=batched, n_sm=n_sm), (G, n, batched)
                S = dev["slices"]
                assert -(-n // S) <= 65535, (G, n, batched, S)


def test_plan_rejects_bad_arguments(lib):
    from paper_2502_06337_gb300 import binding as B

    for n, G in ((0, 512), (-5, 512), (2**31 + 1, 512), (1000, 8), (1000, 4096), (1000, 500)):
        with pytest.raises(B.SprotError):
            B.vote_plan(n, G)
