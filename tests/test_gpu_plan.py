"""The axis vote's work split (gpu: the plan reads the device's SM count; no kernel runs).

For every grid side and pair counts from one to 2^31 - 1, single and batched, the plan that
`sprot_vote_plan` reports must
- partition the rows [0, G) into bands of whole row pairs (the shared tiles hold two rows'
  16-bit counters per 32-bit word), at most SPROT_MAX_BANDS of them, the same for every n;
- give every band a shared tile that fits the vote kernel's shared memory: (2G + 8) bytes a
  row (G + 4 words a row pair, with the pad word that takes a run's end beyond the grid) next
  to the 24 warps' circle tables (9 x 32 words each) and 32 dummy words, in 227 KB less 64
  bytes of static use; a band of columns with the same edges needs (2G + 2) bytes a column;
- cut the pairs into slices of at most 65535 circles, so that no 16-bit counter of a slice's
  tile can wrap (Algorithm 1's accumulator is summed over the slices in 32 bits).
"""
import pytest

pytestmark = pytest.mark.gpu

TILE_BYTES = 227 * 1024 - 64 - (24 * 9 * 32 * 4 + 32 * 4)
SIDES = [16, 32, 64, 128, 256, 512, 1024, 2048]
COUNTS = [1, 2, 999, 65535, 65536, 300_001, 1_000_000, 5_000_000, 123_456_789, 2**31 - 1]


@pytest.mark.parametrize("G", SIDES)
def test_bands_partition_the_rows_and_fit_the_tile(lib, G):
    from paper_2502_06337_gb300 import binding as B

    first = None
    for batched in (False, True):
        for n in COUNTS:
            rows = B.vote_plan(n, G, batched=batched)["band_row0"]
            T = len(rows) - 1
            assert 1 <= T <= B.MAX_BANDS
            assert rows[0] == 0 and rows[-1] == G
            for b in range(T):
                r0, r1 = rows[b], rows[b + 1]
                assert r1 > r0 and r0 % 2 == 0 and r1 % 2 == 0, (G, b, r0, r1)
                assert (r1 - r0) * (2 * G + 8) <= TILE_BYTES, (G, b, r1 - r0)
                assert (r1 - r0) * (2 * G + 2) <= TILE_BYTES
            # the bands depend on G alone
            if first is None:
                first = rows
            assert rows == first, (G, n, batched)


@pytest.mark.parametrize("G", [64, 512, 2048])
@pytest.mark.parametrize("batched", [False, True])
def test_slices_hold_at_most_65535_circles(lib, G, batched):
    from paper_2502_06337_gb300 import binding as B

    for n in COUNTS:
        S = B.vote_plan(n, G, batched=batched)["slices"]
        assert 1 <= S <= n, (n, S)
        assert -(-n // S) <= 65535, (n, S)  # the largest slice: ceil(n / S) circles
        assert B.vote_plan(n, G, batched=batched)["slices"] == S  # deterministic


def test_plan_rejects_bad_arguments(lib):
    from paper_2502_06337_gb300 import binding as B

    for n, G in ((0, 512), (-5, 512), (2**31 + 1, 512), (1000, 8), (1000, 4096), (1000, 500)):
        with pytest.raises(B.SprotError):
            B.vote_plan(n, G)
