"""The axis vote's work split as host code, without a GPU (`sprot_vote_plan_sm` takes the SM
count instead of reading it from a device). For every grid side, pair counts from one to
2^31 - 1, single and batched, and devices of 1 to 4096 SMs, the plan must
- partition the rows [0, G) into bands of whole row pairs (the shared tiles hold two rows'
  16-bit counters per 32-bit word), at most SPROT_MAX_BANDS of them, set by G alone;
- give every band a tile that fits the vote kernel's shared memory: (2G + 8) bytes a row
  (G + 4 words a row pair, with the pad word that takes a run's end beyond the grid) beside
  the 24 warps' circle tables (9 x 32 words each) and 32 dummy words, in 227 KB less 64 bytes
  of static use; a band of columns with the same edges needs (2G + 2) bytes a column;
- cut the pairs into at most n slices of at most 65535 circles each, so that no 16-bit
  counter of a slice's tile can wrap (Algorithm 1's accumulator is summed over the slices in
  32 bits)."""
import pytest

from paper_2502_06337_gb300 import binding as B, build

TILE_BYTES = 227 * 1024 - 64 - (24 * 9 * 32 * 4 + 32 * 4)
SIDES = [16, 32, 64, 128, 256, 512, 1024, 2048]
COUNTS = [1, 2, 999, 65535, 65536, 300_001, 1_000_000, 5_000_000, 123_456_789, 2**31 - 1]
SMS = [1, 8, 76, 148, 152, 160, 4096]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.load(build.build())


@pytest.mark.parametrize("G", SIDES)
def test_bands_partition_the_rows_and_fit_the_tile(G):
    first = None
    for n_sm in SMS:
        for batched in (False, True):
            for n in COUNTS:
                rows = B.vote_plan(n, G, batched=batched, n_sm=n_sm)["band_row0"]
                T = len(rows) - 1
                assert 1 <= T <= B.MAX_BANDS
                assert rows[0] == 0 and rows[-1] == G
                for b in range(T):
                    r0, r1 = rows[b], rows[b + 1]
                    assert r1 > r0 and r0 % 2 == 0 and r1 % 2 == 0, (G, b, r0, r1)
                    assert (r1 - r0) * (2 * G + 8) <= TILE_BYTES, (G, b, r1 - r0)
                    assert (r1 - r0) * (2 * G + 2) <= TILE_BYTES
                if first is None:
                    first = rows
                assert rows == first, (G, n, batched, n_sm)


@pytest.mark.parametrize("G", [16, 512, 2048])
@pytest.mark.parametrize("batched", [False, True])
def test_slices_hold_at_most_65535_circles(G, batched):
    for n_sm in SMS:
        for n in COUNTS:
            S = B.vote_plan(n, G, batched=batched, n_sm=n_sm)["slices"]
            assert 1 <= S <= n, (n, n_sm, S)
            assert -(-n // S) <= 65535, (n, n_sm, S)  # the largest slice: ceil(n / S) circles


def test_single_plan_fills_whole_rounds_of_sms():
    """A single solve takes k rounds of the SMs, the fewest whose 2 T items per slice reach the
    slice count the 16-bit counters force (s_min = ceil(n / 65535)), and the most slices whose
    items fit those rounds: k n_sm - 2T < 2T S <= k n_sm (when n / 512 does not cap S)."""
    for n in (300_001, 1_000_000, 5_000_000, 123_456_789):
        for n_sm in (8, 76, 148, 152, 160):
            p = B.vote_plan(n, 512, n_sm=n_sm)
            per_slice = 2 * (len(p["band_row0"]) - 1)
            s_min = -(-n // 65535)
            k = max(1, -(-(s_min * per_slice) // n_sm))
            items = per_slice * p["slices"]
            assert k * n_sm - per_slice < items <= k * n_sm, (n, n_sm, items, k)
            assert p["slices"] >= s_min


def test_batched_plan_ignores_the_sm_count():
    for n in COUNTS:
        plans = {tuple(B.vote_plan(n, 512, batched=True, n_sm=s)["band_row0"]) +
                 (B.vote_plan(n, 512, batched=True, n_sm=s)["slices"],) for s in SMS}
        assert len(plans) == 1, n


@pytest.mark.parametrize("n,G,n_sm", [(0, 512, 152), (-5, 512, 152), (2**31 + 1, 512, 152), (1000, 8, 152),
                                      (1000, 4096, 152), (1000, 500, 152), (1000, 512, 0), (1000, 512, 4097)])
def test_plan_rejects_bad_arguments(n, G, n_sm):
    with pytest.raises(B.SprotError):
        B.vote_plan(n, G, n_sm=n_sm)
