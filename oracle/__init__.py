"""FP64 CPU oracle of the stereographic-projection rotation vote (arXiv 2502.06337).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or run anything in this package. The CUDA library never calls
it and shares no code with it: a product path that reached this package would be a CPU
fallback, which the library does not have.

Everything here is a plain, slow restatement of the paper's definitions in float64 numpy:
    geometry.py  stereographic projection (Eqs. 11-12), the projected great circle (Eq. 13),
                 Rodrigues (Eq. 2) and the rotation error (Eq. 16);
    vote.py      the axis vote (Algorithm 1, Sec. IV-A), peak and top-k (Sec. IV-D), the
                 angle vote (Algorithm 1, Sec. IV-B), labels and least-squares refinement.

Parity pinning: every function is pinned by the not-gpu tests against closed forms,
invariants, brute force or library routines (see tests/test_oracle_*.py). No function is
"parity unpinned".
"""
from .geometry import (  # noqa: F401
    stereographic_projection,
    inverse_stereographic_projection,
    projected_circle,
    great_circle_curve,
    rodrigues,
    rotation_error,
)
from .vote import (  # noqa: F401
    BAND,
    grid_edges,
    cell_axis,
    subcell_offset,
    subcell_axis,
    circle_cell_extrema,
    axis_vote,
    cell_votes,
    row_votes,
    peak_cell,
    local_maxima,
    top_k_cells,
    window_gate,
    pair_angles,
    angle_vote,
    angle_peak,
    vote_set,
    kabsch,
    refine,
    assign_labels,
    sampled_circle_cells,
    solve,
)
