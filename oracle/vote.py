"""Axis vote, peaks, angle vote and refinement in float64 (test infrastructure; see the
package header).

The steps follow Algorithm 1 (AORESP) and Sec. IV of the paper, in the paper's order:
circle of each correspondence -> 2-D accumulator -> peak cell(s) -> per-pair angle ->
angle histogram -> rotation. Where the paper is silent or ambiguous, the reading taken is
stated at the function that implements it.

Boundary flags. Several steps turn a floating-point test into an integer (a cell counted or
not, a histogram bin, an inlier label). The oracle decides each test in float64 and, beside
the decision, flags the cases whose test lies within ``BAND`` = 1e-6 of its boundary in
normalised units; a float32 implementation may decide those either way. Integer outputs are
therefore returned as the float64 result plus lower/upper bounds that a correct float32
result must lie between.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import inverse_stereographic_projection, rodrigues

#: width of the boundary band (normalised units) inside which a test may go either way
BAND = 1e-6
#: a pair is skipped by the angle vote when p or q lies within this sine of the axis
AXIS_SINE_MIN = 1e-3


# ---------------------------------------------------------------------------------------
# The accumulator grid (Algorithm 1 "two-dimensional accumulator"; Sec. IV-A)
# ---------------------------------------------------------------------------------------

def grid_edges(G: int) -> np.ndarray:
    """Cell edges of the G x G accumulator over the square [-1, 1]^2 of the projection
    plane: e_k = -1 + 2k/G, k = 0..G (exact in binary for power-of-two G).

    Reading (the paper gives no extent for the accumulator): the square covers the whole
    unit disk, i.e. every axis of the southern hemisphere; since r and -r are the same axis
    line, that already holds every rotation axis. The corners outside the disk are kept so
    that the grid is a plain square."""
    return -1.0 + 2.0 * np.arange(G + 1, dtype=np.float64) / G


def cell_axis(G: int, row: int, col: int) -> np.ndarray:
    """The axis of a cell: its centre back-projected by Eq. 12 (Algorithm 1, "the center of
    the block ... is back-projected onto the sphere"). Rows index v, columns index u.
    Canonicalised to the southern hemisphere (r_z <= 0) since r and -r are one axis."""
    u = -1.0 + (2.0 * col + 1.0) / G
    v = -1.0 + (2.0 * row + 1.0) / G
    r = inverse_stereographic_projection(u, v)
    if r[2] > 0:
        r = -r
    return r


def _quadratic_range(c2, c1, lo, hi):
    """min and max of f(x) = c2 x^2 + c1 x over the closed interval [lo, hi].

    A quadratic attains its extremes on an interval at the end points or at its vertex
    -c1/(2 c2) when that lies inside. Broadcasts over all arguments."""
    c2, c1, lo, hi = np.broadcast_arrays(*(np.asarray(x, dtype=np.float64) for x in (c2, c1, lo, hi)))
    f_lo = c2 * lo * lo + c1 * lo
    f_hi = c2 * hi * hi + c1 * hi
    fmin = np.minimum(f_lo, f_hi)
    fmax = np.maximum(f_lo, f_hi)
    with np.errstate(divide="ignore", invalid="ignore"):
        xv = -c1 / (2.0 * c2)
        inside = (c2 != 0) & (xv >= lo) & (xv <= hi)
        fv = np.where(inside, c2 * xv * xv + c1 * xv, 0.0)
    fmin = np.where(inside, np.minimum(fmin, fv), fmin)
    fmax = np.where(inside, np.maximum(fmax, fv), fmax)
    return fmin, fmax


def circle_cell_extrema(d, G: int):
    """min and max of the curve function F of ``d`` over every closed cell.

    F(u, v) = 2 d1 u + 2 d2 v + d3 (u^2 + v^2 - 1) (Eq. 13 with D = 0; see
    ``great_circle_curve``) splits as g(u) + h(v) - d3 with g(u) = d3 u^2 + 2 d1 u and
    h(v) = d3 v^2 + 2 d2 v, so its extremes over a box are sums of 1-D extremes.
    Returns (Fmin, Fmax), each G x G indexed [row (v), col (u)]."""
    d = np.asarray(d, dtype=np.float64)
    e = grid_edges(G)
    gmin, gmax = _quadratic_range(d[2], 2.0 * d[0], e[:-1], e[1:])
    hmin, hmax = _quadratic_range(d[2], 2.0 * d[1], e[:-1], e[1:])
    Fmin = hmin[:, None] + gmin[None, :] - d[2]
    Fmax = hmax[:, None] + gmax[None, :] - d[2]
    return Fmin, Fmax


def _differences(P, Q):
    """d_i = p_i - q_i in float64 (exact for float32 inputs). Algorithm 1 writes y - x and
    Sec. IV writes x - y; the sign does not change the circle. A pair with d_i = 0 exactly
    fixes no circle: it is 'degenerate' and takes no part in any vote."""
    D = np.asarray(P, dtype=np.float64) - np.asarray(Q, dtype=np.float64)
    deg = ~np.any(D != 0.0, axis=1)
    return D, deg


def axis_vote(P, Q, G: int):
    """The 2-D axis accumulator (Algorithm 1; Sec. IV-A; Fig. 3c: "the number in each cell
    represents the number of circles that pass through the cell").

    Reading: circle i passes through cell c iff the curve F_i = 0 meets the CLOSED cell,
    i.e. min_c F_i <= 0 <= max_c F_i (F is continuous and the cell connected). A curve on a
    shared edge therefore counts in both cells. The paper's epsilon-band (Eq. 9) is not
    used: the vote is at cell resolution.

    The decision for (i, c) is flagged when |min_c F_i| or |max_c F_i| is within BAND of 0
    after normalising d_i to unit length.

    Returns dict(grid, lo, hi, n_degenerate): ``grid`` the float64 counts (int64, G x G,
    [row, col]); a float32 implementation is correct iff lo <= its grid <= hi, and must
    equal ``grid`` wherever lo == hi.
    """
    D, deg = _differences(P, Q)
    grid = np.zeros((G, G), dtype=np.int64)
    lo = np.zeros((G, G), dtype=np.int64)
    hi = np.zeros((G, G), dtype=np.int64)
    for i in np.flatnonzero(~deg):
        d = D[i]
        Fmin, Fmax = circle_cell_extrema(d, G)
        voted = (Fmin <= 0.0) & (Fmax >= 0.0)
        tol = BAND * float(np.sqrt(d @ d))
        flag = (np.abs(Fmin) <= tol) | (np.abs(Fmax) <= tol)
        grid += voted
        lo += voted & ~flag
        hi += voted | flag
    return dict(grid=grid, lo=lo, hi=hi, n_degenerate=int(deg.sum()))


def cell_votes(P, Q, G: int, rows, cols):
    """Votes of selected cells over all circles (the same test as ``axis_vote``, evaluated
    cell by cell so that it scales to 10^6 circles). Returns (count, lo, hi) arrays."""
    D, deg = _differences(P, Q)
    e = grid_edges(G)
    nrm = np.sqrt(np.einsum("ij,ij->i", D, D))
    out = np.zeros((3, len(rows)), dtype=np.int64)
    for k, (r, c) in enumerate(zip(rows, cols)):
        gmin, gmax = _quadratic_range(D[:, 2], 2.0 * D[:, 0], e[c], e[c + 1])
        hmin, hmax = _quadratic_range(D[:, 2], 2.0 * D[:, 1], e[r], e[r + 1])
        Fmin = gmin + hmin - D[:, 2]
        Fmax = gmax + hmax - D[:, 2]
        voted = (Fmin <= 0.0) & (Fmax >= 0.0) & ~deg
        flag = ((np.abs(Fmin) <= BAND * nrm) | (np.abs(Fmax) <= BAND * nrm)) & ~deg
        out[0, k] = voted.sum()
        out[1, k] = (voted & ~flag).sum()
        out[2, k] = (voted | flag).sum()
    return out[0], out[1], out[2]


def row_votes(P, Q, G: int, row: int, chunk: int = 8192):
    """Votes of every cell of one row over all circles (the same closed-cell test as
    ``axis_vote``, evaluated for one row at a time, in chunks of circles, so that whole rows
    of a 10^6-circle accumulator can be checked). Returns (count, lo, hi), each of length G."""
    D, deg = _differences(P, Q)
    e = grid_edges(G)
    out = np.zeros((3, G), dtype=np.int64)
    for a in range(0, len(D), chunk):
        d = D[a:a + chunk][~deg[a:a + chunk]]
        nrm = np.sqrt(np.einsum("ij,ij->i", d, d))[:, None]
        hmin, hmax = _quadratic_range(d[:, 2], 2.0 * d[:, 1], e[row], e[row + 1])
        gmin, gmax = _quadratic_range(d[:, 2][:, None], 2.0 * d[:, 0][:, None], e[None, :-1], e[None, 1:])
        Fmin = gmin + (hmin - d[:, 2])[:, None]
        Fmax = gmax + (hmax - d[:, 2])[:, None]
        voted = (Fmin <= 0.0) & (Fmax >= 0.0)
        flag = (np.abs(Fmin) <= BAND * nrm) | (np.abs(Fmax) <= BAND * nrm)
        out[0] += voted.sum(axis=0)
        out[1] += (voted & ~flag).sum(axis=0)
        out[2] += (voted | flag).sum(axis=0)
    return out[0], out[1], out[2]


# ---------------------------------------------------------------------------------------
# Peaks (Algorithm 1; Sec. IV-A; multi-rotation Sec. IV-D)
# ---------------------------------------------------------------------------------------

def peak_cell(grid):
    """The cell with the most votes. Reading: ties go to the smallest row-major index
    (row = v first, then column = u). Returns (row, col, count)."""
    grid = np.asarray(grid)
    G = grid.shape[1]
    flat = int(np.argmax(grid.ravel()))  # first maximum in row-major order
    return flat // G, flat % G, int(grid.ravel()[flat])


def axis_angle_deg(r1, r2) -> float:
    """Angle between two axis LINES, in degrees: min of the angles to r2 and -r2."""
    c = abs(float(np.dot(r1, r2))) / (np.linalg.norm(r1) * np.linalg.norm(r2))
    return math.degrees(math.acos(min(1.0, c)))


def local_maxima(grid):
    """Cells that are peaks of the accumulator: strict local maxima of the key
    (count, -row-major index) over their 8 neighbours (clipped to the grid).

    Reading (Sec. IV-D and Fig. 3d-f detect the rotation axes as the peaks of the 2-D
    histogram but give no definition): a cell is a peak when no neighbour has more votes,
    and among equal counts the smallest index wins, so a plateau resolves to a definite cell
    and a cell on the flank of a larger peak (a shoulder) is never a peak. Returns a
    boolean G x G mask."""
    grid = np.asarray(grid)
    G0, G1 = grid.shape
    idx = np.arange(G0 * G1).reshape(G0, G1)
    peak = np.ones((G0, G1), dtype=bool)
    for dr in (-1, 0, 1):
        for dc in (-1, 0, 1):
            if dr == 0 and dc == 0:
                continue
            # the cell (r, c) against its neighbour (r + dr, c + dc), where it exists
            r0, r1 = max(0, -dr), G0 - max(0, dr)
            c0, c1 = max(0, -dc), G1 - max(0, dc)
            here = grid[r0:r1, c0:c1]
            there = grid[r0 + dr:r1 + dr, c0 + dc:c1 + dc]
            here_i = idx[r0:r1, c0:c1]
            there_i = idx[r0 + dr:r1 + dr, c0 + dc:c1 + dc]
            beaten = (there > here) | ((there == here) & (there_i < here_i))
            peak[r0:r1, c0:c1] &= ~beaten
    return peak


def top_k_cells(grid, k: int, nms_deg: float):
    """Several rotation axes from one accumulator (Sec. IV-D; Fig. 3d-f).

    Reading: the candidates are the accumulator's peaks (``local_maxima``); the paper
    states no rule for separating them, so a greedy non-maximum suppression is applied.
    Peaks are visited by (count descending, row-major index ascending); a peak is taken if
    its count is positive and its axis is more than ``nms_deg`` degrees from every axis
    taken so far. Stops after k peaks. The global maximum is always a peak, so with k = 1
    this is ``peak_cell``. Returns a list of (row, col, count)."""
    grid = np.asarray(grid)
    G = grid.shape[1]
    flat = grid.ravel()
    is_peak = local_maxima(grid).ravel()
    order = np.lexsort((np.arange(flat.size), -flat))
    peaks, axes = [], []
    for idx in order:
        cnt = int(flat[idx])
        if cnt <= 0 or len(peaks) >= k:
            break
        if not is_peak[idx]:
            continue
        row, col = divmod(int(idx), G)
        r = cell_axis(G, row, col)
        if any(axis_angle_deg(r, a) <= nms_deg for a in axes):
            continue
        peaks.append((row, col, cnt))
        axes.append(r)
    return peaks


def subcell_offset(grid, row: int, col: int):
    """Sub-cell position of a peak, in cells, along u (columns) and v (rows).

    Algorithm 1 back-projects the centre of the peak cell (Eq. 12), so the axis carries up
    to half a cell of quantisation. Reading (the paper gives no interpolation): along each
    grid axis a parabola is fitted through the counts of the peak cell and its two edge
    neighbours, c(-1), c(0), c(1), and the peak is placed at its vertex,
        delta = (c(-1) - c(1)) / (2 (c(-1) - 2 c(0) + c(1))),
    clamped to [-1/2, 1/2] (the cell itself). The offset along an axis is 0 when the
    parabola does not open downwards (c(-1) - 2 c(0) + c(1) >= 0) or when the peak lies on
    the grid border along that axis (a neighbour is missing). Returns (du, dv)."""
    grid = np.asarray(grid)
    G = grid.shape[1]
    c0 = float(grid[row, col])

    def vertex(cm, cp):
        den = float(cm) - 2.0 * c0 + float(cp)
        if den >= 0.0:
            return 0.0
        return min(0.5, max(-0.5, 0.5 * (float(cm) - float(cp)) / den))

    du = vertex(grid[row, col - 1], grid[row, col + 1]) if 0 < col < G - 1 else 0.0
    dv = vertex(grid[row - 1, col], grid[row + 1, col]) if 0 < row < G - 1 else 0.0
    return du, dv


def subcell_axis(G: int, row: int, col: int, du: float, dv: float) -> np.ndarray:
    """The axis at the sub-cell point (centre of cell (row, col) moved by du, dv cells),
    back-projected by Eq. 12 and canonicalised to r_z <= 0 like ``cell_axis``."""
    u = -1.0 + (2.0 * col + 1.0 + 2.0 * du) / G
    v = -1.0 + (2.0 * row + 1.0 + 2.0 * dv) / G
    r = inverse_stereographic_projection(u, v)
    if r[2] > 0:
        r = -r
    return r


# ---------------------------------------------------------------------------------------
# Angle vote (Algorithm 1 second loop; Sec. IV-B, Eq. 15)
# ---------------------------------------------------------------------------------------

def window_gate(P, Q, G: int, row: int, col: int, w: int):
    """Which correspondences take part in the angle vote about the axis of cell (row, col).

    Reading: Algorithm 1 lets every pair vote; a pair whose circle misses the found axis
    cannot be an inlier of that axis, so with w >= 0 a pair votes only if its circle meets
    the (2w+1) x (2w+1) window of cells centred on the peak (clipped to the grid), tested
    like a cell of the axis vote on the window's closed box. w < 0 keeps Algorithm 1's
    every-pair vote. Degenerate pairs never vote.
    Returns (gate, flag) boolean arrays."""
    D, deg = _differences(P, Q)
    if w < 0:
        return ~deg, np.zeros_like(deg)
    e = grid_edges(G)
    r0, r1 = max(0, row - w), min(G - 1, row + w)
    c0, c1 = max(0, col - w), min(G - 1, col + w)
    gmin, gmax = _quadratic_range(D[:, 2], 2.0 * D[:, 0], e[c0], e[c1 + 1])
    hmin, hmax = _quadratic_range(D[:, 2], 2.0 * D[:, 1], e[r0], e[r1 + 1])
    Fmin = gmin + hmin - D[:, 2]
    Fmax = gmax + hmax - D[:, 2]
    nrm = np.sqrt(np.einsum("ij,ij->i", D, D))
    gate = (Fmin <= 0.0) & (Fmax >= 0.0) & ~deg
    flag = ((np.abs(Fmin) <= BAND * nrm) | (np.abs(Fmax) <= BAND * nrm)) & ~deg
    return gate, flag


def pair_angles(r, P, Q):
    """Per-pair rotation angle about axis r (Algorithm 1: beta = r x x, gamma = r x y, and
    the angle between them; Eq. 15 solved for theta).

    Reading: Algorithm 1 takes arccos of the normalised beta . gamma, which is unsigned,
    while its angle bins cover [-pi, pi]. The signed angle
        theta = atan2(r . (beta x gamma), beta . gamma)  in (-pi, pi]
    is used; it is the angle of Eq. 2 about +r that carries beta onto gamma.
    Returns (theta, |beta|, |gamma|)."""
    r = np.asarray(r, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    beta = np.cross(r, P)
    gamma = np.cross(r, Q)
    s = np.cross(beta, gamma) @ r
    c = np.einsum("ij,ij->i", beta, gamma)
    return np.arctan2(s, c), np.linalg.norm(beta, axis=1), np.linalg.norm(gamma, axis=1)


def angle_vote(P, Q, r, gate, gate_flag, J: int):
    """The 1-D angle histogram about axis r (Algorithm 1: theta discretised uniformly over
    [-pi, pi] into J bins; "histogram voting", Sec. IV-B).

    Bin b covers [-pi + 2 pi b / J, -pi + 2 pi (b+1) / J); theta = pi falls in bin 0 (the
    same angle as -pi). A pair votes if its gate is set and neither p nor q lies within a
    sine of AXIS_SINE_MIN of the axis (there the angle is undefined or ill-conditioned).

    Flags: a pair's bin is flagged when theta lies within
        eta = BAND (1 + |p|/|beta|) (1 + |q|/|gamma|)
    of a bin edge -- the angle moved by a relative perturbation BAND of the axis, p or q --
    and its validity is flagged when |beta|/|p| is within BAND of AXIS_SINE_MIN (same for q).

    Returns dict(hist, lo, hi, bin, member, member_lo, member_hi, theta) where
    ``member`` is the float64 vote set, ``member_lo`` the certain and ``member_hi`` the
    possible voters, and ``bin`` the bin of every pair (-1 where undefined)."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    theta, nb, ng = pair_angles(r, P, Q)
    npn = np.linalg.norm(P, axis=1)
    nqn = np.linalg.norm(Q, axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        sp = np.where(npn > 0, nb / npn, 0.0)
        sq = np.where(nqn > 0, ng / nqn, 0.0)
        valid = (sp > AXIS_SINE_MIN) & (sq > AXIS_SINE_MIN)
        vflag = ((npn > 0) & (np.abs(sp - AXIS_SINE_MIN) <= BAND)) | (
            (nqn > 0) & (np.abs(sq - AXIS_SINE_MIN) <= BAND))
        x = (theta + math.pi) * J / (2.0 * math.pi)
        b = np.floor(x).astype(np.int64) % J
        frac = x - np.floor(x)
        dist = np.minimum(frac, 1.0 - frac) * (2.0 * math.pi / J)
        eta = BAND * (1.0 + npn / nb) * (1.0 + nqn / ng)
        bflag = dist <= eta
    alt = np.where(frac < 0.5, b - 1, b + 1) % J
    member = gate & valid
    member_lo = gate & ~gate_flag & valid & ~vflag
    member_hi = (gate | gate_flag) & (valid | vflag)
    hist = np.bincount(b[member], minlength=J)
    lo = np.bincount(b[member_lo & ~bflag], minlength=J)
    hi = np.bincount(b[member_hi], minlength=J) + np.bincount(alt[member_hi & bflag], minlength=J)
    binv = np.where(member_hi, b, -1)
    return dict(hist=hist, lo=lo, hi=hi, bin=binv, member=member, member_lo=member_lo,
                member_hi=member_hi, bin_flag=bflag, theta=theta)


def angle_peak(hist):
    """The bin with most votes (ties to the lowest index) and its centre angle."""
    hist = np.asarray(hist)
    J = hist.size
    b = int(np.argmax(hist))
    return b, -math.pi + (b + 0.5) * 2.0 * math.pi / J


def vote_set(av: dict, b: int, J: int, window: int):
    """The pairs that agree with the voted rotation: voters whose bin is within ``window``
    bins of the peak bin b (circularly). Returns (V, V_lo, V_hi) like ``angle_vote``."""
    binv = av["bin"]
    dist = np.minimum((binv - b) % J, (b - binv) % J)
    near = (binv >= 0) & (dist <= window)
    # a bin-flagged pair may sit one bin further out or in
    near_out = (binv >= 0) & (dist <= window + 1)
    near_in = (binv >= 0) & (dist <= max(window - 1, -1))
    V = av["member"] & near
    V_lo = av["member_lo"] & (near_in | (near & ~av["bin_flag"]))
    V_hi = av["member_hi"] & (near | (near_out & av["bin_flag"]))
    return V, V_lo, V_hi


# ---------------------------------------------------------------------------------------
# Recovery and refinement (Sec. IV-C; least squares on the inliers)
# ---------------------------------------------------------------------------------------

def kabsch(P, Q):
    """The rotation minimising sum ||q_i - R p_i||^2 (no translation: Eq. 1 has none).
    M = sum q_i p_i^T = U S V^T, R = U diag(1, 1, det(U V^T)) V^T (numpy SVD)."""
    M = np.asarray(Q, dtype=np.float64).T @ np.asarray(P, dtype=np.float64)
    U, _, Vt = np.linalg.svd(M)
    s = np.sign(np.linalg.det(U @ Vt))
    if s == 0:
        s = 1.0
    return U @ np.diag([1.0, 1.0, s]) @ Vt


def refine(P, Q, V, R_fallback, tau: float):
    """Least-squares refinement (not in the paper, which stops at Rodrigues; Sec. II-A
    names local refinement as the usual last step). R1 = Kabsch over the vote set V (or
    R_fallback if V is empty); inliers C = {i : ||q_i - R1 p_i|| <= tau}, tau being the
    "noise level" input of Algorithm 1; R = Kabsch over C (or R1 if C is empty).

    Label flags: |residual - tau| <= BAND (1 + |p| + |q|).
    Returns dict(R1, R, inlier, inlier_flag, residual)."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    R1 = kabsch(P[V], Q[V]) if V.any() else np.asarray(R_fallback, dtype=np.float64)
    res = np.linalg.norm(Q - P @ R1.T, axis=1)
    inl = res <= tau
    flag = np.abs(res - tau) <= BAND * (1.0 + np.linalg.norm(P, axis=1) + np.linalg.norm(Q, axis=1))
    R = kabsch(P[inl], Q[inl]) if inl.any() else R1
    return dict(R1=R1, R=R, inlier=inl, inlier_flag=flag, residual=res)


def assign_labels(P, Q, R1s, tau: float):
    """Labels for several rotations: pair i goes to the rotation a with the smallest
    residual ||q_i - R1_a p_i|| among those <= tau (ties to the smaller a), else -1.
    Returns (labels, flag). A pair is flagged where any residual is within the band of tau,
    or where two residuals <= tau are within the band of each other (the choice between the
    two rotations is then a float decision at its threshold, as when two found rotations
    approximate the same true one)."""
    P = np.asarray(P, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    scale = BAND * (1.0 + np.linalg.norm(P, axis=1) + np.linalg.norm(Q, axis=1))
    best = np.full(P.shape[0], np.inf)
    labels = np.full(P.shape[0], -1, dtype=np.int32)
    flag = np.zeros(P.shape[0], dtype=bool)
    within = []
    for a, R1 in enumerate(R1s):
        res = np.linalg.norm(Q - P @ np.asarray(R1).T, axis=1)
        flag |= np.abs(res - tau) <= scale
        within.append(np.where(res <= tau + scale, res, np.inf))
        take = (res <= tau) & (res < best)
        labels[take] = a
        best[take] = res[take]
    if len(within) > 1:
        w = np.sort(np.stack(within, axis=1), axis=1)
        two = np.isfinite(w[:, 1])
        flag[two] |= w[two, 1] - w[two, 0] <= scale[two]
    return labels, flag


def eps_axis_vote(P, Q, G: int, eps: float):
    """The consensus accumulator of Eq. 9 at cell resolution: circle i counts in cell c if
    some axis r of the cell satisfies |r . z_i| < eps, z_i = d_i/|d_i|.

    With F/(1 + u^2 + v^2) = d . r(u, v) (Eq. 12, 13), r . z < eps and r . z > -eps read
    F_minus = F - eps |d| (1 + u^2 + v^2) < 0 and F_plus = F + eps |d| (1 + u^2 + v^2) > 0;
    both are separable quadratics (circles of Eq. 13 with D != 0). The cell, being connected,
    meets the band iff min_cell F_minus < 0 and max_cell F_plus > 0. eps = 0 leaves the open
    version of the curve test; eps > 0 adds the cells within angular distance asin(eps) of the
    great circle. The decision is flagged when either extreme is within BAND |d| of zero.
    Returns dict(grid, lo, hi)."""
    D, deg = _differences(P, Q)
    e = grid_edges(G)
    grid = np.zeros((G, G), dtype=np.int64)
    lo = np.zeros((G, G), dtype=np.int64)
    hi = np.zeros((G, G), dtype=np.int64)
    for i in np.flatnonzero(~deg):
        d = D[i]
        nd = float(np.sqrt(d @ d))
        cm, cp = d[2] - eps * nd, d[2] + eps * nd
        # F_minus = cm (u^2 + v^2) + 2 d1 u + 2 d2 v - cp ; F_plus = cp (u^2 + v^2) + 2 d1 u + 2 d2 v - cm
        gmin, _ = _quadratic_range(cm, 2.0 * d[0], e[:-1], e[1:])
        hmin, _ = _quadratic_range(cm, 2.0 * d[1], e[:-1], e[1:])
        _, gmax = _quadratic_range(cp, 2.0 * d[0], e[:-1], e[1:])
        _, hmax = _quadratic_range(cp, 2.0 * d[1], e[:-1], e[1:])
        Fm = hmin[:, None] + gmin[None, :] - cp
        Fp = hmax[:, None] + gmax[None, :] - cm
        voted = (Fm < 0.0) & (Fp > 0.0)
        tol = BAND * nd
        flag = (np.abs(Fm) <= tol) | (np.abs(Fp) <= tol)
        grid += voted
        lo += voted & ~flag
        hi += voted | flag
    return dict(grid=grid, lo=lo, hi=hi)


def eps_cell_votes(P, Q, G: int, eps: float, rows, cols):
    """Votes of selected cells of the eps-band accumulator over all circles (the test of
    ``eps_axis_vote`` evaluated cell by cell, for 10^6 circles). Returns (count, lo, hi)."""
    D, deg = _differences(P, Q)
    e = grid_edges(G)
    nd = np.sqrt(np.einsum("ij,ij->i", D, D))
    cm, cp = D[:, 2] - eps * nd, D[:, 2] + eps * nd
    out = np.zeros((3, len(rows)), dtype=np.int64)
    for k, (r, c) in enumerate(zip(rows, cols)):
        gmin, _ = _quadratic_range(cm, 2.0 * D[:, 0], e[c], e[c + 1])
        hmin, _ = _quadratic_range(cm, 2.0 * D[:, 1], e[r], e[r + 1])
        _, gmax = _quadratic_range(cp, 2.0 * D[:, 0], e[c], e[c + 1])
        _, hmax = _quadratic_range(cp, 2.0 * D[:, 1], e[r], e[r + 1])
        Fm = gmin + hmin - cp
        Fp = gmax + hmax - cm
        voted = (Fm < 0.0) & (Fp > 0.0) & ~deg
        flag = ((np.abs(Fm) <= BAND * nd) | (np.abs(Fp) <= BAND * nd)) & ~deg
        out[0, k] = voted.sum()
        out[1, k] = (voted & ~flag).sum()
        out[2, k] = (voted | flag).sum()
    return out[0], out[1], out[2]


def ls_axis(P, Q, select=None, hint=None):
    """The least-squares rotation axis of a set of pairs (Eq. 10): the unit r minimising
    sum_i (z_i . r)^2 with z_i = (p_i - q_i)/|p_i - q_i|, i.e. the eigenvector of
    S = sum_i z_i z_i^T for its smallest eigenvalue (numpy eigh). ``select`` is a boolean
    mask of the pairs to use (all when None); degenerate pairs are skipped. The sign is chosen
    so that r . hint >= 0, or r_z <= 0 without a hint (ties: r_z < 0, then r_y < 0, ...).

    Returns dict(axis, lam, S, gap) with lam the smallest eigenvalue (the residual sum of
    squares) and gap = (second smallest - smallest) / largest eigenvalue, the conditioning of
    the axis. axis is None when fewer than two independent directions are present."""
    D, deg = _differences(P, Q)
    use = ~deg if select is None else (np.asarray(select, dtype=bool) & ~deg)
    Z = D[use]
    if Z.shape[0] == 0:
        return dict(axis=None, lam=0.0, S=np.zeros((3, 3)), gap=0.0)
    Z = Z / np.linalg.norm(Z, axis=1, keepdims=True)
    S = Z.T @ Z
    w, V = np.linalg.eigh(S)
    if w[1] <= 1e-12 * max(w[2], 1e-300):
        return dict(axis=None, lam=float(w[0]), S=S, gap=0.0)
    r = V[:, 0]
    ref = np.asarray(hint, dtype=np.float64) if hint is not None else None
    if ref is not None:
        if r @ ref < 0:
            r = -r
    else:
        for k in (2, 1, 0):
            if r[k] != 0.0:
                if r[k] > 0:
                    r = -r
                break
    return dict(axis=r, lam=float(w[0]), S=S, gap=float((w[1] - w[0]) / w[2]))


# ---------------------------------------------------------------------------------------
# Algorithm 1's sampled rasteriser (used as a pin of the cell predicate)
# ---------------------------------------------------------------------------------------

def sampled_circle_cells(d, G: int, J: int, alpha0=(0.0, 0.0, 1.0)):
    """Cells hit by J points of the great circle of d, as Algorithm 1 draws it: a basis
    vector alpha1 orthogonal to z = d/|d| by Gram-Schmidt from alpha0, alpha2 = alpha1 x z,
    points alpha1 cos(t_j) + alpha2 sin(t_j) (the printed second cosine is read as a sine),
    stereographic projection (Eq. 11), and the cell that holds each point. Points outside
    the square are dropped. Returns a set of (row, col)."""
    z = np.asarray(d, dtype=np.float64)
    z = z / np.linalg.norm(z)
    a0 = np.asarray(alpha0, dtype=np.float64)
    a1 = a0 - (a0 @ z) * z
    if np.linalg.norm(a1) < 1e-6:
        a0 = np.array([1.0, 0.0, 0.0])
        a1 = a0 - (a0 @ z) * z
    a1 /= np.linalg.norm(a1)
    a2 = np.cross(a1, z)
    t = np.linspace(-math.pi, math.pi, J, endpoint=False)
    pts = np.cos(t)[:, None] * a1 + np.sin(t)[:, None] * a2
    pts = pts[pts[:, 2] < 1.0 - 1e-12]
    uv = np.stack([pts[:, 0] / (1.0 - pts[:, 2]), pts[:, 1] / (1.0 - pts[:, 2])], axis=1)
    inside = (np.abs(uv[:, 0]) < 1.0) & (np.abs(uv[:, 1]) < 1.0)
    uv = uv[inside]
    cols = np.floor((uv[:, 0] + 1.0) * G / 2.0).astype(int)
    rows = np.floor((uv[:, 1] + 1.0) * G / 2.0).astype(int)
    return set(zip(rows.tolist(), cols.tolist()))


#: half-width (plane units, times 1 + 1/|alpha0 - (alpha0.z) z|) of the band around cell edges
#: inside which a float32 sample may fall on either side
SAMPLE_BAND = 1e-5


def sample_basis(d):
    """The basis of the great circle of d used by Algorithm 1: z = d/|d|; alpha0 = e3 unless
    d1 = d2 = 0 exactly (then z = +-e3 and alpha0 = e1); alpha1 = alpha0 - (alpha0 . z) z
    (the projection of Algorithm 1 removed) normalised; alpha2 = alpha1 x z.
    Returns (alpha1, alpha2, |alpha0 - (alpha0 . z) z|).

    Reading: Algorithm 1 leaves alpha0 open; the rule above is one whose branch is decided
    exactly in any precision (d1 = d2 = 0 is a test on the inputs)."""
    d = np.asarray(d, dtype=np.float64)
    z = d / np.linalg.norm(d)
    a0 = np.array([1.0, 0.0, 0.0]) if (d[0] == 0.0 and d[1] == 0.0) else np.array([0.0, 0.0, 1.0])
    a1 = a0 - (a0 @ z) * z
    na = float(np.linalg.norm(a1))
    a1 = a1 / na
    return a1, np.cross(a1, z), na


def sampled_axis_vote(P, Q, G: int, J: int):
    """Algorithm 1's accumulator taken literally: for every pair, the J points
    alpha1 cos(t_j) + alpha2 sin(t_j) of its great circle, t_j = -pi + 2 pi j / J, are
    projected by Eq. 11 and each point inside the square adds one to its cell. A circle can
    therefore vote a cell several times, and a cell it only grazes may get no vote. (The
    printed second cosine is read as a sine.) Degenerate pairs (d = 0) do not vote.

    Flags: a sample whose u or v lies within eta = SAMPLE_BAND (1 + 1/|alpha0 - (alpha0.z)z|)
    of a cell edge (or of the square's border) may land on either side in float32; it counts
    in ``hi`` for every candidate cell and not in ``lo``.
    Returns dict(grid, lo, hi) of int64 G x G arrays [row (v), col (u)]."""
    D, deg = _differences(P, Q)
    t = -math.pi + 2.0 * math.pi * np.arange(J) / J
    ct, st = np.cos(t), np.sin(t)
    grid = np.zeros((G, G), dtype=np.int64)
    lo = np.zeros((G, G), dtype=np.int64)
    hi = np.zeros((G, G), dtype=np.int64)
    half = G / 2.0
    for i in np.flatnonzero(~deg):
        a1, a2, na = sample_basis(D[i])
        pts = ct[:, None] * a1[None, :] + st[:, None] * a2[None, :]
        w = 1.0 - pts[:, 2]
        ok = w > 0.0
        u = np.where(ok, pts[:, 0] / np.where(ok, w, 1.0), np.inf)
        v = np.where(ok, pts[:, 1] / np.where(ok, w, 1.0), np.inf)
        eta = SAMPLE_BAND * (1.0 + 1.0 / na) * half  # in cell units
        fu, fv = (u + 1.0) * half, (v + 1.0) * half
        inside = (np.abs(u) < 1.0) & (np.abs(v) < 1.0)
        with np.errstate(invalid="ignore"):  # points at the pole: inf - inf, never flagged
            near_u = np.abs(fu - np.round(fu)) <= eta
            near_v = np.abs(fv - np.round(fv)) <= eta
        flag = (near_u | near_v) & np.isfinite(fu) & np.isfinite(fv)
        col = np.floor(fu[inside]).astype(np.int64)
        row = np.floor(fv[inside]).astype(np.int64)
        np.add.at(grid, (row, col), 1)
        sure = inside & ~flag
        np.add.at(lo, (np.floor(fv[sure]).astype(np.int64), np.floor(fu[sure]).astype(np.int64)), 1)
        np.add.at(hi, (np.floor(fv[sure]).astype(np.int64), np.floor(fu[sure]).astype(np.int64)), 1)
        for k in np.flatnonzero(flag):
            cols = {int(np.floor(fu[k] - eta)), int(np.floor(fu[k] + eta))}
            rows = {int(np.floor(fv[k] - eta)), int(np.floor(fv[k] + eta))}
            for r in rows:
                for c in cols:
                    if 0 <= r < G and 0 <= c < G:
                        hi[r, c] += 1
    return dict(grid=grid, lo=lo, hi=hi)


# ---------------------------------------------------------------------------------------
# The whole estimator
# ---------------------------------------------------------------------------------------

def solve(P, Q, G: int, J: int, k: int = 1, nms_deg: float = 2.0, w: int = 1,
          window: int = 1, tau: float = 0.05, grid=None, subcell: bool = False):
    """Algorithm 1 end to end, plus the multi-rotation form (Sec. IV-D) and refinement.

    For each of up to k peaks: axis r (Eq. 12 at the cell centre, r_z <= 0), gate, angle
    histogram, peak bin b and its centre theta_hat; if theta_hat < 0 the pair (r, theta) is
    replaced by (-r, -theta) so that theta lies in [0, pi] as in Sec. III-A; R_vote by
    Rodrigues (Eq. 2); vote set V; R1 = Kabsch(V). Then labels against every R1 and
    R = Kabsch over each label class.

    With ``subcell`` the axis of each peak is ``subcell_axis`` at ``subcell_offset`` instead
    of the cell centre (the gate still uses the peak's cells).

    ``grid`` may be passed in (e.g. a float32 implementation's grid) to evaluate the later
    stages on it. Returns a dict with every intermediate."""
    P = np.asarray(P, dtype=np.float32)
    Q = np.asarray(Q, dtype=np.float32)
    out = {}
    if grid is None:
        av = axis_vote(P, Q, G)
        out["axis"] = av
        grid = av["grid"]
    peaks = top_k_cells(grid, k, nms_deg)
    out["peaks"] = peaks
    rots = []
    for (row, col, cnt) in peaks:
        du, dv = subcell_offset(grid, row, col)
        r = subcell_axis(G, row, col, du, dv) if subcell else cell_axis(G, row, col)
        gate, gflag = window_gate(P, Q, G, row, col, w)
        vote = angle_vote(P, Q, r, gate, gflag, J)
        b, th = angle_peak(vote["hist"])
        V, V_lo, V_hi = vote_set(vote, b, J, window)
        axis, theta = (r, th) if th >= 0 else (-r, -th)
        R_vote = rodrigues(axis, theta)
        R1 = kabsch(P[V], Q[V]) if V.any() else R_vote
        rots.append(dict(cell=(row, col), axis_votes=cnt, axis=axis, r_cell=r, theta=theta,
                         cell_offset=(du, dv),
                         bin=b, angle_votes=int(vote["hist"][b]), R_vote=R_vote, gate=gate,
                         gate_flag=gflag, vote=vote, V=V, V_lo=V_lo, V_hi=V_hi, R1=R1))
    labels, lflag = assign_labels(P, Q, [x["R1"] for x in rots], tau)
    for a, x in enumerate(rots):
        sel = labels == a
        x["R"] = kabsch(P[sel], Q[sel]) if sel.any() else x["R1"]
        x["n_inliers"] = int(sel.sum())
    out["rotations"] = rots
    out["labels"] = labels
    out["label_flag"] = lflag
    return out
