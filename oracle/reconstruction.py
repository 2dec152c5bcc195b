"""Oracle reconstruction: MUSCL on primitives and MUSCL-BVD-THINC on phi.

TEST INFRASTRUCTURE ONLY (plain PyTorch CPU float64).

Cites arXiv 2009.14555:
  * Section 3.1: MUSCL reconstruction of cell-centred primitive variables
    (after Johnsen & Colonius) and the MUSCL-BVD-THINC interface steepening;
  * Appendix A: THINC tanh profile, its cell-edge values q_L, q_R through the
    constants A, B, C, the mixed-cell test, the total boundary variation (TBV)
    of each candidate and the BVD choice, and the multi-dimensional
    steepness beta = beta0 |n_d| + 0.01 with a Youngs normal.

Readings: the limiter is minmod (the paper names none), or van Leer's as an
option (the harmonic mean 2 a b / (a + b) of same-sign one-sided
differences, van Leer 1974; 0 otherwise); THINC acts on the
volume fraction phi1 only; "q_max" in the edge formulas is the jump
max(q_{i-1}, q_{i+1}) - q_min; the mixed-cell test is strict on both sides; BVD
picks THINC only when its TBV is strictly smaller; in a non-mixed cell the
THINC candidate is the MUSCL one; in 1D |n_d| = 1.
"""
from __future__ import annotations

import torch

THINC_EPS = 1e-20   # epsilon of Appendix A
THINC_DELTA = 1e-5  # delta of the mixed-cell test, Appendix A
BETA0 = 2.5         # beta0 of Appendix A


def minmod(a, b):
    """minmod(a, b) = sign(a) min(|a|, |b|) if a b > 0 else 0."""
    return torch.where(a * b > 0, torch.sign(a) * torch.minimum(a.abs(), b.abs()),
                       torch.zeros_like(a))


def vanleer(a, b):
    """van Leer's limited slope: 2 a b / (a + b) if a b > 0 else 0."""
    ab = a * b
    pos = ab > 0
    return torch.where(pos, 2.0 * ab / torch.where(pos, a + b, torch.ones_like(a)), torch.zeros_like(a))


def muscl_faces(w, limiter="minmod"):
    """Limited linear reconstruction along the last axis.

    Returns (wL, wR): the values at the left (x_{i-1/2}) and right (x_{i+1/2})
    edges of every cell that has two neighbours; the outermost cells get NaN.
    """
    wL = torch.full_like(w, float("nan"))
    wR = torch.full_like(w, float("nan"))
    lim = {"minmod": minmod, "vanleer": vanleer}[limiter]
    d = lim(w[..., 1:-1] - w[..., :-2], w[..., 2:] - w[..., 1:-1])
    wL[..., 1:-1] = w[..., 1:-1] - 0.5 * d
    wR[..., 1:-1] = w[..., 1:-1] + 0.5 * d
    return wL, wR


def thinc_faces(q, beta):
    """THINC edge values (Appendix A) for every cell with two neighbours.

    Returns (qL, qR, mixed): edge values and the mixed-cell mask.  Outside
    mixed cells the returned values are meaningless (mask them).
    """
    qm, qc, qp = q[..., :-2], q[..., 1:-1], q[..., 2:]
    b = beta[..., 1:-1]
    qmin = torch.minimum(qm, qp)
    qmax = torch.maximum(qm, qp) - qmin          # the jump across the cell
    theta = torch.sign(qp - qm)
    C = (qc - qmin + THINC_EPS) / (qmax + THINC_EPS)
    mixed = (C > THINC_DELTA) & (C < 1 - THINC_DELTA) & ((qp - qc) * (qc - qm) > 0)
    # keep the transcendental arguments finite where the mask is off
    th = torch.where(mixed, theta, torch.ones_like(theta))
    C = torch.where(mixed, C, torch.full_like(C, 0.5))
    Bc = torch.exp(th * b * (2 * C - 1))
    tb = torch.tanh(b)
    Ac = (Bc / torch.cosh(b) - 1) / tb
    qL = qmin + 0.5 * qmax * (1 + th * Ac)
    qR = qmin + 0.5 * qmax * (1 + th * (tb + Ac) / (1 + Ac * tb))
    pad = torch.full_like(q[..., :1], float("nan"))
    padb = torch.zeros_like(q[..., :1], dtype=torch.bool)
    return (torch.cat([pad, qL, pad], -1), torch.cat([pad, qR, pad], -1),
            torch.cat([padb, mixed, padb], -1))


def bvd_select(mL, mR, tL, tR, mixed):
    """BVD choice between the MUSCL (m) and THINC (t) candidates (Appendix A).

    Candidates are defined for cells 1..n-2 along the last axis; the choice is
    made for cells 2..n-3 (it needs the neighbours' candidates).  Returns the
    chosen (L, R) edge values with NaN where no choice is possible.
    """
    tL = torch.where(mixed, tL, mL)
    tR = torch.where(mixed, tR, mR)

    def tbv(pL, pR):
        # the four neighbour combinations of Appendix A
        a_m = (mR[..., 1:-3] - pL[..., 2:-2]).abs()
        a_t = (tR[..., 1:-3] - pL[..., 2:-2]).abs()
        b_m = (pR[..., 2:-2] - mL[..., 3:-1]).abs()
        b_t = (pR[..., 2:-2] - tL[..., 3:-1]).abs()
        return torch.minimum(torch.minimum(a_m + b_m, a_t + b_t),
                             torch.minimum(a_m + b_t, a_t + b_m))

    use_t = tbv(tL, tR) < tbv(mL, mR)
    L = torch.full_like(mL, float("nan"))
    R = torch.full_like(mR, float("nan"))
    L[..., 2:-2] = torch.where(use_t, tL[..., 2:-2], mL[..., 2:-2])
    R[..., 2:-2] = torch.where(use_t, tR[..., 2:-2], mR[..., 2:-2])
    return L, R


def youngs_abs_normal(phi, dx, dy):
    """|n_x|, |n_y| of the Youngs normal on a (ny, nx) array (interior cells).

    Youngs' method: the gradient of phi at the four cell corners (from the 2x2
    blocks that share each corner), averaged to the cell centre.  Where the
    gradient vanishes both components are taken as 1.  The outermost ring of
    cells gets NaN.
    """
    # corner gradients on the (ny-1, nx-1) grid of corners
    gx = (phi[1:, 1:] + phi[:-1, 1:] - phi[1:, :-1] - phi[:-1, :-1]) / (2 * dx)
    gy = (phi[1:, 1:] + phi[1:, :-1] - phi[:-1, 1:] - phi[:-1, :-1]) / (2 * dy)
    cx = 0.25 * (gx[1:, 1:] + gx[:-1, 1:] + gx[1:, :-1] + gx[:-1, :-1])
    cy = 0.25 * (gy[1:, 1:] + gy[:-1, 1:] + gy[1:, :-1] + gy[:-1, :-1])
    n2 = cx * cx + cy * cy
    pos = n2 > 0  # sqrt taken only where positive so that its derivative stays finite
    norm = torch.where(pos, torch.sqrt(torch.where(pos, n2, torch.ones_like(n2))), torch.zeros_like(n2))
    zero = norm == 0
    nx_ = torch.where(zero, torch.ones_like(cx), cx.abs() / torch.where(zero, torch.ones_like(norm), norm))
    ny_ = torch.where(zero, torch.ones_like(cy), cy.abs() / torch.where(zero, torch.ones_like(norm), norm))
    outx = torch.full_like(phi, float("nan"))
    outy = torch.full_like(phi, float("nan"))
    outx[1:-1, 1:-1] = nx_
    outy[1:-1, 1:-1] = ny_
    return outx, outy


def thinc_beta(abs_n):
    """beta = beta0 |n_d| + 0.01 (Appendix A)."""
    return BETA0 * abs_n + 0.01
