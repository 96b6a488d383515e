"""FP64 moving-least-squares transfer between Lagrangian markers and the
lattice (Section "No-slip conditions for moving immersed boundaries").

TEST INFRASTRUCTURE (see the package docstring): never imported by the product.
"""
from __future__ import annotations

import numpy as np

from .lattice import Ef

# support: 3 nodes per axis (9 per plane, 27 in all) inside a cube of side
# 2 r_w = 2.6 dx centred on the marker (Reading M2)
SUPPORT_SIDE = 2.6
ALPHA = 0.3            # Eq. intKernel
PIVOT_TOL = 1e-10      # Reading M4: singular moment matrix -> nearest support node

OFFSETS = np.array([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)],
                   dtype=np.int64)   # k = (dx+1) + 3 (dy+1) + 9 (dz+1)


class Stencil:
    """MLS operator of a set of points: node indices (M,27), interpolation
    weights phi (M,27) and gradient weights grad (M,3,27)."""

    def __init__(self, nodes, phi, grad, weight, fallback=None):
        self.fallback = fallback
        self.nodes = nodes
        self.phi = phi
        self.grad = grad
        self.weight = weight

    def interp(self, values):
        """Eq. uLag: U = sum_k phi_k u^k.  values (N, c) -> (M, c)."""
        return np.einsum("mk,mkc->mc", self.phi, values[self.nodes])

    def gradient(self, values):
        """Linear coefficients a_1..a_3 of the MLS fit: d u_c / d x_j (M, c, 3)."""
        return np.einsum("mjk,mkc->mcj", self.grad, values[self.nodes])


def weight_function(r):
    """Eq. intKernel: W = exp(-(r/alpha)^2) for r <= 1, else 0."""
    return weight_of_r2(np.asarray(r) ** 2)


def weight_of_r2(r2):
    """Eq. intKernel written on r^2: exp(-r^2/alpha^2) for r <= 1, else 0.
    The support test looks at the real part only, so that a complex-step
    perturbation of the point (derivative checks) leaves the support set
    fixed and differentiates the weights."""
    return np.where(np.real(r2) <= 1.0, np.exp(-r2 / ALPHA ** 2), 0.0)


def leading_pivots(A):
    """Pivots of A = L D L^T without pivoting, as ratios of leading principal
    minors: d_j = det(A[:j+1,:j+1]) / det(A[:j,:j])."""
    dets = [np.ones(A.shape[0])] + [np.linalg.det(A[:, :j, :j]) for j in range(1, 5)]
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.stack([dets[j + 1] / dets[j] for j in range(4)], axis=1)


def stencil(lat, X):
    """MLS shape functions of Eq. l2norm at points X (M,3).

    J = sum_k W(x - x^k) [p^T(x^k) a(x) - u^k]^2 with the linear basis
    p = [1, x - X, y - Y, z - Z] (Reading M5) is minimised by
    a = A^{-1} sum_k W_k p_k u^k, A = sum_k W_k p_k p_k^T, so
    U(X) = a_0 gives phi_k = W_k (A^{-1} p_k)_0 and the gradient weights are
    W_k (A^{-1} p_k)_{1..3}.  The support is the 3x3x3 block around the
    nearest node (round half up), r_k = |X - x^k| / 2.6 (Reading M2).
    Reading M4: every Eulerian point of the support takes part, a solid one
    with the state of the wall it lies in (the populations of a solid node
    are the rest equilibrium: rho = 1, u = 0) and one off a non-periodic box
    with the state of the nearest box node (its coordinates clamped to the
    box).  Every support is then the full block, so the moment matrix is
    never singular; the nearest-point fallback below is a guard only.
    Dropping the solid points instead leaves a point near a wall with a few
    fluid points that carry large weights, and the explicit direct forcing
    (Eq. bodyforce) then amplifies the fluid velocity there from step to step.

    X may be complex (complex-step derivatives): every discrete decision (the
    nearest node, the support, the singularity test, the fallback node) is
    taken on the real part, so the shape functions are differentiated at a
    fixed stencil."""
    X = np.asarray(X).reshape(-1, 3)
    if not np.iscomplexobj(X):
        X = X.astype(np.float64)
    M = X.shape[0]
    base = np.floor(np.real(X) + 0.5).astype(np.int64)
    coords = base[:, None, :] + OFFSETS[None, :, :]          # (M,27,3) unwrapped
    pos = coords.astype(np.float64)
    dims = (lat.nx, lat.ny, lat.nz)
    ok = np.ones((M, 27), dtype=bool)
    wrapped = []
    for ax in range(3):
        c = coords[..., ax]
        if lat.periodic[ax]:
            c = c % dims[ax]
        else:
            c = np.clip(c, 0, dims[ax] - 1)
        wrapped.append(c)
    nodes = wrapped[0] + lat.nx * (wrapped[1] + lat.ny * wrapped[2])
    rel = pos - X[:, None, :]
    r2 = (rel * rel).sum(axis=2) / SUPPORT_SIDE ** 2
    Wk = np.where(ok, weight_of_r2(r2), 0.0)
    p = np.concatenate([np.ones((M, 27, 1)), rel], axis=2)    # (M,27,4)
    A = np.einsum("mk,mki,mkj->mij", Wk, p, p)
    piv = np.real(leading_pivots(A))
    a00 = np.real(A[:, 0, 0])
    good = (a00 > 0) & np.all(piv > PIVOT_TOL * np.where(a00 > 0, a00, 1.0)[:, None], axis=1)
    phi = np.zeros((M, 27), dtype=Wk.dtype)
    grad = np.zeros((M, 3, 27), dtype=Wk.dtype)
    if good.any():
        Ainv = np.linalg.inv(A[good])
        coef = np.einsum("mij,mkj->mik", Ainv, p[good]) * Wk[good][:, None, :]   # (m,4,27)
        phi[good] = coef[:, 0, :]
        grad[good] = coef[:, 1:, :]
    bad = ~good
    if bad.any():
        # the nearest support point takes the whole marker (largest W)
        has = np.real(Wk[bad]).max(axis=1) > 0
        kk = np.argmax(np.real(Wk[bad]), axis=1)
        rows = np.nonzero(bad)[0]
        phi[rows[has], kk[has]] = 1.0
    return Stencil(nodes, phi, grad, Wk, bad)


def node_velocity(f, nodes=None):
    """u = sum_i f_i e_i / rho (no force term) at the given nodes; (n,3)."""
    g = f if nodes is None else f[:, nodes]
    rho = g.sum(axis=0)
    return (Ef.T @ g).T / rho[:, None]


def node_density(f, nodes=None):
    g = f if nodes is None else f[:, nodes]
    return g.sum(axis=0)


def interpolate_velocity(f, st):
    """Eq. uLag applied to the fluid velocity u* = sum f e / rho of the current
    populations (Reading T1: the force term of the step is not known yet)."""
    flat = st.nodes.reshape(-1)
    u = node_velocity(f, flat).reshape(st.nodes.shape + (3,))
    return np.einsum("mk,mkc->mc", st.phi, u)


def spread(N, st, F, c):
    """Eq. bodyforce: f_ib^k = sum_l c_l phi^l_k F_l, summed over every marker
    whose support holds node k; c_l = A_l (Reading M3).  Returns (N,3)."""
    contrib = (c[:, None] * st.phi)[:, :, None] * F[:, None, :]
    out = np.zeros((N, 3), dtype=contrib.dtype)
    np.add.at(out, st.nodes.reshape(-1), contrib.reshape(-1, 3))
    return out
