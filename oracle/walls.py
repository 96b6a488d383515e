"""FP64 tagging of a lattice by a triangulated fixed wall and the
Bouzidi-Firdaouss-Lallemand distances measured to the wall's markers
(Section "Boundary conditions on fixed bodies", Eq. qbouzidi).

TEST INFRASTRUCTURE (see the package docstring): never imported by the product.

The paper's rule, step by step:
  1. the markers of a triangulated body are the centroids of its triangles;
  2. a node whose cell holds a marker is solid;
  3. a node that is not solid and has a solid node at x + e_i is a boundary
     node, and a_i = 1 for every such direction i;
  4. q_i = |x_b - x_L| / |x_b - x_s| with x_s = x_b + e_i and x_L "the
     corresponding Lagrangian marker";
  5. every other node is fluid.
Readings (W):
  W1  the cell of a node is the unit cube centred on it: a marker at c lies in
      the cell of the node floor(c + 1/2) per axis (the round-half-up node of
      the MLS support, Reading M2); markers outside a non-periodic box are
      dropped, periodic axes wrap;
  W2  the corresponding marker is, of the markers in the cell of x_s, the one
      nearest to x_b (the smallest q: the wall is at least that close);
  W3  a link toward a node that is solid without holding a marker (a solid
      tag given beforehand, e.g. a box edge) gets q = 1/2 (halfway
      bounce-back), as the analytic voxelisation does for such nodes;
  W4  q is clipped to [1e-6, 1], the range the wall rule takes (a marker in
      the far corner of the cell gives |x_b - x_L| up to |e_i| + sqrt(3)/2);
  W5  distances are taken as sqrt((dx*dx + dy*dy) + dz*dz) in FP64 and q is
      rounded to FP32 once, after the clip.
Links are returned in (node, direction) order, like the analytic voxeliser.
"""
from __future__ import annotations

import numpy as np

from .lattice import E

SOLID = 1
FLUID = 0
Q_MIN = 1e-6


def markers(verts, tris):
    """Step 1: triangle centroids (v0 + v1 + v2) / 3, (M, 3) FP64."""
    V = np.asarray(verts, dtype=np.float64)
    T = np.asarray(tris, dtype=np.int64)
    return (V[T[:, 0]] + V[T[:, 1]] + V[T[:, 2]]) / 3.0


def marker_cells(L, shape, periodic):
    """Reading W1: the node of each marker's cell, as integer coordinates
    (M, 3) (periodic axes wrapped) and a mask of the markers inside the box."""
    dims = np.asarray(shape, dtype=np.int64)
    raw = np.floor(L + 0.5).astype(np.int64)
    ok = np.ones(L.shape[0], dtype=bool)
    cell = raw.copy()
    for ax in range(3):
        if periodic[ax]:
            cell[:, ax] = np.mod(raw[:, ax], dims[ax])
        else:
            ok &= (raw[:, ax] >= 0) & (raw[:, ax] < dims[ax])
    return raw, cell, ok


def voxelise_markers(verts, tris, shape, periodic=(False, False, False), tag_in=None):
    """Steps 1-5 over a box of shape (nx, ny, nz).  tag_in (optional, flat)
    marks nodes that are solid beforehand.  Returns (tag u8 flat, node u32,
    dir u32, q f32) with the links in (node, direction) order."""
    nx, ny, nz = (int(s) for s in shape)
    N = nx * ny * nz
    tag = np.zeros(N, dtype=np.uint8) if tag_in is None else np.array(tag_in, dtype=np.uint8).copy()
    L = markers(verts, tris)
    raw, cell, ok = marker_cells(L, shape, periodic)
    L, raw, cell = L[ok], raw[ok], cell[ok]
    flat = cell[:, 0] + nx * (cell[:, 1] + ny * cell[:, 2])
    # step 2
    tag[flat] = SOLID
    # step 3: boundary nodes and their directions
    n = np.nonzero(tag == FLUID)[0]
    X, Y, Z = n % nx, (n // nx) % ny, n // (nx * ny)
    nodes, dirs = [], []
    for i in range(1, 19):
        s = [X + E[i, 0], Y + E[i, 1], Z + E[i, 2]]
        inside = np.ones(n.shape[0], dtype=bool)
        for ax, d in enumerate((nx, ny, nz)):
            if periodic[ax]:
                s[ax] = np.mod(s[ax], d)
            else:
                inside &= (s[ax] >= 0) & (s[ax] < d)
        nb = np.where(inside, s[0] + nx * (s[1] + ny * s[2]), 0)
        hit = inside & (tag[nb] == SOLID)
        nodes.append(n[hit])
        dirs.append(np.full(int(hit.sum()), i, dtype=np.int64))
    nodes = np.concatenate(nodes)
    dirs = np.concatenate(dirs)
    order = np.lexsort((dirs, nodes))
    nodes, dirs = nodes[order], dirs[order]
    # step 4 with Reading W2: each marker offers its distance to every
    # boundary node b = x_s - e_i of its cell; the link keeps the smallest
    key = nodes * 19 + dirs
    dist = np.full(nodes.shape[0], np.inf)
    for i in range(1, 19):
        if key.shape[0] == 0:
            break
        braw = raw - E[i][None, :]
        bc = braw.copy()
        inside = np.ones(braw.shape[0], dtype=bool)
        for ax, d in enumerate((nx, ny, nz)):
            if periodic[ax]:
                bc[:, ax] = np.mod(braw[:, ax], d)
            else:
                inside &= (braw[:, ax] >= 0) & (braw[:, ax] < d)
        k = np.where(inside, (bc[:, 0] + nx * (bc[:, 1] + ny * bc[:, 2])) * 19 + i, -1)
        pos = np.minimum(np.searchsorted(key, k), key.shape[0] - 1)
        has = inside & (key[pos] == k)
        dx = braw[:, 0].astype(np.float64) - L[:, 0]
        dy = braw[:, 1].astype(np.float64) - L[:, 1]
        dz = braw[:, 2].astype(np.float64) - L[:, 2]
        d = np.sqrt((dx * dx + dy * dy) + dz * dz)
        np.minimum.at(dist, pos[has], d[has])
    elen = np.sqrt((E[dirs] ** 2).sum(axis=1).astype(np.float64))
    q = np.where(np.isfinite(dist), dist / elen, 0.5)       # Reading W3
    q = np.clip(q, Q_MIN, 1.0)                                # Reading W4
    return tag, nodes.astype(np.uint32), dirs.astype(np.uint32), q.astype(np.float32)
