"""Icosphere surface meshes for the bead membranes (Sec. 2.2: each bead is an
icosahedron refined recursively into a triangulated sphere).

This module produces INPUT geometry only (node coordinates and triangle
connectivity).  It holds none of the time-step arithmetic: both the oracle and
the CUDA path receive the arrays it returns and compute everything else
(reference shapes, strains, forces) on their own.

Construction (a reading of Sec. 2.2, which names the method but not its
details): the 12 icosahedron vertices are the cyclic permutations of
(0, +-1, +-phi), normalised to the unit sphere; each refinement splits every
triangle into four through its edge midpoints, and every new midpoint is
projected back onto the unit sphere.  After s refinements the mesh has
V = 10*4^s + 2 nodes, E = 30*4^s edges and F = 20*4^s triangles.  Triangles
are oriented counter-clockwise seen from outside (outward normals).  The node
set is mirror-symmetric in x, y and z.
"""
from __future__ import annotations

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def icosahedron():
    """Return (vertices[12,3] on the unit sphere, faces[20,3] outward)."""
    v = []
    for a in (-1.0, 1.0):
        for b in (-_PHI, _PHI):
            v.append((0.0, a, b))
            v.append((a, b, 0.0))
            v.append((b, 0.0, a))
    v = np.array(v, dtype=np.float64)
    # faces are the vertex triples whose pairwise distances all equal the edge length 2
    faces = []
    n = len(v)
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    adj = np.abs(d2 - 4.0) < 1e-9
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    faces.append([i, j, k])
    faces = np.array(faces, dtype=np.int64)
    assert faces.shape == (20, 3)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, _orient_outward(v, faces)


def _orient_outward(v, faces):
    out = faces.copy()
    for t, (a, b, c) in enumerate(faces):
        n = np.cross(v[b] - v[a], v[c] - v[a])
        if np.dot(n, v[a] + v[b] + v[c]) < 0:
            out[t] = (a, c, b)
    return out


def icosphere(subdiv: int):
    """Unit icosphere after `subdiv` midpoint refinements.

    Returns (nodes[V,3] float64, tris[F,3] int32).  Node order is
    deterministic: the 12 icosahedron vertices first, then midpoints in the
    order they are first created.
    """
    v, f = icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(subdiv):
        cache = {}
        nf = []

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            if key not in cache:
                p = (np.asarray(verts[i]) + np.asarray(verts[j])) * 0.5
                p = p / np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf.extend([(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)])
        f = np.array(nf, dtype=np.int64)
    nodes = np.array(verts, dtype=np.float64)
    return nodes, f.astype(np.int32)


def edges_of(tris):
    """Unique undirected edges of a triangle list (sorted pairs)."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e.sort(axis=1)
    return np.unique(e, axis=0)
