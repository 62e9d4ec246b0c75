"""FP64 oracle of the Fast Gaussian Accumulator (Section 6): the refined icosahedron, the
nearest cell of each normal, the histogram, and peak detection on the cell graph.

TEST INFRASTRUCTURE (see the package docstring): only the tests, the smoke check and the
benchmark's CPU legs use it; the CUDA library shares no code with it.

Definitions (Section 6.1):
  - Level 0 is the icosahedron with the 12 vertices (+-1, +-phi, 0), (0, +-1, +-phi),
    (+-phi, 0, +-1) scaled to unit length, in the order listed in ICO_VERTICES, and the 20 faces
    formed by every triple of mutually adjacent vertices (edge length 2), taken in lexicographic
    order of the sorted triple and oriented counter-clockwise seen from outside.
  - Level l + 1 splits every face (a, b, c) of level l into four, with the edge midpoints
    projected onto the unit sphere: child 0 = (a, ab, ca), 1 = (ab, b, bc), 2 = (ca, bc, c),
    3 = (ab, bc, ca). Face 4 p + j of level l + 1 is child j of face p. The cells of the
    accumulator are the faces of the chosen level.
  - A cell's surface normal is the unit normal of its (flat) face, (b - a) x (c - a) normalised.
  - A normal belongs to the cell whose surface normal is closest to it (Section 6.1.3), i.e. the
    largest dot product; the first such cell on exact ties.
  - Peaks (Section 6.2, on the cell graph instead of the unwrapped image): a cell whose count is
    above v_min and not below the count of any of its 1-ring neighbours (cells sharing a
    vertex), where a plateau keeps its lowest-index cell. Peaks closer than d_peak (Euclidean
    distance of the surface normals) are merged by single-linkage agglomerative clustering into
    the count-weighted mean of their normals, renormalised; clusters are returned by
    decreasing total count.
"""
from __future__ import annotations

import numpy as np

PHI = (1.0 + 5.0 ** 0.5) / 2.0
ICO_VERTICES = np.array([(-1, PHI, 0), (1, PHI, 0), (-1, -PHI, 0), (1, -PHI, 0), (0, -1, PHI), (0, 1, PHI),
                         (0, -1, -PHI), (0, 1, -PHI), (PHI, 0, -1), (PHI, 0, 1), (-PHI, 0, -1), (-PHI, 0, 1)],
                        dtype=np.float64)


def icosahedron(level: int):
    """Refined icosahedron of Section 6.1.1 -> (V float64 [nv, 3] unit vertices, F int64 [20 4^level, 3])."""
    V = [v / np.linalg.norm(v) for v in ICO_VERTICES]
    F = []
    for i in range(12):
        for j in range(i + 1, 12):
            for k in range(j + 1, 12):
                if all(abs(np.linalg.norm(ICO_VERTICES[a] - ICO_VERTICES[b]) - 2.0) < 1e-9
                       for a, b in ((i, j), (j, k), (i, k))):
                    F.append((i, j, k) if np.linalg.det(ICO_VERTICES[[i, j, k]]) > 0 else (i, k, j))
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                p = V[a] + V[b]
                V.append(p / np.linalg.norm(p))
                mid[key] = len(V) - 1
            return mid[key]

        nxt = []
        for a, b, c in F:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nxt += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        F = nxt
    return np.array(V), np.array(F, dtype=np.int64)


def cell_normals(V: np.ndarray, F: np.ndarray) -> np.ndarray:
    """Unit surface normal of every cell (face)."""
    A, B, C = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(B - A, C - A)
    return n / np.linalg.norm(n, axis=1)[:, None]


def neighbours(F: np.ndarray) -> list:
    """1-ring vertex adjacency of every cell (cells sharing at least one vertex), ascending."""
    inc = {}
    for t, f in enumerate(F):
        for v in f:
            inc.setdefault(int(v), set()).add(t)
    return [sorted(set().union(*(inc[int(v)] for v in f)) - {t}) for t, f in enumerate(F)]


def nearest_cell(normals: np.ndarray, N: np.ndarray, chunk: int = 65536) -> np.ndarray:
    """Index of the cell with the largest dot product for every row of `normals` (brute force)."""
    normals = np.asarray(normals, np.float64)
    out = np.empty(len(normals), np.int64)
    for s in range(0, len(normals), chunk):
        out[s:s + chunk] = (normals[s:s + chunk] @ N.T).argmax(1)
    return out


def sampled(normals: np.ndarray, mask, stride: int) -> np.ndarray:
    """Indices of the normals the accumulator integrates: every stride-th triangle (Section 6.3's
    sampling), kept by the mask when there is one, with a finite normal."""
    normals = np.asarray(normals).reshape(-1, 3)
    idx = np.arange(0, len(normals), stride)
    ok = np.isfinite(normals[idx]).all(1)
    if mask is not None:
        ok &= np.asarray(mask).reshape(-1)[idx] != 0
    return idx[ok]


def accumulate(normals: np.ndarray, level: int, mask=None, stride: int = 1):
    """Histogram of Section 6.1 -> (counts int64 [cells], cell of every triangle (-1 if not sampled))."""
    V, F = icosahedron(level)
    N = cell_normals(V, F)
    normals = np.asarray(normals, np.float64).reshape(-1, 3)
    idx = sampled(normals, mask, stride)
    cells = np.full(len(normals), -1, np.int64)
    cells[idx] = nearest_cell(normals[idx], N)
    counts = np.bincount(cells[idx], minlength=len(F))
    return counts, cells


def peaks(counts: np.ndarray, level: int, v_min: float, d_peak: float):
    """Dominant normals from a histogram (definition in the module docstring)
    -> (normals float64 [p, 3], weights int64 [p]), by decreasing weight."""
    V, F = icosahedron(level)
    N = cell_normals(V, F)
    nb = neighbours(F)
    counts = np.asarray(counts)
    pk = [i for i in range(len(F)) if counts[i] > v_min and all(
        counts[i] > counts[j] or (counts[i] == counts[j] and i < j) for j in nb[i])]
    # single linkage: peaks within d_peak of each other end in one cluster
    parent = list(range(len(pk)))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for a in range(len(pk)):
        for b in range(a + 1, len(pk)):
            if np.linalg.norm(N[pk[a]] - N[pk[b]]) < d_peak:
                ra, rb = find(a), find(b)
                if ra != rb:
                    parent[max(ra, rb)] = min(ra, rb)
    clusters = {}
    for a in range(len(pk)):
        clusters.setdefault(find(a), []).append(pk[a])
    out = []
    for members in clusters.values():
        w = counts[members].astype(np.float64)
        v = (N[members] * w[:, None]).sum(0)
        out.append((v / np.linalg.norm(v), int(w.sum()), min(members)))
    out.sort(key=lambda t: (-t[1], t[2]))
    return np.array([o[0] for o in out]).reshape(-1, 3), np.array([o[1] for o in out], np.int64)
