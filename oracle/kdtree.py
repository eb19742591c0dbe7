"""KD-tree ordering of the points into tiles (oracle; test infrastructure).

Section 6 (clustering paragraph): points are split recursively; each cluster is
sorted along the largest dimension of its bounding box and split into a left
cluster of b * 2^(ceil(log2(n/b)) - 1) points (half the power of two of tiles
that covers the cluster, times the tile size) and a right cluster with the
rest, so every leaf holds b points except possibly the last.

Readings where the text is not explicit (also listed in the design notes):
  * "largest dimension": the axis with the largest (max - min) extent of the
    cluster's points; ties go to the lowest axis index.
  * sort key: (coordinate along that axis, original point index), ascending.
  * a cluster of n <= b points is a leaf and keeps the order it arrived in.
"""
from __future__ import annotations

import numpy as np


def _left_size(n: int, b: int) -> int:
    p = 0
    while b * (1 << p) < n:  # smallest p with b * 2^p >= n, i.e. ceil(log2(n/b))
        p += 1
    return b * (1 << (p - 1))


def kd_order(x: np.ndarray, b: int) -> np.ndarray:
    """Return perm (int64, length N): perm[p] = original index of the p-th ordered point."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    out: list[np.ndarray] = []

    def rec(idx: np.ndarray) -> None:
        n = len(idx)
        if n <= b:
            out.append(idx)
            return
        pts = x[idx]
        ext = pts.max(axis=0) - pts.min(axis=0)
        axis = int(np.argmax(ext))  # argmax returns the first maximum: lowest axis on ties
        order = np.lexsort((idx, pts[:, axis]))  # primary key: coordinate, secondary: index
        s = idx[order]
        nl = _left_size(n, b)
        rec(s[:nl])
        rec(s[nl:])

    rec(np.arange(N, dtype=np.int64))
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
