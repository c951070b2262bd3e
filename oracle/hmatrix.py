"""Cluster trees, block cluster tree and admissibility (oracle, FP64).

Follows Sec. 3.1 (Eqs. (3.10)-(3.11)): clusters are bisected by principal
component analysis until #cluster <= b_min; the block cluster tree pairs
clusters from the root I x J; a block is far (low rank) when

    min(diam(tau), diam(sigma)) <= eta dist(tau, sigma)

and near (dense) when it is an inadmissible pair of leaves.  Readings of what
the paper leaves open:

* split: principal axis = eigenvector of the largest eigenvalue of the
  covariance of the cluster's points, signed so that its largest-magnitude
  component is positive; points with projection (about the mean) < 0 go to
  son 1, the rest (ties included) to son 2, each son keeping the original
  order; if a son would be empty, split the sorted projections (stable) at
  the median instead.
* boxes: axis-aligned boxes enclosing the supports of the indices (a point
  for a collocation row, the element for a P0 column, the union of the
  elements around a node for a P1 column); diam = box diagonal,
  dist = box-to-box Euclidean distance (0 when they touch).
* admissible only when dist > 0.
* recursion: admissible -> far leaf; both clusters leaves -> near leaf;
  otherwise split the clusters that have sons.
Pins: partition of I x J (every index pair in exactly one block), leaf
sizes, admissibility of every far block, brute-force PCA on tiny inputs
(tests/test_oracle_hmatrix.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cluster:
    idx: np.ndarray                 # original indices, in cluster order
    lo: np.ndarray
    hi: np.ndarray
    sons: list = field(default_factory=list)
    offset: int = 0                 # position of idx[0] in the permutation

    @property
    def size(self):
        return len(self.idx)

    @property
    def diam(self):
        return float(np.linalg.norm(self.hi - self.lo))


def principal_axis(pts: np.ndarray) -> np.ndarray:
    c = pts - pts.mean(axis=0)
    cov = c.T @ c
    w, v = np.linalg.eigh(cov)
    ax = v[:, int(np.argmax(w))]
    k = int(np.argmax(np.abs(ax)))
    return ax if ax[k] > 0 else -ax


def build_cluster_tree(pts, lo, hi, leaf: int) -> Cluster:
    """PCA bisection of the index set {0..n-1} (points pts, support boxes
    [lo, hi] per index) down to clusters of at most ``leaf`` indices."""
    pts, lo, hi = (np.asarray(a, dtype=np.float64) for a in (pts, lo, hi))

    def rec(idx, offset):
        cl = Cluster(idx=idx, lo=lo[idx].min(axis=0), hi=hi[idx].max(axis=0), offset=offset)
        if len(idx) <= leaf:
            return cl
        p = pts[idx]
        ax = principal_axis(p)
        proj = (p - p.mean(axis=0)) @ ax
        left = proj < 0.0
        if left.all() or (~left).all():
            order = np.argsort(proj, kind="stable")
            half = len(idx) // 2
            left = np.zeros(len(idx), dtype=bool)
            left[order[:half]] = True
        s1 = rec(idx[left], offset)
        s2 = rec(idx[~left], offset + int(left.sum()))
        cl.sons = [s1, s2]
        cl.idx = np.concatenate([s1.idx, s2.idx])
        return cl

    return rec(np.arange(len(pts)), 0)


def box_dist(a: Cluster, b: Cluster) -> float:
    d = np.maximum(0.0, np.maximum(a.lo - b.hi, b.lo - a.hi))
    return float(np.linalg.norm(d))


def admissible(a: Cluster, b: Cluster, eta: float) -> bool:
    dist = box_dist(a, b)
    return dist > 0.0 and min(a.diam, b.diam) <= eta * dist


@dataclass
class Block:
    rows: Cluster
    cols: Cluster
    far: bool


def build_block_tree(rt: Cluster, ct: Cluster, eta: float) -> list[Block]:
    out: list[Block] = []

    def rec(t, s):
        if admissible(t, s, eta):
            out.append(Block(t, s, True))
        elif not t.sons and not s.sons:
            out.append(Block(t, s, False))
        else:
            ts = t.sons if t.sons else [t]
            ss = s.sons if s.sons else [s]
            for a in ts:
                for b in ss:
                    rec(a, b)

    rec(rt, ct)
    return out


def support_boxes(geo, kind: str):
    """(points, lo, hi) for the rows ('centroids' | 'nodes', points) or the
    columns ('elements' | 'p1nodes', supports) of a mesh geometry."""
    if kind == "centroids":
        p = geo.centroid
        return p, p, p
    if kind == "nodes":
        p = geo.xyz
        return p, p, p
    if kind == "elements":
        P = geo.P
        return geo.centroid, P.min(axis=1), P.max(axis=1)
    if kind == "p1nodes":
        P = geo.P
        lo = np.full((geo.n_nodes, 3), np.inf)
        hi = np.full((geo.n_nodes, 3), -np.inf)
        for e, t in enumerate(geo.tri):
            for a in t:
                lo[a] = np.minimum(lo[a], P[e].min(axis=0))
                hi[a] = np.maximum(hi[a], P[e].max(axis=0))
        return geo.xyz, lo, hi
    raise ValueError(kind)
