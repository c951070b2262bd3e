"""Pins of the oracle's cluster/block trees and of the BDF2 convolution
quadrature."""
import math

import numpy as np
import pytest
from scipy import integrate

import synthetic as syn
from oracle import bem, cq, hmatrix


def test_principal_axis_brute_force():
    rng = np.random.default_rng(0)
    pts = rng.normal(size=(40, 3)) * np.array([3.0, 1.0, 0.5])
    ax = hmatrix.principal_axis(pts)
    c = pts - pts.mean(0)
    # brute force over directions on a fine sphere grid
    th, ph = np.meshgrid(np.linspace(0, np.pi, 361), np.linspace(0, 2 * np.pi, 721), indexing="ij")
    d = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1).reshape(-1, 3)
    var = ((c @ d.T) ** 2).sum(0)
    best = d[np.argmax(var)]
    assert abs(abs(best @ ax) - 1.0) < 1e-4


@pytest.mark.parametrize("leaf,eta,lvl", [(4, 2.0, 2), (8, 1.0, 2), (32, 2.0, 3)])
def test_block_tree_partition_and_admissibility(leaf, eta, lvl):
    xyz, tri = syn.icosphere(lvl)
    geo = bem.Geometry(xyz, tri)
    rt = hmatrix.build_cluster_tree(*hmatrix.support_boxes(geo, "nodes"), leaf)
    ct = hmatrix.build_cluster_tree(*hmatrix.support_boxes(geo, "elements"), leaf)
    blocks = hmatrix.build_block_tree(rt, ct, eta)
    cover = np.zeros((geo.n_nodes, geo.n_tris), int)
    for b in blocks:
        cover[np.ix_(b.rows.idx, b.cols.idx)] += 1
        if b.far:
            assert min(b.rows.diam, b.cols.diam) <= eta * hmatrix.box_dist(b.rows, b.cols)
            assert hmatrix.box_dist(b.rows, b.cols) > 0
        else:
            assert b.rows.size <= leaf and b.cols.size <= leaf
    assert (cover == 1).all()
    assert any(b.far for b in blocks)
    # the leaves of a cluster tree partition the index set
    def leaves(c):
        return [c] if not c.sons else leaves(c.sons[0]) + leaves(c.sons[1])
    idx = np.concatenate([c.idx for c in leaves(rt)])
    assert sorted(idx.tolist()) == list(range(geo.n_nodes))


def _conv_exact(kern, g, t):
    return integrate.quad(lambda tau: kern(t - tau) * g(tau), 0.0, t, epsabs=1e-13, epsrel=1e-12, limit=200)[0]


def test_cq_exponential_kernel_second_order():
    """K(s) = 1/(s + a) <-> exp(-a t); BDF2 CQ error O(dt^2)."""
    a, T = 2.0, 1.0
    g = lambda t: t ** 3 * math.exp(-t)
    errs = []
    for N in (20, 40, 80):
        dt = T / N
        tt = dt * np.arange(N + 1)
        y = cq.convolve(lambda s: 1.0 / (s + a), np.array([g(t) for t in tt]), N, dt).real
        ex = np.array([_conv_exact(lambda u: math.exp(-a * u), g, t) for t in tt])
        errs.append(np.abs(y - ex).max())
    assert errs[0] / errs[1] > 3.3 and errs[1] / errs[2] > 3.3
    assert errs[2] < 2e-4


def test_cq_delay_kernel():
    """K(s) = exp(-s d / c) / (4 pi d) <-> g(t - d / c) / (4 pi d)."""
    d, c, T = 0.3, 1.0, 1.0
    g = lambda t: math.sin(3 * t) ** 4
    errs = []
    for N in (40, 80, 160):
        dt = T / N
        tt = dt * np.arange(N + 1)
        y = cq.convolve(lambda s: np.exp(-s * d / c) / (4 * math.pi * d),
                        np.array([g(t) for t in tt]), N, dt).real
        ex = np.array([g(t - d / c) if t > d / c else 0.0 for t in tt]) / (4 * math.pi * d)
        errs.append(np.abs(y - ex).max() * 4 * math.pi * d)
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_cq_differentiation_is_bdf2():
    """K(s) = s: CQ weights are those of BDF2, (3/2 g_n - 2 g_{n-1} + g_{n-2}/2)/dt."""
    N, dt = 30, 0.05
    rng = np.random.default_rng(2)
    g = rng.normal(size=N + 1)
    y = cq.convolve(lambda s: s, g, N, dt).real
    gp = np.concatenate([[0.0, 0.0], g])
    ref = (1.5 * gp[2:] - 2 * gp[1:-1] + 0.5 * gp[:-2]) / dt
    assert np.abs(y - ref).max() < 1e-4 * np.abs(ref).max()
