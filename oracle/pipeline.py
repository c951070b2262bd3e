"""End-to-end oracle of the multi-frequency operator: geometry and
frequencies -> cluster and block trees -> per-block dense tensors ->
3D-ACA + face ACA -> compressed apply (oracle, FP64, test infrastructure).

Sec. 2.4 (Eqs. (2.22)-(2.24)) defines the array of N_Q matrices; Sec. 3
compresses it blockwise (Algorithm 1 per block of the block cluster tree,
Sec. 3.1) and applies it (Eq. (3.15)).
"""
from __future__ import annotations

import numpy as np

from . import aca, bem, hmatrix


def col_kind(kernel):
    return "elements" if kernel in bem.SL_KINDS else "p1nodes"


def trees(op: bem.Operator, leaf: int, eta: float):
    geo = op.geo
    rp = hmatrix.support_boxes(geo, op.rows_kind)
    cp = hmatrix.support_boxes(geo, col_kind(op.kernel))
    rt = hmatrix.build_cluster_tree(*rp, leaf)
    ct = hmatrix.build_cluster_tree(*cp, leaf)
    return rt, ct, hmatrix.build_block_tree(rt, ct, eta)


def compress(op: bem.Operator, s, eps: float, eps_aca: float | None = None,
             leaf: int = 32, eta: float = 2.0, dense_tensor=None):
    """Compressed operator: list of aca.CompressedBlock.  ``dense_tensor``
    (n_rows, n_cols, K, 3, 3) may be passed to avoid recomputing entries."""
    eps_aca = eps / 100.0 if eps_aca is None else eps_aca
    _, _, blocks = trees(op, leaf, eta)
    out = []
    for b in blocks:
        rows, cols = b.rows.idx, b.cols.idx
        if dense_tensor is not None:
            C = dense_tensor[np.ix_(rows, cols)]
        else:
            C = op.block(rows, cols, s)
        out.append(aca.compress_block(C, rows, cols, b.far, eps, eps_aca))
    return out


def stats(blocks, K: int):
    """Compression statistics (Sec. 4.1): stored complex numbers versus the
    dense tensor, ranks per block."""
    stored = 0
    dense = 0
    ranks = []
    for b in blocks:
        m, n = len(b.rows), len(b.cols)
        dense += 9 * m * n * K
        if b.kind == "dense":
            stored += 9 * m * n * K
            ranks.append(K)
        elif b.kind == "rank0":
            ranks.append(0)
        else:
            ranks.append(len(b.faces))
            stored += 9 * K * len(b.fibres)
            for f in b.faces:
                if isinstance(f, aca.LowRank):
                    stored += f.U.size + f.V.size
                else:
                    stored += 9 * m * n
    return {"compression_rate": stored / dense, "ranks": ranks}
