"""3D-ACA (Algorithm 1), matrix-valued ACA with QR/SVD recompression and the
compressed multi-frequency apply (oracle, FP64).

Block tensors are arrays C[i, j, k] of 3 x 3 complex matrices, shape
(m, n, K, 3, 3); the face-fibre product is (H (x) f)[i, j, k] = H[i, j] f[k]
(3 x 3 product, face on the left, because the fibre is normalised by the
inverse of the pivot block from the left, Sec. 3, Algorithm 1).

Readings of Algorithm 1 and Eqs. (3.2)-(3.8):
* k_1 = 0 is the first frequency of the list (0-based).
* The loop is a do-while; the pair that fails the test
  ||H_d||_F ||f_d|| > eps ||C^(d)||_F is discarded (r = d - 1).
* ||f_d|| is the Frobenius norm over all k of the 3 x 3 fibre entries;
  ||C^(d)||_F^2 follows the recursion of Eq. (3.3) in matrix form,
  sum_{p,q} Re tr(M_pq N_qp), M_pq = sum_ij H_p[i,j]^H H_q[i,j],
  N_qp = sum_k f_q[k] f_p[k]^H.
* Pivot (Eq. (3.7)): (i_d, j_d) = argmax sigma_3(H_d[i, j]), ties to the
  smallest row-major index; k_{d+1} = argmax_k sigma_3(f_d[k]) (Eq. (3.8))
  over the frequencies not used yet (f_d[k_d] = I by construction, so the
  unrestricted argmax would return k_d again whenever the other fibre
  entries are smaller than the pivot, as they are at k_1 = 0, the frequency
  of least damping); ties to the smallest k.
* No regular pivot (Sec. 3, after Eq. (3.8)): max sigma_3 <= PIV_TOL times
  the Frobenius norm of the face (or fibre) -> the block is stored dense.
  A face residual that vanishes (||H_d||_F <= TINY ||C^(d-1)||_F) ends the
  loop (r = d - 1); an all-zero block has rank 0.  Reaching r = K stores
  the block dense (the dense limit).

Matrix-valued ACA of a face (Sec. 3.1, Eq. (3.12), after Rjasanow-Weggler
and Haider et al.): partial pivoting on 3 x 3 blocks; start row = first row
of the block; column pivot = argmax sigma_3 in the residual row; next row =
argmax sigma_3 in the new column over rows not yet used; stop when
||u||_F ||v||_F <= eps_aca ||S||_F; then QR of both factors, SVD of
R_U R_V^H, truncation to the smallest rank whose discarded singular values
have Frobenius norm <= eps_aca times the total.  A face without a regular
pivot row is kept dense.
Pins (tests/test_oracle_aca.py): interpolation property at the pivots,
exact recovery of a synthetic separable tensor, recursion = explicit norm,
error <= eps against the dense tensor.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

PIV_TOL = 1e-13
TINY = 1e-14


def sigma3(blocks: np.ndarray) -> np.ndarray:
    """Smallest singular value of every 3 x 3 block (..., 3, 3)."""
    return np.linalg.svd(blocks, compute_uv=False)[..., -1]


def face_fibre(H: np.ndarray, f: np.ndarray) -> np.ndarray:
    """(H (x) f)[i, j, k] = H[i, j] @ f[k] -> (m, n, K, 3, 3)."""
    return np.einsum("ijab,kbc->ijkac", H, f)


@dataclass
class Aca3d:
    kind: str                          # 'aca' | 'dense' | 'rank0'
    ks: list = field(default_factory=list)
    pivots: list = field(default_factory=list)
    faces: list = field(default_factory=list)     # (m, n, 3, 3) each
    fibres: list = field(default_factory=list)    # (K, 3, 3) each
    norm2: float = 0.0

    @property
    def rank(self):
        return len(self.faces)

    def tensor(self, shape=None):
        if self.kind == "rank0":
            return np.zeros(shape, dtype=np.complex128)
        out = 0.0
        for H, f in zip(self.faces, self.fibres):
            out = out + face_fibre(H, f)
        return out


def norm2_recursive(faces, fibres) -> float:
    """||sum_d H_d (x) f_d||_F^2 from the 3 x 3 Gram matrices (Eq. (3.3))."""
    tot = 0.0
    for p in range(len(faces)):
        for q in range(len(faces)):
            M = np.einsum("ijba,ijbc->ac", faces[p].conj(), faces[q])
            N = np.einsum("kab,kcb->ac", fibres[q], fibres[p].conj())
            tot += np.trace(M @ N).real
    return tot


def aca3d(C: np.ndarray, eps: float, k1: int = 0) -> Aca3d:
    """Algorithm 1 on the dense block tensor C (m, n, K, 3, 3)."""
    m, n, K = C.shape[:3]
    res = Aca3d(kind="aca")
    k = k1
    while True:
        d = len(res.faces) + 1
        H = C[:, :, k].copy()
        for Hp, fp in zip(res.faces, res.fibres):
            H -= np.einsum("ijab,bc->ijac", Hp, fp[k])
        nH = np.linalg.norm(H)
        if d == 1 and nH == 0.0:
            return Aca3d(kind="rank0")
        if d > 1 and nH <= TINY * np.sqrt(res.norm2):
            return res
        s3 = sigma3(H)
        flat = int(np.argmax(s3.ravel()))
        if s3.ravel()[flat] <= PIV_TOL * nH:
            return Aca3d(kind="dense")
        i_d, j_d = divmod(flat, n)
        P = H[i_d, j_d]
        fib = C[i_d, j_d].copy()                               # (K, 3, 3)
        for Hp, fp in zip(res.faces, res.fibres):
            fib -= np.einsum("ab,kbc->kac", Hp[i_d, j_d], fp)
        f = np.linalg.solve(P[None], fib)                      # P^{-1} fib[k]
        faces = res.faces + [H]
        fibres = res.fibres + [f]
        norm2 = norm2_recursive(faces, fibres)
        if np.linalg.norm(H) * np.linalg.norm(f) <= eps * np.sqrt(norm2):
            return res                                         # r = d - 1
        res.faces, res.fibres, res.norm2 = faces, fibres, norm2
        res.ks.append(k)
        res.pivots.append((i_d, j_d))
        if d == K:
            return Aca3d(kind="dense")
        s3f = sigma3(f)
        s3f[res.ks] = -1.0
        k = int(np.argmax(s3f))
        if s3f[k] <= PIV_TOL * np.linalg.norm(f):
            return Aca3d(kind="dense")


# --------------------------------------------------------------------------
# matrix-valued ACA of one face + QR/SVD recompression
# --------------------------------------------------------------------------

@dataclass
class LowRank:
    U: np.ndarray          # (3m, rho)
    V: np.ndarray          # (3n, rho), face ~= U V^H

    def matrix(self):
        return self.U @ self.V.conj().T


def aca_matrix(H: np.ndarray, eps_aca: float):
    """Matrix-valued partial-pivot ACA of a face H (m, n, 3, 3).  Returns a
    LowRank in the 3m x 3n matrix layout, or None (keep dense)."""
    m, n = H.shape[:2]
    us, vs = [], []          # u_t (m, 3, 3), v_t (n, 3, 3)
    used = np.zeros(m, dtype=bool)
    i = 0
    norm2 = 0.0
    for _ in range(min(m, n)):
        row = H[i].copy()
        for u, v in zip(us, vs):
            row -= np.einsum("ab,jbc->jac", u[i], v)
        used[i] = True
        s3 = sigma3(row)
        j = int(np.argmax(s3))
        nrow = np.linalg.norm(row)
        if nrow == 0.0 and not us:
            break
        if s3[j] <= PIV_TOL * max(nrow, 1e-300):
            if nrow <= TINY * np.sqrt(max(norm2, 0.0)):
                break
            return None
        col = H[:, j].copy()
        for u, v in zip(us, vs):
            col -= np.einsum("iab,bc->iac", u, v[j])
        Pinv = np.linalg.inv(row[j])
        u = np.einsum("iab,bc->iac", col, Pinv)
        v = row
        # recursive ||S||_F^2 with the new pair
        cross = 0.0
        for up, vp in zip(us, vs):
            M = np.einsum("iba,ibc->ac", up.conj(), u)
            N = np.einsum("jab,jcb->ac", v, vp.conj())
            cross += np.trace(M @ N).real
        M = np.einsum("iba,ibc->ac", u.conj(), u)
        N = np.einsum("jab,jcb->ac", v, v.conj())
        norm2 = norm2 + 2.0 * cross + np.trace(M @ N).real
        us.append(u)
        vs.append(v)
        if np.linalg.norm(u) * np.linalg.norm(v) <= eps_aca * np.sqrt(max(norm2, 0.0)):
            break
        cand = sigma3(u)
        cand[used] = -1.0
        if (cand < 0).all():
            break
        i = int(np.argmax(cand))
    if not us:
        return LowRank(np.zeros((3 * m, 0), complex), np.zeros((3 * n, 0), complex))
    # H ~= sum_t u_t[i] v_t[j]: U = [u_t stacked] (3m x 3r), V^H = [v_t] (3r x 3n)
    U = np.concatenate([u.reshape(3 * m, 3) for u in us], axis=1)
    VH = np.concatenate([v.transpose(1, 0, 2).reshape(3, 3 * n) for v in vs], axis=0)
    return recompress(U, VH.conj().T, eps_aca)


def recompress(U: np.ndarray, V: np.ndarray, eps_aca: float) -> LowRank:
    """QR of U and V, SVD of R_U R_V^H, Frobenius-relative truncation
    (Eq. (3.12))."""
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    W, sig, ZH = np.linalg.svd(Ru @ Rv.conj().T)
    tot = np.sqrt((sig ** 2).sum())
    keep = len(sig)
    tail = 0.0
    while keep > 0:
        t = np.sqrt(tail + sig[keep - 1] ** 2)
        if t > eps_aca * tot:
            break
        tail += sig[keep - 1] ** 2
        keep -= 1
    return LowRank(Qu @ (W[:, :keep] * sig[:keep]), Qv @ ZH[:keep].conj().T)


# --------------------------------------------------------------------------
# compressed operator over a block partition, and its apply
# --------------------------------------------------------------------------

@dataclass
class CompressedBlock:
    rows: np.ndarray
    cols: np.ndarray
    far: bool
    kind: str                       # 'aca' | 'dense' | 'rank0'
    faces: list                     # dense (m, n, 3, 3) or LowRank
    fibres: list                    # (K, 3, 3)
    ks: list
    dense: np.ndarray | None = None  # (m, n, K, 3, 3) when kind == 'dense'


def compress_block(C: np.ndarray, rows, cols, far: bool, eps: float, eps_aca: float):
    r = aca3d(C, eps)
    faces = []
    if r.kind == "aca":
        for H in r.faces:
            lr = aca_matrix(H, eps_aca) if far else None
            faces.append(H if lr is None else lr)
    return CompressedBlock(np.asarray(rows), np.asarray(cols), far, r.kind, faces,
                           r.fibres, r.ks, C.copy() if r.kind == "dense" else None)


def face_dense(face, m, n):
    if isinstance(face, LowRank):
        M = face.matrix()
        return M.reshape(m, 3, n, 3).transpose(0, 2, 1, 3)
    return face


def block_tensor(b: CompressedBlock, K: int) -> np.ndarray:
    m, n = len(b.rows), len(b.cols)
    if b.kind == "dense":
        return b.dense
    out = np.zeros((m, n, K, 3, 3), dtype=np.complex128)
    for face, f in zip(b.faces, b.fibres):
        out += face_fibre(face_dense(face, m, n), f)
    return out


def apply_batched(blocks, X: np.ndarray, n_rows: int) -> np.ndarray:
    """Y[:, k] = C_k X[:, k] for all k; X (n_cols, 3, K) -> Y (n_rows, 3, K)."""
    K = X.shape[2]
    Y = np.zeros((n_rows, 3, K), dtype=np.complex128)
    for b in blocks:
        T = block_tensor(b, K)                                  # (m, n, K, 3, 3)
        Y[b.rows] += np.einsum("ijkab,jbk->iak", T, X[b.cols])
    return Y


def apply_contracted(blocks, W: np.ndarray, n_rows: int) -> np.ndarray:
    """y = sum_k C_k W[:, k] (Eq. (3.15)); W (n_cols, 3, K) -> (n_rows, 3)."""
    return apply_batched(blocks, W, n_rows).sum(axis=2)


def apply_dense(C: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Y[:, :, k] = C[:, :, k] X[:, :, k]: C (M, N, K, 3, 3), X (N, 3, K)."""
    return np.einsum("ijkab,jbk->iak", C, X)


def apply_adjoint_dense(C: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Conjugate-transpose apply, X[:, :, k] = C[:, :, k]^H Y[:, :, k]:
    C (M, N, K, 3, 3), Y (M, 3, K) -> X (N, 3, K).  The 3M x 3N matrix of
    frequency k has block (i, j) = C[i, j, k]; its conjugate transpose has
    block (j, i) = C[i, j, k]^H."""
    return np.einsum("ijkab,iak->jbk", C.conj(), Y)


def receiver_energy(C: np.ndarray, X: np.ndarray, w: np.ndarray) -> float:
    """J = sum_k sum_i w_i |(C_k X_k)[i]|^2 (a receiver response): C (M, N,
    K, 3, 3), X (N, 3, K), w (M,) receiver weights."""
    Y = apply_dense(C, X)
    return float((w[:, None, None] * np.abs(Y) ** 2).sum())


def receiver_energy_speed_gradient(C: np.ndarray, dC: np.ndarray, X: np.ndarray, w: np.ndarray) -> float:
    """dJ/dc for one wave speed c, with dC = dC/dc (same layout as C):
    dJ/dc = 2 Re sum_k sum_i w_i conj(Y_k[i]) . (dC_k X_k)[i], Y = C X (the
    adjoint field of J is 2 w Y)."""
    Y = apply_dense(C, X)
    dY = apply_dense(dC, X)
    return float(2.0 * np.real((w[:, None, None] * np.conj(Y) * dY).sum()))
