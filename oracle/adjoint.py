"""Receiver energy of a traction-driven Neumann problem through convolution
quadrature, and its gradient by the adjoint method (oracle, FP64, test
infrastructure: only tests, the smoke check and the benchmark's CPU leg use
it).

Forward problem.  The paper's Neumann rows (Sec. 2.3, Eq. (2.12)) in the
Laplace domain read (C + K)(s) u^(s) = V(s) t^(s); uniform-step convolution
quadrature (Sec. 2.4, constant steps: the scaled DFT of oracle.cq) maps the
time samples to the L = N + 1 frequencies s_k and back.  For real data the
frequencies come in conjugate pairs (s_{L-k} = conj s_k, Sec. 4.1) and so do
the transforms, so only k = 0 .. K - 1, K = floor(L / 2) + 1, are solved:

    g^_k = forward CQ transform of the traction samples g_n,  k < K
    A_k u^_k = V_k g^_k,  A = C + K (node rows), V single layer (node rows)
    u_n  = inverse CQ transform of the conjugate-extended set (real)
    J    = dt sum_n sum_{r in receivers} |u_n[r]|^2

Gradient (the functional's derivatives with respect to the real traction
samples and to the wave speeds c_p, c_s at fixed density).  With the complex
gradient convention dJ = Re sum conj(G^) du^ (G^ = dJ/dRe + i dJ/dIm):

    G_n     = 2 dt u_n at the receivers, 0 elsewhere
    G^_k    = adjoint of the half-set inverse transform applied to G
    W_k     = A_k^-H G^_k                         (adjoint solve)
    dJ/dg   = adjoint of the half-set forward transform applied to V_k^H W_k
    dJ/dc_a = Re sum_k W_k^H (dV_k/dc_a g^_k - dA_k/dc_a u^_k)

The two adjoint transforms are the adjoints of real-linear maps (real time
samples, complex frequency values) and are written here from their matrices.
Pins (tests/test_oracle_adjoint.py): the half-set transforms against the
full oracle.cq transforms, the defining inner-product identities of both
adjoint transforms, and the gradient against central differences of J in
the traction (J is quadratic: exact up to rounding) and in the wave speeds.
"""
from __future__ import annotations

import numpy as np

from . import bem, cq


def half_count(N: int) -> int:
    """K = floor(L / 2) + 1 frequencies of the half set, L = N + 1."""
    return (N + 1) // 2 + 1


def _phase(N: int):
    L = N + 1
    lam = cq.lam_c(N)
    n = np.arange(L)
    K = half_count(N)
    k = np.arange(K)
    # exp(2 pi i n k / L) with the integer product reduced mod L
    E = np.exp(2j * np.pi * (np.outer(n, k) % L) / L)
    # multiplicity of frequency k in the full set: 1 for k = 0 and (L even)
    # k = L / 2, else 2 (k and its conjugate partner L - k)
    c = np.full(K, 2.0)
    c[0] = 1.0
    if L % 2 == 0:
        c[L // 2] = 1.0
    return L, lam, n, E, c


def cq_forward_half(g: np.ndarray, N: int) -> np.ndarray:
    """g (L, ...) real samples -> g^ (K, ...): the first K rows of the full
    forward transform."""
    return cq.forward(g, N)[:half_count(N)]


def extend(yh: np.ndarray, N: int) -> np.ndarray:
    """Half set (K, ...) -> full set (L, ...) by y^_{L-k} = conj(y^_k)."""
    L = N + 1
    K = half_count(N)
    full = np.empty((L,) + yh.shape[1:], dtype=complex)
    full[:K] = yh
    for k in range(K, L):
        full[k] = np.conj(yh[L - k])
    return full


def cq_inverse_half(yh: np.ndarray, N: int) -> np.ndarray:
    """Half set (K, ...) -> real samples (L, ...): the full inverse
    transform of the conjugate extension (imaginary part zero up to
    rounding, dropped)."""
    return cq.inverse(extend(yh, N), N).real


def cq_inverse_half_adjoint(G: np.ndarray, N: int) -> np.ndarray:
    """Adjoint of cq_inverse_half as a real-linear map: for real G (L, ...)
    the complex G^ (K, ...) with sum_n G_n u_n = Re sum_k conj(G^_k) y^_k
    for u = cq_inverse_half(y^).  u_n = sum_k Re(a_nk y^_k) with
    a_nk = c_k lam^-n exp(2 pi i n k / L) / L, hence G^_k = sum_n conj(a_nk) G_n."""
    L, lam, n, E, c = _phase(N)
    A = c[None, :] * (lam ** (-n.astype(float)))[:, None] * E / L      # a_nk
    return np.tensordot(np.conj(A).T, G, axes=(1, 0))


def cq_forward_half_adjoint(Gh: np.ndarray, N: int) -> np.ndarray:
    """Adjoint of cq_forward_half restricted to real samples: the real
    dg (L, ...) with sum_n dg_n g_n = Re sum_k conj(Gh_k) g^_k.
    g^_k = sum_n b_kn g_n, b_kn = lam^n exp(-2 pi i n k / L), hence
    dg_n = Re sum_k conj(b_kn) Gh_k."""
    L, lam, n, E, c = _phase(N)
    B = (lam ** n.astype(float))[:, None] * np.conj(E)                 # b_kn as [n, k]
    return np.real(np.tensordot(np.conj(B), Gh, axes=(1, 0)))


def operators(xyz, tri, material, s, kernels=(bem.KERNEL_SL, bem.KERNEL_DL)):
    """Dense node-row matrices (3 n_nodes x 3 n_cols) of the given kernels at
    every frequency of s: {kernel: [M_k]}."""
    out = {}
    for kern in kernels:
        C = bem.Operator(xyz, tri, material, bem.ROWS_NODES, kern).dense(s)    # (m, n, K, 3, 3)
        out[kern] = [bem.to_matrix(C[:, :, k]) for k in range(len(s))]
    return out


def receiver_energy(V, A, g: np.ndarray, rec, N: int, dt: float):
    """J and the intermediate states (g^, u^, u): V, A lists of the K dense
    matrices; g (L, n_tris, 3) real; rec receiver node indices."""
    gh = cq_forward_half(g, N)
    K = len(gh)
    uh = np.stack([np.linalg.solve(A[k], V[k] @ gh[k].reshape(-1)) for k in range(K)])
    uh = uh.reshape(K, -1, 3)
    u = cq_inverse_half(uh, N)
    J = dt * float((u[:, rec, :] ** 2).sum())
    return J, gh, uh, u


def receiver_energy_grad(V, A, dV, dA, g: np.ndarray, rec, N: int, dt: float):
    """(J, dJ/dg (L, n_tris, 3), [dJ/dc_a for the pairs (dV_a, dA_a)]) by the
    adjoint method; dV, dA lists (one per wave speed) of lists of K dense
    derivative matrices."""
    J, gh, uh, u = receiver_energy(V, A, g, rec, N, dt)
    K = len(gh)
    G = np.zeros_like(u)
    G[:, rec, :] = 2.0 * dt * u[:, rec, :]
    Gh = cq_inverse_half_adjoint(G, N)
    W = np.stack([np.linalg.solve(A[k].conj().T, Gh[k].reshape(-1)) for k in range(K)])
    Gg = np.stack([V[k].conj().T @ W[k] for k in range(K)]).reshape(gh.shape)
    dg = cq_forward_half_adjoint(Gg, N)
    dc = []
    for dVa, dAa in zip(dV, dA):
        tot = 0.0 + 0.0j
        for k in range(K):
            tot += np.vdot(W[k], dVa[k] @ gh[k].reshape(-1) - dAa[k] @ uh[k].reshape(-1))
        dc.append(float(tot.real))
    return J, dg, dc
