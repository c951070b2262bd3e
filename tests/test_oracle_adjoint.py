"""Pins of oracle/adjoint.py (receiver energy through CQ and its adjoint
gradient) that do not rest on the oracle's own formulas: the half-set
transforms against the full transforms of oracle.cq (pinned in
test_oracle_hmatrix_cq.py), the defining inner-product identities of the two
adjoint transforms, and the adjoint gradient against central differences of
J: in the traction (J is quadratic, so the difference quotient is exact up to
rounding) and in the wave speeds (operators reassembled at perturbed
speeds, O(h^2))."""
import numpy as np
import pytest

import synthetic as syn
from oracle import adjoint, bem, cq


@pytest.mark.parametrize("N", [14, 15])
def test_half_set_transforms_agree_with_full(N):
    L = N + 1
    g = syn.normal(5, L * 6).reshape(L, 2, 3)
    full = cq.forward(g, N)
    assert np.allclose(adjoint.extend(full[:adjoint.half_count(N)], N), full, rtol=0, atol=1e-12 * np.abs(full).max())
    # round trip: the inverse scales by lam^-n (up to 1e5 at n = N), so
    # rounding of the forward sums reaches ~1e-10 relative
    back = adjoint.cq_inverse_half(adjoint.cq_forward_half(g, N), N)
    assert np.abs(back - g).max() < 1e-9 * np.abs(g).max()
    assert np.abs(back - cq.inverse(full, N).real).max() < 1e-9 * np.abs(g).max()
    # a conjugate-symmetric full set inverts to real samples
    assert np.abs(cq.inverse(full, N).imag).max() < 1e-9 * np.abs(g).max()


@pytest.mark.parametrize("N", [14, 15])
def test_adjoint_transform_identities(N):
    L, K = N + 1, adjoint.half_count(N)
    G = syn.normal(1, L * 4).reshape(L, 4)
    yh = syn.complex_normal(2, (K, 4))
    lhs = float((G * adjoint.cq_inverse_half(yh, N)).sum())
    rhs = float(np.real(np.vdot(adjoint.cq_inverse_half_adjoint(G, N), yh)))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)
    g = syn.normal(3, L * 4).reshape(L, 4)
    Gh = syn.complex_normal(4, (K, 4))
    lhs = float((adjoint.cq_forward_half_adjoint(Gh, N) * g).sum())
    rhs = float(np.real(np.vdot(Gh, adjoint.cq_forward_half(g, N))))
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1.0)


def _material(cp, cs, rho=7850.0):
    mu = rho * cs * cs
    return (rho, rho * cp * cp - 2.0 * mu, mu)


@pytest.fixture(scope="module")
def tiny_box():
    xyz, tri = syn.box(1.0, 1.0, 0.5, 0.5)
    N, dt = 9, 5e-5
    s = bem.freqs_bdf2(N, dt, adjoint.half_count(N))
    rho, lam, mu = syn.STEEL
    cp, cs = np.sqrt((lam + 2 * mu) / rho), np.sqrt(mu / rho)
    ops = adjoint.operators(xyz, tri, _material(cp, cs), s,
                            (bem.KERNEL_SL, bem.KERNEL_DL, bem.KERNEL_SL_DCP, bem.KERNEL_SL_DCS,
                             bem.KERNEL_DL_DCP, bem.KERNEL_DL_DCS))
    g = syn.box_traction(xyz, tri, N, dt, width=0.4, t0=2e-4, tw=1e-4)
    g = g + 1e5 * syn.normal(9, g.size).reshape(g.shape)     # every element loaded
    rec = syn.box_receivers(xyz, 4)
    return dict(xyz=xyz, tri=tri, N=N, dt=dt, s=s, cp=cp, cs=cs, ops=ops, g=g, rec=rec)


def test_gradient_in_traction_matches_central_differences(tiny_box):
    b = tiny_box
    o = b["ops"]
    J, dg, dc = adjoint.receiver_energy_grad(o["sl"], o["dl"], [], [], b["g"], b["rec"], b["N"], b["dt"])
    assert J > 0.0
    idx = [(0, 3, 2), (4, 10, 0), (b["N"], 31, 1), (2, 17, 2)]
    for n, e, a in idx:
        h = 1e3
        gp, gm = b["g"].copy(), b["g"].copy()
        gp[n, e, a] += h
        gm[n, e, a] -= h
        Jp = adjoint.receiver_energy(o["sl"], o["dl"], gp, b["rec"], b["N"], b["dt"])[0]
        Jm = adjoint.receiver_energy(o["sl"], o["dl"], gm, b["rec"], b["N"], b["dt"])[0]
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - dg[n, e, a]) <= 1e-7 * np.abs(dg).max(), (n, e, a, fd, dg[n, e, a])


def test_gradient_in_wave_speeds_matches_central_differences(tiny_box):
    b = tiny_box
    o = b["ops"]
    J, dg, dc = adjoint.receiver_energy_grad(o["sl"], o["dl"], [o["sl_dcp"], o["sl_dcs"]],
                                             [o["dl_dcp"], o["dl_dcs"]], b["g"], b["rec"], b["N"], b["dt"])
    for a, (cp, cs) in enumerate(((1, 0), (0, 1))):
        h = 1e-4 * (b["cp"] if a == 0 else b["cs"])
        Js = []
        for sg in (1, -1):
            m = _material(b["cp"] + sg * h * cp, b["cs"] + sg * h * cs)
            oo = adjoint.operators(b["xyz"], b["tri"], m, b["s"])
            Js.append(adjoint.receiver_energy(oo["sl"], oo["dl"], b["g"], b["rec"], b["N"], b["dt"])[0])
        fd = (Js[0] - Js[1]) / (2 * h)
        assert abs(fd - dc[a]) <= 1e-5 * abs(fd), (a, fd, dc[a])
