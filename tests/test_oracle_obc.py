"""Pins of the OBC rescaling in the oracle across its whole range of psi.

The OBC model of Onufriev, Bashford and Case (Proteins 55, 383 (2004)) is the
GB model of the paper's MD (Sec. III.D, "igb=2").  It turns the HCT
descreening sum I of atom i into an effective Born radius through
    1/R = 1/a - tanh(Phi(psi)) / rho,   Phi = alpha psi - beta psi^2 + gamma psi^3,
with psi = a I and a = rho - offset.  The other oracle pins reach this map
only at its ends: psi -> 0 and tanh saturating.  A slip in a coefficient or
a sign of Phi would pass them.  These tests read the map off the oracle's
radii and compare it with facts derived by hand:

* Taylor coefficients at small psi.  With t(psi) = rho (1/a - 1/R) =
  tanh(Phi(psi)) and tanh x = x - x^3/3 + O(x^5),
      t = alpha psi - beta psi^2 + (gamma - alpha^3/3) psi^3
          + alpha^2 beta psi^4 + O(psi^5).
  A least-squares fit of t against psi gives the first four coefficients.
* One term at a time, for psi up to about 3.  With two of alpha, beta and
  gamma set to zero, numpy's arctanh of t is a single monomial of psi.
* dR/dpsi, the derivative the force chain rule uses, against central
  differences of R along the same geometry.

Geometry: atom 0 at the centre of 12 atoms on the vertices of an icosahedron
of radius r.  Each vertex atom descreens atom 0 by the same HCT integral
H(r; a_0, s) (pinned by quadrature elsewhere), so psi_0 = 12 a_0 H(r; a_0, s).
Moving r from 30 A down to 1.6 A sweeps psi_0 from about 1e-4 to about 3.
Only atom 0 is read.
"""
import numpy as np
import pytest

RHO0, SCREEN, RHO_J = 1.5, 0.9, 3.0


def _shell(r):
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s2 * g, 0.0, s1)]
    v = np.array(v)
    v *= r / np.linalg.norm(v[0])
    return np.vstack([np.zeros(3), v])


def _atom0(orc, r, **kw):
    """(psi_0, R_0, dR_0/dpsi_0) with the icosahedron at radius r."""
    x = _shell(r)
    rho = np.array([RHO0] + [RHO_J] * 12)
    scr = np.full(13, SCREEN)
    p = orc.default_params(**kw)
    o = orc.born_radii(x, rho, scr, p)
    a0 = RHO0 - p.offset
    # psi_0 is 12 times one pinned pair integral
    s = SCREEN * (RHO_J - p.offset)
    assert o["psi"][0] == pytest.approx(12.0 * a0 * orc.hct_pair(r, a0, s), rel=1e-13)
    return o["psi"][0], o["R"][0], o["dRdpsi"][0]


def _t(orc, R, **kw):
    p = orc.default_params(**kw)
    a0 = RHO0 - p.offset
    return RHO0 * (1.0 / a0 - 1.0 / R)


@pytest.mark.parametrize("alpha,beta,gamma", [
    (1.0, 0.8, 4.85),           # the workloads' set (OBC-II)
    (0.8, 0.0, 2.909125),       # OBC-I
    (1.0, 0.0, 0.0), (1.0, 1.7, 0.0), (1.0, -0.9, 0.0), (0.6, 0.8, 0.0), (1.0, 0.8, 1.5),
])
def test_taylor_coefficients_at_small_psi(orc, alpha, beta, gamma):
    kw = dict(alpha=alpha, beta=beta, gamma=gamma)
    rs = np.linspace(9.0, 30.0, 60)
    pts = [_atom0(orc, r, **kw) for r in rs]
    psi = np.array([p[0] for p in pts])
    t = np.array([_t(orc, p[1], **kw) for p in pts])
    assert 1e-4 < psi.min() and psi.max() < 0.03
    # t / psi = c1 + c2 psi + c3 psi^2 + c4 psi^3 + ..., fitted in u = psi / max
    u = psi / psi.max()
    V = np.vander(u, 7, increasing=True)
    c, *_ = np.linalg.lstsq(V, t / psi, rcond=None)
    c = c / psi.max() ** np.arange(7)
    assert c[0] == pytest.approx(alpha, abs=1e-9)
    assert c[1] == pytest.approx(-beta, abs=1e-6)
    assert c[2] == pytest.approx(gamma - alpha ** 3 / 3.0, abs=1e-3)
    assert c[3] == pytest.approx(alpha ** 2 * beta, abs=0.2)


@pytest.mark.parametrize("term", ["alpha", "beta", "gamma"])
@pytest.mark.parametrize("coef", [0.8, 1.0, 4.85])
def test_single_terms_across_the_range(orc, term, coef):
    kw = dict(alpha=0.0, beta=0.0, gamma=0.0)
    kw[term] = coef
    power, sign = {"alpha": (1, 1.0), "beta": (2, -1.0), "gamma": (3, 1.0)}[term]
    seen = []
    for r in np.linspace(1.6, 12.0, 80):
        psi, R, _ = _atom0(orc, r, **kw)
        t = _t(orc, R, **kw)
        if abs(t) > 1.0 - 1e-6:           # tanh saturated: arctanh is ill-conditioned
            continue
        want = sign * coef * psi ** power
        assert np.arctanh(t) == pytest.approx(want, rel=1e-9, abs=1e-14), (r, psi)
        seen.append(psi)
    assert min(seen) < 0.01 and max(seen) > 1.0


@pytest.mark.parametrize("alpha,beta,gamma", [(1.0, 0.8, 4.85), (0.8, 0.0, 2.909125), (1.0, -0.9, 0.3)])
def test_dR_dpsi_against_central_differences(orc, alpha, beta, gamma):
    kw = dict(alpha=alpha, beta=beta, gamma=gamma)
    checked = 0
    for r in np.linspace(2.0, 14.0, 25):
        h = 1e-5 * r
        pp, Rp, _ = _atom0(orc, r + h, **kw)
        pm, Rm, _ = _atom0(orc, r - h, **kw)
        psi, R, d = _atom0(orc, r, **kw)
        if abs(pp - pm) < 1e-9 * psi:
            continue
        fd = (Rp - Rm) / (pp - pm)
        assert d == pytest.approx(fd, rel=2e-6, abs=1e-9), (r, psi)
        checked += 1
    assert checked >= 20
