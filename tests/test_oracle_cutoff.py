"""Oracle cutoffs: the Born-radius cutoff rgbmax (the HCT integral restricted
to the ball of radius rgbmax about atom i) and the pair cutoff `cut` of the
GB and Coulomb pair terms (truncation).  Pinned by 2-D quadrature of the
restricted volume integral, by agreement with the uncut closed form (a
different formula) when the ball holds all of sphere j, by finite
differences of the integral and of the energy, and by the additivity of the
truncated pair sum."""
import numpy as np
import pytest
from scipy import integrate

import synth


def hct_by_quadrature_cut(r, a, s, rc):
    """(1/4pi) * integral over the ball (x_j, s) of |y - x_i|^-4 restricted to
    a < |y - x_i| < rc, |x_i - x_j| = r; spherical coordinates about x_j."""
    def inner(u):
        if u == 0.0:
            return 2.0 / r ** 4 if a < r < rc else 0.0
        c_hi = min(1.0, (u * u + r * r - a * a) / (2.0 * u * r))     # |y - x_i| > a
        c_lo = max(-1.0, (u * u + r * r - rc * rc) / (2.0 * u * r))  # |y - x_i| < rc
        if c_hi <= c_lo:
            return 0.0
        val, _ = integrate.quad(lambda c: (u * u + r * r - 2 * u * r * c) ** -2, c_lo, c_hi,
                                epsabs=0, epsrel=1e-12, limit=200)
        return val

    pts = [p for p in (abs(r - a), r + a, r, abs(rc - r), rc + r) if 0 < p < s]
    val, _ = integrate.quad(lambda u: 0.5 * u * u * inner(u), 0.0, s, points=pts or None,
                            epsabs=0, epsrel=1e-11, limit=400)
    return val


@pytest.mark.parametrize("r,a,s,rc,regime", [
    (20.0, 1.5, 1.2, 20.5, "straddling the cutoff"),
    (20.0, 1.5, 1.2, 19.2, "mostly beyond"),
    (20.0, 1.5, 1.2, 18.7, "entirely beyond"),
    (4.0, 1.5, 1.2, 4.6, "disjoint, cut through sphere j"),
    (2.0, 1.5, 1.2, 2.8, "overlapping, cut"),
    (0.3, 0.8, 1.5, 1.0, "engulfed, cut inside the engulfed shells"),
    (0.3, 0.8, 1.5, 1.6, "engulfed, cut beyond"),
    (0.3, 0.8, 1.5, 0.7, "cut inside sphere i"),
])
def test_cut_integral_matches_quadrature(orc, r, a, s, rc, regime):
    ref = hct_by_quadrature_cut(r, a, s, rc)
    got = orc.hct_pair_cut(r, a, s, rc)
    assert abs(got - ref) <= 1e-9 * max(abs(ref), 1e-12) + 1e-15, (regime, got, ref)


@pytest.mark.parametrize("r,a,s", [(4.0, 1.5, 1.2), (2.0, 1.5, 1.2), (1.0, 1.1, 1.5),
                                   (0.3, 0.8, 1.5), (12.0, 1.71, 1.2), (0.2, 1.5, 1.0)])
def test_cut_beyond_sphere_equals_uncut_closed_form(orc, r, a, s):
    assert orc.hct_pair_cut(r, a, s, r + s + 0.5) == pytest.approx(orc.hct_pair(r, a, s), rel=1e-12, abs=1e-16)
    assert orc.hct_pair_cut(r, a, s, 0.0) == orc.hct_pair(r, a, s)


@pytest.mark.parametrize("r,a,s,rc", [(20.0, 1.5, 1.2, 20.5), (20.0, 1.5, 1.2, 19.5), (4.0, 1.5, 1.2, 4.6),
                                      (2.0, 1.5, 1.2, 2.8), (0.3, 0.8, 1.5, 1.0), (0.9, 1.3, 1.6, 1.9)])
def test_cut_derivative_fd(orc, r, a, s, rc):
    h = 1e-5 * max(1.0, r)          # relative step: the values are ~1e-6 at r = 20
    fd = (orc.hct_pair_cut(r + h, a, s, rc) - orc.hct_pair_cut(r - h, a, s, rc)) / (2 * h)
    assert orc.hct_pair_dr_cut(r, a, s, rc) == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_cut_integral_is_continuous_at_the_cutoff(orc):
    """As sphere j leaves the ball (r - s -> rc) the integral goes to zero."""
    a, s, rc = 1.5, 1.2, 20.0
    for eps in (1e-3, 1e-5):
        assert orc.hct_pair_cut(rc + s - eps, a, s, rc) < 1e-8
    assert orc.hct_pair_cut(rc + s + 1e-3, a, s, rc) == 0.0


@pytest.fixture(scope="module")
def mol():
    rep = synth.make_replica(300, 72, [])
    return (rep.xyz.astype(np.float64), rep.q.astype(np.float64), rep.rho.astype(np.float64),
            rep.screen.astype(np.float64))


def test_large_cutoffs_change_nothing(orc, mol):
    x, q, rho, scr = mol
    span = np.linalg.norm(x.max(0) - x.min(0)) + 5.0
    o0 = orc.energy_forces(x, q, rho, scr)
    o1 = orc.energy_forces(x, q, rho, scr, orc.default_params(rgbmax=span, cut=span))
    assert np.allclose(o1["R"], o0["R"], rtol=1e-12)
    assert np.allclose(o1["E"], o0["E"], rtol=1e-12)
    assert np.allclose(o1["F"], o0["F"], rtol=1e-9, atol=1e-10)


def cut_in_gap(x, near):
    """A cutoff near `near` in the middle of the widest gap between pair
    distances there: the truncated energy jumps where a pair crosses the
    cutoff, so finite differences (and numpy's own distances, which may round
    differently from the oracle's) need every pair well away from it."""
    d = np.linalg.norm(x[:, None] - x[None], axis=2)[np.triu_indices(len(x), 1)]
    d = np.sort(d[np.abs(d - near) < 0.2])
    k = int(np.argmax(np.diff(d)))
    assert d[k + 1] - d[k] > 1e-3
    return float(np.float32(0.5 * (d[k] + d[k + 1])))


def test_pair_cutoff_drops_exactly_the_far_pairs(orc, mol):
    """E(cut) = E(no cut) - sum over pairs with r > cut of the pair's GB and
    Coulomb terms at the same Born radii (each pair's terms from a two-atom
    evaluation minus the two self terms)."""
    x, q, rho, scr = mol
    R = orc.born_radii(x, rho, scr)["R"]
    cut = cut_in_gap(x, 9.0)
    E_all = orc.energy_fixed_radii(x, q, R).sum()
    E_cut = orc.energy_fixed_radii(x, q, R, orc.default_params(cut=cut)).sum()
    far = 0.0
    n = len(q)
    for i in range(n):
        for j in range(i + 1, n):
            if np.linalg.norm(x[i] - x[j]) > cut:
                pair = orc.energy_fixed_radii(x[[i, j]], q[[i, j]], R[[i, j]]).sum()
                self_ = (orc.energy_fixed_radii(x[[i]], q[[i]], R[[i]]).sum()
                         + orc.energy_fixed_radii(x[[j]], q[[j]], R[[j]]).sum())
                far += pair - self_
    assert E_cut == pytest.approx(E_all - far, rel=1e-11, abs=1e-9)


def test_pair_cutoff_boundary_is_the_exact_distance(orc):
    """Two ions on either side of the cutoff, within 1e-12 relative of it: on
    the inside the truncated energy equals the untruncated one, on the
    outside it equals the two isolated ions' Born energies (one-atom
    evaluations).  The decision is taken on the exact distance, however close
    the pair lies to the cutoff."""
    cut = 10.0
    q = np.array([0.5, -0.5])
    R = np.array([1.5, 1.7])
    iso = (orc.energy_fixed_radii(np.zeros((1, 3)), q[:1], R[:1]).sum()
           + orc.energy_fixed_radii(np.zeros((1, 3)), q[1:], R[1:]).sum())
    for dx, inside in ((cut * (1 - 1e-12), True), (cut, True), (cut * (1 + 1e-12), False),
                       (cut + 1e-7, False), (cut - 1e-7, True)):
        x = np.array([[0.0, 0.0, 0.0], [dx, 0.0, 0.0]])
        E = orc.energy_fixed_radii(x, q, R, orc.default_params(cut=cut))
        if inside:
            assert E.sum() == pytest.approx(orc.energy_fixed_radii(x, q, R).sum(), rel=1e-14), dx
            assert E[1] != 0.0
        else:
            assert E.sum() == pytest.approx(iso, rel=1e-14), dx
            assert E[1] == 0.0


def test_forces_fd_with_both_cutoffs(orc, mol):
    x, q, rho, scr = mol
    p = orc.default_params(rgbmax=8.0, cut=cut_in_gap(x, 10.0))
    o = orc.energy_forces(x, q, rho, scr, p)
    d = np.linalg.norm(x[:, None] - x[None], axis=2)
    rng = np.random.default_rng(4)
    h = 1e-5
    checked = 0
    for _ in range(40):
        i, k = int(rng.integers(len(q))), int(rng.integers(3))
        if np.any(np.abs(d[i] - p.cut) < 1e-3):     # the truncated energy jumps at r = cut
            continue
        xp, xm = x.copy(), x.copy()
        xp[i, k] += h
        xm[i, k] -= h
        fd = -(orc.energy(xp, q, rho, scr, p) - orc.energy(xm, q, rho, scr, p)) / (2 * h)
        assert o["F"][i, k] == pytest.approx(fd, abs=2e-6 * max(1.0, abs(fd)))
        checked += 1
    assert checked >= 20
