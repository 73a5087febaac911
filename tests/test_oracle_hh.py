"""Pins for the oracle's 4D hyperspherical harmonics (Eq. complex-HSH,
Eq. real-SH, App. A).  Each test checks the oracle against mathematics that
does not go through its own formulas: quadrature on S^3, the addition theorem,
library routines, harmonicity in R^4, closed forms, and counts the paper prints.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dir_from_angles(theta, phi):
    # reading A3: polar axis = z, azimuth in the xy-plane
    return np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi), math.cos(theta)])


def test_counts_match_paper_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "hh_counts.txt")) if l.strip() and not l.startswith("#")]
    for r in rows:
        if r[0] == "record":
            K, deg, total = int(r[1]), int(r[2]), int(r[3])
            assert 2 * K + 3 * oracle.lib().or_n_hh(deg) == total
        else:
            assert oracle.lib().or_n_hh(int(r[0])) == int(r[1])


def test_index_is_a_bijection():
    for deg in range(4):
        seen = []
        for n in range(deg + 1):
            for l in range(n + 1):
                for m in range(-l, l + 1):
                    seen.append(oracle.hh_index(n, l, m))
        assert sorted(seen) == list(range(oracle.lib().or_n_hh(deg)))


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_orthonormal_on_s3_by_quadrature(degree):
    """Gram matrix of the real harmonics under the S^3 measure
    sin^2(gamma) sin(theta) dgamma dtheta dphi is the identity."""
    ng, nt, nphi = 48, 24, 24
    xg, wg = np.polynomial.legendre.leggauss(ng)
    gam = (xg + 1.0) * math.pi / 2.0
    wg = wg * math.pi / 2.0 * np.sin(gam) ** 2
    xt, wt = np.polynomial.legendre.leggauss(nt)  # in cos(theta)
    phis = np.arange(nphi) * 2.0 * math.pi / nphi
    wphi = 2.0 * math.pi / nphi
    Nh = oracle.lib().or_n_hh(degree)
    G = np.zeros((Nh, Nh))
    for g, w1 in zip(gam, wg):
        for ct, w2 in zip(xt, wt):
            th = math.acos(ct)
            for ph in phis:
                h = oracle.hh_all(degree, g, _dir_from_angles(th, ph))
                G += (w1 * w2 * wphi) * np.outer(h, h)
    assert np.abs(G - np.eye(Nh)).max() < 1e-10


def test_printed_normalisation_is_not_orthonormal():
    """The paper prints A_{n,l} with (n-l+1)!; with it the squared norm would be
    (n-l+1) times ours, so the reading A1 is forced (reported in the design notes)."""
    for n in range(4):
        for l in range(n + 1):
            printed = (2.0 ** l * math.factorial(l)) * math.sqrt(
                2.0 * (n + 1) * math.factorial(n - l + 1) / (math.pi * math.factorial(n + l + 1)))
            ours = oracle.lib().or_hh_norm(n, l)
            assert abs((printed / ours) ** 2 - (n - l + 1)) < 1e-12


def test_addition_theorem():
    """sum_{l,m} H_nlm(x)^2 = (n+1)^2 / (2 pi^2) at every point of S^3."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        g = rng.uniform(0, math.pi)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        h = oracle.hh_all(3, g, d)
        for n in range(4):
            s = sum(h[oracle.hh_index(n, l, m)] ** 2 for l in range(n + 1) for m in range(-l, l + 1))
            assert abs(s - (n + 1) ** 2 / (2 * math.pi ** 2)) < 1e-12


def test_gegenbauer_and_legendre_against_scipy():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(1)
    for x in rng.uniform(-1, 1, 25):
        for k in range(6):
            for lam in (1.0, 2.0, 3.0, 4.0, 2.5):
                assert abs(oracle.gegenbauer(k, lam, x) - sp.eval_gegenbauer(k, lam, x)) < 1e-11
        for l in range(5):
            for m in range(l + 1):
                # scipy includes the Condon-Shortley phase (-1)^m, the oracle does not (reading A3)
                assert abs(oracle.legendre(l, m, x) - (-1) ** m * sp.lpmv(m, l, x)) < 1e-11


def test_real_sh_against_scipy_complex():
    """Y_lm = sqrt2 (-1)^m Re Y_l^m (m > 0), Y_l0 = Y_l^0, sqrt2 (-1)^|m| Im Y_l^|m| (m < 0),
    scipy's Y_l^m carrying the Condon-Shortley phase."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(2)
    for _ in range(50):
        th, ph = math.acos(rng.uniform(-1, 1)), rng.uniform(0, 2 * math.pi)
        d = _dir_from_angles(th, ph)
        for l in range(4):
            for m in range(-l, l + 1):
                Yc = complex(sp.sph_harm_y(l, abs(m), th, ph))
                if m == 0:
                    ref = Yc.real
                elif m > 0:
                    ref = math.sqrt(2) * (-1) ** m * Yc.real
                else:
                    ref = math.sqrt(2) * (-1) ** abs(m) * Yc.imag
                assert abs(oracle.sh_real(l, m, d) - ref) < 1e-12


def _F(x, n, l, m):
    """|x|^n H_nlm at the direction of x in R^4, with the paper's coordinates
    x1 = cos g, x2 = sin g cos th, x3 = sin g sin th cos ph, x4 = sin g sin th sin ph."""
    r = np.linalg.norm(x)
    g = math.acos(max(-1.0, min(1.0, x[0] / r)))
    v = np.array([x[2], x[3], x[1]])
    d = v / np.linalg.norm(v)
    return r ** n * oracle.hh_all(3, g, d)[oracle.hh_index(n, l, m)]


def test_harmonic_polynomials_in_r4():
    """r^n H_nlm is a harmonic homogeneous polynomial in R^4: its Laplacian vanishes.
    Pins the Gegenbauer parameter l+1, the sin^l factor and the pairing with Y_l."""
    rng = np.random.default_rng(3)
    h = 1e-3
    for _ in range(6):
        x = rng.standard_normal(4)
        x /= np.linalg.norm(x)
        for n in range(1, 4):
            for l in range(n + 1):
                for m in (-l, 0, l):
                    f0 = _F(x, n, l, m)
                    lap = 0.0
                    for a in range(4):
                        e = np.zeros(4)
                        e[a] = h
                        lap += (_F(x + e, n, l, m) - 2 * f0 + _F(x - e, n, l, m)) / h ** 2
                    # second derivatives are O(1); FD error is O(h^2)
                    assert abs(lap) < 1e-4, (n, l, m, lap)


def test_a_wrong_gegenbauer_parameter_breaks_harmonicity():
    """Control for the test above: with lambda = n + l (the appendix's printed form)
    the same construction is not harmonic, so that test can tell them apart."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(4)
    x /= np.linalg.norm(x)
    n, l, h = 3, 1, 1e-3

    def F(y):
        r = np.linalg.norm(y)
        c = y[0] / r
        s = math.sqrt(max(0.0, 1 - c * c))
        v = np.array([y[2], y[3], y[1]])
        d = v / np.linalg.norm(v)
        return r ** n * s ** l * oracle.gegenbauer(n - l, n + l, c) * oracle.sh_real(l, 0, d)

    lap = sum((F(x + h * e) - 2 * F(x) + F(x - h * e)) / h ** 2 for e in np.eye(4))
    assert abs(lap) > 1e-2


def test_closed_forms():
    # H_000 = Abar_00 C^1_0 Y_00 = sqrt(2/pi) / (2 sqrt(pi)) = 1 / (pi sqrt 2)
    rng = np.random.default_rng(5)
    for _ in range(10):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        assert abs(oracle.hh_all(2, rng.uniform(0, math.pi), d)[0] - 1.0 / (math.pi * math.sqrt(2))) < 1e-15
    # Y_00 = 1 / (2 sqrt pi);  Y_10 = sqrt(3/(4 pi)) z
    d = np.array([0.36, 0.48, 0.8])
    assert abs(oracle.sh_real(0, 0, d) - 0.5 / math.sqrt(math.pi)) < 1e-15
    assert abs(oracle.sh_real(1, 0, d) - math.sqrt(3 / (4 * math.pi)) * 0.8) < 1e-15
    assert abs(oracle.sh_real(1, 1, d) - math.sqrt(3 / (4 * math.pi)) * 0.36) < 1e-15
    assert abs(oracle.sh_real(1, -1, d) - math.sqrt(3 / (4 * math.pi)) * 0.48) < 1e-15


def test_dgamma_matches_finite_difference():
    rng = np.random.default_rng(6)
    for _ in range(20):
        g = rng.uniform(0.05, math.pi - 0.05)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        h = 1e-6
        fd = (oracle.hh_all(3, g + h, d) - oracle.hh_all(3, g - h, d)) / (2 * h)
        assert np.abs(oracle.hh_all_dgamma(3, g, d) - fd).max() < 1e-8
