"""The oracle's PCA over bands, pinned by closed forms and invariants."""
import math

import numpy as np

import oracle


def test_two_bands_closed_form():
    """Covariance [[a, c], [c, b]]: eigenvalues (a+b)/2 +- sqrt(((a-b)/2)^2 + c^2)."""
    rng = np.random.default_rng(0)
    u = rng.normal(0, 1, 4000)
    v = rng.normal(0, 1, 4000)
    x = np.stack([2 * u + 0.5 * v, u - v]).reshape(2, 1, 40, 100)
    mean, comps, var = oracle.pca_fit(x)
    xc = x.reshape(2, -1) - mean[:, None]
    a, b, c = (xc[0] ** 2).mean(), (xc[1] ** 2).mean(), (xc[0] * xc[1]).mean()
    r = math.sqrt(((a - b) / 2) ** 2 + c * c)
    assert math.isclose(var[0], (a + b) / 2 + r, rel_tol=1e-12)
    assert math.isclose(var[1], (a + b) / 2 - r, rel_tol=1e-12)
    # the first component solves (C - l1 I) v = 0
    C = np.array([[a, c], [c, b]])
    assert np.allclose(C @ comps[0], var[0] * comps[0], atol=1e-12)


def test_known_rotation_and_variances():
    """Sources with exactly diagonal sample covariance (9, 4, 1): mixed by a
    rotation R, PCA returns R's columns (signed by the rule) and 9, 4, 1."""
    n = 64
    h = np.array([[1 if bin(i & j).count("1") % 2 == 0 else -1 for j in range(n)] for i in range(n)], float)
    s = np.stack([3 * h[1], 2 * h[2], 1 * h[3]])  # zero-mean, orthogonal rows: covariance diag(9, 4, 1)
    th, ph = 0.7, -0.4
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(ph), -math.sin(ph)], [0, math.sin(ph), math.cos(ph)]])
    R = Rz @ Rx
    x = (R @ s + np.array([[5.0], [-2.0], [0.25]])).reshape(3, 1, 8, 8)
    mean, comps, var = oracle.pca_fit(x)
    assert np.allclose(mean, [5.0, -2.0, 0.25], atol=1e-13)
    assert np.allclose(var, [9, 4, 1], atol=1e-12)
    for k in range(3):
        col = R[:, k] * np.sign(R[np.argmax(np.abs(R[:, k])), k])
        assert np.allclose(comps[k], col, atol=1e-12)


def test_orthonormal_ordered_and_trace():
    rng = np.random.default_rng(1)
    A = rng.normal(0, 1, (6, 6))
    x = (A @ rng.normal(0, 1, (6, 3000))).reshape(6, 3, 20, 50)
    mean, comps, var = oracle.pca_fit(x)
    assert np.allclose(comps @ comps.T, np.eye(6), atol=1e-12)
    assert np.all(np.diff(var) <= 0)
    xc = x.reshape(6, -1) - mean[:, None]
    assert math.isclose(var.sum(), (xc ** 2).mean(axis=1).sum(), rel_tol=1e-12)
    for k in range(6):  # sign rule
        j = int(np.argmax(np.abs(comps[k])))
        assert comps[k, j] > 0


def test_project_inverse_roundtrip_and_moments():
    rng = np.random.default_rng(2)
    A = rng.normal(0, 1, (5, 5))
    x = (A @ rng.normal(0, 1, (5, 2400)) + 3).reshape(5, 4, 20, 30).astype(np.float32)
    mean, comps, var = oracle.pca_fit(x)
    z = oracle.pca_project(x, mean, comps, 5)
    back = oracle.pca_inverse(z, mean, comps)
    assert np.allclose(back, x, atol=1e-5)
    zz = z.reshape(5, -1).astype(np.float64)
    assert np.allclose(zz.mean(axis=1), 0, atol=1e-5)
    assert np.allclose((zz ** 2).mean(axis=1), var, rtol=1e-5)
    # dropping the last component costs exactly its variance (mean square error)
    z4 = oracle.pca_project(x, mean, comps, 4)
    err = oracle.pca_inverse(z4, mean, comps).astype(np.float64) - x
    assert math.isclose((err ** 2).sum(axis=0).mean(), var[4], rel_tol=1e-4)


def test_non_finite_pixels_are_excluded_from_the_fit():
    rng = np.random.default_rng(3)
    x = rng.normal(0, 1, (3, 2, 10, 10))
    y = x.copy()
    y[1, 0, 3, 4] = np.nan
    m1, c1, v1 = oracle.pca_fit(np.delete(x.reshape(3, -1), 34, axis=1).reshape(3, 1, 1, 199))
    m2, c2, v2 = oracle.pca_fit(y)
    assert np.allclose(m1, m2) and np.allclose(c1, c2) and np.allclose(v1, v2)
