"""The bounds behind the render kernels' culling, checked by brute force (CPU only).

The kernels skip work with three conservative tests derived from the truncated ellipsoid
{d : d^T Sigma^-1 d <= 9} (Sec. 3.3's 3-sigma truncation), written in the kernels' exponent
form q(d) = (log2 e / 2) d^T Sigma^-1 d <= T:
  * completing the square along x: q = S(dy, dz) + a (dx - c1 dy - c2 dz)^2 with
    S = Pyy dy^2 + P2yz dy dz + Pzz dz^2 (the per-row exponent of both kernels);
  * the box: |d_k| <= trunc sigma_k on the ellipsoid (the forward's footprint cull);
  * the section through a z-plane: y in k1 dz +- hw, x in (c1 k1 + c2) dz +- hw sqrt(Pyy/a +
    c1^2), hw^2 = (T - kappa dz^2) / Pyy, k1 = -P2yz / (2 Pyy), kappa = Pzz - P2yz^2 / (4 Pyy)
    (the adjoint's row mask and its plane skip).
Each is checked here against dense samples of the ellipsoid for random anisotropic,
rotated Gaussians: every sample lies inside the bound, and the bound is attained.
"""
import numpy as np

T_SIGMA = 3.0
HALF_LOG2E = 0.5 / np.log(2.0)
T = HALF_LOG2E * T_SIGMA ** 2


def _random_sigma(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    s = np.exp(rng.uniform(np.log(0.3), np.log(8.0), 3))
    return R @ np.diag(s * s) @ R.T


def _row_form(A):
    """The kernels' row parameters from the exponent matrix A (q = d^T A d)."""
    a = A[0, 0]
    c1, c2 = -A[0, 1] / a, -A[0, 2] / a
    pyy = A[1, 1] - A[0, 1] ** 2 / a
    p2yz = 2.0 * (A[1, 2] - A[0, 1] * A[0, 2] / a)
    pzz = A[2, 2] - A[0, 2] ** 2 / a
    return a, c1, c2, pyy, p2yz, pzz


def _ellipsoid_surface(sigma, n, rng):
    """Points d with q(d) = T exactly."""
    L = np.linalg.cholesky(sigma)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return (T_SIGMA * u) @ L.T


def test_completed_square_equals_quadratic_form():
    rng = np.random.default_rng(0)
    for _ in range(50):
        sigma = _random_sigma(rng)
        A = HALF_LOG2E * np.linalg.inv(sigma)
        a, c1, c2, pyy, p2yz, pzz = _row_form(A)
        d = rng.normal(scale=5.0, size=(200, 3))
        q = np.einsum("ni,ij,nj->n", d, A, d)
        S = pyy * d[:, 1] ** 2 + p2yz * d[:, 1] * d[:, 2] + pzz * d[:, 2] ** 2
        qr = S + a * (d[:, 0] - c1 * d[:, 1] - c2 * d[:, 2]) ** 2
        assert np.allclose(qr, q, rtol=1e-10, atol=1e-10)
        assert pyy > 0 and pzz - p2yz ** 2 / (4 * pyy) > 0  # the row shadow is positive definite


def test_box_half_extents_bound_the_ellipsoid():
    rng = np.random.default_rng(1)
    for _ in range(50):
        sigma = _random_sigma(rng)
        ext = T_SIGMA * np.sqrt(np.diag(sigma))
        d = _ellipsoid_surface(sigma, 20000, rng)
        m = np.abs(d).max(axis=0)
        assert np.all(m <= ext * (1 + 1e-12))
        assert np.all(m >= ext * (1 - 1e-2))  # attained (up to sampling)


def test_plane_sections_bound_y_and_x():
    rng = np.random.default_rng(2)
    for _ in range(30):
        sigma = _random_sigma(rng)
        A = HALF_LOG2E * np.linalg.inv(sigma)
        a, c1, c2, pyy, p2yz, pzz = _row_form(A)
        k1 = -p2yz / (2 * pyy)
        kappa = pzz - p2yz ** 2 / (4 * pyy)
        zmax = np.sqrt(T / kappa)
        assert np.isclose(zmax, T_SIGMA * np.sqrt(sigma[2, 2]), rtol=1e-9)
        for dz in rng.uniform(-0.999 * zmax, 0.999 * zmax, 6):
            hw = np.sqrt((T - kappa * dz * dz) / pyy)
            yc, xc = k1 * dz, (c1 * k1 + c2) * dz
            hwx = hw * np.sqrt(pyy / a + c1 * c1)
            # the section {(dx, dy): q(dx, dy, dz) <= T}, sampled on its boundary: for dy in
            # the y-interval, dx = c1 dy + c2 dz +- sqrt((T - S) / a)
            dy = yc + hw * np.cos(np.linspace(0, np.pi, 4001))
            S = pyy * dy ** 2 + p2yz * dy * dz + pzz * dz ** 2
            r = np.sqrt(np.maximum(T - S, 0.0) / a)
            dx = np.concatenate([c1 * dy + c2 * dz + r, c1 * dy + c2 * dz - r])
            assert np.all(np.abs(dy - yc) <= hw * (1 + 1e-12))
            assert np.all(np.abs(dx - xc) <= hwx * (1 + 1e-9))
            assert np.abs(dx - xc).max() >= hwx * (1 - 1e-4)  # attained
            # no point of the plane outside the y-interval reaches q <= T
            dy_out = yc + hw * (1 + 1e-6) * np.array([-1.0, 1.0])
            S_out = pyy * dy_out ** 2 + p2yz * dy_out * dz + pzz * dz ** 2
            assert np.all(S_out > T)
