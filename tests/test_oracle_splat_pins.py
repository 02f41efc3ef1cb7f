"""Pins of the oracle's particle renderer (App. D.2: spheres splatted into a depth buffer, a bilateral
filter scaled by camera distance, normals and lighting from the smoothed depth).

The splat is checked against exact ray-sphere geometry, the filter against fields it must keep
(constants, linear ramps, edges much deeper than its range sigma) and against the width it must have
at a given depth, the normals against planes whose depth comes from ray-plane intersection, and the
shading against Lambert's closed form."""
import math

import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(777)


def _cam(W=96, H=80, f=90.0, rot=None, eye=(0.0, 0.0, 0.0)):
    return oracle.Camera(W, H, f, f * 1.1, W / 2 + 0.3, H / 2 - 0.2, eye, np.eye(3) if rot is None else rot)


def _ray(cam, i, j):
    return np.array([(i + 0.5 - cam.cx) / cam.fx, (j + 0.5 - cam.cy) / cam.fy, 1.0])


def test_splat_of_one_sphere_follows_ray_geometry():
    cam = _cam()
    r = 0.06
    c = np.array([0.05, -0.03, 1.4])
    rp = oracle.RenderParams(r, 0.01, 0.01, 3)
    depth, amb, drawn = oracle.splat_depth(cam, rp, c.reshape(3, 1))
    assert drawn == 1
    checked = 0
    for j in range(cam.height):
        for i in range(cam.width):
            d = _ray(cam, i, j)
            # ray t d (z = t) against the sphere |t d - c| = r: t^2 |d|^2 - 2 t d.c + |c|^2 - r^2 = 0
            A, B, C = d @ d, -2 * d @ c, c @ c - r * r
            disc = B * B - 4 * A * C
            if abs(disc) < 2e-3 * B * B or amb[j, i]:
                continue  # near the silhouette: the sprite disk and the true outline differ there
            checked += 1
            if disc < 0:
                assert not np.isfinite(depth[j, i])
                continue
            t = (-B - math.sqrt(disc)) / (2 * A)
            assert np.isfinite(depth[j, i])
            # the sprite is the sphere seen orthographically: exact at the centre, off by O(r (r/z)) elsewhere
            assert abs(depth[j, i] - t) < 2.0 * r * r / c[2]
    assert checked > 100
    # at the pixel whose ray passes nearest the centre, the depth is z - r sqrt(1 - s^2) with s small
    u = cam.fx * c[0] / c[2] + cam.cx
    v = cam.fy * c[1] / c[2] + cam.cy
    i, j = int(u), int(v)
    s2 = ((i + 0.5 - u) / (cam.fx * r / c[2])) ** 2 + ((j + 0.5 - v) / (cam.fy * r / c[2])) ** 2
    assert abs(depth[j, i] - (c[2] - r * math.sqrt(1 - s2))) < 1e-14


def test_splat_keeps_the_nearest_and_ignores_order_and_hidden_particles():
    cam = _cam()
    rp = oracle.RenderParams(0.05, 0.01, 0.01, 3)
    x = np.stack([RNG.uniform(-0.3, 0.3, 200), RNG.uniform(-0.25, 0.25, 200), RNG.uniform(1.0, 2.0, 200)])
    x[2, :5] = -1.0  # behind the camera
    d_all, _, drawn = oracle.splat_depth(cam, rp, x)
    assert drawn == 195
    perm = RNG.permutation(200)
    d_perm, _, _ = oracle.splat_depth(cam, rp, x[:, perm])
    assert np.array_equal(d_all, d_perm)
    d_a, _, _ = oracle.splat_depth(cam, rp, x[:, :100])
    d_b, _, _ = oracle.splat_depth(cam, rp, x[:, 100:])
    assert np.array_equal(d_all, np.minimum(d_a, d_b))


def test_splat_respects_the_camera_pose():
    """Moving the camera and the particles by the same rigid motion leaves the image unchanged."""
    from scipy.spatial.transform import Rotation
    rp = oracle.RenderParams(0.05, 0.01, 0.01, 3)
    x = np.stack([RNG.uniform(-0.3, 0.3, 60), RNG.uniform(-0.25, 0.25, 60), RNG.uniform(1.0, 2.0, 60)])
    d0, _, _ = oracle.splat_depth(_cam(), rp, x)
    Q = Rotation.from_rotvec([0.3, -0.5, 0.2]).as_matrix()
    t = np.array([0.4, -0.1, 0.7])
    xw = Q @ x + t[:, None]
    cam = _cam(rot=Q.T, eye=tuple(t))  # camera frame = the moved frame
    d1, _, _ = oracle.splat_depth(cam, rp, xw)
    fin = np.isfinite(d0)
    assert np.array_equal(fin, np.isfinite(d1))
    assert np.abs(d0[fin] - d1[fin]).max() < 1e-12


def test_bilateral_keeps_constants_linear_ramps_and_deep_edges():
    cam = _cam(W=40, H=36)
    K = 4
    rp = oracle.RenderParams(0.05, 0.02, 1e6, K)  # range sigma huge: a plain Gaussian
    const = np.full((36, 40), 1.7)
    assert np.abs(oracle.bilateral(cam, rp, const) - 1.7).max() < 1e-14
    jj, ii = np.indices((36, 40))
    ramp = 1.5 + 0.01 * ii - 0.007 * jj
    out = oracle.bilateral(cam, rp, ramp)
    inner = (slice(K, 36 - K), slice(K, 40 - K))
    assert np.abs(out[inner] - ramp[inner]).max() < 1e-12
    # a step of 0.5 with range sigma 0.005: each side keeps its own depth
    step = np.where(ii < 20, 1.2, 1.7)
    rp_edge = oracle.RenderParams(0.05, 0.02, 0.005, K)
    out = oracle.bilateral(cam, rp_edge, step)
    assert np.abs(out - step).max() < 1e-12
    # empty pixels stay empty and are not averaged in
    holes = const.copy()
    holes[10:14, 10:14] = np.inf
    out = oracle.bilateral(cam, rp, holes)
    assert np.all(np.isinf(out[10:14, 10:14]))
    assert np.abs(out[np.isfinite(out)] - 1.7).max() < 1e-14


@pytest.mark.parametrize("d0", [0.8, 1.6, 3.0])
def test_bilateral_width_scales_with_distance(d0):
    """An impulse eps at one pixel of a flat field at depth d0: the filtered increments at horizontal
    offsets 1 and 2 from it are in the ratio exp(-(4 - 1) / (2 sigma^2)), which gives the filter's
    width sigma; it must be fx * smooth / d0 (capped at K / 2)."""
    cam = _cam(W=41, H=41, f=100.0)
    K, smooth = 6, 0.03
    rp = oracle.RenderParams(0.05, smooth, 1e6, K)
    z = np.full((41, 41), d0)
    eps = 1e-6
    z[20, 20] += eps
    out = oracle.bilateral(cam, rp, z)
    inc1 = out[20, 21] - d0
    inc2 = out[20, 22] - d0
    sigma = math.sqrt(3.0 / (2.0 * math.log(inc1 / inc2)))
    expect = min(cam.fx * smooth / d0, K / 2)
    assert abs(sigma - expect) < 1e-4 * expect


def _plane_depth(cam, n, h):
    """Per-pixel depth of the plane n . P = h seen by the camera (ray-plane intersection)."""
    jj, ii = np.indices((cam.height, cam.width))
    rx = (ii + 0.5 - cam.cx) / cam.fx
    ry = (jj + 0.5 - cam.cy) / cam.fy
    return h / (n[0] * rx + n[1] * ry + n[2])


def test_normals_of_planes_and_lambert_shading():
    cam = _cam(W=50, H=40)
    rp = oracle.RenderParams(0.05, 0.02, 0.01, 3, light=(0.2, -0.3, -1.0), albedo=(0.9, 0.5, 0.2), ambient=0.3,
                             background=(0.1, 0.2, 0.3))
    for _ in range(5):
        n = np.array([RNG.uniform(-0.4, 0.4), RNG.uniform(-0.4, 0.4), -1.0])
        n /= np.linalg.norm(n)  # facing the camera
        z = _plane_depth(cam, n, -1.5)
        z[:3, :5] = np.inf
        nrm, rgb, amb = oracle.shade(cam, rp, z)
        fin = np.isfinite(z)
        assert np.abs(nrm[fin] - n).max() < 1e-9
        l = np.array(rp.light) / np.linalg.norm(rp.light)
        lam = max(0.0, n @ l)
        expect = np.array(rp.albedo) * (rp.ambient + (1 - rp.ambient) * lam)
        assert np.abs(rgb[fin] - expect).max() < 1e-9
        assert np.all(rgb[~fin] == np.array(rp.background))
        assert np.all(nrm[~fin] == 0)


def test_normals_pick_the_side_that_stays_on_the_surface():
    """At the border of a near plane in front of a far one, the one-sided differences of the near
    plane's pixels use the near side, so their normal is the near plane's."""
    cam = _cam(W=40, H=30)
    rp = oracle.RenderParams(0.05, 0.02, 0.01, 3)
    near = np.array([0.0, 0.0, -1.0])
    z = np.full((30, 40), 3.0)
    z[:, :20] = _plane_depth(cam, np.array([0.2, 0.1, -1.0]) / np.linalg.norm([0.2, 0.1, -1.0]), -1.0)[:, :20]
    nrm, _, amb = oracle.shade(cam, rp, z)
    n_left = np.array([0.2, 0.1, -1.0]) / np.linalg.norm([0.2, 0.1, -1.0])
    assert np.abs(nrm[1:-1, 19] - n_left).max() < 1e-9  # last column of the near plane
    assert np.abs(nrm[1:-1, 20] - near).max() < 1e-9    # first column of the far (fronto-parallel) one
