"""Pins of the oracle's particle form of the contact (Sec. 3's default coupling; Algorithm 1 "compute
penalty forces" and "accumulate equivalent rigid-body forces and torques") and of its SDF volumes.

Hand-solved single-particle cases fix every branch of the penalty law (spring, approach damper,
viscous and Coulomb-capped friction, moving and spinning bodies, separation, no contact); the balance
of linear and angular momentum between the material and the bodies pins the reaction and its moment;
lattice-exact fields (planes, samples) and the piecewise-linear box pin the trilinear SDF volume."""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(20240)
KAPPA, BETA = 2.0e6, 1.5e3
PEN = oracle.Penalty(KAPPA, BETA)


def _params(n=32, gravity=(0.0, -9.8, 0.0), bound=3):
    return oracle.Params(n=n, dt=2e-4, gravity=gravity, bound=bound, p_vol=2e-6)


def _one(x, v):
    x = np.asarray(x, np.float64).reshape(3, 1)
    v = np.asarray(v, np.float64).reshape(3, 1)
    return oracle.State.from_arrays(x, v, np.zeros((9, 1)), np.eye(3).reshape(9, 1))


def _accel(col, x, v, t=0.0, P=None):
    P = P or _params()
    a, w, amb, nc = oracle.penalty_accel(P, PEN, _one(x, v), [col], t)
    return a[:, 0], w[0], bool(amb[0]), nc


BOX = oracle.Collider(oracle.BOX, (0.1, 0.08, 0.06), 0.5, pos=(0.5, 0.5, 0.5))


def test_penalty_spring_on_the_depth():
    d = 0.01  # below the +y face
    x = (0.52, 0.5 + 0.08 - d, 0.49)
    a, w, amb, nc = _accel(BOX, x, (0, 0, 0))
    assert nc == 1 and not amb
    np.testing.assert_allclose(a, [0.0, KAPPA * d, 0.0], rtol=1e-12, atol=1e-9)
    P = _params()
    m = P.c().p_mass
    imp = -P.dt * m * a
    np.testing.assert_allclose(w[:3], imp, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(w[3:], np.cross(np.array(x) - 0.5, imp), rtol=1e-12, atol=1e-18)


def test_penalty_damper_only_on_approach():
    d = 0.01
    x = (0.52, 0.5 + 0.08 - d, 0.49)
    a_in, *_ = _accel(BOX, x, (0, -0.3, 0))   # moving into the body
    a_out, *_ = _accel(BOX, x, (0, 0.3, 0))   # leaving it
    np.testing.assert_allclose(a_in, [0.0, KAPPA * d + BETA * 0.3, 0.0], rtol=1e-12)
    np.testing.assert_allclose(a_out, [0.0, KAPPA * d, 0.0], rtol=1e-12)


def test_penalty_friction_viscous_then_capped():
    d = 0.01
    x = (0.52, 0.5 + 0.08 - d, 0.49)
    an = KAPPA * d
    slow = 1e-3  # beta |v_t| = 1.5 m/s^2 < mu a_n = 1e4
    a, *_ = _accel(BOX, x, (slow, 0, 0))
    np.testing.assert_allclose(a, [-BETA * slow, an, 0.0], rtol=1e-12)
    fast = 20.0  # beta |v_t| = 3e4 > mu a_n
    a, *_ = _accel(BOX, x, (0, 0, -fast))
    np.testing.assert_allclose(a, [0.0, an, 0.5 * an], rtol=1e-12)


def test_penalty_moving_and_spinning_body():
    d = 0.01
    x = np.array([0.52, 0.5 + 0.08 - d, 0.49])
    lifted = oracle.Collider(oracle.BOX, BOX.half, 0.5, pos=BOX.pos, lin_vel=(0.0, 0.2, 0.0))
    a, *_ = _accel(lifted, x, (0, 0, 0))  # the face moves up into a resting particle
    np.testing.assert_allclose(a, [0.0, KAPPA * d + BETA * 0.2, 0.0], rtol=1e-12)
    # spinning about y through the centre: the body moves at w x r past the particle, friction drags it
    w = 3.0
    spin = oracle.Collider(oracle.BOX, BOX.half, 0.5, pos=BOX.pos, ang_vel=(0.0, w, 0.0))
    r = x - 0.5
    vc = np.cross([0.0, w, 0.0], r)
    a, wr, *_ = _accel(spin, x, (0, 0, 0))
    vt = -vc  # relative velocity of the particle, all tangential
    visc = BETA * np.linalg.norm(vt)
    cap = 0.5 * KAPPA * d
    at = -min(visc, cap) * vt / np.linalg.norm(vt)
    np.testing.assert_allclose(a, at + [0.0, KAPPA * d, 0.0], rtol=1e-12, atol=1e-9)
    # the reaction's moment about the centre of mass opposes the spin
    assert wr[4] * w < 0


def test_penalty_no_contact_outside_and_time_moves_the_body():
    x = (0.52, 0.5 + 0.08 + 0.005, 0.49)  # 5 mm above the face
    a, w, amb, nc = _accel(BOX, x, (0, -1.0, 0))
    assert nc == 0 and np.all(a == 0) and np.all(w == 0)
    # the same body moving up at 1 m/s reaches the particle after 5 ms: at t = 7 ms it is 2 mm deep
    up = oracle.Collider(oracle.BOX, BOX.half, 0.5, pos=BOX.pos, lin_vel=(0.0, 1.0, 0.0))
    a, w, amb, nc = _accel(up, x, (0, 0, 0), t=0.007)
    assert nc == 1
    np.testing.assert_allclose(a, [0.0, KAPPA * 0.002 + BETA * 1.0, 0.0], rtol=1e-9)
    com_t = np.array([0.5, 0.507, 0.5])
    np.testing.assert_allclose(w[3:], np.cross(np.array(x) - com_t, w[:3]), rtol=1e-9, atol=1e-18)


def test_penalty_laws_hold_over_random_contacts():
    """Over random particles and bodies: a_n >= 0, the friction part opposes the sliding velocity and
    stays in the Coulomb cone |a_t| <= mu a_n."""
    cap = oracle.Collider(oracle.CAPSULE, (0.04, 0.05, 0.0), 0.7, pos=(0.5, 0.5, 0.5), quat=(0.9, 0.1, -0.3, 0.2),
                          lin_vel=(0.1, -0.2, 0.05), ang_vel=(1.0, -2.0, 0.5), com=(0.5, 0.51, 0.49))
    n_checked = 0
    for _ in range(400):
        x = 0.5 + RNG.uniform(-0.07, 0.07, 3)
        v = RNG.normal(0, 0.5, 3)
        phi, nrm, amb = oracle.collider_sdf(cap, 0.0, x)
        a, w, _, nc = _accel(cap, x, v)
        if phi >= 0:
            assert nc == 0 and np.all(a == 0)
            continue
        n_checked += 1
        an = a @ nrm
        at = a - an * nrm
        R, p, com = oracle.collider_pose(cap, 0.0)
        vr = v - (np.array(cap.lin_vel) + np.cross(cap.ang_vel, x - com))
        vt = vr - (vr @ nrm) * nrm
        assert an >= -1e-9
        assert np.linalg.norm(at) <= 0.7 * an * (1 + 1e-12) + 1e-9
        if np.linalg.norm(at) > 0:
            assert at @ vt < 0
            assert np.linalg.norm(np.cross(at, vt)) <= 1e-9 * np.linalg.norm(at) * np.linalg.norm(vt)
    assert n_checked > 50


def _random_state(N, seed, lo=0.35, hi=0.65):
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, (3, N))
    v = rng.normal(0, 0.5, (3, N))
    C = rng.normal(0, 3.0, (9, N))
    F = (np.eye(3).reshape(9, 1) + rng.normal(0, 0.03, (9, N)))
    return oracle.State.from_arrays(x, v, C, F)


def _two_bodies():
    box = oracle.Collider(oracle.BOX, (0.08, 0.05, 0.07), 0.4, pos=(0.45, 0.5, 0.52), quat=(0.95, 0.2, 0.1, -0.2),
                          lin_vel=(0.3, 0.0, -0.1), ang_vel=(0.5, 1.5, -1.0), com=(0.46, 0.49, 0.52))
    cap = oracle.Collider(oracle.CAPSULE, (0.03, 0.06, 0.0), 0.6, pos=(0.58, 0.47, 0.5), quat=(0.8, 0.0, 0.6, 0.0),
                          lin_vel=(-0.2, 0.1, 0.0), ang_vel=(0.0, 0.0, 2.0))
    return [box, cap]


def test_penalty_momentum_balance_with_the_bodies():
    """What P2G adds to the grid's momentum through the forces is exactly what the bodies lose: the
    linear part equals minus the summed impulses, and the angular part (sum over nodes of x_i x mv_i)
    minus the summed angular impulses about the origin (tau_k + com_k(t) x J_k)."""
    P = _params(gravity=(0, 0, 0), bound=0)
    s = _random_state(3000, 7)
    cols = _two_bodies()
    t = 0.003
    acc, w, amb, nc = oracle.penalty_accel(P, PEN, s, cols, t)
    assert nc > 200
    g_with = oracle.p2g_forces(P, s, acc)
    g_without = oracle.p2g(P, s)
    n = P.n
    dmv = (g_with[..., 1:] - g_without[..., 1:]).reshape(-1, 3)
    idx = np.indices((n, n, n)).reshape(3, -1).T / n
    J = w[:, :3].sum(0)
    scale = np.abs(w[:, :3]).sum()
    np.testing.assert_allclose(dmv.sum(0), -J, atol=1e-12 * scale)
    L_grid = np.cross(idx, dmv).sum(0)
    L_bodies = np.zeros(3)
    for k, c in enumerate(cols):
        _, _, com = oracle.collider_pose(c, t)
        L_bodies += w[k, 3:] + np.cross(com, w[k, :3])
    np.testing.assert_allclose(L_grid, -L_bodies, atol=1e-11 * scale)
    # and the mass is untouched by the forces
    assert np.array_equal(g_with[..., 0], g_without[..., 0])


def test_penalty_substep_without_bodies_is_the_plain_substep():
    P = _params()
    s1 = _random_state(500, 8)
    s2 = s1.copy()
    oracle.substep(P, s1)
    oracle.substep_penalty(P, PEN, s2)
    for a in ("x", "v", "C", "F"):
        assert np.array_equal(getattr(s1, a), getattr(s2, a))


def test_penalty_pushes_a_particle_out_of_a_resting_body():
    """A lone particle placed inside a resting box with no gravity: the depth falls every substep until
    the particle leaves the body (the sign and the grid round trip of the force)."""
    P = _params(gravity=(0, 0, 0), bound=0)
    x = np.array([0.52, 0.5 + 0.08 - 0.004, 0.49])
    s = _one(x, (0, 0, 0))
    depth = [-oracle.collider_sdf(BOX, 0.0, s.x[:, 0])[0]]
    for _ in range(40):
        oracle.substep_penalty(P, PEN, s, [BOX])
        depth.append(-oracle.collider_sdf(BOX, 0.0, s.x[:, 0])[0])
        if depth[-1] < 0:
            break
    assert depth[-1] < 0, depth
    assert np.all(np.diff([d for d in depth if d > 0]) < 0)


# ------------------------------------------------------------------ SDF volumes

def _volume_collider(field, h, origin, **kw):
    return oracle.Collider(oracle.SDF_VOLUME, (0.0, 0.0, 0.0), kw.pop("friction", 0.5), kw.pop("pos", (0.0, 0.0, 0.0)),
                           sdf=field, sdf_origin=origin, sdf_h=h, **kw)


def test_sdf_volume_reproduces_samples_and_linear_fields():
    """Trilinear interpolation returns every lattice sample exactly and reproduces an affine field
    (value and gradient) everywhere inside the lattice."""
    res = (7, 5, 6)
    h = 0.013
    origin = (-0.04, -0.03, -0.035)
    ii = np.indices(res).astype(np.float64)
    pts = np.stack([origin[a] + h * ii[a] for a in range(3)])
    nrm = np.array([0.3, -0.5, 0.81])
    plane = np.tensordot(nrm, pts, axes=1) + 0.004
    col = _volume_collider(plane, h, origin)
    rand = RNG.normal(size=res)
    colr = _volume_collider(rand, h, origin)
    for i, j, k in [(0, 0, 0), (6, 4, 5), (3, 2, 1), (6, 0, 2)]:
        val, _, _ = oracle.sdf_volume(colr, pts[:, i, j, k])
        assert abs(val - rand[i, j, k]) <= 1e-12 * abs(rand).max()
    for _ in range(100):
        l = np.array([RNG.uniform(origin[a], origin[a] + h * (res[a] - 1)) for a in range(3)])
        val, g, _ = oracle.sdf_volume(col, l)
        assert abs(val - (nrm @ l + 0.004)) < 1e-14
        np.testing.assert_allclose(g, nrm, atol=1e-12)


def test_sdf_volume_outside_the_lattice_is_no_contact_and_pose_applies():
    res = (5, 5, 5)
    h = 0.02
    origin = (-0.04, -0.04, -0.04)
    field = -np.ones(res)  # "inside" everywhere on the lattice
    from scipy.spatial.transform import Rotation
    q = Rotation.from_rotvec([0.3, -0.2, 0.5])
    qw = q.as_quat()
    col = _volume_collider(field, h, origin, pos=(0.5, 0.5, 0.5), quat=(qw[3], qw[0], qw[1], qw[2]))
    phi, nrm, _ = oracle.collider_sdf(col, 0.0, 0.5 + q.apply([0.01, -0.02, 0.03]))
    assert phi == -1.0 and np.all(nrm == 0)  # constant field: no gradient, no normal
    assert oracle.sdf_volume(col, np.array([0.05, 0.0, 0.0])) is None
    phi, nrm, _ = oracle.collider_sdf(col, 0.0, 0.5 + q.apply([0.041, 0.0, 0.0]))
    assert phi == 1e30
    # an affine field: the world normal is the rotated field gradient
    ii = np.indices(res).astype(np.float64)
    pts = np.stack([origin[a] + h * ii[a] for a in range(3)])
    gl = np.array([0.0, 0.6, 0.8])
    col = _volume_collider(np.tensordot(gl, pts, axes=1), h, origin, pos=(0.5, 0.5, 0.5),
                           quat=(qw[3], qw[0], qw[1], qw[2]))
    phi, nrm, _ = oracle.collider_sdf(col, 0.0, 0.5 + q.apply([0.01, 0.01, -0.02]))
    assert abs(phi - (0.6 * 0.01 - 0.8 * 0.02)) < 1e-14
    np.testing.assert_allclose(nrm, q.apply(gl), atol=1e-12)


def _box_volume(half, h, pad=3):
    half = np.asarray(half)
    res = tuple(int(np.ceil(2 * (half[a] + pad * h) / h)) + 1 for a in range(3))
    origin = tuple(-(res[a] - 1) * h / 2 for a in range(3))
    ii = np.indices(res).astype(np.float64)
    pts = np.stack([origin[a] + h * ii[a] for a in range(3)]).reshape(3, -1).T
    box = oracle.Collider(oracle.BOX, tuple(half), 0.5, pos=(0.0, 0.0, 0.0))
    field = np.array([oracle.collider_sdf(box, 0.0, p)[0] for p in pts]).reshape(res)
    return field, origin


def test_sdf_volume_of_a_box_equals_the_box_away_from_its_ridges():
    """The box SDF is linear wherever one face is the nearest (inside) or the only one exceeded
    (outside): in lattice cells whose corners all lie in one such region the volume equals the analytic
    box, value and normal; the penalty computed from either collider is then the same."""
    half = (0.05, 0.035, 0.04)
    h = 0.01
    field, origin = _box_volume(half, h)
    from scipy.spatial.transform import Rotation
    q = Rotation.from_rotvec([0.2, 0.4, -0.1])
    qw = q.as_quat()
    kw = dict(pos=(0.5, 0.5, 0.5), quat=(qw[3], qw[0], qw[1], qw[2]), lin_vel=(0.1, 0.0, -0.2), ang_vel=(0, 1.0, 0))
    vol = _volume_collider(field, h, origin, **kw)
    box = oracle.Collider(oracle.BOX, half, 0.5, **kw)
    hv = np.asarray(half)

    def region(l):  # which linear piece of the box SDF holds l (None on a ridge-crossing piece)
        qv = np.abs(l) - hv
        if np.all(qv < 0):
            return ("in", int(np.argmax(qv)), bool(l[np.argmax(qv)] >= 0))
        pos = qv > 0
        if pos.sum() == 1:
            ax = int(np.argmax(pos))
            return ("out", ax, bool(l[ax] >= 0))
        return None

    checked = 0
    for _ in range(3000):
        l = RNG.uniform(-1.3, 1.3, 3) * hv
        c = np.floor((l - origin) / h)
        corners = [origin + h * (c + np.array(o)) for o in np.ndindex(2, 2, 2)]
        r = {region(p) for p in corners}
        if len(r) != 1 or None in r:
            continue
        checked += 1
        x = 0.5 + q.apply(l)
        pv, nv, _ = oracle.collider_sdf(vol, 0.0, x)
        pb, nb, _ = oracle.collider_sdf(box, 0.0, x)
        assert abs(pv - pb) < 1e-13
        np.testing.assert_allclose(nv, nb, atol=1e-12)
        if pb < 0:
            v = RNG.normal(0, 0.3, 3)
            a1, w1, *_ = _accel(vol, x, v)
            a2, w2, *_ = _accel(box, x, v)
            np.testing.assert_allclose(a1, a2, rtol=1e-11, atol=1e-6)
    assert checked > 300
