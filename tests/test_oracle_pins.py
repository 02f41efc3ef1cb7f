"""Pins of the FP64 oracle against facts fixed by the mathematics, not by the oracle itself.

Each test names what pins it: a closed form, an exact invariant of the APIC/MLS
transfers (Jiang et al. 2015; Hu et al. 2018), a brute-force evaluation on tiny
inputs, a library routine (numpy / scipy) for a textbook sub-problem, or a
hand-solved case. A plausible slip in the oracle (a dropped term, a wrong sign
or index, a transposed operand) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2302_04659_gb300 import scenes

RNG = np.random.default_rng(12345)


def rand_rot(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


# ---------------------------------------------------------------------------- weights (A2, A4)

@pytest.mark.parametrize("n", [4, 6, 8, 32, 64])
def test_weight_moments_closed_form(n):
    """The quadratic B-spline stencil has sum w = 1, sum w d = 0, sum w d d^T = dx^2/4 I.
    Three moments per axis fix the three weights uniquely, so this pins the weights."""
    dx = 1.0 / n
    for _ in range(200):
        x = RNG.uniform(1.5 * dx, 1 - 2.5 * dx, size=3)
        base, idx, w, d = oracle.stencil(n, x)
        assert abs(w.sum() - 1.0) < 1e-14
        assert np.abs((w[:, None] * d).sum(0)).max() < 1e-15
        M = (w[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0)
        assert np.abs(M - dx * dx / 4 * np.eye(3)).max() < 1e-17 * 1e2
        assert (w >= 0).all()


@pytest.mark.parametrize("n", [4, 5, 8])
def test_stencil_brute_force_tiny_grid(n):
    """Brute force: evaluate the B-spline product at EVERY node of a tiny grid; the 27-node stencil
    must hold exactly the nonzero weights, at the right node indices."""
    dx = 1.0 / n
    nodes = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3) * dx
    for _ in range(50):
        x = RNG.uniform(1.0 * dx, 1 - 2.0 * dx, size=3)
        u = (x[None, :] - nodes) / dx
        wbf = np.prod([[oracle.bspline(ui) for ui in row] for row in u], axis=1)
        base, idx, w, d = oracle.stencil(n, x)
        dense = np.zeros(n ** 3)
        np.add.at(dense, idx, w)
        assert np.abs(dense - wbf).max() < 1e-15
        assert np.allclose(d, nodes[idx] - x[None, :], atol=1e-15)


def test_bspline_values():
    """The 1-D kernel at a few points (textbook values of the quadratic B-spline)."""
    assert oracle.bspline(0.0) == 0.75
    assert oracle.bspline(0.5) == 0.5
    assert oracle.bspline(-0.5) == 0.5
    assert oracle.bspline(1.0) == 0.125
    assert oracle.bspline(1.5) == 0.0
    assert oracle.bspline(2.0) == 0.0


# ---------------------------------------------------------------------------- material constants

def test_lame_inverse_relations():
    """mu, lambda must reproduce E and nu through the inverse relations of linear elasticity."""
    for E, nu in [(5e3, 0.3), (1e4, 0.3), (3e5, 0.3), (1e6, 0.45)]:
        mu, la = oracle.lame(E, nu)
        assert abs(mu * (3 * la + 2 * mu) / (la + mu) - E) < 1e-9 * E
        assert abs(la / (2 * (la + mu)) - nu) < 1e-14


# ---------------------------------------------------------------------------- SVD

def _svd_cases():
    cases = [np.eye(3), np.diag([2.0, 2.0, 0.5]), np.diag([1.0, 1.0, 1.0]) * 0.7, rand_rot(RNG),
             np.diag([1.5, 0.9, -0.8]), np.diag([3.0, 1e-9, 1e-9]) @ rand_rot(RNG)]
    for _ in range(200):
        cases.append(np.eye(3) + 0.3 * RNG.normal(size=(3, 3)))
    for _ in range(50):
        cases.append(RNG.normal(size=(3, 3)))
    return cases


def test_svd_against_numpy():
    """One-sided Jacobi SVD: reconstruction, orthogonality, rotations only, and the singular values
    of numpy.linalg.svd (LAPACK) up to the sign convention for det F < 0."""
    for F in _svd_cases():
        U, S, V, sweeps = oracle.svd3(F)
        scale = max(1.0, np.abs(F).max())
        assert np.abs(U @ np.diag(S) @ V.T - F).max() < 1e-13 * scale
        assert np.abs(U.T @ U - np.eye(3)).max() < 1e-13
        assert np.abs(V.T @ V - np.eye(3)).max() < 1e-13
        assert abs(np.linalg.det(U) - 1) < 1e-13 and abs(np.linalg.det(V) - 1) < 1e-13
        ref = np.linalg.svd(F, compute_uv=False)
        assert np.abs(np.sort(np.abs(S))[::-1] - ref).max() < 1e-13 * scale
        assert (S[2] < 0) == (np.linalg.det(F) < 0) or abs(S[2]) < 1e-12
        assert sweeps < 60


# ---------------------------------------------------------------------------- stress (A1)

def _psi(mu, la, F):
    """Fixed-corotated energy density mu ||F - R||^2 + lambda/2 (J - 1)^2 through numpy's SVD."""
    s = np.linalg.svd(F, compute_uv=False)
    J = np.linalg.det(F)
    return mu * ((s - 1) ** 2).sum() + 0.5 * la * (J - 1) ** 2


def test_stress_is_energy_derivative():
    """tau = (d psi / d F) F^T, the derivative taken by central finite differences of the energy."""
    mu, la = oracle.lame(5e3, 0.3)
    for _ in range(30):
        F = np.eye(3) + 0.2 * RNG.normal(size=(3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        P = np.zeros((3, 3))
        h = 1e-6
        for i in range(3):
            for j in range(3):
                E = np.zeros((3, 3)); E[i, j] = h
                P[i, j] = (_psi(mu, la, F + E) - _psi(mu, la, F - E)) / (2 * h)
        tau_fd = P @ F.T
        tau = oracle.stress(mu, la, F)
        assert np.abs(tau - tau_fd).max() < 1e-5 * max(1.0, np.abs(tau).max())


def test_stress_closed_forms_and_frame_indifference():
    mu, la = oracle.lame(5e3, 0.3)
    assert np.abs(oracle.stress(mu, la, np.eye(3))).max() < 1e-12
    # F = sI: R = I, so (F - R) F^T = s (s - 1) I and J = s^3
    for s in [0.8, 1.0, 1.3]:
        tau = oracle.stress(mu, la, s * np.eye(3))
        expect = (2 * mu * s * (s - 1) + la * s ** 3 * (s ** 3 - 1)) * np.eye(3)
        assert np.abs(tau - expect).max() < 1e-9 * la
    for _ in range(20):
        F = np.eye(3) + 0.2 * RNG.normal(size=(3, 3))
        if np.linalg.det(F) < 0.2:
            continue
        Q = rand_rot(RNG)
        tau = oracle.stress(mu, la, F)
        assert np.abs(tau - tau.T).max() < 1e-9 * mu
        assert np.abs(oracle.stress(mu, la, Q @ F) - Q @ tau @ Q.T).max() < 1e-9 * mu
        assert np.abs(oracle.stress(mu, la, F @ Q) - tau).max() < 1e-9 * mu


# ---------------------------------------------------------------------------- return map (A5)

def test_return_map_invariants():
    """Von Mises in Hencky strain: projected states lie on the yield sphere, keep tr(log sigma),
    keep the singular vectors; states inside are returned bit-for-bit unchanged."""
    mu, la = oracle.lame(5e3, 0.3)
    ty = 50.0
    radius = ty / (2 * mu)
    n_proj = 0
    for _ in range(300):
        F = np.eye(3) + 0.05 * RNG.normal(size=(3, 3))
        Fn, proj, cl = oracle.return_map(mu, ty, F)
        s0 = np.linalg.svd(F, compute_uv=False)
        s1 = np.linalg.svd(Fn, compute_uv=False)
        e0, e1 = np.log(s0), np.log(s1)
        dev0 = np.linalg.norm(e0 - e0.mean())
        dev1 = np.linalg.norm(e1 - e1.mean())
        assert not cl
        if dev0 <= radius:
            assert not proj
            assert np.array_equal(Fn, F)
        else:
            n_proj += 1
            assert proj
            assert abs(dev1 - radius) < 1e-12
            assert abs(e1.sum() - e0.sum()) < 1e-12
            # coaxial: Fn F^-1 = U diag(s1/s0) U^T is symmetric positive definite
            M = Fn @ np.linalg.inv(F)
            assert np.abs(M - M.T).max() < 1e-12
    assert n_proj > 50


def test_return_map_isotropy_and_diagonal_case():
    mu, la = oracle.lame(5e3, 0.3)
    ty = 50.0
    radius = ty / (2 * mu)
    for _ in range(30):
        F = np.eye(3) + 0.08 * RNG.normal(size=(3, 3))
        Q1, Q2 = rand_rot(RNG), rand_rot(RNG)
        Fn, _, _ = oracle.return_map(mu, ty, F)
        Fr, _, _ = oracle.return_map(mu, ty, Q1 @ F @ Q2)
        assert np.abs(Fr - Q1 @ Fn @ Q2).max() < 1e-12
    # diagonal F: projection along the deviatoric direction of log(diag), closed form
    d = np.array([1.08, 0.97, 0.95])
    e = np.log(d)
    dev = e - e.mean()
    e_new = e.mean() + dev * radius / np.linalg.norm(dev)
    Fn, proj, _ = oracle.return_map(mu, ty, np.diag(d))
    assert proj
    assert np.abs(Fn - np.diag(np.exp(e_new))).max() < 1e-13


# ---------------------------------------------------------------------------- colliders (A3)

def test_collider_pose_translation_rotation():
    from scipy.spatial.transform import Rotation
    q0 = Rotation.from_rotvec([0.3, -0.2, 0.5])
    qw = q0.as_quat()  # x y z w
    col = oracle.Collider(oracle.BOX, (0.1, 0.05, 0.02), 0.5, pos=(0.4, 0.5, 0.6),
                          quat=(qw[3], qw[0], qw[1], qw[2]), lin_vel=(0.3, -0.1, 0.2),
                          ang_vel=(1.0, 2.0, -0.5), com=(0.45, 0.5, 0.58))
    for t in [0.0, 1e-3, 0.05, 0.4]:
        R, p, com = oracle.collider_pose(col, t)
        Rt = (Rotation.from_rotvec(np.array(col.ang_vel) * t) * q0).as_matrix()
        assert np.abs(R - Rt).max() < 1e-14
        assert np.abs(com - (np.array(col.com) + t * np.array(col.lin_vel))).max() < 1e-15
        # the frame origin is carried rigidly about the centre of mass
        d0 = np.array(col.pos) - np.array(col.com)
        assert np.abs((p - com) - Rotation.from_rotvec(np.array(col.ang_vel) * t).apply(d0)).max() < 1e-14
    # velocity of a body point = lin_vel + w x (x - com)  (finite difference in time)
    t, h = 0.1, 1e-6
    xb = np.array([0.02, -0.01, 0.03])
    R1, p1, c1 = oracle.collider_pose(col, t - h)
    R2, p2, c2 = oracle.collider_pose(col, t + h)
    R0, p0, c0 = oracle.collider_pose(col, t)
    vfd = ((p2 + R2 @ xb) - (p1 + R1 @ xb)) / (2 * h)
    x0 = p0 + R0 @ xb
    vex = np.array(col.lin_vel) + np.cross(col.ang_vel, x0 - c0)
    assert np.abs(vfd - vex).max() < 1e-8


def _surface_samples_box(h, m=60):
    pts = []
    g = np.linspace(-1, 1, m)
    A, B = np.meshgrid(g, g, indexing="ij")
    for ax in range(3):
        o = [a for a in range(3) if a != ax]
        for s in (-1, 1):
            P = np.zeros((m * m, 3))
            P[:, ax] = s * h[ax]
            P[:, o[0]] = A.ravel() * h[o[0]]
            P[:, o[1]] = B.ravel() * h[o[1]]
            pts.append(P)
    return np.concatenate(pts)


def test_sdf_box_brute_force():
    h = np.array([0.1, 0.05, 0.07])
    col = oracle.Collider(oracle.BOX, tuple(h), 0.5, pos=(0.5, 0.5, 0.5))
    S = _surface_samples_box(h) + 0.5
    spacing = 2 * h.max() / 59
    for _ in range(200):
        x = 0.5 + RNG.uniform(-0.2, 0.2, size=3)
        phi, nrm, amb = oracle.collider_sdf(col, 0.0, x)
        inside = np.all(np.abs(x - 0.5) < h)
        assert (phi < 0) == inside
        dist = np.sqrt(((S - x) ** 2).sum(1)).min()
        assert abs(abs(phi) - dist) < spacing
        assert abs(np.linalg.norm(nrm) - 1) < 1e-12
        if not amb:
            e = 1e-7
            g = np.array([(oracle.collider_sdf(col, 0.0, x + e * np.eye(3)[a])[0] -
                           oracle.collider_sdf(col, 0.0, x - e * np.eye(3)[a])[0]) / (2 * e) for a in range(3)])
            assert np.abs(g - nrm).max() < 1e-5


def test_sdf_capsule_brute_force():
    r, hl = 0.02, 0.05
    from scipy.spatial.transform import Rotation
    q = Rotation.from_rotvec([0.4, 0.1, -0.3])
    qw = q.as_quat()
    col = oracle.Collider(oracle.CAPSULE, (r, hl, 0.0), 0.5, pos=(0.5, 0.5, 0.5), quat=(qw[3], qw[0], qw[1], qw[2]))
    a = 0.5 + q.apply([0, 0, -hl])
    b = 0.5 + q.apply([0, 0, hl])
    ts = np.linspace(0, 1, 20001)
    seg = a[None, :] + ts[:, None] * (b - a)[None, :]
    for _ in range(200):
        x = 0.5 + RNG.uniform(-0.1, 0.1, size=3)
        phi, nrm, amb = oracle.collider_sdf(col, 0.0, x)
        dist = np.sqrt(((seg - x) ** 2).sum(1)).min() - r
        assert abs(phi - dist) < 1e-7
        e = 1e-7
        g = np.array([(oracle.collider_sdf(col, 0.0, x + e * np.eye(3)[k])[0] -
                       oracle.collider_sdf(col, 0.0, x - e * np.eye(3)[k])[0]) / (2 * e) for k in range(3)])
        assert np.abs(g - nrm).max() < 1e-5


def _one_node_grid(n, node, m, v):
    g = np.zeros((n, n, n, 4))
    g[node][0] = m
    g[node][1:] = m * np.asarray(v)
    return g


def test_grid_update_hand_solved_contact():
    """Single-node Coulomb cases solved by hand: stick, slip, separating, moving body, wall band."""
    n = 16
    dx = 1.0 / n
    P = oracle.Params(n=n, dt=1e-3, gravity=(0.0, 0.0, 0.0), bound=3)
    node = (8, 8, 8)
    xi = np.array(node) * dx
    # static box whose +y face lies just above the node: the node is inside, normal +y
    h = (0.2, 0.1, 0.2)
    box = oracle.Collider(oracle.BOX, h, 0.5, pos=(xi[0], xi[1] - h[1] + 0.01, xi[2]))
    m = 2.0
    cases = [
        ((0.3, -1.0, 0.0), (0.0, 0.0, 0.0)),       # |vt| = 0.3 <= 0.5 * 1: stick
        ((2.0, -1.0, 0.0), (1.5, 0.0, 0.0)),       # slip: vt (1 - 0.5 * 1 / 2)
        ((0.3, 1.0, 0.0), (0.3, 1.0, 0.0)),        # separating: unchanged
        ((0.0, -1.0, 0.0), (0.0, 0.0, 0.0)),       # head-on: stick
    ]
    for vin, vout in cases:
        g, w, _ = oracle.grid_update(P, _one_node_grid(n, node, m, vin), [box], 0.0)
        assert np.abs(g[node][1:] - vout).max() < 1e-14, (vin, g[node][1:])
        assert g[node][0] == m
        imp = m * (np.array(vin) - np.array(vout))
        assert np.abs(w[0, :3] - imp).max() < 1e-14
        assert np.abs(w[0, 3:] - np.cross(xi - np.array(box.pos), imp)).max() < 1e-14
    # moving box pushes a resting node: relative velocity -0.5 along the normal, sticks to the body
    mov = oracle.Collider(oracle.BOX, h, 0.5, pos=box.pos, lin_vel=(0.0, 0.5, 0.0))
    g, w, _ = oracle.grid_update(P, _one_node_grid(n, node, m, (0.0, 0.0, 0.0)), [mov], 0.0)
    assert np.abs(g[node][1:] - np.array([0.0, 0.5, 0.0])).max() < 1e-14
    assert np.abs(w[0, :3] - np.array([0.0, -1.0, 0.0])).max() < 1e-14
    # spinning capsule about z through its com: body velocity at the node is w x (x - com)
    r, hl = 0.05, 0.2
    cap = oracle.Collider(oracle.CAPSULE, (r, hl, 0.0), 0.0, pos=(xi[0] + 0.04, xi[1], xi[2]),
                          ang_vel=(0.0, 0.0, 2.0), com=(xi[0] + 0.04, xi[1], xi[2]))
    # node at -0.04 x from the axis, inside; normal -x; body velocity (0, 2*(-0.04), 0) = (0,-0.08,0)
    vin = np.array([0.3, 0.1, 0.0])  # moving +x into the body: vn = -0.3; friction 0 -> keep tangential
    g, w, _ = oracle.grid_update(P, _one_node_grid(n, node, m, vin), [cap], 0.0)
    vc = np.array([0.0, -0.08, 0.0])
    vr = vin - vc
    expect = vc + np.array([0.0, vr[1], vr[2]])
    assert np.abs(g[node][1:] - expect).max() < 1e-14
    # wall band zeroes velocity without touching the wrench
    band = (1, 8, 8)
    g, w, _ = oracle.grid_update(P, _one_node_grid(n, band, m, (0.3, 0.2, 0.1)), [], 0.0)
    assert np.all(g[band][1:] == 0.0)
    # gravity adds dt g before contact
    P2 = oracle.Params(n=n, dt=1e-3, gravity=(0.0, -9.8, 0.0), bound=3)
    g, _, _ = oracle.grid_update(P2, _one_node_grid(n, node, m, (0.1, 0.2, 0.3)), [], 0.0)
    assert np.abs(g[node][1:] - np.array([0.1, 0.2 - 9.8e-3, 0.3])).max() < 1e-15


def test_grid_update_massless_nodes_get_zero_velocity():
    n = 8
    P = oracle.Params(n=n, dt=1e-3)
    g = np.zeros((n, n, n, 4))
    g[..., 1:] = 5.0  # momentum without mass must not produce velocity
    out, _, _ = oracle.grid_update(P, g)
    assert np.all(out[..., 1:] == 0.0)


# ---------------------------------------------------------------------------- transfers (A2, A4)

def _tiny_state(n, N, kind, seed):
    rng = np.random.default_rng(seed)
    dx = 1.0 / n
    x = rng.uniform(2 * dx, 1 - 2 * dx, size=(3, N))
    v = rng.normal(size=(3, N))
    C = rng.normal(size=(9, N)) * 3
    F = (np.eye(3).reshape(9, 1) + 0.1 * rng.normal(size=(9, N)))
    J = rng.uniform(0.8, 1.2, size=N)
    return oracle.State.from_arrays(x, v, C, F if kind == oracle.PLASTICINE else None,
                                    J if kind == oracle.FLUID else None)


@pytest.mark.parametrize("kind", [oracle.PLASTICINE, oracle.FLUID])
def test_p2g_brute_force(kind):
    """P2G equals a brute-force double loop over (particle, every node) with the B-spline product."""
    n, N = 8, 25
    s = _tiny_state(n, N, kind, 7)
    P = oracle.Params(n=n, dt=1e-3, kind=kind, p_vol=1e-3)
    pc = P.c()
    grid = oracle.p2g(P, s)
    dx = 1.0 / n
    nodes = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3) * dx
    ref = np.zeros((n ** 3, 4))
    bs = np.vectorize(oracle.bspline)
    for p in range(N):
        xp = s.x[:, p]
        w = np.prod(bs((nodes - xp[None, :]) / dx), axis=1)
        if kind == oracle.PLASTICINE:
            tau = oracle.stress(pc.mu, pc.lam, s.F[:, p].reshape(3, 3))
        else:
            tau = pc.lam * s.J[p] * (s.J[p] - 1) * np.eye(3)
        A = pc.p_mass * s.C[:, p].reshape(3, 3) - P.dt * P.p_vol * 4 / dx ** 2 * tau
        d = nodes - xp[None, :]
        ref[:, 0] += w * pc.p_mass
        ref[:, 1:] += w[:, None] * (pc.p_mass * s.v[:, p][None, :] + d @ A.T)
    assert np.abs(grid.reshape(-1, 4) - ref).max() < 1e-12 * np.abs(ref).max()


def _mls_energy(P, pc, s, node, disp, stencils):
    """Total elastic energy sum_p V0 psi(F_p(x^)) after moving one grid node by `disp`, with each
    particle's deformation gradient carried by the MLS-MPM update that the node positions define:
    F_p(x^) = (I + D^-1 sum_i w_ip (x^_i - x_i)(x_i - x_p)^T) F_p, D^-1 = 4/dx^2 (Hu et al. 2018).
    Only the moved node contributes to the sum. Plasticine: fixed-corotated psi through numpy's SVD;
    fluid: psi(J) = lambda/2 (J - 1)^2 with J_p(x^) = J_p det(I + ...)."""
    dx = 1.0 / P.n
    Dinv = 4.0 / dx ** 2
    E = 0.0
    for p, (idx, w, d) in enumerate(stencils):
        G = np.eye(3)
        for q in range(27):
            if idx[q] == node:
                G = G + Dinv * w[q] * np.outer(disp, d[q])
        if P.kind == oracle.PLASTICINE:
            E += P.p_vol * _psi(pc.mu, pc.lam, G @ s.F[:, p].reshape(3, 3))
        else:
            J = s.J[p] * np.linalg.det(G)
            E += P.p_vol * 0.5 * pc.lam * (J - 1.0) ** 2
    return E


@pytest.mark.parametrize("kind", [oracle.PLASTICINE, oracle.FLUID])
def test_p2g_stress_momentum_is_minus_dt_energy_gradient(kind):
    """The stress half of the particle-to-grid momentum (Algorithm 1's "forces"; MLS-MPM, Hu et al.
    2018) is dt times the grid force f_i = -dE/dx^_i, the derivative of the total elastic energy with
    respect to the node position taken here by central finite differences of E through the MLS
    deformation-gradient update and numpy's SVD. With v = 0 and C = 0 the transfer's momentum is that
    term alone, so this fixes its sign, the D^-1 = 4/dx^2 scale, V0, dt and tau = (dpsi/dF) F^T, none
    of which the momentum-conservation pins can see."""
    n, N = 8, 6
    rng = np.random.default_rng(21)
    dx = 1.0 / n
    x = rng.uniform(2.2 * dx, 1 - 2.2 * dx, size=(3, N))
    F = np.empty((9, N))
    for p in range(N):
        while True:
            Fp = np.eye(3) + 0.15 * rng.normal(size=(3, 3))
            if np.linalg.det(Fp) > 0.3:
                break
        F[:, p] = Fp.reshape(9)
    J = rng.uniform(0.7, 1.3, size=N)
    s = oracle.State.from_arrays(x, np.zeros((3, N)), np.zeros((9, N)), F if kind == oracle.PLASTICINE else None,
                                 J if kind == oracle.FLUID else None)
    P = oracle.Params(n=n, dt=1e-3, kind=kind, p_vol=2e-3)
    pc = P.c()
    mom = oracle.p2g(P, s).reshape(-1, 4)[:, 1:]
    stencils = []
    for p in range(N):
        _, idx, w, d = oracle.stencil(n, s.x[:, p])
        stencils.append((idx, w, d))
    nodes = sorted({int(i) for idx, _, _ in stencils for i in idx})
    h = 1e-7
    worst = 0.0
    scale = np.abs(mom).max()
    assert scale > 0.0
    for node in nodes:
        grad = np.zeros(3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            grad[a] = (_mls_energy(P, pc, s, node, e, stencils) - _mls_energy(P, pc, s, node, -e, stencils)) / (2 * h)
        worst = max(worst, np.abs(mom[node] - (-P.dt * grad)).max())
    assert worst < 1e-6 * scale
    # nodes outside every stencil receive nothing
    others = np.setdiff1d(np.arange(n ** 3), nodes)
    assert np.abs(mom[others]).max() == 0.0


def test_return_map_singular_value_clamp_branch():
    """Singular values below 1e-6 are raised to 1e-6 before the logarithm and F is rebuilt from the
    clamped values, even when the clamped state lies inside the yield surface (closed forms)."""
    mu, la = oracle.lame(5e3, 0.3)
    ty = 50.0
    radius = ty / (2 * mu)
    rng = np.random.default_rng(5)
    U, V = rand_rot(rng), rand_rot(rng)
    # all three below the floor: log sigma = log(1e-6) (1, 1, 1) has no deviatoric part, so no projection;
    # F comes back as 1e-6 U V^T
    Ftr = U @ np.diag([3e-8, 1e-9, 5e-7]) @ V.T
    Fn, proj, cl = oracle.return_map(mu, ty, Ftr)
    assert cl and not proj
    assert np.abs(Fn - 1e-6 * U @ V.T).max() < 1e-18
    # one below the floor: clamped, then projected onto the yield sphere with the trace kept
    Ftr = U @ np.diag([1e-9, 1.02, 0.99]) @ V.T
    Fn, proj, cl = oracle.return_map(mu, ty, Ftr)
    assert cl and proj
    e = np.log([1e-6, 1.02, 0.99])
    dev = e - e.mean()
    e_new = e.mean() + dev * radius / np.linalg.norm(dev)
    assert np.abs(Fn - U @ np.diag(np.exp(e_new)) @ V.T).max() < 1e-12
    # just above the floor: no clamp, and inside the yield surface nothing changes
    Ftr = U @ np.diag([1.001, 1.0, 0.999]) @ V.T
    Fn, proj, cl = oracle.return_map(mu, ty, Ftr)
    assert not cl and not proj and np.array_equal(Fn, Ftr)


def test_g2p_reproduces_affine_velocity_fields():
    """APIC reproduces affine fields exactly: grid v_i = a + B x_i gives v_p = a + B x_p, C_p = B."""
    n, N = 16, 40
    dx = 1.0 / n
    rng = np.random.default_rng(3)
    a = rng.normal(size=3)
    B = rng.normal(size=(3, 3))
    nodes = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3) * dx
    grid = np.zeros((n ** 3, 4))
    grid[:, 0] = 1.0
    grid[:, 1:] = a[None, :] + nodes @ B.T
    s = _tiny_state(n, N, oracle.FLUID, 4)
    x0 = s.x.copy()
    J0 = s.J.copy()
    P = oracle.Params(n=n, dt=1e-3, kind=oracle.FLUID, p_vol=1e-3)
    oracle.g2p(P, grid, s)
    vp = a[:, None] + B @ x0
    assert np.abs(s.v - vp).max() < 1e-12
    assert np.abs(s.C.reshape(3, 3, N) - B[:, :, None]).max() < 1e-10
    assert np.abs(s.x - np.clip(x0 + P.dt * vp, 2 * dx, 1 - 2 * dx)).max() < 1e-15
    assert np.abs(s.J - J0 * np.linalg.det(np.eye(3) + P.dt * B)).max() < 1e-12


def test_g2p_uniform_dilation_updates_F_without_yield():
    """A pure dilation v = alpha (x - x0) is volumetric, so plasticity never acts: F -> (1 + dt alpha) F."""
    n, N = 16, 30
    dx = 1.0 / n
    alpha = 3.0
    nodes = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3) * dx
    grid = np.zeros((n ** 3, 4))
    grid[:, 0] = 1.0
    grid[:, 1:] = alpha * (nodes - 0.5)
    rng = np.random.default_rng(9)
    x = rng.uniform(0.3, 0.7, size=(3, N))
    F = np.tile(np.eye(3).reshape(9, 1), (1, N))
    s = oracle.State.from_arrays(x, np.zeros((3, N)), np.zeros((9, N)), F)
    P = oracle.Params(n=n, dt=1e-3, p_vol=1e-3)
    oracle.g2p(P, grid, s)
    assert np.abs(s.F - (1 + P.dt * alpha) * F).max() < 1e-12


# ---------------------------------------------------------------------------- conservation through a substep

def _free_state(seed):
    sc = scenes.cube_scene("ff")
    v, C, F = scenes.random_state(sc.N, seed)
    return sc, oracle.State.from_arrays(sc.x, v, C, F)


def _angular_momentum(s, mass, dx):
    L = (mass * np.cross(s.x.T, s.v.T)).sum(0)
    C = s.C.reshape(3, 3, -1)
    # (dx^2/4) eps_abc C_cb for each particle
    spin = np.stack([C[2, 1] - C[1, 2], C[0, 2] - C[2, 0], C[1, 0] - C[0, 1]])
    return L + mass * dx * dx / 4 * spin.sum(1)


def test_mass_after_p2g_exact():
    sc, s = _free_state(5)
    P = oracle.Params(n=sc.n, dt=sc.dt, p_vol=sc.material.p_vol)
    grid = oracle.p2g(P, s)
    total = grid[..., 0].sum()
    expect = sc.N * P.c().p_mass
    assert abs(total - expect) < 1e-13 * expect


@pytest.mark.parametrize("kind", [oracle.PLASTICINE, oracle.FLUID])
def test_linear_and_angular_momentum_conserved(kind):
    """Without gravity, walls or colliders, a full substep conserves total linear momentum and the
    APIC angular momentum sum m_p [x_p x v_p + dx^2/4 eps:C_p] exactly (Jiang et al. 2015)."""
    sc, s = _free_state(6)
    if kind == oracle.FLUID:
        s = oracle.State.from_arrays(s.x, s.v, s.C, None, np.linalg.det(s.F.T.reshape(-1, 3, 3)))
    P = oracle.Params(n=sc.n, dt=sc.dt, gravity=(0, 0, 0), bound=0, kind=kind, p_vol=sc.material.p_vol)
    m = P.c().p_mass
    dx = 1.0 / sc.n
    p0 = m * s.v.sum(1)
    L0 = _angular_momentum(s, m, dx)
    scale_p = m * np.abs(s.v).sum()
    scale_L = m * np.abs(np.cross(s.x.T, s.v.T)).sum()
    for _ in range(3):
        oracle.substep(P, s)
        assert np.abs(m * s.v.sum(1) - p0).max() < 1e-12 * scale_p
        assert np.abs(_angular_momentum(s, m, dx) - L0).max() < 1e-12 * scale_L


def test_free_fall_closed_form():
    """A stress-free block far from the walls falls ballistically: v_k = v0 + k g dt,
    x_k = x0 + k dt v0 + g dt^2 k (k + 1) / 2 (velocity updated before the position)."""
    sc = scenes.cube_scene("ff")
    N = sc.N
    v0 = np.array([0.1, 0.2, -0.3])
    s = oracle.State.from_arrays(sc.x, np.tile(v0[:, None], (1, N)), np.zeros((9, N)), sc.F)
    x0 = s.x.copy()
    P = oracle.Params(n=sc.n, dt=sc.dt, p_vol=sc.material.p_vol)
    g = np.array(P.gravity)
    for k in range(1, 51):
        oracle.substep(P, s)
        vk = v0 + k * g * P.dt
        xk = x0 + k * P.dt * v0[:, None] + (g * P.dt ** 2 * k * (k + 1) / 2)[:, None]
        assert np.abs(s.v - vk[:, None]).max() < 1e-12
        assert np.abs(s.x - xk).max() < 1e-13
    assert np.abs(s.C).max() < 1e-9


def test_clamp_keeps_stencils_inside():
    n = 16
    dx = 1.0 / n
    x = np.array([[2.05 * dx, 0.5, 1 - 2.05 * dx], [0.5] * 3, [0.5] * 3])
    v = np.array([[-100.0, 0.0, 100.0], [0.0] * 3, [0.0] * 3])
    s = oracle.State.from_arrays(x, v, np.zeros((9, 3)), np.tile(np.eye(3).reshape(9, 1), (1, 3)))
    P = oracle.Params(n=n, dt=1e-3, gravity=(0, 0, 0), bound=0, p_vol=1e-3)
    ncl, _, _ = oracle.substep(P, s)
    assert ncl == 2
    assert s.x[0, 0] == 2 * dx and s.x[0, 2] == 1 - 2 * dx


# ---------------------------------------------------------------------------- surrogate window (extension)

def test_surrogate_window_reduces_to_a_substep_and_scales_with_k():
    """With no correction and k = 1 the window is exactly one substep; with k > 1 the grid-to-particle
    pass moves by k times the one-substep displacement with the same v and C (the gathered velocity does
    not depend on the step), and F takes (I + k dt C)."""
    sc = scenes.cube_scene("rand")
    m = sc.material
    P = oracle.Params(n=sc.n, dt=sc.dt, kind=m.kind, E=m.E, nu=m.nu, yield_stress=1e9, rho=m.rho, p_vol=m.p_vol)
    base = oracle.State.from_arrays(sc.x, sc.v, sc.C, sc.F)
    dv = np.zeros((sc.n, sc.n, sc.n, 3))
    box = (0, 0, 0, sc.n, sc.n, sc.n)
    a = oracle.State.from_arrays(sc.x, sc.v, sc.C, sc.F)
    oracle.substep(P, a)
    b = oracle.State.from_arrays(sc.x, sc.v, sc.C, sc.F)
    oracle.surrogate_window(P, b, dv, box, 0.01, 1)
    for f in ("x", "v", "C", "F"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    c = oracle.State.from_arrays(sc.x, sc.v, sc.C, sc.F)
    sums = oracle.surrogate_window(P, c, dv, box, 0.01, 4)
    free = (b.x > 2.0 / sc.n + 1e-9) & (b.x < 1 - 2.0 / sc.n - 1e-9)  # not clamped
    np.testing.assert_allclose((c.x - base.x)[free], 4 * (b.x - base.x)[free], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(c.v, b.v, rtol=0, atol=0)
    np.testing.assert_allclose(c.C, b.C, rtol=0, atol=0)
    C = b.C.T.reshape(-1, 3, 3)
    F0 = base.F.T.reshape(-1, 3, 3)
    Fk = np.einsum("pab,pbc->pac", np.eye(3) + 4 * sc.dt * C, F0)  # no yielding at this yield stress
    np.testing.assert_allclose(c.F.T.reshape(-1, 3, 3), Fk, rtol=1e-12, atol=1e-14)
    # a uniform correction shifts the corrected momentum by M * unit * dv at nodes off the wall band
    d = oracle.State.from_arrays(sc.x, sc.v, sc.C, sc.F)
    dv1 = np.zeros_like(dv)
    dv1[..., 1] = 1.0
    s1 = oracle.surrogate_window(P, d, dv1, box, 0.01, 4)
    assert s1["P_hat"][1] > sums["P_hat"][1]
    np.testing.assert_allclose(s1["P_hat"][[0, 2]], sums["P_hat"][[0, 2]], rtol=1e-12, atol=1e-15)
