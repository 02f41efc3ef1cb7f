/*
 * mpm_oracle.c -- plain FP64 CPU oracle of one MLS-MPM substep.
 *
 * TEST INFRASTRUCTURE ONLY (see mpm_oracle.h): called by the tests, the smoke
 * check and the benchmark's CPU-baseline leg, never by the product path.
 *
 * Each function names the step of the paper's soft step (Algorithm 1, App. D.1)
 * it carries out and the published method the paper points to for its
 * equations (Sec. 3: MLS-MPM as in PlasticineLab). Loops are in index order,
 * without blocking, sorting or fusion, so each step can be read against its
 * definition.
 */
#include "mpm_oracle.h"

#include <math.h>
#include <string.h>

/* ---------------------------------------------------------------- 3x3 helpers */

static void mat_mul(const double A[9], const double B[9], double out[9]) {
    double r[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * B[k * 3 + j];
            r[i * 3 + j] = s;
        }
    memcpy(out, r, sizeof r);
}

/* A * B^T */
static void mat_mul_bt(const double A[9], const double B[9], double out[9]) {
    double r[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i * 3 + k] * B[j * 3 + k];
            r[i * 3 + j] = s;
        }
    memcpy(out, r, sizeof r);
}

static double mat_det(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static void cross3(const double a[3], const double b[3], double out[3]) {
    double r0 = a[1] * b[2] - a[2] * b[1];
    double r1 = a[2] * b[0] - a[0] * b[2];
    double r2 = a[0] * b[1] - a[1] * b[0];
    out[0] = r0; out[1] = r1; out[2] = r2;
}

/* ---------------------------------------------------------------- material constants */

/* Lame parameters of an isotropic solid from E and nu (Table 4 lists E and nu). */
void orc_lame(double E, double nu, double* mu, double* lambda) {
    *mu = E / (2.0 * (1.0 + nu));
    *lambda = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* ---------------------------------------------------------------- kernel (A2, A4) */

/* Quadratic B-spline (Jiang et al. 2015, Hu et al. 2018): the MLS-MPM weight function. */
double orc_bspline(double u) {
    u = fabs(u);
    if (u < 0.5) return 0.75 - u * u;
    if (u < 1.5) return 0.5 * (1.5 - u) * (1.5 - u);
    return 0.0;
}

/* Base node and fractional offset of a particle along one axis, then the three weights.
 * base = floor(x/dx - 0.5) puts x/dx - base in [0.5, 1.5), so the particle's distances in cells to
 * nodes base, base+1, base+2 are fx, fx-1, fx-2. */
static void axis_weights(double xdx, int* base, double* fx, double w[3]) {
    int b = (int)floor(xdx - 0.5);
    double f = xdx - (double)b;
    *base = b;
    *fx = f;
    w[0] = orc_bspline(f);
    w[1] = orc_bspline(f - 1.0);
    w[2] = orc_bspline(f - 2.0);
}

void orc_stencil(int n, const double x[3], int base[3], int idx[27], double w[27], double dpos[81]) {
    double dx = 1.0 / n;
    double wa[3][3], fa[3];
    for (int a = 0; a < 3; ++a) axis_weights(x[a] * n, &base[a], &fa[a], wa[a]);
    int q = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k, ++q) {
                idx[q] = ((base[0] + i) * n + (base[1] + j)) * n + (base[2] + k);
                w[q] = wa[0][i] * wa[1][j] * wa[2][k];
                dpos[q * 3 + 0] = ((double)i - fa[0]) * dx;
                dpos[q * 3 + 1] = ((double)j - fa[1]) * dx;
                dpos[q * 3 + 2] = ((double)k - fa[2]) * dx;
            }
}

/* ---------------------------------------------------------------- SVD (A1, A5) */

/* One-sided Jacobi SVD (Hestenes 1958; Golub & Van Loan, Sec. 8.6.3): rotate column pairs of
 * W = F V until all columns are mutually orthogonal; then sig_i = |W e_i|, U e_i = W e_i / sig_i. */
int orc_svd3(const double F[9], double U[9], double sig[3], double V[9]) {
    double W[9];
    memcpy(W, F, sizeof W);
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    static const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    int sweep;
    for (sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int pi = 0; pi < 3; ++pi) {
            int p = pairs[pi][0], q = pairs[pi][1];
            double alpha = 0.0, beta = 0.0, gamma = 0.0;
            for (int r = 0; r < 3; ++r) {
                alpha += W[r * 3 + p] * W[r * 3 + p];
                beta += W[r * 3 + q] * W[r * 3 + q];
                gamma += W[r * 3 + p] * W[r * 3 + q];
            }
            if (fabs(gamma) <= 1e-15 * sqrt(alpha * beta) || gamma == 0.0) continue;
            rotated = 1;
            /* angle that makes the new columns p, q orthogonal: t = tan(theta) is the smaller root of
             * t^2 + 2 zeta t - 1 = 0 with zeta = (beta - alpha) / (2 gamma) */
            double zeta = (beta - alpha) / (2.0 * gamma);
            double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double c = 1.0 / sqrt(1.0 + t * t);
            double s = c * t;
            for (int r = 0; r < 3; ++r) {
                double wp = W[r * 3 + p], wq = W[r * 3 + q];
                W[r * 3 + p] = c * wp - s * wq;
                W[r * 3 + q] = s * wp + c * wq;
                double vp = V[r * 3 + p], vq = V[r * 3 + q];
                V[r * 3 + p] = c * vp - s * vq;
                V[r * 3 + q] = s * vp + c * vq;
            }
        }
        if (!rotated) break;
    }
    double nrm[3];
    for (int c = 0; c < 3; ++c)
        nrm[c] = sqrt(W[c] * W[c] + W[3 + c] * W[3 + c] + W[6 + c] * W[6 + c]);
    /* sort columns by norm, descending (selection sort on three entries) */
    int order[3] = {0, 1, 2};
    for (int a = 0; a < 2; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (nrm[order[b]] > nrm[order[a]]) { int tmp = order[a]; order[a] = order[b]; order[b] = tmp; }
    double Ws[9], Vs[9];
    for (int c = 0; c < 3; ++c) {
        sig[c] = nrm[order[c]];
        for (int r = 0; r < 3; ++r) {
            Ws[r * 3 + c] = W[r * 3 + order[c]];
            Vs[r * 3 + c] = V[r * 3 + order[c]];
        }
    }
    memcpy(V, Vs, sizeof Vs);
    /* U columns; a zero column (rank-deficient F) is completed to an orthonormal frame */
    double scale = sig[0] > 0.0 ? sig[0] : 1.0;
    for (int c = 0; c < 3; ++c) {
        if (sig[c] > 1e-300 && sig[c] > 1e-14 * scale) {
            for (int r = 0; r < 3; ++r) U[r * 3 + c] = Ws[r * 3 + c] / sig[c];
        } else {
            double u0[3], u1[3], e[3];
            if (c == 0) { U[0] = 1.0; U[3] = 0.0; U[6] = 0.0; continue; }
            u0[0] = U[0]; u0[1] = U[3]; u0[2] = U[6];
            if (c == 1) {
                /* any unit vector orthogonal to u0 */
                e[0] = fabs(u0[0]) < 0.9 ? 1.0 : 0.0; e[1] = fabs(u0[0]) < 0.9 ? 0.0 : 1.0; e[2] = 0.0;
                cross3(u0, e, u1);
                double l = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
                U[1] = u1[0] / l; U[4] = u1[1] / l; U[7] = u1[2] / l;
            } else {
                u1[0] = U[1]; u1[1] = U[4]; u1[2] = U[7];
                cross3(u0, u1, e);
                U[2] = e[0]; U[5] = e[1]; U[8] = e[2];
            }
            sig[c] = 0.0;
        }
    }
    /* rotations only: det V = +1 (flip last columns of V and U together, F V = U S unchanged),
     * then det U = +1 by flipping the last column of U and the sign of the smallest singular value */
    if (mat_det(V) < 0.0) {
        for (int r = 0; r < 3; ++r) { V[r * 3 + 2] = -V[r * 3 + 2]; U[r * 3 + 2] = -U[r * 3 + 2]; }
    }
    if (mat_det(U) < 0.0) {
        for (int r = 0; r < 3; ++r) U[r * 3 + 2] = -U[r * 3 + 2];
        sig[2] = -sig[2];
    }
    return sweep;
}

/* ---------------------------------------------------------------- constitutive model (A1) */

/* Fixed-corotated Kirchhoff stress (Stomakhin et al. 2012): tau = P F^T with
 * P = 2 mu (F - R) + lambda (J - 1) J F^-T, i.e. tau = 2 mu (F - R) F^T + lambda J (J - 1) I. */
void orc_stress_fixed_corotated(double mu, double lambda, const double F[9], double tau[9]) {
    double U[9], S[3], V[9], R[9], FmR[9];
    orc_svd3(F, U, S, V);
    mat_mul_bt(U, V, R);
    double J = mat_det(F);
    for (int i = 0; i < 9; ++i) FmR[i] = F[i] - R[i];
    mat_mul_bt(FmR, F, tau);
    for (int i = 0; i < 9; ++i) tau[i] *= 2.0 * mu;
    double vol = lambda * J * (J - 1.0);
    tau[0] += vol; tau[4] += vol; tau[8] += vol;
}

/* Von Mises plasticity in Hencky strain (as in PlasticineLab): eps = log sig, project the deviatoric
 * part of eps back onto the sphere ||dev eps|| = tau_Y / (2 mu) when it lies outside; the trace of eps
 * (volume) is kept. F = U exp(eps) V^T. Inside the yield surface F is returned unchanged. */
int orc_return_map(double mu, double yield_stress, const double Ftr[9], double Fout[9], int* clamped) {
    double U[9], S[3], V[9];
    orc_svd3(Ftr, U, S, V);
    int clamp = 0;
    double eps[3];
    for (int i = 0; i < 3; ++i) {
        double s = S[i];
        if (s < 1e-6) { s = 1e-6; clamp = 1; }
        eps[i] = log(s);
    }
    double tr = eps[0] + eps[1] + eps[2];
    double dev[3] = {eps[0] - tr / 3.0, eps[1] - tr / 3.0, eps[2] - tr / 3.0};
    double dnorm = sqrt(dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]);
    double dgamma = dnorm - yield_stress / (2.0 * mu);
    if (clamped) *clamped = clamp;
    if (dgamma <= 0.0 && !clamp) {
        memcpy(Fout, Ftr, 9 * sizeof(double));
        return 0;
    }
    if (dgamma > 0.0)
        for (int i = 0; i < 3; ++i) eps[i] -= dgamma * dev[i] / dnorm;
    double US[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) US[r * 3 + c] = U[r * 3 + c] * exp(eps[c]);
    mat_mul_bt(US, V, Fout);
    return dgamma > 0.0;
}

/* ---------------------------------------------------------------- colliders (A3) */

static void quat_to_mat(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double l = sqrt(w * w + x * x + y * y + z * z);
    w /= l; x /= l; y /= l; z /= l;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Rigid motion with constant velocities since the pose was set (Algorithm 1 copies poses and velocities
 * once per rigid step; between copies the body moves kinematically): the centre of mass translates with
 * lin_vel and the body turns about it by the rotation vector ang_vel * t (Rodrigues' formula). */
void orc_collider_pose(const orc_collider* c, double t, double R[9], double p[3], double com[3]) {
    double R0[9], Q[9];
    quat_to_mat(c->quat, R0);
    double th[3] = {c->ang_vel[0] * t, c->ang_vel[1] * t, c->ang_vel[2] * t};
    double a = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
    for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
    if (a > 0.0) {
        double k[3] = {th[0] / a, th[1] / a, th[2] / a};
        double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
        double K2[9];
        mat_mul(K, K, K2);
        double sa = sin(a), ca = 1.0 - cos(a);
        for (int i = 0; i < 9; ++i) Q[i] += sa * K[i] + ca * K2[i];
    }
    mat_mul(Q, R0, R);
    for (int i = 0; i < 3; ++i) com[i] = c->com[i] + t * c->lin_vel[i];
    double d[3] = {c->pos[0] - c->com[0], c->pos[1] - c->com[1], c->pos[2] - c->com[2]};
    for (int i = 0; i < 3; ++i) p[i] = com[i] + Q[i * 3] * d[0] + Q[i * 3 + 1] * d[1] + Q[i * 3 + 2] * d[2];
}

/* SDF volume of a mesh (Sec. 3 stores one per mesh as a 3-D texture): the trilinear interpolant of the
 * lattice samples. In lattice units u = (l - origin) / h the point lies in cell c = floor(u) (the last
 * cell on the upper faces) at fraction f = u - c; the value is the sum over the cell's 8 corners of
 * prod_a (f_a or 1 - f_a) times the sample, and the gradient is the interpolant's derivative: along
 * axis a, the blend by the other two axes' weights of the four edge differences along a, divided by h. */
int orc_sdf_volume(const orc_collider* c, const double l[3], double* phi, double grad[3], int* ambiguous) {
    int cell[3];
    double f[3];
    int amb = 0;
    for (int a = 0; a < 3; ++a) {
        double u = (l[a] - c->sdf_origin[a]) / c->sdf_h;
        if (!(u >= 0.0) || u > (double)(c->res[a] - 1)) return 0;
        int ci = (int)floor(u);
        if (ci > c->res[a] - 2) ci = c->res[a] - 2;
        cell[a] = ci;
        f[a] = u - (double)ci;
        if (f[a] < 1e-5 || f[a] > 1.0 - 1e-5) amb = 1;
    }
    double smp[2][2][2]; /* [di][dj][dk] */
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk)
                smp[di][dj][dk] = c->sdf[(cell[0] + di) +
                                         (size_t)c->res[0] * ((cell[1] + dj) + (size_t)c->res[1] * (cell[2] + dk))];
    double val = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk) {
                double wi = di ? f[0] : 1.0 - f[0], wj = dj ? f[1] : 1.0 - f[1], wk = dk ? f[2] : 1.0 - f[2];
                val += wi * wj * wk * smp[di][dj][dk];
            }
    /* the derivative along each axis: the bilinear blend of the cell's four edge differences */
    for (int e = 0; e < 2; ++e)
        for (int o = 0; o < 2; ++o) {
            double w1 = e ? f[1] : 1.0 - f[1], w2 = o ? f[2] : 1.0 - f[2];
            g[0] += w1 * w2 * (smp[1][e][o] - smp[0][e][o]);
            double w0 = e ? f[0] : 1.0 - f[0];
            g[1] += w0 * w2 * (smp[e][1][o] - smp[e][0][o]);
            double w1b = o ? f[1] : 1.0 - f[1];
            g[2] += w0 * w1b * (smp[e][o][1] - smp[e][o][0]);
        }
    *phi = val;
    for (int a = 0; a < 3; ++a) grad[a] = g[a] / c->sdf_h;
    if (ambiguous) *ambiguous = amb;
    return 1;
}

/* Analytic signed distances of the primitive shapes of Sec. 3 (box, capsule) and SDF volumes, in the
 * shape frame. A point outside an SDF volume's lattice is outside the body (phi = +1e30, no normal). */
double orc_collider_sdf(const orc_collider* c, double t, const double x[3], double normal[3], int* ambiguous) {
    double R[9], p[3], com[3];
    orc_collider_pose(c, t, R, p, com);
    double d[3] = {x[0] - p[0], x[1] - p[1], x[2] - p[2]};
    double l[3];
    for (int i = 0; i < 3; ++i) l[i] = R[i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2]; /* R^T d */
    double nl[3] = {0.0, 0.0, 0.0};
    double phi;
    int amb = 0;
    if (c->type == ORC_BOX) {
        double q[3], qo[3];
        for (int i = 0; i < 3; ++i) {
            q[i] = fabs(l[i]) - c->half[i];
            qo[i] = q[i] > 0.0 ? q[i] : 0.0;
        }
        double outside = sqrt(qo[0] * qo[0] + qo[1] * qo[1] + qo[2] * qo[2]);
        int am = 0;
        if (q[1] > q[am]) am = 1;
        if (q[2] > q[am]) am = 2;
        double qmax = q[am];
        phi = outside + (qmax < 0.0 ? qmax : 0.0);
        if (outside > 0.0) {
            for (int i = 0; i < 3; ++i) nl[i] = (l[i] >= 0.0 ? 1.0 : -1.0) * qo[i] / outside;
        } else {
            nl[am] = l[am] >= 0.0 ? 1.0 : -1.0;
            /* inside: the nearest face switches where two q's tie */
            for (int i = 0; i < 3; ++i)
                if (i != am && fabs(q[i] - qmax) < 1e-6) amb = 1;
            if (fabs(l[am]) < 1e-6) amb = 1;
        }
    } else if (c->type == ORC_SDF_VOLUME) {
        double g[3];
        if (!orc_sdf_volume(c, l, &phi, g, &amb)) {
            phi = 1e30;
        } else {
            double gl = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            if (gl > 0.0)
                for (int i = 0; i < 3; ++i) nl[i] = g[i] / gl;
        }
    } else {
        double r = c->half[0], h = c->half[1];
        double cz = l[2] < -h ? -h : (l[2] > h ? h : l[2]);
        double e[3] = {l[0], l[1], l[2] - cz};
        double el = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        phi = el - r;
        if (el > 0.0) {
            for (int i = 0; i < 3; ++i) nl[i] = e[i] / el;
        } else {
            nl[0] = 1.0;
        }
        if (el < 1e-6) amb = 1;
    }
    for (int i = 0; i < 3; ++i) normal[i] = R[i * 3] * nl[0] + R[i * 3 + 1] * nl[1] + R[i * 3 + 2] * nl[2];
    if (fabs(phi) < 1e-6) amb = 1;
    if (ambiguous) *ambiguous = amb;
    return phi;
}

/* ---------------------------------------------------------------- P2G (A1, A2) */

/* Algorithm 1, "MPM particle to grid (mass, momentum, forces)": with the MLS-MPM fused force term
 * (Hu et al. 2018), each particle adds to the 27 nodes of its stencil
 *   m_i  += w_ip m_p
 *   mv_i += w_ip (m_p v_p + A_p (x_i - x_p)),   A_p = m_p C_p - dt V0 (4/dx^2) tau_p. */
void orc_p2g(const orc_params* P, int np, const double* x, const double* v, const double* C,
             const double* F, const double* J, double* grid) {
    orc_p2g_forces(P, np, x, v, C, F, J, 0, grid);
}

/* The same transfer with Algorithm 1's "forces": an external acceleration a_p adds the impulse
 * dt m_p a_p to the momentum the particle scatters. */
void orc_p2g_forces(const orc_params* P, int np, const double* x, const double* v, const double* C,
                    const double* F, const double* J, const double* accel, double* grid) {
    int n = P->n;
    double dx = 1.0 / n;
    size_t nn = (size_t)n * n * n;
    memset(grid, 0, nn * 4 * sizeof(double));
    double Dinv = 4.0 / (dx * dx);
    for (int p = 0; p < np; ++p) {
        double xp[3] = {x[p], x[np + p], x[2 * np + p]};
        double vp[3] = {v[p], v[np + p], v[2 * np + p]};
        if (accel)
            for (int a = 0; a < 3; ++a) vp[a] += P->dt * accel[(size_t)a * np + p];
        double Cp[9], tau[9], A[9];
        for (int i = 0; i < 9; ++i) Cp[i] = C[(size_t)i * np + p];
        if (P->kind == ORC_PLASTICINE) {
            double Fp[9];
            for (int i = 0; i < 9; ++i) Fp[i] = F[(size_t)i * np + p];
            orc_stress_fixed_corotated(P->mu, P->lambda, Fp, tau);
        } else {
            double Jp = J[p];
            memset(tau, 0, sizeof tau);
            tau[0] = tau[4] = tau[8] = P->lambda * Jp * (Jp - 1.0);
        }
        for (int i = 0; i < 9; ++i) A[i] = P->p_mass * Cp[i] - P->dt * P->p_vol * Dinv * tau[i];
        int base[3], idx[27];
        double w[27], dpos[81];
        orc_stencil(n, xp, base, idx, w, dpos);
        for (int q = 0; q < 27; ++q) {
            double* g = grid + (size_t)idx[q] * 4;
            const double* d = dpos + q * 3;
            g[0] += w[q] * P->p_mass;
            for (int a = 0; a < 3; ++a) {
                double Ad = A[a * 3] * d[0] + A[a * 3 + 1] * d[1] + A[a * 3 + 2] * d[2];
                g[1 + a] += w[q] * (P->p_mass * vp[a] + Ad);
            }
        }
    }
}

/* ---------------------------------------------------------------- grid update (A3) */

/* Algorithm 1, "MPM grid compute velocity", with the grid form of the contact of Sec. 3: for each
 * node with mass, v = mv/m + dt g; then every collider in index order: if the node is inside
 * (phi < 0) and approaching (v_n < 0 relative to the body's velocity there) the relative velocity is
 * projected by Coulomb friction -- stick (v_r = 0) when |v_t| <= -mu v_n, else slip
 * v_r = v_t (1 + mu v_n / |v_t|); the momentum removed, m (v_before - v_after), is the impulse on the
 * body (Algorithm 1's force-torque buffers), with its moment about the centre of mass. Finally the
 * sticky wall band sets v = 0. */
void orc_grid_update(const orc_params* P, double* grid, int ncol, const orc_collider* cols, double t,
                     double* wrench, unsigned char* ambiguous) {
    int n = P->n;
    double dx = 1.0 / n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                size_t node = ((size_t)i * n + j) * n + k;
                double* g = grid + node * 4;
                if (ambiguous) ambiguous[node] = 0;
                if (!(g[0] > 0.0)) {
                    g[1] = g[2] = g[3] = 0.0;
                    continue;
                }
                double m = g[0];
                double v[3];
                for (int a = 0; a < 3; ++a) v[a] = g[1 + a] / m + P->dt * P->gravity[a];
                double xi[3] = {i * dx, j * dx, k * dx};
                for (int c = 0; c < ncol; ++c) {
                    double nrm[3];
                    int amb = 0;
                    double phi = orc_collider_sdf(&cols[c], t, xi, nrm, &amb);
                    if (amb && ambiguous) ambiguous[node] = 1;
                    if (!(phi < 0.0)) continue;
                    double R[9], p[3], com[3];
                    orc_collider_pose(&cols[c], t, R, p, com);
                    double rel[3] = {xi[0] - com[0], xi[1] - com[1], xi[2] - com[2]};
                    double wxr[3];
                    cross3(cols[c].ang_vel, rel, wxr);
                    double vc[3], vr[3];
                    for (int a = 0; a < 3; ++a) {
                        vc[a] = cols[c].lin_vel[a] + wxr[a];
                        vr[a] = v[a] - vc[a];
                    }
                    double vn = vr[0] * nrm[0] + vr[1] * nrm[1] + vr[2] * nrm[2];
                    if (!(vn < 0.0)) continue;
                    double vt[3];
                    for (int a = 0; a < 3; ++a) vt[a] = vr[a] - vn * nrm[a];
                    double tn = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
                    double mu = cols[c].friction;
                    double vnew[3];
                    if (tn <= -mu * vn) {
                        for (int a = 0; a < 3; ++a) vnew[a] = vc[a];
                    } else {
                        double s = 1.0 + mu * vn / tn;
                        for (int a = 0; a < 3; ++a) vnew[a] = vc[a] + vt[a] * s;
                    }
                    if (wrench) {
                        double imp[3], tq[3];
                        for (int a = 0; a < 3; ++a) imp[a] = m * (v[a] - vnew[a]);
                        cross3(rel, imp, tq);
                        for (int a = 0; a < 3; ++a) {
                            wrench[c * 6 + a] += imp[a];
                            wrench[c * 6 + 3 + a] += tq[a];
                        }
                    }
                    for (int a = 0; a < 3; ++a) v[a] = vnew[a];
                }
                int b = P->bound;
                if (i < b || j < b || k < b || i >= n - b || j >= n - b || k >= n - b) v[0] = v[1] = v[2] = 0.0;
                for (int a = 0; a < 3; ++a) g[1 + a] = v[a];
            }
}

/* ---------------------------------------------------------------- G2P + integration (A4, A5) */

/* Algorithm 1, "MPM grid to particle (velocity)" and "integrate MPM particles": APIC gather
 * v_p = sum w v_i, C_p = (4/dx^2) sum w v_i (x_i - x_p)^T; advect x_p += dt v_p and clamp it to
 * [2dx, 1-2dx] so every stencil stays inside the grid; F <- (I + dt C) F then the plastic return map,
 * or for the fluid J <- J det(I + dt C). */
int orc_g2p(const orc_params* P, int np, const double* grid, double* x, double* v, double* C,
            double* F, double* J, int* sv_clamped) {
    int n = P->n;
    double dx = 1.0 / n;
    double Dinv = 4.0 / (dx * dx);
    double lo = 2.0 * dx, hi = 1.0 - 2.0 * dx;
    int nclamp = 0, nsv = 0;
    for (int p = 0; p < np; ++p) {
        double xp[3] = {x[p], x[np + p], x[2 * np + p]};
        int base[3], idx[27];
        double w[27], dpos[81];
        orc_stencil(n, xp, base, idx, w, dpos);
        double vn[3] = {0, 0, 0}, B[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int q = 0; q < 27; ++q) {
            const double* g = grid + (size_t)idx[q] * 4;
            for (int a = 0; a < 3; ++a) {
                vn[a] += w[q] * g[1 + a];
                for (int b = 0; b < 3; ++b) B[a * 3 + b] += w[q] * g[1 + a] * dpos[q * 3 + b];
            }
        }
        double Cn[9];
        for (int i = 0; i < 9; ++i) Cn[i] = Dinv * B[i];
        for (int a = 0; a < 3; ++a) {
            double xn = xp[a] + P->dt * vn[a];
            if (xn < lo) { xn = lo; ++nclamp; }
            if (xn > hi) { xn = hi; ++nclamp; }
            x[(size_t)a * np + p] = xn;
            v[(size_t)a * np + p] = vn[a];
        }
        for (int i = 0; i < 9; ++i) C[(size_t)i * np + p] = Cn[i];
        double G[9];
        for (int i = 0; i < 9; ++i) G[i] = ((i % 4 == 0) ? 1.0 : 0.0) + P->dt * Cn[i];
        if (P->kind == ORC_PLASTICINE) {
            double Fp[9], Ftr[9], Fnew[9];
            for (int i = 0; i < 9; ++i) Fp[i] = F[(size_t)i * np + p];
            mat_mul(G, Fp, Ftr);
            int cl = 0;
            orc_return_map(P->mu, P->yield_stress, Ftr, Fnew, &cl);
            nsv += cl;
            for (int i = 0; i < 9; ++i) F[(size_t)i * np + p] = Fnew[i];
        } else {
            J[p] = J[p] * mat_det(G);
        }
    }
    if (sv_clamped) *sv_clamped = nsv;
    return nclamp;
}

int orc_substep(const orc_params* P, int np, double* x, double* v, double* C, double* F, double* J,
                int ncol, const orc_collider* cols, double t, double* wrench, double* grid,
                unsigned char* ambiguous) {
    orc_p2g(P, np, x, v, C, F, J, grid);
    orc_grid_update(P, grid, ncol, cols, t, wrench, ambiguous);
    return orc_g2p(P, np, grid, x, v, C, F, J, 0);
}

/* ---------------------------------------------------------------- particle contact (Sec. 3) */

/* Algorithm 1 "compute penalty forces" and "accumulate equivalent rigid-body forces and torques".
 * For a particle inside body c (phi < 0), with the body's velocity at the particle
 * v_c = v_lin + w x (x_p - com), relative velocity v_r = v_p - v_c, its normal part v_n = v_r . n and
 * tangential part v_t = v_r - v_n n, the penalty acceleration is
 *   a = a_n n - min(damping |v_t|, friction a_n) v_t / |v_t|,
 *   a_n = stiffness (-phi) + damping max(-v_n, 0)  (>= 0: a spring on the depth, a damper on approach).
 * The body receives the opposite impulse, -dt m_p a, and its moment about the centre of mass. */
int orc_penalty_accel(const orc_params* P, const orc_penalty* pen, int np, const double* x, const double* v,
                      int ncol, const orc_collider* cols, double t, double* accel, double* wrench,
                      unsigned char* ambiguous) {
    int contacts = 0;
    for (int p = 0; p < np; ++p) {
        double xp[3] = {x[p], x[np + p], x[2 * np + p]};
        double vp[3] = {v[p], v[np + p], v[2 * np + p]};
        double acc[3] = {0.0, 0.0, 0.0};
        if (ambiguous) ambiguous[p] = 0;
        for (int c = 0; c < ncol; ++c) {
            double nrm[3];
            int amb = 0;
            double phi = orc_collider_sdf(&cols[c], t, xp, nrm, &amb);
            if (amb && ambiguous) ambiguous[p] = 1;
            if (!(phi < 0.0)) continue;
            ++contacts;
            double R[9], org[3], com[3];
            orc_collider_pose(&cols[c], t, R, org, com);
            double rel[3] = {xp[0] - com[0], xp[1] - com[1], xp[2] - com[2]};
            double wxr[3];
            cross3(cols[c].ang_vel, rel, wxr);
            double vr[3];
            for (int a = 0; a < 3; ++a) vr[a] = vp[a] - (cols[c].lin_vel[a] + wxr[a]);
            double vn = vr[0] * nrm[0] + vr[1] * nrm[1] + vr[2] * nrm[2];
            double an = pen->stiffness * (-phi) + pen->damping * (vn < 0.0 ? -vn : 0.0);
            double vt[3];
            for (int a = 0; a < 3; ++a) vt[a] = vr[a] - vn * nrm[a];
            double tn = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
            double ft = 0.0; /* tangential acceleration per unit sliding speed */
            if (tn > 0.0) {
                double cap = cols[c].friction * an;
                double visc = pen->damping * tn;
                ft = (visc < cap ? visc : cap) / tn;
            }
            double a_c[3];
            for (int a = 0; a < 3; ++a) {
                a_c[a] = an * nrm[a] - ft * vt[a];
                acc[a] += a_c[a];
            }
            if (wrench) {
                double imp[3], tq[3];
                for (int a = 0; a < 3; ++a) imp[a] = -P->dt * P->p_mass * a_c[a];
                cross3(rel, imp, tq);
                for (int a = 0; a < 3; ++a) {
                    wrench[c * 6 + a] += imp[a];
                    wrench[c * 6 + 3 + a] += tq[a];
                }
            }
        }
        for (int a = 0; a < 3; ++a) accel[(size_t)a * np + p] = acc[a];
    }
    return contacts;
}

int orc_substep_penalty(const orc_params* P, const orc_penalty* pen, int np, double* x, double* v, double* C,
                        double* F, double* J, int ncol, const orc_collider* cols, double t, double* wrench,
                        double* grid, double* accel, unsigned char* ambiguous) {
    orc_penalty_accel(P, pen, np, x, v, ncol, cols, t, accel, wrench, ambiguous);
    orc_p2g_forces(P, np, x, v, C, F, J, accel, grid);
    orc_grid_update(P, grid, 0, cols, t, 0, 0);
    return orc_g2p(P, np, grid, x, v, C, F, J, 0);
}
