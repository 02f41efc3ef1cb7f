/*
 * mpm_oracle.h -- plain FP64 CPU oracle of one MLS-MPM substep.
 *
 * TEST INFRASTRUCTURE ONLY. This code exists to check the CUDA path: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may call it. The
 * product path never links or loads it, and it shares no code, header, table
 * or helper with the CUDA sources.
 *
 * What it computes. The paper (Sec. 3, "Rigid-soft Coupling"; App. D.1,
 * Algorithm 1) names the solver -- MLS-MPM (Hu et al. 2018) in the style of
 * PlasticineLab -- and the order of one soft step: particle to grid (mass,
 * momentum, forces), grid velocity, grid to particle (velocity), particle
 * integration, with rigid-body forces and torques accumulated per body. It does
 * not print the equations; the ones used here are the published methods the
 * paper names:
 *   - quadratic B-spline kernel and APIC/MLS affine transfer (Jiang et al.
 *     2015; Hu et al. 2018), D^-1 = 4/dx^2;
 *   - fixed-corotated Kirchhoff stress tau = 2mu(F-R)F^T + lambda J(J-1) I
 *     (Stomakhin et al. 2012; SIGGRAPH 2016 MPM course);
 *   - von Mises return mapping in Hencky (log) strain for plasticine, the yield
 *     stress of Table 4 entering as ||dev log sigma|| <= tau_Y / (2 mu);
 *   - a weakly compressible fluid as fixed-corotated with mu = 0, lambda = K,
 *     carrying only J, updated by J <- J det(I + dt C);
 *   - grid-node contact against analytic box / capsule signed distances with
 *     Coulomb friction (the grid form of Sec. 3's coupling), the impulse taken
 *     from each node summed per body with its moment about the body's centre of
 *     mass (Algorithm 1, force-torque buffers);
 *   - the particle form of the coupling (Sec. 3's default; Algorithm 1 "compute
 *     penalty forces"): a spring-damper penalty acceleration at every particle
 *     inside a body, with viscous friction capped by Coulomb's law, entering
 *     P2G as a momentum source, its reaction summed per body;
 *   - signed distances of meshes as SDF volumes (Sec. 3), read by trilinear
 *     interpolation with the interpolant's own gradient as the normal.
 *
 * Layout. Particle state is structure-of-arrays in FP64: x[3][np], v[3][np],
 * C[9][np], F[9][np] (3x3 matrices row-major: component r*3+c of particle p at
 * [(r*3+c)*np + p]); a fluid carries J[np] instead of F. The grid is dense, n
 * nodes per axis, node (i,j,k) at (i,j,k)*dx with dx = 1/n, stored as
 * grid[((i*n + j)*n + k)*4 + {0: mass, 1..3: momentum or velocity}].
 *
 * Every loop runs in index order with no blocking, sorting or fusion. The
 * compile flags forbid FMA contraction so that results do not depend on the
 * compiler's choice.
 */
#ifndef MPM_ORACLE_H
#define MPM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PLASTICINE = 0, ORC_FLUID = 1 };
enum { ORC_BOX = 0, ORC_CAPSULE = 1, ORC_SDF_VOLUME = 2 };

typedef struct {
    int n;               /* grid nodes per axis, dx = 1/n */
    double dt;           /* substep length */
    double gravity[3];
    int bound;           /* sticky wall band: nodes with any index < bound or >= n-bound get v = 0 */
    int kind;            /* ORC_PLASTICINE or ORC_FLUID */
    double mu, lambda;   /* Lame parameters; fluid: mu = 0, lambda = bulk modulus */
    double yield_stress; /* plasticine von Mises yield stress */
    double p_vol;        /* initial particle volume V0 */
    double p_mass;       /* particle mass rho * V0 */
} orc_params;

typedef struct {
    int type;            /* ORC_BOX, ORC_CAPSULE or ORC_SDF_VOLUME */
    double half[3];      /* box half extents | capsule (radius, half length along local z, unused) */
    double friction;     /* Coulomb coefficient */
    double pos[3];       /* shape-frame origin at t = 0 (world) */
    double quat[4];      /* shape-frame orientation at t = 0, (w, x, y, z) */
    double lin_vel[3];   /* velocity of the centre of mass (world) */
    double ang_vel[3];   /* angular velocity (world) */
    double com[3];       /* centre of mass at t = 0 (world) */
    /* ORC_SDF_VOLUME only: signed distances sampled on a lattice in the shape frame, sample (i,j,k) at
     * sdf_origin + sdf_h * (i,j,k), stored at sdf[i + res[0] * (j + res[1] * k)]; res[a] >= 2 */
    const double* sdf;
    int res[3];
    double sdf_origin[3];
    double sdf_h;
} orc_collider;

/* Penalty contact at the particles (Sec. 3's default coupling): per unit of particle mass, a normal
 * acceleration stiffness * depth + damping * (approach speed), and a tangential one that opposes the
 * sliding velocity, damping * |v_t| capped by friction * (normal acceleration). */
typedef struct {
    double stiffness;    /* 1/s^2 */
    double damping;      /* 1/s */
} orc_penalty;

/* Lame parameters from Young's modulus and Poisson ratio (Table 4 gives E, nu). */
void orc_lame(double E, double nu, double* mu, double* lambda);

/* 1-D quadratic B-spline N(u); nonzero for |u| < 1.5. */
double orc_bspline(double u);

/* The 27-node stencil of a particle at x: node indices (flattened i*n*n+j*n+k),
 * weights w and offsets dpos = x_node - x_p. Returns the base node per axis in base[3]. */
void orc_stencil(int n, const double x[3], int base[3], int idx[27], double w[27], double dpos[81]);

/* SVD of a 3x3 matrix by one-sided (Hestenes) Jacobi rotations, F = U diag(sig) V^T,
 * det U = det V = +1, |sig| sorted descending, sig[2] < 0 iff det F < 0. Returns sweeps used. */
int orc_svd3(const double F[9], double U[9], double sig[3], double V[9]);

/* Fixed-corotated Kirchhoff stress tau = 2 mu (F - R) F^T + lambda J (J - 1) I, R = polar rotation of F. */
void orc_stress_fixed_corotated(double mu, double lambda, const double F[9], double tau[9]);

/* Von Mises return map in Hencky strain; returns 1 if the state was projected.
 * *clamped is set to 1 if a singular value was raised to 1e-6 before the log. */
int orc_return_map(double mu, double yield_stress, const double Ftr[9], double Fout[9], int* clamped);

/* Pose of a collider at time t after it was set: rotation R (row-major), frame origin p, centre of mass c. */
void orc_collider_pose(const orc_collider* c, double t, double R[9], double p[3], double com[3]);

/* Signed distance of world point x to the collider at time t, with the unit outward normal (world).
 * *ambiguous is set when the normal's branch is within 1e-6 of switching (box face tie, capsule axis). */
double orc_collider_sdf(const orc_collider* c, double t, const double x[3], double normal[3], int* ambiguous);

/* Step A1+A2: clear the grid, then scatter mass and APIC momentum with the stress impulse. */
void orc_p2g(const orc_params* P, int np, const double* x, const double* v, const double* C,
             const double* F, const double* J, double* grid);

/* Step A1+A2 with external particle accelerations accel[3][np] (SoA; NULL = none): the momentum each
 * particle scatters is m_p (v_p + dt a_p) + A_p (x_i - x_p). */
void orc_p2g_forces(const orc_params* P, int np, const double* x, const double* v, const double* C,
                    const double* F, const double* J, const double* accel, double* grid);

/* Trilinear interpolation of a collider's SDF volume at the shape-frame point l: the value and its
 * gradient (shape frame). Returns 0 (and leaves phi, grad untouched) when l lies outside the lattice.
 * *ambiguous is set when l is within 1e-5 cells of a cell face (where the gradient is discontinuous). */
int orc_sdf_volume(const orc_collider* c, const double l[3], double* phi, double grad[3], int* ambiguous);

/* Algorithm 1 "compute penalty forces" and "accumulate equivalent rigid-body forces and torques" at
 * collider time t: accel[3][np] (SoA) receives each particle's penalty acceleration summed over the
 * colliders (index order, each from the particle's velocity at the start of the substep); wrench[6*k]
 * (may be NULL) accumulates per collider the impulse -dt m_p a and its moment about the centre of mass.
 * ambiguous[np] (may be NULL) marks particles whose inside test or normal branch is within 1e-6 of
 * flipping. Returns the number of particle-collider contacts. */
int orc_penalty_accel(const orc_params* P, const orc_penalty* pen, int np, const double* x, const double* v,
                      int ncol, const orc_collider* cols, double t, double* accel, double* wrench,
                      unsigned char* ambiguous);

/* Step A3: v = mv/m + dt g on nodes with m > 0, colliders in index order, then sticky walls.
 * wrench[6*k] accumulates (impulse, angular impulse about the com) per collider; may be NULL.
 * ambiguous (n^3 bytes, may be NULL) marks nodes whose inside test or normal branch is within 1e-6
 * of flipping. Nodes with m == 0 keep m = 0 and get v = 0. */
void orc_grid_update(const orc_params* P, double* grid, int ncol, const orc_collider* cols, double t,
                     double* wrench, unsigned char* ambiguous);

/* Steps A4+A5: gather v and C, advect and clamp x to [2dx, 1-2dx], update F (return map) or J.
 * Returns the number of clamped coordinates; *sv_clamped counts singular values raised to 1e-6. */
int orc_g2p(const orc_params* P, int np, const double* grid, double* x, double* v, double* C,
            double* F, double* J, int* sv_clamped);

/* One full substep at collider time t (A1..A5). grid is caller scratch of 4*n^3 doubles.
 * Returns the number of clamped coordinates. */
int orc_substep(const orc_params* P, int np, double* x, double* v, double* C, double* F, double* J,
                int ncol, const orc_collider* cols, double t, double* wrench, double* grid,
                unsigned char* ambiguous);

/* One full substep with the particle form of the contact (Algorithm 1 in order): penalty
 * accelerations and body impulses at collider time t, P2G with those forces, the grid update without
 * colliders (gravity, sticky walls), G2P. accel is caller scratch of 3*np doubles; ambiguous (np bytes,
 * may be NULL) as orc_penalty_accel. Returns the number of clamped coordinates. */
int orc_substep_penalty(const orc_params* P, const orc_penalty* pen, int np, double* x, double* v, double* C,
                        double* F, double* J, int ncol, const orc_collider* cols, double t, double* wrench,
                        double* grid, double* accel, unsigned char* ambiguous);

#ifdef __cplusplus
}
#endif
#endif
