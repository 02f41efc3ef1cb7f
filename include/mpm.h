/*
 * mpm.h -- C-ABI of the GB300 MLS-MPM soft-body substep library (libmpm_gb300.so).
 *
 * The calls follow the coupling loop of the paper's soft-body engine (Sec. 3,
 * "Rigid-soft Coupling"; App. D.1, Algorithm 1):
 *   - collision shapes are copied into the soft scene once       -> mpm_set_shapes
 *   - after every rigid step, body poses and velocities are copied
 *     in and the force-torque buffers are reset                   -> mpm_set_colliders
 *   - soft steps: particle to grid (mass, momentum, forces), grid
 *     velocity, grid to particle, particle integration             -> mpm_substep
 *   - accumulated body forces / torques are read back              -> mpm_read_wrench
 *   - particles are handed to a consumer by one GPU-GPU copy       -> mpm_read_state
 *     (App. D.2), or to the host.
 * Contact comes in the two forms Sec. 3 describes (mpm_set_contact): the grid
 * form (signed distances evaluated on grid nodes, as in PlasticineLab, with a
 * Coulomb friction projection; the default) and the particle form the paper
 * prefers (signed distances evaluated at the particles, penalty forces entering
 * the particle-to-grid transfer). Bodies are boxes, capsules or SDF volumes
 * (Sec. 3: meshes become signed-distance volumes).
 *
 * Conventions
 *   - Everything is FP32 except the wrench accumulators (FP64).
 *   - Particle arrays are structure-of-arrays with the particle index fastest:
 *     x[3][n], v[3][n], C[9][n], F[9][n]; 3x3 matrices row-major, so entry (r,c)
 *     of particle p is at [(r*3 + c)*n + p].
 *   - The domain is the unit cube; the grid has cfg.n nodes per axis, node i at
 *     i*dx with dx = 1/n. Particles are kept inside [2dx, 1-2dx] (clamped, with
 *     a status flag), so every quadratic B-spline stencil lies in the grid.
 *   - Memory: the caller owns all device memory. mpm_create receives one device
 *     workspace of mpm_workspace_size() bytes (256-byte aligned, e.g. a torch
 *     tensor) that must outlive the handle; the library allocates no device
 *     memory and owns only the small host-side handle.
 *   - Streams: every call takes a cudaStream_t as void* (NULL = legacy default
 *     stream) and only enqueues work on it, except those documented as
 *     synchronizing. Calls on one handle must be issued from one host thread at a
 *     time and on one stream (or streams the caller orders).
 *   - Errors: each call returns an mpm_status; argument errors are detected on
 *     the host before anything is enqueued. Conditions found on the device
 *     (clamping, non-finite values) set sticky flag bits read by
 *     mpm_get_status; the kernels never trap or abort.
 */
#ifndef MPM_GB300_H
#define MPM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPM_MAX_COLLIDERS 32

typedef struct mpm_sim mpm_sim; /* opaque handle, host memory owned by the library */

typedef enum {
    MPM_OK = 0,
    MPM_ERR_INVALID_ARG = 1, /* a pointer, size or enum is out of range; nothing was enqueued */
    MPM_ERR_CUDA = 2,        /* a CUDA runtime call failed; the message is kept for mpm_last_error */
    MPM_ERR_WORKSPACE = 3,   /* workspace NULL, misaligned or smaller than mpm_workspace_size */
    MPM_ERR_CAPACITY = 4     /* more particles or colliders than the handle was created for */
} mpm_status;

/* Sticky device flag bits (mpm_get_status). None of them stops the simulation. */
#define MPM_FLAG_CLAMPED 0x1u    /* a particle coordinate was clamped to [2dx, 1-2dx] */
#define MPM_FLAG_NONFINITE 0x2u  /* a non-finite coordinate or velocity was met (position clamped) */
#define MPM_FLAG_SV_CLAMPED 0x4u /* a singular value of F was raised to 1e-6 before its logarithm */
#define MPM_FLAG_FAR_MOVE 0x8u   /* a particle moved >= 1 cell in one substep (served by a slower path) */

enum { MPM_PLASTICINE = 0, MPM_FLUID = 1 };
enum { MPM_BOX = 0, MPM_CAPSULE = 1, MPM_SDF_VOLUME = 2 };
enum { MPM_CONTACT_GRID = 0, MPM_CONTACT_PARTICLE = 1 };

typedef struct {
    int n;              /* grid nodes per axis: a multiple of 4 in [8, 256]; dx = 1/n */
    float dt;           /* substep length (s) */
    float gravity[3];   /* m/s^2 */
    int bound;          /* sticky wall band: nodes with an index < bound or >= n-bound get v = 0 */
    int max_particles;  /* capacity, >= 1 */
    int max_colliders;  /* capacity, 0..MPM_MAX_COLLIDERS */
} mpm_config;

typedef struct {
    int kind;           /* MPM_PLASTICINE (fixed-corotated + von Mises in Hencky strain) or MPM_FLUID */
    float rho;          /* density; particle mass = rho * p_vol */
    float E, nu;        /* plasticine Young's modulus and Poisson ratio (Table 4) */
    float yield_stress; /* plasticine von Mises yield stress (Table 4) */
    float bulk_modulus; /* fluid: lambda = bulk_modulus, mu = 0 */
    float p_vol;        /* initial particle volume V0 (Table 4 "particle volume") */
} mpm_material;

typedef struct {
    int type;           /* MPM_BOX, MPM_CAPSULE or MPM_SDF_VOLUME */
    float half[3];      /* box half extents | capsule (radius, half length along local z, ignored) */
    float friction;     /* Coulomb coefficient >= 0 */
    /* MPM_SDF_VOLUME only (Sec. 3: a mesh's signed distances as a volume): samples on a lattice in the
     * shape frame, sample (i,j,k) at sdf_origin + sdf_h * (i,j,k) stored at
     * sdf[i + res[0] * (j + res[1] * k)], FP32, in DEVICE memory owned by the caller, which keeps it
     * alive and unchanged while the shape is in use. res[a] >= 2, sdf_h > 0. The library interpolates
     * trilinearly (in FP32, not with texture filtering) and takes the interpolant's gradient as the
     * normal; a point outside the lattice is outside the body. */
    const float* sdf;
    int res[3];
    float sdf_origin[3];
    float sdf_h;
} mpm_shape;

/* Bytes of device workspace a handle with this configuration needs. */
mpm_status mpm_workspace_size(const mpm_config* cfg, const mpm_material* mat, size_t* bytes);

/* ---- Batches of environments.
 * One handle can hold many independent environments (envs), each with its own grid, material,
 * particles and colliders; all advance together with the same launches (the vectorized simulation the
 * paper leaves as future work, App. D.3). A single-scene handle (mpm_create) is a batch of one.
 * Arrays that span envs are concatenations in env order: particle arrays are SoA over all particles
 * (stride = total count), collider arrays list all envs' colliders. The shared mpm_config supplies dt,
 * gravity and bound; its n, max_particles and max_colliders are taken per env from mpm_env. */
typedef struct {
    int n;              /* grid nodes per axis of this env: a multiple of 4 in [8, 256] */
    int max_particles;  /* capacity of this env, >= 1 */
    int max_colliders;  /* capacity of this env, >= 0 */
    mpm_material material;
} mpm_env;

#define MPM_MAX_ENVS 16384

mpm_status mpm_workspace_size_batch(const mpm_config* cfg, int nenv, const mpm_env* envs, size_t* bytes);
mpm_status mpm_create_batch(const mpm_config* cfg, int nenv, const mpm_env* envs, void* d_workspace, size_t bytes,
                            void* stream, mpm_sim** out);
/* counts[nenv] particles per env; arrays SoA over all sum(counts) particles, as mpm_set_particles. */
mpm_status mpm_set_particles_batch(mpm_sim* sim, const int* counts, const float* x, const float* v, const float* C,
                                   const float* F, int src_on_device, void* stream);
/* counts[nenv] shapes per env, shapes concatenated in env order. */
mpm_status mpm_set_shapes_batch(mpm_sim* sim, const int* counts, const mpm_shape* shapes);
int mpm_num_envs(const mpm_sim* sim);

/* Launch shape of the substep kernels (the autotuner's knobs): most particles per chunk of a bin
 * (chunk, 32..128, multiple of 32), resident CTAs per SM of the fused particle pass (1..7) and of the grid
 * update (1..8). 0 keeps a value. Takes effect at the next mpm_substep. */
mpm_status mpm_set_launch(mpm_sim* sim, int chunk, int fused_ctas_per_sm, int grid_ctas_per_sm);
mpm_status mpm_get_launch(const mpm_sim* sim, int* chunk, int* fused_ctas_per_sm, int* grid_ctas_per_sm);

/* Create a handle over a caller-owned device workspace; zeroes what must start at zero on `stream`.
 * cfg / mat are copied. On error *out is NULL. */
mpm_status mpm_create(const mpm_config* cfg, const mpm_material* mat, void* d_workspace, size_t bytes,
                      void* stream, mpm_sim** out);

/* Replace the particle state (Algorithm 1 "initialize soft scene"). n <= max_particles; n = 0 empties
 * the scene. Arrays are SoA with stride n, in host memory (src_on_device = 0: copied in, the call
 * returns once the host arrays may be reused) or device memory (src_on_device = 1: read on `stream`).
 * v and C may be NULL (zero); F may be NULL (identity). For MPM_FLUID only J = det F is kept.
 * Positions outside [2dx, 1-2dx] are clamped and flagged. Resets the grid; keeps colliders. */
mpm_status mpm_set_particles(mpm_sim* sim, int n, const float* x, const float* v, const float* C,
                             const float* F, int src_on_device, void* stream);

/* Collision shapes, copied once (Algorithm 1 "copy rigid body shapes ... to soft scene").
 * Host memory; k <= max_colliders. Takes effect at the next mpm_set_colliders. */
mpm_status mpm_set_shapes(mpm_sim* sim, int k, const mpm_shape* shapes);

/* Body poses and velocities after a rigid step (Algorithm 1 "copy rigid body poses to soft scene",
 * "initialize force-torque buffers per rigid body"). Host arrays, k = number of shapes set:
 *   pose    k x 7: frame origin (x, y, z) and orientation quaternion (w, x, y, z)
 *   lin_vel k x 3: velocity of the centre of mass;  ang_vel k x 3: angular velocity (world frame)
 *   com     k x 3: centre of mass (world frame); NULL = frame origin
 * ang_vel may be NULL (zero). Between two calls each body moves rigidly with these constant
 * velocities, evaluated in closed form at the start of every substep (tabulated on the device for the
 * first 64 substeps). The arrays are copied into a library-owned pinned staging buffer and uploaded
 * on `stream`: they may be reused when the call returns. The wrench accumulators and the substep
 * count are zeroed. For a batch, k is the total over envs and the arrays are concatenated in env order. */
mpm_status mpm_set_colliders(mpm_sim* sim, int k, const float* pose, const float* lin_vel,
                             const float* ang_vel, const float* com, void* stream);

/* Advance n_substeps >= 0 substeps (Algorithm 1's inner loop: P2G, grid velocity with gravity,
 * colliders and sticky walls, G2P with F update and return mapping). Asynchronous: no host sync. */
mpm_status mpm_substep(mpm_sim* sim, int n_substeps, void* stream);

/* Contact form (Sec. 3), for all envs of the handle; takes effect at the next substep.
 *   MPM_CONTACT_GRID (default): colliders act on grid nodes in the grid update; stiffness and damping
 *     are ignored.
 *   MPM_CONTACT_PARTICLE: Algorithm 1 "compute penalty forces": at the start of every substep each
 *     particle inside a body (phi < 0) gets, per unit mass and per body (index order), the acceleration
 *       a = a_n n - min(damping |v_t|, friction a_n) v_t / |v_t|,
 *       a_n = stiffness (-phi) + damping max(-v_n, 0),
 *     from its velocity relative to the body's surface velocity (v_n along the outward normal n, v_t
 *     the tangential rest); the particle-to-grid transfer adds dt m_p a to its momentum and the body's
 *     force-torque buffer receives -dt m_p a and its moment. The grid update then applies gravity and
 *     the walls only. stiffness >= 0 in 1/s^2 with stiffness dt^2 <= 1, damping >= 0 in 1/s with
 *     damping dt <= 1 (explicit stability). Each mpm_substep call then ends on a grid-to-particle pass alone, so that the next call's first
 *     transfer sees the poses of the mpm_set_colliders in between.
 * Not available while a surrogate network is attached (mpm_surrogate_attach). */
mpm_status mpm_set_contact(mpm_sim* sim, int mode, float stiffness, float damping);

/* Particle state in the caller's original order. Any pointer may be NULL (skipped). Arrays SoA with
 * stride n. dst_on_device = 1: written on `stream` (the paper's single GPU-GPU copy), no sync.
 * dst_on_device = 0: host memory, the call synchronizes `stream`. dst_on_device = 2: page-locked host
 * memory (cudaHostAlloc / cudaHostRegister), the copies enqueued on `stream` without waiting: the arrays
 * hold the state once `stream` reaches this call (MPM_ERR_INVALID_ARG for other memory). A fluid
 * reports F = J^(1/3) I. */
mpm_status mpm_read_state(mpm_sim* sim, float* x, float* v, float* C, float* F, int dst_on_device,
                          void* stream);

/* Force-torque buffers (Algorithm 1 "apply accumulated forces and torques"): for each collider the
 * impulse (3) and angular impulse about its centre of mass (3) that the body received from the soft
 * material since the last mpm_set_colliders, as k x 6 doubles in host memory; *n_substeps (may be NULL) gets
 * the substeps accumulated, so the mean force is impulse / (n_substeps * dt). Synchronizes `stream`. */
mpm_status mpm_read_wrench(mpm_sim* sim, double* impulse_torque, int* n_substeps, void* stream);

/* mpm_read_wrench into page-locked host memory, enqueued on `stream` without waiting: impulse_torque
 * (k x 6 doubles) and *n_substeps (may be NULL) hold the values once `stream` reaches this call. A loop
 * that reads every step's impulses back can so keep the device busy. MPM_ERR_INVALID_ARG if a destination
 * is not page-locked. */
mpm_status mpm_read_wrench_async(mpm_sim* sim, double* impulse_torque, unsigned* n_substeps, void* stream);

/* Sticky device flags (MPM_FLAG_*), ORed since creation or the last clear. Synchronizes `stream`. */
mpm_status mpm_get_status(mpm_sim* sim, unsigned* flags, int clear, void* stream);

/* Current particle count (host-side, no sync). */
int mpm_num_particles(const mpm_sim* sim);

/* Diagnostics: the grid holding the particle-to-grid transfer of the current state (mass and momentum,
 * before the grid velocity update), densely as float[n][n][n][4] = (m, mv_x, mv_y, mv_z) with node
 * (i,j,k) at ((i*n + j)*n + k)*4. Device destination only; enqueued on `stream`. For a batch, the envs'
 * grids follow one another in env order (env e's n_e^3 * 4 floats). */
mpm_status mpm_read_grid(mpm_sim* sim, float* d_out, void* stream);

/* Diagnostics: kernel timing. Every launch of a kernel kind whose bit (1 << MPM_K_*) is set in
 * kernel_mask is bracketed by CUDA events on its stream (inside replayed graphs too: the events are
 * swapped on every replay); 0 turns timing off. mpm_read_timing synchronizes and returns, per kernel kind,
 * the summed milliseconds and launch counts since the last reset (arrays of MPM_K_COUNT entries, either
 * may be NULL). Kinds: load (set_particles), scan and assign (bin sort after set_particles), p2g
 * (transfer after set_particles), grid (sort-assign + grid update, once per substep), g2p2g (fused
 * grid-to-particle / particle-to-grid with the bin scan, once per substep), read (readbacks),
 * colliders (collider upload). */
enum { MPM_K_LOAD = 0, MPM_K_SCAN, MPM_K_ASSIGN, MPM_K_P2G, MPM_K_GRID, MPM_K_G2P2G, MPM_K_READ,
       MPM_K_COLLIDERS, MPM_K_COUNT };
mpm_status mpm_set_timing(mpm_sim* sim, unsigned kernel_mask);
mpm_status mpm_read_timing(mpm_sim* sim, double* ms, long long* launches, int reset);

/* CUDA-graph replay of mpm_substep (default on): the launches of a call are captured once per distinct
 * (substep count, particle count, collider count, timing mask, pipeline state) and replayed with one
 * graph launch on the caller's stream. Off: every launch is issued directly. Calls on a stream that the
 * caller is capturing are always issued directly, so they land in the caller's graph. */
mpm_status mpm_set_graphs(mpm_sim* sim, int enable);

/* Number of kernels the handle has launched since creation (host counter, no sync). */
long long mpm_launch_count(const mpm_sim* sim);

/* Particle-to-grid transfer without any device allocation. The paper has no counterpart: this entry
 * serves callers that cannot call cudaMalloc -- a plugin inside a host simulator that owns all device
 * memory, or a real-time loop where cudaMalloc's implicit device synchronization is not allowed.
 * It computes what mpm_read_grid returns after mpm_set_particles (mass and momentum with the stress
 * impulse, before the grid velocity update) for the particle set given, straight into grid_out.
 *   x, v, C, F  device SoA arrays with stride n, as for mpm_set_particles (v, C NULL = zero; F NULL =
 *               identity; a fluid uses J = det F); positions are clamped into [2dx, 1-2dx] when read
 *   grid_out    device float[cfg->n]^3 [4] = (m, mv_x, mv_y, mv_z), 16-byte aligned; zeroed by the call
 * Scratch (bin keys and ranks, bin offsets, chunk list, sorted order; about 0.9 MB) lives in a device
 * array owned by the library, resident on every GPU that loads it until the process exits. Limits:
 * n <= 65,536 particles and cfg->n <= 64, else MPM_ERR_CAPACITY (nothing enqueued). Of cfg only n (a
 * multiple of 4, at least 8) and dt (> 0) are used and checked, with the material (MPM_ERR_INVALID_ARG).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress, once per
 * device, with that device current) and keeps it for the life of the process: make that first call
 * before any stream capture, and do not call this entry again on a device after cudaDeviceReset (or a
 * reset of its primary context), which may move the array. Every call on a device shares the array, so
 * calls that overlap on the GPU (different streams, or different host threads) race; serialize them.
 * Enqueued on `stream`, no host synchronization; allocates nothing. */
mpm_status mpm_p2g_static(const mpm_config* cfg, const mpm_material* mat, int n, const float* x, const float* v,
                          const float* C, const float* F, float* grid_out, void* stream);

/* ---- Learned-surrogate window. An extension of the method (the paper's simulator has no learned
 * component): k substeps are replaced by one plain grid update (gravity, colliders, sticky walls, as in
 * mpm_substep), a correction dv of the updated node velocities computed by the caller's network, and one
 * grid-to-particle transfer with time step k*dt (advection, C, and F <- (I + k dt C) F with the return
 * map), followed by the particle-to-grid transfer of the new state. One-env handles only
 * (MPM_ERR_INVALID_ARG otherwise). Boxes are in grid-node indices (axis order i, j, k of the grid). */
typedef struct {
    int i0, j0, k0; /* first node of the box (may be negative: nodes outside the grid read as empty) */
    int D, H, W;    /* nodes along i, j, k */
} mpm_box;

/* Bounding box of the grid nodes with mass (the active 4^3 bins) of the current state, grown by
 * `margin` nodes on every side and clamped to the grid. Synchronizes `stream`. */
mpm_status mpm_surrogate_box(mpm_sim* sim, int margin, mpm_box* box, void* stream);

/* Start a window: the sort-assign and the plain grid update of the current state, then the network
 * input over `box`: d_feat (float[D*H*W][4], 16-byte aligned) = (m * m_scale, v_x, v_y, v_z * v_scale)
 * of the updated nodes, channels-last with i slowest; d_mask (one byte per node) = m > 0. Enqueued
 * only. Until mpm_surrogate_advance ends the window, mpm_substep is refused. */
mpm_status mpm_surrogate_features(mpm_sim* sim, const mpm_box* box, float m_scale, float v_scale, float* d_feat,
                                  uint8_t* d_mask, void* stream);

/* The fallback gate of a started window, for the correction d_dv (float[D*H*W][3]; velocity change =
 * d_dv * dv_unit at nodes with mass; zero in the sticky wall band). Writes out[0] = mass residual
 * |sum_i m_i - sum_p m_p| / sum_p m_p, out[1] = momentum residual |P_hat - P_exp| / (M v_ref), where
 * P_hat is the momentum of the corrected nodes and P_exp = P_0 + (k + 1)/2 (P_1 - P_0) the first-order
 * mean momentum over k substeps from the momentum before (P_0) and after (P_1) one plain grid update;
 * out[2] = M, out[3] = |P_hat - P_exp|. v_ref = 0 takes the scene's own velocity scale: the
 * mass-weighted RMS node speed of the transfer at the window start, sqrt(sum_i |m v_i|^2 / m_i / M).
 * MPM_ERR_INVALID_ARG for v_ref < 0. Synchronizes `stream`. */
mpm_status mpm_surrogate_check(mpm_sim* sim, const mpm_box* box, const float* d_dv, float dv_unit, int k,
                               double v_ref, double* out, void* stream);

/* End a window. With d_dv: apply the correction, then one grid-to-particle pass with time step k*dt;
 * body impulses of the window are the first substep's times k; the substep counter advances by k.
 * With d_dv == NULL (the fallback): the plain grid-to-particle pass and k - 1 plain substeps. */
mpm_status mpm_surrogate_advance(mpm_sim* sim, const mpm_box* box, const float* d_dv, float dv_unit, int k,
                                 void* stream);

/* The surrogate network attached to a handle, so that whole environment steps of windows run inside
 * the library (graph-replayed, the gate decided on the device, no host synchronization per window).
 * Network: four 3x3x3 convolutions 4 -> 32 -> 32 -> 32 -> 3 (ReLU between), weights packed for the
 * tensor-core forward (mpm_conv3d_pack_tc in mpm_net.h), biases FP32, all device memory the caller owns
 * and keeps alive while attached. */
typedef struct {
    const void* w_packed[4];
    const float* bias[4];
    float m_scale, v_scale;  /* network input: (m * m_scale, v * v_scale) */
    float dv_unit;           /* m/s per network output unit */
    double v_ref;            /* velocity scale of the momentum residual (m/s); 0: the scene's RMS node speed */
    double threshold;        /* fallback when the mass or momentum residual exceeds this */
    int k;                   /* substeps per window, odd */
    int margin;              /* nodes added around the material's bins for the box */
} mpm_surrogate_net;

/* Device workspace for the network's buffers over boxes of up to max_voxels nodes and the start-of-step
 * snapshot of up to max_particles particles (the per-step fallback). */
size_t mpm_surrogate_workspace_size(int max_voxels, int max_particles);

/* Attach (net != NULL) or detach the network. One-env handles whose bins fit the fused scan only. */
mpm_status mpm_surrogate_attach(mpm_sim* sim, const mpm_surrogate_net* net, void* d_workspace, size_t bytes,
                                int max_voxels);

/* n_substeps (a multiple of k) as windows of the attached network, from one box computed for the call
 * (one host synchronization), enqueued as one graph launch. The gate:
 *   0  off: every window uses the network;
 *   1  per step: every window uses the network while the gate records its residuals on the device; one
 *      readback at the end of the call, and if any window exceeded the threshold the step is redone
 *      from a snapshot of its start (state, body impulses, substep count) with n_substeps plain substeps;
 *   2  per window: each window whose residuals exceed the threshold runs as k plain substeps instead,
 *      both branches enqueued and decided on the device.
 * A box larger than max_voxels runs plain substeps. */
mpm_status mpm_surrogate_step(mpm_sim* sim, int n_substeps, int gate, void* stream);

/* Counters of gated windows: windows run, windows that ran as plain substeps (failed windows with gate 2,
 * every window of a redone step with gate 1), and the last window's (mass, momentum) residuals;
 * reset != 0 zeroes the counters. Synchronizes `stream`. */
mpm_status mpm_surrogate_stats(mpm_sim* sim, long long* windows, long long* fallbacks, double* residuals, int reset,
                               void* stream);

/* Release the host handle (the workspace stays the caller's). Safe on NULL. Does not synchronize:
 * the caller must not free the workspace before work enqueued on it has finished. */
void mpm_destroy(mpm_sim* sim);

const char* mpm_status_string(mpm_status s);

/* Last CUDA error message seen by any call in this process (thread-local), or "". */
const char* mpm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
