/*
 * mpm_render.h -- C ABI of the particle renderer (screen-space splatting).
 *
 * App. D.2 of the paper renders MPM particles for visual observations by
 * screen-space splatting: particles drawn as spheres into a depth buffer, a
 * bilateral filter smoothing that depth with a width scaled by the distance
 * from the camera, then normals and lighting computed from the smoothed depth;
 * the particle positions reach the renderer by one GPU-GPU copy. Here the four
 * steps are CUDA kernels writing headless device buffers, and mpm_render_sim
 * reads a simulation handle's particle positions in place (no copy at all).
 *
 * The steps, for a pinhole camera (camera frame x right, y down, z forward;
 * x_cam = rot (x_world - eye); pixel (i, j) -- column i, row j -- has its centre
 * at (i + 0.5, j + 0.5); u = fx x/z + cx, v = fy y/z + cy):
 *   1. splat: a particle at camera depth z > near_z covers the pixels whose
 *      centres lie inside its projected ellipse of radii (fx r / z, fy r / z);
 *      at normalised distance s from the ellipse centre it has depth
 *      z - r sqrt(1 - s^2) clamped at 0 (the point-sprite sphere); each pixel
 *      keeps the nearest depth, +inf where nothing was drawn;
 *   2. bilateral filter: at a drawn pixel of depth d0, the weighted mean of the
 *      drawn pixels of the (2K+1)^2 window, weight
 *      exp(-(a^2 + b^2) / (2 s^2) - (d - d0)^2 / (2 sigma_depth^2)) for offset
 *      (a, b) and depth d, s = min(fx smooth / d0, K / 2) pixels;
 *   3. normals: camera-frame points from the smoothed depth; along x and along
 *      y the one-sided difference to the neighbour with the smaller depth jump
 *      (forward on ties); n = normalize(dy x dx), facing the camera; (0,0,-1)
 *      when a direction has no drawn neighbour;
 *   4. Lambert: rgb = albedo (ambient + (1 - ambient) max(0, n . l)); the
 *      background colour where nothing was drawn.
 * Arithmetic is FP32. Images are row-major [height][width] (normals and rgb
 * with 3 floats per pixel), in DEVICE memory owned by the caller.
 */
#ifndef MPM_RENDER_H
#define MPM_RENDER_H

#include <stddef.h>

#include "mpm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MPM_RENDER_MAX_SIDE 8192
#define MPM_RENDER_MAX_WINDOW 16

typedef struct {
    int width, height;  /* pixels, 1..MPM_RENDER_MAX_SIDE */
    float fx, fy;       /* focal lengths in pixels, > 0 */
    float cx, cy;       /* principal point in pixels */
    float eye[3];       /* camera position (world) */
    float rot[9];       /* world -> camera rotation, row-major */
    float near_z;       /* particles at camera depth <= near_z are not drawn; > 0 */
} mpm_camera;

typedef struct {
    float radius;        /* sphere radius of every particle (world), > 0 */
    float smooth;        /* bilateral spatial width, world units at the pixel's depth, > 0 */
    float sigma_depth;   /* bilateral range sigma (world), > 0 */
    int window;          /* bilateral half window K in pixels, 0..MPM_RENDER_MAX_WINDOW (0: no filter) */
    float light[3];      /* direction towards the light, camera frame (normalised here), nonzero */
    float albedo[3];
    float ambient;       /* 0..1 */
    float background[3];
} mpm_render_params;

/* Bytes of device workspace mpm_render needs for an image of this size (two depth planes). */
size_t mpm_render_workspace_size(int width, int height);

/* Render n particles with positions d_x (device, SoA [3][stride]: x at d_x[p], y at d_x[stride + p],
 * z at d_x[2 stride + p]; stride >= n). Outputs (device, each may be NULL except d_rgb):
 *   d_depth  [H][W]     step 1 (+inf where empty)
 *   d_smooth [H][W]     step 2
 *   d_normal [H][W][3]  step 3 (zero where empty)
 *   d_rgb    [H][W][3]  step 4
 * d_workspace: device, 256-byte aligned, >= mpm_render_workspace_size bytes. Enqueued on `stream`, no
 * host sync. Errors: MPM_ERR_INVALID_ARG for a NULL or out-of-range argument (nothing enqueued),
 * MPM_ERR_WORKSPACE for a missing, misaligned or small workspace, MPM_ERR_CUDA for a launch failure. */
mpm_status mpm_render(const mpm_camera* cam, const mpm_render_params* params, int n, int stride, const float* d_x,
                      float* d_depth, float* d_smooth, float* d_normal, float* d_rgb, void* d_workspace, size_t bytes,
                      void* stream);

/* The same for the particles of a simulation handle (all envs), read where the simulation keeps them:
 * the paper's GPU-GPU copy to the renderer becomes no copy. Stream-ordered after the handle's work. */
mpm_status mpm_render_sim(mpm_sim* sim, const mpm_camera* cam, const mpm_render_params* params, float* d_depth,
                          float* d_smooth, float* d_normal, float* d_rgb, void* d_workspace, size_t bytes,
                          void* stream);

#ifdef __cplusplus
}
#endif
#endif
