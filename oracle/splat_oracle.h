/*
 * splat_oracle.h -- plain FP64 CPU oracle of the particle renderer.
 *
 * TEST INFRASTRUCTURE ONLY (like mpm_oracle.h): called by the tests, the smoke
 * check and the benchmark's CPU-baseline leg, never by the product path; it
 * shares no code with the CUDA sources.
 *
 * What it computes. App. D.2 of the paper renders MPM particles by screen-space
 * splatting (Cords & Staadt 2008; as in NVIDIA Flex): particles drawn as
 * spheres into a depth buffer, the depth smoothed by a bilateral filter whose
 * width is scaled by the distance from the camera, then normals and lighting
 * computed from the smoothed depth. The paper gives no formulas; the ones here
 * are the standard screen-space forms of those steps (van der Laan, Green &
 * Sainz 2009, "Screen space fluid rendering with curvature flow"):
 *   1. splat: pinhole projection; a particle at camera-space depth z covers the
 *      pixels whose centres fall inside its projected disk (an ellipse when
 *      fx != fy), at depth z - r sqrt(1 - s^2) clamped at 0, s the normalised
 *      distance from the disk centre (the point-sprite sphere); the buffer keeps
 *      the minimum;
 *   2. bilateral filter: for each covered pixel with depth d0, over a fixed
 *      (2K+1)^2 window (K = 0: no filter), weights exp(-|offset|^2 / (2 sigma_s^2)) *
 *      exp(-(d - d0)^2 / (2 sigma_d^2)) on covered pixels, with the spatial
 *      width sigma_s = min(fx * smooth / d0, K / 2) pixels (world width
 *      `smooth` seen at depth d0: the distance scaling of App. D.2);
 *   3. normals: camera-space points from the smoothed depth, one-sided
 *      differences along x and y taking the side with the smaller depth jump
 *      (the side that stays on the surface), n = normalize(dy x dx), facing
 *      the camera;
 *   4. Lambert shading: albedo * (ambient + (1 - ambient) max(0, n . l)),
 *      background where nothing was drawn.
 *
 * Conventions. Camera frame: x right, y down, z forward (depth > 0 in front).
 * x_cam = rot (x_world - eye), rot row-major. Pixel (i, j) (column i, row j) has
 * its centre at (i + 0.5, j + 0.5); u = fx x/z + cx, v = fy y/z + cy. Images are
 * row-major [j][i]; an empty pixel has depth +inf.
 */
#ifndef SPLAT_ORACLE_H
#define SPLAT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int width, height;
    double fx, fy, cx, cy;
    double eye[3];
    double rot[9];
    double near_z;
} orc_camera;

typedef struct {
    double radius;        /* particle sphere radius (world) */
    double smooth;        /* bilateral spatial width (world units at the pixel's depth) */
    double sigma_depth;   /* bilateral range sigma (world) */
    int window;           /* half window K (pixels) */
    double light[3];      /* direction towards the light, camera frame (normalised here) */
    double albedo[3];
    double ambient;
    double background[3];
} orc_render;

/* Step 1: depth[H*W] = min splat depth (+inf where empty). ambiguous[H*W] (may be NULL): pixels where
 * some particle's coverage test is within 1e-4 of flipping (|s^2 - 1| < 1e-4) and that particle would
 * be at least as near as the pixel's depth. Returns the number of particles drawn (in front of near_z). */
int orc_splat_depth(const orc_camera* cam, const orc_render* R, int n, const double* x, double* depth,
                    unsigned char* ambiguous);

/* Step 2: smoothed[H*W] from depth[H*W]. */
void orc_bilateral(const orc_camera* cam, const orc_render* R, const double* depth, double* smoothed);

/* Steps 3 and 4: normal[H*W*3] (camera frame; zero where empty) and rgb[H*W*3] from the smoothed
 * depth. ambiguous[H*W] (may be NULL) marks pixels whose difference side is within 1e-5 * depth of
 * switching. */
void orc_shade(const orc_camera* cam, const orc_render* R, const double* smoothed, double* normal, double* rgb,
               unsigned char* ambiguous);

#ifdef __cplusplus
}
#endif
#endif
