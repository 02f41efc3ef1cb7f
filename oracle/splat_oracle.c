/*
 * splat_oracle.c -- plain FP64 CPU oracle of the particle renderer (App. D.2).
 *
 * TEST INFRASTRUCTURE ONLY (see splat_oracle.h). Each step is written as its
 * definition: every particle against every pixel of its footprint, every pixel
 * against every tap of its window, in index order.
 */
#include "splat_oracle.h"

#include <math.h>

static double inf(void) { return HUGE_VAL; }

/* App. D.2 "render soft-body particles as spheres": the point-sprite sphere of every particle. */
int orc_splat_depth(const orc_camera* cam, const orc_render* R, int n, const double* x, double* depth,
                    unsigned char* ambiguous) {
    const int W = cam->width, H = cam->height;
    for (int p = 0; p < W * H; ++p) {
        depth[p] = inf();
        if (ambiguous) ambiguous[p] = 0;
    }
    int drawn = 0;
    for (int q = 0; q < n; ++q) {
        double d[3] = {x[q] - cam->eye[0], x[n + q] - cam->eye[1], x[2 * n + q] - cam->eye[2]};
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = cam->rot[a * 3] * d[0] + cam->rot[a * 3 + 1] * d[1] + cam->rot[a * 3 + 2] * d[2];
        if (!(c[2] > cam->near_z)) continue;
        ++drawn;
        double up = cam->fx * c[0] / c[2] + cam->cx, vp = cam->fy * c[1] / c[2] + cam->cy;
        double rx = cam->fx * R->radius / c[2], ry = cam->fy * R->radius / c[2];
        /* every pixel whose centre could fall inside the ellipse (one pixel to spare on each side) */
        int i0 = (int)floor(up - rx - 0.5) - 1, i1 = (int)ceil(up + rx - 0.5) + 1;
        int j0 = (int)floor(vp - ry - 0.5) - 1, j1 = (int)ceil(vp + ry - 0.5) + 1;
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > W - 1) i1 = W - 1;
        if (j1 > H - 1) j1 = H - 1;
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                double du = ((double)i + 0.5 - up) / rx, dv = ((double)j + 0.5 - vp) / ry;
                double s2 = du * du + dv * dv;
                if (!(s2 < 1.0)) continue;
                double z = c[2] - R->radius * sqrt(1.0 - s2);
                if (z < 0.0) z = 0.0; /* a sphere reaching behind the camera */
                if (z < depth[j * W + i]) depth[j * W + i] = z;
            }
    }
    if (!ambiguous) return drawn;
    /* A pixel is ambiguous when a particle's coverage test there is within 1e-4 of flipping (FP32
     * evaluates s^2 to about that) and the particle, if it covered the pixel, would be at least as
     * near as what the pixel holds: only then can the flip change the depth. */
    for (int q = 0; q < n; ++q) {
        double d[3] = {x[q] - cam->eye[0], x[n + q] - cam->eye[1], x[2 * n + q] - cam->eye[2]};
        double c[3];
        for (int a = 0; a < 3; ++a) c[a] = cam->rot[a * 3] * d[0] + cam->rot[a * 3 + 1] * d[1] + cam->rot[a * 3 + 2] * d[2];
        if (!(c[2] > cam->near_z)) continue;
        double up = cam->fx * c[0] / c[2] + cam->cx, vp = cam->fy * c[1] / c[2] + cam->cy;
        double rx = cam->fx * R->radius / c[2], ry = cam->fy * R->radius / c[2];
        int i0 = (int)floor(up - rx - 0.5) - 1, i1 = (int)ceil(up + rx - 0.5) + 1;
        int j0 = (int)floor(vp - ry - 0.5) - 1, j1 = (int)ceil(vp + ry - 0.5) + 1;
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > W - 1) i1 = W - 1;
        if (j1 > H - 1) j1 = H - 1;
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                double du = ((double)i + 0.5 - up) / rx, dv = ((double)j + 0.5 - vp) / ry;
                double s2 = du * du + dv * dv;
                if (fabs(s2 - 1.0) < 1e-4 && c[2] - R->radius * 0.01 <= depth[j * W + i]) ambiguous[j * W + i] = 1;
            }
    }
    return drawn;
}

/* App. D.2 "a bilateral filter to smooth the depth buffer", its width scaled with the distance from
 * the camera. */
void orc_bilateral(const orc_camera* cam, const orc_render* R, const double* depth, double* smoothed) {
    const int W = cam->width, H = cam->height, K = R->window;
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            double d0 = depth[j * W + i];
            if (K == 0 || !(d0 < inf())) { /* no filter, or nothing drawn here */
                smoothed[j * W + i] = d0;
                continue;
            }
            double ss = cam->fx * R->smooth / d0;
            if (ss > 0.5 * K) ss = 0.5 * K;
            double sum = 0.0, wsum = 0.0;
            for (int b = -K; b <= K; ++b)
                for (int a = -K; a <= K; ++a) {
                    int ii = i + a, jj = j + b;
                    if (ii < 0 || jj < 0 || ii >= W || jj >= H) continue;
                    double d = depth[jj * W + ii];
                    if (!(d < inf())) continue;
                    double dd = d - d0;
                    double w = exp(-(double)(a * a + b * b) / (2.0 * ss * ss)) *
                               exp(-dd * dd / (2.0 * R->sigma_depth * R->sigma_depth));
                    sum += w * d;
                    wsum += w;
                }
            smoothed[j * W + i] = sum / wsum;
        }
}

/* Camera-space point of pixel (i, j) at depth d. */
static void unproject(const orc_camera* cam, int i, int j, double d, double P[3]) {
    P[0] = d * ((double)i + 0.5 - cam->cx) / cam->fx;
    P[1] = d * ((double)j + 0.5 - cam->cy) / cam->fy;
    P[2] = d;
}

/* One-sided difference along (di, dj) at pixel (i, j): the side with the smaller depth jump; returns 0
 * when neither neighbour is drawn. */
static int side_difference(const orc_camera* cam, const double* z, int i, int j, int di, int dj, double out[3],
                           int* ambiguous) {
    const int W = cam->width, H = cam->height;
    double d0 = z[j * W + i];
    int fi = i + di, fj = j + dj, bi = i - di, bj = j - dj;
    int has_f = fi < W && fj < H && z[fj * W + fi] < inf();
    int has_b = bi >= 0 && bj >= 0 && z[bj * W + bi] < inf();
    if (!has_f && !has_b) return 0;
    double P0[3], P1[3];
    unproject(cam, i, j, d0, P0);
    int use_f = has_f;
    if (has_f && has_b) {
        double jf = fabs(z[fj * W + fi] - d0), jb = fabs(z[bj * W + bi] - d0);
        use_f = jf <= jb;
        if (fabs(jf - jb) < 1e-5 * d0) *ambiguous = 1;
    }
    if (use_f) {
        unproject(cam, fi, fj, z[fj * W + fi], P1);
        for (int a = 0; a < 3; ++a) out[a] = P1[a] - P0[a];
    } else {
        unproject(cam, bi, bj, z[bj * W + bi], P1);
        for (int a = 0; a < 3; ++a) out[a] = P0[a] - P1[a];
    }
    return 1;
}

/* App. D.2 "compute normal and lighting on the smoothed soft-body depth". */
void orc_shade(const orc_camera* cam, const orc_render* R, const double* z, double* normal, double* rgb,
               unsigned char* ambiguous) {
    const int W = cam->width, H = cam->height;
    double l[3] = {R->light[0], R->light[1], R->light[2]};
    double ll = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    for (int a = 0; a < 3; ++a) l[a] /= ll;
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            int p = j * W + i;
            int amb = 0;
            double* nrm = normal + 3 * p;
            nrm[0] = nrm[1] = nrm[2] = 0.0;
            if (!(z[p] < inf())) {
                for (int a = 0; a < 3; ++a) rgb[3 * p + a] = R->background[a];
                if (ambiguous) ambiguous[p] = 0;
                continue;
            }
            double dx[3], dy[3];
            int okx = side_difference(cam, z, i, j, 1, 0, dx, &amb);
            int oky = side_difference(cam, z, i, j, 0, 1, dy, &amb);
            if (okx && oky) {
                /* n = dy x dx: towards the camera (-z) for a surface facing it */
                double c[3] = {dy[1] * dx[2] - dy[2] * dx[1], dy[2] * dx[0] - dy[0] * dx[2],
                               dy[0] * dx[1] - dy[1] * dx[0]};
                double cl = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
                if (cl > 0.0)
                    for (int a = 0; a < 3; ++a) nrm[a] = c[a] / cl;
                else
                    nrm[2] = -1.0;
            } else {
                nrm[2] = -1.0; /* an isolated pixel or line: facing the camera */
            }
            double ndl = nrm[0] * l[0] + nrm[1] * l[1] + nrm[2] * l[2];
            double diff = ndl > 0.0 ? ndl : 0.0;
            for (int a = 0; a < 3; ++a) rgb[3 * p + a] = R->albedo[a] * (R->ambient + (1.0 - R->ambient) * diff);
            if (ambiguous) ambiguous[p] = (unsigned char)amb;
        }
}
