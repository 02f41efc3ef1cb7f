// render_kernels.cu -- the particle renderer of App. D.2 (screen-space splatting), FP32, sm_103a.
//
// Three launches per frame after the depth plane is cleared:
//   k_splat      one thread per particle: project, walk the pixels of its projected ellipse, keep the
//                nearest point-sprite depth per pixel with an integer atomicMin on the FP32 bits
//                (depths are >= 0, where the bit order is the numeric order)
//   k_bilateral  one thread per pixel over a shared-memory tile with a K-pixel halo: the
//                distance-scaled bilateral filter of the depth
//   k_shade      one thread per pixel: normals from one-sided differences of the smoothed depth,
//                Lambert shading into the colour plane
// The formulas are stated in mpm_render.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mpm_internal.h"
#include "mpm_render.h"

namespace mpm {

namespace {

constexpr uint32_t kInfBits = 0x7f800000u;
constexpr int kTile = 16;  // bilateral / shading tile (kTile x kTile threads)

__global__ void __launch_bounds__(256) k_depth_clear(uint32_t* __restrict__ d, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) d[i] = kInfBits;
}

// Step 1. A particle behind near_z draws nothing; the pixel loop covers the ellipse's bounding box,
// clamped to the image before any float -> int conversion.
__global__ void __launch_bounds__(256) k_splat(mpm_camera cam, float r, int n, int stride,
                                               const float* __restrict__ x, uint32_t* __restrict__ depth) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float d[3] = {x[p] - cam.eye[0], x[(size_t)stride + p] - cam.eye[1], x[2 * (size_t)stride + p] - cam.eye[2]};
    float c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = cam.rot[a * 3] * d[0] + cam.rot[a * 3 + 1] * d[1] + cam.rot[a * 3 + 2] * d[2];
    if (!(c[2] > cam.near_z)) return;
    const float up = cam.fx * c[0] / c[2] + cam.cx, vp = cam.fy * c[1] / c[2] + cam.cy;
    const float rx = cam.fx * r / c[2], ry = cam.fy * r / c[2];
    const float W = (float)cam.width, H = (float)cam.height;
    // pixel centres i + 0.5 inside [up - rx, up + rx]: floor / ceil leave up to a pixel of slack
    const float fi0 = fminf(fmaxf(floorf(up - rx - 0.5f), 0.0f), W);
    const float fi1 = fminf(fmaxf(ceilf(up + rx - 0.5f), -1.0f), W - 1.0f);
    const float fj0 = fminf(fmaxf(floorf(vp - ry - 0.5f), 0.0f), H);
    const float fj1 = fminf(fmaxf(ceilf(vp + ry - 0.5f), -1.0f), H - 1.0f);
    if (!(fi0 <= fi1) || !(fj0 <= fj1)) return;  // off screen (or NaN)
    const int i0 = (int)fi0, i1 = (int)fi1, j0 = (int)fj0, j1 = (int)fj1;
    const float irx = 1.0f / rx, iry = 1.0f / ry;
    for (int j = j0; j <= j1; ++j) {
        const float dv = ((float)j + 0.5f - vp) * iry;
        for (int i = i0; i <= i1; ++i) {
            const float du = ((float)i + 0.5f - up) * irx;
            const float s2 = du * du + dv * dv;
            if (!(s2 < 1.0f)) continue;
            const float z = fmaxf(c[2] - r * sqrtf(1.0f - s2), 0.0f);
            atomicMin(&depth[(size_t)j * cam.width + i], __float_as_uint(z));
        }
    }
}

// Step 2. The tile and its halo are staged in shared memory (empty pixels as +inf); K == 0 copies.
__global__ void __launch_bounds__(kTile * kTile) k_bilateral(mpm_camera cam, float smooth, float sigma_depth, int K,
                                                            const uint32_t* __restrict__ depth,
                                                            float* __restrict__ out) {
    extern __shared__ float tile[];
    const int side = kTile + 2 * K;
    const int ti = blockIdx.x * kTile, tj = blockIdx.y * kTile;
    const int W = cam.width, H = cam.height;
    for (int t = threadIdx.y * kTile + threadIdx.x; t < side * side; t += kTile * kTile) {
        const int gi = ti - K + t % side, gj = tj - K + t / side;
        tile[t] = (gi >= 0 && gj >= 0 && gi < W && gj < H) ? __uint_as_float(depth[(size_t)gj * W + gi])
                                                           : __uint_as_float(kInfBits);
    }
    __syncthreads();
    const int i = ti + threadIdx.x, j = tj + threadIdx.y;
    if (i >= W || j >= H) return;
    const float d0 = tile[(threadIdx.y + K) * side + threadIdx.x + K];
    if (K == 0 || !(d0 < INFINITY)) {
        out[(size_t)j * W + i] = d0;
        return;
    }
    const float ss = fminf(cam.fx * smooth / d0, 0.5f * (float)K);
    const float inv_s = 1.0f / (2.0f * ss * ss), inv_r = 1.0f / (2.0f * sigma_depth * sigma_depth);
    float sum = 0.0f, wsum = 0.0f;
    for (int b = -K; b <= K; ++b) {
        const float* row = tile + (threadIdx.y + K + b) * side + threadIdx.x + K;
        for (int a = -K; a <= K; ++a) {
            const float d = row[a];
            if (!(d < INFINITY)) continue;
            const float dd = d - d0;
            const float w = expf(-(float)(a * a + b * b) * inv_s - dd * dd * inv_r);
            sum += w * d;
            wsum += w;
        }
    }
    out[(size_t)j * W + i] = sum / wsum;
}

__device__ __forceinline__ void unproject(const mpm_camera& cam, int i, int j, float d, float P[3]) {
    P[0] = d * ((float)i + 0.5f - cam.cx) / cam.fx;
    P[1] = d * ((float)j + 0.5f - cam.cy) / cam.fy;
    P[2] = d;
}

// One-sided difference along (di, dj): to the drawn neighbour with the smaller depth jump (forward on
// ties); false when neither neighbour is drawn.
__device__ __forceinline__ bool side_difference(const mpm_camera& cam, const float* __restrict__ z, int i, int j,
                                                int di, int dj, float d0, float out[3]) {
    const int W = cam.width, H = cam.height;
    const int fi = i + di, fj = j + dj, bi = i - di, bj = j - dj;
    const float zf = (fi < W && fj < H) ? z[(size_t)fj * W + fi] : INFINITY;
    const float zb = (bi >= 0 && bj >= 0) ? z[(size_t)bj * W + bi] : INFINITY;
    const bool has_f = zf < INFINITY, has_b = zb < INFINITY;
    if (!has_f && !has_b) return false;
    const bool use_f = has_f && (!has_b || fabsf(zf - d0) <= fabsf(zb - d0));
    float P0[3], P1[3];
    unproject(cam, i, j, d0, P0);
    if (use_f) {
        unproject(cam, fi, fj, zf, P1);
#pragma unroll
        for (int a = 0; a < 3; ++a) out[a] = P1[a] - P0[a];
    } else {
        unproject(cam, bi, bj, zb, P1);
#pragma unroll
        for (int a = 0; a < 3; ++a) out[a] = P0[a] - P1[a];
    }
    return true;
}

// Steps 3 and 4.
__global__ void __launch_bounds__(kTile * kTile) k_shade(mpm_camera cam, mpm_render_params rp, float3 l,
                                                        const float* __restrict__ z, float* __restrict__ normal,
                                                        float* __restrict__ rgb) {
    const int i = blockIdx.x * kTile + threadIdx.x, j = blockIdx.y * kTile + threadIdx.y;
    if (i >= cam.width || j >= cam.height) return;
    const size_t p = (size_t)j * cam.width + i;
    const float d0 = z[p];
    float n[3] = {0.0f, 0.0f, 0.0f};
    float col[3];
    if (!(d0 < INFINITY)) {
#pragma unroll
        for (int a = 0; a < 3; ++a) col[a] = rp.background[a];
    } else {
        float dx[3], dy[3];
        const bool okx = side_difference(cam, z, i, j, 1, 0, d0, dx);
        const bool oky = side_difference(cam, z, i, j, 0, 1, d0, dy);
        n[2] = -1.0f;
        if (okx && oky) {
            const float c[3] = {dy[1] * dx[2] - dy[2] * dx[1], dy[2] * dx[0] - dy[0] * dx[2], dy[0] * dx[1] - dy[1] * dx[0]};
            const float cl = sqrtf(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
            if (cl > 0.0f) {
#pragma unroll
                for (int a = 0; a < 3; ++a) n[a] = c[a] / cl;
            }
        }
        const float diff = fmaxf(n[0] * l.x + n[1] * l.y + n[2] * l.z, 0.0f);
#pragma unroll
        for (int a = 0; a < 3; ++a) col[a] = rp.albedo[a] * (rp.ambient + (1.0f - rp.ambient) * diff);
    }
    if (normal) {
#pragma unroll
        for (int a = 0; a < 3; ++a) normal[3 * p + a] = n[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) rgb[3 * p + a] = col[a];
}

bool finite3(const float* v, int k) {
    for (int a = 0; a < k; ++a)
        if (!std::isfinite(v[a])) return false;
    return true;
}

}  // namespace

size_t render_workspace_bytes(int width, int height) {
    const size_t plane = ((size_t)width * height * sizeof(float) + 255) / 256 * 256;
    return 2 * plane;
}

bool render_args_valid(const mpm_camera* cam, const mpm_render_params* rp) {
    if (!cam || !rp) return false;
    if (cam->width < 1 || cam->height < 1 || cam->width > MPM_RENDER_MAX_SIDE || cam->height > MPM_RENDER_MAX_SIDE)
        return false;
    if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy)) return false;
    if (!std::isfinite(cam->cx) || !std::isfinite(cam->cy) || !finite3(cam->eye, 3) || !finite3(cam->rot, 9)) return false;
    if (!(cam->near_z > 0.0f) || !std::isfinite(cam->near_z)) return false;
    if (!(rp->radius > 0.0f) || !std::isfinite(rp->radius)) return false;
    if (!(rp->smooth > 0.0f) || !std::isfinite(rp->smooth)) return false;
    if (!(rp->sigma_depth > 0.0f) || !std::isfinite(rp->sigma_depth)) return false;
    if (rp->window < 0 || rp->window > MPM_RENDER_MAX_WINDOW) return false;
    if (!finite3(rp->light, 3) || !finite3(rp->albedo, 3) || !finite3(rp->background, 3)) return false;
    if (!(rp->ambient >= 0.0f && rp->ambient <= 1.0f)) return false;
    const float ll = rp->light[0] * rp->light[0] + rp->light[1] * rp->light[1] + rp->light[2] * rp->light[2];
    return ll > 0.0f && std::isfinite(ll);
}

mpm_status render_enqueue(const mpm_camera& cam, const mpm_render_params& rp, int n, int stride, const float* d_x,
                          float* d_depth, float* d_smooth, float* d_normal, float* d_rgb, void* ws, size_t bytes,
                          cudaStream_t st) {
    if (!d_rgb || n < 0 || stride < n || (n > 0 && !d_x)) return MPM_ERR_INVALID_ARG;
    if (!ws || reinterpret_cast<uintptr_t>(ws) % 256 || bytes < render_workspace_bytes(cam.width, cam.height))
        return MPM_ERR_WORKSPACE;
    const int npx = cam.width * cam.height;
    const size_t plane = render_workspace_bytes(cam.width, cam.height) / 2;
    uint32_t* depth = d_depth ? reinterpret_cast<uint32_t*>(d_depth) : static_cast<uint32_t*>(ws);
    float* smooth = d_smooth ? d_smooth : reinterpret_cast<float*>(static_cast<char*>(ws) + plane);
    k_depth_clear<<<std::min((npx + 255) / 256, 152 * 8), 256, 0, st>>>(depth, npx);
    if (n > 0) k_splat<<<(n + 255) / 256, 256, 0, st>>>(cam, rp.radius, n, stride, d_x, depth);
    const dim3 tiles((cam.width + kTile - 1) / kTile, (cam.height + kTile - 1) / kTile);
    const dim3 threads(kTile, kTile);
    const int side = kTile + 2 * rp.window;
    k_bilateral<<<tiles, threads, side * side * sizeof(float), st>>>(cam, rp.smooth, rp.sigma_depth, rp.window, depth,
                                                                     smooth);
    const float ll = sqrtf(rp.light[0] * rp.light[0] + rp.light[1] * rp.light[1] + rp.light[2] * rp.light[2]);
    const float3 l = make_float3(rp.light[0] / ll, rp.light[1] / ll, rp.light[2] / ll);
    k_shade<<<tiles, threads, 0, st>>>(cam, rp, l, smooth, d_normal, d_rgb);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda_error(e, "render");
    return MPM_OK;
}

}  // namespace mpm

extern "C" {

size_t mpm_render_workspace_size(int width, int height) {
    if (width < 1 || height < 1 || width > MPM_RENDER_MAX_SIDE || height > MPM_RENDER_MAX_SIDE) return 0;
    return mpm::render_workspace_bytes(width, height);
}

mpm_status mpm_render(const mpm_camera* cam, const mpm_render_params* params, int n, int stride, const float* d_x,
                      float* d_depth, float* d_smooth, float* d_normal, float* d_rgb, void* d_workspace, size_t bytes,
                      void* stream) {
    if (!mpm::render_args_valid(cam, params)) return MPM_ERR_INVALID_ARG;
    return mpm::render_enqueue(*cam, *params, n, stride, d_x, d_depth, d_smooth, d_normal, d_rgb, d_workspace, bytes,
                               static_cast<cudaStream_t>(stream));
}

}  // extern "C"
