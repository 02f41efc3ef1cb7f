// net_kernels.cu -- the learned grid surrogate's network: 3x3x3 convolutions (forward, input gradient,
// weight gradient), masked MSE loss and Adam, behind include/mpm_net.h.
//
// Two precisions. FP32: plain CUDA-core kernels, one output element per thread (the reference mode the
// gradient checks hold to 1e-5). BF16: implicit-GEMM tensor-core kernels (mma.sync m16n8k16, FP32
// accumulate). A convolution is the GEMM y[M = voxels][N = cout] = A[M][K] B[K][N] with K = 27 * cin
// ordered (tap, ci), A[p][(t, ci)] = x[p + o_t][ci], B[(t, ci)][co] = w[t][co][ci]. A CTA owns a tile of
// 4 x 4 x 8 output voxels: it stages the 6 x 6 x 10 input halo (channels-last, padded rows) and the whole
// weight matrix (rows = output channels, k contiguous, padded) in shared memory and loops persistently
// over tiles, so each CTA loads the weights once. Each of 4 warps computes 32 voxels x all channels.
// The input gradient is the same kernel on the flipped, transposed weights (w'[t][ci][co] =
// w[26 - t][co][ci]) with the ReLU mask of the layer below folded into the epilogue. The weight gradient
// is, per tap, the GEMM dw[t][co][ci] = sum_p dy[p][co] x[p + o_t][ci] (M = cout, N = cin, K = voxels),
// accumulated per CTA in shared memory over its tiles and added to the output with one FP32 atomic per
// entry per CTA.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "mpm_internal.h"
#include "mpm_net.h"

namespace mpm {
namespace net {
namespace {

constexpr int TZ = 4, TY = 4, TX = 8, TM = TZ * TY * TX;  // output voxels per tile (128)
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2, HV = HZ * HY * HX;  // halo voxels (360)
constexpr int kThreads = 128;

__host__ __device__ __forceinline__ int ceil_to(int v, int m) { return (v + m - 1) / m * m; }

// shared-memory row strides (bf16 elements): +8 keeps the 8 rows a fragment load touches on distinct banks
__host__ __device__ __forceinline__ int x_stride(int cin) { return cin % 16 == 0 ? cin + 8 : cin; }
__host__ __device__ __forceinline__ int k_pad(int cin) { return ceil_to(27 * cin, 16); }
__host__ __device__ __forceinline__ int w_stride(int cin) { return k_pad(cin) + 8; }

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A B + D for one m16n8k16 tile (A row-major 16x16 bf16, B column-major 16x8 bf16, FP32 D)
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct Box {
    int D, H, W;
    int tz, ty, tx;  // tiles per axis
    __host__ __device__ int tiles() const { return tz * ty * tx; }
};

Box make_box(int D, int H, int W) {
    Box b{D, H, W, (D + TZ - 1) / TZ, (H + TY - 1) / TY, (W + TX - 1) / TX};
    return b;
}

__device__ __forceinline__ void tile_origin(const Box& b, int tile, int& z0, int& y0, int& x0) {
    x0 = (tile % b.tx) * TX;
    y0 = ((tile / b.tx) % b.ty) * TY;
    z0 = (tile / (b.tx * b.ty)) * TZ;
}

// Stage the halo of a tile: Xs[h][c] for h in [0, HV), channels-last with row stride xs, zeros outside.
__device__ void stage_halo(__nv_bfloat16* Xs, const __nv_bfloat16* __restrict__ x, const Box& b, int cin, int xs,
                           int z0, int y0, int x0) {
    if (cin % 8 == 0) {
        const int vec = cin / 8;  // 16-byte pieces per voxel
        for (int i = threadIdx.x; i < HV * vec; i += blockDim.x) {
            const int h = i / vec, q = i % vec;
            const int z = z0 - 1 + h / (HY * HX), y = y0 - 1 + (h / HX) % HY, xx = x0 - 1 + h % HX;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (z >= 0 && z < b.D && y >= 0 && y < b.H && xx >= 0 && xx < b.W)
                v = reinterpret_cast<const uint4*>(x + (((size_t)z * b.H + y) * b.W + xx) * cin)[q];
            *reinterpret_cast<uint4*>(Xs + h * xs + q * 8) = v;
        }
    } else {
        for (int i = threadIdx.x; i < HV * cin; i += blockDim.x) {
            const int h = i / cin, c = i % cin;
            const int z = z0 - 1 + h / (HY * HX), y = y0 - 1 + (h / HX) % HY, xx = x0 - 1 + h % HX;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (z >= 0 && z < b.D && y >= 0 && y < b.H && xx >= 0 && xx < b.W)
                v = x[(((size_t)z * b.H + y) * b.W + xx) * cin + c];
            Xs[h * xs + c] = v;
        }
    }
}

// ------------------------------------------------------------------------ BF16 forward / input gradient
//
// Forward tiles are 4 x 8 x 8 voxels (256 GEMM rows, 8 warps x 32 rows) with a 6 x 10 x 10 halo. Fragments
// come from shared memory with ldmatrix: the A rows of an m16 tile are 16 voxels whose halo rows (one
// voxel's channels, 16-byte aligned, padded to 80 bytes for 32 channels) fall on distinct banks; B rows are
// output channels with k contiguous. With a tile flag array, a tile whose flag is 0 is written as zeros
// instead of computed (the surrogate needs outputs only near the material).

constexpr int FZ = 4, FY = 8, FX = 8, FM = FZ * FY * FX;                // 256 output voxels per tile
constexpr int GZ = FZ + 2, GY = FY + 2, GX = FX + 2, GV = GZ * GY * GX;  // 600 halo voxels
constexpr int kFwdThreads = 256;

__host__ __device__ __forceinline__ int fwd_tiles(const Box& b, int& tx, int& ty) {
    tx = (b.W + FX - 1) / FX;
    ty = (b.H + FY - 1) / FY;
    return tx * ty * ((b.D + FZ - 1) / FZ);
}

__device__ __forceinline__ int fwd_tap_offset(int t) {
    return ((t / 9) * GY + (t / 3) % 3) * GX + t % 3;
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const __nv_bfloat16* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x2(uint32_t& r0, uint32_t& r1, const __nv_bfloat16* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

struct ConvMma {
    Box box;
    int cin, cout;                  // of this GEMM (for the input gradient: cin = original cout, ...)
    const __nv_bfloat16* x;         // [vox][cin]
    const __nv_bfloat16* w;         // original [27][co][ci] layout of the layer
    int transpose;                  // 1: input gradient (use w[26 - t][c][n] for output n, input c)
    int w_cin;                      // the layer's cin (row length of w)
    const float* bias;
    int relu;
    const __nv_bfloat16* mask;      // [vox][cout] or null: output *= (mask > 0)
    void* y;                        // [vox][cout], bf16 or f32
    int y_f32;
    const uint8_t* tile_need;       // per forward tile, or null: compute every tile
};

template <int HZ_, int HY_, int HX_>
__device__ void stage_halo_t(__nv_bfloat16* Xs, const __nv_bfloat16* __restrict__ x, const Box& b, int cin, int xs,
                             int z0, int y0, int x0) {
    constexpr int HV_ = HZ_ * HY_ * HX_;
    if (cin % 8 == 0) {
        const int vec = cin / 8;  // 16-byte pieces per voxel
        for (int i = threadIdx.x; i < HV_ * vec; i += blockDim.x) {
            const int h = i / vec, q = i % vec;
            const int z = z0 - 1 + h / (HY_ * HX_), y = y0 - 1 + (h / HX_) % HY_, xx = x0 - 1 + h % HX_;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (z >= 0 && z < b.D && y >= 0 && y < b.H && xx >= 0 && xx < b.W)
                v = reinterpret_cast<const uint4*>(x + (((size_t)z * b.H + y) * b.W + xx) * cin)[q];
            *reinterpret_cast<uint4*>(Xs + h * xs + q * 8) = v;
        }
    } else {
        for (int i = threadIdx.x; i < HV_ * cin; i += blockDim.x) {
            const int h = i / cin, c = i % cin;
            const int z = z0 - 1 + h / (HY_ * HX_), y = y0 - 1 + (h / HX_) % HY_, xx = x0 - 1 + h % HX_;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (z >= 0 && z < b.D && y >= 0 && y < b.H && xx >= 0 && xx < b.W)
                v = x[(((size_t)z * b.H + y) * b.W + xx) * cin + c];
            Xs[h * xs + c] = v;
        }
    }
}

template <int NT>  // n8 tiles: cout <= 8 * NT
__global__ void __launch_bounds__(kFwdThreads, 2) k_conv_mma(ConvMma a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cin = a.cin, xs = x_stride(cin), K = 27 * cin, KP = k_pad(cin), ws = w_stride(cin);
    __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(smem_raw);                 // [NT*8][ws]
    __nv_bfloat16* Xs = Ws + NT * 8 * ws;                                            // [GV][xs]
    // weights: Ws[n][k], k = t * cin + c; zero for n >= cout or k >= K
    for (int i = threadIdx.x; i < NT * 8 * KP; i += blockDim.x) {
        const int n = i / KP, k = i % KP;
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (n < a.cout && k < K) {
            const int t = k / cin, c = k % cin;
            v = a.transpose ? a.w[((size_t)(26 - t) * cin + c) * a.w_cin + n]   // w[26-t][co = c][ci = n]
                            : a.w[((size_t)t * a.cout + n) * cin + c];
        }
        Ws[n * ws + k] = v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, kk = (lane & 3) * 2;
    const int lq = lane >> 3, lr = lane & 7;
    // halo index (centre tap) of the rows this lane addresses for ldmatrix (A) and holds in the mma layout
    int hA[2], hb[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int m = warp * 32 + mt * 16 + lr + (lq & 1) * 8;
        hA[mt] = ((m / (FY * FX)) * GY + (m / FX) % FY) * GX + m % FX;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int mm = warp * 32 + mt * 16 + g + r * 8;
            hb[mt][r] = ((mm / (FY * FX)) * GY + (mm / FX) % FY) * GX + mm % FX;
        }
    }
    const int a_koff = (lq >> 1) * 8;
    const bool fast = cin % 16 == 0;
    int tx, ty;
    const int tiles = fwd_tiles(a.box, tx, ty);
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int x0 = (tile % tx) * FX, y0 = ((tile / tx) % ty) * FY, z0 = (tile / (tx * ty)) * FZ;
        if (a.tile_need && !a.tile_need[tile]) {  // not needed: zeros (uniform across the CTA)
            for (int i = threadIdx.x; i < FM * a.cout; i += blockDim.x) {
                const int m = i / a.cout, n = i % a.cout;
                const int z = z0 + m / (FY * FX), y = y0 + (m / FX) % FY, xx = x0 + m % FX;
                if (z >= a.box.D || y >= a.box.H || xx >= a.box.W) continue;
                const size_t o = (((size_t)z * a.box.H + y) * a.box.W + xx) * a.cout + n;
                if (a.y_f32) static_cast<float*>(a.y)[o] = 0.0f;
                else static_cast<__nv_bfloat16*>(a.y)[o] = __float2bfloat16(0.0f);
            }
            continue;
        }
        __syncthreads();  // previous tile's reads of Xs done (and, first time, Ws written)
        stage_halo_t<GZ, GY, GX>(Xs, a.x, a.box, cin, xs, z0, y0, x0);
        __syncthreads();
        float acc[2][NT][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
        for (int k0 = 0; k0 < KP; k0 += 16) {
            uint32_t af[2][4];
            if (fast) {  // the 16 k of this step are channels c0..c0+15 of one tap
                const int t = k0 / cin, c0 = k0 % cin, off = fwd_tap_offset(t);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) ldsm_x4(af[mt], Xs + (hA[mt] + off) * xs + c0 + a_koff);
            } else {  // gather element by element (few input channels)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = q & 1, kq = k0 + kk + (q >> 1) * 8;
                        __nv_bfloat16 e0 = __float2bfloat16(0.0f), e1 = e0;
                        if (kq < K) e0 = Xs[(hb[mt][r] + fwd_tap_offset(kq / cin)) * xs + kq % cin];
                        if (kq + 1 < K) e1 = Xs[(hb[mt][r] + fwd_tap_offset((kq + 1) / cin)) * xs + (kq + 1) % cin];
                        af[mt][q] = pack2(e0, e1);
                    }
            }
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {  // two n8 tiles per ldmatrix.x4
                uint32_t b[4];
                ldsm_x4(b, Ws + ((np * 2 + (lq >> 1)) * 8 + lr) * ws + k0 + (lq & 1) * 8);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma16816(acc[mt][2 * np], af[mt], b[0], b[1]);
                    mma16816(acc[mt][2 * np + 1], af[mt], b[2], b[3]);
                }
            }
            if constexpr (NT % 2 == 1) {
                uint32_t b0, b1;
                ldsm_x2(b0, b1, Ws + ((NT - 1) * 8 + lr) * ws + k0 + (lq & 1) * 8);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][NT - 1], af[mt], b0, b1);
            }
        }
        // epilogue: bias, ReLU, mask, store (rows g / g + 8, columns kk / kk + 1 of each n8 tile)
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int m = warp * 32 + mt * 16 + g + r * 8;
                const int z = z0 + m / (FY * FX), y = y0 + (m / FX) % FY, xx = x0 + m % FX;
                if (z >= a.box.D || y >= a.box.H || xx >= a.box.W) continue;
                const size_t vox = ((size_t)z * a.box.H + y) * a.box.W + xx;
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int n = nt * 8 + kk + c;
                        if (n >= a.cout) continue;
                        float v = acc[mt][nt][r * 2 + c];
                        if (a.bias) v += a.bias[n];
                        if (a.relu) v = fmaxf(v, 0.0f);
                        if (a.mask && !(__bfloat162float(a.mask[vox * a.cout + n]) > 0.0f)) v = 0.0f;
                        if (a.y_f32)
                            static_cast<float*>(a.y)[vox * a.cout + n] = v;
                        else
                            static_cast<__nv_bfloat16*>(a.y)[vox * a.cout + n] = __float2bfloat16(v);
                    }
            }
    }
}

// Per forward tile: 1 if any voxel of the tile (dilate = 0), or of the tile and its 26 neighbours
// (dilate = 1), has a nonzero mask byte.
__global__ void k_tile_flags(Box b, const uint8_t* __restrict__ mask, int dilate, uint8_t* __restrict__ flags) {
    int tx, ty;
    const int tiles = fwd_tiles(b, tx, ty);
    const int tz = tiles / (tx * ty);
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int cx = tile % tx, cy = (tile / tx) % ty, cz = tile / (tx * ty);
        const int r = dilate ? 1 : 0;
        int any = 0;
        for (int dz = -r; dz <= r && !any; ++dz)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx) {
                    const int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                    if (nx < 0 || ny < 0 || nz < 0 || nx >= tx || ny >= ty || nz >= tz) continue;
                    for (int i = threadIdx.x; i < FM; i += blockDim.x) {
                        const int z = nz * FZ + i / (FY * FX), y = ny * FY + (i / FX) % FY, xx = nx * FX + i % FX;
                        if (z < b.D && y < b.H && xx < b.W && mask[((size_t)z * b.H + y) * b.W + xx]) any = 1;
                    }
                }
        any = __syncthreads_or(any);
        if (threadIdx.x == 0) flags[tile] = any ? 1 : 0;
    }
}

size_t conv_mma_smem(int cin, int nt) {
    return (size_t)(nt * 8 * w_stride(cin) + GV * x_stride(cin)) * sizeof(__nv_bfloat16);
}

// ------------------------------------------------------------------------ BF16 weight gradient

struct WgradMma {
    Box box;
    int cin, cout;
    const __nv_bfloat16* x;   // [vox][cin]
    const __nv_bfloat16* dy;  // [vox][cout]
    float* dw;                // [27][cout][cin], zeroed before
    float* db;                // [cout], zeroed before
};

// MT m16 tiles over cout, NT n8 tiles over cin. Warp w handles taps w, w + 4, ...
template <int MT, int NT>
__global__ void __launch_bounds__(kThreads) k_wgrad_mma(WgradMma a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int cin = a.cin, xs = x_stride(cin);
    constexpr int DS = TM + 8;  // row stride of dy^T (voxels contiguous per output channel)
    float* ACC = reinterpret_cast<float*>(smem_raw);                       // [27][MT*16][NT*8]
    float* DB = ACC + 27 * MT * 16 * NT * 8;                                // [MT*16]
    __nv_bfloat16* DYs = reinterpret_cast<__nv_bfloat16*>(DB + MT * 16);   // [MT*16][DS]
    __nv_bfloat16* Xs = DYs + MT * 16 * DS;                                 // [HV][xs]
    for (int i = threadIdx.x; i < 27 * MT * 16 * NT * 8 + MT * 16; i += blockDim.x) ACC[i] = 0.0f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, kk = (lane & 3) * 2;
    for (int tile = blockIdx.x; tile < a.box.tiles(); tile += gridDim.x) {
        int z0, y0, x0;
        tile_origin(a.box, tile, z0, y0, x0);
        __syncthreads();
        stage_halo(Xs, a.x, a.box, cin, xs, z0, y0, x0);
        // dy^T of the tile's voxels (zero outside the box and for channels >= cout)
        for (int i = threadIdx.x; i < TM * MT * 16; i += blockDim.x) {
            const int m = i / (MT * 16), co = i % (MT * 16);
            const int z = z0 + m / (TY * TX), y = y0 + (m / TX) % TY, xx = x0 + m % TX;
            __nv_bfloat16 v = __float2bfloat16(0.0f);
            if (co < a.cout && z < a.box.D && y < a.box.H && xx < a.box.W)
                v = a.dy[(((size_t)z * a.box.H + y) * a.box.W + xx) * a.cout + co];
            DYs[co * DS + m] = v;
        }
        __syncthreads();
        if (threadIdx.x < a.cout) {
            float s = 0.0f;
            for (int m = 0; m < TM; ++m) s += __bfloat162float(DYs[threadIdx.x * DS + m]);
            DB[threadIdx.x] += s;
        }
        for (int t = warp; t < 27; t += 4) {
            const int off = (t / 9 * HY + (t / 3) % 3) * HX + t % 3;
            float acc[MT][NT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.0f;
#pragma unroll 2
            for (int k0 = 0; k0 < TM; k0 += 16) {
                uint32_t af[MT][4];
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const __nv_bfloat16* r0 = DYs + (mt * 16 + g) * DS + k0 + kk;
                    const __nv_bfloat16* r1 = r0 + 8 * DS;
                    af[mt][0] = lds32(r0);
                    af[mt][1] = lds32(r1);
                    af[mt][2] = lds32(r0 + 8);
                    af[mt][3] = lds32(r1 + 8);
                }
                // B[k = voxel][n = ci]: x at the voxel shifted by tap t (two voxels per register)
                int hk[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int m = k0 + kk + (q & 1) + (q >> 1) * 8;
                    hk[q] = ((m / (TY * TX)) * HY + (m / TX) % TY) * HX + m % TX + off;
                }
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    const int n = nt * 8 + g;
                    uint32_t b0 = 0u, b1 = 0u;
                    if (n < cin) {
                        b0 = pack2(Xs[hk[0] * xs + n], Xs[hk[1] * xs + n]);
                        b1 = pack2(Xs[hk[2] * xs + n], Xs[hk[3] * xs + n]);
                    }
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) mma16816(acc[mt][nt], af[mt], b0, b1);
                }
            }
            float* At = ACC + t * MT * 16 * NT * 8;
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int row = mt * 16 + g + (q >> 1) * 8, col = nt * 8 + kk + (q & 1);
                        At[row * NT * 8 + col] += acc[mt][nt][q];
                    }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 27 * a.cout * cin; i += blockDim.x) {
        const int t = i / (a.cout * cin), co = (i / cin) % a.cout, ci = i % cin;
        const float v = ACC[(t * MT * 16 + co) * NT * 8 + ci];
        if (v != 0.0f) atomicAdd(&a.dw[i], v);
    }
    if (threadIdx.x < a.cout) atomicAdd(&a.db[threadIdx.x], DB[threadIdx.x]);
}

size_t wgrad_smem(int cin, int mt, int nt) {
    return (size_t)(27 * mt * 16 * nt * 8 + mt * 16) * sizeof(float) +
           (size_t)(mt * 16 * (TM + 8) + HV * x_stride(cin)) * sizeof(__nv_bfloat16);
}

// ------------------------------------------------------------------------ FP32 reference kernels

__global__ void k_conv_f32(Box b, int cin, int cout, const float* __restrict__ x, const float* __restrict__ w,
                           const float* __restrict__ bias, int relu, float* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nvox = (size_t)b.D * b.H * b.W;
    if (i >= nvox * cout) return;
    const int co = (int)(i % cout);
    const size_t p = i / cout;
    const int xx = (int)(p % b.W), y = (int)((p / b.W) % b.H), z = (int)(p / ((size_t)b.W * b.H));
    float s = bias ? bias[co] : 0.0f;
    for (int t = 0; t < 27; ++t) {
        const int zz = z + t / 9 - 1, yy = y + (t / 3) % 3 - 1, xq = xx + t % 3 - 1;
        if (zz < 0 || zz >= b.D || yy < 0 || yy >= b.H || xq < 0 || xq >= b.W) continue;
        const float* xv = x + (((size_t)zz * b.H + yy) * b.W + xq) * cin;
        const float* wr = w + ((size_t)t * cout + co) * cin;
        for (int c = 0; c < cin; ++c) s = fmaf(xv[c], wr[c], s);
    }
    out[i] = relu ? fmaxf(s, 0.0f) : s;
}

__global__ void k_conv_bwd_data_f32(Box b, int cin, int cout, const float* __restrict__ dy,
                                    const float* __restrict__ w, const float* __restrict__ act_in,
                                    float* __restrict__ dx) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nvox = (size_t)b.D * b.H * b.W;
    if (i >= nvox * cin) return;
    const int ci = (int)(i % cin);
    const size_t q = i / cin;
    const int xx = (int)(q % b.W), y = (int)((q / b.W) % b.H), z = (int)(q / ((size_t)b.W * b.H));
    float s = 0.0f;
    for (int t = 0; t < 27; ++t) {  // dy at q - o_t
        const int zz = z - (t / 9 - 1), yy = y - ((t / 3) % 3 - 1), xq = xx - (t % 3 - 1);
        if (zz < 0 || zz >= b.D || yy < 0 || yy >= b.H || xq < 0 || xq >= b.W) continue;
        const float* d = dy + (((size_t)zz * b.H + yy) * b.W + xq) * cout;
        for (int co = 0; co < cout; ++co) s = fmaf(d[co], w[((size_t)t * cout + co) * cin + ci], s);
    }
    if (act_in && !(act_in[i] > 0.0f)) s = 0.0f;
    dx[i] = s;
}

// One CTA per (tap, out channel): threads over (in channel, voxel stripes), shared reduction.
__global__ void k_conv_bwd_weight_f32(Box b, int cin, int cout, const float* __restrict__ x,
                                      const float* __restrict__ dy, float* __restrict__ dw,
                                      float* __restrict__ db) {
    const int t = blockIdx.x / cout, co = blockIdx.x % cout;
    const int oz = t / 9 - 1, oy = (t / 3) % 3 - 1, ox = t % 3 - 1;
    const size_t nvox = (size_t)b.D * b.H * b.W;
    __shared__ float part[256];
    for (int ci = 0; ci <= cin; ++ci) {  // ci == cin: the bias gradient (tap 13 CTAs only)
        if (ci == cin && t != 13) break;
        float s = 0.0f;
        for (size_t p = threadIdx.x; p < nvox; p += blockDim.x) {
            const float g = dy[p * cout + co];
            if (ci == cin) {
                s += g;
                continue;
            }
            const int xx = (int)(p % b.W), y = (int)((p / b.W) % b.H), z = (int)(p / ((size_t)b.W * b.H));
            const int zz = z + oz, yy = y + oy, xq = xx + ox;
            if (zz < 0 || zz >= b.D || yy < 0 || yy >= b.H || xq < 0 || xq >= b.W) continue;
            s = fmaf(g, x[(((size_t)zz * b.H + yy) * b.W + xq) * cin + ci], s);
        }
        part[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (ci == cin)
                db[co] = part[0];
            else
                dw[((size_t)t * cout + co) * cin + ci] = part[0];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------ loss, optimizer, casts

__global__ void k_mask_count(int nvox, const uint8_t* __restrict__ mask, float* count) {
    float c = 0.0f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += gridDim.x * blockDim.x) c += mask[i] ? 1.0f : 0.0f;
    c += __shfl_xor_sync(0xffffffffu, c, 16);
    c += __shfl_xor_sync(0xffffffffu, c, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    if ((threadIdx.x & 31) == 0 && c != 0.0f) atomicAdd(count, c);
}

template <typename PT, typename DT>
__global__ void k_mse(int nvox, int C, const PT* __restrict__ pred, const float* __restrict__ target,
                      const uint8_t* __restrict__ mask, const float* __restrict__ count, float* loss, DT* dpred) {
    const float inv = 1.0f / fmaxf(*count * (float)C, 1.0f);
    float s = 0.0f;
    const size_t n = (size_t)nvox * C;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float d = 0.0f;
        if (mask[i / C]) {
            float p;
            if constexpr (sizeof(PT) == 2) p = __bfloat162float(pred[i]); else p = pred[i];
            d = p - target[i];
            s += d * d;
        }
        const float gd = 2.0f * d * inv;
        if constexpr (sizeof(DT) == 2) dpred[i] = __float2bfloat16(gd); else dpred[i] = gd;
    }
    s += __shfl_xor_sync(0xffffffffu, s, 16);
    s += __shfl_xor_sync(0xffffffffu, s, 8);
    s += __shfl_xor_sync(0xffffffffu, s, 4);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if ((threadIdx.x & 31) == 0 && s != 0.0f) atomicAdd(loss, s * inv);
}

__global__ void k_adam(int n, float* p, const float* g, float* m, float* v, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16* pb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16(pi);
}

__global__ void k_cast_to_bf16(int n, const float* __restrict__ s, __nv_bfloat16* __restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = __float2bfloat16(s[i]);
}

__global__ void k_cast_to_f32(int n, const __nv_bfloat16* __restrict__ s, float* __restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = __bfloat162float(s[i]);
}

// ------------------------------------------------------------------------ launch helpers

unsigned blocks_for(size_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

int persistent_ctas(int tiles, const void* kernel, size_t smem, int threads = kThreads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    return std::max(1, std::min(tiles, std::max(per_sm, 1) * std::max(sms, 1)));
}

template <int NT>
cudaError_t launch_conv_mma(const ConvMma& a, cudaStream_t s) {
    const size_t smem = conv_mma_smem(a.cin, NT);
    cudaError_t e = cudaFuncSetAttribute(k_conv_mma<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int tx, ty;
    const int tiles = fwd_tiles(a.box, tx, ty);
    const int grid = persistent_ctas(tiles, (const void*)k_conv_mma<NT>, smem, kFwdThreads);
    k_conv_mma<NT><<<grid, kFwdThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t conv_mma(const ConvMma& a, cudaStream_t s) {
    const int nt = (a.cout + 7) / 8;
    switch (nt) {
        case 1: return launch_conv_mma<1>(a, s);
        case 2: return launch_conv_mma<2>(a, s);
        case 3: return launch_conv_mma<3>(a, s);
        case 4: return launch_conv_mma<4>(a, s);
        case 5: return launch_conv_mma<5>(a, s);
        case 6: return launch_conv_mma<6>(a, s);
        case 7: return launch_conv_mma<7>(a, s);
        default: return launch_conv_mma<8>(a, s);
    }
}

template <int MT, int NT>
cudaError_t launch_wgrad(const WgradMma& a, cudaStream_t s) {
    const size_t smem = wgrad_smem(a.cin, MT, NT);
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_mma<MT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = persistent_ctas(a.box.tiles(), (const void*)k_wgrad_mma<MT, NT>, smem);
    k_wgrad_mma<MT, NT><<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int MT>
cudaError_t wgrad_nt(const WgradMma& a, cudaStream_t s) {
    switch ((a.cin + 7) / 8) {
        case 1: return launch_wgrad<MT, 1>(a, s);
        case 2: return launch_wgrad<MT, 2>(a, s);
        case 3: return launch_wgrad<MT, 3>(a, s);
        case 4: return launch_wgrad<MT, 4>(a, s);
        default: return cudaErrorInvalidValue;  // more than 32 input channels: not instantiated
    }
}

cudaError_t wgrad_mma(const WgradMma& a, cudaStream_t s) {
    switch ((a.cout + 15) / 16) {
        case 1: return wgrad_nt<1>(a, s);
        case 2: return wgrad_nt<2>(a, s);
        default: return cudaErrorInvalidValue;  // more than 32 output channels: not instantiated
    }
}

bool valid_dims(int D, int H, int W, int cin, int cout) {
    return D > 0 && H > 0 && W > 0 && cin > 0 && cout > 0 && cin <= MPM_NET_MAX_CHANNELS &&
           cout <= MPM_NET_MAX_CHANNELS && (size_t)D * H * W < (size_t)1 << 31;
}

}  // namespace
}  // namespace net
}  // namespace mpm

using namespace mpm::net;

extern "C" {

mpm_status mpm_conv3d_forward(int dtype, int D, int H, int W, int cin, int cout, const void* x, const void* w,
                              const float* bias, int relu, int y_f32, void* y, void* stream) {
    if (!valid_dims(D, H, W, cin, cout) || !x || !w || !y) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Box b = make_box(D, H, W);
    cudaError_t e;
    if (dtype == MPM_NET_F32) {
        const size_t n = (size_t)D * H * W * cout;
        k_conv_f32<<<blocks_for(n, 256), 256, 0, st>>>(b, cin, cout, static_cast<const float*>(x),
                                                        static_cast<const float*>(w), bias, relu,
                                                        static_cast<float*>(y));
        e = cudaGetLastError();
    } else if (dtype == MPM_NET_BF16) {
        ConvMma a{b, cin, cout, static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(w), 0, cin,
                  bias, relu, nullptr, y, y_f32, nullptr};
        e = conv_mma(a, st);
    } else {
        return MPM_ERR_INVALID_ARG;
    }
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_forward");
}

mpm_status mpm_conv3d_forward_tiled(int D, int H, int W, int cin, int cout, const void* x, const void* w,
                                    const float* bias, int relu, int y_f32, void* y, const uint8_t* tile_flags,
                                    void* stream) {
    if (!valid_dims(D, H, W, cin, cout) || !x || !w || !y || !tile_flags) return MPM_ERR_INVALID_ARG;
    ConvMma a{make_box(D, H, W), cin, cout, static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(w),
              0, cin, bias, relu, nullptr, y, y_f32, tile_flags};
    cudaError_t e = conv_mma(a, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_forward_tiled");
}

int mpm_conv3d_tile_count(int D, int H, int W) {
    if (D <= 0 || H <= 0 || W <= 0) return 0;
    int tx, ty;
    return fwd_tiles(make_box(D, H, W), tx, ty);
}

mpm_status mpm_conv3d_tile_flags(int D, int H, int W, const uint8_t* mask, int dilate, uint8_t* flags,
                                 void* stream) {
    if (D <= 0 || H <= 0 || W <= 0 || !mask || !flags) return MPM_ERR_INVALID_ARG;
    const Box b = make_box(D, H, W);
    int tx, ty;
    const int tiles = fwd_tiles(b, tx, ty);
    k_tile_flags<<<std::min(tiles, 4096), 256, 0, static_cast<cudaStream_t>(stream)>>>(b, mask, dilate ? 1 : 0,
                                                                                      flags);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_tile_flags");
}

mpm_status mpm_conv3d_backward_data(int dtype, int D, int H, int W, int cin, int cout, const void* dy,
                                    const void* w, const void* act_in, void* dx, void* stream) {
    if (!valid_dims(D, H, W, cin, cout) || !dy || !w || !dx) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Box b = make_box(D, H, W);
    cudaError_t e;
    if (dtype == MPM_NET_F32) {
        const size_t n = (size_t)D * H * W * cin;
        k_conv_bwd_data_f32<<<blocks_for(n, 256), 256, 0, st>>>(b, cin, cout, static_cast<const float*>(dy),
                                                                 static_cast<const float*>(w),
                                                                 static_cast<const float*>(act_in),
                                                                 static_cast<float*>(dx));
        e = cudaGetLastError();
    } else if (dtype == MPM_NET_BF16) {
        // a forward pass over dy (cout channels in) to cin channels out with flipped, transposed weights
        ConvMma a{b, cout, cin, static_cast<const __nv_bfloat16*>(dy), static_cast<const __nv_bfloat16*>(w), 1, cin,
                  nullptr, 0, static_cast<const __nv_bfloat16*>(act_in), dx, 0, nullptr};
        e = conv_mma(a, st);
    } else {
        return MPM_ERR_INVALID_ARG;
    }
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_backward_data");
}

mpm_status mpm_conv3d_backward_weight(int dtype, int D, int H, int W, int cin, int cout, const void* x,
                                      const void* dy, float* dw, float* db, void* stream) {
    if (!valid_dims(D, H, W, cin, cout) || !x || !dy || !dw || !db) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Box b = make_box(D, H, W);
    cudaError_t e;
    if (dtype == MPM_NET_F32) {
        k_conv_bwd_weight_f32<<<27 * cout, 256, 0, st>>>(b, cin, cout, static_cast<const float*>(x),
                                                        static_cast<const float*>(dy), dw, db);
        e = cudaGetLastError();
    } else if (dtype == MPM_NET_BF16) {
        if (cin > 32 || cout > 32) return MPM_ERR_INVALID_ARG;
        e = cudaMemsetAsync(dw, 0, sizeof(float) * 27 * cin * cout, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(db, 0, sizeof(float) * cout, st);
        if (e == cudaSuccess) {
            WgradMma a{b, cin, cout, static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(dy), dw,
                       db};
            e = wgrad_mma(a, st);
        }
    } else {
        return MPM_ERR_INVALID_ARG;
    }
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_backward_weight");
}

mpm_status mpm_mse_loss(int dtype, int nvox, int C, const void* pred, int pred_f32, const float* target,
                        const uint8_t* mask, float* loss, void* dpred, void* stream) {
    if (nvox <= 0 || C <= 0 || !pred || !target || !mask || !loss || !dpred) return MPM_ERR_INVALID_ARG;
    if (dtype != MPM_NET_F32 && dtype != MPM_NET_BF16) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* count = loss + 1;  // loss[0]: the loss, loss[1]: the masked voxel count
    cudaError_t e = cudaMemsetAsync(loss, 0, 2 * sizeof(float), st);
    if (e == cudaSuccess) {
        k_mask_count<<<std::min(blocks_for(nvox, 256), 1024u), 256, 0, st>>>(nvox, mask, count);
        const unsigned grid = std::min(blocks_for((size_t)nvox * C, 256), 4096u);
        if (dtype == MPM_NET_F32)
            k_mse<float, float><<<grid, 256, 0, st>>>(nvox, C, static_cast<const float*>(pred), target, mask, count,
                                                    loss, static_cast<float*>(dpred));
        else if (pred_f32)
            k_mse<float, __nv_bfloat16><<<grid, 256, 0, st>>>(nvox, C, static_cast<const float*>(pred), target, mask,
                                                            count, loss, static_cast<__nv_bfloat16*>(dpred));
        else
            k_mse<__nv_bfloat16, __nv_bfloat16><<<grid, 256, 0, st>>>(
                nvox, C, static_cast<const __nv_bfloat16*>(pred), target, mask, count, loss,
                static_cast<__nv_bfloat16*>(dpred));
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_mse_loss");
}

mpm_status mpm_adam_step(int n, float* p, const float* g, float* m, float* v, int t, float lr, float beta1,
                         float beta2, float eps, void* p_bf16, void* stream) {
    if (n <= 0 || !p || !g || !m || !v || t < 1) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float c1 = 1.0f - powf(beta1, (float)t), c2 = 1.0f - powf(beta2, (float)t);
    k_adam<<<blocks_for(n, 256), 256, 0, st>>>(n, p, g, m, v, lr, beta1, beta2, eps, c1, c2,
                                              static_cast<__nv_bfloat16*>(p_bf16));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_adam_step");
}

mpm_status mpm_cast_f32_to_bf16(int n, const float* src, void* dst, void* stream) {
    if (n <= 0 || !src || !dst) return MPM_ERR_INVALID_ARG;
    k_cast_to_bf16<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, src, static_cast<__nv_bfloat16*>(dst));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_cast_f32_to_bf16");
}

mpm_status mpm_cast_bf16_to_f32(int n, const void* src, float* dst, void* stream) {
    if (n <= 0 || !src || !dst) return MPM_ERR_INVALID_ARG;
    k_cast_to_f32<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, static_cast<const __nv_bfloat16*>(src), dst);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_cast_bf16_to_f32");
}

}  // extern "C"
