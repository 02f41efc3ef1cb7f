// mpm_noalloc.cu -- mpm_p2g_static: the particle-to-grid transfer without any device allocation.
//
// Some callers cannot call cudaMalloc: a plugin running inside a host simulator that owns every byte of
// device memory, or a real-time control loop where cudaMalloc's implicit device synchronization is not
// allowed. For them this entry point runs the bin-sorted particle-to-grid transfer with its sort scratch
// (bin keys and ranks, bin offsets, the chunk list, the sorted order) in a file-scope device array that
// the library owns, so the caller passes only its particle arrays and the output grid. The array is
// loaded with the library and stays resident on every GPU that uses it until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "mpm.h"
#include "mpm_internal.h"

using namespace mpm;

namespace {

constexpr int kStaticMaxParticles = 65536;
constexpr int kStaticMaxGrid = 64;  // nodes per axis
constexpr int kStaticMaxBins = (kStaticMaxGrid / 4) * (kStaticMaxGrid / 4) * (kStaticMaxGrid / 4);
constexpr int kStaticMaxChunks = kStaticMaxParticles / kChunk + kStaticMaxBins + 1;

constexpr size_t round256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffKeyrank = 0;
constexpr size_t kOffPerm = kOffKeyrank + round256(sizeof(uint2) * kStaticMaxParticles);
constexpr size_t kOffHist = kOffPerm + round256(sizeof(uint32_t) * kStaticMaxParticles);
constexpr size_t kOffCursor = kOffHist + round256(sizeof(uint32_t) * kStaticMaxBins);
constexpr size_t kOffChunks = kOffCursor + round256(sizeof(uint32_t) * kStaticMaxBins);
constexpr size_t kOffCounters = kOffChunks + round256(sizeof(int4) * kStaticMaxChunks);
constexpr size_t kStaticBytes = kOffCounters + 256;  // num_chunks, status (about 0.9 MB in all)

// The scratch. Host code must not use this name as an address: it is a host-side stand-in for the
// symbol. The device address comes from cudaGetSymbolAddress, once per device, and is cached for the
// life of the process: a cudaDeviceReset (or a reset of the device's primary context) reloads the module
// and may move the array, after which the cached address is stale, so this entry point must not be
// called again on that device in the same process.
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

mpm_status scratch_address(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return MPM_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return MPM_OK;
}

// Bin key and rank of every particle (position clamped into the domain first), counted per bin.
__global__ void __launch_bounds__(256) k_static_keys(Geometry g, int N, const float* __restrict__ x,
                                                     uint32_t* hist, uint2* keyrank) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t key = 0xffffffffu;
    if (p < N) {
        int b[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float xa = fminf(fmaxf(x[(size_t)a * N + p], g.lo), g.hi);
            b[a] = cell_base(xa, g.inv_dx) >> 2;
        }
        key = block_index(b[0], b[1], b[2], g.nb);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader && key != 0xffffffffu) base = atomicAdd(&hist[key], (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader) + __popc(peers & ((1u << lane) - 1u));
    if (p < N) keyrank[p] = make_uint2(key, base);
}

// Particle-to-grid transfer of the sorted particles straight into the caller's dense grid: per particle
// A = m C - dt V0 (4/dx^2) tau and, at each of its 27 nodes, m += w m_p, mv += w (m_p v + A (x_i - x_p)).
template <int KIND>
__global__ void __launch_bounds__(kChunk) k_static_p2g(Geometry g, Material mat, int N, const float* __restrict__ x,
                                                       const float* __restrict__ v, const float* __restrict__ C,
                                                       const float* __restrict__ F, const uint32_t* __restrict__ perm,
                                                       const int4* __restrict__ chunks,
                                                       const uint32_t* __restrict__ num_chunks, float4* grid) {
    const uint32_t nch = *num_chunks;
    for (uint32_t w = blockIdx.x; w < nch; w += gridDim.x) {
        const int4 ch = chunks[w];
        if ((int)threadIdx.x >= ch.z) continue;
        const uint32_t src = perm[ch.y + threadIdx.x];
        float xp[3], vp[3], Cp[3][3], tau[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xp[a] = fminf(fmaxf(x[(size_t)a * N + src], g.lo), g.hi);
            vp[a] = v ? v[(size_t)a * N + src] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Cp[r][c] = C ? C[(size_t)(r * 3 + c) * N + src] : 0.0f;
        float Fp[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Fp[r][c] = F ? F[(size_t)(r * 3 + c) * N + src] : (r == c ? 1.0f : 0.0f);
        if (KIND == MPM_PLASTICINE) {
            fixed_corotated_stress(Fp, mat, tau);
        } else {
            const float J = det3(Fp);
            const float s = mat.lambda * J * (J - 1.0f);
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) tau[r][c] = r == c ? s : 0.0f;
        }
        float A[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) A[r][c] = mat.p_mass * Cp[r][c] + mat.stress_scale * tau[r][c];
        int bs[3];
        float f[3], wt[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            bs[a] = cell_base(xp[a], g.inv_dx);
            f[a] = cell_frac(xp[a], g.inv_dx, bs[a]);
            bspline_weights(f[a], wt[a]);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float wk = wt[0][i] * wt[1][j] * wt[2][k];
                    const float d[3] = {((float)i - f[0]) * g.dx, ((float)j - f[1]) * g.dx, ((float)k - f[2]) * g.dx};
                    float mom[3];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
                        mom[r] = wk * (mat.p_mass * vp[r] + A[r][0] * d[0] + A[r][1] * d[1] + A[r][2] * d[2]);
                    const size_t node = ((size_t)(bs[0] + i) * g.n + (bs[1] + j)) * g.n + (bs[2] + k);
                    atomicAdd(&grid[node], make_float4(wk * mat.p_mass, mom[0], mom[1], mom[2]));
                }
    }
}

}  // namespace

extern "C" mpm_status mpm_p2g_static(const mpm_config* cfg, const mpm_material* mat, int n, const float* x,
                                     const float* v, const float* C, const float* F, float* grid_out,
                                     void* stream) {
    // only the fields this entry uses are checked: the grid size, dt and the material
    if (!cfg || !mat || n < 0 || (n > 0 && !x) || !grid_out) return MPM_ERR_INVALID_ARG;
    if (cfg->n < 8 || cfg->n > 256 || (cfg->n % 4) != 0) return MPM_ERR_INVALID_ARG;
    if (!(cfg->dt > 0.0f) || !std::isfinite(cfg->dt)) return MPM_ERR_INVALID_ARG;
    mpm_status r = check_material(mat);
    if (r != MPM_OK) return r;
    if (n > kStaticMaxParticles || cfg->n > kStaticMaxGrid) return MPM_ERR_CAPACITY;
    if ((reinterpret_cast<uintptr_t>(grid_out) & 15u) != 0) return MPM_ERR_INVALID_ARG;
    unsigned char* s = nullptr;
    r = scratch_address(&s);
    if (r != MPM_OK) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Geometry g{};
    g.n = cfg->n;
    g.nb = cfg->n / 4;
    g.nblocks = g.nb * g.nb * g.nb;
    g.nb_recip = 0xFFFFFFFFu / (uint32_t)g.nb + 1u;
    g.dx = (float)(1.0 / cfg->n);
    g.inv_dx = (float)cfg->n;
    g.dt = cfg->dt;
    g.lo = (float)(2.0 / cfg->n);
    g.hi = (float)(1.0 - 2.0 / cfg->n);
    double mu = 0.0, lambda = mat->bulk_modulus;
    if (mat->kind == MPM_PLASTICINE) {
        mu = (double)mat->E / (2.0 * (1.0 + mat->nu));
        lambda = (double)mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu));
    }
    Material m{};
    m.mu = (float)mu;
    m.lambda = (float)lambda;
    m.yield_radius = mu > 0.0 ? (float)(mat->yield_stress / (2.0 * mu)) : 0.0f;
    m.p_mass = (float)((double)mat->rho * mat->p_vol);
    m.stress_scale = (float)(-(double)cfg->dt * mat->p_vol * 4.0 * cfg->n * cfg->n);

    uint2* keyrank = reinterpret_cast<uint2*>(s + kOffKeyrank);
    uint32_t* perm = reinterpret_cast<uint32_t*>(s + kOffPerm);
    uint32_t* hist = reinterpret_cast<uint32_t*>(s + kOffHist);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(s + kOffCursor);
    int4* chunks = reinterpret_cast<int4*>(s + kOffChunks);
    uint32_t* num_chunks = reinterpret_cast<uint32_t*>(s + kOffCounters);

    const size_t grid_bytes = (size_t)g.n * g.n * g.n * sizeof(float4);
    if (cudaMemsetAsync(grid_out, 0, grid_bytes, st) != cudaSuccess) return MPM_ERR_CUDA;
    if (n == 0) return MPM_OK;
    // the counts must start at zero on every call: the array keeps whatever the last call (or an
    // interrupted one) left, and the first call finds it uninitialised. The scan reads the counts in
    // groups of four bins, so the group padding is cleared too. This clear must stay.
    if (cudaMemsetAsync(hist, 0, sizeof(uint32_t) * ((g.nblocks + 3) & ~3), st) != cudaSuccess) return MPM_ERR_CUDA;
    k_static_keys<<<(n + 255) / 256, 256, 0, st>>>(g, n, x, hist, keyrank);
    if (cudaGetLastError() != cudaSuccess) return MPM_ERR_CUDA;
    if (launch_scan(hist, cursor, chunks, num_chunks, g.nblocks, kChunk, st) != cudaSuccess) return MPM_ERR_CUDA;
    if (launch_assign(n, keyrank, cursor, perm, st) != cudaSuccess) return MPM_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MPM_ERR_CUDA;
    float4* grid = reinterpret_cast<float4*>(grid_out);
    if (mat->kind == MPM_PLASTICINE)
        k_static_p2g<MPM_PLASTICINE><<<sms * 4, kChunk, 0, st>>>(g, m, n, x, v, C, F, perm, chunks, num_chunks, grid);
    else
        k_static_p2g<MPM_FLUID><<<sms * 4, kChunk, 0, st>>>(g, m, n, x, v, C, F, perm, chunks, num_chunks, grid);
    if (cudaGetLastError() != cudaSuccess) return MPM_ERR_CUDA;
    return MPM_OK;
}
