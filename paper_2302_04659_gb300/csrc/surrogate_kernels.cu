// surrogate_kernels.cu -- grid-side kernels of the learned surrogate window (an extension of the method:
// the paper's simulator has no learned component). A window replaces k substeps by one plain grid update,
// a network correction of the updated node velocities, and one grid-to-particle transfer with time step
// k*dt. These kernels read the network input off the updated grid, add the network's correction back,
// and sum the mass and momentum the fallback gate compares.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mpm_internal.h"

namespace mpm {
namespace {

constexpr uint32_t kLocalMask = (1u << kLocalBinBits) - 1u;

// The block's totals of v[0..NV), left in thread 0's v (warps shuffle, then warp 0 sums the warps').
template <int NV>
__device__ __forceinline__ void block_pair_sum(Pair (&v)[NV], Pair (&part)[32][NV]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[q] = pair_add(v[q], pair_shfl_xor(v[q], off));
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) part[warp][q] = v[q];
    __syncthreads();
    if (warp == 0) {  // warp 0 ends with the block's totals in v (lane 0 reads them)
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            Pair t = lane < nw ? part[lane][q] : Pair{0.0f, 0.0f};
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t = pair_add(t, pair_shfl_xor(t, off));
            v[q] = t;
        }
    }
}

// Block-wide sum of NV pairs (blockDim a multiple of 32, at most 1024) added to out[NV] (FP64) without
// contended atomics: each block stores its total in partials[block][NV]; the last block to finish
// (ticket) sums the blocks' totals, adds them to out and resets the ticket. Returns true in that last
// block (all of its threads), after out is written.
template <int NV>
__device__ __forceinline__ bool block_sum_last(Pair (&v)[NV], Pair* partials, uint32_t* ticket, double* out) {
    __shared__ Pair part[32][NV];
    __shared__ bool last;
    block_pair_sum<NV>(v, part);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) partials[(size_t)blockIdx.x * NV + q] = v[q];
        __threadfence();  // the totals are visible before the ticket is taken
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // the blocks' totals, spread over the threads (L2 reads, all in flight), then the same block sum
    Pair t[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) t[q] = Pair{0.0f, 0.0f};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const float2 u = __ldcg(reinterpret_cast<const float2*>(&partials[(size_t)b * NV + q]));
            t[q] = pair_add(t[q], Pair{u.x, u.y});
        }
    __syncthreads();  // part[] is reused
    block_pair_sum<NV>(t, part);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) out[q] += pair_value(t[q]);
        *ticket = 0u;
    }
    __syncthreads();
    return true;
}

// Block-wide sum of NV pairs added to out[NV] (FP64) by one atomic per component per block: for sums that
// nothing in the same launch waits on.
template <int NV>
__device__ __forceinline__ void block_sum_atomic(Pair (&v)[NV], double* out) {
    __shared__ Pair part[32][NV];
    block_pair_sum<NV>(v, part);
    if (threadIdx.x == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q)
            if (v[q].hi != 0.0f) atomicAdd(&out[q], pair_value(v[q]));
}

// Bin bounds of the active bins (the grid's bin list), one block: box[0..2] = min bin per axis,
// box[3..5] = max (box[3] = -1 when there are none).
__global__ void k_sur_box(const uint32_t* __restrict__ list, const uint32_t* __restrict__ count, int nb, int* box) {
    const uint32_t n = *count;
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int b = (int)(list[i] & kLocalMask);
        const int c[3] = {b / (nb * nb), (b / nb) % nb, b % nb};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = min(lo[a], c[a]);
            hi[a] = max(hi[a], c[a]);
        }
    }
    __shared__ int red[6][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], off));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], off));
        }
        if (lane == 0) {
            red[a][warp] = lo[a];
            red[3 + a][warp] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int q = threadIdx.x;
        int v = q < 3 ? (1 << 30) : -1;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = q < 3 ? min(v, red[q][w]) : max(v, red[q][w]);
        box[q] = v;
    }
}

// The start of a gated step: save the body impulses and the substep count, clear the step's flag.
__global__ void k_sur_step_begin(const double* wrench, double* wrench_saved, int n6, const uint32_t* counter,
                                 uint32_t* words) {
    for (int i = threadIdx.x; i < n6; i += blockDim.x) wrench_saved[i] = wrench[i];
    if (threadIdx.x == 0) {
        words[0] = 0u;        // a window failed the gate
        words[1] = *counter;  // the substep count at the start
    }
}

// Undo a step's bookkeeping: the impulses and the substep count as they were at its start.
__global__ void k_sur_step_restore(double* wrench, const double* wrench_saved, int n6, uint32_t* counter,
                                   const uint32_t* words) {
    for (int i = threadIdx.x; i < n6; i += blockDim.x) wrench[i] = wrench_saved[i];
    if (threadIdx.x == 0) *counter = words[1];
}

// Mass and momentum of the transfer, before the grid update (nodes hold (m, m v)), into sums[0..4), and
// sum_i |m v_i|^2 / m_i (twice the nodes' kinetic energy) into sums[kSumK0].
__global__ void k_sur_moments(const float4* __restrict__ grid, const uint32_t* __restrict__ list,
                              const uint32_t* __restrict__ count, double* sums) {
    const uint32_t n = *count;
    Pair v[4] = {};
    Pair ke[1] = {};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n * kBlkNodes; i += gridDim.x * blockDim.x) {
        const uint32_t b = list[i / kBlkNodes] & kLocalMask;
        const float4 g = grid[(size_t)b * kBlkNodes + i % kBlkNodes];
        v[0] = pair_add(v[0], g.x);
        v[1] = pair_add(v[1], g.y);
        v[2] = pair_add(v[2], g.z);
        v[3] = pair_add(v[3], g.w);
        if (g.x > 0.0f) ke[0] = pair_add(ke[0], (g.y * g.y + g.z * g.z + g.w * g.w) / g.x);
    }
    block_sum_atomic<4>(v, sums);
    block_sum_atomic<1>(ke, sums + kSumK0);
}

__device__ __forceinline__ bool box_node(const SurBox& b, size_t t, int& i, int& j, int& k) {
    k = b.k0 + (int)(t % b.W);
    j = b.j0 + (int)((t / b.W) % b.H);
    i = b.i0 + (int)(t / ((size_t)b.W * b.H));
    return true;
}

// Network input over the box from the updated grid (nodes hold (v, m)): (m * m_scale, v * v_scale),
// the mass mask, and the momentum sum of the updated grid.
__global__ void k_sur_features(const float4* __restrict__ grid, int n, int nb, SurBox box, float m_scale,
                               float v_scale, float* __restrict__ feat, __nv_bfloat16* __restrict__ feat_bf16,
                               uint8_t* __restrict__ mask, double* sums) {
    const size_t nv = (size_t)box.D * box.H * box.W;
    Pair p[3] = {};
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (size_t)gridDim.x * blockDim.x) {
        int i, j, k;
        box_node(box, t, i, j, k);
        float4 g = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (i >= 0 && i < n && j >= 0 && j < n && k >= 0 && k < n) g = grid[node_index(i, j, k, nb)];
        const float m = g.w;
        const float4 f = make_float4(m * m_scale, g.x * v_scale, g.y * v_scale, g.z * v_scale);
        if (feat) reinterpret_cast<float4*>(feat)[t] = f;
        if (feat_bf16) {  // the network input, 8 bytes per node
            const __nv_bfloat162 lo = __floats2bfloat162_rn(f.x, f.y), hi = __floats2bfloat162_rn(f.z, f.w);
            reinterpret_cast<uint2*>(feat_bf16)[t] = make_uint2(*reinterpret_cast<const uint32_t*>(&lo),
                                                                *reinterpret_cast<const uint32_t*>(&hi));
        }
        mask[t] = m > 0.0f ? 1 : 0;
        p[0] = pair_add(p[0], m * g.x);
        p[1] = pair_add(p[1], m * g.y);
        p[2] = pair_add(p[2], m * g.z);
    }
    if (sums) block_sum_atomic<3>(p, sums);
}

__device__ __forceinline__ bool in_wall(int i, int j, int k, int n, int bound) {
    const int hi = n - bound;
    return i < bound || j < bound || k < bound || i >= hi || j >= hi || k >= hi;
}

// The corrected velocity of a node: v + dv * unit where it has mass, zero in the sticky wall band.
// apply != 0 writes it back; the momentum of the corrected grid is summed either way.
__global__ void k_sur_correct(float4* __restrict__ grid, int n, int nb, int bound, SurBox box,
                              const float* __restrict__ dv, float unit, int apply, double* sums) {
    const size_t nv = (size_t)box.D * box.H * box.W;
    Pair p[3] = {};
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (size_t)gridDim.x * blockDim.x) {
        int i, j, k;
        box_node(box, t, i, j, k);
        if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n) continue;
        float4* node = &grid[node_index(i, j, k, nb)];
        float4 g = *node;
        if (!(g.w > 0.0f)) continue;
        const float* d = dv + t * 3;
        float v[3] = {g.x + d[0] * unit, g.y + d[1] * unit, g.z + d[2] * unit};
        if (in_wall(i, j, k, n, bound)) v[0] = v[1] = v[2] = 0.0f;
        p[0] = pair_add(p[0], g.w * v[0]);
        p[1] = pair_add(p[1], g.w * v[1]);
        p[2] = pair_add(p[2], g.w * v[2]);
        if (apply) *node = make_float4(v[0], v[1], v[2], g.w);
    }
    block_sum_atomic<3>(p, sums);
}

// The gate in one launch: the corrected grid's momentum summed like k_sur_correct (without writing it
// back), then the last block to finish computes the residuals, sets the gate, records the stats, and
// zeroes the sums for the next window (so no separate clearing is needed).
struct GateArgs {
    const float4* grid;
    int n, nb, bound;
    SurBox box;
    const float* dv;
    float unit;
    double* sums;            // M, P0[3] (k_sur_moments), P1[3] (k_sur_features), P_hat[3] (here), K0
    double m_particles, v_ref, threshold;
    int k;
    uint32_t* gate;
    unsigned long long* stats;
    uint32_t* any_failed;    // per-step mode, or null
    uint32_t* ticket;
    Pair* partials;           // per-block totals (kReduceBlocks x 3)
};

// The residuals of a window from its sums S = (M, P0[3], P1[3], P_hat[3], K0): the grid mass against the
// particles', and the corrected grid's momentum against the momentum the first substep's change predicts
// for the window, P0 + (k + 1)/2 (P1 - P0), relative to M v_ref. v_ref = 0 takes the scene's own velocity
// scale, the mass-weighted RMS node speed of the transfer sqrt(K0 / M) (K0 = sum_i |m v_i|^2 / m_i).
__device__ __forceinline__ void window_residuals(const double* S, double m_particles, int k, double v_ref,
                                                 double& r_mass, double& r_mom) {
    const double M = S[0];
    if (!(v_ref > 0.0)) v_ref = M > 0.0 && S[kSumK0] > 0.0 ? sqrt(S[kSumK0] / M) : 1e-30;
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double pexp = S[1 + a] + 0.5 * (k + 1) * (S[4 + a] - S[1 + a]);
        d2 += (S[7 + a] - pexp) * (S[7 + a] - pexp);
    }
    r_mass = m_particles > 0.0 ? fabs(M - m_particles) / m_particles : 0.0;
    r_mom = M > 0.0 ? sqrt(d2) / (M * v_ref) : 0.0;
}

// The gate's decision from the complete sums: residuals, gate word, stats; the sums are zeroed for the
// next window. One thread.
__device__ void gate_decide(const GateArgs& g) {
    double S[kSumWindow];
    for (int q = 0; q < kSumWindow; ++q) S[q] = __ldcg(&g.sums[q]);
    double r_mass, r_mom;
    window_residuals(S, g.m_particles, g.k, g.v_ref, r_mass, r_mom);
    const bool ok = r_mass <= g.threshold && r_mom <= g.threshold;  // a NaN residual fails
    *g.gate = ok ? 1u : 0u;
    if (!ok && g.any_failed) *g.any_failed = 1u;
    g.stats[0] += 1ull;
    if (!ok && !g.any_failed) g.stats[1] += 1ull;
    reinterpret_cast<double*>(g.stats)[2] = r_mass;
    reinterpret_cast<double*>(g.stats)[3] = r_mom;
    for (int q = 0; q < kSumWindow; ++q) g.sums[q] = 0.0;
}

__global__ void k_sur_check_gate(GateArgs g) {
    const size_t nv = (size_t)g.box.D * g.box.H * g.box.W;
    Pair p[3] = {};
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (size_t)gridDim.x * blockDim.x) {
        int i, j, k;
        box_node(g.box, t, i, j, k);
        if (i < 0 || i >= g.n || j < 0 || j >= g.n || k < 0 || k >= g.n) continue;
        const float4 gv = g.grid[node_index(i, j, k, g.nb)];
        if (!(gv.w > 0.0f)) continue;
        const float* d = g.dv + t * 3;
        float v[3] = {gv.x + d[0] * g.unit, gv.y + d[1] * g.unit, gv.z + d[2] * g.unit};
        if (in_wall(i, j, k, g.n, g.bound)) v[0] = v[1] = v[2] = 0.0f;
        p[0] = pair_add(p[0], gv.w * v[0]);
        p[1] = pair_add(p[1], gv.w * v[1]);
        p[2] = pair_add(p[2], gv.w * v[2]);
    }
    if (!block_sum_last<3>(p, g.partials, g.ticket, g.sums + 7) || threadIdx.x != 0) return;
    gate_decide(g);
}

// Body impulses over a window: the first substep's share, counted k times in all.
__global__ void k_wrench_extrapolate(double* wrench, const double* before, int n6, double extra,
                                     const uint32_t* gate, uint32_t gate_run) {
    if (gate && *gate != gate_run) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n6) wrench[i] += extra * (wrench[i] - before[i]);
}

// The fallback gate of a window, on the device (one thread).
__global__ void k_sur_gate(const double* sums, double m_particles, int k, double v_ref, double threshold,
                           uint32_t* gate, unsigned long long* stats, uint32_t* any_failed) {
    double r_mass, r_mom;
    window_residuals(sums, m_particles, k, v_ref, r_mass, r_mom);
    const bool ok = r_mass <= threshold && r_mom <= threshold;  // a NaN residual fails
    *gate = ok ? 1u : 0u;
    if (!ok && any_failed) *any_failed = 1u;  // per-step fallback: the host counts the redone windows
    stats[0] += 1ull;
    if (!ok && !any_failed) stats[1] += 1ull;
    reinterpret_cast<double*>(stats)[2] = r_mass;
    reinterpret_cast<double*>(stats)[3] = r_mom;
}

// The per-step gate over the windows of a step, one warp: window w's sums are slots[kSumWindow w ..]; a window
// that fails marks the step (any_failed) for a plain redo. The stats count the windows and keep the last
// window's residuals; the slots are zeroed for the next step.
__global__ void k_sur_decide(double* slots, int nwin, double m_particles, int k, double v_ref, double threshold,
                             unsigned long long* stats, uint32_t* any_failed) {
    const int lane = threadIdx.x;
    bool failed = false;
    for (int w0 = 0; w0 < nwin; w0 += 32) {
        const int w = w0 + lane;
        if (w < nwin) {
            double* S = slots + (size_t)w * kSumWindow;
            double r_mass, r_mom;
            window_residuals(S, m_particles, k, v_ref, r_mass, r_mom);
            failed |= !(r_mass <= threshold && r_mom <= threshold);  // a NaN residual fails
            if (w == nwin - 1) {
                reinterpret_cast<double*>(stats)[2] = r_mass;
                reinterpret_cast<double*>(stats)[3] = r_mom;
            }
#pragma unroll
            for (int q = 0; q < kSumWindow; ++q) S[q] = 0.0;
        }
    }
    if (__any_sync(0xffffffffu, failed) && lane == 0) *any_failed = 1u;
    if (lane == 0) stats[0] += (unsigned long long)nwin;
}

// The corrected velocities written back (when the gate passed, if there is one); block 0 also advances
// the substep counter by k - 1 (the grid update before it counted the first) and counts the first substep's
// body impulses k times. With sums, the corrected grid's momentum is added to sums[0..3).
__global__ void k_sur_apply_gated(float4* __restrict__ grid, int n, int nb, int bound, SurBox box,
                                  const float* __restrict__ dv, float unit, const uint32_t* gate, uint32_t* counter,
                                  int k, double* wrench, const double* wrench_before, int n6, double* sums) {
    if (gate && *gate != 1u) return;
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) *counter += (uint32_t)(k - 1);
        for (int i = threadIdx.x; i < n6; i += blockDim.x) wrench[i] += (double)(k - 1) * (wrench[i] - wrench_before[i]);
    }
    const size_t nv = (size_t)box.D * box.H * box.W;
    Pair p[3] = {};
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nv; t += (size_t)gridDim.x * blockDim.x) {
        int i, j, k;
        box_node(box, t, i, j, k);
        if (i < 0 || i >= n || j < 0 || j >= n || k < 0 || k >= n) continue;
        float4* node = &grid[node_index(i, j, k, nb)];
        const float4 g = *node;
        if (!(g.w > 0.0f)) continue;
        const float* d = dv + t * 3;
        float v[3] = {g.x + d[0] * unit, g.y + d[1] * unit, g.z + d[2] * unit};
        if (in_wall(i, j, k, n, bound)) v[0] = v[1] = v[2] = 0.0f;
        if (sums) {  // (uniform)
            p[0] = pair_add(p[0], g.w * v[0]);
            p[1] = pair_add(p[1], g.w * v[1]);
            p[2] = pair_add(p[2], g.w * v[2]);
        }
        *node = make_float4(v[0], v[1], v[2], g.w);
    }
    if (sums) block_sum_atomic<3>(p, sums);
}

__global__ void k_cast_bf16(int n, const float* __restrict__ s, __nv_bfloat16* __restrict__ d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = __float2bfloat16(s[i]);
}

unsigned grid_for(size_t n, int threads, unsigned cap) {
    size_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

cudaError_t launch_sur_box(const uint32_t* list, const uint32_t* count, int nb, int nbins_cap, int* box,
                           cudaStream_t s) {
    (void)nbins_cap;
    k_sur_box<<<1, 1024, 0, s>>>(list, count, nb, box);
    return cudaGetLastError();
}

cudaError_t launch_sur_step_begin(const double* wrench, double* saved, int n6, const uint32_t* counter, uint32_t* words,
                                  cudaStream_t s) {
    k_sur_step_begin<<<1, 256, 0, s>>>(wrench, saved, n6, counter, words);
    return cudaGetLastError();
}

cudaError_t launch_sur_step_restore(double* wrench, const double* saved, int n6, uint32_t* counter,
                                    const uint32_t* words, cudaStream_t s) {
    k_sur_step_restore<<<1, 256, 0, s>>>(wrench, saved, n6, counter, words);
    return cudaGetLastError();
}

cudaError_t launch_sur_moments(const float4* grid, const uint32_t* list, const uint32_t* count, int nbins_cap,
                               double* sums, cudaStream_t s) {
    k_sur_moments<<<grid_for((size_t)nbins_cap * kBlkNodes, 256, kReduceBlocks), 256, 0, s>>>(grid, list, count, sums);
    return cudaGetLastError();
}

cudaError_t launch_sur_features(const float4* grid, int n, int nb, const SurBox& box, float m_scale,
                                float v_scale, float* feat, uint8_t* mask, double* sums, cudaStream_t s,
                                void* feat_bf16) {
    const size_t nv = (size_t)box.D * box.H * box.W;
    k_sur_features<<<grid_for(nv, 256, kReduceBlocks), 256, 0, s>>>(grid, n, nb, box, m_scale, v_scale, feat,
                                                                    static_cast<__nv_bfloat16*>(feat_bf16), mask, sums);
    return cudaGetLastError();
}

cudaError_t launch_sur_correct(float4* grid, int n, int nb, int bound, const SurBox& box, const float* dv,
                               float unit, int apply, double* sums, cudaStream_t s) {
    const size_t nv = (size_t)box.D * box.H * box.W;
    k_sur_correct<<<grid_for(nv, 256, kReduceBlocks), 256, 0, s>>>(grid, n, nb, bound, box, dv, unit, apply, sums);
    return cudaGetLastError();
}

cudaError_t launch_wrench_extrapolate(double* wrench, const double* before, int n6, double extra, cudaStream_t s,
                                      const uint32_t* gate, uint32_t gate_run) {
    if (n6 <= 0) return cudaSuccess;
    k_wrench_extrapolate<<<(n6 + 255) / 256, 256, 0, s>>>(wrench, before, n6, extra, gate, gate_run);
    return cudaGetLastError();
}

cudaError_t launch_sur_gate(const double* sums, double m_particles, int k, double v_ref, double threshold,
                            uint32_t* gate, unsigned long long* stats, cudaStream_t s, uint32_t* any_failed) {
    k_sur_gate<<<1, 1, 0, s>>>(sums, m_particles, k, v_ref, threshold, gate, stats, any_failed);
    return cudaGetLastError();
}

cudaError_t launch_sur_check_gate(const float4* grid, int n, int nb, int bound, const SurBox& box, const float* dv,
                                  float unit, double* sums, double m_particles, int k, double v_ref, double threshold,
                                  uint32_t* gate, unsigned long long* stats, uint32_t* any_failed,
                                  const ReduceScratch& r, cudaStream_t s) {
    const size_t nv = (size_t)box.D * box.H * box.W;
    GateArgs g{grid, n, nb, bound, box, dv, unit, sums, m_particles, v_ref, threshold, k, gate, stats, any_failed,
               r.ticket, r.partials};
    k_sur_check_gate<<<grid_for(nv, 256, kReduceBlocks), 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_sur_decide(double* slots, int nwin, double m_particles, int k, double v_ref, double threshold,
                              unsigned long long* stats, uint32_t* any_failed, cudaStream_t s) {
    k_sur_decide<<<1, 32, 0, s>>>(slots, nwin, m_particles, k, v_ref, threshold, stats, any_failed);
    return cudaGetLastError();
}

cudaError_t launch_sur_apply(float4* grid, int n, int nb, int bound, const SurBox& box, const float* dv, float unit,
                             const uint32_t* gate, uint32_t* counter, int k, double* wrench,
                             const double* wrench_before, int n6, cudaStream_t s, double* sums) {
    const size_t nv = (size_t)box.D * box.H * box.W;
    k_sur_apply_gated<<<grid_for(nv, 256, 2048), 256, 0, s>>>(grid, n, nb, bound, box, dv, unit, gate, counter, k,
                                                              wrench, wrench_before, n6, sums);
    return cudaGetLastError();
}

cudaError_t launch_cast_to_bf16(int n, const float* src, void* dst, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_cast_bf16<<<(n + 255) / 256, 256, 0, s>>>(n, src, static_cast<__nv_bfloat16*>(dst));
    return cudaGetLastError();
}

}  // namespace mpm
