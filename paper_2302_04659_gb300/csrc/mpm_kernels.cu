// mpm_kernels.cu -- the CUDA kernels of the MLS-MPM substep (FP32, sm_103a).
//
// One substep (Algorithm 1's soft step: particle to grid, grid velocity, grid to particle, particle
// integration) of every environment (env) of a handle runs as two launches:
//   k_assign_grid   sorted slot of every particle of the state the previous launch wrote (counting sort
//                   into 4^3-node bins), and the grid update of the transfer it scattered:
//                   v = mv/m + dt g, box/capsule Coulomb contact with per-body impulse sums, sticky walls;
//                   zeroes the previous grid's active bins
//   k_g2p2g         per chunk of a bin: gather v and C from a shared-memory tile of the updated grid,
//                   advect, update F with the plastic return map (or J), and in the same pass scatter the
//                   new state's mass and momentum (with its stress) into a shared-memory tile of the next
//                   grid, flushed with vector atomics; counts the new bins, and its last CTA scans them
//                   (with many bins, k_scan_tiles + k_scan_apply do that instead)
// Fusing grid-to-particle with the next substep's particle-to-grid (the "G2P2G" pattern of Wang et
// al. 2020) reads each particle's x and F once per substep and its v, C not at all: they are
// recomputed by the gather. k_p2g is the standalone transfer used after the state is replaced.
#include <cuda_runtime.h>

#include <algorithm>

#include "mpm_device.cuh"
#include "mpm_internal.h"

namespace mpm {

namespace {

// Local bin of a position in an env's grid.
__device__ __forceinline__ uint32_t local_bin_of(const float x[3], const Geometry& g) {
    int b0 = cell_base(x[0], g.inv_dx) >> 2;
    int b1 = cell_base(x[1], g.inv_dx) >> 2;
    int b2 = cell_base(x[2], g.inv_dx) >> 2;
    return block_index(b0, b1, b2, g.nb);
}

// Clamp a coordinate into [lo, hi]; a NaN goes to lo. Returns flag bits.
__device__ __forceinline__ uint32_t clamp_coord(float& x, float lo, float hi) {
    uint32_t f = 0;
    if (!isfinite(x)) f |= 0x2u;
    if (!(x >= lo) || !(x <= hi)) f |= 0x1u;
    x = fminf(fmaxf(x, lo), hi);
    return f;
}

// Programmatic dependent launch: the two per-substep kernels are launched so that the next one may be
// scheduled while the previous one drains. A kernel waits for its predecessor's completion (and memory)
// before touching its outputs, and releases its successor once its own main work is issued.
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void release_successor() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Warp-aggregated histogram increment; every lane of the warp must call it (key = ~0u: no count).
// Returns the lane's rank among all particles counted into the same key (when want_base).
__device__ __forceinline__ uint32_t warp_hist_add(uint32_t* hist, uint32_t key, bool want_base) {
    uint32_t peers = __match_any_sync(0xffffffffu, key);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader && key != 0xffffffffu) base = atomicAdd(&hist[key], (uint32_t)__popc(peers));
    if (want_base) {
        base = __shfl_sync(0xffffffffu, base, leader);
        base += __popc(peers & ((1u << lane) - 1u));
    }
    return base;
}

// Env of particle p (caller order): the last env whose first particle is <= p.
__device__ __forceinline__ int env_of_particle(const EnvDesc* envs, int nenv, uint32_t p) {
    int lo = 0, hi = nenv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (envs[mid].part_first <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Copy an env descriptor into shared memory (threads 0..19).
__device__ __forceinline__ void load_env(EnvDesc& dst, const EnvDesc* envs, int e) {
    static_assert(sizeof(EnvDesc) % 4 == 0, "EnvDesc is copied as words");
    constexpr int kWords = (int)(sizeof(EnvDesc) / 4);
    if ((int)threadIdx.x < kWords)
        reinterpret_cast<uint32_t*>(&dst)[threadIdx.x] = reinterpret_cast<const uint32_t*>(envs + e)[threadIdx.x];
}

// ------------------------------------------------------------------------ scatter tile
//
// The particle-to-grid scatter of one chunk (at most kChunk particles of one bin) goes into a shared
// tile of the 8^3 nodes its particles can reach, accumulated with 32-bit integer atomics: shared-memory
// integer adds are single native instructions, FP32 ones are not. Values are fixed point:
//   mass      sum of weights, scaled by 2^22 (a node sums at most kChunk = 256 weights <= 0.75^3 each, so
//             the sum stays below 108 * 2^22 < 2^31);
//   momentum  scaled by 2^k with k = 22 - e, where 2^e bounds (from above, within a factor 2) the largest
//             per-particle magnitude B_p = max_a (m |v_a| + 1.5 dx sum_c |A_ac|) of the chunk, so every node
//             sum stays below 108 * 2^22 as well. Rounding is then at most 2^-23 of that bound per term.
// A chunk has two such tiles. The chunk records which FP32 exponents its particles' bounds B_p take (a
// 256-bit map); particles whose exponent lies more than kSlowShift below the largest go to the second
// tile, scaled from the largest exponent among them. A slow particle sharing a chunk with a fast one
// (material at rest beside a moving tool) is then rounded relative to the slow particles' range, not the
// fast one's: a term is rounded at most 2^-18 of its particle's bound in the first tile (its bounds lie
// within 2^5 of the largest), and relative to the largest slow bound in the second.
// Every scaled term a b is below 2^22, so one FP32 fused multiply-add rounds it to an integer:
// a b + 1.5 * 2^23 lands where one unit is one ulp, so the low mantissa bits hold round-to-nearest-even
// of the exact product, offset by the bit pattern 0x4B400000 of the constant, which is subtracted.
// The tiles are flushed in FP32 with one 16-byte vector atomic per touched node, and zeroed as they are
// read, so a chunk finds them clear.

constexpr int kMassBits = 22;
constexpr int kSlowShift = 4;  // a bound whose exponent field is this far below the chunk's largest is slow

// Layers of the class-layered order a chunk gives the particles that stay in its bin: one per particle
// of a class at most, so as many as a chunk holds particles.
constexpr int kLayers = kChunk;

// Tile storage: node (lx, ly, lz) of a chunk's tile sits at slot lx * kPitchX + ly * kPitchY + lz, with
// kPitchX = 4 (mod 32). The 64 cells (c0, c1, c2) of a bin then start at bank 4 (c0 + 2 c1) + c2 (mod 32):
// two cells per bank, so for any one stencil offset the nodes of particles in 32 different bank classes
// ((c0 + 2 c1) mod 8, c2) fall in 32 different banks. The map is additive, so a particle's 27 nodes are
// one base register plus compile-time offsets.
constexpr int kPitchY = 8;
constexpr int kPitchX = 68;
constexpr int kScatterSlots = 7 * kPitchX + 7 * kPitchY + 8;  // 540, a multiple of 4 (cleared as int4)
constexpr int kGatherSlots = 5 * kPitchX + 5 * kPitchY + 6;   // 386: the 6^3 gather tile

__device__ __forceinline__ int tile_slot(int lx, int ly, int lz) { return lx * kPitchX + ly * kPitchY + lz; }

// Bank class of cell (c0, c1, c2) of a bin (each in 0..3).
__device__ __forceinline__ uint32_t bank_class(int c0, int c1, int c2) {
    return ((uint32_t)((c0 + 2 * c1) & 7) << 2) | (uint32_t)c2;
}

struct __align__(16) ScatterTile {
    int q[2][4][kScatterSlots];  // [fast, slow tile][m, mx, my, mz][slot]
    uint32_t touched[27];
    uint32_t expo_map[8];  // bit e set: some particle of the chunk has a bound B_p with FP32 exponent field e
    uint32_t class_count[32];      // staying particles per bank class so far
    uint32_t layer_mask[kLayers];  // per layer, its classes
    uint32_t stay_base;            // the staying group's first rank in the bin
};

__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// Scale exponent k for bounds whose FP32 exponent field is at most `field` (clamped so 2^k and 2^-k stay
// normal): such a bound is below 2^e with e = field - 126, and k = 22 - e.
__device__ __forceinline__ int momentum_scale_exp(int field) {
    const int k = kMassBits - (field - 126);
    return min(max(k, -100), 100);
}

// B_p: bound on |m v_a + (A (x_i - x_p))_a| over the 27 nodes, (x_i - x_p) within 1.5 dx per axis.
__device__ __forceinline__ float particle_bound(float m, const float vn[3], const float (&A)[3][3], float dx) {
    float b = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float r = fmaf(1.5f * dx, fabsf(A[a][0]) + fabsf(A[a][1]) + fabsf(A[a][2]), m * fabsf(vn[a]));
        b = fmaxf(b, r);
    }
    return b;
}

// Flag global bin b of the output grid as active; the thread that sets the flag appends the packed
// (env, local bin) entry to the bin list.
__device__ __forceinline__ void mark_bin(const TransferParams& p, uint32_t b, uint32_t entry) {
    if (__ldcg(&p.flags_out[b]) == 0u && atomicExch(&p.flags_out[b], 1u) == 0u)
        p.list_out[atomicAdd(p.list_count_out, 1u)] = entry;
}

// Scatter one particle's mass and momentum to its 27 nodes: mom(node) = w (m v + A (x_i - x_p)),
// expanded per node index as base_mom + i Ad0 + j Ad1 + k Ad2 with Ad[c] = dx * column c of A.
// The tile covers nodes [o, o+8) per axis with o = 4 * bin - 1; a particle outside it (one that moved a
// cell or more since it was binned) updates the global grid directly in FP32 and marks the bins it
// touches. Returns flag bits.
__device__ __forceinline__ uint32_t scatter_particle(ScatterTile& T, const TransferParams& p, const EnvDesc& E,
                                                     int env, const int o[3], const float xn[3], const float vn[3],
                                                     const float (&A)[3][3], int tile, float mscale) {
    const Geometry& g = E.geo;
    int bs[3];
    float f[3], w[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        bs[a] = cell_base(xn[a], g.inv_dx);
        f[a] = cell_frac(xn[a], g.inv_dx, bs[a]);
        bspline_weights(f[a], w[a]);
    }
    const float m = E.mat.p_mass;
    const int l0 = bs[0] - o[0], l1 = bs[1] - o[1], l2 = bs[2] - o[2];
    const bool in_tile = (unsigned)l0 <= 5u && (unsigned)l1 <= 5u && (unsigned)l2 <= 5u;
    // In the tile the momentum terms are in the chunk's fixed-point units: the scale folds into dx and m.
    const float su = in_tile ? g.dx * mscale : g.dx, sm = in_tile ? m * mscale : m;
    float Ad[3][3];  // Ad[c] = su * column c of A; the y and z rows as pairs
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Ad[c][0] = su * A[0][c];
        const float2 yz = __fmul2_rn(make_float2(su, su), make_float2(A[1][c], A[2][c]));
        Ad[c][1] = yz.x;
        Ad[c][2] = yz.y;
    }
    float bm[3];
    {
        float2 byz = __fmul2_rn(make_float2(sm, sm), make_float2(vn[1], vn[2]));
        float bx = sm * vn[0];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            byz = __ffma2_rn(make_float2(-f[c], -f[c]), make_float2(Ad[c][1], Ad[c][2]), byz);
            bx = fmaf(-f[c], Ad[c][0], bx);
        }
        bm[0] = bx;
        bm[1] = byz.x;
        bm[2] = byz.y;
    }
    if (in_tile) {
        // Node (i, j, k) receives round(w 2^22) and round(w m_k) with m_k = bm + i Ad0 + j Ad1 + k Ad2 (scaled).
        // Packed FP32x2 pairs: (mass, x) with the pair (2^22, m_k.x), and (y, z); each lane is rounded as
        // a scalar fused multiply-add would round it.
        const float wscale = pow2f(kMassBits);
        const float2 magic = make_float2(12582912.0f, 12582912.0f);
        const float2 ad2x = make_float2(0.0f, Ad[2][0]);
        const float2 ad2yz = make_float2(Ad[2][1], Ad[2][2]);
        int* tm = T.q[tile][0] + tile_slot(l0, l1, l2);
        int* tx = T.q[tile][1] + tile_slot(l0, l1, l2);
        int* ty = T.q[tile][2] + tile_slot(l0, l1, l2);
        int* tz = T.q[tile][3] + tile_slot(l0, l1, l2);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float wij = w[0][i] * w[1][j];
                const float2 mx = make_float2(wscale, bm[0] + i * Ad[0][0] + j * Ad[1][0]);
                float2 myz = make_float2(bm[1], bm[2]);
                if (i) myz = __ffma2_rn(make_float2((float)i, (float)i), make_float2(Ad[0][1], Ad[0][2]), myz);
                if (j) myz = __ffma2_rn(make_float2((float)j, (float)j), make_float2(Ad[1][1], Ad[1][2]), myz);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float wk = wij * w[2][k];
                    const float2 wk2 = make_float2(wk, wk);
                    const float kf = (float)k;
                    const float2 vx = k ? __ffma2_rn(make_float2(kf, kf), ad2x, mx) : mx;
                    const float2 vyz = k ? __ffma2_rn(make_float2(kf, kf), ad2yz, myz) : myz;
                    const float2 qmx = __ffma2_rn(wk2, vx, magic);
                    const float2 qyz = __ffma2_rn(wk2, vyz, magic);
                    const int o = i * kPitchX + j * kPitchY + k;
                    atomicAdd(tm + o, __float_as_int(qmx.x) - 0x4B400000);
                    atomicAdd(tx + o, __float_as_int(qmx.y) - 0x4B400000);
                    atomicAdd(ty + o, __float_as_int(qyz.x) - 0x4B400000);
                    atomicAdd(tz + o, __float_as_int(qyz.y) - 0x4B400000);
                }
            }
        return 0;
    }
    float4* grid = p.grid_out + E.node_base;
    // rare path: rolled loops, weights picked by selects (no run-time indexing of register arrays)
#pragma unroll 1
    for (int i = 0; i < 3; ++i)
#pragma unroll 1
        for (int j = 0; j < 3; ++j)
#pragma unroll 1
            for (int k = 0; k < 3; ++k) {
                const float wi = i == 0 ? w[0][0] : (i == 1 ? w[0][1] : w[0][2]);
                const float wj = j == 0 ? w[1][0] : (j == 1 ? w[1][1] : w[1][2]);
                const float wkk = k == 0 ? w[2][0] : (k == 1 ? w[2][1] : w[2][2]);
                float wk = wi * wj * wkk;
                int gx = bs[0] + i, gy = bs[1] + j, gz = bs[2] + k;
                float4 add = make_float4(wk * m, wk * (bm[0] + i * Ad[0][0] + j * Ad[1][0] + k * Ad[2][0]),
                                         wk * (bm[1] + i * Ad[0][1] + j * Ad[1][1] + k * Ad[2][1]),
                                         wk * (bm[2] + i * Ad[0][2] + j * Ad[1][2] + k * Ad[2][2]));
                atomicAdd(&grid[node_index(gx, gy, gz, g.nb)], add);
                const uint32_t lb = block_index(gx >> 2, gy >> 2, gz >> 2, g.nb);
                mark_bin(p, E.bin_base + lb, pack_bin((uint32_t)env, lb));
            }
    return 0x8u;
}

// Zero both tiles (once per launch; afterwards the flush zeroes what it reads).
__device__ __forceinline__ void tile_zero(ScatterTile& T) {
    int4* q = reinterpret_cast<int4*>(&T.q[0][0][0]);
    for (int t = threadIdx.x; t < 2 * kScatterSlots; t += blockDim.x) q[t] = make_int4(0, 0, 0, 0);
}

// The per-chunk bookkeeping of a tile (the node values are already zero).
__device__ __forceinline__ void tile_clear(ScatterTile& T) {
    if (threadIdx.x < 27) T.touched[threadIdx.x] = 0u;
    if (threadIdx.x < 8) T.expo_map[threadIdx.x] = 0u;
    if (threadIdx.x < 32) T.class_count[threadIdx.x] = 0u;
    for (int t = threadIdx.x; t < kLayers; t += blockDim.x) T.layer_mask[t] = 0u;
}

// Record the exponent of this thread's particle bound in the chunk's map; every thread of the CTA must
// call it. A warp whose bounds share one map word (the usual case) sets its bits with one atomic.
__device__ __forceinline__ void tile_bound(ScatterTile& T, float bp, bool active) {
    const uint32_t field = (__float_as_uint(bp) >> 23) & 0xffu;
    const uint32_t word = field >> 5, bit = 1u << (field & 31u);
    const uint32_t lo = __reduce_min_sync(0xffffffffu, active ? word : 0xffffu);
    const uint32_t hi = __reduce_max_sync(0xffffffffu, active ? word : 0u);
    if (lo == hi) {
        const uint32_t bits = __reduce_or_sync(0xffffffffu, active ? bit : 0u);
        if ((threadIdx.x & 31) == 0) atomicOr(&T.expo_map[lo], bits);
    } else if (active) {
        atomicOr(&T.expo_map[word], bit);
    }
}

// The chunk's two scales from its exponent map (read after the barrier that follows tile_bound): the
// largest exponent field `top` sets the first tile's scale k_fast; the largest field below
// top - kSlowShift, if any, the second tile's k_slow (slow = false: no particle goes there).
struct TileScales {
    int k_fast, k_slow, split;  // a particle with exponent field < split uses the second tile
    bool slow;
};

__device__ __forceinline__ TileScales tile_scales(const ScatterTile& T) {
    // every thread reads the same words (broadcast); the loops are uniform across the CTA
    int wt = 7;
    while (wt > 0 && T.expo_map[wt] == 0u) --wt;
    const uint32_t mt = T.expo_map[wt];
    const int top = mt ? wt * 32 + 31 - __clz(mt) : 0;
    TileScales t;
    t.split = top - kSlowShift;
    int low = -1;
    if (t.split > 0) {
        int ws = (t.split - 1) >> 5;  // word of the highest field below split
        uint32_t w = T.expo_map[ws] & (0xffffffffu >> (31 - ((t.split - 1) & 31)));
        while (w == 0u && ws > 0) w = T.expo_map[--ws];
        if (w) low = ws * 32 + 31 - __clz(w);
    }
    t.k_fast = momentum_scale_exp(top);
    t.slow = low >= 0;
    t.k_slow = momentum_scale_exp(t.slow ? low : 0);
    return t;
}

// The tile a particle scatters into (0 fast, 1 slow) and its momentum scale.
__device__ __forceinline__ int tile_of(float bp, const TileScales& ts, float& mscale) {
    const bool slow = (int)((__float_as_uint(bp) >> 23) & 0xffu) < ts.split;
    mscale = pow2f(slow ? ts.k_slow : ts.k_fast);
    return slow ? 1 : 0;
}

// Add the tiles' nonzero nodes to the env's global grid (FP32, one vector atomic each), zero them, then
// mark the bins that received mass. bin = (bx, by, bz) of the particles; the tile origin is 4 * bin - 1.
// The slow tile is read only when a particle of the chunk used it (ts.slow, uniform over the CTA).
__device__ __forceinline__ void tile_flush(ScatterTile& T, const TransferParams& p, const EnvDesc& E, int env,
                                           int bx, int by, int bz, const TileScales& ts) {
    const int nb = E.geo.nb;
    float4* grid = p.grid_out + E.node_base;
    const float mass_unit = E.mat.p_mass * pow2f(-kMassBits);
    const float inv_f = pow2f(-ts.k_fast), inv_s = pow2f(-ts.k_slow);
    const bool slow_used = ts.slow;
    for (int t = threadIdx.x; t < kScatterNodes; t += blockDim.x) {
        const int ti = t >> 6, tj = (t >> 3) & 7, tk = t & 7;  // a warp reads 32 consecutive slots
        const int sl = tile_slot(ti, tj, tk);
        const int mf = T.q[0][0][sl];
        const int ms = slow_used ? T.q[1][0][sl] : 0;
        if ((mf | ms) == 0) continue;  // no weight reached the node (momentum is then zero too)
        float4 add = make_float4((float)(mf + ms) * mass_unit, 0.0f, 0.0f, 0.0f);
        if (mf) {
            add.y = (float)T.q[0][1][sl] * inv_f;
            add.z = (float)T.q[0][2][sl] * inv_f;
            add.w = (float)T.q[0][3][sl] * inv_f;
            T.q[0][0][sl] = T.q[0][1][sl] = T.q[0][2][sl] = T.q[0][3][sl] = 0;
        }
        if (ms) {
            add.y += (float)T.q[1][1][sl] * inv_s;
            add.z += (float)T.q[1][2][sl] * inv_s;
            add.w += (float)T.q[1][3][sl] * inv_s;
            T.q[1][0][sl] = T.q[1][1][sl] = T.q[1][2][sl] = T.q[1][3][sl] = 0;
        }
        int gx = 4 * bx - 1 + ti, gy = 4 * by - 1 + tj, gz = 4 * bz - 1 + tk;
        atomicAdd(&grid[node_index(gx, gy, gz, nb)], add);
        int qx = (gx >> 2) - bx + 1, qy = (gy >> 2) - by + 1, qz = (gz >> 2) - bz + 1;
        T.touched[(qx * 3 + qy) * 3 + qz] = 1u;
    }
    __syncthreads();
    if (threadIdx.x < 27 && T.touched[threadIdx.x]) {
        int q = threadIdx.x;
        int qx = q / 9, qy = (q / 3) % 3, qz = q % 3;
        const uint32_t lb = block_index(bx + qx - 1, by + qy - 1, bz + qz - 1, nb);
        mark_bin(p, E.bin_base + lb, pack_bin((uint32_t)env, lb));
    }
}

__device__ __forceinline__ void load_mat(const float* base, int N, uint32_t i, float (&M)[3][3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M[r][c] = base[(size_t)(r * 3 + c) * N + i];
}

__device__ __forceinline__ void store_mat(float* base, int N, uint32_t i, const float (&M)[3][3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) base[(size_t)(r * 3 + c) * N + i] = M[r][c];
}

// A = m C - dt V0 (4/dx^2) tau: the MLS-MPM affine momentum with the stress impulse folded in.
__device__ __forceinline__ void affine(const Material& mat, const float (&C)[3][3], const float (&tau)[3][3],
                                       float (&A)[3][3]) {
    const float2 m2 = make_float2(mat.p_mass, mat.p_mass), s2 = make_float2(mat.stress_scale, mat.stress_scale);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float2 a = __ffma2_rn(s2, make_float2(tau[r][0], tau[r][1]), __fmul2_rn(m2, make_float2(C[r][0], C[r][1])));
        A[r][0] = a.x;
        A[r][1] = a.y;
        A[r][2] = fmaf(mat.stress_scale, tau[r][2], mat.p_mass * C[r][2]);
    }
}

// Local bin b (< nb^3) to its block coordinates, dividing by nb with its 32-bit reciprocal: for b < 2^19
// the rounding error of umulhi(b, ceil(2^32 / nb)) is below 2^-13, and b / nb's fraction is at most
// 1 - 1/nb with nb <= 64, so the quotient is exact.
__device__ __forceinline__ void decode_bin(int b, const Geometry& g, int& bx, int& by, int& bz) {
    const uint32_t q1 = __umulhi((uint32_t)b, g.nb_recip), q2 = __umulhi(q1, g.nb_recip);
    bz = b - (int)q1 * g.nb;
    by = (int)q1 - (int)q2 * g.nb;
    bx = (int)q2;
}

}  // namespace

// ------------------------------------------------------------------------ set_particles

// Copy the caller's particles in (clamped), with identity pid, and count them into bins with ranks.
__global__ void __launch_bounds__(256) k_load(LoadParams p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < p.N;
    uint32_t flags = 0, key = 0xffffffffu;
    if (active) {
        const int e = env_of_particle(p.envs, p.nenv, (uint32_t)i);
        const EnvDesc& E = p.envs[e];
        const Geometry& g = E.geo;
        const int N = p.N;
        float xp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xp[a] = p.x[(size_t)a * N + i];
            flags |= clamp_coord(xp[a], g.lo, g.hi);
            p.dst.x[(size_t)a * N + i] = xp[a];
            p.dst.v[(size_t)a * N + i] = p.v ? p.v[(size_t)a * N + i] : 0.0f;
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) p.dst.C[(size_t)c * N + i] = p.C ? p.C[(size_t)c * N + i] : 0.0f;
        if (E.kind == 0) {
#pragma unroll
            for (int c = 0; c < 9; ++c)
                p.dst.F[(size_t)c * N + i] = p.F ? p.F[(size_t)c * N + i] : ((c % 4 == 0) ? 1.0f : 0.0f);
        } else {
            float J = 1.0f;
            if (p.F) {
                float M[3][3];
                load_mat(p.F, N, i, M);
                J = det3(M);
            }
            p.dst.F[i] = J;
        }
        p.dst.pid[i] = (uint32_t)i;
        key = E.bin_base + local_bin_of(xp, g);
    }
    const uint32_t rank = warp_hist_add(p.hist, key, true);
    if (active) p.keyrank[i] = make_uint2(key, rank);
    if (flags) atomicOr(p.status, flags);
}

// ------------------------------------------------------------------------ counting sort into bins

// One CTA (a multiple of 32 threads, at most 1024): exclusive scan of the bin counts -> bin start
// offsets (cursor) and the chunk list: each bin is cut into chunks of at most `chunk` particles, one
// chunk per CTA iteration of the particle passes, tagged with the bin's env. The counts are read from L2
// (they were accumulated by other CTAs' atomics) and zeroed for the next histogram. Each thread owns a run
// of 4-bin groups, read as 16-byte vectors in batches of independent loads so one L2 round trip covers
// 32 (then 16) bins. The count and env arrays are padded to a multiple of 4 bins (zeros).
// CHUNK > 0 fixes the chunk size at compile time (the divisions become shifts); 0 takes `chunk`.
template <int CHUNK>
__device__ __forceinline__ void scan_bins(uint32_t* hist, uint32_t* cursor, int4* chunks, uint32_t* num_chunks,
                                          const uint32_t* bin_env, int nblocks, int chunk_arg,
                                          uint32_t (&warp_tot)[2][32]) {
    const int chunk = CHUNK > 0 ? CHUNK : chunk_arg;
    const int tid = threadIdx.x;
    const int nq = (nblocks + 3) >> 2;
    const int per = (nq + blockDim.x - 1) / blockDim.x;
    const int q0 = min(tid * per, nq), q1 = min(q0 + per, nq);
    uint4* H = reinterpret_cast<uint4*>(hist);
    uint32_t cnt = 0, nch = 0;
    for (int q = q0; q < q1; q += 8) {
        uint4 h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) h[u] = q + u < q1 ? __ldcg(&H[q + u]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const uint32_t c4[4] = {h[u].x, h[u].y, h[u].z, h[u].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                cnt += c4[e];
                nch += (c4[e] + chunk - 1) / chunk;
            }
        }
    }
    // block-wide exclusive scan of (cnt, nch)
    const int lane = tid & 31, wid = tid >> 5;
    uint32_t ic = cnt, in = nch;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t tc = __shfl_up_sync(0xffffffffu, ic, d), tn = __shfl_up_sync(0xffffffffu, in, d);
        if (lane >= d) { ic += tc; in += tn; }
    }
    if (lane == 31) { warp_tot[0][wid] = ic; warp_tot[1][wid] = in; }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        uint32_t vc = lane < nw ? warp_tot[0][lane] : 0u, vn = lane < nw ? warp_tot[1][lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t tc = __shfl_up_sync(0xffffffffu, vc, d), tn = __shfl_up_sync(0xffffffffu, vn, d);
            if (lane >= d) { vc += tc; vn += tn; }
        }
        if (lane < nw) { warp_tot[0][lane] = vc; warp_tot[1][lane] = vn; }
    }
    __syncthreads();
    uint32_t off = ic - cnt + (wid > 0 ? warp_tot[0][wid - 1] : 0u);
    uint32_t coff = in - nch + (wid > 0 ? warp_tot[1][wid - 1] : 0u);
    uint4* Cur = reinterpret_cast<uint4*>(cursor);
    const uint4* BE = reinterpret_cast<const uint4*>(bin_env);  // null: every bin is env 0's
    for (int q = q0; q < q1; q += 4) {
        // four 4-bin groups per batch: counts and (for several envs) the bins' envs, all loads in flight
        uint4 h[4], be[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            h[u] = q + u < q1 ? __ldcg(&H[q + u]) : make_uint4(0u, 0u, 0u, 0u);
            be[u] = (BE && q + u < q1) ? BE[q + u] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (q + u >= q1) break;
            const uint32_t c4[4] = {h[u].x, h[u].y, h[u].z, h[u].w};
            const uint32_t e4[4] = {be[u].x, be[u].y, be[u].z, be[u].w};
            uint32_t o4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t c = c4[e];
                o4[e] = off;
                const int b = 4 * (q + u) + e;
                for (uint32_t s = 0; s < c; s += chunk)
                    chunks[coff++] = make_int4(b, (int)(off + s), (int)min((uint32_t)chunk, c - s), (int)e4[e]);
                off += c;
            }
            Cur[q + u] = make_uint4(o4[0], o4[1], o4[2], o4[3]);
            H[q + u] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (tid == blockDim.x - 1) *num_chunks = coff;
}

__global__ void __launch_bounds__(1024) k_scan(uint32_t* hist, uint32_t* cursor, int4* chunks,
                                               uint32_t* num_chunks, const uint32_t* bin_env, int nblocks,
                                               int chunk) {
    __shared__ uint32_t warp_tot[2][32];
    if (chunk == kChunk)
        scan_bins<kChunk>(hist, cursor, chunks, num_chunks, bin_env, nblocks, chunk, warp_tot);
    else
        scan_bins<0>(hist, cursor, chunks, num_chunks, bin_env, nblocks, chunk, warp_tot);
}

// The bin counts' exclusive prefix into shared memory (cur_sh, total_bins padded to 4), each count read
// from L2 once: a thread copies its run of 4-bin groups into cur_sh while summing, the CTA scans the
// per-thread sums, and each thread turns its run into offsets in place. With `writer` the CTA also
// writes the global offsets, the chunk list (chunks of at most `chunk` particles, tagged with the bin's
// env) and its length. The counts are left in place.
template <int CHUNK>
__device__ __forceinline__ void scan_counts_shared(const uint32_t* hist, uint32_t* cur_sh, int nblocks, int chunk_arg,
                                                   bool writer, uint32_t* cursor, int4* chunks, uint32_t* num_chunks,
                                                   const uint32_t* bin_env, uint32_t (&warp_tot)[2][32]) {
    const int chunk = CHUNK > 0 ? CHUNK : chunk_arg;
    const int tid = threadIdx.x;
    const int nq = (nblocks + 3) >> 2;
    const int per = (nq + blockDim.x - 1) / blockDim.x;
    const int q0 = min(tid * per, nq), q1 = min(q0 + per, nq);
    const uint4* H = reinterpret_cast<const uint4*>(hist);
    uint4* S = reinterpret_cast<uint4*>(cur_sh);
    uint32_t cnt = 0, nch = 0;
    for (int q = q0; q < q1; q += 8) {
        uint4 h[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) h[u] = q + u < q1 ? __ldcg(&H[q + u]) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (q + u < q1) S[q + u] = h[u];
            const uint32_t c4[4] = {h[u].x, h[u].y, h[u].z, h[u].w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                cnt += c4[e];
                nch += (c4[e] + chunk - 1) / chunk;
            }
        }
    }
    const int lane = tid & 31, wid = tid >> 5;
    uint32_t ic = cnt, in = nch;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t tc = __shfl_up_sync(0xffffffffu, ic, d), tn = __shfl_up_sync(0xffffffffu, in, d);
        if (lane >= d) { ic += tc; in += tn; }
    }
    if (lane == 31) { warp_tot[0][wid] = ic; warp_tot[1][wid] = in; }
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        uint32_t vc = lane < nw ? warp_tot[0][lane] : 0u, vn = lane < nw ? warp_tot[1][lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t tc = __shfl_up_sync(0xffffffffu, vc, d), tn = __shfl_up_sync(0xffffffffu, vn, d);
            if (lane >= d) { vc += tc; vn += tn; }
        }
        if (lane < nw) { warp_tot[0][lane] = vc; warp_tot[1][lane] = vn; }
    }
    __syncthreads();
    uint32_t off = ic - cnt + (wid > 0 ? warp_tot[0][wid - 1] : 0u);
    uint32_t coff = in - nch + (wid > 0 ? warp_tot[1][wid - 1] : 0u);
    const uint4* BE = reinterpret_cast<const uint4*>(bin_env);  // null: every bin is env 0's
    for (int q = q0; q < q1; ++q) {
        const uint4 h = S[q];
        const uint32_t c4[4] = {h.x, h.y, h.z, h.w};
        const uint4 be = (writer && BE) ? BE[q] : make_uint4(0u, 0u, 0u, 0u);
        const uint32_t e4[4] = {be.x, be.y, be.z, be.w};
        uint32_t o4[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            o4[e] = off;
            if (writer)
                for (uint32_t s = 0; s < c4[e]; s += chunk)
                    chunks[coff++] = make_int4(4 * q + e, (int)(off + s), (int)min((uint32_t)chunk, c4[e] - s), (int)e4[e]);
            off += c4[e];
        }
        S[q] = make_uint4(o4[0], o4[1], o4[2], o4[3]);
        if (writer) reinterpret_cast<uint4*>(cursor)[q] = S[q];
    }
    if (writer && tid == blockDim.x - 1) *num_chunks = coff;
}

// Grid-wide scan for many bins, kernel 1: per tile of kScanTile bins, the sums of particles and chunks.
__global__ void __launch_bounds__(256) k_scan_tiles(ScanParams p) {
    wait_for_predecessor();
    const int t = blockIdx.x;
    const int b0 = t * kScanTile;
    uint32_t cnt = 0, nch = 0;
    for (int b = b0 + (int)threadIdx.x; b < min(b0 + kScanTile, p.total_bins); b += blockDim.x) {
        const uint32_t c = __ldcg(&p.hist[b]);
        cnt += c;
        nch += (c + p.chunk - 1) / p.chunk;
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    nch = __reduce_add_sync(0xffffffffu, nch);
    __shared__ uint32_t part[2][8];
    if ((threadIdx.x & 31) == 0) { part[0][threadIdx.x >> 5] = cnt; part[1][threadIdx.x >> 5] = nch; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += part[0][w]; b += part[1][w]; }
        p.tile_sums[t] = make_uint2(a, b);
    }
}

// Grid-wide scan, kernel 2: each tile adds up the sums of the tiles before it, scans its own bins into
// offsets and chunk entries, and zeroes its counts. The last tile stores the chunk total.
__global__ void __launch_bounds__(kScanTile) k_scan_apply(ScanParams p) {
    __shared__ uint32_t warp_tot[2][32];
    __shared__ uint32_t base[2];
    const int t = blockIdx.x;
    uint32_t pc = 0, pn = 0;
    for (int u = (int)threadIdx.x; u < t; u += blockDim.x) {
        const uint2 s = __ldcg(&p.tile_sums[u]);
        pc += s.x;
        pn += s.y;
    }
    pc = __reduce_add_sync(0xffffffffu, pc);
    pn = __reduce_add_sync(0xffffffffu, pn);
    if ((threadIdx.x & 31) == 0) { warp_tot[0][threadIdx.x >> 5] = pc; warp_tot[1][threadIdx.x >> 5] = pn; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += warp_tot[0][w]; b += warp_tot[1][w]; }
        base[0] = a;
        base[1] = b;
    }
    __syncthreads();
    // one bin per thread: block-wide exclusive scan of (count, chunks)
    const int b = t * kScanTile + (int)threadIdx.x;
    const uint32_t c = b < p.total_bins ? __ldcg(&p.hist[b]) : 0u;
    const uint32_t n = (c + p.chunk - 1) / p.chunk;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t ic = c, in = n;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t tc = __shfl_up_sync(0xffffffffu, ic, d), tn = __shfl_up_sync(0xffffffffu, in, d);
        if (lane >= d) { ic += tc; in += tn; }
    }
    __syncthreads();
    if (lane == 31) { warp_tot[0][wid] = ic; warp_tot[1][wid] = in; }
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t vc = lane < nw ? warp_tot[0][lane] : 0u, vn = lane < nw ? warp_tot[1][lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t tc = __shfl_up_sync(0xffffffffu, vc, d), tn = __shfl_up_sync(0xffffffffu, vn, d);
            if (lane >= d) { vc += tc; vn += tn; }
        }
        if (lane < nw) { warp_tot[0][lane] = vc; warp_tot[1][lane] = vn; }
    }
    __syncthreads();
    const uint32_t off = base[0] + ic - c + (wid > 0 ? warp_tot[0][wid - 1] : 0u);
    uint32_t coff = base[1] + in - n + (wid > 0 ? warp_tot[1][wid - 1] : 0u);
    if (b < p.total_bins) {
        p.cursor[b] = off;
        if (c) {
            const int env = (int)p.bin_env[b];
            for (uint32_t s = 0; s < c; s += p.chunk)
                p.chunks[coff++] = make_int4(b, (int)(off + s), (int)min((uint32_t)p.chunk, c - s), env);
        }
        p.hist[b] = 0u;
    }
    if (t == (int)gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *p.num_chunks = coff;
}

// Sorted slot of particle j: slot = start of its bin + its rank within the bin. The rank was handed out
// with the particle's bin count (a chunk's staying particles from one atomic per chunk, in class-layered
// order; the others one atomic per warp and bin), so this pass needs no atomics.
__device__ __forceinline__ void assign_slot(int j, int N, const uint2* __restrict__ keyrank,
                                            const uint32_t* __restrict__ cursor, uint32_t* __restrict__ perm) {
    if (j >= N) return;
    const uint2 kr = keyrank[j];
    perm[cursor[kr.x] + kr.y] = (uint32_t)j;
}

// Four consecutive particles per thread (two 16-byte loads, four independent offset lookups in flight).
constexpr int kAssignPerThread = 4;
__device__ __forceinline__ void assign_slots4(int t, int N, const uint2* __restrict__ keyrank,
                                              const uint32_t* __restrict__ cursor, uint32_t* __restrict__ perm) {
    const int j0 = t * kAssignPerThread;
    if (j0 + kAssignPerThread <= N) {
        const uint4* q = reinterpret_cast<const uint4*>(keyrank + j0);
        const uint4 a = q[0], b = q[1];
        const uint32_t c0 = cursor[a.x], c1 = cursor[a.z], c2 = cursor[b.x], c3 = cursor[b.z];
        perm[c0 + a.y] = (uint32_t)j0;
        perm[c1 + a.w] = (uint32_t)(j0 + 1);
        perm[c2 + b.y] = (uint32_t)(j0 + 2);
        perm[c3 + b.w] = (uint32_t)(j0 + 3);
    } else {
        for (int j = j0; j < N; ++j) assign_slot(j, N, keyrank, cursor, perm);
    }
}

__global__ void __launch_bounds__(256) k_assign(int N, const uint2* __restrict__ keyrank,
                                                const uint32_t* __restrict__ cursor, uint32_t* __restrict__ perm) {
    assign_slots4(blockIdx.x * blockDim.x + threadIdx.x, N, keyrank, cursor, perm);
}

// ------------------------------------------------------------------------ standalone P2G

// ------------------------------------------------------------------------ particle contact

// Penalty acceleration of a particle at x with velocity v against one body (Sec. 3's particle form of
// the coupling, Algorithm 1 "compute penalty forces"): inside the body (phi < 0),
//   a = a_n n - min(damping |v_t|, friction a_n) v_t / |v_t|,  a_n = stiffness (-phi) + damping max(-v_n, 0),
// with v_n, v_t the normal and tangential parts of the velocity relative to the body's surface
// velocity there. rel receives x - com, the lever arm of the reaction.
__device__ __forceinline__ bool penalty_one(const ColliderNow& cn, const float x[3], const float v[3], float stiffness,
                                            float damping, float a[3], float rel[3]) {
    const float o[3] = {x[0] - cn.p[0], x[1] - cn.p[1], x[2] - cn.p[2]};
    if (o[0] * o[0] + o[1] * o[1] + o[2] * o[2] > cn.reach2) return false;  // beyond the body's ball
    float nrm[3];
    const float phi = collider_sdf(cn, x, nrm);
    if (!(phi < 0.0f)) return false;
#pragma unroll
    for (int i = 0; i < 3; ++i) rel[i] = x[i] - cn.com[i];
    const float vr[3] = {v[0] - (cn.lin[0] + cn.ang[1] * rel[2] - cn.ang[2] * rel[1]),
                         v[1] - (cn.lin[1] + cn.ang[2] * rel[0] - cn.ang[0] * rel[2]),
                         v[2] - (cn.lin[2] + cn.ang[0] * rel[1] - cn.ang[1] * rel[0])};
    const float vn = vr[0] * nrm[0] + vr[1] * nrm[1] + vr[2] * nrm[2];
    const float an = stiffness * (-phi) + damping * fmaxf(-vn, 0.0f);
    const float vt[3] = {vr[0] - vn * nrm[0], vr[1] - vn * nrm[1], vr[2] - vn * nrm[2]};
    const float tn = sqrtf(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
    const float ft = tn > 0.0f ? fminf(damping * tn, cn.friction * an) / tn : 0.0f;
#pragma unroll
    for (int i = 0; i < 3; ++i) a[i] = an * nrm[i] - ft * vt[i];
    return true;
}

// Pose of collider c at substep `step` for the penalty: this CTA's shared copy (few colliders), the
// table mpm_set_colliders filled (first kPoseSteps substeps), else evaluated here.
__device__ __forceinline__ void penalty_pose(const TransferParams& p, const ColliderNow* cs, bool shared_poses, int c,
                                             uint32_t step, float dt, ColliderNow& cn) {
    if (shared_poses)
        cn = cs[c];
    else if (step < (uint32_t)kPoseSteps)
        cn = p.poses[(size_t)step * p.k_total + c];
    else
        collider_at(p.cols[c], (float)step * dt, cn);
}

// A particle's penalty acceleration summed over its env's bodies (index order), and the reactions
// (Algorithm 1 "accumulate equivalent rigid-body forces and torques"): -dt m a and its moment about
// the centre of mass, summed over the warp, then into this CTA's shared sums (few colliders) or the
// FP64 buffers. All threads of the CTA call it (the loop bound is the chunk's env).
__device__ __forceinline__ void penalty_accel(const TransferParams& p, const EnvDesc& E, const ColliderNow* cs,
                                              float* cw, bool shared_poses, uint32_t step, bool active,
                                              const float x[3], const float v[3], float acc[3]) {
    const float dt = E.geo.dt, m = E.mat.p_mass;
    acc[0] = acc[1] = acc[2] = 0.0f;
    const int c1 = E.col_first + E.col_count;
    for (int c = E.col_first; c < c1; ++c) {
        ColliderNow cn;
        penalty_pose(p, cs, shared_poses, c, step, dt, cn);
        float a[3], rel[3];
        const bool hit = active && penalty_one(cn, x, v, p.stiffness, p.damping, a, rel);
        float w6[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (hit) {
            const float imp[3] = {-dt * m * a[0], -dt * m * a[1], -dt * m * a[2]};
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                acc[i] += a[i];
                w6[i] = imp[i];
            }
            w6[3] = rel[1] * imp[2] - rel[2] * imp[1];
            w6[4] = rel[2] * imp[0] - rel[0] * imp[2];
            w6[5] = rel[0] * imp[1] - rel[1] * imp[0];
        }
        if (__any_sync(0xffffffffu, hit)) {
#pragma unroll
            for (int q = 0; q < 6; ++q)
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) w6[q] += __shfl_xor_sync(0xffffffffu, w6[q], off);
            if ((threadIdx.x & 31) == 0) {
                if (shared_poses) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) atomicAdd(&cw[c * 6 + q], w6[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < 6; ++q) atomicAdd(&p.wrench[(size_t)c * 6 + q], (double)w6[q]);
                }
            }
        }
    }
}

// Shared poses and reaction sums of a CTA that applies penalties (few colliders): poses at `step`.
__device__ __forceinline__ void penalty_begin(const TransferParams& p, ColliderNow* cs, float* cw, uint32_t step,
                                              float dt) {
    if ((int)threadIdx.x < p.k_total) collider_at(p.cols[threadIdx.x], (float)step * dt, cs[threadIdx.x]);
    for (int t = threadIdx.x; t < p.k_total * 6; t += blockDim.x) cw[t] = 0.0f;
}

__device__ __forceinline__ void penalty_end(const TransferParams& p, const float* cw) {
    for (int t = threadIdx.x; t < p.k_total * 6; t += blockDim.x)
        if (cw[t] != 0.0f) atomicAdd(&p.wrench[t], (double)cw[t]);
}

__global__ void __launch_bounds__(kChunk) k_p2g(TransferParams p) {
    __shared__ ScatterTile T;
    __shared__ EnvDesc E;
    __shared__ ColliderNow cs[kSharedPoses];
    __shared__ float cw[kSharedPoses * 6];
    const int N = p.N;
    uint32_t flags = 0;
    const uint32_t nchunks = *p.num_chunks;
    const bool shared_poses = p.k_total <= kSharedPoses;
    const uint32_t step = p.contact ? *p.substep_counter : 0u;
    if (p.contact && shared_poses) {
        penalty_begin(p, cs, cw, step, p.env0.geo.dt);
        __syncthreads();
    }
    tile_zero(T);
    for (uint32_t w = blockIdx.x; w < nchunks; w += gridDim.x) {
        const int4 ch = p.chunks[w];
        const int env = ch.w;
        load_env(E, p.envs, env);
        tile_clear(T);
        __syncthreads();
        int bx, by, bz;
        decode_bin(ch.x - (int)E.bin_base, E.geo, bx, by, bz);
        const int o[3] = {4 * bx - 1, 4 * by - 1, 4 * bz - 1};
        const bool active = (int)threadIdx.x < ch.z;
        float x[3] = {0.0f, 0.0f, 0.0f}, v[3] = {0.0f, 0.0f, 0.0f}, A[3][3];
        float bp = 0.0f;
        if (active) {
            const uint32_t src = p.perm[ch.y + threadIdx.x];
            float C[3][3], tau[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x[a] = p.in.x[(size_t)a * N + src];
                v[a] = p.in.v[(size_t)a * N + src];
            }
            load_mat(p.in.C, N, src, C);
            if (E.kind == 0) {
                float F[3][3];
                load_mat(p.in.F, N, src, F);
                fixed_corotated_stress(F, E.mat, tau);
            } else {
                const float J = p.in.F[src];
                const float s = E.mat.lambda * J * (J - 1.0f);
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) tau[r][c] = r == c ? s : 0.0f;
            }
            affine(E.mat, C, tau, A);
        }
        if (p.contact) {  // the penalty impulse joins the momentum this particle transfers
            float acc[3];
            penalty_accel(p, E, cs, cw, shared_poses, step, active, x, v, acc);
#pragma unroll
            for (int a = 0; a < 3; ++a) v[a] += E.geo.dt * acc[a];
        }
        if (active) bp = particle_bound(E.mat.p_mass, v, A, E.geo.dx);
        tile_bound(T, bp, active);
        __syncthreads();
        const TileScales ts = tile_scales(T);
        float mscale;
        const int tile = tile_of(bp, ts, mscale);
        if (active) flags |= scatter_particle(T, p, E, env, o, x, v, A, tile, mscale);
        __syncthreads();
        tile_flush(T, p, E, env, bx, by, bz, ts);
        __syncthreads();
    }
    if (p.contact && shared_poses) penalty_end(p, cw);
    if (flags) atomicOr(p.status, flags);
}

// ------------------------------------------------------------------------ fused G2P -> P2G

// The env of a chunk: the kernel parameters' copy for a one-env handle, else the shared double buffer.
template <bool ONE_ENV>
__device__ __forceinline__ const EnvDesc& chunk_env(const TransferParams& p, const EnvDesc (&Es)[2], int it) {
    if constexpr (ONE_ENV) return p.env0;
    else return Es[it & 1];
}

// KIND: the material of every env (0 plasticine, 1 fluid) or -1 for a per-env choice at run time.
// ONE_ENV: one env whose descriptor comes from the kernel parameters (constant bank operands) rather
// than from shared memory, which keeps the single-scene kernel's register budget.
// CTA: threads per CTA = the most particles of a chunk it takes (128 or 256). Dense scenes (many
// particles per bin) run 256-particle chunks at 4 resident CTAs per SM (64 registers): measured 6 % faster
// per env step than 128-particle chunks at 7 CTAs (72 registers) on the 200k and the 600k pinch scene — a
// chunk's gather-tile load and scatter-tile flush then serve twice the particles — and faster than 3 or 5
// CTAs, or chunks of 384 or 512. Sparse batches keep 128-thread CTAs, whose threads chunks fill.
// PEN: the particle form of the contact (penalty accelerations join the transfer; the grid update
// applies no colliders then).
template <int KIND, bool ONE_ENV, bool PEN, int CTA>
__global__ void __launch_bounds__(CTA, CTA == 256 ? (PEN ? 3 : 4) : (PEN ? 6 : 7)) k_g2p2g(TransferParams p) {
    // gather tile: node velocities of [4 bin, 4 bin + 6) per axis, one FP32 array per component, slots laid
    // out like the scatter tile so the 27 reads of a warp spread over the banks
    __shared__ float Gx[kGatherSlots], Gy[kGatherSlots], Gz[kGatherSlots];
    __shared__ ScatterTile T;
    static_assert(CTA <= kLayers, "a cell's layer index stays below kLayers");
    __shared__ EnvDesc Es[2];  // several envs: the current chunk's env and the next one's
    __shared__ ColliderNow cs[PEN ? kSharedPoses : 1];
    __shared__ float cw[PEN ? kSharedPoses * 6 : 1];
    const int N = p.N;
    uint32_t flags = 0;
    wait_for_predecessor();
    if (p.gate && *p.gate != p.gate_run) {  // the other branch of a gated window runs instead
        release_successor();
        return;
    }
    // the substep the transfer belongs to (the grid update before this launch counted the last one)
    const bool pen = PEN && p.scatter;
    const bool shared_poses = p.k_total <= kSharedPoses;
    const uint32_t step = pen ? *p.substep_counter : 0u;
    if (pen && shared_poses) penalty_begin(p, cs, cw, step, p.env0.geo.dt);
    // the first chunk is requested with the count (its index does not depend on it), then dropped if
    // past the end
    int4 next = (int)blockIdx.x < p.chunk_cap ? p.chunks[blockIdx.x] : make_int4(0, 0, 0, 0);
    const uint32_t nchunks = *p.num_chunks;
    if (blockIdx.x >= nchunks) next = make_int4(0, 0, 0, 0);
    // A CTA's first two chunks are blockIdx.x and blockIdx.x + gridDim.x; later ones are handed out in list
    // order by a counter (p.work), two chunks ahead, so that SMs that drew short chunks take more. Thread 0
    // asks for chunk it + 2 at the top of iteration it and publishes it in slot (it & 1) of s_next before
    // the iteration's last barrier; the atomic's round trip overlaps the iteration's work. A CTA asks
    // only when it will run the iteration that reads the answer (chunk it + 1 exists), so every index
    // handed out below nchunks is processed. The last CTA resets the counter.
    __shared__ uint32_t s_next[2];
    tile_zero(T);  // ordered before the first scatter by the first chunk's barriers
    if constexpr (!ONE_ENV) {
        load_env(Es[0], p.envs, next.w);
        __syncthreads();
    }
    int it = 0;
    uint32_t w = blockIdx.x, wn = blockIdx.x + gridDim.x;
    for (; w < nchunks; ++it) {
        const int4 ch = next;
        const int env = ONE_ENV ? 0 : ch.w;
        const EnvDesc& E = chunk_env<ONE_ENV>(p, Es, it);
        const int kind = KIND >= 0 ? KIND : E.kind;
        const Geometry& g = E.geo;
        const float dt = g.dt;
        if (it > 0) wn = s_next[(it + 1) & 1];  // published before the previous iteration's last barrier
        uint32_t ticket = 0;
        if (threadIdx.x == 0 && wn < nchunks) ticket = atomicAdd(p.work, 1u);  // chunk it + 2 (used later)
        if (wn < nchunks) next = p.chunks[wn];  // prefetch the next descriptor
        int bx, by, bz;
        decode_bin(ch.x - (int)E.bin_base, g, bx, by, bz);
        const int ox = 4 * bx, oy = 4 * by, oz = 4 * bz;
        // this thread's particle: its loads are issued first so they overlap the tile load below. A chunk
        // never holds more particles than the CTA has threads (the list is recut when the chunk size
        // changes); should one, the rest are left alone and the internal-error flag is raised.
        if (ch.z > CTA && threadIdx.x == 0) flags |= kFlagInternal;
        const bool active = (int)threadIdx.x < min(ch.z, CTA);
        const uint32_t slot = (uint32_t)(ch.y + threadIdx.x);
        uint32_t src = 0;
        float x[3] = {0.5f, 0.5f, 0.5f};
        if (active) {
            src = p.perm[slot];
#pragma unroll
            for (int a = 0; a < 3; ++a) x[a] = p.in.x[(size_t)a * N + src];
        }
        const float4* grid_in = p.grid_in + E.node_base;
        for (int t = threadIdx.x; t < kGatherNodes; t += blockDim.x) {
            const int i = t / 36, j = (t / 6) % 6, k = t % 6;
            const int gx = ox + i, gy = oy + j, gz = oz + k;
            float4 val = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (gx < g.n && gy < g.n && gz < g.n) val = grid_in[node_index(gx, gy, gz, g.nb)];
            const int s = tile_slot(i, j, k);
            Gx[s] = val.x;
            Gy[s] = val.y;
            Gz[s] = val.z;
        }
        tile_clear(T);
        __syncthreads();
        if constexpr (!ONE_ENV)
            if (wn < nchunks) load_env(Es[(it + 1) & 1], p.envs, next.w);
        float xn[3] = {0.0f, 0.0f, 0.0f}, vn[3] = {0.0f, 0.0f, 0.0f}, A[3][3];
        float bp = 0.0f;
        uint32_t newkey = 0xffffffffu;
        if (active) {
            // ---- G2P: v = sum w v_i, C = 4/dx sum w v_i (i - f)^T (offsets in cells)
            int bs[3];
            float f[3], w3[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                bs[a] = cell_base(x[a], g.inv_dx);
                f[a] = cell_frac(x[a], g.inv_dx, bs[a]);
                bspline_weights(f[a], w3[a]);
            }
            int l0 = bs[0] - ox, l1 = bs[1] - oy, l2 = bs[2] - oz;
            if ((unsigned)l0 > 3u || (unsigned)l1 > 3u || (unsigned)l2 > 3u) {
                flags |= kFlagInternal;
                l0 = min(max(l0, 0), 3);
                l1 = min(max(l1, 0), 3);
                l2 = min(max(l2, 0), 3);
            }
            // 27 weighted reads into 12 sums, M[a][c] = sum_ijk w_i w_j w_k (index_c) v_a and v, contracted
            // one axis at a time: over k the sums with weights w_k and k w_k, over j with w_j and j w_j,
            // over i with w_i and i w_i. The x and y components travel as one packed FP32x2 operand
            // (one instruction for both, each lane rounded as a scalar fused multiply-add would be).
            const float* gx = Gx + tile_slot(l0, l1, l2);
            const float* gy = Gy + tile_slot(l0, l1, l2);
            const float* gz = Gz + tile_slot(l0, l1, l2);
            // (the z component's sums with weights w and k w travel as a pair too)
            float2 vxy = make_float2(0.0f, 0.0f), Mxy[3] = {vxy, vxy, vxy};
            float2 vz2 = make_float2(0.0f, 0.0f);  // (v_z, M_z2)
            float Mz0 = 0.0f, Mz1 = 0.0f;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float2 b0 = make_float2(0.0f, 0.0f), bj = b0, bk = b0;
                float2 bz2 = make_float2(0.0f, 0.0f);  // (b0z, bkz)
                float bjz = 0.0f;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float2 a0 = make_float2(0.0f, 0.0f), ak = a0;
                    float2 az2 = make_float2(0.0f, 0.0f);  // (a0z, akz)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int o = i * kPitchX + j * kPitchY + k;
                        const float2 g = make_float2(gx[o], gy[o]);
                        const float wk = w3[2][k], gzo = gz[o];
                        a0 = k ? __ffma2_rn(make_float2(wk, wk), g, a0) : __fmul2_rn(make_float2(wk, wk), g);
                        if (k) {
                            const float kw = (float)k * wk;
                            ak = __ffma2_rn(make_float2(kw, kw), g, ak);
                            az2 = __ffma2_rn(make_float2(wk, kw), make_float2(gzo, gzo), az2);
                        } else {
                            az2.x = wk * gzo;
                        }
                    }
                    const float wj = w3[1][j];
                    b0 = __ffma2_rn(make_float2(wj, wj), a0, b0);
                    bk = __ffma2_rn(make_float2(wj, wj), ak, bk);
                    bz2 = __ffma2_rn(make_float2(wj, wj), az2, bz2);
                    if (j) {
                        const float jw = (float)j * wj;
                        bj = __ffma2_rn(make_float2(jw, jw), a0, bj);
                        bjz = fmaf(jw, az2.x, bjz);
                    }
                }
                const float wi = w3[0][i];
                vxy = __ffma2_rn(make_float2(wi, wi), b0, vxy);
                vz2 = __ffma2_rn(make_float2(wi, wi), bz2, vz2);
                if (i) {
                    const float iw = (float)i * wi;
                    Mxy[0] = __ffma2_rn(make_float2(iw, iw), b0, Mxy[0]);
                    Mz0 = fmaf(iw, bz2.x, Mz0);
                }
                Mxy[1] = __ffma2_rn(make_float2(wi, wi), bj, Mxy[1]);
                Mxy[2] = __ffma2_rn(make_float2(wi, wi), bk, Mxy[2]);
                Mz1 = fmaf(wi, bjz, Mz1);
            }
            vn[0] = vxy.x;
            vn[1] = vxy.y;
            vn[2] = vz2.x;
            const float M[3][3] = {{Mxy[0].x, Mxy[1].x, Mxy[2].x}, {Mxy[0].y, Mxy[1].y, Mxy[2].y}, {Mz0, Mz1, vz2.y}};
            float Cn[3][3];
            const float cs = 4.0f * g.inv_dx;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) Cn[a][c] = cs * (M[a][c] - vn[a] * f[c]);
            // ---- advect and clamp
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xn[a] = x[a] + dt * vn[a];
                if (!isfinite(vn[a])) flags |= 0x2u;
                flags |= clamp_coord(xn[a], g.lo, g.hi);
            }
            // ---- F (or J) update, return map, stress of the new state
            float Gm[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) Gm[a][c] = (a == c ? 1.0f : 0.0f) + dt * Cn[a][c];
            float tau[3][3];
            if (kind == 0) {
                float F[3][3], Ft[3][3];
                load_mat(p.in.F, N, src, F);
                matmul3(Gm, F, Ft);
                flags |= plastic_update_and_stress(Ft, E.mat, tau);
                store_mat(p.out.F, N, slot, Ft);
            } else {
                const float J = p.in.F[src] * det3(Gm);
                const float s = E.mat.lambda * J * (J - 1.0f);
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) tau[r][c] = r == c ? s : 0.0f;
                p.out.F[slot] = J;
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                p.out.x[(size_t)a * N + slot] = xn[a];
                p.out.v[(size_t)a * N + slot] = vn[a];
            }
            store_mat(p.out.C, N, slot, Cn);
            p.out.pid[slot] = p.in.pid[src];
            newkey = E.bin_base + local_bin_of(xn, g);
            affine(E.mat, Cn, tau, A);
        }
        if constexpr (PEN) {
            if (pen) {  // the penalty impulse joins the momentum the new state transfers
                float acc[3];
                penalty_accel(p, E, cs, cw, shared_poses, step, active, xn, vn, acc);
#pragma unroll
                for (int a = 0; a < 3; ++a) vn[a] += dt * acc[a];
            }
        }
        if (active) bp = particle_bound(E.mat.p_mass, vn, A, g.dx);
        // Rank within the new bin. The 64 cells of a bin fall in 32 bank classes (bank_class): for every
        // stencil offset, tile nodes of cells in different classes lie in different banks (tile_slot).
        // The particles that stay in the chunk's bin take consecutive ranks in class-layered order: layer r
        // holds the r-th staying particle (in slot order) of each class, the classes in a fixed order; so
        // while layers are full, any 32 consecutive ranks -- a warp of the next substep, wherever the group
        // starts -- hold 32 classes and gather and scatter without bank conflicts. The others take a
        // warp-aggregated rank. The atomics' results are only stored after the scatter, so their round
        // trips overlap the work in between.
        const bool stay = p.scatter && active && newkey == (uint32_t)ch.x;
        uint32_t class_key = 0;  // layer * 32 + class
        if (stay) {
            const int c0 = cell_base(xn[0], g.inv_dx) - ox, c1 = cell_base(xn[1], g.inv_dx) - oy,
                      c2 = cell_base(xn[2], g.inv_dx) - oz;  // each in 0..3: xn is in this bin
            const uint32_t cls = bank_class(c0, c1, c2);
            const uint32_t lay = atomicAdd(&T.class_count[cls], 1u);  // < particles in the chunk
            atomicOr(&T.layer_mask[lay], 1u << cls);
            class_key = lay * 32u + cls;
        }
        // (a staying particle's rank is its layered position until the group's base is known)
        uint32_t rank = warp_hist_add(p.hist, stay ? 0xffffffffu : newkey, true);
        if (p.scatter) {
            tile_bound(T, bp, active);
            const int nstay = __syncthreads_count(stay);
            if (threadIdx.x == 0 && nstay > 0) T.stay_base = atomicAdd(&p.hist[ch.x], (uint32_t)nstay);
            if (stay) {  // the earlier layers, then this layer's classes before this one
                const uint32_t lay = class_key >> 5, cls = class_key & 31u;
                uint32_t pos = 0;
                for (uint32_t q = 0; q < lay; ++q) pos += __popc(T.layer_mask[q]);
                rank = pos + __popc(T.layer_mask[lay] & ((1u << cls) - 1u));
            }
            // ---- P2G of the new state into the next grid
            const TileScales ts = tile_scales(T);
            const int o[3] = {ox - 1, oy - 1, oz - 1};
            float mscale;
            const int tile = tile_of(bp, ts, mscale);
            if (active) flags |= scatter_particle(T, p, E, env, o, xn, vn, A, tile, mscale);
            if (active && !stay) p.keyrank_out[slot] = make_uint2(newkey, rank);
            __syncthreads();
            if (stay) p.keyrank_out[slot] = make_uint2(newkey, T.stay_base + rank);
            if (threadIdx.x == 0 && wn < nchunks) s_next[it & 1] = 2u * gridDim.x + ticket;
            tile_flush(T, p, E, env, bx, by, bz, ts);
        } else {
            if (active) p.keyrank_out[slot] = make_uint2(newkey, rank);
            if (threadIdx.x == 0 && wn < nchunks) s_next[it & 1] = 2u * gridDim.x + ticket;
        }
        // With the scatter, the barriers above already order this chunk's reads of the shared tiles before
        // the next chunk's writes: the gather tile is last read before the bound barrier, the scatter tile
        // before the flush's barrier, and a thread clearing T.touched[t] is the one that read it. Without
        // the scatter, the next gather tile must wait here.
        if (!p.scatter) __syncthreads();
        w = wn;
    }
    if constexpr (PEN)
        if (pen && shared_poses) penalty_end(p, cw);
    if (flags) atomicOr(p.status, flags);
    release_successor();
    // The last CTA to finish resets the chunk counter and, with few bins, turns the new bin counts into
    // offsets and the next chunk list. Every CTA has read its chunks and added to the counts before
    // taking its ticket.
    __shared__ uint32_t warp_tot[2][32];
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(p.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) *p.work = 0u;
    if (p.tail_scan) {
        __threadfence();
        if (p.chunk == kChunk)
            scan_bins<kChunk>(p.hist, p.cursor, p.chunks_next, p.num_chunks_next, p.bin_env, p.total_bins, kChunk,
                              warp_tot);
        else
            scan_bins<0>(p.hist, p.cursor, p.chunks_next, p.num_chunks_next, p.bin_env, p.total_bins, p.chunk,
                         warp_tot);
    }
    if (threadIdx.x == 0) *p.done = 0u;
}

// ------------------------------------------------------------------------ grid update

// A persistent CTA of 256 threads works through the active bins, four at a time (one node per thread,
// so each warp holds half of one bin): first the previous grid's bins (zeroed), then this grid's
// (updated). Each bin's env supplies its geometry and colliders. Collider poses of the substep are
// evaluated by each CTA into shared memory when the handle has few colliders, else read from the table
// filled at mpm_set_colliders (evaluated on the fly after kPoseSteps substeps). A body's impulse and
// angular impulse are summed over the warp's nodes before one FP64 atomic per component.
template <bool ONE_ENV>
__device__ __forceinline__ const EnvDesc& bin_env_desc(const GridParams& p, int env) {
    if constexpr (ONE_ENV) return p.env0;
    else return p.envs[env];
}

template <bool ONE_ENV, bool SHARED_POSES>
__device__ __forceinline__ void grid_update_cta(const GridParams& p, int cta) {
    __shared__ ColliderNow cs[SHARED_POSES ? kSharedPoses : 1];
    __shared__ float cw[SHARED_POSES ? kSharedPoses * 6 : 1];  // this CTA's wrench sums (few colliders)
    const int grp = threadIdx.x >> 6, ln = threadIdx.x & 63, lane = threadIdx.x & 31;
    // The group takes entry `item` of both bin lists per pass. The list counts and the first pass's
    // entries (their index does not depend on the counts) are requested before the pose evaluation and
    // its barrier, so the first node load waits for one round trip less.
    const uint32_t stride = (uint32_t)(p.ctas * 4);
    uint32_t item = (uint32_t)(cta * 4 + grp);
    uint32_t e_old = item < (uint32_t)p.list_cap ? p.list_old[item] : 0u;
    uint32_t e_new = item < (uint32_t)p.list_cap ? p.list[item] : 0u;
    const uint32_t n_old = *p.list_count_old, n_new = *p.list_count;
    const uint32_t step = *p.substep_counter;
    constexpr bool shared_poses = SHARED_POSES;
    if (shared_poses && p.grid_colliders) {
        if ((int)threadIdx.x < p.k_total) collider_at(p.cols[threadIdx.x], (float)step * p.dt, cs[threadIdx.x]);
        if ((int)threadIdx.x < p.k_total * 6) cw[threadIdx.x] = 0.0f;
        __syncthreads();
    }
    constexpr uint32_t kLocalMask = (1u << kLocalBinBits) - 1u;
    Pair p0[5] = {};  // mass, momentum and sum |m v|^2 / m of the transfer (for a surrogate's gate)
    for (; item < max(n_old, n_new); item += stride) {
        // item, and so env and bin, are uniform across each warp
        if (item < n_old) {  // a bin of the previous grid: zeroed for its next use
            const uint32_t lbo = e_old & kLocalMask;
            const EnvDesc& Eo = bin_env_desc<ONE_ENV>(p, (int)(e_old >> kLocalBinBits));
            p.grid_old[Eo.node_base + (size_t)lbo * kBlkNodes + ln] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (ln == 0) p.flags_old[Eo.bin_base + lbo] = 0u;
        }
        const uint32_t nx = item + stride;  // the next pass's entries, requested early
        const uint32_t e_old_next = nx < n_old ? p.list_old[nx] : 0u;
        if (item >= n_new) {
            e_old = e_old_next;
            continue;
        }
        const uint32_t entry = e_new;
        e_new = nx < n_new ? p.list[nx] : 0u;
        e_old = e_old_next;
        const int env = (int)(entry >> kLocalBinBits);
        const uint32_t lb = entry & kLocalMask;
        const EnvDesc& E = bin_env_desc<ONE_ENV>(p, env);
        const Geometry& g = E.geo;
        float4* node = &p.grid[E.node_base + (size_t)lb * kBlkNodes + ln];
        const float4 gv = *node;
        if (p.p0_sums) {  // (uniform)
            p0[0] = pair_add(p0[0], gv.x);
            p0[1] = pair_add(p0[1], gv.y);
            p0[2] = pair_add(p0[2], gv.z);
            p0[3] = pair_add(p0[3], gv.w);
            if (gv.x > 0.0f) p0[4] = pair_add(p0[4], (gv.y * gv.y + gv.z * gv.z + gv.w * gv.w) / gv.x);
        }
        const bool has_mass = gv.x > 0.0f;
        const float m = gv.x;
        const float im = has_mass ? 1.0f / m : 0.0f;
        float v[3] = {gv.y * im + p.dt * p.gravity[0], gv.z * im + p.dt * p.gravity[1],
                      gv.w * im + p.dt * p.gravity[2]};
        int bx, by, bz;
        decode_bin((int)lb, g, bx, by, bz);
        const int i = 4 * bx + (ln >> 4), j = 4 * by + ((ln >> 2) & 3), k = 4 * bz + (ln & 3);
        const float xi[3] = {i * g.dx, j * g.dx, k * g.dx};
        const int c_end = p.grid_colliders && __any_sync(0xffffffffu, has_mass) ? E.col_first + E.col_count : 0;
        for (int c = E.col_first; c < c_end; ++c) {
            ColliderNow cn;
            if (shared_poses)
                cn = cs[c];
            else if (step < (uint32_t)kPoseSteps)
                cn = p.poses[(size_t)step * p.k_total + c];
            else
                collider_at(p.cols[c], (float)step * p.dt, cn);
            float nrm[3] = {0.0f, 0.0f, 0.0f};
            const float o[3] = {xi[0] - cn.p[0], xi[1] - cn.p[1], xi[2] - cn.p[2]};
            const bool near = o[0] * o[0] + o[1] * o[1] + o[2] * o[2] <= cn.reach2;  // else surely outside
            const float phi = near ? collider_sdf(cn, xi, nrm) : 1e30f;
            const float rel[3] = {xi[0] - cn.com[0], xi[1] - cn.com[1], xi[2] - cn.com[2]};
            const float vc[3] = {cn.lin[0] + cn.ang[1] * rel[2] - cn.ang[2] * rel[1],
                                 cn.lin[1] + cn.ang[2] * rel[0] - cn.ang[0] * rel[2],
                                 cn.lin[2] + cn.ang[0] * rel[1] - cn.ang[1] * rel[0]};
            const float vr[3] = {v[0] - vc[0], v[1] - vc[1], v[2] - vc[2]};
            const float vnrm = vr[0] * nrm[0] + vr[1] * nrm[1] + vr[2] * nrm[2];
            const bool contact = has_mass && phi < 0.0f && vnrm < 0.0f;
            float w6[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (contact) {
                const float vt[3] = {vr[0] - vnrm * nrm[0], vr[1] - vnrm * nrm[1], vr[2] - vnrm * nrm[2]};
                const float tn = sqrtf(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
                const float mu = cn.friction;
                float vnew[3];
                if (tn <= -mu * vnrm) {
                    vnew[0] = vc[0]; vnew[1] = vc[1]; vnew[2] = vc[2];
                } else {
                    const float s = 1.0f + mu * vnrm / tn;
                    vnew[0] = vc[0] + vt[0] * s; vnew[1] = vc[1] + vt[1] * s; vnew[2] = vc[2] + vt[2] * s;
                }
                const float imp[3] = {m * (v[0] - vnew[0]), m * (v[1] - vnew[1]), m * (v[2] - vnew[2])};
                w6[0] = imp[0];
                w6[1] = imp[1];
                w6[2] = imp[2];
                w6[3] = rel[1] * imp[2] - rel[2] * imp[1];
                w6[4] = rel[2] * imp[0] - rel[0] * imp[2];
                w6[5] = rel[0] * imp[1] - rel[1] * imp[0];
                v[0] = vnew[0]; v[1] = vnew[1]; v[2] = vnew[2];
            }
            if (__any_sync(0xffffffffu, contact)) {
#pragma unroll
                for (int q = 0; q < 6; ++q)
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) w6[q] += __shfl_xor_sync(0xffffffffu, w6[q], off);
                if (lane == 0) {
                    if (shared_poses) {
#pragma unroll
                        for (int q = 0; q < 6; ++q) atomicAdd(&cw[c * 6 + q], w6[q]);
                    } else {
                        double* wr = p.wrench + (size_t)c * 6;
#pragma unroll
                        for (int q = 0; q < 6; ++q) atomicAdd(&wr[q], (double)w6[q]);
                    }
                }
            }
        }
        if (!has_mass) continue;
        const int lo = p.bound, hi = g.n - p.bound;
        if (i < lo || j < lo || k < lo || i >= hi || j >= hi || k >= hi) v[0] = v[1] = v[2] = 0.0f;
        *node = make_float4(v[0], v[1], v[2], m);
    }
    release_successor();  // the CTA's nodes are written: the next launch may be scheduled (it still waits)
    if (p.p0_sums) {  // (uniform) this CTA's sums as FP32 pairs, one FP64 atomic per component
        __shared__ Pair ps[8][5];
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) p0[q] = pair_add(p0[q], pair_shfl_xor(p0[q], off));
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 5; ++q) ps[threadIdx.x >> 5][q] = p0[q];
        __syncthreads();
        if (threadIdx.x < 5) {
            Pair t{0.0f, 0.0f};
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = pair_add(t, ps[w][threadIdx.x]);
            // M and P0 at p0_sums[0..4), K0 at p0_sums[kSumK0]
            if (t.hi != 0.0f) atomicAdd(&p.p0_sums[threadIdx.x < 4 ? threadIdx.x : kSumK0], pair_value(t));
        }
    }
    __syncthreads();
    if (shared_poses && p.grid_colliders && (int)threadIdx.x < p.k_total * 6 && cw[threadIdx.x] != 0.0f)
        atomicAdd(&p.wrench[threadIdx.x], (double)cw[threadIdx.x]);
    // the last CTA to finish empties the previous grid's bin list (every CTA has read its count) and
    // counts the substep (every CTA has read the count)
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(p.done, 1u) == (uint32_t)p.ctas - 1u;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        *p.list_count_old = 0u;
        *p.substep_counter = step + 1u;
        *p.done = 0u;
    }
}

// The sort-assign of the state the previous fused pass wrote (first assign_ctas CTAs) and the grid
// update of the transfer it scattered (the remaining CTAs): independent work, one launch.
// With p.scan (few bins, counts not yet scanned), every sort-assign CTA first scans the bin counts into
// shared memory for itself (a few tens of KB read from L2), so no CTA waits for another: CTA 0 also
// writes the global offsets and the next chunk list, and the last of them to finish reading the counts
// clears them for the next substep. The scan so runs beside the grid update instead of at the end of
// the fused pass, where the other SMs would idle.
template <bool ONE_ENV, bool SHARED_POSES>
__global__ void __launch_bounds__(256) k_assign_grid(AssignGridParams p) {
    extern __shared__ uint4 dyn_sh[];  // p.scan: the bin offsets (total_bins, padded to 4)
    // the next launch is scheduled once every CTA has signalled (near its end) or exited; it still waits
    // for this launch to complete before it touches memory
    wait_for_predecessor();
    if (p.gate && *p.gate != p.gate_run) return;  // the other branch of a gated window runs instead
    if ((int)blockIdx.x < p.assign_ctas) {
        if (!p.scan) {
            release_successor();
            assign_slots4(blockIdx.x * blockDim.x + threadIdx.x, p.N, p.keyrank, p.cursor, p.perm);
            return;
        }
        __shared__ uint32_t warp_tot[2][32];
        uint32_t* cur_sh = reinterpret_cast<uint32_t*>(dyn_sh);
        // this thread's (bin, rank) pairs are requested before the scan, which does not need them: a CTA
        // takes kScanAssignRounds runs of blockDim.x * kAssignPerThread particles, four per thread per run
        int j0[kScanAssignRounds];
        bool full[kScanAssignRounds];
        uint4 kr[kScanAssignRounds][2];
#pragma unroll
        for (int r = 0; r < kScanAssignRounds; ++r) {
            j0[r] = ((blockIdx.x * kScanAssignRounds + r) * blockDim.x + threadIdx.x) * kAssignPerThread;
            full[r] = j0[r] + kAssignPerThread <= p.N;
            kr[r][0] = kr[r][1] = make_uint4(0u, 0u, 0u, 0u);
            if (full[r]) {
                const uint4* q = reinterpret_cast<const uint4*>(p.keyrank + j0[r]);
                kr[r][0] = q[0];
                kr[r][1] = q[1];
            }
        }
        const bool writer = blockIdx.x == 0;
        if (p.chunk == kChunk)
            scan_counts_shared<kChunk>(p.hist, cur_sh, p.total_bins, kChunk, writer, p.cursor_out, p.chunks,
                                       p.num_chunks, p.bin_env, warp_tot);
        else
            scan_counts_shared<0>(p.hist, cur_sh, p.total_bins, p.chunk, writer, p.cursor_out, p.chunks,
                                  p.num_chunks, p.bin_env, warp_tot);
        __syncthreads();  // this CTA's reads of the counts are done, its offsets are in shared memory
        // count this CTA as done reading (no answer awaited: the first grid-update CTA clears the counts)
        if (threadIdx.x == 0) atomicAdd(p.scan_done, 1u);
        release_successor();  // only the stores of the permutation remain
#pragma unroll
        for (int r = 0; r < kScanAssignRounds; ++r) {
            if (full[r]) {
                p.perm[cur_sh[kr[r][0].x] + kr[r][0].y] = (uint32_t)j0[r];
                p.perm[cur_sh[kr[r][0].z] + kr[r][0].w] = (uint32_t)(j0[r] + 1);
                p.perm[cur_sh[kr[r][1].x] + kr[r][1].y] = (uint32_t)(j0[r] + 2);
                p.perm[cur_sh[kr[r][1].z] + kr[r][1].w] = (uint32_t)(j0[r] + 3);
            } else {
                for (int j = j0[r]; j < min(p.N, j0[r] + kAssignPerThread); ++j) assign_slot(j, p.N, p.keyrank, cur_sh, p.perm);
            }
        }
        return;
    }
    grid_update_cta<ONE_ENV, SHARED_POSES>(p.grid, blockIdx.x - p.assign_ctas);
    if (p.scan && (int)blockIdx.x == p.assign_ctas) {
        // Every sort-assign CTA has read the counts once scan_done reaches their number: clear the counts
        // for the next substep. They have lower block indices, so they were scheduled before this CTA.
        __shared__ bool ok;
        if (threadIdx.x == 0) {
            uint32_t n = 0;
            for (uint32_t it = 0; it < (1u << 20); ++it) {
                n = *(volatile uint32_t*)p.scan_done;
                if (n >= (uint32_t)p.assign_ctas) break;
            }
            ok = n >= (uint32_t)p.assign_ctas;
            if (!ok) atomicOr(p.status, kFlagInternal);
        }
        __syncthreads();
        if (ok) {
            uint4* H = reinterpret_cast<uint4*>(p.hist);
            for (int q = threadIdx.x; q < (p.total_bins + 3) >> 2; q += blockDim.x) H[q] = make_uint4(0u, 0u, 0u, 0u);
            if (threadIdx.x == 0) *p.scan_done = 0u;
        }
    }
}

// ------------------------------------------------------------------------ readback

__global__ void __launch_bounds__(256) k_read_state(int N, const EnvDesc* envs, int nenv, StateView s, float* x,
                                                    float* v, float* C, float* F) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const uint32_t p = s.pid[j];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (x) x[(size_t)a * N + p] = s.x[(size_t)a * N + j];
        if (v) v[(size_t)a * N + p] = s.v[(size_t)a * N + j];
    }
    if (C) {
#pragma unroll
        for (int i = 0; i < 9; ++i) C[(size_t)i * N + p] = s.C[(size_t)i * N + j];
    }
    if (F) {
        if (envs[env_of_particle(envs, nenv, p)].kind == 0) {
#pragma unroll
            for (int i = 0; i < 9; ++i) F[(size_t)i * N + p] = s.F[(size_t)i * N + j];
        } else {
            const float c = cbrtf(s.F[j]);
#pragma unroll
            for (int i = 0; i < 9; ++i) F[(size_t)i * N + p] = (i % 4 == 0) ? c : 0.0f;
        }
    }
}

__global__ void __launch_bounds__(256) k_read_grid(Geometry g, const float4* __restrict__ grid, float4* out) {
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t total = (size_t)g.n * g.n * g.n;
    if (t >= total) return;
    int k = (int)(t % g.n), j = (int)((t / g.n) % g.n), i = (int)(t / ((size_t)g.n * g.n));
    out[t] = grid[node_index(i, j, k, g.nb)];
}

// A collider upload of at most kSharedPoses bodies travels in the kernel parameters (no copy).
__global__ void k_set_colliders_small(ColliderUpload u, ColliderSet* table, double* wrench, uint32_t* counter) {
    const int t = threadIdx.x;
    if (t < u.k) table[t] = u.c[t];
    if (t < u.k * 6) wrench[t] = 0.0;
    if (t == 0) *counter = 0u;
}

// After a larger upload (copied to the table): the wrench and substep count restart from zero, and the
// pose table is filled: pose of collider c after s substeps for s < kPoseSteps (one thread per entry).
__global__ void k_set_colliders(const ColliderSet* cols, int k, ColliderNow* poses, double* wrench,
                                uint32_t* counter, float dt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k * 6) wrench[t] = 0.0;
    if (t == 0) *counter = 0u;
    if (k > kSharedPoses && t < k * kPoseSteps) {
        const int s = t / k, c = t % k;
        collider_at(cols[c], (float)s * dt, poses[t]);
    }
}

__global__ void __launch_bounds__(256) k_hist_from_cursor(const uint32_t* __restrict__ cursor,
                                                          uint32_t* __restrict__ hist, int total_bins, uint32_t n) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= total_bins) return;
    hist[b] = (b + 1 < total_bins ? cursor[b + 1] : n) - cursor[b];
}

__global__ void k_advance_counter(uint32_t* counter, int n, const uint32_t* gate, uint32_t gate_run) {
    if (gate && *gate != gate_run) return;
    if (threadIdx.x == 0) *counter += (uint32_t)n;
}

// ------------------------------------------------------------------------ launch wrappers

static inline unsigned ceil_div(size_t a, size_t b) { return (unsigned)((a + b - 1) / b); }

// Launch with programmatic stream serialization: the kernel may start while its predecessor on the
// stream drains; it orders itself with wait_for_predecessor().
template <typename P>
static cudaError_t launch_dependent(void (*kernel)(P), unsigned grid, unsigned block, cudaStream_t s, const P& p,
                                    size_t smem = 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, p);
}

cudaError_t launch_load(const LoadParams& p, cudaStream_t s) {
    if (p.N <= 0) return cudaSuccess;
    k_load<<<ceil_div(p.N, 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_scan(uint32_t* hist, uint32_t* cursor, int4* chunks, uint32_t* num_chunks, int nblocks,
                        int chunk, cudaStream_t s) {
    return launch_scan_binned(hist, cursor, chunks, num_chunks, nullptr, nblocks, chunk, s);
}

cudaError_t launch_scan_binned(uint32_t* hist, uint32_t* cursor, int4* chunks, uint32_t* num_chunks,
                               const uint32_t* bin_env, int nbins, int chunk, cudaStream_t s) {
    k_scan<<<1, 1024, 0, s>>>(hist, cursor, chunks, num_chunks, bin_env, nbins, chunk);
    return cudaGetLastError();
}

cudaError_t launch_scan_grid(const ScanParams& p, cudaStream_t s) {
    const unsigned tiles = ceil_div(p.total_bins, kScanTile);
    cudaError_t e = launch_dependent(k_scan_tiles, tiles, 256, s, p);
    if (e != cudaSuccess) return e;
    k_scan_apply<<<tiles, kScanTile, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_assign(int N, const uint2* keyrank, const uint32_t* cursor, uint32_t* perm, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    k_assign<<<ceil_div(N, 256 * kAssignPerThread), 256, 0, s>>>(N, keyrank, cursor, perm);
    return cudaGetLastError();
}

cudaError_t launch_p2g(const TransferParams& p, int grid_ctas, cudaStream_t s) {
    k_p2g<<<grid_ctas, kChunk, 0, s>>>(p);
    return cudaGetLastError();
}

using TransferKernel = void (*)(TransferParams);

template <int CTA>
static TransferKernel g2p2g_variant_cta(int kind_all, bool one_env, bool pen) {
    if (pen) {  // the particle contact: one-env variants per material, one for every batch
        if (one_env) return kind_all == 1 ? k_g2p2g<1, true, true, CTA> : k_g2p2g<0, true, true, CTA>;
        return k_g2p2g<-1, false, true, CTA>;
    }
    if (one_env) return kind_all == 1 ? k_g2p2g<1, true, false, CTA> : k_g2p2g<0, true, false, CTA>;
    if (kind_all == 0) return k_g2p2g<0, false, false, CTA>;
    if (kind_all == 1) return k_g2p2g<1, false, false, CTA>;
    return k_g2p2g<-1, false, false, CTA>;
}

int fused_cta_threads(int chunk) { return chunk > 128 ? 256 : 128; }

static TransferKernel g2p2g_variant(int kind_all, bool one_env, bool pen, int chunk) {
    return fused_cta_threads(chunk) == 256 ? g2p2g_variant_cta<256>(kind_all, one_env, pen)
                                           : g2p2g_variant_cta<128>(kind_all, one_env, pen);
}

cudaError_t launch_g2p2g(const TransferParams& p, int grid_ctas, cudaStream_t s) {
    return launch_dependent(g2p2g_variant(p.kind_all, p.one_env != 0, p.contact != 0, p.chunk), grid_ctas,
                            fused_cta_threads(p.chunk), s, p);
}

size_t assign_scan_smem(int total_bins) { return (size_t)((total_bins + 3) & ~3) * sizeof(uint32_t); }

cudaError_t launch_assign_grid(const AssignGridParams& p, cudaStream_t s) {
    const bool sp = p.grid.k_total <= kSharedPoses;
    auto k = p.grid.one_env ? (sp ? k_assign_grid<true, true> : k_assign_grid<true, false>)
                            : (sp ? k_assign_grid<false, true> : k_assign_grid<false, false>);
    const size_t smem = p.scan ? assign_scan_smem(p.total_bins) : 0;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return launch_dependent(k, p.assign_ctas + p.grid.ctas, 256, s, p, smem);
}

cudaError_t launch_read_state(int N, const EnvDesc* envs, int nenv, StateView src, float* x, float* v, float* C,
                              float* F, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    k_read_state<<<ceil_div(N, 256), 256, 0, s>>>(N, envs, nenv, src, x, v, C, F);
    return cudaGetLastError();
}

cudaError_t launch_read_grid(const Geometry& g, const float4* grid, float* out, cudaStream_t s) {
    size_t total = (size_t)g.n * g.n * g.n;
    k_read_grid<<<ceil_div(total, 256), 256, 0, s>>>(g, grid, reinterpret_cast<float4*>(out));
    return cudaGetLastError();
}

cudaError_t launch_set_colliders_small(const ColliderUpload& u, ColliderSet* table, double* wrench,
                                       uint32_t* counter, cudaStream_t s) {
    k_set_colliders_small<<<1, 128, 0, s>>>(u, table, wrench, counter);
    return cudaGetLastError();
}

cudaError_t launch_set_colliders(const ColliderSet* cols, int k, ColliderNow* poses, double* wrench,
                                 uint32_t* counter, float dt, cudaStream_t s) {
    const int threads = std::max(k > kSharedPoses ? k * kPoseSteps : k * 6, 1);
    k_set_colliders<<<ceil_div(threads, 256), 256, 0, s>>>(cols, k, poses, wrench, counter, dt);
    return cudaGetLastError();
}

cudaError_t launch_hist_from_cursor(const uint32_t* cursor, uint32_t* hist, int total_bins, uint32_t n,
                                    cudaStream_t s) {
    k_hist_from_cursor<<<ceil_div((size_t)total_bins, 256), 256, 0, s>>>(cursor, hist, total_bins, n);
    return cudaGetLastError();
}

cudaError_t launch_advance_counter(uint32_t* counter, int n, cudaStream_t s) {
    k_advance_counter<<<1, 32, 0, s>>>(counter, n, nullptr, 0u);
    return cudaGetLastError();
}

cudaError_t launch_advance_counter_gated(uint32_t* counter, int n, const uint32_t* gate, uint32_t gate_run,
                                         cudaStream_t s) {
    k_advance_counter<<<1, 32, 0, s>>>(counter, n, gate, gate_run);
    return cudaGetLastError();
}

int transfer_ctas_per_sm(bool fused, int kind_all, bool one_env, bool pen, int chunk) {
    int n = 0;
    cudaError_t e = fused ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, g2p2g_variant(kind_all, one_env, pen, chunk),
                                                                          fused_cta_threads(chunk), 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_p2g, kChunk, 0);
    if (e != cudaSuccess || n < 1) n = 1;
    return n;
}

}  // namespace mpm
