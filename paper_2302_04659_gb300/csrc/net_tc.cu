// net_tc.cu -- the surrogate network's forward convolution on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), behind mpm_conv3d_forward_tc (include/mpm_net.h).
//
// Implicit GEMM per tile of 1 x 16 x 8 output voxels (M = 128 rows, N = the output channels padded to 16
// or 32, K = 27 taps x input channels). The input halo (3 x 18 x 10 voxels) lands in shared memory by
// tensor-map bulk copies (TMA, zero fill outside the box) as planes of 8 channels, one 16-byte row per voxel, so the 8 voxels of a row of the tile form one
// 8 x 16-byte core matrix and the next row of the tile sits 10 voxels (160 bytes) further: the A
// operand of a tap is the plane shifted by the tap's voxel offset, described with no swizzle (leading
// byte offset = the next 8 channels, stride byte offset = 160 bytes). The weights, packed once per update
// in the same canonical K-major layout (one block per K step), arrive in each CTA by one bulk copy
// (cp.async.bulk, completion on an mbarrier). One thread issues the MMAs of a tile
// into a 32-column FP32 accumulator in tensor memory and commits them to an mbarrier; the four warps then
// read their 32 rows back (tcgen05.ld 32x32b), add the bias, apply ReLU and store. Every wait on the
// mbarrier is bounded: past the limit the kernel records an error word and leaves, freeing its tensor
// memory. Input channels: 4 (padded to 8: the two dx taps of a row pair up in one K step) or a multiple
// of 16 up to 32; output channels up to 32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "mpm_internal.h"
#include "mpm_net.h"

namespace mpm {
namespace net_tc {
namespace {

constexpr int TY = 16, TX = 8, TM = TY * TX;          // 128 rows per tile (one z plane)
constexpr int HZ = 3, HY = TY + 2, HX = TX + 2, HV = HZ * HY * HX;  // 540 halo voxels
constexpr int kPlanePad = 20;                          // zero voxels after each plane (dx over-read)
constexpr int kPlaneVox = HV + kPlanePad;
constexpr int kPlaneBytes = kPlaneVox * 16;            // 8960: planes start on 128-byte boundaries (TMA)
constexpr int kThreads = 128;
constexpr uint32_t kTmemCols = 32;
constexpr uint32_t kWaitLimit = 1u << 22;              // mbarrier polls before giving up

__device__ uint32_t g_tc_error;  // nonzero after a bounded wait ran out (mpm_net_tc_status)

struct Args {
    int D, H, W;
    int cin, cout;
    const __nv_bfloat16* x;  // [vox][cin]
    const unsigned char* wp; // weights packed in the kernel's shared-memory layout (mpm_conv3d_pack_tc)
    const float* bias;
    int relu;
    int y_f32;
    void* y;
    const uint8_t* tile_dist;  // per tile: distance to the nearest mask voxel (capped), or null
    int radius;                // with tile_dist: compute tiles within this distance
    const __nv_bfloat16* act;  // if set, [vox][cout]: outputs are zeroed where act <= 0 (a ReLU's derivative)
};

// BF16 bits that are > 0 (sign clear, not zero); a NaN's sign bit is arbitrary, it never occurs here.
__device__ __forceinline__ bool bf16_positive(uint32_t bits16) { return (bits16 & 0x8000u) == 0u && (bits16 & 0x7fffu) != 0u; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulate, BF16 A and B, both K-major, N x M.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int N>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float (&v)[N]);

template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// K steps: CG = input channel groups of 8 (1 for 4 channels, 2 or 4 for 16 or 32).
__host__ __device__ constexpr int k_steps(int cg) { return cg == 1 ? 18 : 27 * cg / 2; }

// One tile of the tensor map (channels 8 q .. 8 q + 7 of a 10 x 18 x 3 voxel box) into shared memory.
__device__ __forceinline__ void tma_plane(uint32_t dst, const CUtensorMap* map, int c, int x, int y, int z,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

// Stage the halo of tile (z0, y0, x0) into one plane buffer with asynchronous copies (4 input channels:
// 8 bytes per voxel, zero-filled outside the box; the rows' other 8 bytes stay zero).
template <int CG>
__device__ __forceinline__ void stage_async(const Args& a, uint32_t buf, int z0, int y0, int x0) {
    static_assert(CG == 1, "wider inputs arrive by tensor-map copies");
    for (int h = threadIdx.x; h < HV; h += kThreads) {
        const int z = z0 - 1 + h / (HY * HX), yy = y0 - 1 + (h / HX) % HY, xq = x0 - 1 + h % HX;
        const bool in = z >= 0 && z < a.D && yy >= 0 && yy < a.H && xq >= 0 && xq < a.W;
        const __nv_bfloat16* src = in ? a.x + (((size_t)z * a.H + yy) * a.W + xq) * a.cin : a.x;
        cp_async8(buf + h * 16, src, in ? 8u : 0u);
    }
}

template <int NPAD>
__device__ __forceinline__ void epilogue(const Args& a, uint32_t tmem_acc, int z0, int y0, int x0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = warp * 32 + lane;
    const int y = y0 + m / TX, xx = x0 + m % TX;
    float acc[NPAD];
    tmem_load<NPAD>(tmem_acc + ((uint32_t)(warp * 32) << 16), acc);
    if (y >= a.H || xx >= a.W) return;
    const size_t vox = ((size_t)z0 * a.H + y) * a.W + xx;
    if (!a.y_f32 && a.cout == 32) {
        uint32_t packed[16], am[16];
        if (a.act) {  // the ReLU mask of the layer that produced this gradient's input
            const uint4* src = reinterpret_cast<const uint4*>(a.act + vox * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 u = src[q];
                am[4 * q] = u.x; am[4 * q + 1] = u.y; am[4 * q + 2] = u.z; am[4 * q + 3] = u.w;
            }
        }
#pragma unroll
        for (int n = 0; n < 32; n += 2) {
            float v0 = acc[n] + (a.bias ? a.bias[n] : 0.0f), v1 = acc[n + 1] + (a.bias ? a.bias[n + 1] : 0.0f);
            if (a.relu) { v0 = fmaxf(v0, 0.0f); v1 = fmaxf(v1, 0.0f); }
            if (a.act) {
                if (!bf16_positive(am[n / 2] & 0xffffu)) v0 = 0.0f;
                if (!bf16_positive(am[n / 2] >> 16)) v1 = 0.0f;
            }
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(v0, v1);
            packed[n / 2] = *reinterpret_cast<const uint32_t*>(&p2);
        }
        uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.y) + vox * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
    } else {
#pragma unroll
        for (int n = 0; n < NPAD; ++n) {
            if (n >= a.cout) break;
            float v = acc[n] + (a.bias ? a.bias[n] : 0.0f);
            if (a.relu) v = fmaxf(v, 0.0f);
            if (a.act && !bf16_positive(reinterpret_cast<const uint16_t*>(a.act)[vox * a.cout + n])) v = 0.0f;
            if (a.y_f32) static_cast<float*>(a.y)[vox * a.cout + n] = v;
            else static_cast<__nv_bfloat16*>(a.y)[vox * a.cout + n] = __float2bfloat16(v);
        }
    }
}

// Programmatic dependent launch: wait for the previous launch's memory, and let the next one start.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void trigger_dependents() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// 4 input channels (the first layer), persistent, software-pipelined: while the tensor core runs the MMAs
// of tile j (accumulator j % 2), the next tile's halo lands in the other plane buffer by asynchronous
// 8-byte copies from all threads (a 4-channel voxel row is too narrow for a tensor-map copy), and the
// threads store tile j - 1 from the other accumulator. Wider inputs use k_conv_tc_ring.
template <int NPAD, int CG>
__global__ void __launch_bounds__(kThreads, 1) k_conv_tc(Args a, const __grid_constant__ CUtensorMap /*tmap*/) {
    static_assert(CG == 1, "16 or 32 input channels run k_conv_tc_ring");
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int S = k_steps(CG);
    constexpr int kBBlock = NPAD * 32;  // bytes of one K step of B: 2 k-groups x NPAD/8 n-groups x 128
    constexpr int kBuf = CG * kPlaneBytes;
    unsigned char* planes = smem;                                   // 2 buffers of CG planes
    unsigned char* bsm = smem + 2 * kBuf;                           // S blocks of kBBlock
    // [0], [1]: MMAs of a buffer done; [2]: weights landed
    uint64_t* bar = reinterpret_cast<uint64_t*>(bsm + S * kBBlock);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 5);
    const int tid = threadIdx.x, warp = tid >> 5;

    // zero both buffers: every row's upper 8 bytes (channels 4..7) and the plane padding stay zero
    for (int i = tid; i < 2 * kBuf / 16; i += kThreads)
        *reinterpret_cast<uint4*>(planes + i * 16) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int b = 0; b < 5; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + b)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar + 2)),
                     "r"((uint32_t)(S * kBBlock))
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(bsm)),
            "l"(a.wp), "r"((uint32_t)(S * kBBlock)), "r"(smem_u32(bar + 2))
            : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeroed padding, for the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // The setup above touches no data of earlier launches (the weights are static), so with programmatic
    // dependent launch it overlaps the end of the previous kernel; the input and the tile map are read
    // only after the wait. The next launch may begin its own setup once every CTA is past this point.
    grid_dependency_wait();
    trigger_dependents();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(TM, NPAD);
    const uint32_t planes_addr = smem_u32(planes), b_addr = smem_u32(bsm);
    const int tx = (a.W + TX - 1) / TX, ty = (a.H + TY - 1) / TY, tiles = tx * ty * a.D;

    auto origin = [&](int tile, int& z0, int& y0, int& x0) {
        x0 = (tile % tx) * TX;
        y0 = ((tile / tx) % ty) * TY;
        z0 = tile / (tx * ty);
    };
    // the first needed tile >= tile on this CTA's stride (or tiles); tiles passed over are zero-filled
    auto next_needed = [&](int tile) {
        for (; tile < tiles; tile += gridDim.x) {
            if (!a.tile_dist || a.tile_dist[tile] <= a.radius) return tile;
            int z0, y0, x0;
            origin(tile, z0, y0, x0);
            const int m = tid, y = y0 + m / TX, xx = x0 + m % TX;
            if (y < a.H && xx < a.W) {
                const size_t vox = ((size_t)z0 * a.H + y) * a.W + xx;
                for (int n = 0; n < a.cout; ++n) {
                    if (a.y_f32) static_cast<float*>(a.y)[vox * a.cout + n] = 0.0f;
                    else static_cast<__nv_bfloat16*>(a.y)[vox * a.cout + n] = __float2bfloat16(0.0f);
                }
            }
        }
        return tiles;
    };
    // load a tile's halo into buffer b (by all threads; waited before the buffer is used)
    auto load_halo = [&](int tile, int b) {
        int z0, y0, x0;
        origin(tile, z0, y0, x0);
        stage_async<CG>(a, planes_addr + b * kBuf, z0, y0, x0);
    };

    bool failed = !mbar_wait(smem_u32(bar + 2), 0);  // the weights
    failed = __syncthreads_or(failed) != 0;
    uint32_t ph_mma0 = 0u, ph_mma1 = 0u;
    int cur = failed ? tiles : next_needed(blockIdx.x);
    int prev = -1;  // tile whose accumulator awaits its epilogue
    int j = 0;
    if (cur < tiles) {
        load_halo(cur, 0);
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    while (cur < tiles) {
        const int b = j & 1;
        const int nxt = next_needed(cur + gridDim.x);
        if (tid == 0 && !failed) {  // the MMAs of tile `cur` from plane buffer b into accumulator b
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            // a K step pairs the dx = 0, 1 taps of a row (the second k-group is the next voxel along x,
            // 16 bytes on), then dx = 2 with an empty half. Step descriptors = base + compile-time offsets.
            const uint64_t ad0 = smem_desc(planes_addr + b * kBuf, 16u, HX * 16);
            const uint64_t bd0 = smem_desc(b_addr, (NPAD / 8) * 128, 128);
#pragma unroll
            for (int s = 0; s < S; ++s) {
                const int pair = s >> 1, half = s & 1;
                const int off = ((pair / 3) * HY + pair % 3) * HX + (half ? 2 : 0);
                mma_bf16(tmem + b * kTmemCols, ad0 + (uint64_t)off, bd0 + (uint64_t)((s * kBBlock) >> 4), idesc,
                         s > 0 ? 1u : 0u);
            }
            mma_commit(smem_u32(bar + b));
        }
        __syncwarp();
        if (prev >= 0) {  // tile prev's MMAs (buffer and accumulator 1 - b) must be done
            uint32_t& ph = b ? ph_mma0 : ph_mma1;
            if (!mbar_wait(smem_u32(bar + (1 - b)), ph)) failed = true;
            ph ^= 1u;
        }
        failed = __syncthreads_or(failed) != 0;
        if (failed) break;
        if (nxt < tiles) load_halo(nxt, 1 - b);  // overlaps the MMAs of `cur`
        if (prev >= 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int z0, y0, x0;
            origin(prev, z0, y0, x0);
            epilogue<NPAD>(a, tmem + (1 - b) * kTmemCols, z0, y0, x0);
        }
        cp_async_wait_all();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        prev = cur;
        cur = nxt;
        ++j;
    }
    if (prev >= 0 && !failed) {  // the last tile
        const int b = (j - 1) & 1;
        uint32_t& ph = b ? ph_mma1 : ph_mma0;
        if (!mbar_wait(smem_u32(bar + b), ph)) failed = true;
        failed = __syncthreads_or(failed) != 0;
        if (!failed) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int z0, y0, x0;
            origin(prev, z0, y0, x0);
            epilogue<NPAD>(a, tmem + b * kTmemCols, z0, y0, x0);
        }
    }
    if (failed && tid == 0) atomicExch(&g_tc_error, 1u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols));
}

// ---- the tensor-map path (16 or 32 input channels) with a ring of halo buffers
//
// Each CTA owns the tiles blockIdx.x, blockIdx.x + gridDim.x, ... (those within reach of the material).
// Thread 0 issues the weights' bulk copy and the halo copies of the first NB tiles at once, then, for
// tile i, waits for its halo, issues its MMAs into accumulator i % 2 and commits; after the MMAs of tile
// i - 1 are done, their halo buffer takes the copy of tile i - 1 + NB and the four warps store tile i - 1
// from its accumulator while the tensor core runs tile i. Copies are NB - 1 tiles ahead of the MMAs, so
// their latency is hidden once the ring is full.
template <int NPAD, int CG>
__host__ __device__ constexpr int ring_depth() {
    return (4 * CG * kPlaneBytes + k_steps(CG) * NPAD * 32 + 1024 <= 227 * 1024) ? 4
           : (3 * CG * kPlaneBytes + k_steps(CG) * NPAD * 32 + 1024 <= 227 * 1024) ? 3 : 2;
}

template <int NPAD, int CG>
__host__ __device__ constexpr size_t ring_smem_bytes() {
    return (size_t)ring_depth<NPAD, CG>() * CG * kPlaneBytes + (size_t)k_steps(CG) * NPAD * 32 +
           (ring_depth<NPAD, CG>() + 3) * 8 + 16;
}

template <int NPAD, int CG>
__global__ void __launch_bounds__(kThreads, 1) k_conv_tc_ring(Args a, const __grid_constant__ CUtensorMap tmap) {
    static_assert(CG >= 2, "the ring path reads its halos through the tensor map");
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int S = k_steps(CG), NB = ring_depth<NPAD, CG>();
    constexpr int kBBlock = NPAD * 32, kBuf = CG * kPlaneBytes;
    unsigned char* planes = smem;                                    // NB buffers of CG planes
    unsigned char* bsm = smem + NB * kBuf;                           // S blocks of kBBlock
    // [0, NB): a buffer's halo landed; NB, NB + 1: MMAs into an accumulator done; NB + 2: weights landed
    uint64_t* bar = reinterpret_cast<uint64_t*>(bsm + S * kBBlock);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + NB + 3);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tx = (a.W + TX - 1) / TX, ty = (a.H + TY - 1) / TY, tiles = tx * ty * a.D;
    const uint32_t planes_addr = smem_u32(planes), b_addr = smem_u32(bsm);
    auto bar_addr = [&](int k) { return smem_u32(bar + k); };
    auto needed = [&](int t) { return !a.tile_dist || a.tile_dist[t] <= a.radius; };
    auto advance = [&](int t) {  // the first needed tile >= t on this CTA's stride (or tiles)
        for (; t < tiles; t += gridDim.x)
            if (needed(t)) return t;
        return tiles;
    };
    auto origin = [&](int tile, int& z0, int& y0, int& x0) {
        x0 = (tile % tx) * TX;
        y0 = ((tile / tx) % ty) * TY;
        z0 = tile / (tx * ty);
    };
    auto issue_halo = [&](int tile, int b) {  // thread 0
        int z0, y0, x0;
        origin(tile, z0, y0, x0);
        const uint32_t full = bar_addr(b);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full), "r"((uint32_t)(CG * HV * 16))
                     : "memory");
        for (int q = 0; q < CG; ++q)
            tma_plane(planes_addr + b * kBuf + q * kPlaneBytes, &tmap, q * 8, x0 - 1, y0 - 1, z0 - 1, full);
    };

    // The setup up to the wait touches no data of earlier launches (the weights are static), so with
    // programmatic dependent launch it overlaps the end of the previous kernel; the tile map, the input
    // halos and the outputs are touched only after the wait. The next launch may begin its own setup
    // once every CTA is past the wait.
    // the planes' zero padding (the dx over-read) in every buffer
    for (int i = tid; i < NB * kBuf / 16; i += kThreads)
        if ((i % (kBuf / 16)) % kPlaneVox >= HV) *reinterpret_cast<uint4*>(planes + i * 16) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int k = 0; k < NB + 3; ++k) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_addr(k)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_addr(NB + 2)),
                     "r"((uint32_t)(S * kBBlock))
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(b_addr),
            "l"(a.wp), "r"((uint32_t)(S * kBBlock)), "r"(bar_addr(NB + 2))
            : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    grid_dependency_wait();
    trigger_dependents();
    // zero outputs of skipped tiles
    for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
        if (needed(t)) continue;
        int z0, y0, x0;
        origin(t, z0, y0, x0);
        const int y = y0 + tid / TX, xx = x0 + tid % TX;
        if (y < a.H && xx < a.W) {
            const size_t vox = ((size_t)z0 * a.H + y) * a.W + xx;
            for (int n = 0; n < a.cout; ++n) {
                if (a.y_f32) static_cast<float*>(a.y)[vox * a.cout + n] = 0.0f;
                else static_cast<__nv_bfloat16*>(a.y)[vox * a.cout + n] = __float2bfloat16(0.0f);
            }
        }
    }
    int pf = tiles;       // thread 0: the next tile to prefetch
    int issued = 0;       // thread 0: halo copies issued (copy q went to buffer q % NB, phase (q / NB) & 1)
    if (tid == 0) {
        pf = advance(blockIdx.x);
        for (; issued < NB && pf < tiles; ++issued) {
            issue_halo(pf, issued);
            pf = advance(pf + gridDim.x);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeroed padding, for the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(TM, NPAD);

    bool failed = false;
    int commits = 0;  // thread 0: MMA groups committed (group c to barrier NB + c % 2, phase (c / 2) & 1)
    int cur = advance(blockIdx.x), prev = -1, i = 0;
    while (cur < tiles) {
        const int b = i % NB, acc = i & 1;
        if (tid == 0) {
            if (i == 0 && !mbar_wait(bar_addr(NB + 2), 0)) failed = true;     // the weights
            if (!failed && !mbar_wait(bar_addr(b), (i / NB) & 1)) failed = true;  // this tile's halo
            if (!failed) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // the descriptors of step st are the tile's base descriptors plus compile-time offsets
                // (addresses stay below 256 KB, so the 14-bit address field never carries)
                const uint64_t ad0 = smem_desc(planes_addr + b * kBuf, kPlaneBytes, HX * 16);
                const uint64_t bd0 = smem_desc(b_addr, (NPAD / 8) * 128, 128);
                const uint32_t d = tmem + acc * kTmemCols;
#pragma unroll
                for (int st = 0; st < S; ++st) {
                    constexpr int half = CG / 2;
                    const int tap = st / half, q = (st % half) * 2;
                    const int off = ((tap / 9) * HY + (tap / 3) % 3) * HX + tap % 3;
                    mma_bf16(d, ad0 + (uint64_t)((q * kPlaneBytes + off * 16) >> 4),
                             bd0 + (uint64_t)((st * kBBlock) >> 4), idesc, st > 0 ? 1u : 0u);
                }
                mma_commit(bar_addr(NB + acc));
                ++commits;
            }
        }
        __syncwarp();
        if (prev >= 0 && !mbar_wait(bar_addr(NB + (1 - acc)), ((i - 1) >> 1) & 1)) failed = true;  // tile i - 1
        failed = __syncthreads_or(failed) != 0;
        if (failed) break;
        if (prev >= 0) {
            if (tid == 0 && pf < tiles) {  // tile i - 1's buffer is free: the copy NB tiles ahead
                issue_halo(pf, issued % NB);
                ++issued;
                pf = advance(pf + gridDim.x);
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int z0, y0, x0;
            origin(prev, z0, y0, x0);
            epilogue<NPAD>(a, tmem + (1 - acc) * kTmemCols, z0, y0, x0);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        prev = cur;
        cur = advance(cur + gridDim.x);
        ++i;
    }
    if (prev >= 0 && !failed) {  // the last tile
        const int acc = (i - 1) & 1;
        if (!mbar_wait(bar_addr(NB + acc), ((i - 1) >> 1) & 1)) failed = true;
        failed = __syncthreads_or(failed) != 0;
        if (!failed) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int z0, y0, x0;
            origin(prev, z0, y0, x0);
            epilogue<NPAD>(a, tmem + acc * kTmemCols, z0, y0, x0);
        }
    }
    if (failed && tid == 0) {
        atomicExch(&g_tc_error, 1u);
        // leave nothing in flight: the copies not yet consumed (from copy i on) and the last MMA group
        for (int q = i; q < issued; ++q) mbar_wait(bar_addr(q % NB), (q / NB) & 1);
        if (commits > 0) mbar_wait(bar_addr(NB + ((commits - 1) & 1)), ((commits - 1) >> 1) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols));
}

size_t smem_bytes(int npad, int cg) {
    return 2 * (size_t)cg * kPlaneBytes + (size_t)k_steps(cg) * npad * 32 + 5 * 8 + 16;
}

int npad_of(int cout) { return cout <= 16 ? 16 : 32; }
int cg_of(int cin) { return cin == 4 ? 1 : cin / 8; }
size_t packed_bytes(int cin, int cout) { return (size_t)k_steps(cg_of(cin)) * npad_of(cout) * 32; }

// The weights in the kernel's canonical K-major layout: block s (K step), k-group kg, n-group ng,
// row r (output channel), column c (k), zero where the step has no tap or channel. With `adjoint`, w is a
// forward layer's weights ([27][fwd_cout][fwd_cin]) and the layer packed is its input gradient, a
// convolution of the output gradient (fwd_cout channels, padded to cin) into fwd_cin = cout channels:
// its weight for tap t, output n, input ci is the forward weight of the mirrored tap 26 - t with the
// channel roles swapped, w[26 - t][ci][n].
__global__ void k_pack(const __nv_bfloat16* __restrict__ w, int cin, int cout, int npad, int cg,
                       __nv_bfloat16* __restrict__ out, int adjoint = 0, int fwd_cin = 0, int fwd_cout = 0) {
    const int S = k_steps(cg);
    const int total = S * 16 * npad;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = i & 7, r = (i >> 3) & 7, ng = (i >> 6) % (npad / 8), kg = (i / (8 * npad)) & 1;
        const int s = i / (16 * npad);
        const int n = ng * 8 + r;
        int tap, ci;
        bool zero = false;
        if (cg == 1) {  // a step pairs the dx = 0, 1 taps of a row, then dx = 2 with an empty half
            const int pair = s >> 1, half = s & 1;
            zero = half && kg;
            tap = pair * 3 + (half ? 2 : kg);
            ci = c;
        } else {
            tap = s / (cg / 2);
            ci = (s % (cg / 2)) * 16 + kg * 8 + c;
        }
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (!adjoint) {
            if (!zero && n < cout && ci < cin) v = w[((size_t)tap * cout + n) * cin + ci];
        } else {  // output n = a forward input channel, input ci = a forward output channel
            if (!zero && n < fwd_cin && ci < fwd_cout) v = w[((size_t)(26 - tap) * fwd_cout + ci) * fwd_cin + n];
        }
        out[i] = v;
    }
}

// Per tile: the Chebyshev distance (in voxels, capped at kDistCap) from the tile to the nearest voxel
// whose mask byte is set.
constexpr int kDistCap = 4;
constexpr int kDistThreads = 256;
__global__ void __launch_bounds__(kDistThreads, 4) k_tile_dist(int D, int H, int W, const uint8_t* __restrict__ mask,
                                                               uint8_t* __restrict__ dist) {
    const int tx = (W + TX - 1) / TX, ty = (H + TY - 1) / TY, tiles = tx * ty * D;
    constexpr int R = kDistCap;
    constexpr int EZ = 1 + 2 * R, EY = TY + 2 * R, EX = TX + 2 * R;
    constexpr int NE = EZ * EY * EX, PER = (NE + kDistThreads - 1) / kDistThreads;
    __shared__ int wmin[kDistThreads / 32];
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int x0 = (tile % tx) * TX, y0 = ((tile / tx) % ty) * TY, z0 = tile / (tx * ty);
        // this thread's voxels of the expanded box: their distances to the tile, and every mask byte
        // requested before any is used
        uint8_t dv[PER], m[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = (int)threadIdx.x + k * kDistThreads;
            const int z = z0 - R + i / (EY * EX), y = y0 - R + (i / EX) % EY, xx = x0 - R + i % EX;
            const bool in = i < NE && z >= 0 && z < D && y >= 0 && y < H && xx >= 0 && xx < W;
            const int dz = z < z0 ? z0 - z : (z > z0 ? z - z0 : 0);
            const int dy = y < y0 ? y0 - y : (y >= y0 + TY ? y - (y0 + TY - 1) : 0);
            const int dx = xx < x0 ? x0 - xx : (xx >= x0 + TX ? xx - (x0 + TX - 1) : 0);
            dv[k] = (uint8_t)max(dz, max(dy, dx));  // <= R inside the expanded box
            m[k] = in ? mask[((size_t)z * H + y) * W + xx] : (uint8_t)0;
        }
        int best = R + 1;
#pragma unroll
        for (int k = 0; k < PER; ++k)
            if (m[k]) best = min(best, (int)dv[k]);
        for (int off = 16; off > 0; off >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, off));
        if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            int b = R + 1;
            for (int w = 0; w < kDistThreads / 32; ++w) b = min(b, wmin[w]);
            dist[tile] = (uint8_t)b;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------ weight gradient
//
// dW[t][co][ci] = sum_q dy[q - o_t][co] x[q][ci] and db[co] = sum_q dy[q][co], q over the box (dy and x zero
// outside), as implicit GEMMs with K = the 128 voxels of a tile: for each of the 9 (dz, dy) rows of taps,
// D[(j, co)][ci] += sum_q A[(j, co)][q] B[q][ci] with A = dy at q - (dz, dy, j - 1) and B = x at q. Both
// operands are read MN-major from the channel planes the forward uses (one 16-byte row of 8 channels per
// voxel, so any voxel shift is 16-byte aligned): A from three copies of dy's halo, copy j loaded shifted by
// j - 1 voxels along x so that one descriptor stride (a plane) steps from copy to copy, B from the tile's
// voxels of x. M = 128 rows (three copies of up to 32 channels; rows past them are read and dropped), N =
// the input channels padded to 16 or 32, 8 K steps of 16 voxels (two rows of 8 along x). The 9
// accumulators (9 N columns of tensor memory) stay on the CTA across its tiles and reach dW once, by
// vector atomics; db is summed from the unshifted copy.
struct WgArgs {
    int D, H, W;
    int cin, cout;
    const __nv_bfloat16* x;   // [vox][cin] (cin 4, 16 or 32)
    const __nv_bfloat16* dy;  // [vox][cd], cd = the output channels padded to 4, 16 or 32 (zero past cout)
    float* dw;                // [27][cout][cin], accumulated into (zeroed by the caller)
    float* db;                // [cout], accumulated into
};

constexpr int kWgTilePlane = TM * 16;  // 2048: 8 channels of a tile's 128 voxels (row y at y * 128 bytes)
constexpr int kWgAPlanes = 16;         // the 128 rows of A span 16 planes from its base
constexpr size_t kWgSmem = (size_t)kWgAPlanes * kPlaneBytes + 2 * 4 * kWgTilePlane + 64;

// Descriptor of an MN-major operand without swizzle: core matrices of 8 K rows (voxels) x 16 bytes (8
// channels); the leading byte offset holds the stride between 8-voxel groups along K, the stride byte
// offset the stride between 8-channel groups along MN (as for K-major operands, where the K stride is
// also the leading one). Checked against the FP64 oracle; the other assignment gives wrong sums.
__device__ __forceinline__ uint64_t wg_desc(uint32_t addr, uint32_t k_stride, uint32_t mn_stride) {
    return smem_desc(addr, k_stride, mn_stride);
}

// kind::f16 instruction descriptor with both operands MN-major (the transpose bits 15 and 16 set).
__host__ __device__ constexpr uint32_t instr_desc_mn(int m, int n) { return instr_desc(m, n) | (1u << 15) | (1u << 16); }

// Stage tile (z0, y0, x0): dy's halo (the 10 x 18 x 3 box at x0 - 1, y0 - 1, z0 - 1, one row of all 8 CGD
// channels per voxel: fewer and wider tensor-map requests than plane by plane) into the staging area at
// `st_addr`, and x's tile voxels into the B buffer at `b_addr`. The tensor-map parts
// complete on `bar` (thread 0 issues them); the 4-channel parts are 8-byte asynchronous copies by every
// thread into the low half of each row (the high half stays zero), waited for with cp_async_wait_all.
template <int CGX, int CGD>
__device__ __forceinline__ void wg_stage(const WgArgs& a, const CUtensorMap* map_dy, const CUtensorMap* map_x,
                                         uint32_t st_addr, uint32_t b_addr, uint32_t bar, int z0, int y0, int x0) {
    constexpr uint32_t tma_bytes = (CGD >= 2 ? (uint32_t)CGD * HV * 16 : 0u) + (CGX >= 2 ? (uint32_t)CGX * kWgTilePlane : 0u);
    if constexpr (tma_bytes > 0) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tma_bytes) : "memory");
            if constexpr (CGD >= 2)
                tma_plane(st_addr, map_dy, 0, x0 - 1, y0 - 1, z0 - 1, bar);
            if constexpr (CGX >= 2)
                for (int q = 0; q < CGX; ++q)
                    asm volatile(
                        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
                        "[%6];" ::"r"(b_addr + q * kWgTilePlane),
                        "l"(reinterpret_cast<uint64_t>(map_x)), "r"(q * 8), "r"(x0), "r"(y0), "r"(z0), "r"(bar)
                        : "memory");
        }
    }
    if constexpr (CGD == 1) {  // dy of 4 channels
        for (int h = threadIdx.x; h < HV; h += kThreads) {
            const int z = z0 - 1 + h / (HY * HX), yy = y0 - 1 + (h / HX) % HY, xq = x0 - 1 + h % HX;
            const bool in = z >= 0 && z < a.D && yy >= 0 && yy < a.H && xq >= 0 && xq < a.W;
            const __nv_bfloat16* src = in ? a.dy + (((size_t)z * a.H + yy) * a.W + xq) * 4 : a.dy;
            cp_async8(st_addr + h * 16, src, in ? 8u : 0u);
        }
    }
    if constexpr (CGX == 1) {  // x of 4 channels: the tile's voxels
        for (int m = threadIdx.x; m < TM; m += kThreads) {
            const int yy = y0 + m / TX, xq = x0 + m % TX;
            const bool in = yy < a.H && xq < a.W;
            const __nv_bfloat16* src = in ? a.x + (((size_t)z0 * a.H + yy) * a.W + xq) * 4 : a.x;
            cp_async8(b_addr + m * 16, src, in ? 8u : 0u);
        }
    }
    if constexpr (CGD == 1 || CGX == 1) asm volatile("cp.async.commit_group;" ::: "memory");
}

// The three shifted copies of the staged halo, in planes of 8 channels: copy j holds, at halo voxel (hz, hy,
// hx), the staged voxel (hz, hy, hx + 1 - j) -- dy at (hz, hy, hx) of the box shifted by j - 1 along x --
// for hx in 1..8, the columns the MMAs read.
template <int CGD>
__device__ __forceinline__ void wg_expand(unsigned char* smem) {
    constexpr int kRows = HZ * HY * TX;  // 432 rows of 16 bytes per plane and copy
    const unsigned char* st = smem + 3 * CGD * kPlaneBytes;  // staged rows of 16 CGD bytes
    for (int i = threadIdx.x; i < 3 * CGD * kRows; i += kThreads) {
        const int jq = i / kRows, r = i % kRows, j = jq / CGD, q = jq % CGD;
        const int h = (r / TX) * HX + r % TX + 1;  // (hz, hy) = r / TX, hx = r % TX + 1
        const uint4 v = *reinterpret_cast<const uint4*>(st + (h + 1 - j) * 16 * CGD + q * 16);
        *reinterpret_cast<uint4*>(smem + (j * CGD + q) * kPlaneBytes + h * 16) = v;
    }
}

// CGX: x's planes (1: 4 channels, by 8-byte copies; 2 or 4: 16 or 32 channels, by the tensor map); CGD:
// dy's planes (1: 4 channels; 2 or 4: 16 or 32). One CTA per SM over the tiles blockIdx.x, blockIdx.x +
// gridDim.x, ..., two stages deep: tile i + 1's halo and x land (staging planes, the other B buffer) while
// the tensor core runs tile i's 72 MMAs; then the threads expand the halo into the three copies.
template <int CGX, int CGD>
__global__ void __launch_bounds__(kThreads, 1)
    k_wgrad_tc(WgArgs a, const __grid_constant__ CUtensorMap map_dy, const __grid_constant__ CUtensorMap map_x) {
    constexpr int N = CGX == 4 ? 32 : 16;               // columns of one accumulator
    constexpr int kB = (N / 8) * kWgTilePlane;          // one B buffer
    constexpr uint32_t kCols = 9 * N > 256 ? 512 : 256;  // tensor memory allocated (a power of two)
    constexpr bool kTma = CGX >= 2 || CGD >= 2, kAsync = CGX == 1 || CGD == 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    // [0, 16 planes): the copies (planes [0, 3 CGD)), the staged halo (planes [3 CGD, 4 CGD)), the rest only read
    // as A's dropped rows; then the two B buffers; then the barriers (0: staged, 1: MMAs done)
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kWgAPlanes * kPlaneBytes + 2 * kB);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 2);
    __shared__ float db_part[kThreads];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tx = (a.W + TX - 1) / TX, ty = (a.H + TY - 1) / TY, tiles = tx * ty * a.D;
    const uint32_t a_addr = smem_u32(smem), st_addr = a_addr + 3 * CGD * kPlaneBytes;
    const uint32_t b_addr = a_addr + kWgAPlanes * kPlaneBytes;
    const uint32_t staged = smem_u32(bar), done = smem_u32(bar + 1);
    // the planes' unwritten halves and pads are zero (the 8-byte copies fill only the low half of a row)
    for (int i = tid; i < (kWgAPlanes * kPlaneBytes + 2 * kB) / 16; i += kThreads)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(staged));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc_mn(TM, N);
    auto stage = [&](int t, int buf) {
        const int x0 = (t % tx) * TX, y0 = ((t / tx) % ty) * TY, z0 = t / (tx * ty);
        wg_stage<CGX, CGD>(a, &map_dy, &map_x, st_addr, b_addr + buf * kB, staged, z0, y0, x0);
    };
    const int co_db = tid % 32;  // this thread's bias-gradient channel, over voxels tid / 32 + 4 k
    float db = 0.0f;
    bool failed = false;
    int i = 0;
    if (blockIdx.x < tiles) stage(blockIdx.x, 0);
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++i) {
        // tile i staged, and tile i - 1's MMAs (readers of the copies and of the other B buffer) done
        if constexpr (kTma)
            if (!mbar_wait(staged, i & 1)) failed = true;
        if constexpr (kAsync) asm volatile("cp.async.wait_group 0;" ::: "memory");
        if (i > 0 && !mbar_wait(done, (i - 1) & 1)) failed = true;
        failed = __syncthreads_or(failed) != 0;
        if (failed) break;
        wg_expand<CGD>(smem);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the copies, for the tensor core
        __syncthreads();
        if (tile + (int)gridDim.x < tiles) stage(tile + gridDim.x, (i + 1) & 1);
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t bb = b_addr + (i & 1) * kB;
#pragma unroll
            for (int g = 0; g < 9; ++g) {
                const int dz = g / 3 - 1, dyo = g % 3 - 1;
#pragma unroll
                for (int ks = 0; ks < TM / 16; ++ks) {
                    // A: the copies' voxel (1 - dz, 2 ks + 1 - dy, 1) of the halo; B: the tile's row 2 ks
                    const uint32_t ao = a_addr + (((1 - dz) * HY + 2 * ks + 1 - dyo) * HX + 1) * 16;
                    const uint32_t bo = bb + 2 * ks * TX * 16;
                    mma_bf16(tmem + g * N, wg_desc(ao, HX * 16, kPlaneBytes), wg_desc(bo, TX * 16, kWgTilePlane),
                             idesc, (i > 0 || ks > 0) ? 1u : 0u);
                }
            }
            mma_commit(done);
        }
        // the bias gradient from the unshifted copy (copy 1) at the tile's voxels, while the MMAs run
        if (co_db < a.cout) {
            const unsigned char* c1 = smem + (CGD + co_db / 8) * kPlaneBytes;
            for (int m = tid / 32; m < TM; m += kThreads / 32) {
                const int h = (HY + m / TX + 1) * HX + m % TX + 1;
                db += __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(c1 + h * 16)[co_db % 8]);
            }
        }
    }
    if (!failed && i > 0) {  // the last tile's MMAs
        if (!mbar_wait(done, (i - 1) & 1)) failed = true;
        failed = __syncthreads_or(failed) != 0;
    }
    if (failed && tid == 0) {
        atomicExch(&g_tc_error, 1u);
        // leave nothing in flight: tile i's staging (if its wait ran out) and the last MMA group
        if constexpr (kTma) mbar_wait(staged, i & 1);
        if (i > 0) mbar_wait(done, (i - 1) & 1);
    }
    if constexpr (kAsync) asm volatile("cp.async.wait_all;" ::: "memory");
    if (!failed && i > 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int r = warp * 32 + lane, j = r / (CGD * 8), co = r % (CGD * 8);
#pragma unroll 1
        for (int gg = 0; gg < 9; ++gg) {
            const int g = (gg + blockIdx.x) % 9;  // CTAs start on different taps: fewer atomics on one address
            float v[N];
            tmem_load<N>(tmem + ((uint32_t)(warp * 32) << 16) + g * N, v);
            if (j >= 3 || co >= a.cout) continue;
            const int t = (g / 3) * 9 + (g % 3) * 3 + j;
            float* dst = a.dw + ((size_t)t * a.cout + co) * a.cin;
            if (a.cin % 4 == 0) {
#pragma unroll
                for (int c = 0; c < N; c += 4)
                    if (c < a.cin) atomicAdd(reinterpret_cast<float4*>(dst + c), make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]));
            } else {
#pragma unroll
                for (int c = 0; c < N; ++c)
                    if (c < a.cin) atomicAdd(dst + c, v[c]);
            }
        }
    }
    db_part[tid] = db;
    __syncthreads();
    if (!failed && tid < a.cout) {
        float s = 0.0f;
        for (int k = tid; k < kThreads; k += 32) s += db_part[k];
        atomicAdd(&a.db[tid], s);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// A 4-D tensor map (channels, W, H, D) of BF16 activations with `c` channels and the given box.
cudaError_t encode_act_map(CUtensorMap* map, const __nv_bfloat16* base, int c, int W, int H, int D,
                           const cuuint32_t (&box)[4]) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[4] = {(cuuint64_t)c, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D};
    const cuuint64_t strides[3] = {(cuuint64_t)c * 2, (cuuint64_t)W * c * 2, (cuuint64_t)H * W * c * 2};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(base), dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int CGX, int CGD>
cudaError_t launch_wgrad(const WgArgs& a, cudaStream_t s) {
    auto kernel = k_wgrad_tc<CGX, CGD>;
    static int sms = 0;
    if (sms == 0) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
        if (e != cudaSuccess) return e;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sms = std::max(sms, 1);
    }
    const int tiles = ((a.W + TX - 1) / TX) * ((a.H + TY - 1) / TY) * a.D;
    CUtensorMap map_dy{}, map_x{};
    if constexpr (CGD >= 2) {
        const cuuint32_t box[4] = {8 * CGD, HX, HY, HZ};  // all channels of a voxel in one row
        cudaError_t e = encode_act_map(&map_dy, a.dy, 8 * CGD, a.W, a.H, a.D, box);
        if (e != cudaSuccess) return e;
    }
    if constexpr (CGX >= 2) {
        const cuuint32_t box[4] = {8, TX, TY, 1};
        cudaError_t e = encode_act_map(&map_x, a.x, 8 * CGX, a.W, a.H, a.D, box);
        if (e != cudaSuccess) return e;
    }
    k_wgrad_tc<CGX, CGD><<<std::min(tiles, sms), kThreads, kWgSmem, s>>>(a, map_dy, map_x);
    return cudaGetLastError();
}

template <int CGX>
cudaError_t launch_wgrad_cd(const WgArgs& a, int cgd, cudaStream_t s) {
    return cgd == 1 ? launch_wgrad<CGX, 1>(a, s) : (cgd == 2 ? launch_wgrad<CGX, 2>(a, s) : launch_wgrad<CGX, 4>(a, s));
}

template <int NPAD, int CG>
cudaError_t launch(const Args& a, cudaStream_t s) {
    using Kernel = void (*)(Args, const CUtensorMap);
    Kernel kernel;
    size_t smem;
    if constexpr (CG >= 2) {
        kernel = k_conv_tc_ring<NPAD, CG>;
        smem = ring_smem_bytes<NPAD, CG>();
    } else {
        kernel = k_conv_tc<NPAD, CG>;
        smem = smem_bytes(NPAD, CG);
    }
    // resident CTAs, set up once per process (the kernels of one library run on GPUs of one kind)
    static int slots = 0;
    if (slots == 0) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
        slots = std::max(per_sm, 1) * std::max(sms, 1);
    }
    const int tiles = ((a.W + TX - 1) / TX) * ((a.H + TY - 1) / TY) * a.D;
    const int grid = std::max(1, std::min(tiles, slots));
    CUtensorMap map{};
    if (CG >= 2) {  // the activations as a 4-D tensor (channels, W, H, D); boxes of 8 x 10 x 18 x 3
        static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
        if (!encode) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
            if (e != cudaSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
        const cuuint64_t dims[4] = {(cuuint64_t)a.cin, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.D};
        const cuuint64_t strides[3] = {(cuuint64_t)a.cin * 2, (cuuint64_t)a.W * a.cin * 2,
                                       (cuuint64_t)a.H * a.W * a.cin * 2};
        const cuuint32_t box[4] = {8, HX, HY, HZ};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(a.x), dims,
                                  strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a, static_cast<const CUtensorMap>(map));
}

__global__ void k_pad_channels(size_t nvox, int c, int c_pad, const __nv_bfloat16* __restrict__ src,
                               __nv_bfloat16* __restrict__ dst) {
    const size_t total = nvox * (size_t)c_pad;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t v = i / c_pad;
        const int ch = (int)(i % c_pad);
        dst[i] = ch < c ? src[v * c + ch] : __float2bfloat16(0.0f);
    }
}

}  // namespace
}  // namespace net_tc
}  // namespace mpm

using namespace mpm::net_tc;

extern "C" {

int mpm_conv3d_tc_packed_bytes(int cin, int cout) {
    if ((cin != 4 && cin != 16 && cin != 32) || cout < 1 || cout > 32) return 0;
    return (int)packed_bytes(cin, cout);
}

mpm_status mpm_conv3d_pack_tc(int cin, int cout, const void* w, void* packed, void* stream) {
    if ((cin != 4 && cin != 16 && cin != 32) || cout < 1 || cout > 32 || !w || !packed) return MPM_ERR_INVALID_ARG;
    const int total = (int)(packed_bytes(cin, cout) / 2);
    k_pack<<<(total + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16*>(w), cin, cout, npad_of(cout), cg_of(cin), static_cast<__nv_bfloat16*>(packed));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_pack_tc");
}

int mpm_conv3d_tc_tile_count(int D, int H, int W) {
    if (D <= 0 || H <= 0 || W <= 0) return 0;
    return ((W + TX - 1) / TX) * ((H + TY - 1) / TY) * D;
}

mpm_status mpm_conv3d_tc_tile_dist(int D, int H, int W, const uint8_t* mask, uint8_t* dist, void* stream) {
    if (D <= 0 || H <= 0 || W <= 0 || !mask || !dist) return MPM_ERR_INVALID_ARG;
    const int tiles = mpm_conv3d_tc_tile_count(D, H, W);
    k_tile_dist<<<std::min(tiles, 8192), kDistThreads, 0, static_cast<cudaStream_t>(stream)>>>(D, H, W, mask, dist);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_tc_tile_dist");
}

mpm_status mpm_conv3d_forward_tc(int D, int H, int W, int cin, int cout, const void* x, const void* w_packed,
                                 const float* bias, int relu, int y_f32, void* y, const uint8_t* tile_dist,
                                 int radius, void* stream) {
    if (D <= 0 || H <= 0 || W <= 0 || !x || !w_packed || !y || cout < 1 || cout > 32 || radius < 0 ||
        (size_t)D * H * W >= ((size_t)1 << 31))
        return MPM_ERR_INVALID_ARG;
    if (cin != 4 && cin != 16 && cin != 32) return MPM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(w_packed) % 16 || reinterpret_cast<uintptr_t>(x) % 16) return MPM_ERR_INVALID_ARG;
    Args a{D, H, W, cin, cout, static_cast<const __nv_bfloat16*>(x), static_cast<const unsigned char*>(w_packed), bias,
           relu, y_f32, y, tile_dist, radius, nullptr};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const bool n16 = cout <= 16;
    if (cin == 4) e = n16 ? launch<16, 1>(a, st) : launch<32, 1>(a, st);
    else if (cin == 16) e = n16 ? launch<16, 2>(a, st) : launch<32, 2>(a, st);
    else e = n16 ? launch<16, 4>(a, st) : launch<32, 4>(a, st);
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_forward_tc");
}

mpm_status mpm_pad_channels_bf16(int nvox, int c, int c_pad, const void* src, void* dst, void* stream) {
    if (nvox < 0 || c < 1 || c_pad < c || !src || !dst) return MPM_ERR_INVALID_ARG;
    if (nvox == 0) return MPM_OK;
    const size_t total = (size_t)nvox * c_pad;
    const unsigned blocks = (unsigned)std::min<size_t>((total + 255) / 256, 152 * 16);
    k_pad_channels<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        (size_t)nvox, c, c_pad, static_cast<const __nv_bfloat16*>(src), static_cast<__nv_bfloat16*>(dst));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_pad_channels_bf16");
}

// Channel count of the tensor-core kernels' input for c channels (the padded width).
static int tc_cin_of(int c) { return c <= 4 ? 4 : (c <= 16 ? 16 : 32); }

int mpm_conv3d_tc_adjoint_packed_bytes(int cin, int cout) {
    if (cin < 1 || cin > 32 || cout < 1 || cout > 32) return 0;
    return (int)packed_bytes(tc_cin_of(cout), cin);
}

mpm_status mpm_conv3d_pack_tc_adjoint(int cin, int cout, const void* w, void* packed, void* stream) {
    if (cin < 1 || cin > 32 || cout < 1 || cout > 32 || !w || !packed) return MPM_ERR_INVALID_ARG;
    const int acin = tc_cin_of(cout), acout = cin;
    const int total = (int)(packed_bytes(acin, acout) / 2);
    k_pack<<<(total + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat16*>(w), acin, acout, npad_of(acout), cg_of(acin),
        static_cast<__nv_bfloat16*>(packed), 1, cin, cout);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_pack_tc_adjoint");
}

mpm_status mpm_conv3d_backward_data_tc(int D, int H, int W, int cin, int cout, const void* dy, const void* w_adj_packed,
                                       const void* act_in, void* dx, void* stream) {
    if (D <= 0 || H <= 0 || W <= 0 || !dy || !w_adj_packed || !dx || cin < 1 || cin > 32 || cout < 1 || cout > 32 ||
        (size_t)D * H * W >= ((size_t)1 << 31))
        return MPM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(w_adj_packed) % 16 || reinterpret_cast<uintptr_t>(dy) % 16 ||
        (act_in && cin == 32 && reinterpret_cast<uintptr_t>(act_in) % 16))
        return MPM_ERR_INVALID_ARG;
    const int acin = tc_cin_of(cout);
    Args a{D, H, W, acin, cin, static_cast<const __nv_bfloat16*>(dy), static_cast<const unsigned char*>(w_adj_packed),
           nullptr, 0, 0, dx, nullptr, 0, static_cast<const __nv_bfloat16*>(act_in)};
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    const bool n16 = cin <= 16;
    if (acin == 4) e = n16 ? launch<16, 1>(a, st) : launch<32, 1>(a, st);
    else if (acin == 16) e = n16 ? launch<16, 2>(a, st) : launch<32, 2>(a, st);
    else e = n16 ? launch<16, 4>(a, st) : launch<32, 4>(a, st);
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_backward_data_tc");
}

mpm_status mpm_conv3d_backward_weight_tc(int D, int H, int W, int cin, int cout, const void* x, const void* dy,
                                         float* dw, float* db, void* stream) {
    if (D <= 0 || H <= 0 || W <= 0 || !x || !dy || !dw || !db || cout < 1 || cout > 32 ||
        (size_t)D * H * W >= ((size_t)1 << 31))
        return MPM_ERR_INVALID_ARG;
    if (cin != 4 && cin != 16 && cin != 32) return MPM_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(x) % 16 || reinterpret_cast<uintptr_t>(dy) % 16 ||
        reinterpret_cast<uintptr_t>(dw) % 16)
        return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * 27 * cout * cin, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(db, 0, sizeof(float) * cout, st);
    if (e == cudaSuccess) {
        const WgArgs a{D, H, W, cin, cout, static_cast<const __nv_bfloat16*>(x), static_cast<const __nv_bfloat16*>(dy),
                       dw, db};
        const int cgd = cg_of(tc_cin_of(cout));
        e = cin == 4 ? launch_wgrad_cd<1>(a, cgd, st) : (cin == 16 ? launch_wgrad_cd<2>(a, cgd, st) : launch_wgrad_cd<4>(a, cgd, st));
    }
    return e == cudaSuccess ? MPM_OK : mpm::record_cuda_error(e, "mpm_conv3d_backward_weight_tc");
}

mpm_status mpm_net_tc_status(unsigned* flags, int clear, void* stream) {
    if (!flags) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_tc_error, sizeof(v), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && clear) {
        static const unsigned zero = 0;
        e = cudaMemcpyToSymbolAsync(g_tc_error, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return mpm::record_cuda_error(e, "mpm_net_tc_status");
    *flags = v;
    return MPM_OK;
}

}  // extern "C"
