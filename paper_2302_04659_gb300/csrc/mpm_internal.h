// mpm_internal.h -- launch parameters shared by the kernels (mpm_kernels.cu) and the C-ABI host code
// (mpm_abi.cu). Not part of the public interface.
//
// A handle simulates one or more independent environments (envs) together: each env has its own grid,
// material, particles and colliders; all of them advance with the same launches. Bins get global ids
// (the env's first bin + its local bin), particles global indices (the caller's concatenated order).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm.h"
#include "mpm_device.cuh"
#include "mpm_render.h"

namespace mpm {

// Most particles per chunk of a bin = threads per CTA of the particle passes.
constexpr int kChunk = 256;

// With at most kSharedPoses colliders in a handle, each grid-update CTA evaluates the poses of the
// substep into shared memory. With more, mpm_set_colliders tabulates them for the next kPoseSteps
// substeps (later substeps evaluate them on the fly).
constexpr int kSharedPoses = 16;
constexpr int kPoseSteps = 64;

// Above this many bins (all envs), the bin counts are scanned by two grid-wide kernels instead of the
// last CTA of the fused pass.
constexpr int kTailScanMaxBins = 16384;
constexpr int kScanTile = 1024;  // bins per CTA of the grid-wide scan

// Sort-assign CTAs that also scan the bin counts take this many runs of 1,024 particles each (one scan
// per CTA serves them all).
constexpr int kScanAssignRounds = 2;

// A surrogate window's gate sums: M, P0[3], P1[3], P_hat[3] and K0 = sum_i |m v_i|^2 / m_i of the
// transfer (the scene's velocity scale), kSumWindow doubles per window.
constexpr int kSumK0 = 10;
constexpr int kSumWindow = 12;

// Internal-consistency flag: a particle was found outside the bin it was sorted into.
constexpr uint32_t kFlagInternal = 0x80000000u;

// Particle state, structure of arrays with stride N (all particles of all envs):
//   x[3N] v[3N] C[9N] F[9N] (a fluid keeps J in the first N entries of F), pid[N] after the floats.
struct StateView {
    float* x;
    float* v;
    float* C;
    float* F;
    uint32_t* pid;
};

struct Geometry {
    int n, nb;      // nodes and blocks per axis
    int nblocks;    // nb^3
    uint32_t nb_recip;  // ceil(2^32 / nb): b / nb = umulhi(b, nb_recip) exactly for b < 2^19 and nb <= 64
    float dx, inv_dx, dt;
    float lo, hi;   // particle clamp range [2dx, 1-2dx]
};

struct __align__(16) EnvDesc {
    Geometry geo;
    Material mat;
    int kind;            // MPM_PLASTICINE / MPM_FLUID
    uint32_t bin_base;   // first global bin
    uint32_t node_base;  // first node of its grids (block-major, nblocks * 64 nodes)
    int col_first, col_count;
    uint32_t part_first, part_count;  // its particles in the caller's order
};

// A bin list entry packs the env and the local bin.
constexpr int kLocalBinBits = 18;  // nb <= 64
__host__ __device__ __forceinline__ uint32_t pack_bin(uint32_t env, uint32_t local) {
    return (env << kLocalBinBits) | local;
}

struct TransferParams {  // particle passes: the fused G2P->P2G substep and the standalone P2G
    const EnvDesc* envs;
    EnvDesc env0;           // a handle of one env: its descriptor, read from the kernel parameters
    int one_env;            // 1: a single env (env0), no per-chunk descriptor loads
    int kind_all;           // the material of every env, or -1 when they differ
    int N;                  // particles of all envs (SoA stride)
    StateView in;           // read through perm
    StateView out;          // written at the sorted slot (fused pass only)
    const uint32_t* perm;   // sorted slot -> position in `in`
    uint2* keyrank_out;     // fused pass: (global bin of the new position, rank within that bin)
    uint32_t* hist;         // fused pass: particles per global bin of the new positions
    const float4* grid_in;  // fused pass: node velocities (x, y, z, mass)
    float4* grid_out;       // mass and momentum accumulated (m, mx, my, mz)
    uint32_t* flags_out;    // global bins of grid_out that received anything
    uint32_t* list_out;     // ... as packed (env, local bin) entries, each appended once
    uint32_t* list_count_out;
    const int4* chunks;     // (global bin, first sorted slot, count, env)
    const uint32_t* num_chunks;
    int chunk_cap;          // entries the chunk list can hold
    uint32_t* status;
    uint32_t* substep_counter;
    // fused pass with few bins: the last CTA to finish scans `hist` into these (the same buffers as
    // chunks / num_chunks, rewritten once every CTA is done reading them)
    int tail_scan;
    int total_bins;
    int chunk;              // most particles per chunk (<= kChunk)
    const uint32_t* gate;   // if set, the launch runs only when *gate == gate_run (read after the wait)
    uint32_t gate_run;
    const uint32_t* bin_env;  // env of every global bin (for the chunk list)
    uint32_t* cursor;
    int4* chunks_next;
    uint32_t* num_chunks_next;
    uint32_t* done;         // CTAs finished, reset by the last one
    uint32_t* work;         // fused pass: chunks handed out after each CTA's first, reset by the last CTA
    // the particle form of the contact (mpm_set_contact): penalty accelerations added to the momentum
    // each particle transfers, at the collider poses of substep *substep_counter
    int contact;            // 1: particle penalty contact
    float stiffness, damping;
    const ColliderSet* cols;
    const ColliderNow* poses;  // pose table (k_total > kSharedPoses), rows of k_total per substep
    int k_total;
    double* wrench;
    int scatter;            // fused pass: 0 = grid-to-particle only, no transfer into the next grid
};

struct ScanParams {  // grid-wide scan of the bin counts (many bins)
    uint32_t* hist;
    uint32_t* cursor;
    int4* chunks;
    uint32_t* num_chunks;
    uint2* tile_sums;       // (particles, chunks) per tile of kScanTile bins
    const uint32_t* bin_env;
    int total_bins;
    int chunk;
};

struct GridParams {
    const EnvDesc* envs;
    EnvDesc env0;             // a one-env handle's descriptor (see TransferParams)
    int one_env;
    float dt;
    float gravity[3];
    int bound;
    float4* grid;             // (m, mv) in, (v, m) out
    const uint32_t* list;     // active bins of grid (packed) and their count
    const uint32_t* list_count;
    int list_cap;             // entries either bin list can hold
    float4* grid_old;         // the previous grid, zeroed here (its active bins) for its next use
    uint32_t* flags_old;      // its bin flags, cleared
    const uint32_t* list_old;
    uint32_t* list_count_old; // reset by the last CTA to finish
    uint32_t* done;           // CTAs finished, reset by the last one
    const ColliderSet* cols;  // all envs' colliders, as set
    const ColliderNow* poses; // [kPoseSteps][k_total] poses after each substep count (k_total > kSharedPoses)
    int k_total;              // colliders of all envs
    uint32_t* substep_counter;  // read at the start, advanced by the last CTA
    double* wrench;           // k_total x 6
    int ctas;                 // CTAs of the (persistent) grid update
    int grid_colliders;       // 1: the grid form of the contact acts here (0: particle form, no colliders)
    double* p0_sums;          // if set: mass and momentum of the transfer (before the update) added here (4)
};

struct AssignGridParams {  // the sort-assign of the new state and the grid update, one launch
    GridParams grid;
    int N;
    const uint2* keyrank;
    const uint32_t* cursor;
    uint32_t* perm;
    int assign_ctas;          // the first assign_ctas CTAs assign sorted slots (0: no assign)
    // scan = 1: the counts in `hist` are not scanned yet; each assign CTA scans them for itself (the first
    // also writes cursor_out, chunks and num_chunks) and counts itself in scan_done; the first grid-update
    // CTA waits (bounded) for all of them, then clears hist and scan_done
    int scan;
    uint32_t* hist;
    uint32_t* cursor_out;
    int4* chunks;
    uint32_t* num_chunks;
    const uint32_t* bin_env;
    int total_bins;
    int chunk;
    uint32_t* scan_done;      // assign CTAs done reading the counts, reset by the CTA that clears hist
    uint32_t* status;         // error flags (a bounded wait that ran out sets kFlagInternal)
    const uint32_t* gate;     // if set, the launch runs only when *gate == gate_run (read after the wait)
    uint32_t gate_run;
};

// Argument check of a material (mpm_material rules in mpm.h); shared by the entry points.
mpm_status check_material(const mpm_material* m);

struct LoadParams {  // mpm_set_particles*: copy in, clamp, bin keys and ranks
    const EnvDesc* envs;
    int nenv;
    int N;
    const float* x;
    const float* v;
    const float* C;
    const float* F;
    StateView dst;
    uint2* keyrank;
    uint32_t* hist;
    uint32_t* status;
};

// Record a CUDA error for mpm_last_error(); returns MPM_ERR_CUDA (mpm_abi.cu).
mpm_status record_cuda_error(cudaError_t e, const char* what);

// launch wrappers (mpm_kernels.cu); each returns cudaGetLastError() after enqueueing
cudaError_t launch_load(const LoadParams& p, cudaStream_t s);
cudaError_t launch_scan(uint32_t* hist, uint32_t* cursor, int4* chunks, uint32_t* num_chunks, int nblocks,
                        int chunk, cudaStream_t s);
cudaError_t launch_scan_binned(uint32_t* hist, uint32_t* cursor, int4* chunks, uint32_t* num_chunks,
                               const uint32_t* bin_env, int nbins, int chunk, cudaStream_t s);
cudaError_t launch_scan_grid(const ScanParams& p, cudaStream_t s);
cudaError_t launch_assign(int N, const uint2* keyrank, const uint32_t* cursor, uint32_t* perm, cudaStream_t s);
cudaError_t launch_p2g(const TransferParams& p, int grid_ctas, cudaStream_t s);
cudaError_t launch_g2p2g(const TransferParams& p, int grid_ctas, cudaStream_t s);
cudaError_t launch_assign_grid(const AssignGridParams& p, cudaStream_t s);
cudaError_t launch_read_state(int N, const EnvDesc* envs, int nenv, StateView src, float* x, float* v, float* C,
                              float* F, cudaStream_t s);
cudaError_t launch_read_grid(const Geometry& g, const float4* grid, float* out, cudaStream_t s);
struct ColliderUpload {  // at most kSharedPoses colliders, passed by value to the upload kernel
    int k;
    ColliderSet c[kSharedPoses];
};
cudaError_t launch_set_colliders_small(const ColliderUpload& u, ColliderSet* table, double* wrench,
                                       uint32_t* counter, cudaStream_t s);
cudaError_t launch_set_colliders(const ColliderSet* cols, int k, ColliderNow* poses, double* wrench,
                                 uint32_t* counter, float dt, cudaStream_t s);
cudaError_t launch_advance_counter(uint32_t* counter, int n, cudaStream_t s);
// hist[b] = particles of global bin b, recovered from the exclusive offsets cursor (n particles in all)
cudaError_t launch_hist_from_cursor(const uint32_t* cursor, uint32_t* hist, int total_bins, uint32_t n,
                                    cudaStream_t s);

// surrogate window (surrogate_kernels.cu): a box of grid nodes [i0, i0 + D) x [j0, j0 + H) x [k0, k0 + W)
struct SurBox {
    int i0, j0, k0, D, H, W;
};
cudaError_t launch_sur_box(const uint32_t* list, const uint32_t* count, int nb, int nbins_cap, int* box,
                           cudaStream_t s);
cudaError_t launch_sur_step_begin(const double* wrench, double* saved, int n6, const uint32_t* counter, uint32_t* words,
                                  cudaStream_t s);
cudaError_t launch_sur_step_restore(double* wrench, const double* saved, int n6, uint32_t* counter,
                                    const uint32_t* words, cudaStream_t s);
// Scratch of the gate's one-launch check: per-block totals and the last-block ticket (reductions launch at
// most kReduceBlocks blocks: 8 resident 256-thread blocks on each of the 152 SMs).
constexpr int kReduceBlocks = 152 * 8;
struct ReduceScratch {
    Pair* partials;    // kReduceBlocks x 4 per-block totals
    uint32_t* ticket;  // zero between launches
};
// The surrogate's sums are added to `sums` (FP64, one atomic per component per block of FP32-pair totals):
// the transfer's mass and momentum (before the grid update), the updated grid's momentum over the box
// (with the network input), the corrected grid's momentum.
cudaError_t launch_sur_moments(const float4* grid, const uint32_t* list, const uint32_t* count, int nbins_cap,
                               double* sums, cudaStream_t s);
cudaError_t launch_sur_features(const float4* grid, int n, int nb, const SurBox& box, float m_scale,
                                float v_scale, float* feat, uint8_t* mask, double* sums, cudaStream_t s,
                                void* feat_bf16 = nullptr);
cudaError_t launch_sur_correct(float4* grid, int n, int nb, int bound, const SurBox& box, const float* dv,
                               float unit, int apply, double* sums, cudaStream_t s);
cudaError_t launch_wrench_extrapolate(double* wrench, const double* before, int n6, double extra, cudaStream_t s,
                                      const uint32_t* gate = nullptr, uint32_t gate_run = 1);
// The device-side gate of a window: from the sums (M, P0, P1, P_hat) the mass and momentum residuals;
// gate = 1 if both are within threshold, else 0; stats[0..1] += (windows, fallbacks), stats[2..3] the
// residuals (doubles after the two 64-bit counters).
cudaError_t launch_sur_gate(const double* sums, double m_particles, int k, double v_ref, double threshold,
                            uint32_t* gate, unsigned long long* stats, cudaStream_t s, uint32_t* any_failed = nullptr);
// The corrected grid's momentum and the gate in one launch (last block decides; sums re-zeroed).
cudaError_t launch_sur_check_gate(const float4* grid, int n, int nb, int bound, const SurBox& box, const float* dv,
                                  float unit, double* sums, double m_particles, int k, double v_ref, double threshold,
                                  uint32_t* gate, unsigned long long* stats, uint32_t* any_failed, const ReduceScratch& r,
                                  cudaStream_t s);
// The per-step gate over nwin windows whose sums are slots[10 w .. 10 w + 10): any_failed = 1 if one fails;
// stats[0] += nwin, stats[2..3] the last window's residuals; the slots are zeroed.
cudaError_t launch_sur_decide(double* slots, int nwin, double m_particles, int k, double v_ref, double threshold,
                              unsigned long long* stats, uint32_t* any_failed, cudaStream_t s);
// The correction written back (only if *gate == 1 when gate is set), with the window's substep-counter and
// body-impulse bookkeeping; with sums, the corrected grid's momentum is added to sums[0..3).
cudaError_t launch_sur_apply(float4* grid, int n, int nb, int bound, const SurBox& box, const float* dv, float unit,
                             const uint32_t* gate, uint32_t* counter, int k, double* wrench,
                             const double* wrench_before, int n6, cudaStream_t s, double* sums = nullptr);
cudaError_t launch_advance_counter_gated(uint32_t* counter, int n, const uint32_t* gate, uint32_t gate_run,
                                         cudaStream_t s);
cudaError_t launch_cast_to_bf16(int n, const float* src, void* dst, cudaStream_t s);

// the particle renderer (render_kernels.cu)
size_t render_workspace_bytes(int width, int height);
bool render_args_valid(const mpm_camera* cam, const mpm_render_params* rp);
mpm_status render_enqueue(const mpm_camera& cam, const mpm_render_params& rp, int n, int stride, const float* d_x,
                          float* d_depth, float* d_smooth, float* d_normal, float* d_rgb, void* ws, size_t bytes,
                          cudaStream_t st);

// occupancy of the particle kernels (CTAs per SM at kChunk threads), for the variant launch_g2p2g picks
int transfer_ctas_per_sm(bool fused, int kind_all, bool one_env, bool pen = false, int chunk = kChunk);
// threads per CTA of the fused pass for a chunk size (128 or 256)
int fused_cta_threads(int chunk);

}  // namespace mpm
