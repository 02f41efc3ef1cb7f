// mpm_internal.h -- launch parameters shared by the kernels (mpm_kernels.cu) and the C-ABI host code
// (mpm_abi.cu). Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mpm_device.cuh"

namespace mpm {

// Particles per chunk of a bin = threads per CTA of the particle passes.
constexpr int kChunk = 128;

// Internal-consistency flag: a particle was found outside the bin it was sorted into.
constexpr uint32_t kFlagInternal = 0x80000000u;

// Particle state, structure of arrays with stride N (current count):
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
    float dx, inv_dx, dt;
    float lo, hi;   // particle clamp range [2dx, 1-2dx]
};

struct TransferParams {  // particle passes: the fused G2P->P2G substep and the standalone P2G
    Geometry geo;
    Material mat;
    int N;
    StateView in;           // read through perm
    StateView out;          // written at the sorted slot (fused pass only)
    const uint32_t* perm;   // sorted slot -> position in `in`
    uint2* keyrank_out;     // fused pass: (bin of the new position, rank within that bin), per sorted slot
    uint32_t* hist;         // fused pass: particles per bin of the new positions
    const float4* grid_in;  // fused pass: node velocities (x, y, z, mass)
    float4* grid_out;       // mass and momentum accumulated (m, mx, my, mz)
    uint32_t* flags_out;    // bins of grid_out that received anything
    uint32_t* list_out;     // ... and the same bins as a list, each appended once (when its flag is set)
    uint32_t* list_count_out;
    const int4* chunks;     // (bin, first sorted slot, count, 0)
    const uint32_t* num_chunks;
    uint32_t* status;
    uint32_t* substep_counter;
    // fused pass only: the last CTA to finish scans `hist` into these (the same buffers as chunks /
    // num_chunks, rewritten once every CTA is done reading them)
    uint32_t* cursor;
    int4* chunks_next;
    uint32_t* num_chunks_next;
    uint32_t* done;           // CTAs finished, reset by the last one
};

struct GridParams {
    Geometry geo;
    float gravity[3];
    int bound;
    float4* grid;             // (m, mv) in, (v, m) out
    const uint32_t* list;     // active bins of grid and their count
    const uint32_t* list_count;
    float4* grid_old;         // the previous grid, zeroed here (its active bins) for its next use
    uint32_t* flags_old;      // its bin flags, cleared
    const uint32_t* list_old;
    uint32_t* list_count_old; // reset by the last CTA to finish
    uint32_t* done;           // CTAs finished, reset by the last one
    const ColliderSet* cols;  // as set; posed at t = substep counter * dt
    int ncol;
    const uint32_t* substep_counter;
    double* wrench;           // ncol x 6
    int ctas;                 // CTAs of the (persistent) grid update
};

struct AssignGridParams {  // the sort-assign of the new state and the grid update, one launch
    GridParams grid;
    int N;
    const uint2* keyrank;
    const uint32_t* cursor;
    uint32_t* perm;
    int assign_ctas;          // the first assign_ctas CTAs assign sorted slots (0: no assign)
};

struct ColliderUpload {
    int k;
    ColliderSet c[kMaxColliders];
};

// launch wrappers (mpm_kernels.cu); each returns cudaGetLastError() after enqueueing
cudaError_t launch_load(const Geometry& g, int kind, int N, const float* x, const float* v, const float* C,
                        const float* F, StateView dst, uint2* keyrank, uint32_t* hist, uint32_t* status,
                        cudaStream_t s);
cudaError_t launch_scan(uint32_t* hist, uint32_t* cursor, int4* chunks, uint32_t* num_chunks, int nblocks,
                        int chunk, cudaStream_t s);
cudaError_t launch_assign(int N, const uint2* keyrank, const uint32_t* cursor, uint32_t* perm, cudaStream_t s);
cudaError_t launch_p2g(const TransferParams& p, int kind, int grid_ctas, int threads, cudaStream_t s);
cudaError_t launch_g2p2g(const TransferParams& p, int kind, int grid_ctas, int threads, cudaStream_t s);
cudaError_t launch_grid_update(const GridParams& p, cudaStream_t s);
cudaError_t launch_assign_grid(const AssignGridParams& p, cudaStream_t s);
cudaError_t launch_read_state(int kind, int N, StateView src, float* x, float* v, float* C, float* F,
                              cudaStream_t s);
cudaError_t launch_read_grid(const Geometry& g, const float4* grid, float* out, cudaStream_t s);
cudaError_t launch_set_colliders(const ColliderUpload& u, ColliderSet* table, double* wrench, uint32_t* counter,
                                 cudaStream_t s);
cudaError_t launch_advance_counter(uint32_t* counter, int n, cudaStream_t s);

// occupancy of the particle kernels (CTAs per SM at the given block size)
int transfer_ctas_per_sm(int kind, int threads, bool fused);

}  // namespace mpm
