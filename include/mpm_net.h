/* mpm_net.h -- C-ABI of the learned grid surrogate's network kernels (libmpm_gb300.so).
 *
 * The surrogate is an extension of the method: the paper's simulator has no learned component. Its
 * network is four 3x3x3 convolutions over a box of grid nodes (4 -> 32 -> 32 -> 32 -> 3 channels,
 * ReLU between them, zero "same" padding); these entry points are its forward and backward passes,
 * loss and optimizer step, on device memory the caller owns, enqueued on `stream` (a cudaStream_t).
 *
 * Layouts: activations are channels-last over a D x H x W box, element ((z*H + y)*W + x)*C + c;
 * weights are [27][cout][cin] with tap t = (dz*3 + dy)*3 + dx for the input offset (dz-1, dy-1, dx-1)
 * along (D, H, W); biases are float[cout]. The convolution is a cross-correlation:
 *   y[p][co] = bias[co] + sum_{t,ci} x[p + o_t][ci] * w[t][co][ci], x = 0 outside the box.
 *
 * Precision (`dtype`): MPM_NET_F32 runs FP32 CUDA-core kernels (the reference mode of the gradient
 * checks); MPM_NET_BF16 takes BF16 activations and weights and runs tensor-core (mma.sync m16n8k16)
 * kernels that accumulate in FP32. Channel counts 1..64.
 *
 * Errors: MPM_ERR_INVALID_ARG for null pointers, non-positive sizes or unsupported channel counts;
 * MPM_ERR_CUDA if a launch fails (mpm_last_error() has the detail). Nothing is allocated. */
#ifndef MPM_NET_H
#define MPM_NET_H

#include <stddef.h>
#include <stdint.h>

#include "mpm.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { MPM_NET_F32 = 0, MPM_NET_BF16 = 1 };
#define MPM_NET_MAX_CHANNELS 64

/* Forward convolution. x: D*H*W*cin, w: 27*cout*cin, y: D*H*W*cout, all of `dtype`, except that with
 * MPM_NET_BF16 and y_f32 != 0 the output y is FP32. bias may be NULL. relu != 0 applies max(., 0). */
mpm_status mpm_conv3d_forward(int dtype, int D, int H, int W, int cin, int cout, const void* x, const void* w,
                              const float* bias, int relu, int y_f32, void* y, void* stream);

/* Tiled forward (BF16 only): the forward pass over tiles of 4 x 8 x 8 voxels (D, H, W), computing only the
 * tiles whose byte in tile_flags is nonzero and writing zeros to the others. Tiles are numbered
 * ((tz * ty_count) + ty) * tx_count + tx with tx along W; mpm_conv3d_tile_count gives their number. */
mpm_status mpm_conv3d_forward_tiled(int D, int H, int W, int cin, int cout, const void* x, const void* w,
                                    const float* bias, int relu, int y_f32, void* y, const uint8_t* tile_flags,
                                    void* stream);
int mpm_conv3d_tile_count(int D, int H, int W);

/* Tile flags from a voxel mask (one byte per voxel): a tile is flagged if any voxel of it (dilate = 0),
 * or of it and its 26 neighbouring tiles (dilate = 1), is nonzero. flags: mpm_conv3d_tile_count bytes. */
mpm_status mpm_conv3d_tile_flags(int D, int H, int W, const uint8_t* mask, int dilate, uint8_t* flags,
                                 void* stream);

/* Forward pass on the 5th-generation tensor cores (tcgen05.mma, FP32 accumulators in tensor memory), BF16
 * in and out (FP32 out when y_f32 != 0). cin: 4, 16 or 32; cout: 1..32. The weights are given packed
 * (mpm_conv3d_pack_tc). Tiles are 1 x 16 x 8 voxels (D, H, W); with tile_dist (may be NULL, see
 * mpm_conv3d_tc_tile_dist) only tiles at distance <= radius are computed and the others written as
 * zeros. x and w_packed 16-byte aligned. A wait that runs out records an error word readable with
 * mpm_net_tc_status; the call returns normally. */
mpm_status mpm_conv3d_forward_tc(int D, int H, int W, int cin, int cout, const void* x, const void* w_packed,
                                 const float* bias, int relu, int y_f32, void* y, const uint8_t* tile_dist,
                                 int radius, void* stream);

/* Bytes of a layer's packed weights (0 for unsupported channel counts), and the packing of w
 * ([27][cout][cin] BF16) into that layout. */
int mpm_conv3d_tc_packed_bytes(int cin, int cout);
mpm_status mpm_conv3d_pack_tc(int cin, int cout, const void* w, void* packed, void* stream);

/* Input gradient of a layer (cin -> cout; the definition of mpm_conv3d_backward_data, with the ReLU mask of
 * act_in when it is not NULL) on the 5th-generation tensor cores: a convolution of the output gradient
 * with the layer's adjoint weights (mirrored taps, swapped channel roles), packed for it by
 * mpm_conv3d_pack_tc_adjoint from the layer's BF16 weights [27][cout][cin]
 * (mpm_conv3d_tc_adjoint_packed_bytes bytes, 0 for unsupported counts). dy: D*H*W*cp BF16 with
 * cp = 4, 16 or 32 (the smallest of those >= cout), channels beyond cout zero (mpm_pad_channels_bf16);
 * act_in and dx: D*H*W*cin BF16. cin, cout in 1..32. dy, w_adj_packed 16-byte aligned (act_in too when
 * cin = 32). */
int mpm_conv3d_tc_adjoint_packed_bytes(int cin, int cout);
mpm_status mpm_conv3d_pack_tc_adjoint(int cin, int cout, const void* w, void* packed, void* stream);
mpm_status mpm_conv3d_backward_data_tc(int D, int H, int W, int cin, int cout, const void* dy, const void* w_adj_packed,
                                       const void* act_in, void* dx, void* stream);
/* Copy nvox voxels of c BF16 channels into c_pad >= c channels, zero-filling the rest. */
mpm_status mpm_pad_channels_bf16(int nvox, int c, int c_pad, const void* src, void* dst, void* stream);

/* Tiles of the tensor-core forward over a D x H x W box, and per tile the Chebyshev distance (in voxels,
 * capped at 5) from the tile to the nearest voxel whose mask byte is set. dist: one byte per tile. */
int mpm_conv3d_tc_tile_count(int D, int H, int W);
mpm_status mpm_conv3d_tc_tile_dist(int D, int H, int W, const uint8_t* mask, uint8_t* dist, void* stream);

/* Weight and bias gradients on the tensor cores (tcgen05), the same quantities as mpm_conv3d_backward_weight:
 * dw[t][co][ci] = sum_p dy[p][co] x[p + o_t][ci] (o_t = (t/9 - 1, (t/3)%3 - 1, t%3 - 1) in (z, y, x), x zero
 * outside the box), db[co] = sum_p dy[p][co]. BF16 products, FP32 accumulation. x: D*H*W*cin BF16 with cin 4,
 * 16 or 32; dy: D*H*W*cd BF16 with cd = cout padded to 4, 16 or 32 (the padding channels zero, as
 * mpm_pad_channels_bf16 writes them); x, dy and dw 16-byte aligned. dw (27*cout*cin) and db (cout) are FP32,
 * overwritten (zeroed on the stream, then accumulated by one persistent CTA per SM). A bounded wait that runs
 * out sets the error word of mpm_net_tc_status. */
mpm_status mpm_conv3d_backward_weight_tc(int D, int H, int W, int cin, int cout, const void* x, const void* dy,
                                         float* dw, float* db, void* stream);

/* The tensor-core kernels' error word (nonzero: a wait ran out); clear != 0 resets it. Synchronizes. */
mpm_status mpm_net_tc_status(unsigned* flags, int clear, void* stream);

/* Input gradient (the adjoint of the forward map in x): dx[q][ci] = sum_{t,co} dy[q - o_t][co] w[t][co][ci],
 * multiplied by (act_in[q][ci] > 0) when act_in != NULL (the ReLU of the layer that produced x).
 * dy: D*H*W*cout, act_in and dx: D*H*W*cin, of `dtype`. */
mpm_status mpm_conv3d_backward_data(int dtype, int D, int H, int W, int cin, int cout, const void* dy,
                                    const void* w, const void* act_in, void* dx, void* stream);

/* Weight and bias gradients: dw[t][co][ci] = sum_p dy[p][co] x[p + o_t][ci], db[co] = sum_p dy[p][co].
 * x: D*H*W*cin and dy: D*H*W*cout of `dtype`; dw (27*cout*cin) and db (cout) are FP32, overwritten. */
mpm_status mpm_conv3d_backward_weight(int dtype, int D, int H, int W, int cin, int cout, const void* x,
                                      const void* dy, float* dw, float* db, void* stream);

/* Masked mean squared error over nvox voxels of C channels: L = sum_{mask} (pred - target)^2 / (n_mask*C),
 * dpred = 2 (pred - target) mask / (n_mask*C) (zero off the mask). pred and dpred of `dtype` (with
 * MPM_NET_BF16, pred may be FP32 when pred_f32 != 0); target FP32; mask one byte per voxel (nonzero =
 * counted). loss: two floats, overwritten with the loss and the number of masked voxels. */
mpm_status mpm_mse_loss(int dtype, int nvox, int C, const void* pred, int pred_f32, const float* target,
                        const uint8_t* mask, float* loss, void* dpred, void* stream);

/* One Adam step (Kingma & Ba 2015, bias-corrected, step t >= 1) on n FP32 parameters p with gradient g
 * and moments m, v (updated in place). If p_bf16 != NULL the updated parameters are also written there
 * rounded to BF16. */
mpm_status mpm_adam_step(int n, float* p, const float* g, float* m, float* v, int t, float lr, float beta1,
                         float beta2, float eps, void* p_bf16, void* stream);

/* Round n FP32 values to BF16 (round to nearest even), or widen n BF16 values to FP32. */
mpm_status mpm_cast_f32_to_bf16(int n, const float* src, void* dst, void* stream);
mpm_status mpm_cast_bf16_to_f32(int n, const void* src, float* dst, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MPM_NET_H */
