/*
 * gpair_unet.h -- C ABI of the kernels behind the learned warm start: a 3-D U-Net that maps the
 * adjoint back-projection A^T b of measured signals to initial Gaussian amplitudes.
 *
 * The paper motivates this part only indirectly: its Discussion proposes the operators as a
 * differentiable physics layer inside learned pipelines and the ImageReconstructor (the adjoint
 * alone) as an initialiser for iterative reconstruction.  The network, its layer sizes and its
 * training are this library's design.
 *
 * Tensors are single volumes in channels-last layout, element (z, y, x, c) at
 * ((z * H + y) * W + x) * C + c.  Activations and weights are bf16 (uint16_t bit patterns);
 * every kernel accumulates in FP32.  Convolutions are 3x3x3 (taps = 27, zero padding 1, stride 1)
 * or 1x1x1 (taps = 1); weights are [Cout][taps][Cin] with tap = (dz+1)*9 + (dy+1)*3 + (dx+1).
 * Channel counts: Cin a multiple of 16, Cout a multiple of 8 (the tensor-core fragment sizes).
 * All pointers are device memory; calls are asynchronous on `stream`; return gpair_status
 * (include/gpair.h).
 */
#ifndef GPAIR_UNET_H
#define GPAIR_UNET_H

#include <stdint.h>

#include "gpair.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef uint16_t gpair_bf16;

/* Convolution path of gpair_conv3d_fwd / _dgrad.  The 5th-generation tensor-core kernel (tcgen05
 * MMAs with accumulators in tensor memory, operands loaded by TMA) takes shapes with Cin and Cout
 * multiples of 16, 1 or 27 taps and 16-byte aligned tensors.  Mode 1 (default) uses it for every
 * eligible shape and the mma.sync kernel for the others; mode 2 uses it alone (an ineligible shape
 * returns GPAIR_ERR_UNSUPPORTED); mode 0 uses the mma.sync kernel alone.  Other values only
 * query.  Returns the mode in force. */
int gpair_unet_tensor_path(int mode);
/* 1 if a bounded wait of the tensor-core convolution gave up since the last call (then cleared). */
int gpair_unet_tc_status(void);

/* out = act(conv(in, w) + bias): bias FP32 [Cout] or NULL; relu != 0 applies max(., 0). */
gpair_status gpair_conv3d_fwd(const gpair_bf16* in, int D, int H, int W, int Cin, const gpair_bf16* w,
                              const float* bias, int Cout, int taps, int relu, gpair_bf16* out, void* stream);

/* din = dL/d(in) of the convolution given dout = dL/d(conv output) (before any activation):
 * the transposed convolution, computed as a convolution with flipped taps and transposed channels.
 * wt_scratch: device bf16 buffer of Cout * taps * Cin elements for the transposed weights. */
gpair_status gpair_conv3d_dgrad(const gpair_bf16* dout, int D, int H, int W, int Cout, const gpair_bf16* w,
                                int Cin, int taps, gpair_bf16* wt_scratch, gpair_bf16* din, void* stream);

/* dw[co][t][ci] += sum_v dout[v][co] in[v + off(t)][ci] (FP32, accumulated: zero it first) and
 * db[co] += sum_v dout[v][co] (db may be NULL). */
gpair_status gpair_conv3d_wgrad(const gpair_bf16* in, const gpair_bf16* dout, int D, int H, int W, int Cin, int Cout,
                                int taps, float* dw, float* db, void* stream);

/* g *= (act > 0), n elements (ReLU backward through the stored activation). */
gpair_status gpair_relu_bwd(const gpair_bf16* act, gpair_bf16* g, int64_t n, void* stream);

/* 2x2x2 average pooling (D, H, W even): out has D/2 x H/2 x W/2; and its transpose. */
gpair_status gpair_pool2_fwd(const gpair_bf16* in, int D, int H, int W, int C, gpair_bf16* out, void* stream);
gpair_status gpair_pool2_bwd(const gpair_bf16* dout, int D, int H, int W, int C, gpair_bf16* din, void* stream);

/* nearest x2 upsampling from (D, H, W) to (2D, 2H, 2W); and its transpose (sum of 8 children). */
gpair_status gpair_up2_fwd(const gpair_bf16* in, int D, int H, int W, int C, gpair_bf16* out, void* stream);
gpair_status gpair_up2_bwd(const gpair_bf16* dout, int D, int H, int W, int C, gpair_bf16* din, void* stream);

/* channel concatenation out[v] = (a[v] (Ca channels), b[v] (Cb channels)) over nv voxels, and split. */
gpair_status gpair_concat_fwd(const gpair_bf16* a, int Ca, const gpair_bf16* b, int Cb, int64_t nv, gpair_bf16* out,
                              void* stream);
gpair_status gpair_concat_bwd(const gpair_bf16* dout, int Ca, int Cb, int64_t nv, gpair_bf16* da, gpair_bf16* db,
                              void* stream);

/* out = a + b elementwise (n bf16 values; out may alias a or b). */
gpair_status gpair_add_bf16(const gpair_bf16* a, const gpair_bf16* b, gpair_bf16* out, int64_t n, void* stream);

/* x (FP32 [nv]) * scale into channel 0 of a bf16 [nv][C] tensor, other channels 0. */
gpair_status gpair_pack_input(const float* x, float scale, int64_t nv, int C, gpair_bf16* out, void* stream);
/* channel 0 of a bf16 [nv][C] tensor times scale -> FP32 [nv] (relu != 0 clamps at 0). */
gpair_status gpair_unpack_output(const gpair_bf16* in, int64_t nv, int C, float scale, int relu, float* x,
                                 void* stream);

/* Loss on channel 0 of pred (bf16 [nv][C]) against target (FP32 [nv]):
 * loss_out[0] += sum (pred - target)^2 (FP64), dpred = 2 (pred - target) / nv in channel 0, 0 elsewhere. */
gpair_status gpair_mse_loss(const gpair_bf16* pred, const float* target, int64_t nv, int C, gpair_bf16* dpred,
                            double* loss_out, void* stream);

/* Adam on FP32 master weights w (n), gradients g, moments m, v; writes the bf16 copy wb. */
gpair_status gpair_adam_bf16(float* w, const float* g, float* m, float* v, gpair_bf16* wb, int64_t n, float lr,
                             float b1, float b2, float eps, int t, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GPAIR_UNET_H */
