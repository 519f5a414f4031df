// Kernels of the surrogate network (nn.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace se2n {
namespace nn {

// 3x3 convolution, padding 1, NHWC bf16. The input is `in` (Cin channels),
// or, when lo != null, the channel concatenation [nearest-upsample(lo) (C1
// channels, half resolution), in (Cin - C1 channels)]. out = relu?(conv + bias),
// pixel p's Cout channels at out + p * ldo (ldo >= Cout, a multiple of 8).
cudaError_t conv_forward(const __nv_bfloat16 *in, const __nv_bfloat16 *lo, int C1, int B, int H, int W, int Cin,
                         const __nv_bfloat16 *w, const float *bias, int Cout, int relu, __nv_bfloat16 *out, int ldo,
                         cudaStream_t s);
// Gradient w.r.t. the input from the pre-activation gradient gz [P][Cout];
// channels < split go to din (multiplied by act > 0 when act != null),
// channels >= split to din2. wt_scratch (Cout*9*Cin elements) receives the
// rearranged weights of the tensor-core path.
cudaError_t conv_backward_data(const __nv_bfloat16 *gz, int B, int H, int W, int Cout, const __nv_bfloat16 *w, int Cin,
                               const __nv_bfloat16 *act, __nv_bfloat16 *din, __nv_bfloat16 *din2, int split,
                               __nv_bfloat16 *wt_scratch, cudaStream_t s);
// 1 in *host_flag if a tensor-core convolution gave up on a wait (never
// expected); reset clears it. Synchronous.
cudaError_t tc_fault(int *host_flag, bool reset);

// The network's 1x1 head and input skip, fused into the last convolution:
// y[p] = f[p] (mask[p] != 0) + hb + sum_c hw[c] d[p][c].
struct HeadArgs {
    const float *hw, *hb, *f;
    const uint8_t *mask;
    float *y;
};
// TMA tensor-core paths (conv_tma.cu); cudaErrorNotSupported when the shape
// is outside them (tiles of 128 pixels of one image, channel counts in
// multiples of 32), and the caller uses the general kernels.
cudaError_t conv_forward_tma(const __nv_bfloat16 *in, int B, int H, int W, int Cin, const __nv_bfloat16 *w,
                             const float *bias, int Cout, int relu, __nv_bfloat16 *out, int ldo, const HeadArgs *head,
                             cudaStream_t s);
cudaError_t conv_dgrad_tma(const __nv_bfloat16 *gz, int B, int H, int W, int Cout, const __nv_bfloat16 *wt, int Cin,
                           const __nv_bfloat16 *act, __nv_bfloat16 *din, __nv_bfloat16 *din2, int split,
                           cudaStream_t s);
cudaError_t tma_fault(int *host_flag, bool reset);
// Weight gradient on the tensor cores (MN-major TMA operands): dw [Cout][9 C] +=
// sum over pixels of x[p shifted by tap][ci] gz[p][co]; x, gz dense NHWC.
cudaError_t conv_wgrad_tma(const __nv_bfloat16 *x, int B, int H, int W, int C, const __nv_bfloat16 *gz, int Cout,
                           float *dw, cudaStream_t s);
// Channels 0..C1-1 of out (ldo channels per pixel, H x W) = nearest-upsample(lo)
// (C1 channels, H/2 x W/2).
cudaError_t upsample_into(const __nv_bfloat16 *lo, int C1, __nv_bfloat16 *out, int ldo, int B, int H, int W,
                          cudaStream_t s);
// First layer straight from the image: out = relu(conv3x3([bf16(f m), m]) + b)
// with w the layer's bf16 weights [32][9][8] (input channels 0 and 1 used).
cudaError_t conv0_direct(const float *f, const uint8_t *mask, const __nv_bfloat16 *w, const float *bias,
                         __nv_bfloat16 *out, int B, int H, int W, cudaStream_t s);
// dw[Cout][9*Cin] += weight gradient (FP32, atomically accumulated).
cudaError_t conv_backward_weight(const __nv_bfloat16 *gz, int B, int H, int W, int Cout, const __nv_bfloat16 *in,
                                 const __nv_bfloat16 *lo, int C1, int Cin, float *dw, cudaStream_t s);
cudaError_t colsum(const __nv_bfloat16 *g, long long P, int C, float *db, cudaStream_t s);
cudaError_t pack_input(const float *f, const uint8_t *mask, __nv_bfloat16 *x, long long P, cudaStream_t s);
// in: C channels per pixel at in + p * ldi; out dense (C per pixel).
cudaError_t pool(const __nv_bfloat16 *in, int ldi, __nv_bfloat16 *out, int B, int H, int W, int C, cudaStream_t s);
// e: C channels per pixel at e + p * lde.
cudaError_t pool_backward_add_mask(const __nv_bfloat16 *gp, const __nv_bfloat16 *gskip, const __nv_bfloat16 *e, int lde,
                                   __nv_bfloat16 *ge, int B, int H, int W, int C, cudaStream_t s);
cudaError_t up_backward_mask(const __nv_bfloat16 *gup, const __nv_bfloat16 *d, __nv_bfloat16 *gd, int B, int Hl,
                             int Wl, int C, cudaStream_t s);
// out[p] = f[p] (mask[p] != 0) + sum_c w[c] d[p][c] + b: the 1x1 head plus
// the input skip (FP32 f, not its bf16 copy).
cudaError_t head(const __nv_bfloat16 *d, const float *w, const float *b, const float *f, const uint8_t *mask,
                 float *out, long long P, int C, cudaStream_t s);
cudaError_t loss_head_backward(const float *out, const float *target, const __nv_bfloat16 *d, const float *w,
                               __nv_bfloat16 *gd, float *gw, float *gb, float *loss, long long P, int C,
                               cudaStream_t s);
cudaError_t adam(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, long long n, float lr, float b1,
                 float b2, float eps, int t, cudaStream_t s);
cudaError_t to_bf16(const float *p, __nv_bfloat16 *pb, long long n, cudaStream_t s);
cudaError_t known_residual(const float *out, const float *f, const uint8_t *mask, int B, int HW, float *r,
                           cudaStream_t s);

}  // namespace nn
}  // namespace se2n
