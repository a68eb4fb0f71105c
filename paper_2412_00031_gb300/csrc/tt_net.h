// Kernels of the warm-start network (tt_net.cu): input features, 3x3x3 convolutions and
// their gradients, the masked mean squared error and the Adam step. Fields are
// channels-last, [grid][n_r][n_t][n_p][C], FP32.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "tt_common.cuh"

namespace ttgb {

constexpr int kNetLayers = 4;
constexpr int kNetCin[kNetLayers] = {6, 32, 32, 32};
constexpr int kNetCout[kNetLayers] = {32, 32, 32, 1};
constexpr int kNetHidden = 32;
constexpr int kNetFeatures = 6;
constexpr float kNetFeatureScaleKm = 100.0f;
constexpr float kNetClampLo = -0.5f, kNetClampHi = 1.0f;

// Offset of layer l's weights W[27][cin][cout] in the flat parameter vector; its biases
// follow them.
inline int net_weight_offset(int l) {
    int k = 0;
    for (int q = 0; q < l; ++q) k += 27 * kNetCin[q] * kNetCout[q] + kNetCout[q];
    return k;
}
inline int net_param_count() { return net_weight_offset(kNetLayers); }

struct ConvDims {
    int nb, D, H, W;  // grids in the batch and their extent
};

// The grid the warm-start network runs on: every c-th node of the solver grid along each
// axis, the last node of an axis always included (node a of an axis sits at min(a c, n - 1)),
// so nr = ceil((n_r - 1) / c) + 1 and likewise. c = 1: the solver grid itself.
struct NetGrid {
    int c, nr, nt, np;
};
inline int net_axis(int n, int c) { return c == 1 ? n : (n + c - 2) / c + 1; }
inline NetGrid net_grid_of(const GridC &g, int c) {
    return NetGrid{c, net_axis(g.nr, c), net_axis(g.nt, c), net_axis(g.np, c)};
}

// Partial sums of the weight gradient: one row of 28 x 32 x 32 per reduction block.
constexpr int kWgradBlocks = 152;
inline size_t wgrad_partial_floats() { return (size_t)kWgradBlocks * 28 * 32 * 32; }

// out = conv(in) (+ bias), ReLU applied to the inputs when relu_in, and the outputs
// zeroed where gate <= 0 when gate is given. cout is 32 or 1.
cudaError_t run_conv3d(const ConvDims &d, int cin, int cout, const float *in, bool relu_in,
                       const float *w, const float *bias, const float *gate, float *out,
                       cudaStream_t st);
// Gradient of sum(dy * conv(act(in))) with respect to W[27][cin][cout] and b[cout],
// written (overwriting) to gw and gb; partial is the scratch of wgrad_partial_floats().
cudaError_t run_conv3d_wgrad(const ConvDims &d, int cin, int cout, const float *in,
                             bool relu_in, const float *dy, float *partial, float *gw,
                             float *gb, cudaStream_t st);
// wt[26 - t][co][ci] = w[t][ci][co]: the weights of the transposed convolution.
cudaError_t run_conv3d_flip(int cin, int cout, const float *w, float *wt, cudaStream_t st);
// Masked mean squared error of y against tau - 1 (target = tau) over `total` nodes: *loss
// (device double) and dy = d loss / d y. scratch: at least 2 * 1024 + 1 doubles.
cudaError_t run_mse(long long total, const float *y, const float *target, const float *mask,
                    float *dy, double *scratch, double *loss, cudaStream_t st);
cudaError_t run_adam(int n, float *theta, const float *grad, float *m, float *v, int step,
                     float lr, float beta1, float beta2, float eps, cudaStream_t st);
// Features of sources [b0, b0 + nb) of a set-up batch (SrcC, angle tables of B sources) at
// the nodes of the network grid ng: x[b - b0][net node][6] = (s / s0 - 1, xi, eta,
// D / 100 km) of the solver node it sits on.
template <typename F>
cudaError_t run_net_features(const GridC &g, const NetGrid &ng, int B, int b0, int nb,
                             const SrcC *src, const Vec2<F> *tabT, const Vec2<F> *tabP,
                             const F *rad, const F *cost, const F *s, const F *xi, const F *eta,
                             float *x, cudaStream_t st);
// tau[node][b0 + b] = 1 + clamp(y[b][node], -0.5, 1) for b < nb, y on the network grid ng:
// with ng.c > 1 the clamped prediction is interpolated trilinearly to every solver node.
template <typename F>
cudaError_t run_warm_tau(const GridC &g, const NetGrid &ng, int B, int b0, int nb,
                         const float *y, F *tau, cudaStream_t st);
// Inference (warm start, tt_umma.cu): the four convolutions on the tensor cores (tcgen05,
// BF16 operands, FP32 accumulation in tensor memory) over the padded row layout of the
// activations: features x [nb][node][6] (FP32) are packed into b, the layers run
// b -> a -> b -> a -> y, y [nb][node] FP32. a and b hold net_rows(d) rows of 32 BF16 per
// grid. theta: the FP32 (BF16-rounded) parameters (biases); img: the weight images of
// run_net_weight_images. A device-side wait that exceeds limit_ns sets *err = 1.
size_t net_rows(const ConvDims &d);
size_t net_weight_image_elems();
cudaError_t run_net_weight_images(const float *theta, __nv_bfloat16 *img, cudaStream_t st);
cudaError_t run_net_infer(const ConvDims &d, const float *theta, const __nv_bfloat16 *img,
                          const float *x, __nv_bfloat16 *a, __nv_bfloat16 *b, float *y, int n_sm,
                          int *err, unsigned long long limit_ns, cudaStream_t st);
// Training with the convolutions on the tensor cores (tt_umma.cu): the forward pass, the
// input gradients (transposed convolutions gated by the ReLU of the layer below) and the
// weight and bias gradients (input rows times output-gradient rows, summed over the rows)
// run on tcgen05 with BF16 operands and FP32 accumulation, over the padded row layout.
// Writes the masked MSE to *loss (device double) and its gradient to grad (FP32, overwritten).
// Workspace: img (net_weight_image_elems), timg (net_tweight_image_elems), wt (27 x 32 x 32
// floats), rows (net_train_row_elems), y and dy (nb x nodes floats), partial
// (wgrad_partial_floats), scratch (4096 doubles).
size_t net_tweight_image_elems();
size_t net_train_row_elems(const ConvDims &d);
cudaError_t run_net_loss_grad_tc(const ConvDims &d, const float *theta, const float *x,
                                 const float *target, const float *mask, float *grad,
                                 double *loss, __nv_bfloat16 *img, __nv_bfloat16 *timg,
                                 float *wt, __nv_bfloat16 *rows, float *y, float *dy,
                                 float *partial, double *scratch, int n_sm, int *err,
                                 unsigned long long limit_ns, cudaStream_t st);
// Fixed-order sum of `parts` partial rows ([parts][28][1024]: rows t < 27 hold the taps'
// [cin][cout] sums, row 27 the bias sums) into gw [27][cin][cout] and gb [cout] (FP64 sums).
cudaError_t run_wgrad_reduce(int cin, int cout, int parts, const float *partial, float *gw,
                             float *gb, cudaStream_t st);
// Rounds every value to the nearest BF16 (kept in FP32 storage).
cudaError_t run_round_bf16(int n, const float *in, float *out, cudaStream_t st);

}  // namespace ttgb
