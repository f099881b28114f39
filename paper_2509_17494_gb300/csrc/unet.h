// Kernel argument blocks and launchers of the learned coarse corrector.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace th {

// 3x3 convolution, zero padding, as an implicit GEMM on the tensor cores
struct ConvArgs {
  const __nv_bfloat16* x;  // input NHWC: element (p, c) at x[p * xs + xo + c]
  int xs, xo;              // channel stride / offset (multiples of 8)
  const unsigned char* w;  // packed weights (launch_pack_weights), nchunk chunks
  const float* bias;       // cout values (mode 0) or null
  int B, H, W;             // batch and spatial size
  int C8;                  // input channel units of 8 (channels padded to 8 C8)
  int nchunk;              // conv_chunks(C8)
  int cout;                // output channels, multiple of 16 (more than 256: several launches)
  int wrows;               // rows of each packed weight chunk (0: cout); a launch reads rows [0, cout) of them
  int mode;                // 0: z = acc + bias and act = silu(z) as BF16; 1: y = acc as FP32
  __nv_bfloat16* z;        // mode 0 outputs: z[p * zs + zo + c], act[p * as + ao + c]
  int zs, zo;
  __nv_bfloat16* act;
  int as, ao;
  float* y;                // mode 1 output: y[p * ys + yo + c]
  int ys, yo;
  int* err;                // device flag, set when a bounded wait gives up
};
size_t conv_smem_bytes(int cout);
int conv_chunks(int c8);
size_t packed_weight_elems(int rows, int c8);
cudaError_t launch_conv_umma(const ConvArgs& a, cudaStream_t s);
// FP32 [cout][9][cin] -> packed BF16 operand: forward (rows = cout, K over c8 * 8
// input channels) or transpose = 1 (rows = 8 * c8 input channels, K over cout
// output channels, taps flipped) for the input-gradient convolution
cudaError_t launch_pack_weights(const float* w, __nv_bfloat16* out, int cout, int cin, int c8, int transpose,
                                cudaStream_t s);

// weight and bias gradients of a 3x3 convolution
struct WgradArgs {
  const __nv_bfloat16* gz;  // output gradient (after silu'), [p][cout], stride gs
  int gs;
  const __nv_bfloat16* x;   // the convolution's input, [p * xs + xo + c]
  int xs, xo;
  int B, H, W, cout, cin, slices;
  float* part;              // slices * cout * 9 * cin scratch
};
cudaError_t launch_wgrad(const WgradArgs& a, float* dw, float* db, const __nv_bfloat16* gz_for_bias, cudaStream_t s);

// gz = (g + gp/4 (pooled gradient of the coarser level, optional) + gk (skip, optional)) * silu'(z)
struct GradActArgs {
  const float* g;   // [p * gsd + go + c] or null
  int gsd, go;
  const float* gp;  // [P/4][C] or null
  const float* gk;  // [p * gks + gko + c] or null
  int gks, gko;
  const __nv_bfloat16* z;  // [p * zs + c]
  int zs;
  __nv_bfloat16* out;      // [p][C]
  int B, H, W, C;
};
cudaError_t launch_grad_act(const GradActArgs& a, cudaStream_t s);
cudaError_t launch_avgpool2(const __nv_bfloat16* in, int is, __nv_bfloat16* out, int B, int H, int W, int C,
                            cudaStream_t s);
cudaError_t launch_up2(const __nv_bfloat16* in, int C, __nv_bfloat16* out, int os, int oo, int B, int H, int W,
                       cudaStream_t s);
cudaError_t launch_up2_backward(const float* g, int gsd, int go, float* out, int B, int H, int W, int C,
                                cudaStream_t s);
cudaError_t launch_head(const __nv_bfloat16* act, int C, const float* w, float* out, long long npix, cudaStream_t s);
cudaError_t launch_head_backward(const float* gout, const __nv_bfloat16* act, int C, const float* w, float* ga,
                                 float* part, float* dw, long long npix, int slices, cudaStream_t s);
template <typename C>
cudaError_t launch_make_input(const C* rc, long long ldr, int m, int mp, int B, const float* eta, double* s,
                              __nv_bfloat16* x, cudaStream_t st);
cudaError_t launch_pack_input(const float* in, long long npix, __nv_bfloat16* x, cudaStream_t s);
cudaError_t launch_loss(const float* out, const double2* uc, long long ldu, const double* s, int m, int mp, int B,
                        double* num, double* den, float* gout, cudaStream_t st);
template <typename C>
cudaError_t launch_write_correction(const float* out, const double* s, int m, int mp, int B, C* uc, long long ldu,
                                    cudaStream_t st);
cudaError_t launch_adam(float* w, const float* g, float* m1, float* m2, long long n, float lr, float b1, float b2,
                        float c1, float c2, float eps, cudaStream_t s);

}  // namespace th
