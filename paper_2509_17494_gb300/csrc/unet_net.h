// The learned coarse corrector's network: buffers, parameters and the
// forward / backward / training / inference sequences over the kernels of
// unet.cu.  Owned by a context; all device memory is its own (cudaMalloc).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

namespace th {

class UNet {
 public:
  // levels >= 2, base a multiple of 16 with base * 2^(levels-1) <= 128 (the
  // widest concatenation, 3 base 2^(levels-2), stays <= 256 MMA columns);
  // m = coarse nodes per direction; eta = k h_c at the m x m nodes.
  static int check(int levels, int base);
  static size_t param_count(int levels, int base);
  UNet(int levels, int base, int batch_max, int m, const std::vector<float>& eta, int* err);
  ~UNet();
  bool ok() const { return ok_; }
  size_t nparams() const { return np_; }
  int padded() const { return mp_; }
  int batch_max() const { return bmax_; }

  cudaError_t set_params(const float* host, cudaStream_t s);  // FP32 master, oracle order
  cudaError_t get_params(float* host, cudaStream_t s);
  // network only (test hooks): x [B][mp][mp][3] FP32 -> out [B][mp][mp][2] FP32
  cudaError_t forward_from(const float* x_dev, float* out_dev, int B, cudaStream_t s);
  // gradients (FP32, oracle order) of sum(out * gout) after the last forward
  cudaError_t backward_to(const float* gout_dev, float* grads_dev, int B, cudaStream_t s);
  // one Adam step on relative-error loss for pairs (rc, uc) (complex FP64 [B][m*m])
  cudaError_t train_step(const double2* rc, const double2* uc, int B, double lr, double* loss, cudaStream_t s);
  // uc = s UNet(rc / s); rc, uc complex [B][ld]
  template <typename C>
  cudaError_t correct(const C* rc, C* uc, long long ld, int B, cudaStream_t s);
  int launches_per_forward() const;

 private:
  struct Conv {
    int cin, c8, cout;  // c8 = padded input channels / 8
    size_t woff, boff;  // master offsets (weights [cout][9][cin], bias [cout])
    unsigned char* wf = nullptr;  // packed forward operand
    unsigned char* wb = nullptr;  // packed input-gradient operand (null for the first layer)
  };
  cudaError_t forward(int B, cudaStream_t s);
  cudaError_t backward(int B, cudaStream_t s);
  cudaError_t pack(cudaStream_t s);
  cudaError_t conv(const Conv& c, int level, int B, const __nv_bfloat16* x, int xs, __nv_bfloat16* z,
                   __nv_bfloat16* act, int as, int ao, cudaStream_t s);
  cudaError_t conv_back(const Conv& c, int level, int B, const __nv_bfloat16* gz, float* gx, cudaStream_t s);
  cudaError_t wgrad(const Conv& c, int level, int B, const __nv_bfloat16* gz, const __nv_bfloat16* x, int xs,
                    cudaStream_t s);
  template <typename T>
  T* alloc(size_t n);

  bool ok_ = true;
  int L_, base_, bmax_, m_, mp_;
  std::vector<int> C_;
  size_t np_ = 0, head_off_ = 0;
  int* err_;
  std::vector<void*> owned_;
  std::vector<Conv> enc_a_, enc_b_, dec_a_, dec_b_;  // per level
  float *w_ = nullptr, *g_ = nullptr, *m1_ = nullptr, *m2_ = nullptr, *eta_ = nullptr, *wpart_ = nullptr;
  size_t wpart_n_ = 0;
  long long step_ = 0;
  double *s_ = nullptr, *num_ = nullptr, *den_ = nullptr;
  // activations (BF16) per level
  __nv_bfloat16* x_ = nullptr;
  std::vector<__nv_bfloat16*> zea_, aea_, zeb_, cat_, pool_, zda_, ada_, zdb_, out_;
  __nv_bfloat16* bottom_ = nullptr;
  __nv_bfloat16* gz_ = nullptr;
  float* head_out_ = nullptr;
  float* gout_ = nullptr;
  float *ga_ = nullptr, *gb_ = nullptr;  // level-0-sized FP32 scratch
  std::vector<float*> gcat_, gp_;        // per level: concat gradient, pooled-input gradient
  float* glow_ = nullptr;
};

}  // namespace th
