// Learned coarse corrector (no counterpart in the paper; it stands in for the
// coarse solve of Algorithm 1): the kernels of a small convolutional U-Net on
// the coarse node grid, forward, backward and Adam.
//
// Activations are NHWC in BF16 ([pixel][channel], a channel stride and offset
// per tensor, so the decoder's concatenation [skip, up2(lower)] is one buffer
// written by two producers); gradients are FP32.
//
// k_conv_umma: 3x3 convolution with zero padding as an implicit GEMM on the
// tensor cores (tcgen05.mma, kind::f16, BF16 operands, FP32 accumulators in
// tensor memory): D[pixel][c_out] = sum over K of A[pixel][K] B[c_out][K], with
// K = (tap, input channel) taken in units of 8 channels (one 16-byte load of
// one pixel at one tap is one row of an 8 x 16-byte core matrix).  M = 128
// consecutive pixels per CTA, N = c_out (16..256), K in chunks of 8 units (4
// MMAs of K = 16) through a 4-deep ring.  The weights are stored per chunk in
// the core-matrix layout, so each chunk is one bulk copy (TMA engine); the
// pixel operand is gathered by producer warps.  Epilogue (warps 4-7, one
// tensor-memory lane per pixel): z = acc + bias, a = silu(z), both stored as
// BF16 (forward); or acc stored as FP32 (the input gradient, for which the
// same kernel runs with tap-flipped, channel-transposed weights: the gradient
// of a cross-correlation is the cross-correlation of the output gradient with
// the flipped kernel).  Every wait has an iteration limit and raises the
// device error flag when it gives up.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ptx.cuh"
#include "unet.h"

namespace th {
namespace {

constexpr int kUnits = 8;  // 8-channel units per K chunk (64 K)
constexpr int kStages = 4;
constexpr int kConvThreads = 384;
constexpr int kProducers = 7 * 32;  // warps 1-3 and 8-11

__device__ __forceinline__ unsigned su32(const void* p) { return ptx::smem_addr(p); }
using ptx::mbar_arrive;
using ptx::mbar_init;
using ptx::tmem_ld16;
using ptx::umma_bf16;
using ptx::umma_commit;
using ptx::umma_desc;
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

__global__ void __launch_bounds__(kConvThreads, 1) k_conv_umma(const ConvArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int cout = a.cout;
  const unsigned a_bytes = 128u * kUnits * 16u;             // pixel tile, one chunk
  const unsigned b_bytes = (unsigned)cout * kUnits * 16u;   // weight tile, one chunk
  unsigned char* abuf = smraw;                              // [kStages][a_bytes]
  unsigned char* bbuf = smraw + (size_t)kStages * a_bytes;  // [kStages][b_bytes]
  uint64_t* bars = reinterpret_cast<uint64_t*>(bbuf + (size_t)kStages * b_bytes);
  uint64_t* full = bars;               // [kStages]: producers + the weight copy
  uint64_t* empty = bars + kStages;    // [kStages]: MMAs of the chunk done
  uint64_t* done = bars + 2 * kStages;
  __shared__ unsigned tmem_base;
  __shared__ volatile int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long npix = (long long)a.B * a.H * a.W;
  const long long p0 = (long long)blockIdx.x * 128;
  const unsigned ncols = cout <= 32 ? 32u : (cout <= 64 ? 64u : (cout <= 128 ? 128u : 256u));
  const int nchunk = a.nchunk;
  const int lim = ptx::wait_limit(a.err, 1 << 20);
  if (lim == 0) {  // waits disabled: record a timeout before any barrier, copy or MMA
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }

  if (tid == 0) {
    failed = 0;
    for (int i = 0; i < kStages; ++i) {
      mbar_init(full + i, kProducers + 1);
      mbar_init(empty + i, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ weight copies + MMAs
      int issued = 0;
      auto issue = [&](int t) {
        if (t >= nchunk || failed) return;
        const int s = t % kStages, use = t / kStages;
        if (!ptx::mbar_wait_shared_flag(empty + s, (unsigned)((use & 1) ^ 1), &failed, lim)) return;
        ptx::mbar_arrive_expect_tx(full + s, b_bytes);
        const size_t wchunk = (size_t)(a.wrows ? a.wrows : cout) * kUnits * 16u;  // bytes per packed chunk
        ptx::bulk_g2s(bbuf + (size_t)s * b_bytes, a.w + (size_t)t * wchunk, b_bytes, full + s);
        issued = t + 1;
      };
      // D f32, A/B bf16, both K-major, N = cout, M = 128
      const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(cout >> 3) << 17) | (8u << 24);
      for (int t = 0; t < kStages - 1; ++t) issue(t);
      int t = 0;
      for (; t < nchunk && !failed; ++t) {
        const int s = t % kStages, use = t / kStages;
        if (!ptx::mbar_wait_shared_flag(full + s, (unsigned)(use & 1), &failed, lim)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned as = su32(abuf + (size_t)s * a_bytes), bs = su32(bbuf + (size_t)s * b_bytes);
        for (int j = 0; j < kUnits / 2; ++j) {
          const uint64_t da = umma_desc(as + (unsigned)j * 256, 128, kUnits * 128);
          const uint64_t db = umma_desc(bs + (unsigned)j * 256, 128, kUnits * 128);
          umma_bf16(tmem, da, db, idesc, (t > 0 || j > 0) ? 1u : 0u);
        }
        umma_commit(empty + s);
        issue(t + kStages - 1);
      }
      umma_commit(done);
      volatile int ignore = 0;
      ptx::mbar_wait_shared_flag(done, 0u, &ignore, ptx::kDrainPolls);
      for (int u = t; u < issued; ++u) ptx::mbar_wait_shared_flag(full + (u % kStages), (unsigned)((u / kStages) & 1), &ignore, ptx::kDrainPolls);
    }
  } else if (warp >= 4 && warp <= 7) {
    // ------------------------------------------------ epilogue
    const int q = warp - 4;
    const long long p = p0 + q * 32 + lane;
    if (!failed) ptx::mbar_wait_shared_flag(done, 0u, &failed, lim);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    for (int c0 = 0; c0 < cout; c0 += 16) {
      unsigned r[16];
      tmem_ld16(tmem + ((unsigned)(q * 32) << 16) + (unsigned)c0, r);
      if (p < npix && !failed) {
        if (a.mode == 0) {
          __align__(16) __nv_bfloat16 zb[16], ab[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float z = __uint_as_float(r[j]) + (a.bias ? a.bias[c0 + j] : 0.f);
            zb[j] = __float2bfloat16_rn(z);
            ab[j] = __float2bfloat16_rn(silu_f(z));
          }
          uint4* zd = reinterpret_cast<uint4*>(a.z + (size_t)p * a.zs + a.zo + c0);
          uint4* ad = reinterpret_cast<uint4*>(a.act + (size_t)p * a.as + a.ao + c0);
          zd[0] = reinterpret_cast<const uint4*>(zb)[0];
          zd[1] = reinterpret_cast<const uint4*>(zb)[1];
          ad[0] = reinterpret_cast<const uint4*>(ab)[0];
          ad[1] = reinterpret_cast<const uint4*>(ab)[1];
        } else {
          float4* yd = reinterpret_cast<float4*>(a.y + (size_t)p * a.ys + a.yo + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            yd[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
        }
      }
    }
  } else {
    // ------------------------------------------------ pixel-operand producers
    const int pidx = (warp <= 3) ? tid - 32 : tid - 32 - 128;  // 0 .. kProducers - 1
    const int C8 = a.C8, U = 9 * C8;
    for (int t = 0; t < nchunk; ++t) {
      const int s = t % kStages, use = t / kStages;
      if (!failed) ptx::mbar_wait_shared_flag(empty + s, (unsigned)((use & 1) ^ 1), &failed, lim);
      unsigned char* dst = abuf + (size_t)s * a_bytes;
      for (int idx = pidx; idx < 128 * kUnits; idx += kProducers) {
        const int row = idx / kUnits, uu = idx - row * kUnits;
        const int u = t * kUnits + uu;
        uint4 v = make_uint4(0, 0, 0, 0);
        const long long p = p0 + row;
        if (u < U && p < npix) {
          const int tap = u / C8, c8 = u - tap * C8;
          const int b = (int)(p / ((long long)a.H * a.W));
          const int rem = (int)(p - (long long)b * a.H * a.W);
          const int y = rem / a.W + tap / 3 - 1, x = rem % a.W + tap % 3 - 1;
          if (y >= 0 && y < a.H && x >= 0 && x < a.W)
            v = *reinterpret_cast<const uint4*>(a.x + ((size_t)((long long)b * a.H + y) * a.W + x) * a.xs + a.xo +
                                               c8 * 8);
        }
        *reinterpret_cast<uint4*>(dst + ((size_t)((row >> 3) * kUnits + uu) * 128 + (row & 7) * 16)) = v;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(full + s);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && failed) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
  }
}

// ---------------------------------------------------------------- weights
// FP32 master [c_out][tap][c_in] -> the chunked core-matrix operand of the
// forward (transpose = 0) or of the input-gradient convolution (transpose = 1:
// rows are input channels, K = (tap, output channel) with the taps flipped).
__global__ void k_pack_weights(const float* w, __nv_bfloat16* out, int cout, int cin, int rows, int kc8,
                               int nchunk, int transpose) {
  const long long total = (long long)nchunk * rows * kUnits * 8;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i & 7);
    const int r8 = (int)((i >> 3) & 7);
    const long long rest = i >> 6;
    const int uu = (int)(rest % kUnits);
    const long long rest2 = rest / kUnits;
    const int rb = (int)(rest2 % (rows / 8));
    const int chunk = (int)(rest2 / (rows / 8));
    const int row = rb * 8 + r8;
    const int u = chunk * kUnits + uu;
    const int tap = u / kc8, c = (u - tap * kc8) * 8 + e;
    float v = 0.f;
    if (tap < 9) {
      if (!transpose) {
        if (row < cout && c < cin) v = w[((size_t)row * 9 + tap) * cin + c];
      } else {
        // row = input channel, c = output channel, tap flipped
        if (row < cin && c < cout) v = w[((size_t)c * 9 + (8 - tap)) * cin + row];
      }
    }
    out[i] = __float2bfloat16_rn(v);
  }
}

// ---------------------------------------------------------------- weight gradient
// dW[co][tap][ci] = sum_p gz[p][co] x[p + off(tap)][ci]; CTA = (16 co x 16 ci
// tile, pixel slice); partial sums [slice][co][tap][ci], reduced in slice order.
__global__ void __launch_bounds__(256) k_wgrad(const WgradArgs a) {
  __shared__ float gs[32][17];
  __shared__ float xs[32][9][17];
  const int tiles_ci = (a.cin + 15) / 16;
  const int tile = blockIdx.x % (tiles_ci * ((a.cout + 15) / 16));
  const int slice = blockIdx.x / (tiles_ci * ((a.cout + 15) / 16));
  const int co0 = (tile / tiles_ci) * 16, ci0 = (tile % tiles_ci) * 16;
  const long long npix = (long long)a.B * a.H * a.W;
  const long long per = (npix + a.slices - 1) / a.slices;
  const long long pb = slice * per, pe = min(npix, pb + per);
  float acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = 0.f;
  const int tid = threadIdx.x;
  const int oc = tid >> 4, ic = tid & 15;  // this thread: (co0 + oc, all taps, ci0 + ic)
  for (long long q0 = pb; q0 < pe; q0 += 32) {
    __syncthreads();
    for (int i = tid; i < 32 * 16; i += 256) {
      const int pp = i >> 4, c = i & 15;
      const long long p = q0 + pp;
      gs[pp][c] = (p < pe && co0 + c < a.cout) ? __bfloat162float(a.gz[(size_t)p * a.gs + co0 + c]) : 0.f;
    }
    for (int i = tid; i < 32 * 9 * 16; i += 256) {
      const int pp = i / 144, rem = i - pp * 144, tap = rem >> 4, c = rem & 15;
      const long long p = q0 + pp;
      float v = 0.f;
      if (p < pe && ci0 + c < a.cin) {
        const int b = (int)(p / ((long long)a.H * a.W));
        const int r = (int)(p - (long long)b * a.H * a.W);
        const int y = r / a.W + tap / 3 - 1, x = r % a.W + tap % 3 - 1;
        if (y >= 0 && y < a.H && x >= 0 && x < a.W)
          v = __bfloat162float(a.x[((size_t)((long long)b * a.H + y) * a.W + x) * a.xs + a.xo + ci0 + c]);
      }
      xs[pp][tap][c] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int pp = 0; pp < 32; ++pp) {
      const float g = gs[pp][oc];
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) acc[tap] += g * xs[pp][tap][ic];
    }
  }
  if (co0 + oc < a.cout && ci0 + ic < a.cin) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
      a.part[(((size_t)slice * a.cout + co0 + oc) * 9 + tap) * a.cin + ci0 + ic] = acc[tap];
  }
}

__global__ void k_sum_slices(const float* part, float* out, long long n, int slices) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < slices; ++k) s += part[(size_t)k * n + i];
    out[i] = s;
  }
}

// bias gradient: db[c] = sum_p gz[p][c], slices then k_sum_slices
__global__ void k_bias_grad(const __nv_bfloat16* gz, int gs, int C, long long npix, int slices, float* part) {
  const int slice = blockIdx.x;
  const long long per = (npix + slices - 1) / slices;
  const long long pb = slice * per, pe = min(npix, pb + per);
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float s = 0.f;
    for (long long p = pb; p < pe; ++p) s += __bfloat162float(gz[(size_t)p * gs + c]);
    part[(size_t)slice * C + c] = s;
  }
}

// ---------------------------------------------------------------- elementwise
// gz = (g [+ pooled-up gradient gp/4 of the coarser level] [+ skip gradient gk]) * silu'(z)
__global__ void k_grad_act(const GradActArgs a) {
  const long long n = (long long)a.B * a.H * a.W * a.C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % a.C);
    const long long p = i / a.C;
    float g = a.g ? a.g[(size_t)p * a.gsd + a.go + c] : 0.f;
    if (a.gp) {
      const int b = (int)(p / ((long long)a.H * a.W));
      const int r = (int)(p - (long long)b * a.H * a.W);
      const int y = r / a.W, x = r % a.W;
      const size_t pc = ((size_t)b * (a.H / 2) + y / 2) * (a.W / 2) + x / 2;
      g += 0.25f * a.gp[pc * a.C + c];
    }
    if (a.gk) g += a.gk[(size_t)p * a.gks + a.gko + c];
    const float z = __bfloat162float(a.z[(size_t)p * a.zs + c]);
    a.out[(size_t)p * a.C + c] = __float2bfloat16_rn(g * dsilu_f(z));
  }
}

// out[P][c] = mean of the 2x2 block of in (BF16), c < C
__global__ void k_avgpool2(const __nv_bfloat16* in, int is, __nv_bfloat16* out, int B, int H, int W, int C) {
  const long long n = (long long)B * (H / 2) * (W / 2) * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x = (int)(q % (W / 2));
    q /= (W / 2);
    const int y = (int)(q % (H / 2));
    const int b = (int)(q / (H / 2));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        s += __bfloat162float(in[(((size_t)b * H + 2 * y + dy) * W + 2 * x + dx) * is + c]);
    out[i] = __float2bfloat16_rn(0.25f * s);
  }
}

// out[b][y][x][oo + c] = in[b][y/2][x/2][c] (nearest doubling into a concatenation slot)
__global__ void k_up2(const __nv_bfloat16* in, int C, __nv_bfloat16* out, int os, int oo, int B, int H, int W) {
  const long long n = (long long)B * H * W * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const long long p = i / C;
    const int b = (int)(p / ((long long)H * W));
    const int r = (int)(p - (long long)b * H * W);
    const int y = r / W, x = r % W;
    out[(size_t)p * os + oo + c] = in[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
  }
}

// out[P][c] = sum over the 2x2 block of g[.][go + c] (FP32), coarse grid H/2 x W/2
__global__ void k_up2_backward(const float* g, int gsd, int go, float* out, int B, int H, int W, int C) {
  const long long n = (long long)B * (H / 2) * (W / 2) * C;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x = (int)(q % (W / 2));
    q /= (W / 2);
    const int y = (int)(q % (H / 2));
    const int b = (int)(q / (H / 2));
    float s = 0.f;
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) s += g[(((size_t)b * H + 2 * y + dy) * W + 2 * x + dx) * gsd + go + c];
    out[i] = s;
  }
}

// head: out[p][j] = b[j] + sum_c w[j][c] a[p][c], j < 2 (FP32 output)
__global__ void k_head(const __nv_bfloat16* act, int C, const float* w, float* out, long long npix) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix; p += (long long)gridDim.x * blockDim.x) {
    float s0 = w[2 * C], s1 = w[2 * C + 1];
    for (int c = 0; c < C; ++c) {
      const float v = __bfloat162float(act[(size_t)p * C + c]);
      s0 += w[c] * v;
      s1 += w[C + c] * v;
    }
    out[2 * p] = s0;
    out[2 * p + 1] = s1;
  }
}

// head backward: ga[p][c] = sum_j gout[p][j] w[j][c]; per-slice partial parameter gradients
__global__ void k_head_backward(const float* gout, const __nv_bfloat16* act, int C, const float* w, float* ga,
                                float* part, long long npix, int slices) {
  const int slice = blockIdx.x;
  const long long per = (npix + slices - 1) / slices;
  const long long pb = slice * per, pe = min(npix, pb + per);
  for (long long p = pb + threadIdx.x; p < pe; p += blockDim.x)
    for (int c = 0; c < C; ++c) ga[(size_t)p * C + c] = gout[2 * p] * w[c] + gout[2 * p + 1] * w[C + c];
  // partials in the packed parameter order: [w (2 x C)][b (2)]
  for (int o = threadIdx.x; o < 2 * (C + 1); o += blockDim.x) {
    const int j = o < 2 * C ? o / C : o - 2 * C;
    const int c = o < 2 * C ? o - j * C : C;
    float s = 0.f;
    for (long long p = pb; p < pe; ++p)
      s += gout[2 * p + j] * (c < C ? __bfloat162float(act[(size_t)p * C + c]) : 1.f);
    part[(size_t)slice * 2 * (C + 1) + o] = s;
  }
}

// ---------------------------------------------------------------- inputs, loss, output
// per sample: s = RMS(rc) over the m x m nodes (one CTA per sample, fixed-order tree)
template <typename C>
__global__ void k_rms(const C* rc, long long ldr, int nn, double* s) {
  __shared__ double red[256];
  const C* r = rc + (size_t)blockIdx.x * ldr;
  double acc = 0;
  for (int i = threadIdx.x; i < nn; i += 256) acc += (double)r[i].x * r[i].x + (double)r[i].y * r[i].y;
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double v = sqrt(red[0] / nn);
    s[blockIdx.x] = v > 0 ? v : 1.0;
  }
}

// x[b][y][x][0..7] = (Re r/s, Im r/s, eta, 0...) on the m x m nodes, 0 on the padding
template <typename C>
__global__ void k_make_input(const C* rc, long long ldr, const double* s, const float* eta, int m, int mp, int B,
                             __nv_bfloat16* x) {
  const long long n = (long long)B * mp * mp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / ((long long)mp * mp));
    const int r = (int)(i - (long long)b * mp * mp);
    const int y = r / mp, xx = r % mp;
    __align__(16) __nv_bfloat16 v[8];
    for (int c = 0; c < 8; ++c) v[c] = __float2bfloat16_rn(0.f);
    if (y < m && xx < m) {
      const C q = rc[(size_t)b * ldr + (size_t)y * m + xx];
      const double inv = 1.0 / s[b];
      v[0] = __float2bfloat16_rn((float)(q.x * inv));
      v[1] = __float2bfloat16_rn((float)(q.y * inv));
      v[2] = __float2bfloat16_rn(eta[(size_t)y * m + xx]);
    }
    *reinterpret_cast<uint4*>(x + (size_t)i * 8) = *reinterpret_cast<const uint4*>(v);
  }
}

// the same from an FP32 [B][mp][mp][3] array (test hook: the network alone)
__global__ void k_pack_input(const float* in, long long n, __nv_bfloat16* x) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    __align__(16) __nv_bfloat16 v[8];
    for (int c = 0; c < 8; ++c) v[c] = __float2bfloat16_rn(c < 3 ? in[3 * i + c] : 0.f);
    *reinterpret_cast<uint4*>(x + (size_t)i * 8) = *reinterpret_cast<const uint4*>(v);
  }
}

// per sample: num = ||out - t||^2, den = ||t||^2 over the m x m nodes, t = uc / s
__global__ void k_loss_sums(const float* out, const double2* uc, long long ldu, const double* s, int m, int mp,
                            double* num, double* den) {
  __shared__ double rn[256], rd[256];
  const int b = blockIdx.x;
  double an = 0, ad = 0;
  for (int i = threadIdx.x; i < m * m; i += 256) {
    const int y = i / m, x = i % m;
    const double2 u = uc[(size_t)b * ldu + i];
    const double tr = u.x / s[b], ti = u.y / s[b];
    const float* o = out + (((size_t)b * mp + y) * mp + x) * 2;
    const double dr = o[0] - tr, di = o[1] - ti;
    an += dr * dr + di * di;
    ad += tr * tr + ti * ti;
  }
  rn[threadIdx.x] = an;
  rd[threadIdx.x] = ad;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rn[threadIdx.x] += rn[threadIdx.x + w];
      rd[threadIdx.x] += rd[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    num[b] = rn[0];
    den[b] = rd[0] > 0 ? rd[0] : 1.0;
  }
}

// gout = 2 (out - t) / (den_b B) on the nodes, 0 on the padding
__global__ void k_loss_grad(const float* out, const double2* uc, long long ldu, const double* s, const double* den,
                            int m, int mp, int B, float* gout) {
  const long long n = (long long)B * mp * mp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / ((long long)mp * mp));
    const int r = (int)(i - (long long)b * mp * mp);
    const int y = r / mp, x = r % mp;
    float g0 = 0.f, g1 = 0.f;
    if (y < m && x < m) {
      const double2 u = uc[(size_t)b * ldu + (size_t)y * m + x];
      const double f = 2.0 / (den[b] * B);
      g0 = (float)((out[2 * i] - u.x / s[b]) * f);
      g1 = (float)((out[2 * i + 1] - u.y / s[b]) * f);
    }
    gout[2 * i] = g0;
    gout[2 * i + 1] = g1;
  }
}

// uc = s (out_re + i out_im) on the nodes
template <typename C>
__global__ void k_write_correction(const float* out, const double* s, int m, int mp, int B, C* uc, long long ldu) {
  const long long n = (long long)B * m * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / ((long long)m * m));
    const int r = (int)(i - (long long)b * m * m);
    const int y = r / m, x = r % m;
    const float* o = out + (((size_t)b * mp + y) * mp + x) * 2;
    C v;
    v.x = (decltype(v.x))(s[b] * o[0]);
    v.y = (decltype(v.y))(s[b] * o[1]);
    uc[(size_t)b * ldu + r] = v;
  }
}

// Adam on the FP32 master parameters (bias corrections from the host)
__global__ void k_adam(float* w, const float* g, float* m1, float* m2, long long n, float lr, float b1, float b2,
                       float c1, float c2, float eps) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = v;
    w[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
  }
}

inline unsigned blocks_for(long long n, int threads = 256) {
  long long b = (n + threads - 1) / threads;
  if (b > 8 * 152) b = 8 * 152;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

// ---------------------------------------------------------------- launchers
size_t conv_smem_bytes(int cout) {
  return (size_t)kStages * (128u * kUnits * 16u + (size_t)cout * kUnits * 16u) + (2 * kStages + 1) * sizeof(uint64_t);
}
int conv_chunks(int c8) { return (9 * c8 + kUnits - 1) / kUnits; }
size_t packed_weight_elems(int rows, int c8) { return (size_t)conv_chunks(c8) * rows * kUnits * 8; }

// One tcgen05 MMA has N <= 256: wider outputs (the input gradient of a decoder
// convolution, whose output channels are the concatenation's 3 C) run as
// launches over output-channel ranges of at most 256, each reading its rows of
// every packed weight chunk and writing its channel range.
cudaError_t launch_conv_umma(const ConvArgs& a, cudaStream_t s) {
  if (a.cout < 16 || (a.cout & 15) || a.cout > 1024) return cudaErrorInvalidValue;
  if ((a.xs & 7) || (a.xo & 7)) return cudaErrorInvalidValue;
  const long long npix = (long long)a.B * a.H * a.W;
  for (int c0 = 0; c0 < a.cout; c0 += 256) {
    ConvArgs b = a;
    b.cout = std::min(256, a.cout - c0);
    b.wrows = a.wrows ? a.wrows : a.cout;
    b.w = a.w + (size_t)c0 * kUnits * 16u;  // rows c0.. of each chunk (rows are 8-row groups, row-group major)
    if (a.bias) b.bias = a.bias + c0;
    b.zo = a.zo + c0;
    b.ao = a.ao + c0;
    b.yo = a.yo + c0;
    const size_t smem = conv_smem_bytes(b.cout);
    cudaError_t e = cudaFuncSetAttribute(k_conv_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_conv_umma<<<(unsigned)((npix + 127) / 128), kConvThreads, smem, s>>>(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_pack_weights(const float* w, __nv_bfloat16* out, int cout, int cin, int c8, int transpose,
                                cudaStream_t s) {
  // forward: rows = cout, K = 9 x (c8 = cin padded / 8); input gradient: rows = cin (padded), K = 9 x cout / 8
  const int rows = transpose ? c8 * 8 : cout;
  const int kc8 = transpose ? cout / 8 : c8;
  const int nchunk = conv_chunks(kc8);
  k_pack_weights<<<blocks_for((long long)nchunk * rows * kUnits * 8), 256, 0, s>>>(w, out, cout, cin, rows, kc8,
                                                                                  nchunk, transpose);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const WgradArgs& a, float* dw, float* db, const __nv_bfloat16* gz_for_bias, cudaStream_t s) {
  const int tiles = ((a.cout + 15) / 16) * ((a.cin + 15) / 16);
  k_wgrad<<<(unsigned)(tiles * a.slices), 256, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)a.cout * 9 * a.cin;
  k_sum_slices<<<blocks_for(n), 256, 0, s>>>(a.part, dw, n, a.slices);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const long long npix = (long long)a.B * a.H * a.W;
  k_bias_grad<<<(unsigned)a.slices, 128, 0, s>>>(gz_for_bias, a.gs, a.cout, npix, a.slices, a.part);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_sum_slices<<<blocks_for(a.cout), 256, 0, s>>>(a.part, db, a.cout, a.slices);
  return cudaGetLastError();
}

cudaError_t launch_grad_act(const GradActArgs& a, cudaStream_t s) {
  k_grad_act<<<blocks_for((long long)a.B * a.H * a.W * a.C), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_avgpool2(const __nv_bfloat16* in, int is, __nv_bfloat16* out, int B, int H, int W, int C,
                            cudaStream_t s) {
  k_avgpool2<<<blocks_for((long long)B * H * W * C / 4), 256, 0, s>>>(in, is, out, B, H, W, C);
  return cudaGetLastError();
}
cudaError_t launch_up2(const __nv_bfloat16* in, int C, __nv_bfloat16* out, int os, int oo, int B, int H, int W,
                       cudaStream_t s) {
  k_up2<<<blocks_for((long long)B * H * W * C), 256, 0, s>>>(in, C, out, os, oo, B, H, W);
  return cudaGetLastError();
}
cudaError_t launch_up2_backward(const float* g, int gsd, int go, float* out, int B, int H, int W, int C,
                                cudaStream_t s) {
  k_up2_backward<<<blocks_for((long long)B * H * W * C / 4), 256, 0, s>>>(g, gsd, go, out, B, H, W, C);
  return cudaGetLastError();
}
cudaError_t launch_head(const __nv_bfloat16* act, int C, const float* w, float* out, long long npix, cudaStream_t s) {
  k_head<<<blocks_for(npix), 256, 0, s>>>(act, C, w, out, npix);
  return cudaGetLastError();
}
cudaError_t launch_head_backward(const float* gout, const __nv_bfloat16* act, int C, const float* w, float* ga,
                                 float* part, float* dw, long long npix, int slices, cudaStream_t s) {
  k_head_backward<<<(unsigned)slices, 256, 0, s>>>(gout, act, C, w, ga, part, npix, slices);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_slices<<<1, 256, 0, s>>>(part, dw, 2 * (C + 1), slices);
  return cudaGetLastError();
}
template <typename C>
cudaError_t launch_make_input(const C* rc, long long ldr, int m, int mp, int B, const float* eta, double* s,
                              __nv_bfloat16* x, cudaStream_t st) {
  k_rms<C><<<(unsigned)B, 256, 0, st>>>(rc, ldr, m * m, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_make_input<C><<<blocks_for((long long)B * mp * mp), 256, 0, st>>>(rc, ldr, s, eta, m, mp, B, x);
  return cudaGetLastError();
}
template cudaError_t launch_make_input<double2>(const double2*, long long, int, int, int, const float*, double*,
                                                __nv_bfloat16*, cudaStream_t);
template cudaError_t launch_make_input<float2>(const float2*, long long, int, int, int, const float*, double*,
                                               __nv_bfloat16*, cudaStream_t);
cudaError_t launch_pack_input(const float* in, long long npix, __nv_bfloat16* x, cudaStream_t s) {
  k_pack_input<<<blocks_for(npix), 256, 0, s>>>(in, npix, x);
  return cudaGetLastError();
}
cudaError_t launch_loss(const float* out, const double2* uc, long long ldu, const double* s, int m, int mp, int B,
                        double* num, double* den, float* gout, cudaStream_t st) {
  k_loss_sums<<<(unsigned)B, 256, 0, st>>>(out, uc, ldu, s, m, mp, num, den);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_loss_grad<<<blocks_for((long long)B * mp * mp), 256, 0, st>>>(out, uc, ldu, s, den, m, mp, B, gout);
  return cudaGetLastError();
}
template <typename C>
cudaError_t launch_write_correction(const float* out, const double* s, int m, int mp, int B, C* uc, long long ldu,
                                    cudaStream_t st) {
  k_write_correction<C><<<blocks_for((long long)B * m * m), 256, 0, st>>>(out, s, m, mp, B, uc, ldu);
  return cudaGetLastError();
}
template cudaError_t launch_write_correction<double2>(const float*, const double*, int, int, int, double2*, long long,
                                                      cudaStream_t);
template cudaError_t launch_write_correction<float2>(const float*, const double*, int, int, int, float2*, long long,
                                                     cudaStream_t);
cudaError_t launch_adam(float* w, const float* g, float* m1, float* m2, long long n, float lr, float b1, float b2,
                        float c1, float c2, float eps, cudaStream_t s) {
  k_adam<<<blocks_for(n), 256, 0, s>>>(w, g, m1, m2, n, lr, b1, b2, c1, c2, eps);
  return cudaGetLastError();
}

}  // namespace th
