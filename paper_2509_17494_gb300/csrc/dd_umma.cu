// K3b: the subdomain inverse-row products for a batch of right-hand sides on
// the fifth-generation tensor cores (tcgen05.mma, Section 4.1 / Algorithm 2:
// V_i = W_i R_i r for every right-hand side at once).
//
// Per subdomain the product is a complex GEMM V = W X^T, W: NR x NC rows
// (NR <= 128), X: NB x NC gathered residuals (NB = 64, 32 or 16 right-hand sides
// per tile, the widest whose doubled X buffer fits shared memory: 64 for the
// 289-column rows of the 2-D Q4 subdomains, so that every row crosses HBM once
// for 64 sources; 16 for the 729-column rows of the 3-D Q2 subdomains).  In real
// arithmetic, with A = W (M = 128 rows, K-major) and B = X (N = NB, K-major):
//   D_re = W_re X_re^T - W_im X_im^T,   D_im = W_re X_im^T + W_im X_re^T,
// four MMAs per K-step of 16 (the minus sign through the A-negate bit), with
// BF16 operands and FP32 accumulators in tensor memory.
//
// Operand layout in shared memory: "core matrices" of 8 rows x 16 bytes,
// arranged [row/8][k/8] with k/8 fastest, no swizzle; the descriptors carry
// the K step (128 bytes) and the row step (the number of k/8 blocks times 128
// bytes).  W is stored in global memory already in this layout, split into
// K-chunks of 64 so each chunk is one contiguous bulk copy (TMA engine) per
// real/imaginary part; rows 88..127 of the A tile are never loaded (their
// results are discarded).  X is gathered from the FP32 residual, rounded to
// BF16 and written in the same layout by producer warps.
//
// Roles in a persistent CTA (one per SM): warp 0 lane 0 issues the bulk copies
// and the MMAs; warps 4-7 move the accumulators from tensor memory to global
// memory; all other warps gather X.  W chunks go through a ring of 3 (NB = 64)
// or 4 slots,
// X and the accumulators are double-buffered; everything is ordered by
// mbarriers.  Every wait has an iteration limit; when one gives up the CTA
// raises `failed`, stops issuing work, drains what it issued (bounded) and
// frees its tensor memory before returning.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace th {
namespace {

constexpr int kKC = 8;       // k/8 blocks per W chunk (64 columns)
constexpr int kMaxDepth = 4;  // W chunk slots at most (barrier arrays)
// one W chunk slot: re + im parts of M8 row groups x 64 columns
__host__ __device__ inline size_t w_slot_bytes(int M8) { return (size_t)2 * M8 * kKC * 128; }
constexpr int kThreads = 512;

__device__ __forceinline__ unsigned su32(const void* p) { return ptx::smem_addr(p); }
using ptx::mbar_arrive;
using ptx::mbar_init;
using ptx::tmem_ld16;
using ptx::umma_bf16;
using ptx::umma_commit;
using ptx::umma_desc;

}  // namespace

size_t dd_umma_bytes_per_sub(int NR, int NC) {
  const int M8 = (NR + 7) / 8;
  const int K8 = 2 * ((NC + 15) / 16);
  return (size_t)K8 * 2 * M8 * 128;
}

template <int kNB, int kDepth, bool D3>
__global__ void __launch_bounds__(kThreads, 1) k_dd_umma(const DDUmmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int M8 = a.M8, K8 = a.K8;
  const int NKC = (K8 + kKC - 1) / kKC;
  const size_t xbuf_bytes = (size_t)2 * (kNB / 8) * K8 * 128;  // re + im
  const size_t kSlotBytes = w_slot_bytes(M8);                  // a multiple of 1024 bytes
  unsigned char* wslot = smraw;                                 // [kDepth][kSlotBytes]
  unsigned char* xbuf = smraw + (size_t)kDepth * kSlotBytes;    // [2][xbuf_bytes]
  uint64_t* bars = reinterpret_cast<uint64_t*>(xbuf + 2 * xbuf_bytes);
  uint64_t* wfull = bars;           // [kDepth]
  uint64_t* wempty = bars + 4;      // [kDepth]
  uint64_t* xfull = bars + 8;       // [2]
  uint64_t* xempty = bars + 10;     // [2]
  uint64_t* afull = bars + 12;      // [2]
  uint64_t* aempty = bars + 14;     // [2]
  uint64_t* done = bars + 16;       // every MMA of this CTA has completed
  __shared__ unsigned tmem_base;
  __shared__ volatile int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = blockIdx.y * kNB;
  const int nmine = (a.nsub - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const bool producer = (warp >= 1 && warp <= 3) || warp >= 8;
  const int nprod = 11 * 32;
  const int pidx = (warp <= 3) ? tid - 32 : tid - 32 - 128;  // 0..351 among producers
  const int lim = ptx::wait_limit(a.err, 1 << 20);
  if (lim == 0) {  // waits disabled: record a timeout before any barrier, copy or MMA
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }

  if (tid == 0) {
    failed = 0;
    for (int i = 0; i < kDepth; ++i) { mbar_init(wfull + i, 1); mbar_init(wempty + i, 1); }
    for (int i = 0; i < 2; ++i) {
      mbar_init(xfull + i, nprod);
      mbar_init(xempty + i, 1);
      mbar_init(afull + i, 1);
      mbar_init(aempty + i, 128);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(4 * kNB)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ TMA + MMA issuer
      const int total = nmine * NKC;
      const size_t sub_bytes = (size_t)K8 * 2 * M8 * 128;
      int issued = 0;  // W chunks handed to the bulk-copy engine
      auto issue = [&](int t) {
        if (t >= total || failed) return;
        const int i = t / NKC, kc = t - i * NKC;
        const int sub = blockIdx.x + i * gridDim.x;
        const int kcs = min(kKC, K8 - kc * kKC);
        const unsigned part = (unsigned)(M8 * kcs * 128);
        const int slot = t % kDepth, use = t / kDepth;
        if (!ptx::mbar_wait_shared_flag(wempty + slot, (unsigned)((use & 1) ^ 1), &failed, lim)) return;
        ptx::mbar_arrive_expect_tx(wfull + slot, 2 * part);
        const unsigned char* src = a.W + (size_t)sub * sub_bytes + (size_t)kc * kKC * 2 * M8 * 128;
        unsigned char* dst = wslot + (size_t)slot * kSlotBytes;
        ptx::bulk_g2s(dst, src, part, wfull + slot);                          // real part
        ptx::bulk_g2s(dst + kSlotBytes / 2, src + part, part, wfull + slot);  // imaginary part
        issued = t + 1;
      };
      // instruction descriptors: D f32, A/B bf16, K-major, N = kNB, M = 128
      const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kNB >> 3) << 17) | (8u << 24);
      const unsigned idesc_neg = idesc | (1u << 13);
      for (int t = 0; t < kDepth - 1; ++t) issue(t);
      int t = 0;
      for (int i = 0; i < nmine && !failed; ++i) {
        const int xb = i & 1, ux = i >> 1, ab = i & 1;
        if (!ptx::mbar_wait_shared_flag(xfull + xb, (unsigned)(ux & 1), &failed, lim)) break;
        if (!ptx::mbar_wait_shared_flag(aempty + ab, (unsigned)((ux & 1) ^ 1), &failed, lim)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned d_re = tmem + (unsigned)(ab * 2 * kNB), d_im = d_re + kNB;
        const unsigned xre = su32(xbuf + (size_t)xb * xbuf_bytes), xim = xre + (unsigned)(xbuf_bytes / 2);
        for (int kc = 0; kc < NKC; ++kc, ++t) {
          const int slot = t % kDepth, use = t / kDepth;
          if (!ptx::mbar_wait_shared_flag(wfull + slot, (unsigned)(use & 1), &failed, lim)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int kcs = min(kKC, K8 - kc * kKC);
          const unsigned wre = su32(wslot + (size_t)slot * kSlotBytes), wim = wre + kSlotBytes / 2;
          const unsigned a_sbo = (unsigned)kcs * 128, b_sbo = (unsigned)K8 * 128;
          for (int j = 0; j < kcs / 2; ++j) {
            const unsigned ka = (unsigned)j * 256;                    // within the chunk
            const unsigned kb = (unsigned)(kc * kKC + 2 * j) * 128;   // within X
            const uint64_t Are = umma_desc(wre + ka, 128, a_sbo), Aim = umma_desc(wim + ka, 128, a_sbo);
            const uint64_t Bre = umma_desc(xre + kb, 128, b_sbo), Bim = umma_desc(xim + kb, 128, b_sbo);
            const unsigned acc = (kc > 0 || j > 0) ? 1u : 0u;
            umma_bf16(d_re, Are, Bre, idesc, acc);
            umma_bf16(d_re, Aim, Bim, idesc_neg, 1u);
            umma_bf16(d_im, Are, Bim, idesc, acc);
            umma_bf16(d_im, Aim, Bre, idesc, 1u);
          }
          umma_commit(wempty + slot);
          issue(t + kDepth - 1);  // refill the slot freed by the previous chunk's MMAs
        }
        if (failed) break;
        umma_commit(afull + ab);
        umma_commit(xempty + xb);
      }
      // every MMA issued above completes before tensor memory is released
      umma_commit(done);
      volatile int ignore = 0;
      ptx::mbar_wait_shared_flag(done, 0u, &ignore, ptx::kDrainPolls);
      // bulk copies issued but not consumed (only after a failure)
      for (int u = t; u < issued; ++u) ptx::mbar_wait_shared_flag(wfull + (u % kDepth), (unsigned)((u / kDepth) & 1), &ignore, ptx::kDrainPolls);
    }
  } else if (warp >= 4 && warp <= 7) {
    // ------------------------------------------------ epilogue: TMEM -> V
    const int q = warp - 4;  // lanes 32q .. 32q + 31 of tensor memory
    const int row = q * 32 + lane;
    for (int i = 0; i < nmine; ++i) {
      const int ab = i & 1, ua = i >> 1;
      const int sub = blockIdx.x + i * gridDim.x;
      if (!failed) ptx::mbar_wait_shared_flag(afull + ab, (unsigned)(ua & 1), &failed, lim);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned base = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(ab * 2 * kNB);
      for (int c0 = 0; c0 < kNB; c0 += 16) {
        unsigned re[16], im[16];
        tmem_ld16(base + (unsigned)c0, re);
        tmem_ld16(base + (unsigned)(kNB + c0), im);
        if (row < a.NR && !failed) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int rhs = r0 + c0 + j;
            if (rhs < a.nrhs)
              a.V[((size_t)rhs * a.nsub + sub) * a.NR + row] = make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(aempty + ab);
    }
  } else if (producer) {
    // ------------------------------------------------ X producers: gather, round to BF16
    const int KP = K8 * 8;
    for (int i = 0; i < nmine; ++i) {
      const int xb = i & 1, ux = i >> 1;
      const int sub = blockIdx.x + i * gridDim.x;
      if (!failed) ptx::mbar_wait_shared_flag(xempty + xb, (unsigned)((ux & 1) ^ 1), &failed, lim);
      const int* bb = a.box + (size_t)sub * 12;
      const int ox = bb[0], oy = bb[1], wx = bb[2], wy = bb[3], oz = D3 ? bb[8] : 0, wz = D3 ? bb[9] : 1;
      const int L2 = a.Lw * a.Lw;
      __nv_bfloat16* xr = reinterpret_cast<__nv_bfloat16*>(xbuf + (size_t)xb * xbuf_bytes);
      __nv_bfloat16* xi = xr + xbuf_bytes / 4;
      // one column c per producer thread at a time: its box coordinates once,
      // then the kNB right-hand sides as independent loads
      for (int c = pidx; c < KP; c += nprod) {
        const int cz = D3 ? c / L2 : 0, cr = D3 ? c - cz * L2 : c;
        const int cy = cr / a.Lw, cx = cr - cy * a.Lw;
        const bool in = c < a.NC && cx < wx && cy < wy && cz < wz;
        const size_t gidx = in ? ((size_t)(oz + cz) * a.m + (oy + cy)) * a.m + (ox + cx) : 0;
        const size_t cbase = (size_t)(c >> 3) * 64 + (c & 7);
#pragma unroll 8
        for (int n = 0; n < kNB; ++n) {
          const int rhs = r0 + n;
          float2 v = make_float2(0.f, 0.f);
          if (in && rhs < a.nrhs) v = a.r[(size_t)rhs * a.N + gidx];
          const size_t off = (size_t)(n >> 3) * K8 * 64 + cbase + (n & 7) * 8;
          xr[off] = __float2bfloat16_rn(v.x);
          xi[off] = __float2bfloat16_rn(v.y);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(xfull + xb);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && failed) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * kNB) : "memory");
  }
}

template <int kNB, int kDepth>
static size_t dd_umma_smem(const DDUmmaArgs& a) {
  const size_t xbuf_bytes = (size_t)2 * (kNB / 8) * a.K8 * 128;
  return (size_t)kDepth * w_slot_bytes(a.M8) + 2 * xbuf_bytes + 17 * sizeof(uint64_t);
}

template <int kNB, int kDepth, bool D3>
static cudaError_t launch_dd_umma_k(const DDUmmaArgs& a, int sms, cudaStream_t s) {
  const size_t smem = dd_umma_smem<kNB, kDepth>(a);
  cudaError_t e =
      cudaFuncSetAttribute(k_dd_umma<kNB, kDepth, D3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(a.nsub < sms ? a.nsub : sms), (unsigned)((a.nrhs + kNB - 1) / kNB));
  k_dd_umma<kNB, kDepth, D3><<<grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}
template <int kNB, int kDepth>
static cudaError_t launch_dd_umma_nb(const DDUmmaArgs& a, int sms, cudaStream_t s) {
  return a.dim3 ? launch_dd_umma_k<kNB, kDepth, true>(a, sms, s) : launch_dd_umma_k<kNB, kDepth, false>(a, sms, s);
}

cudaError_t launch_dd_umma(const DDUmmaArgs& a, int sms, cudaStream_t s) {
  if (a.NR > 128 || (a.K8 & 1) || a.M8 * 8 > 128) return cudaErrorInvalidValue;
  // 64 right-hand sides per tile when they fit (the rows then cross HBM once for
  // all 64; a ring of three W slots), else 32 or 16 (MMA N >= 16 with M = 128)
  if (a.nrhs > 32 && dd_umma_smem<64, 3>(a) <= 225 * 1024) return launch_dd_umma_nb<64, 3>(a, sms, s);
  if (a.nrhs > 16 && dd_umma_smem<32, 4>(a) <= 225 * 1024) return launch_dd_umma_nb<32, 4>(a, sms, s);
  if (dd_umma_smem<16, 4>(a) <= 225 * 1024) return launch_dd_umma_nb<16, 4>(a, sms, s);
  return cudaErrorInvalidValue;
}

}  // namespace th
