// K8c: the separator product and the spike correction of the partitioned
// coarse solve (Algorithm 1, "solve A_c u_c = r_c"; the three stages are
// described in coarse_part.cu) for groups of up to 64 right-hand sides on the
// fifth-generation tensor cores.  Every operand is held as a pair of BF16
// numbers, v = hi + lo with hi = bf16(v) and lo = bf16(v - hi) (16 significant
// bits), and a product is the sum of the three MMAs hi*hi + hi*lo + lo*hi
// (the lo*lo term is below 2^-16 relative): the rounding of one BF16 number
// (2^-9) alone makes the solve on large coarse grids, whose chunk systems
// amplify these products' errors, too inexact for the outer iteration.  The
// FP64 set-up and the FP32 chunk sweep are those of the other forms.
//
//   MODE 0: xhat = Sinv rhat.  A = Sinv (nred x nred), B = rhat (nred values
//           per right-hand side, written as split BF16 by k_reduced_rhs).  The
//           epilogue stores xhat into the separator rows of x (FP32) and a
//           split-BF16 copy of every separator's values for MODE 1; with the
//           K range split over CTAs (nsplit > 1, to fill the SMs) it stores
//           partial products instead, which k_sep_split_sum adds in split order.
//   MODE 1: x_c -= [L | R]_c [x_left; x_right] on every chunk c.  A = the
//           chunk's spikes (L_c mc rows; one column block per adjacent
//           separator), B = the split-BF16 copies of those separators' values.
//
// Both operands lie in global memory already in the tensor cores' K-major
// layout without swizzle, cut into chunks of 32 columns: an A chunk is 128
// rows (32 KB), a B chunk 64 right-hand sides (16 KB), each made of four parts
// (re hi, im hi, re lo, im lo) of core matrices of 8 rows x 16 bytes arranged
// [row/8][k/8] (umma_off32 in kernels.h).  One bulk copy per operand brings a
// chunk into a ring of four shared-memory stages; per K step of 16 and per
// (hi, lo) pairing four MMAs (M = 128, N = 64, BF16 operands, FP32
// accumulators in tensor memory) form
//   D_re += A_re B_re - A_im B_im,   D_im += A_re B_im + A_im B_re
// (the minus sign through the A-negate bit of the instruction descriptor).
// Tiles of 128 rows are dealt round-robin to persistent CTAs (one per SM);
// the accumulators are double-buffered so that the epilogue of one tile
// overlaps the MMAs of the next.  Roles: warp 0 lane 0 issues the copies and
// the MMAs, warps 4-7 move the accumulators out (warp 4 + q reads tensor
// memory lanes 32q .. 32q + 31).  Every wait is bounded (ptx.cuh); a CTA whose
// wait gives up stops issuing, drains its own copies and MMAs, frees its
// tensor memory and sets err[0].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "launch.cuh"
#include "ptx.cuh"

namespace th {
namespace {

constexpr int kStages = 4;
constexpr int kAPart = 128 * 32 * 2;            // one part of an A chunk (bytes)
constexpr int kBPart = 64 * 32 * 2;             // one part of a B chunk
constexpr int kAChunk = 4 * kAPart;             // 32 KB: re hi, im hi, re lo, im lo
constexpr int kBChunk = 4 * kBPart;             // 16 KB
constexpr int kStageBytes = kAChunk + kBChunk;  // 48 KB
constexpr int kThreads = 256;
constexpr int kTmemCols = 256;                  // two accumulators of 64 + 64 columns

// v = hi + lo in BF16 (hi = bf16(v), lo = bf16(v - hi)) for the real and the
// imaginary part: parts re hi, im hi, re lo, im lo, `part` elements apart
__device__ __forceinline__ void store_split(__nv_bfloat16* st, int part, int off, float vr, float vi) {
  const __nv_bfloat16 hr = __float2bfloat16_rn(vr), hi = __float2bfloat16_rn(vi);
  st[off] = hr;
  st[part + off] = hi;
  st[2 * part + off] = __float2bfloat16_rn(vr - __bfloat162float(hr));
  st[3 * part + off] = __float2bfloat16_rn(vi - __bfloat162float(hi));
}

constexpr size_t coarse_umma_smem() { return (size_t)kStages * kStageBytes + (2 * kStages + 5) * sizeof(uint64_t); }

}  // namespace

template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_coarse_umma(const CoarseUmmaArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* stage = smraw;  // [kStages][A chunk | B chunk]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + (size_t)kStages * kStageBytes);
  uint64_t* full = bars;                 // [kStages] copies landed
  uint64_t* empty = bars + kStages;      // [kStages] MMAs reading the stage completed
  uint64_t* afull = bars + 2 * kStages;  // [2] accumulator complete
  uint64_t* aempty = afull + 2;          // [2] accumulator read out
  uint64_t* done = aempty + 2;           // every MMA of this CTA completed
  __shared__ unsigned tmem_base;
  __shared__ volatile int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grp = blockIdx.y;  // group of 64 right-hand sides
  const int ntiles = MODE == 0 ? a.ntiles_s : a.ntiles_l;
  const CoarseTile* tiles = MODE == 0 ? a.tiles_s : a.tiles_l;
  const int nmine = (ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  ptx::grid_dep_wait();  // launched with a programmatic dependency inside the cycle
  ptx::grid_dep_launch();
  const int lim = ptx::wait_limit(a.err, 1 << 20);
  if (lim == 0) {  // waits disabled: record a timeout before any barrier, copy or MMA
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }
  if (nmine <= 0) return;  // uniform over the CTA

  if (tid == 0) {
    failed = 0;
    for (int i = 0; i < kStages; ++i) {
      ptx::mbar_init(full + i, 1);
      ptx::mbar_init(empty + i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(afull + i, 1);
      ptx::mbar_init(aempty + i, 128);
    }
    ptx::mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     ptx::smem_addr(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_base;
  const unsigned char* Ag = MODE == 0 ? a.As : a.Al;
  const unsigned char* Bg = MODE == 0 ? a.rst + (size_t)grp * a.nkc_s * kBChunk
                                      : a.xst + (size_t)grp * a.nsep * a.nkc_m * kBChunk;

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------ bulk copies + MMAs
      int pi = 0, pkc = 0;  // copy cursor: tile ordinal of this CTA, chunk within it
      int issued = 0;       // chunks handed to the copy engine
      auto issue = [&]() {  // the next chunk in order, into the stage it frees
        if (pi >= nmine || failed) return;
        const CoarseTile& tl = tiles[blockIdx.x + pi * gridDim.x];
        const int t = issued, slot = t % kStages, use = t / kStages;
        if (!ptx::mbar_wait_shared_flag(empty + slot, (unsigned)((use & 1) ^ 1), &failed, lim)) return;
        const unsigned char* asrc = Ag + tl.a_off + (size_t)pkc * kAChunk;
        const unsigned char* bsrc;
        if (MODE == 0) {
          bsrc = Bg + (size_t)(tl.b0 + pkc) * kBChunk;
        } else {
          const int side = pkc < a.nkc_m ? 0 : 1;
          const int sp = side ? tl.b1 : tl.b0;
          bsrc = Bg + ((size_t)sp * a.nkc_m + (pkc - side * a.nkc_m)) * kBChunk;
        }
        unsigned char* dst = stage + (size_t)slot * kStageBytes;
        ptx::mbar_arrive_expect_tx(full + slot, (unsigned)kStageBytes);
        ptx::bulk_g2s(dst, asrc, (unsigned)kAChunk, full + slot);
        ptx::bulk_g2s(dst + kAChunk, bsrc, (unsigned)kBChunk, full + slot);
        issued = t + 1;
        if (++pkc == tl.nkc) {
          pkc = 0;
          ++pi;
        }
      };
      // instruction descriptor: D f32, A/B bf16, both K-major, N = 64, M = 128
      const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(64 >> 3) << 17) | (8u << 24);
      const unsigned idesc_neg = idesc | (1u << 13);
      for (int q = 0; q < kStages - 1; ++q) issue();
      int t = 0;
      for (int i = 0; i < nmine && !failed; ++i) {
        const int nkc = tiles[blockIdx.x + i * gridDim.x].nkc;
        const int ab = i & 1, ua = i >> 1;
        if (!ptx::mbar_wait_shared_flag(aempty + ab, (unsigned)((ua & 1) ^ 1), &failed, lim)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const unsigned d_re = tmem + (unsigned)(ab * 128), d_im = d_re + 64;
        for (int kc = 0; kc < nkc; ++kc, ++t) {
          const int slot = t % kStages, use = t / kStages;
          if (!ptx::mbar_wait_shared_flag(full + slot, (unsigned)(use & 1), &failed, lim)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const unsigned sa = ptx::smem_addr(stage + (size_t)slot * kStageBytes), sb = sa + kAChunk;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const unsigned ko = (unsigned)j * 256;  // two core matrices along K
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {  // (hi, hi), (hi, lo), (lo, hi)
              const unsigned pa = pr == 2 ? 2u : 0u, pb = pr == 1 ? 2u : 0u;
              const uint64_t Are = ptx::umma_desc(sa + pa * kAPart + ko, 128, 512);
              const uint64_t Aim = ptx::umma_desc(sa + (pa + 1) * kAPart + ko, 128, 512);
              const uint64_t Bre = ptx::umma_desc(sb + pb * kBPart + ko, 128, 512);
              const uint64_t Bim = ptx::umma_desc(sb + (pb + 1) * kBPart + ko, 128, 512);
              const unsigned acc = (kc > 0 || j > 0 || pr > 0) ? 1u : 0u;
              ptx::umma_bf16(d_re, Are, Bre, idesc, acc);
              ptx::umma_bf16(d_re, Aim, Bim, idesc_neg, 1u);
              ptx::umma_bf16(d_im, Are, Bim, idesc, acc);
              ptx::umma_bf16(d_im, Aim, Bre, idesc, 1u);
            }
          }
          ptx::umma_commit(empty + slot);
          issue();
        }
        if (failed) break;
        ptx::umma_commit(afull + ab);
      }
      // every MMA issued above completes before tensor memory is released
      ptx::umma_commit(done);
      volatile int ignore = 0;
      ptx::mbar_wait_shared_flag(done, 0u, &ignore, ptx::kDrainPolls);
      // copies issued but not consumed (only after a failure)
      for (int u = t; u < issued; ++u)
        ptx::mbar_wait_shared_flag(full + (u % kStages), (unsigned)((u / kStages) & 1), &ignore, ptx::kDrainPolls);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------ epilogue: tensor memory -> x
    const int q = warp - 4, row = q * 32 + lane;
    for (int i = 0; i < nmine; ++i) {
      const CoarseTile tl = tiles[blockIdx.x + i * gridDim.x];
      const int ab = i & 1, ua = i >> 1;
      if (!failed) ptx::mbar_wait_shared_flag(afull + ab, (unsigned)(ua & 1), &failed, lim);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned base = tmem + ((unsigned)(q * 32) << 16) + (unsigned)(ab * 128);
      const bool live = row < tl.rows && !failed;
      int k = 0, e = 0;
      if (MODE == 0) {
        const int idx = tl.row0 + row;  // reduced index
        k = idx / a.mc;
        e = idx - k * a.mc;
      }
#pragma unroll 1
      for (int c0 = 0; c0 < 64; c0 += 16) {
        unsigned re[16], im[16];
        ptx::tmem_ld16(base + (unsigned)c0, re);
        ptx::tmem_ld16(base + (unsigned)(64 + c0), im);
        if (!live) continue;
        const int nb = min(16, a.nrhs - (grp * 64 + c0));  // right-hand sides of this slice
        if (MODE == 0 && a.nsplit > 1) {  // a partial product of one K split
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (j >= nb) break;
            const int rhs = grp * 64 + c0 + j;
            a.spart[((size_t)tl.b1 * a.nrhs_cap + rhs) * a.nred + tl.row0 + row] =
                make_float2(__uint_as_float(re[j]), __uint_as_float(im[j]));
          }
        } else if (MODE == 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (j >= nb) break;
            const int n = c0 + j, rhs = grp * 64 + n;
            const float vr = __uint_as_float(re[j]), vi = __uint_as_float(im[j]);
            a.x[(size_t)rhs * a.Nc + (size_t)a.sep[k] * a.mc + e] = make_float2(vr, vi);
            __nv_bfloat16* st = reinterpret_cast<__nv_bfloat16*>(
                a.xst + (((size_t)grp * a.nsep + k) * a.nkc_m + (e >> 5)) * kBChunk);
            store_split(st, kBPart / 2, umma_off32(n, e & 31), vr, vi);
          }
        } else {
          // every load of the slice before the first store (they are independent)
          float2* p0 = a.x + (size_t)(grp * 64 + c0) * a.Nc + tl.row0 + row;
          float2 v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j < nb) v[j] = p0[(size_t)j * a.Nc];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (j < nb) {
              v[j].x -= __uint_as_float(re[j]);
              v[j].y -= __uint_as_float(im[j]);
              p0[(size_t)j * a.Nc] = v[j];
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      ptx::mbar_arrive(aempty + ab);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && failed) atomicExch(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// The separator values from the K splits' partial products, added in split
// order: into the separator rows of x and the split-BF16 copy for MODE 1.
__global__ void __launch_bounds__(256) k_sep_split_sum(const CoarseUmmaArgs a) {
  ptx::grid_dep_wait();
  ptx::grid_dep_launch();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x, rhs = blockIdx.y;
  if (idx >= a.nred || rhs >= a.nrhs) return;
  float vr = 0.f, vi = 0.f;
  for (int sp = 0; sp < a.nsplit; ++sp) {
    const float2 v = a.spart[((size_t)sp * a.nrhs_cap + rhs) * a.nred + idx];
    vr += v.x;
    vi += v.y;
  }
  const int k = idx / a.mc, e = idx - k * a.mc, grp = rhs >> 6, n = rhs & 63;
  a.x[(size_t)rhs * a.Nc + (size_t)a.sep[k] * a.mc + e] = make_float2(vr, vi);
  __nv_bfloat16* st =
      reinterpret_cast<__nv_bfloat16*>(a.xst + (((size_t)grp * a.nsep + k) * a.nkc_m + (e >> 5)) * kBChunk);
  store_split(st, kBPart / 2, umma_off32(n, e & 31), vr, vi);
}

cudaError_t launch_coarse_umma(const CoarseUmmaArgs& a, int mode, int sms, cudaStream_t s) {
  if (a.nrhs < 1 || a.mc < 1 || (mode != 0 && mode != 1)) return cudaErrorInvalidValue;
  const int ntiles = mode == 0 ? a.ntiles_s : a.ntiles_l;
  if (ntiles < 1) return cudaSuccess;
  const size_t smem = coarse_umma_smem();
  const int groups = (a.nrhs + 63) / 64;
  const dim3 grid((unsigned)(ntiles < sms ? ntiles : sms), (unsigned)groups);
  cudaError_t e;
  if (mode == 0) {
    e = cudaFuncSetAttribute(k_coarse_umma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = launch_pdl(k_coarse_umma<0>, grid, dim3(kThreads), smem, s, 0, a);
    if (e != cudaSuccess || a.nsplit <= 1) return e;
    return launch_pdl(k_sep_split_sum, dim3((unsigned)((a.nred + 255) / 256), (unsigned)a.nrhs), dim3(256), 0, s, 0,
                      a);
  }
  e = cudaFuncSetAttribute(k_coarse_umma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_coarse_umma<1>, grid, dim3(kThreads), smem, s, 0, a);
}

}  // namespace th
