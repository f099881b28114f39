// Inline-PTX building blocks shared by the kernels that use mbarriers, bulk
// (TMA) copies and the fifth-generation tensor cores, and the one bounded-wait
// policy they all follow.
//
// Bounded waits.  Every wait on an mbarrier polls it at most `limit` times and
// then reports failure; the kernel records the failure in its status word
// (err[0]), waits (again bounded) for its own copies still in flight, releases
// any tensor memory it holds and returns.  The limit of a launch is read from
// the context's status words at kernel start:
//   err[kWaitLimitWord] == 0  -> the kernel's default limit (about a second),
//   err[kWaitLimitWord] >  0  -> that many polls,
//   err[kWaitLimitWord] <  0  -> no polls at all: the kernel records a timeout
//                               and returns before its first mbarrier, bulk
//                               copy, st.async or MMA (th_set_wait_limit, used
//                               to test the error path without a stuck GPU).
#pragma once

#include <cstdint>

namespace th {
namespace ptx {

constexpr int kWaitLimitWord = 63;  // index into the context's 64 device status words
// polls of the waits that drain a CTA's own copies and MMAs after a failure
// (whatever the launch's limit: nothing may still be in flight at exit)
constexpr int kDrainPolls = 1 << 20;

__device__ __forceinline__ int wait_limit(const int* err, int dflt) {
  if (!err) return dflt;
  const int v = *reinterpret_cast<const volatile int*>(err + kWaitLimitWord);
  return v == 0 ? dflt : (v > 0 ? v : 0);
}

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// ------------------------------------------------------------------ mbarriers
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(b)) : "memory");
}
// arrive and add `bytes` to the transaction count of the current phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}
// one poll of the phase with the given parity (returns after a short
// hardware-chosen time if the phase is not complete)
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(ok)
               : "r"(smem_addr(b)), "r"(parity)
               : "memory");
  return ok != 0;
}
// one poll during which the thread may be suspended for up to 10 us (it
// resumes as soon as the phase completes), so waiting warps leave the issue
// slots to the others
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 10000;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// one poll with acquire semantics at cluster scope (the transactions that
// complete the phase are st.async stores of other CTAs of the cluster)
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait with the suspending poll: false after `limit` polls
__device__ __forceinline__ bool mbar_wait_suspend(uint64_t* b, unsigned parity, int limit) {
  for (int it = 0; it < limit; ++it)
    if (mbar_try_wait_suspend(b, parity)) return true;
  return false;
}
// bounded wait shared by the threads of a CTA: false after `limit` polls, or
// early once another thread of the CTA has set *failed (checked every 256
// polls); a wait that gives up sets *failed
__device__ __forceinline__ bool mbar_wait_shared_flag(uint64_t* b, unsigned parity, volatile int* failed, int limit) {
  for (int it = 0; it < limit; ++it) {
    if (mbar_try_wait(b, parity)) return true;
    if ((it & 255) == 255 && *failed) return false;
  }
  *failed = 1;
  return false;
}

// ------------------------------------------------- programmatic dependent launch
// Wait until every grid this one depends on programmatically has completed and
// its memory operations are visible; a no-op in a launch without such a
// dependency.  A kernel launched with one must pass here before it touches
// anything an earlier kernel of the stream writes or reads.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// Let the next grid of the stream, if launched with a programmatic dependency,
// be scheduled (it still waits in grid_dep_wait for this grid to complete).
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ------------------------------------------------------------ bulk copies
// one-dimensional bulk copy global -> shared (16-byte aligned addresses, size
// a multiple of 16), completing `bytes` transactions on bar
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// ------------------------------------------------------------ tcgen05
// shared-memory matrix descriptor, no swizzle: start address, leading and
// stride byte offsets (each >> 4, 14 bits), descriptor version 1 (bit 46)
__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// D[tmem] (+)= A[smem] B[smem], kind::f16 (both operands BF16 here), one CTA
__device__ __forceinline__ void umma_bf16(unsigned d_tmem, uint64_t a, uint64_t b, unsigned idesc, unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on bar once every MMA issued so far by this thread has completed
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_addr(bar))
               : "memory");
}
// 16 consecutive 32-bit columns of tensor memory, lane = thread, then wait
__device__ __forceinline__ void tmem_ld16(unsigned addr, unsigned* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

}  // namespace ptx
}  // namespace th
