// Inline PTX building blocks of the tcgen05 / TMA kernels (sm_103a):
// mbarrier waits with a time bound, 2-D TMA tile loads, shared-memory matrix
// descriptors, the K = 16 BF16 MMAs of one 64-wide K block, and the FP64 ->
// BF16 hi/lo split of the split-precision products.
//
// Every translation unit that includes this header has its own copy of the
// wait bound `g_wait_ns` (a __device__ variable); tc_set_wait_ns() in that
// unit sets it.  A wait that runs past the bound sets the kernel's error flag
// and returns false; the kernels then stop, wait for their own copies and
// MMAs in flight (mbar_wait_drain, bounded by kDrainNs whatever g_wait_ns
// is), free their tensor memory and return, so the context stays usable.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tcptx {

constexpr uint64_t kDefaultWaitNs = 4000000000ull;  // 4 s
constexpr uint64_t kDrainNs = 1000000000ull;        // 1 s for in-flight work at exit

static __device__ uint64_t g_wait_ns = kDefaultWaitNs;
// Test of the error path: when set, each kernel's MMA issuer first waits on
// a barrier that nothing completes, so that wait runs out after g_wait_ns.
static __device__ int g_stall_test = 0;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity; false on timeout or when
// another role has already given up (error flag set).  The first try_wait is
// the fast path (no timer read); while waiting, the flag and the clock are
// checked every 32 tries only, so that a completed phase is seen within one
// try_wait, not after a global-memory round trip.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
  const uint32_t a = smem_u32(b);
  if (mbar_try(a, parity)) return true;
  const uint64_t t0 = gtime();
  const uint64_t limit = g_wait_ns;
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(a, parity)) return true;
    if ((i & 31) == 0) {
      if (*(volatile int*)err) return false;
      if (gtime() - t0 > limit) {
        atomicExch(err, 1);
        return false;
      }
    }
  }
}
// Wait at exit for work this CTA has already issued (TMA copies, MMAs): only
// the fixed kDrainNs bound ends it, not the error flag, so tensor memory and
// shared memory are released only after that work has landed.
__device__ __forceinline__ bool mbar_wait_drain(uint64_t* b, uint32_t parity, int* err) {
  const uint32_t a = smem_u32(b);
  const uint64_t t0 = gtime();
  for (uint32_t i = 0;; ++i) {
    if (mbar_try(a, parity)) return true;
    if ((i & 31) == 31 && gtime() - t0 > kDrainNs) {
      atomicExch(err, 1);
      return false;
    }
  }
}

// The stall of g_stall_test: a wait on `never` (initialised, never arrived
// on); false when it ran out (the error flag is then set).
__device__ __forceinline__ bool stall_test_wait(uint64_t* never, int* err) {
  if (!g_stall_test) return true;
  return mbar_wait(never, 0, err);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_load_2d_u(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row swizzle atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                  // descriptor version
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

// The four K = 16 MMAs of one product over a 64-wide K block.  ad / bd
// describe the stage's first 16 columns; the next ones start 32 bytes further,
// i.e. +2 in the descriptor's address field (addresses stay below 256 KB, so
// no carry).  The first MMA accumulates if `accum`, the other three always.
__device__ __forceinline__ void mma_ktile(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p, q;\n .reg .b64 a1, a2, a3, b1, b2, b3;\n"
      " setp.ne.b32 p, %4, 0;\n setp.eq.u32 q, %3, %3;\n"
      " add.s64 a1, %1, 2;\n add.s64 a2, %1, 4;\n add.s64 a3, %1, 6;\n"
      " add.s64 b1, %2, 2;\n add.s64 b2, %2, 4;\n add.s64 b3, %2, 6;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], a1, b1, %3, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], a2, b2, %3, q;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], a3, b3, %3, q;\n}\n" ::"r"(d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}

// Split two values into BF16 hi parts and BF16 lo parts (the rounding error of
// hi).  The operand is first rounded to FP32 (one conversion on the narrow FP64
// pipe); hi and lo then come from FP32 arithmetic, and hi + lo keeps about 16
// significant bits, well inside FP32's 24.
__device__ __forceinline__ void split_bf16(float x0, float x1, __nv_bfloat162* hi, __nv_bfloat162* lo) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
  const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
  const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
  *hi = __halves2bfloat162(h0, h1);
  *lo = __halves2bfloat162(l0, l1);
}

}  // namespace tcptx
