// tcgen05 / TMEM / mbarrier helpers shared by the tensor-core kernels.
//
// The contractions run as bf16 x bf16 -> f32 MMAs (tcgen05.mma, kind::f16) on
// three-piece bf16 splits of both operands (x = x0 + x1 + x2, each piece the
// bf16 rounding of what the previous ones leave), keeping the six products of
// total order <= 2: every product of two pieces is exact in FP32, the dropped
// ones are below 2^-24 of the result.  Operand tiles are K-major with the
// 128-byte swizzle: row r of a 64-wide bf16 tile is 128 bytes, its 16-byte
// chunk c stored at chunk c ^ (r mod 8), rows in 8-row atoms of 1 KB.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>

namespace fep3m {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__host__ __device__ __forceinline__ uint32_t sw128_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 1 KB between 8-row atoms
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor: bf16 A and B (K-major), f32 accumulator, M = m (128, or 64), N = n (a
// multiple of 16 for M = 128, of 8 for M = 64; <= 256).  Accumulator layout in TMEM: M = 128, row r
// in lane r; M = 64 (cta_group::1), row r in lane 32 (r / 16) + r mod 16 (the first 16 lanes of each
// warp's lane quarter).
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t n, uint32_t m = 128) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                   tmem_d),
               "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {   // one full warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t tmem, uint32_t ncols) {   // the allocating warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// bounded wait for the phase with the given parity; false if it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity)
                 : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void sts128(uint32_t addr, const uint32_t v[4]) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t v[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
// 16 lanes x 32 columns (16 x 64-bit, 16 repetitions): thread t of the warp receives, in register j,
// lane (t / 4) + 8 (t mod 2) of the 16 and column 2 j + (t / 2) mod 2
__device__ __forceinline__ void tmem_ld16x64b(uint32_t taddr, uint32_t v[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x64b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// three-piece bf16 split of two consecutive values, packed in pairs (low half
// the first value): each piece the round-to-nearest bf16 of what the previous
// ones leave, two values per conversion; a bf16 widens to FP32 exactly by a
// 16-bit shift
__device__ __forceinline__ void bf16_split2(float xa, float xb, uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  auto pack = [](float lo, float hi) -> uint32_t {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
  };
  auto lo_f = [](uint32_t w) { return __uint_as_float(w << 16); };
  auto hi_f = [](uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); };
  p0 = pack(xa, xb);
  const float ra = xa - lo_f(p0), rb = xb - hi_f(p0);
  p1 = pack(ra, rb);
  p2 = pack(ra - lo_f(p1), rb - hi_f(p1));
}

// host: three bf16 pieces (round to nearest even) of a finite double
inline void bf16_pieces(double v, uint16_t out[3]) {
  for (int p = 0; p < 3; ++p) {
    const float f = (float)v;
    uint32_t u;
    __builtin_memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    out[p] = (uint16_t)(u >> 16);
    const uint32_t w = (uint32_t)out[p] << 16;
    float g;
    __builtin_memcpy(&g, &w, 4);
    v -= (double)g;
  }
}

}  // namespace tc
}  // namespace fep3m
