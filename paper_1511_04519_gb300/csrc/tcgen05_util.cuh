// Building blocks of the error-free bf16 tensor-core products (the Ozaki
// scheme: Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012) shared by the recombination and
// the wide panels of the triangular solves: the base-64 digit split of FP64
// values, the K-major core-matrix tile layout, and tcgen05 / bulk-copy /
// mbarrier operations as inline PTX.
//
// A K step is 32 values of the reduction (two MMAs of K = 16); an operand
// value split into 9 signed digits below 64 gives products below 2^12, so a
// sum over at most 455 values and nine digit pairs stays below 2^24, an
// integer that the FP32 accumulator holds exactly.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace matex {
namespace tcx {

constexpr int kTcK = 32;           // reduction values per K step (two MMAs of K = 16)
constexpr int kTcS = 9;            // slices per operand, pairs p + q <= kTcS - 1
constexpr int kTcChunk = 448;      // reduction values summed exactly before a drain (<= 455)
constexpr int kTcSbo = (kTcK / 8) * 128;    // bytes between 8-row groups of a tile

// Byte offset of element (r, k) in a K-major tile of 8x8 core matrices
// (8 rows of 16 bytes each, contiguous): core matrices along k are 128 bytes
// apart, 8-row groups kTcSbo apart.
__device__ __forceinline__ int tc_off(int r, int k) {
  return (r >> 3) * kTcSbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// The nine base-64 digits of r in (-1, 1), signed like r:
// r = sum_p s[p] 64^-(p+1) + e, |e| < 2^-54.  |r| 2^54 is scaled exactly (a
// power of two) and truncated to an integer below 2^54 once; the digits are
// its 6-bit fields, taken with integer operations (the FP64 pipe does one
// multiply and one conversion per value).
__device__ __forceinline__ void slice9(double r, float (&s)[kTcS]) {
  const unsigned long long q = __double2ull_rz(fabs(r) * 0x1p54);
  const float sg = r < 0.0 ? -1.f : 1.f;
#pragma unroll
  for (int p = 0; p < kTcS; ++p) s[p] = sg * (float)(unsigned)((q >> (6 * (kTcS - 1 - p))) & 63ull);
}

// Power of two 2^e with max < 2^e (1 for max = 0).
__device__ __forceinline__ double pow2_above(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);  // mx = f 2^e, f in [0.5, 1)
  return ldexp(1.0, e);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
  const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
  return a | (b << 16);
}

// ---- tcgen05 building blocks (inline PTX) ------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major tile without swizzle: start
// address, byte offset between core matrices along K (leading) and along
// M/N (stride), descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: FP32 accumulator, bf16 A and B, both K-major, M x N.
constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count));
}

// Bounded wait for the phase with parity `ph` of barrier b; false when it
// did not complete within about two seconds.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t ph) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(b)), "r"(ph)
        : "memory");
    if (done) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 2000000000ull) return false;
  }
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                 "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

}  // namespace tcx
}  // namespace matex
