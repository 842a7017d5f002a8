// tc_ops.cuh -- building blocks of the tensor-core (tcgen05) kernels on sm_103a: mbarrier
// waits with an iteration limit, shared-memory matrix descriptors, the MMA and its commit,
// TMEM loads, the exponential tile sum of the epilogue, and the packing of the operand rows
// (the whole base-2 exponent of a pair carried in the MMA's K dimension).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace dsmc {
namespace tc {

// Iterations of a bounded mbarrier wait (about a second) before it gives up.
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// One test of phase `parity`: true once that phase of the barrier has completed.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// The bounded wait of a kernel whose roles stop together: it also gives up as soon as
// another role has set *abort (polled every 64 tries).
__device__ __forceinline__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, const volatile int* abort) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63u) == 63u && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// No-swizzle K-major operand: 16-byte K chunks 128 bytes apart (leading), 8-row groups 256
// bytes apart (stride), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(256u >> 4) << 32) | ((uint64_t)1 << 46);
}

// The MMA shape of every tensor-core kernel here: M = 128 rows (one TMEM lane each),
// N = 128 columns.
constexpr int kMmaM = 128;
constexpr int kMmaN = 128;

// kind::f16 with BF16 operands, or kind::tf32; FP32 accumulator; both K-major; M x N.
template <int KIND>
__device__ __forceinline__ uint32_t instr_desc() {
  const uint32_t fmt = KIND == DSMC_BF16 ? 1u : 2u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kMmaN >> 3) << 17) |
         ((uint32_t)(kMmaM >> 4) << 24);
}

template <int KIND>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t accum) {
  const uint32_t idesc = instr_desc<KIND>();
  if (KIND == DSMC_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accum));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(accum));
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

// Issue a 32x32b.x32 TMEM load (one row per lane, 32 consecutive columns); the registers
// are valid after tmem_wait().
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,"
      "%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Sum over 32 columns of 2^acc with packed FP32 adds (pairs of columns); columns at or
// beyond `valid` contribute nothing.  The order of the additions is fixed.
template <bool MASK>
__device__ __forceinline__ float exp_sum32(const uint32_t* acc, int valid) {
  float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int q2 = 0; q2 < 16; ++q2) {
    float2 e = make_float2(ex2(__uint_as_float(acc[2 * q2])), ex2(__uint_as_float(acc[2 * q2 + 1])));
    if (MASK) {
      e.x = 2 * q2 < valid ? e.x : 0.f;
      e.y = 2 * q2 + 1 < valid ? e.y : 0.f;
    }
    s2 = __fadd2_rn(s2, e);
  }
  return __fadd_rn(s2.x, s2.y);
}


// Tensor-core operand rows.  The K dimension holds the D state coordinates followed by
// four extra columns that carry the per-row and per-column exponent terms exactly as
// two-term (hi + lo) splits in the MMA type:
//   row i    (U): [u_i, alpha_hi, alpha_lo, 1, 1]
//   column j (V): [v_j, 1, 1, beta_hi, beta_lo]
// so that the MMA accumulates alpha_i + beta_j + u_i . v_j.  K is cut into 32-byte planes
// (16 BF16 or 8 TF32 values); plane p of a combination is a [Nr][32 B] array in the
// canonical no-swizzle K-major layout (8-row x 16-byte core matrices: row group g at
// g*256 B, 16-byte chunk c at c*128 B).  Entries beyond D + 4 are zero.
template <int D, int KIND>
__device__ __forceinline__ void store_mma_row_t(unsigned char* base, int Nr, int r, const float* x,
                                                const float* ext) {
  constexpr int kp = KIND == DSMC_BF16 ? 16 : 8;      // values per 32-byte plane
  constexpr int kc = KIND == DSMC_BF16 ? 8 : 4;       // values per 16-byte chunk
  constexpr int np = (D + 4 + kp - 1) / kp;
  unsigned char* row = base + (size_t)(r / 8) * 256 + (size_t)(r % 8) * 16;
#pragma unroll
  for (int ch = 0; ch < 2 * np; ++ch) {  // one 16-byte store per chunk
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (KIND == DSMC_BF16) {
        const int k0 = ch * kc + 2 * q;
        const float v0 = k0 < D ? x[k0] : (k0 < D + 4 ? ext[k0 - D] : 0.f);
        const float v1 = k0 + 1 < D ? x[k0 + 1] : (k0 + 1 < D + 4 ? ext[k0 + 1 - D] : 0.f);
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        w[q] = *reinterpret_cast<const uint32_t*>(&h);
      } else {
        const int k = ch * kc + q;
        const float v = k < D ? x[k] : (k < D + 4 ? ext[k - D] : 0.f);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w[q]) : "f"(v));
      }
    }
    *reinterpret_cast<uint4*>(row + (size_t)(ch / 2) * Nr * 32 + (ch % 2) * 128) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int D>
__device__ __forceinline__ void store_mma_row(unsigned char* base, int Nr, int r, const float* x,
                                              const float* ext, int compute) {
  if (compute == DSMC_BF16) store_mma_row_t<D, DSMC_BF16>(base, Nr, r, x, ext);
  else store_mma_row_t<D, DSMC_TF32>(base, Nr, r, x, ext);
}

// hi + lo split of x in the MMA type (the two values the tensor core reads).
__device__ __forceinline__ void split_mma(float x, int compute, float* hi, float* lo) {
  if (compute == DSMC_BF16) {
    *hi = __bfloat162float(__float2bfloat16_rn(x));
    *lo = __bfloat162float(__float2bfloat16_rn(x - *hi));
  } else {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
    *hi = __uint_as_float(t);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x - *hi));
    *lo = __uint_as_float(t);
  }
}


}  // namespace tc
}  // namespace dsmc
