// rowsum_tc.cu -- the N x N exponent / tile-sum pass of Algorithm 1 with the Gaussian
// cross term u_i . v_j on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One CTA computes 128 rows (one TMEM lane each) of one combination against a chunk of
// columns, in blocks of 128 columns.  The operands carry the whole base-2 exponent: row i is
// [u_i, alpha_hi, alpha_lo, 1, 1] and column j is [v_j, 1, 1, beta_hi, beta_lo] (two-term
// splits of alpha_i and beta_j in the MMA type), so the accumulator holds
// e_ij = alpha_i + beta_j + u_i . v_j and the epilogue is only 2^e and the tile sums:
//   - a control warp stages the row tile once and each 128-column block of the columns with
//     TMA bulk copies (cp.async.bulk, operands pre-laid out by the prologue in the canonical
//     no-swizzle K-major layout, one 32-byte K plane = 16 BF16 or 8 TF32 values per copy), and
//     issues P tcgen05.mma (M = 128, N = 128, one per K plane) per block into one of two
//     128-column TMEM accumulators; every MMA commits to its accumulator's barrier and to
//     its column slot's, every row tile's last MMA to the tile's, and the control warp
//     refills a slot or a tile as soon as the MMAs that read it have completed;
//   - eight epilogue warps (two per TMEM lane quarter, splitting the block's columns) read the
//     accumulator with tcgen05.ld, take 2^x on MUFU and keep the per-tile sums, while the
//     tensor core already computes the next block; when one chunk covers the whole row they
//     also keep their half's running row total, which the row-CDF kernel adds up.
// Every wait is bounded; on a timeout the CTA records DSMC_ERR_TIMEOUT, waits (bounded) for
// its own outstanding MMA, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace dsmc {

namespace {

constexpr int kTcRows = 128;                   // MMA M: one TMEM lane per row
constexpr int kTcCols = 128;                   // MMA N: columns per block
constexpr int kEpiWarps = 8;
constexpr int kTcThreads = (kEpiWarps + 1) * 32;
constexpr int kTileBytes = 128 * 32;           // 128 rows (or columns) x 32 bytes of K
constexpr uint32_t kTmemCols = 2 * kTcCols;    // two accumulators
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// No-swizzle K-major operand: 16-byte K chunks 128 bytes apart (leading), 8-row groups 256
// bytes apart (stride), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)(256u >> 4) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 with BF16 operands, or kind::tf32; FP32 accumulator; both K-major; M x N.
template <int KIND>
__device__ __forceinline__ uint32_t instr_desc() {
  const uint32_t fmt = KIND == DSMC_BF16 ? 1u : 2u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTcCols >> 3) << 17) |
         ((uint32_t)(kTcRows >> 4) << 24);
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

// Work item = (combination s, 128-row tile rt, column chunk ch); the grid is persistent
// (two CTAs per SM) and each CTA walks items blockIdx.x, blockIdx.x + gridDim.x, ...
struct Item {
  int s, rt, j0, j1, nblk;
};

__device__ __forceinline__ Item item_of(const MergeArgs& a, int it) {
  const int RT = (a.N + kTcRows - 1) / kTcRows;
  Item r;
  r.s = it / (RT * a.CH);
  const int rem = it % (RT * a.CH);
  r.rt = rem / a.CH;
  r.j0 = (rem % a.CH) * a.CW;
  r.j1 = min(r.j0 + a.CW, a.N);
  r.nblk = (r.j1 - r.j0 + kTcCols - 1) / kTcCols;
  return r;
}

// Column blocks staged ahead (P = 1: 16 x 4 KB, P = 2: 10 x 8 KB, P = 3: 6 x 12 KB); a slot
// is refilled once the MMA that read it has completed.
template <int P>
__host__ __device__ constexpr int v_slots() {
  return P == 1 ? 16 : (P == 2 ? 10 : 6);
}

template <int KIND, int P>
__global__ void __launch_bounds__(kTcThreads, 2) rowsum_tc_kernel(MergeArgs a, int n_items) {
  constexpr int kVSlots = v_slots<P>();
  constexpr int kSlotBytes = P * kTileBytes;
  extern __shared__ __align__(128) unsigned char dsm[];
  unsigned char* sA = dsm;                                        // [2][P][4 KB] row tiles
  unsigned char* sV = dsm + 2 * kSlotBytes;                       // [kVSlots][P][4 KB] column blocks
  // bar_a / bar_v: a row tile / column block landed (TMA); bar_afree / bar_vfree: the MMAs
  // that read it completed (tcgen05.commit), so the buffer may be refilled; bar_mma: a block's
  // accumulator is complete; bar_epi: the epilogue has read it out of TMEM
  __shared__ __align__(8) uint64_t bar_a[2], bar_afree[2], bar_v[kVSlots], bar_vfree[kVSlots], bar_mma[2],
      bar_epi[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_s;

  const int N = a.N, B = a.B;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    abort_s = 0;
    for (int q = 0; q < 2; ++q) {
      mbar_init(smem_u32(&bar_a[q]), 1);
      mbar_init(smem_u32(&bar_afree[q]), 1);
      mbar_init(smem_u32(&bar_mma[q]), 1);
      mbar_init(smem_u32(&bar_epi[q]), kEpiWarps);
    }
    for (int q = 0; q < kVSlots; ++q) {
      mbar_init(smem_u32(&bar_v[q]), 1);
      mbar_init(smem_u32(&bar_vfree[q]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tb = tmem_base;

  if (warp == kEpiWarps) {
    // ------------------------------------------------------------ control: TMA + MMA
    if (lane == 0) {
      bool ok = true;
      int issued = 0;
      // load cursor over the CTA's block sequence
      int l_it = blockIdx.x, l_b = 0, lq = 0;
      Item li = item_of(a, l_it);
      const size_t plane = (size_t)a.Nr * 32;  // bytes of one K plane of one combination
      auto load_next = [&]() {  // the P planes of the next column block, one barrier
        if (l_it >= n_items) return;
        const unsigned char* src =
            a.ws.Vb + (size_t)li.s * P * plane + ((size_t)li.j0 + (size_t)l_b * kTcCols) * 32;
        const int slot = lq % kVSlots;
        const uint32_t bar = smem_u32(&bar_v[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)kSlotBytes)
                     : "memory");
#pragma unroll
        for (int p = 0; p < P; ++p)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(sV + (size_t)slot * kSlotBytes + (size_t)p * kTileBytes)),
              "l"(src + (size_t)p * plane), "r"((uint32_t)kTileBytes), "r"(bar)
              : "memory");
        ++lq;
        if (++l_b == li.nblk) {
          l_b = 0;
          l_it += gridDim.x;
          if (l_it < n_items) li = item_of(a, l_it);
        }
      };
      auto load_a = [&](int it, int slot) {
        if (it >= n_items) return;
        const Item t = item_of(a, it);
        const unsigned char* src = a.ws.Ub + (size_t)t.s * P * plane + (size_t)t.rt * kTileBytes;
        const uint32_t bar = smem_u32(&bar_a[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)kSlotBytes)
                     : "memory");
#pragma unroll
        for (int p = 0; p < P; ++p)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(sA + (size_t)slot * kSlotBytes + (size_t)p * kTileBytes)),
              "l"(src + (size_t)p * plane), "r"((uint32_t)kTileBytes), "r"(bar)
              : "memory");
      };
      // Buffers are refilled as soon as the MMAs that read them complete (their commits):
      // column block q + kVSlots - 2 is loaded after block q's MMA is issued (into the slot of
      // block q - 2), and item k + 1's row tile after item k's first MMA (into item k - 1's
      // buffer).
      load_a(blockIdx.x, 0);
      load_a(blockIdx.x + gridDim.x, 1);
      for (int q = 0; q < kVSlots; ++q) load_next();
      int q = 0;  // global block index of this CTA
      int k = 0;  // item index of this CTA
      int last_item = -1;
      for (int it = blockIdx.x; it < n_items && ok; it += gridDim.x, ++k) {
        const Item cur = item_of(a, it);
        ok = mbar_wait(smem_u32(&bar_a[k & 1]), (uint32_t)(k >> 1) & 1);
        const uint32_t sa = smem_u32(sA + (size_t)(k & 1) * kSlotBytes);
        for (int b = 0; b < cur.nblk && ok; ++b, ++q) {
          const int buf = q & 1;
          const int slot = q % kVSlots;
          if (q >= 2) ok = mbar_wait(smem_u32(&bar_epi[buf]), (uint32_t)((q >> 1) - 1) & 1);
          if (ok) ok = mbar_wait(smem_u32(&bar_v[slot]), (uint32_t)(q / kVSlots) & 1);
          if (!ok) break;
          if (a.stall) continue;  // test switch: nothing is issued, no accumulator completes
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sv = smem_u32(sV + (size_t)slot * kSlotBytes);
#pragma unroll
          for (int p = 0; p < P; ++p)
            mma<KIND>(tb + (uint32_t)buf * kTcCols, smem_desc(sa + p * kTileBytes), smem_desc(sv + p * kTileBytes),
                      p > 0 ? 1u : 0u);
          mma_commit(smem_u32(&bar_mma[buf]));
          mma_commit(smem_u32(&bar_vfree[slot]));
          if (b == cur.nblk - 1) {
            mma_commit(smem_u32(&bar_afree[k & 1]));
            last_item = k;
          }
          ++issued;
          if (q >= 2) {  // off the issue path: block q - 2's MMA is long complete
            ok = mbar_wait(smem_u32(&bar_vfree[(q - 2) % kVSlots]), (uint32_t)((q - 2) / kVSlots) & 1);
            if (!ok) break;
            load_next();
          }
          if (b == 0 && k >= 1) {  // item k - 1's MMAs are done: its buffer takes item k + 1
            ok = mbar_wait(smem_u32(&bar_afree[(k - 1) & 1]), (uint32_t)((k - 1) >> 1) & 1);
            if (!ok) break;
            load_a(it + gridDim.x, (k + 1) & 1);
          }
        }
      }
      // every committed MMA must be complete (and its barrier arrivals landed) before TMEM
      // and the shared memory are released
      if (issued > 0) {
        const int qq = issued - 1;
        mbar_wait(smem_u32(&bar_mma[qq & 1]), (uint32_t)(qq >> 1) & 1);
        mbar_wait(smem_u32(&bar_vfree[qq % kVSlots]), (uint32_t)(qq / kVSlots) & 1);
      }
      if (last_item >= 0) mbar_wait(smem_u32(&bar_afree[last_item & 1]), (uint32_t)(last_item >> 1) & 1);
      if (!ok) {
        atomicExch(&abort_s, 1);
        record_status(a.ws.status, DSMC_ERR_TIMEOUT);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    const int g = warp & 3, h = warp >> 2;
    int q = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
      const Item cur = item_of(a, it);
      const int s = cur.s;
      const int row = cur.rt * kTcRows + 32 * g + lane;
      float* Trow = a.ws.T + ((size_t)s * N + (row < N ? row : 0)) * a.nTp;
      float racc = 0.f;  // this half's tile weights of the row, blocks in order
      bool stop = false;
      for (int b = 0; b < cur.nblk; ++b, ++q) {
        const int buf = q & 1;
        const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bar_mma[buf]), (uint32_t)(q >> 1) & 1)) &&
                        !*reinterpret_cast<volatile int*>(&abort_s);
        if (!ok) {  // warp-uniform
          if (lane == 0) {
            atomicExch(&abort_s, 1);
            record_status(a.ws.status, DSMC_ERR_TIMEOUT);
          }
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int col0 = cur.j0 + b * kTcCols + 64 * h;
        uint32_t acc0[32], acc1[32];
        const uint32_t taddr = tb + ((uint32_t)(32 * g) << 16) + (uint32_t)buf * kTcCols + 64 * h;
        tmem_ld32(taddr, acc0);
        tmem_ld32(taddr + 32, acc1);
        tmem_wait();
        // the accumulator is in registers: release the TMEM buffer to the MMA issuer now
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_epi[buf]));
        float t0, t1;
        if (col0 + 64 <= cur.j1) {
          t0 = exp_sum32<false>(acc0, 32);
          t1 = exp_sum32<false>(acc1, 32);
        } else {
          t0 = exp_sum32<true>(acc0, cur.j1 - col0);
          t1 = exp_sum32<true>(acc1, cur.j1 - col0 - 32);
        }
        racc = __fadd_rn(racc, __fadd_rn(t0, t1));
        if (row < N) {
          if (B == 32) {  // tiles col0 / 32 (even: chunks start at multiples of 128) and + 1
            if (col0 + 32 < cur.j1)
              *reinterpret_cast<float2*>(Trow + col0 / 32) = make_float2(t0, t1);
            else if (col0 < cur.j1)
              Trow[col0 / 32] = t0;
          } else if (col0 < cur.j1) {
            Trow[col0 / 64] = __fadd_rn(t0, t1);
          }
        }
      }
      if (stop) break;
      // one column chunk: the item covers the whole row, so its two halves' sums are the
      // row total's two parts (the row-CDF kernel adds them instead of re-reading T)
      if (a.CH == 1 && row < N) a.ws.rowpart[((size_t)s * 2 + h) * N + row] = racc;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(kTmemCols));
  }
}

// Dynamic shared memory: 2 row tiles + the column-block ring (72 KB at P = 1, 96 KB at
// P = 2 and at P = 3), padded so that at most two CTAs (2 x 256 TMEM columns) share an SM.
constexpr size_t kDynSmem = 100 * 1024;
static_assert((2 + v_slots<1>()) * kTileBytes <= kDynSmem, "staging buffers, one K plane");
static_assert((2 + v_slots<2>()) * 2 * kTileBytes <= kDynSmem, "staging buffers, two K planes");
static_assert((2 + v_slots<3>()) * 3 * kTileBytes <= kDynSmem, "staging buffers, three K planes");

template <int KIND, int P>
cudaError_t launch_t(const MergeArgs& a, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(rowsum_tc_kernel<KIND, P>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDynSmem);
  if (e != cudaSuccess) return e;
  const int RT = (a.N + kTcRows - 1) / kTcRows;
  const int n_items = a.mc * RT * a.CH;
  const int grid = n_items < 2 * 152 ? n_items : 2 * 152;
  rowsum_tc_kernel<KIND, P><<<grid, kTcThreads, kDynSmem, st>>>(a, n_items);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rowsum_tc(const MergeArgs& a, cudaStream_t s) {
  if (a.compute == DSMC_BF16 && a.mma_planes == 1) return launch_t<DSMC_BF16, 1>(a, s);
  if (a.compute == DSMC_BF16 && a.mma_planes == 2) return launch_t<DSMC_BF16, 2>(a, s);
  if (a.compute == DSMC_BF16 && a.mma_planes == 3) return launch_t<DSMC_BF16, 3>(a, s);
  if (a.compute == DSMC_TF32 && a.mma_planes == 3) return launch_t<DSMC_TF32, 3>(a, s);
  if (a.compute == DSMC_TF32 && a.mma_planes == 1) return launch_t<DSMC_TF32, 1>(a, s);
  if (a.compute == DSMC_TF32 && a.mma_planes == 2) return launch_t<DSMC_TF32, 2>(a, s);
  return cudaErrorInvalidValue;
}

}  // namespace dsmc
