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
//     tensor core already computes the next block.
// Every wait is bounded; on a timeout the CTA records DSMC_ERR_TIMEOUT, waits (bounded) for
// its own outstanding MMA and for every bulk copy it issued but did not consume, frees its
// TMEM and returns.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tc_ops.cuh"

namespace dsmc {

namespace {

using namespace tc;

constexpr int kTcRows = 128;                   // MMA M: one TMEM lane per row
constexpr int kTcCols = 128;                   // MMA N: columns per block
constexpr int kEpiWarps = 8;
constexpr int kTcThreads = (kEpiWarps + 1) * 32;
constexpr int kTileBytes = 128 * 32;           // 128 rows (or columns) x 32 bytes of K
constexpr uint32_t kTmemCols = 2 * kTcCols;    // two accumulators
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
      // load cursor over the CTA's block sequence; a_armed / a_seen count the row tiles
      // loaded and waited for, q_seen the column blocks waited for (lq counts those loaded)
      int l_it = blockIdx.x, l_b = 0, lq = 0;
      int a_armed = 0, a_seen = 0, q_seen = 0;
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
        ++a_armed;
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
        if (ok) ++a_seen;
        const uint32_t sa = smem_u32(sA + (size_t)(k & 1) * kSlotBytes);
        for (int b = 0; b < cur.nblk && ok; ++b, ++q) {
          const int buf = q & 1;
          const int slot = q % kVSlots;
          if (q >= 2) ok = mbar_wait(smem_u32(&bar_epi[buf]), (uint32_t)((q >> 1) - 1) & 1);
          if (ok) ok = mbar_wait(smem_u32(&bar_v[slot]), (uint32_t)(q / kVSlots) & 1);
          if (!ok) break;
          q_seen = q + 1;
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
      // bulk copies issued but never waited for (an aborted walk) must land before the
      // shared memory is released: one bounded wait on each pending phase (a slot or row
      // buffer has at most one pending phase, since it is refilled only after it was read)
      for (int qq = q_seen; qq < lq; ++qq)
        mbar_wait(smem_u32(&bar_v[qq % kVSlots]), (uint32_t)(qq / kVSlots) & 1);
      for (int kk = a_seen; kk < a_armed; ++kk)
        mbar_wait(smem_u32(&bar_a[kk & 1]), (uint32_t)(kk >> 1) & 1);
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
  const int full = 2 * (a.sms > 0 ? a.sms : 1);  // two resident CTAs per SM
  const int grid = n_items < full ? n_items : full;
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
