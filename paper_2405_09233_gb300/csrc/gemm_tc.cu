// Per-Fourier-slice complex products on the 5th-generation tensor cores (tcgen05), the
// low-precision operator of the mixed-precision inner solve:
//     Y_k = A_k X_k - X_k B_k      (Eq. (2) in the Fourier domain, Algorithm 1 step 2)
// with BF16 or TF32 inputs and FP32 accumulation in tensor memory.
//
// Planar complex, four real products per K step into two TMEM accumulators:
//     Re Y += Ar Xr - Ai Xi,   Im Y += Ai Xr + Ar Xi              (l over n)
//     Re Y += -Xr Br + Xi Bi,  Im Y += -Xr Bi - Xi Br             (l over s)
// The minus signs are the instruction descriptor's negate-A bit, so no negated copies exist.
// Keeping the operands planar (rather than a realified 2n x 2n matrix) halves the bytes of A_k
// that stream from HBM, which matters because for s ~ 256 the product sits at the HBM/tensor
// ridge point.
//
// Operand layouts (all K-major, i.e. the reduction index l contiguous; rows padded to ld):
//   A_k planes  [k][i][l]  (row-major A_k, prepared once per operator)
//   X_k planes  [k][j][l]  (column-major X_k, written by the planar DFT)        -> B operand
//   X_k planes  [k][i][l]  (row-major X_k, a transposed copy)                    -> A operand
//   B_k planes  [k][j][l]  (column-major B_k, prepared once per operator)        -> B operand
//
// One CTA computes a 128 x BN output tile of one slice.  Warp roles (192 threads):
//   warps 0-3  epilogue: TMEM -> registers -> Y (float2, column-major), TMEM lanes 32w..32w+31
//   warp 4     TMA producer: 4 tiles per stage (A re/im, B re/im), 128-byte swizzle
//   warp 5     TMEM allocator and MMA issuer (one elected lane)
// Stages are recycled through full/empty mbarriers; tcgen05.commit arrives on "empty" when the
// MMAs reading a stage have completed.  Every wait is bounded: on expiry the kernel records an
// error code, skips the rest of its work, still frees its TMEM and returns.
#include <algorithm>
#include <cstdlib>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include "internal.cuh"
#include "tc.cuh"
#include "tcgen05.cuh"
#include "tune.cuh"
#include "fft_reg.cuh"

namespace ts {
namespace {

constexpr int kTileM = 128;
constexpr int kStageBytesMax = 200 * 1024;
using namespace tcg;



template <int BN, int ESZ>
struct TcCfg {
  static constexpr int kElemsK = 128 / ESZ;                  // K elements per 128-byte row
  static constexpr int kTileA = kTileM * 128;                // bytes of one A plane tile
  static constexpr int kTileB = BN * 128;                    // bytes of one B plane tile
  static constexpr int kStage = 2 * kTileA + 2 * kTileB;
  static constexpr int kStages = (kStageBytesMax / kStage) > 4 ? 4 : (kStageBytesMax / kStage);
  static constexpr int kSmem = kStages * kStage + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int kTmemCols = 2 * BN;                   // Re and Im accumulators
  static constexpr int kSubK = 128 / 32;                     // MMA K steps per stage (32 bytes each)
};

// PARTS = 1: one product per operand pair.  PARTS = 3 (split TF32): every l-block is visited three
// times, hi*hi, hi*lo and lo*hi, accumulating in the same FP32 TMEM accumulators (FP32-level
// accuracy on the TF32 tensor pipe).
// One 128 x BN output tile (rows i0.., columns j0..) of slice k; Y holds K slices of column-major
// n x s float2 matrices.  `maps` may live in kernel parameter space or in global memory.
template <int BN, int ESZ, int PARTS>
__device__ __forceinline__ void tc_sylv_tile(const TcMaps& maps, float2* __restrict__ Y, int n, int s, int nyq,
                                             int k, int i0, int j0, int* err, int stall,
                                             unsigned long long wait_ns) {
  using Cfg = TcCfg<BN, ESZ>;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * Cfg::kStages + 1);
  const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + Cfg::kStages);
  const uint32_t bar_acc = smem_u32(bars + 2 * Cfg::kStages);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool real = (k == 0) || (k == nyq);
  const int it1 = (n + Cfg::kElemsK - 1) / Cfg::kElemsK;      // stages of the A_k X_k product
  const int it2 = (s + Cfg::kElemsK - 1) / Cfg::kElemsK;      // stages of the X_k B_k product
  const int iters = PARTS * (it1 + it2);

  if (threadIdx.x == 0) {
    for (int q = 0; q < Cfg::kStages; ++q) {
      mbar_init(bar_full + 8 * q, 1);
      mbar_init(bar_empty + 8 * q, 1);
    }
    mbar_init(bar_acc, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(Cfg::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    if (lane == 0) {
      int issued = 0;   // stages whose loads were issued
      for (int it = 0; it < iters; ++it) {
        const int slot = it % Cfg::kStages;
        const uint32_t phase = (uint32_t)(it / Cfg::kStages) & 1u;
        if (!mbar_wait(bar_empty + 8 * slot, phase ^ 1u, err, 1, wait_ns)) break;
        if (stall) continue;   // test aid: arm no stage, so the MMA warp's wait expires
        const uint32_t full = bar_full + 8 * slot;
        // a real slice (k = 0 or p/2) multiplies the real planes only, so only those are loaded
        mbar_expect_tx(full, real ? Cfg::kTileA + Cfg::kTileB : Cfg::kStage);
        const uint32_t sA = base + slot * Cfg::kStage;
        const uint32_t sAi = sA + Cfg::kTileA, sB = sA + 2 * Cfg::kTileA, sBi = sB + Cfg::kTileB;
        const int blk = it / PARTS, part = it % PARTS;
        const bool alo = part == 2, blo = part == 1;
        if (blk < it1) {
          const int l0 = blk * Cfg::kElemsK;
          tma_load_3d(sA, alo ? &maps.a_re_lo : &maps.a_re, l0, i0, k, full);
          tma_load_3d(sB, blo ? &maps.xc_re_lo : &maps.xc_re, l0, j0, k, full);
          if (!real) {
            tma_load_3d(sAi, alo ? &maps.a_im_lo : &maps.a_im, l0, i0, k, full);
            tma_load_3d(sBi, blo ? &maps.xc_im_lo : &maps.xc_im, l0, j0, k, full);
          }
        } else {
          const int l0 = (blk - it1) * Cfg::kElemsK;
          tma_load_3d(sA, alo ? &maps.xr_re_lo : &maps.xr_re, l0, i0, k, full);
          tma_load_3d(sB, blo ? &maps.b_re_lo : &maps.b_re, l0, j0, k, full);
          if (!real) {
            tma_load_3d(sAi, alo ? &maps.xr_im_lo : &maps.xr_im, l0, i0, k, full);
            tma_load_3d(sBi, blo ? &maps.b_im_lo : &maps.b_im, l0, j0, k, full);
          }
        }
        issued = it + 1;
      }
      // Every stage this warp loaded lands before the CTA exits, also when an error stopped the MMA
      // warp from consuming it: bounded waits on the last kStages loads (immediate when all were used).
      for (int it = issued > Cfg::kStages ? issued - Cfg::kStages : 0; it < issued; ++it)
        mbar_wait(bar_full + 8 * (it % Cfg::kStages), (uint32_t)(it / Cfg::kStages) & 1u, err, 4, wait_ns);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      constexpr int fmt = ESZ == 2 ? 1 : 2;
      constexpr uint32_t idp = make_idesc(fmt, kTileM, BN, false);
      constexpr uint32_t idn = make_idesc(fmt, kTileM, BN, true);
      const uint32_t d_re = tmem, d_im = tmem + BN;
      bool ok = true;
      for (int it = 0; it < iters && ok; ++it) {
        const int slot = it % Cfg::kStages;
        const uint32_t phase = (uint32_t)(it / Cfg::kStages) & 1u;
        if (!mbar_wait(bar_full + 8 * slot, phase, err, 2, wait_ns)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sA = base + slot * Cfg::kStage;
        const uint64_t dAr = smem_desc_sw128(sA), dAi = smem_desc_sw128(sA + Cfg::kTileA);
        const uint64_t dBr = smem_desc_sw128(sA + 2 * Cfg::kTileA);
        const uint64_t dBi = smem_desc_sw128(sA + 2 * Cfg::kTileA + Cfg::kTileB);
#pragma unroll
        for (int kk = 0; kk < Cfg::kSubK; ++kk) {
          const uint64_t o = (uint64_t)(kk * 2);   // 32 bytes >> 4
          const uint32_t first = (it == 0 && kk == 0) ? 0u : 1u;
          if (it / PARTS < it1) {
            mma_issue(d_re, dAr + o, dBr + o, idp, first, ESZ == 4);
            if (!real) {
              mma_issue(d_re, dAi + o, dBi + o, idn, 1u, ESZ == 4);
              mma_issue(d_im, dAi + o, dBr + o, idp, first, ESZ == 4);
              mma_issue(d_im, dAr + o, dBi + o, idp, 1u, ESZ == 4);
            }
          } else {
            mma_issue(d_re, dAr + o, dBr + o, idn, 1u, ESZ == 4);
            if (!real) {
              mma_issue(d_re, dAi + o, dBi + o, idp, 1u, ESZ == 4);
              mma_issue(d_im, dAr + o, dBi + o, idn, 1u, ESZ == 4);
              mma_issue(d_im, dAi + o, dBr + o, idn, 1u, ESZ == 4);
            }
          }
        }
        mma_commit(bar_empty + 8 * slot);
      }
      mma_commit(bar_acc);
      // after an error the MMAs already issued still complete before TMEM is freed
      if (!ok) mbar_wait(bar_acc, 0u, err, 5, wait_ns);
    }
  } else {
    // Epilogue: warp w reads TMEM lanes 32w..32w+31 (= output rows i0 + 32w + lane).
    const bool ok = mbar_wait(bar_acc, 0u, err, 3, wait_ns);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      const int row = i0 + warp * 32 + lane;
      float2* Yk = Y + (long long)k * n * s;
      const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float re[32], im[32];
        tmem_ld32(lane_base + c0, re);
        if (!real) {
          tmem_ld32(lane_base + BN + c0, im);
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c) im[c] = 0.f;
        }
        if (row < n) {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int j = j0 + c0 + c;
            if (j < s) Yk[(long long)j * n + row] = make_float2(re[c], im[c]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kTmemCols));
  }
}

template <int BN, int ESZ, int PARTS>
__global__ void __launch_bounds__(192, 1)
    k_tc_sylv(const __grid_constant__ TcMaps maps, float2* __restrict__ Y, int n, int s, int nyq, int* err, int stall,
              unsigned long long wait_ns) {
  tc_sylv_tile<BN, ESZ, PARTS>(maps, Y, n, s, nyq, blockIdx.z, blockIdx.y * kTileM, blockIdx.x * BN, err, stall,
                               wait_ns);
}

template <typename OpT> __device__ __forceinline__ OpT to_op(float v);
template <> __device__ __forceinline__ __nv_bfloat16 to_op<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <> __device__ __forceinline__ float to_op<float>(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// Low part of the split-TF32 representation: tf32(v - tf32(v)).
__device__ __forceinline__ float tf32_lo(float v) { return to_op<float>(v - to_op<float>(v)); }

// ------------------------------------------------------------------------------------------------
// Batched form: one CTA per (instance, slice, tile) work item; every instance has its own tensor
// maps (a table in global memory, written from the host before the launch) and output.
// ------------------------------------------------------------------------------------------------
template <int BN, int ESZ, int PARTS>
__global__ void __launch_bounds__(192, 1)
    k_b_tc(const TcMaps* __restrict__ maps, const BTcInst* __restrict__ inst, const int* __restrict__ active,
           const int4* __restrict__ items, int* err) {
  const int4 it = items[blockIdx.x];
  if (!active[it.x]) return;   // instance not in the current inner cycle (uniform over the CTA)
  const BTcInst& b = inst[it.x];
  tc_sylv_tile<BN, ESZ, PARTS>(maps[it.x], b.Y, b.n, b.s, b.nyq, it.y, it.z, it.w, err, 0, kWaitNs);
}

// Persistent batched form: gridDim.x CTAs (at most one per SM) walk the cost-sorted work list with
// stride gridDim.x, skipping instances outside the current inner cycle.  Barriers are initialised
// and tensor memory is allocated once per CTA; the TMA / MMA stage ring runs on from one item to the
// next (one stage counter for the whole walk), and two accumulator sets in tensor memory let the
// epilogue of item t drain while item t + 1 is multiplied (acc_full / acc_empty barriers per set).
// Per item the MMAs and their order are those of k_b_tc, so both give bitwise the same products.
// Every wait is bounded; after an expired wait each role stops where it is, the producer waits for
// the stages it loaded, the MMA warp for the MMAs it issued, and tensor memory is freed.
template <int BN, int ESZ, int PARTS>
__global__ void __launch_bounds__(192, 1)
    k_b_tc_persist(const TcMaps* __restrict__ maps, const BTcInst* __restrict__ inst, const int* __restrict__ active,
                   const int4* __restrict__ items, int nitems, int* err) {
  using Cfg = TcCfg<BN, ESZ>;
  constexpr int kCols = 2 * Cfg::kTmemCols;   // two accumulator sets of (Re, Im)
  static_assert(kCols <= 512, "tensor memory");
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Cfg::kStages * Cfg::kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * Cfg::kStages + 5);
  const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + Cfg::kStages);
  const uint32_t bar_accf = smem_u32(bars + 2 * Cfg::kStages);       // [2]: accumulator set ready
  const uint32_t bar_acce = smem_u32(bars + 2 * Cfg::kStages + 2);   // [2]: accumulator set drained
  const uint32_t bar_done = smem_u32(bars + 2 * Cfg::kStages + 4);   // every issued MMA completed
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int q = 0; q < Cfg::kStages; ++q) {
      mbar_init(bar_full + 8 * q, 1);
      mbar_init(bar_empty + 8 * q, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_accf + 8 * b, 1);
      mbar_init(bar_acce + 8 * b, 4);   // one arrival per epilogue warp
    }
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  auto iters_of = [&](const BTcInst& b) {
    return PARTS * ((b.n + Cfg::kElemsK - 1) / Cfg::kElemsK + (b.s + Cfg::kElemsK - 1) / Cfg::kElemsK);
  };

  if (warp == 4) {
    if (lane == 0) {
      long long g = 0, issued = 0;   // stages walked / whose loads were issued
      bool ok = true;
      for (int q = blockIdx.x; q < nitems && ok; q += gridDim.x) {
        const int4 it = items[q];
        if (!active[it.x]) continue;
        const BTcInst& b = inst[it.x];
        const TcMaps& m = maps[it.x];
        const int k = it.y, i0 = it.z, j0 = it.w;
        const bool real = (k == 0) || (k == b.nyq);
        const int it1 = (b.n + Cfg::kElemsK - 1) / Cfg::kElemsK, iters = iters_of(b);
        for (int u = 0; u < iters; ++u, ++g) {
          const int slot = (int)(g % Cfg::kStages);
          const uint32_t phase = (uint32_t)(g / Cfg::kStages) & 1u;
          if (!mbar_wait(bar_empty + 8 * slot, phase ^ 1u, err, 1)) {
            ok = false;
            break;
          }
          const uint32_t full = bar_full + 8 * slot;
          mbar_expect_tx(full, real ? Cfg::kTileA + Cfg::kTileB : Cfg::kStage);
          const uint32_t sA = base + slot * Cfg::kStage;
          const uint32_t sAi = sA + Cfg::kTileA, sB = sA + 2 * Cfg::kTileA, sBi = sB + Cfg::kTileB;
          const int blk = u / PARTS, part = u % PARTS;
          const bool alo = part == 2, blo = part == 1;
          if (blk < it1) {
            const int l0 = blk * Cfg::kElemsK;
            tma_load_3d(sA, alo ? &m.a_re_lo : &m.a_re, l0, i0, k, full);
            tma_load_3d(sB, blo ? &m.xc_re_lo : &m.xc_re, l0, j0, k, full);
            if (!real) {
              tma_load_3d(sAi, alo ? &m.a_im_lo : &m.a_im, l0, i0, k, full);
              tma_load_3d(sBi, blo ? &m.xc_im_lo : &m.xc_im, l0, j0, k, full);
            }
          } else {
            const int l0 = (blk - it1) * Cfg::kElemsK;
            tma_load_3d(sA, alo ? &m.xr_re_lo : &m.xr_re, l0, i0, k, full);
            tma_load_3d(sB, blo ? &m.b_re_lo : &m.b_re, l0, j0, k, full);
            if (!real) {
              tma_load_3d(sAi, alo ? &m.xr_im_lo : &m.xr_im, l0, i0, k, full);
              tma_load_3d(sBi, blo ? &m.b_im_lo : &m.b_im, l0, j0, k, full);
            }
          }
          issued = g + 1;
        }
      }
      for (long long u = issued > Cfg::kStages ? issued - Cfg::kStages : 0; u < issued; ++u)
        mbar_wait(bar_full + 8 * (int)(u % Cfg::kStages), (uint32_t)(u / Cfg::kStages) & 1u, err, 4);
    }
  } else if (warp == 5) {
    if (lane == 0) {
      constexpr int fmt = ESZ == 2 ? 1 : 2;
      constexpr uint32_t idp = make_idesc(fmt, kTileM, BN, false);
      constexpr uint32_t idn = make_idesc(fmt, kTileM, BN, true);
      long long g = 0;
      int t = 0;   // items multiplied by this CTA
      bool ok = true;
      for (int q = blockIdx.x; q < nitems && ok; q += gridDim.x) {
        const int4 it = items[q];
        if (!active[it.x]) continue;
        const BTcInst& b = inst[it.x];
        const bool real = (it.y == 0) || (it.y == b.nyq);
        const int it1 = (b.n + Cfg::kElemsK - 1) / Cfg::kElemsK, iters = iters_of(b);
        const int set = t & 1;
        // the epilogue has drained this accumulator set's previous item (t - 2)
        if (t >= 2 && !mbar_wait(bar_acce + 8 * set, (uint32_t)((t >> 1) + 1) & 1u, err, 6)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d_re = tmem + set * Cfg::kTmemCols, d_im = d_re + BN;
        for (int u = 0; u < iters; ++u, ++g) {
          const int slot = (int)(g % Cfg::kStages);
          const uint32_t phase = (uint32_t)(g / Cfg::kStages) & 1u;
          if (!mbar_wait(bar_full + 8 * slot, phase, err, 2)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sA = base + slot * Cfg::kStage;
          const uint64_t dAr = smem_desc_sw128(sA), dAi = smem_desc_sw128(sA + Cfg::kTileA);
          const uint64_t dBr = smem_desc_sw128(sA + 2 * Cfg::kTileA);
          const uint64_t dBi = smem_desc_sw128(sA + 2 * Cfg::kTileA + Cfg::kTileB);
#pragma unroll
          for (int kk = 0; kk < Cfg::kSubK; ++kk) {
            const uint64_t o = (uint64_t)(kk * 2);
            const uint32_t first = (u == 0 && kk == 0) ? 0u : 1u;
            if (u / PARTS < it1) {
              mma_issue(d_re, dAr + o, dBr + o, idp, first, ESZ == 4);
              if (!real) {
                mma_issue(d_re, dAi + o, dBi + o, idn, 1u, ESZ == 4);
                mma_issue(d_im, dAi + o, dBr + o, idp, first, ESZ == 4);
                mma_issue(d_im, dAr + o, dBi + o, idp, 1u, ESZ == 4);
              }
            } else {
              mma_issue(d_re, dAr + o, dBr + o, idn, 1u, ESZ == 4);
              if (!real) {
                mma_issue(d_re, dAi + o, dBi + o, idp, 1u, ESZ == 4);
                mma_issue(d_im, dAr + o, dBi + o, idn, 1u, ESZ == 4);
                mma_issue(d_im, dAi + o, dBr + o, idn, 1u, ESZ == 4);
              }
            }
          }
          mma_commit(bar_empty + 8 * slot);
        }
        if (!ok) break;
        mma_commit(bar_accf + 8 * set);
        ++t;
      }
      // every MMA issued (also on an error path) completes before tensor memory is freed
      mma_commit(bar_done);
      mbar_wait(bar_done, 0u, err, 5);
    }
  } else {
    // Epilogue: warp w reads TMEM lanes 32w..32w+31 (= output rows i0 + 32w + lane) of set t & 1.
    int t = 0;
    for (int q = blockIdx.x; q < nitems; q += gridDim.x) {
      const int4 it = items[q];
      if (!active[it.x]) continue;
      const BTcInst& b = inst[it.x];
      const int k = it.y, i0 = it.z, j0 = it.w;
      const bool real = (k == 0) || (k == b.nyq);
      const int set = t & 1;
      if (!mbar_wait(bar_accf + 8 * set, (uint32_t)(t >> 1) & 1u, err, 3)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = i0 + warp * 32 + lane;
      float2* Yk = b.Y + (long long)k * b.n * b.s;
      const uint32_t lane_base = tmem + set * Cfg::kTmemCols + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        float re[32], im[32];
        tmem_ld32(lane_base + c0, re);
        if (!real) {
          tmem_ld32(lane_base + BN + c0, im);
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c) im[c] = 0.f;
        }
        if (row < b.n) {
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int j = j0 + c0 + c;
            if (j < b.s) Yk[(long long)j * b.n + row] = make_float2(re[c], im[c]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_acce + 8 * set);
      ++t;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 5) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
}

// Planar copies of the FP32 spectra of a batch: per (instance, slice, 32 x 32 tile) work item,
// column-major planes [k][j][ldn] and row-major planes [k][i][lds] of Re and Im (TF32 or BF16), and
// with SPLIT the low parts v - tf32(v) of both.
template <typename OpT, bool SPLIT>
__global__ void __launch_bounds__(256) k_b_planes(const BTcPlanes* __restrict__ pl, const int* __restrict__ active,
                                                  const int4* __restrict__ items) {
  __shared__ float tr[32][33], ti[32][33];
  const int4 it = items[blockIdx.x];
  if (!active[it.x]) return;
  const BTcPlanes& P = pl[it.x];
  const int k = it.y, i0 = it.z, j0 = it.w;
  const float2* Xk = P.Xh + (long long)k * P.n * P.s;
  const long long oc = (long long)k * P.s * P.ldn, orow = (long long)k * P.n * P.lds;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {     // column j0 + q, rows i0 + tx
    const int i = i0 + threadIdx.x, j = j0 + q;
    float2 v = make_float2(0.f, 0.f);
    if (i < P.n && j < P.s) v = Xk[(long long)j * P.n + i];
    if (k == 0 || k == P.nyq) v.y = 0.f;
    tr[q][threadIdx.x] = v.x;
    ti[q][threadIdx.x] = v.y;
    if (i < P.n && j < P.s) {
      const long long o = oc + (long long)j * P.ldn + i;
      static_cast<OpT*>(P.xc_re)[o] = to_op<OpT>(v.x);
      static_cast<OpT*>(P.xc_im)[o] = to_op<OpT>(v.y);
      if (SPLIT) {
        static_cast<float*>(P.xc_re_lo)[o] = tf32_lo(v.x);
        static_cast<float*>(P.xc_im_lo)[o] = tf32_lo(v.y);
      }
    }
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {     // row i0 + q, columns j0 + tx
    const int i = i0 + q, j = j0 + threadIdx.x;
    if (i < P.n && j < P.s) {
      const long long o = orow + (long long)i * P.lds + j;
      const float vr = tr[threadIdx.x][q], vi = ti[threadIdx.x][q];
      static_cast<OpT*>(P.xr_re)[o] = to_op<OpT>(vr);
      static_cast<OpT*>(P.xr_im)[o] = to_op<OpT>(vi);
      if (SPLIT) {
        static_cast<float*>(P.xr_re_lo)[o] = tf32_lo(vr);
        static_cast<float*>(P.xr_im_lo)[o] = tf32_lo(vi);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Operand preparation
// ------------------------------------------------------------------------------------------------
// A_k (double2, column-major n x n) -> planes [k][i][ld] (row-major), via a 32 x 32 tile transpose.
// With lo planes given, re/im receive tf32(v) and re_lo/im_lo receive tf32(v - tf32(v)).
template <typename OpT>
__global__ void k_prep_A(const double2* __restrict__ Ah, OpT* __restrict__ re, OpT* __restrict__ im, int n, int ld,
                         float* __restrict__ re_lo, float* __restrict__ im_lo) {
  __shared__ float tr[32][33], ti[32][33];
  const int k = blockIdx.z;
  const int i0 = blockIdx.x * 32, l0 = blockIdx.y * 32;
  const double2* A = Ah + (long long)k * n * n;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {   // read column l0+q, rows i0 + tx
    const int i = i0 + threadIdx.x, l = l0 + q;
    double2 v = make_double2(0.0, 0.0);
    if (i < n && l < n) v = A[(long long)l * n + i];
    tr[q][threadIdx.x] = (float)v.x;
    ti[q][threadIdx.x] = (float)v.y;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {   // write row i0+q, columns l0 + tx
    const int i = i0 + q, l = l0 + threadIdx.x;
    if (i < n && l < ld) {
      const long long o = (long long)k * n * ld + (long long)i * ld + l;
      const float vr = l < n ? tr[threadIdx.x][q] : 0.f, vi = l < n ? ti[threadIdx.x][q] : 0.f;
      re[o] = to_op<OpT>(vr);
      im[o] = to_op<OpT>(vi);
      if (re_lo) {
        re_lo[o] = tf32_lo(vr);
        im_lo[o] = tf32_lo(vi);
      }
    }
  }
}

// B_k (double2, column-major s x s) -> planes [k][j][ld] (no transpose), negative-free.
template <typename OpT>
__global__ void k_prep_B(const double2* __restrict__ Bh, OpT* __restrict__ re, OpT* __restrict__ im, int s, int ld,
                         int K, float* __restrict__ re_lo, float* __restrict__ im_lo) {
  const long long total = (long long)K * s * ld;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(e % ld);
    const long long r = e / ld;
    const int j = (int)(r % s), k = (int)(r / s);
    double2 v = make_double2(0.0, 0.0);
    if (l < s) v = Bh[(long long)k * s * s + (long long)j * s + l];
    re[e] = to_op<OpT>((float)v.x);
    im[e] = to_op<OpT>((float)v.y);
    if (re_lo) {
      re_lo[e] = tf32_lo((float)v.x);
      im_lo[e] = tf32_lo((float)v.y);
    }
  }
}

// Planar DFT along mode 3 of an FP32 tensor: X (n x s x p) -> planes [k][j][ldn] (column-major X_k).
template <typename OpT, int PMAX>
__global__ void __launch_bounds__(256) k_rfft_planar(const float* __restrict__ X, OpT* __restrict__ re,
                                                     OpT* __restrict__ im, int n, int s, int p, int ldn,
                                                     float* __restrict__ re_lo, float* __restrict__ im_lo) {
  __shared__ float tc[PMAX], tsn[PMAX];
  for (int r = threadIdx.x; r < p; r += blockDim.x) {
    double sv, cv;
    sincospi(2.0 * r / p, &sv, &cv);
    tc[r] = (float)cv;
    tsn[r] = (float)sv;
  }
  __syncthreads();
  const int K = p / 2 + 1;
  const long long T = (long long)n * s;
  const long long Tp = (long long)ldn * s;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < Tp; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % ldn);
    const long long j = e / ldn;
    float x[PMAX];
#pragma unroll
    for (int t = 0; t < PMAX; ++t) x[t] = (t < p && i < n) ? X[t * T + j * n + i] : 0.f;
#pragma unroll 1
    for (int kk = 0; kk < K; ++kk) {
      float a = 0.f, b = 0.f;
      int r = 0;
#pragma unroll
      for (int t = 0; t < PMAX; ++t) {
        if (t < p) {
          a = fmaf(x[t], tc[r], a);
          b = fmaf(-x[t], tsn[r], b);
          r += kk;
          if (r >= p) r -= p;
        }
      }
      re[kk * Tp + e] = to_op<OpT>(a);
      im[kk * Tp + e] = to_op<OpT>(b);
      if (re_lo) {
        re_lo[kk * Tp + e] = tf32_lo(a);
        im_lo[kk * Tp + e] = tf32_lo(b);
      }
    }
  }
}

// planes [k][j][ldn] (column-major X_k) -> planes [k][i][lds] (row-major X_k).
// Power-of-two p: both planar layouts in one pass.  A CTA of 32 x 8 threads owns a tile of 32 rows
// (i) x TJ columns (j) of tubes (TJ = 32, or 16 with the split-TF32 low parts); each thread runs
// the register FFT of TJ / 8 tubes, writes the column-major planes [k][j][ldn] directly (coalesced
// along i) and keeps the tile in shared memory, from which the row-major planes [k][i][lds] are
// written coalesced along j.  Entries outside n x s are written as zeros in both layouts.  The
// separate transpose re-read the column-major planes from memory (a third of the traffic of the
// pair) and moved 64-byte rows.
template <typename OpT, int P, bool SPLIT>
__global__ void __launch_bounds__(256) k_rfft_planar_fused(const float* __restrict__ X, OpT* __restrict__ cre,
                                                           OpT* __restrict__ cim, OpT* __restrict__ rre,
                                                           OpT* __restrict__ rim, float* __restrict__ cre_lo,
                                                           float* __restrict__ cim_lo, float* __restrict__ rre_lo,
                                                           float* __restrict__ rim_lo, int n, int s, int ldn,
                                                           int lds) {
  constexpr int K = P / 2 + 1, TJ = SPLIT ? 16 : 32, NQ = TJ / 8;
  extern __shared__ uint8_t pf_smem[];
  OpT* tre = reinterpret_cast<OpT*>(pf_smem);             // [K][TJ][33]
  OpT* tim = tre + K * TJ * 33;
  float* tlr = reinterpret_cast<float*>(tim + K * TJ * 33);   // split: low parts, same shape
  float* tli = tlr + (SPLIT ? K * TJ * 33 : 0);
  __shared__ float tc[P], tsn[P];
  for (int r = threadIdx.y * 32 + threadIdx.x; r < P; r += 256) {
    double sv, cv;
    sincospi(2.0 * r / P, &sv, &cv);
    tc[r] = (float)cv;
    tsn[r] = (float)sv;
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * TJ;
  const long long T = (long long)n * s;
  const long long Tc = (long long)ldn * s, Tr = (long long)n * lds;
  const int i = i0 + tx;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int jj = ty + 8 * q, j = j0 + jj;
    const bool live = i < n && j < s;
    rfft_reg<float, P>([&](int t) { return live ? X[t * T + (long long)j * n + i] : 0.f; },
                       [&](int kk, float a, float b) {
                         const OpT ha = to_op<OpT>(a), hb = to_op<OpT>(b);
                         tre[(kk * TJ + jj) * 33 + tx] = ha;
                         tim[(kk * TJ + jj) * 33 + tx] = hb;
                         float la = 0.f, lb = 0.f;
                         if constexpr (SPLIT) {
                           la = tf32_lo(a);
                           lb = tf32_lo(b);
                           tlr[(kk * TJ + jj) * 33 + tx] = la;
                           tli[(kk * TJ + jj) * 33 + tx] = lb;
                         }
                         if (j < s && i < ldn) {
                           const long long o = kk * Tc + (long long)j * ldn + i;
                           cre[o] = ha;
                           cim[o] = hb;
                           if constexpr (SPLIT) {
                             cre_lo[o] = la;
                             cim_lo[o] = lb;
                           }
                         }
                       },
                       tc, tsn);
  }
  __syncthreads();
  // row-major planes: rows i0 + r (r < 32), columns j0 + c (c < TJ), all K slices
  for (int e = ty * 32 + tx; e < K * 32 * TJ; e += 256) {
    const int c = e % TJ, r = (e / TJ) % 32, kk = e / (TJ * 32);
    const int ir = i0 + r, jc = j0 + c;
    if (ir < n && jc < lds) {
      const long long o = kk * Tr + (long long)ir * lds + jc;
      rre[o] = tre[(kk * TJ + c) * 33 + r];
      rim[o] = tim[(kk * TJ + c) * 33 + r];
      if constexpr (SPLIT) {
        rre_lo[o] = tlr[(kk * TJ + c) * 33 + r];
        rim_lo[o] = tli[(kk * TJ + c) * 33 + r];
      }
    }
  }
}

template <typename OpT, int P, bool SPLIT>
constexpr int planar_fused_smem() {
  constexpr int K = P / 2 + 1, TJ = SPLIT ? 16 : 32;
  return K * TJ * 33 * (2 * (int)sizeof(OpT) + (SPLIT ? 8 : 0));
}

template <typename OpT>
__global__ void k_transpose_planes(const OpT* __restrict__ cre, const OpT* __restrict__ cim, OpT* __restrict__ rre,
                                   OpT* __restrict__ rim, int n, int s, int ldn, int lds) {
  __shared__ OpT tr[32][33], ti[32][33];
  const int k = blockIdx.z, i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const OpT* cr = cre + (long long)k * s * ldn;
  const OpT* ci = cim + (long long)k * s * ldn;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int j = j0 + q, i = i0 + threadIdx.x;
    OpT a = to_op<OpT>(0.f), b = to_op<OpT>(0.f);
    if (j < s && i < n) {
      a = cr[(long long)j * ldn + i];
      b = ci[(long long)j * ldn + i];
    }
    tr[q][threadIdx.x] = a;
    ti[q][threadIdx.x] = b;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int i = i0 + q, j = j0 + threadIdx.x;
    if (i < n && j < lds) {
      const long long o = (long long)k * n * lds + (long long)i * lds + j;
      rre[o] = j < s ? tr[threadIdx.x][q] : to_op<OpT>(0.f);
      rim[o] = j < s ? ti[threadIdx.x][q] : to_op<OpT>(0.f);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------------
inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

template <int BN, int ESZ, int PARTS>
void launch_tc(const TcMaps& maps, float2* Y, int n, int s, int K, int nyq, int* err, int stall,
               unsigned long long wait_ns, cudaStream_t st) {
  using Cfg = TcCfg<BN, ESZ>;
  set_max_dynamic_smem((const void*)k_tc_sylv<BN, ESZ, PARTS>, Cfg::kSmem);
  dim3 grid((s + BN - 1) / BN, (n + kTileM - 1) / kTileM, K);
  k_tc_sylv<BN, ESZ, PARTS><<<grid, 192, Cfg::kSmem, st>>>(maps, Y, n, s, nyq, err, stall, wait_ns);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename OpT>
void prepare_operator(ts_op* op, TcOperands& t, cudaStream_t st) {
  const int n = op->n, s = op->s, K = op->K;
  dim3 blk(32, 8);
  k_prep_A<OpT><<<dim3((n + 31) / 32, (t.ldn + 31) / 32, K), blk, 0, st>>>(
      op->Ah, (OpT*)t.a_re, (OpT*)t.a_im, n, t.ldn, (float*)t.a_re_lo, (float*)t.a_im_lo);
  count_launch();
  TS_CUDA(cudaGetLastError());
  const long long tot = (long long)K * s * t.lds;
  int g = (int)((tot + 255) / 256);
  if (g > 152 * 16) g = 152 * 16;
  k_prep_B<OpT><<<g, 256, 0, st>>>(op->Bh, (OpT*)t.b_re, (OpT*)t.b_im, s, t.lds, K, (float*)t.b_re_lo,
                                   (float*)t.b_im_lo);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename OpT, int P, bool SPLIT>
void planar_fused_p(const float* X, TcWork& w, int n, int s, int ldn, int lds, cudaStream_t st) {
  constexpr int smem = planar_fused_smem<OpT, P, SPLIT>(), TJ = SPLIT ? 16 : 32;
  set_max_dynamic_smem((const void*)k_rfft_planar_fused<OpT, P, SPLIT>, smem);
  const dim3 grid((unsigned)((std::max(n, ldn) + 31) / 32), (unsigned)((std::max(s, lds) + TJ - 1) / TJ), 1);
  k_rfft_planar_fused<OpT, P, SPLIT><<<grid, dim3(32, 8), smem, st>>>(
      X, (OpT*)w.xc_re, (OpT*)w.xc_im, (OpT*)w.xr_re, (OpT*)w.xr_im, (float*)w.xc_re_lo, (float*)w.xc_im_lo,
      (float*)w.xr_re_lo, (float*)w.xr_im_lo, n, s, ldn, lds);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <typename OpT, bool SPLIT>
void planar_fused(const float* X, TcWork& w, int n, int s, int p, int ldn, int lds, cudaStream_t st) {
  if (p == 2) planar_fused_p<OpT, 2, SPLIT>(X, w, n, s, ldn, lds, st);
  else if (p == 4) planar_fused_p<OpT, 4, SPLIT>(X, w, n, s, ldn, lds, st);
  else if (p == 8) planar_fused_p<OpT, 8, SPLIT>(X, w, n, s, ldn, lds, st);
  else if (p == 16) planar_fused_p<OpT, 16, SPLIT>(X, w, n, s, ldn, lds, st);
  else planar_fused_p<OpT, 32, SPLIT>(X, w, n, s, ldn, lds, st);
}

template <typename OpT>
void planar_dft(const float* X, TcWork& w, int n, int s, int p, int ldn, int lds, cudaStream_t st) {
  const long long Tp = (long long)ldn * s;
  int g = (int)((Tp + 255) / 256);
  if (g > 152 * 16) g = 152 * 16;
  OpT* cre = (OpT*)w.xc_re; OpT* cim = (OpT*)w.xc_im;
  float* lre = (float*)w.xc_re_lo; float* lim = (float*)w.xc_im_lo;
  if (p == 2 || p == 4 || p == 8 || p == 16 || p == 32) {   // both layouts in one pass
    if (lre) planar_fused<OpT, true>(X, w, n, s, p, ldn, lds, st);
    else planar_fused<OpT, false>(X, w, n, s, p, ldn, lds, st);
    return;
  }
  if (p <= 4) k_rfft_planar<OpT, 4><<<g, 256, 0, st>>>(X, cre, cim, n, s, p, ldn, lre, lim);
  else if (p <= 8) k_rfft_planar<OpT, 8><<<g, 256, 0, st>>>(X, cre, cim, n, s, p, ldn, lre, lim);
  else if (p <= 16) k_rfft_planar<OpT, 16><<<g, 256, 0, st>>>(X, cre, cim, n, s, p, ldn, lre, lim);
  else if (p <= 32) k_rfft_planar<OpT, 32><<<g, 256, 0, st>>>(X, cre, cim, n, s, p, ldn, lre, lim);
  else throw Error{TS_ERR_UNSUPPORTED, "tensor-core path supports p <= 32"};
  count_launch();
  TS_CUDA(cudaGetLastError());
  const int K = p / 2 + 1;
  const dim3 tg((n + 31) / 32, (lds + 31) / 32, K);
  k_transpose_planes<OpT><<<tg, dim3(32, 8), 0, st>>>(cre, cim, (OpT*)w.xr_re, (OpT*)w.xr_im, n, s, ldn, lds);
  count_launch();
  TS_CUDA(cudaGetLastError());
  if (lre) {
    k_transpose_planes<float><<<tg, dim3(32, 8), 0, st>>>(lre, lim, (float*)w.xr_re_lo, (float*)w.xr_im_lo, n, s,
                                                            ldn, lds);
    count_launch();
    TS_CUDA(cudaGetLastError());
  }
}

template <int PARTS>
void launch_by_bn(int esz, int bn, const TcMaps& maps, float2* Yh, int n, int s, int K, int nyq, int* err,
                  int stall, unsigned long long wait_ns, cudaStream_t st) {
  if (esz == 2) {
    if (bn == 64) launch_tc<64, 2, PARTS>(maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
    else if (bn == 128) launch_tc<128, 2, PARTS>(maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
    else launch_tc<256, 2, PARTS>(maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
  } else {
    if (bn == 64) launch_tc<64, 4, PARTS>(maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
    else if (bn == 128) launch_tc<128, 4, PARTS>(maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
    else launch_tc<256, 4, PARTS>(maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
  }
}

}  // namespace

namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw Error{TS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable"};
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 3-D map over planes [K][rows][ld] of ESZ-byte elements, box = (128 bytes of l) x box_rows x 1.
}  // namespace

void make_map(CUtensorMap* m, const void* base, int esz, int ld, int cols, int rows, int K, int box_rows) {
  TS_REQUIRE((reinterpret_cast<uintptr_t>(base) & 15) == 0, "TMA base must be 16-byte aligned");
  TS_REQUIRE(((long long)ld * esz) % 16 == 0, "TMA row pitch must be a multiple of 16 bytes");
  const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)K};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * esz, (cuuint64_t)ld * esz * rows};
  const cuuint32_t box[3] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = encode_fn()(m, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{TS_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r)};
}


// Build (once per operator and precision) the tensor-core operand planes of A_k and B_k.
void tc_prepare(ts_op* op, int precision, cudaStream_t st) {
  if (op->tc_prec == precision && op->tc) return;
  const int esz = precision == TS_MIXED_BF16 ? 2 : 4;
  const bool split = precision == TS_MIXED_TF32X3;
  TcOperands* t = op->tc ? op->tc : new TcOperands();
  op->tc = t;
  t->release();
  t->esz = esz;
  t->split = split;
  t->ldn = round_up(op->n, 64);
  t->lds = round_up(op->s, 64);
  const size_t na = (size_t)op->K * op->n * t->ldn * esz, nb = (size_t)op->K * op->s * t->lds * esz;
  op_alloc_on(t->a_re, na, st);
  op_alloc_on(t->a_im, na, st);
  op_alloc_on(t->b_re, nb, st);
  op_alloc_on(t->b_im, nb, st);
  if (split) {
    op_alloc_on(t->a_re_lo, na, st);
    op_alloc_on(t->a_im_lo, na, st);
    op_alloc_on(t->b_re_lo, nb, st);
    op_alloc_on(t->b_im_lo, nb, st);
  }
  if (esz == 2) prepare_operator<__nv_bfloat16>(op, *t, st);
  else prepare_operator<float>(op, *t, st);
  op->tc_prec = precision;
}

void tc_apply(ts_ctx* ctx, ts_op* op, int precision, const float* X, float2* Yh, cudaStream_t st) {
  tc_prepare(op, precision, st);
  TcOperands& t = *op->tc;
  const int n = op->n, s = op->s, p = op->p, K = op->K, esz = t.esz;
  TcWork w;
  const size_t nx = (size_t)K * s * t.ldn * esz, nr = (size_t)K * n * t.lds * esz;
  w.xc_re = ctx->ws.get("tc_xc_re", nx);
  w.xc_im = ctx->ws.get("tc_xc_im", nx);
  w.xr_re = ctx->ws.get("tc_xr_re", nr);
  w.xr_im = ctx->ws.get("tc_xr_im", nr);
  if (t.split) {
    w.xc_re_lo = ctx->ws.get("tc_xc_re_lo", nx);
    w.xc_im_lo = ctx->ws.get("tc_xc_im_lo", nx);
    w.xr_re_lo = ctx->ws.get("tc_xr_re_lo", nr);
    w.xr_im_lo = ctx->ws.get("tc_xr_im_lo", nr);
  }
  int* err = static_cast<int*>(ctx->ws.get("tc_err", sizeof(int) * 4));
  KernelTimer& tm = ctx->timer;
  tm.begin(st, 1, 4.0 * n * s * p + 2.0 * K * n * s * esz * 2 * (t.split ? 2 : 1));
  if (esz == 2) planar_dft<__nv_bfloat16>(X, w, n, s, p, t.ldn, t.lds, st);
  else planar_dft<float>(X, w, n, s, p, t.ldn, t.lds, st);
  tm.end(st);
  // The column tile BN (64, 128 or 256 output columns per CTA; tiles more than twice s are not
  // tried) is chosen by the autotuner on the first application of this shape and precision.  The
  // accumulation order of every output entry does not depend on BN, so neither does the result.
  auto build = [&](int bn) {
    TcMaps maps;
    make_map(&maps.a_re, t.a_re, esz, t.ldn, n, n, K, kTileM);
    make_map(&maps.a_im, t.a_im, esz, t.ldn, n, n, K, kTileM);
    make_map(&maps.xc_re, w.xc_re, esz, t.ldn, n, s, K, bn);
    make_map(&maps.xc_im, w.xc_im, esz, t.ldn, n, s, K, bn);
    make_map(&maps.xr_re, w.xr_re, esz, t.lds, s, n, K, kTileM);
    make_map(&maps.xr_im, w.xr_im, esz, t.lds, s, n, K, kTileM);
    make_map(&maps.b_re, t.b_re, esz, t.lds, s, s, K, bn);
    make_map(&maps.b_im, t.b_im, esz, t.lds, s, s, K, bn);
    if (t.split) {
      make_map(&maps.a_re_lo, t.a_re_lo, esz, t.ldn, n, n, K, kTileM);
      make_map(&maps.a_im_lo, t.a_im_lo, esz, t.ldn, n, n, K, kTileM);
      make_map(&maps.xc_re_lo, w.xc_re_lo, esz, t.ldn, n, s, K, bn);
      make_map(&maps.xc_im_lo, w.xc_im_lo, esz, t.ldn, n, s, K, bn);
      make_map(&maps.xr_re_lo, w.xr_re_lo, esz, t.lds, s, n, K, kTileM);
      make_map(&maps.xr_im_lo, w.xr_im_lo, esz, t.lds, s, n, K, kTileM);
      make_map(&maps.b_re_lo, t.b_re_lo, esz, t.lds, s, s, K, bn);
      make_map(&maps.b_im_lo, t.b_im_lo, esz, t.lds, s, s, K, bn);
    } else {
      maps.a_re_lo = maps.a_re; maps.a_im_lo = maps.a_im; maps.xc_re_lo = maps.xc_re; maps.xc_im_lo = maps.xc_im;
      maps.xr_re_lo = maps.xr_re; maps.xr_im_lo = maps.xr_im; maps.b_re_lo = maps.b_re; maps.b_im_lo = maps.b_im;
    }
    return maps;
  };
  const int nyq = nyquist_index(p);
  // Test aid for the failure path: with TSTAR_TEST_STALL_TMA=1 in the environment the TMA producer
  // arms no stage, so the MMA warp's bounded wait expires (after 50 ms instead of the usual limit),
  // the kernel records the error, frees its tensor memory and returns; the caller then sees
  // TS_ERR_TIMEOUT.  Read on every application, so a test can turn it on and off around one call.
  const char* stall_env = std::getenv("TSTAR_TEST_STALL_TMA");
  const int stall = stall_env && stall_env[0] == '1';
  const unsigned long long wait_ns = stall ? 50000000ull : kWaitNs;
  auto run = [&](int bn) {
    const TcMaps maps = build(bn);
    if (t.split) launch_by_bn<3>(esz, bn, maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
    else launch_by_bn<1>(esz, bn, maps, Yh, n, s, K, nyq, err, stall, wait_ns, st);
  };
  std::vector<int> cands;
  for (int c : {64, 128, 256})
    if (c == 64 || c / 2 < s) cands.push_back(c);
  const std::string key = "tc:" + std::to_string(n) + "x" + std::to_string(s) + "x" + std::to_string(K) + ":" +
                          std::to_string(precision);
  const int bn = tune_pick(ctx, key, cands, run, st);
  tm.begin(st, 2, gemm_flops_tc(n, s, K, nyq));
  run(bn);
  tm.end(st);
}

// ------------------------------------------------------------------------------------------------
// Batched tensor-core products (host side)
// ------------------------------------------------------------------------------------------------
namespace {
inline size_t align256(size_t b) { return (b + 255) / 256 * 256; }

template <typename OpT, int ESZ, int PARTS, bool SPLIT, int BN>
void batch_preload_bn() {
  using Cfg = TcCfg<BN, ESZ>;
  cudaFuncAttributes fa;
  TS_CUDA(cudaFuncGetAttributes(&fa, (const void*)k_b_tc<BN, ESZ, PARTS>));
  set_max_dynamic_smem((const void*)k_b_tc<BN, ESZ, PARTS>, Cfg::kSmem);
  TS_CUDA(cudaFuncGetAttributes(&fa, (const void*)k_b_tc_persist<BN, ESZ, PARTS>));
  set_max_dynamic_smem((const void*)k_b_tc_persist<BN, ESZ, PARTS>, Cfg::kSmem);
}

int device_sms() {
  static int cached[64] = {0};
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return 152;
  if (!cached[dev]) TS_CUDA(cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev));
  return cached[dev];
}

template <typename OpT, int ESZ, int PARTS, bool SPLIT>
void batch_preload_t() {
  cudaFuncAttributes fa;
  TS_CUDA(cudaFuncGetAttributes(&fa, (const void*)k_b_planes<OpT, SPLIT>));
  batch_preload_bn<OpT, ESZ, PARTS, SPLIT, 64>();
  batch_preload_bn<OpT, ESZ, PARTS, SPLIT, 128>();
}

template <typename OpT, int ESZ, int PARTS, bool SPLIT>
void batch_products_t(int sched, const BTcPlanes* planes, const int4* pitems, int npitems, const TcMaps* maps,
                      const BTcInst* inst, const int* active, const int4* items, int nitems, int* err,
                      cudaStream_t st) {
  k_b_planes<OpT, SPLIT><<<npitems, dim3(32, 8), 0, st>>>(planes, active, pitems);
  count_launch();
  TS_CUDA(cudaGetLastError());
  const int bn = tc_batch_bn(sched);
  if (tc_batch_persistent(sched)) {
    const int grid = std::min(nitems, device_sms());
    if (bn == 128)
      k_b_tc_persist<128, ESZ, PARTS><<<grid, 192, TcCfg<128, ESZ>::kSmem, st>>>(maps, inst, active, items, nitems,
                                                                                err);
    else
      k_b_tc_persist<64, ESZ, PARTS><<<grid, 192, TcCfg<64, ESZ>::kSmem, st>>>(maps, inst, active, items, nitems,
                                                                              err);
  } else if (bn == 128) {
    k_b_tc<128, ESZ, PARTS><<<nitems, 192, TcCfg<128, ESZ>::kSmem, st>>>(maps, inst, active, items, err);
  } else {
    k_b_tc<64, ESZ, PARTS><<<nitems, 192, TcCfg<64, ESZ>::kSmem, st>>>(maps, inst, active, items, err);
  }
  count_launch();
  TS_CUDA(cudaGetLastError());
}
}  // namespace

size_t tc_batch_plane_bytes(int n, int s, int K, int precision) {
  const int esz = precision == TS_MIXED_BF16 ? 2 : 4;
  const bool split = precision == TS_MIXED_TF32X3;
  const size_t nx = align256((size_t)K * s * round_up(n, 64) * esz);
  const size_t nr = align256((size_t)K * n * round_up(s, 64) * esz);
  return (split ? 4 : 2) * (nx + nr);
}

void tc_batch_instance(ts_op* op, int precision, const float2* Xh, void* base, BTcPlanes* pl, TcMaps* maps, int bn) {
  TS_REQUIRE(op->tc && op->tc_prec == precision, "tc_batch_instance: operator planes not prepared");
  const TcOperands& t = *op->tc;
  const int n = op->n, s = op->s, K = op->K, esz = t.esz;
  const size_t nx = align256((size_t)K * s * t.ldn * esz), nr = align256((size_t)K * n * t.lds * esz);
  char* b = static_cast<char*>(base);
  *pl = BTcPlanes{};
  pl->Xh = Xh;
  pl->xc_re = b; b += nx;
  pl->xc_im = b; b += nx;
  pl->xr_re = b; b += nr;
  pl->xr_im = b; b += nr;
  if (t.split) {
    pl->xc_re_lo = b; b += nx;
    pl->xc_im_lo = b; b += nx;
    pl->xr_re_lo = b; b += nr;
    pl->xr_im_lo = b; b += nr;
  }
  pl->n = n; pl->s = s; pl->ldn = t.ldn; pl->lds = t.lds; pl->nyq = nyquist_index(op->p);
  make_map(&maps->a_re, t.a_re, esz, t.ldn, n, n, K, kTileM);
  make_map(&maps->a_im, t.a_im, esz, t.ldn, n, n, K, kTileM);
  make_map(&maps->xc_re, pl->xc_re, esz, t.ldn, n, s, K, bn);
  make_map(&maps->xc_im, pl->xc_im, esz, t.ldn, n, s, K, bn);
  make_map(&maps->xr_re, pl->xr_re, esz, t.lds, s, n, K, kTileM);
  make_map(&maps->xr_im, pl->xr_im, esz, t.lds, s, n, K, kTileM);
  make_map(&maps->b_re, t.b_re, esz, t.lds, s, s, K, bn);
  make_map(&maps->b_im, t.b_im, esz, t.lds, s, s, K, bn);
  if (t.split) {
    make_map(&maps->a_re_lo, t.a_re_lo, esz, t.ldn, n, n, K, kTileM);
    make_map(&maps->a_im_lo, t.a_im_lo, esz, t.ldn, n, n, K, kTileM);
    make_map(&maps->xc_re_lo, pl->xc_re_lo, esz, t.ldn, n, s, K, bn);
    make_map(&maps->xc_im_lo, pl->xc_im_lo, esz, t.ldn, n, s, K, bn);
    make_map(&maps->xr_re_lo, pl->xr_re_lo, esz, t.lds, s, n, K, kTileM);
    make_map(&maps->xr_im_lo, pl->xr_im_lo, esz, t.lds, s, n, K, kTileM);
    make_map(&maps->b_re_lo, t.b_re_lo, esz, t.lds, s, s, K, bn);
    make_map(&maps->b_im_lo, t.b_im_lo, esz, t.lds, s, s, K, bn);
  } else {
    maps->a_re_lo = maps->a_re; maps->a_im_lo = maps->a_im; maps->xc_re_lo = maps->xc_re;
    maps->xc_im_lo = maps->xc_im; maps->xr_re_lo = maps->xr_re; maps->xr_im_lo = maps->xr_im;
    maps->b_re_lo = maps->b_re; maps->b_im_lo = maps->b_im;
  }
}

void tc_batch_preload(int precision) {
  if (precision == TS_MIXED_BF16) batch_preload_t<__nv_bfloat16, 2, 1, false>();
  else if (precision == TS_MIXED_TF32) batch_preload_t<float, 4, 1, false>();
  else batch_preload_t<float, 4, 3, true>();
}

void tc_batch_products(int precision, int sched, const BTcPlanes* planes, const int4* pitems, int npitems,
                       const TcMaps* maps, const BTcInst* inst, const int* active, const int4* items, int nitems,
                       int* err, cudaStream_t st) {
  TS_REQUIRE(nitems > 0 && npitems > 0, "tc_batch_products: empty work list");
  if (precision == TS_MIXED_BF16)
    batch_products_t<__nv_bfloat16, 2, 1, false>(sched, planes, pitems, npitems, maps, inst, active, items, nitems,
                                                 err, st);
  else if (precision == TS_MIXED_TF32)
    batch_products_t<float, 4, 1, false>(sched, planes, pitems, npitems, maps, inst, active, items, nitems, err, st);
  else
    batch_products_t<float, 4, 3, true>(sched, planes, pitems, npitems, maps, inst, active, items, nitems, err, st);
}

double gemm_flops_tc(int n, int s, int K, int nyq) {
  const int nreal = 1 + (nyq >= 0 ? 1 : 0);
  const double per = (double)n * s * ((double)n + s);
  return per * (8.0 * (K - nreal) + 2.0 * nreal);
}

void TcOperands::release() {
  op_free(a_re);
  op_free(a_im);
  op_free(b_re);
  op_free(b_im);
  op_free(a_re_lo);
  op_free(a_im_lo);
  op_free(b_re_lo);
  op_free(b_im_lo);
  a_re = a_im = b_re = b_im = nullptr;
  a_re_lo = a_im_lo = b_re_lo = b_im_lo = nullptr;
}

}  // namespace ts
