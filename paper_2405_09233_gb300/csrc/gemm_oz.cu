// Emulated FP64 per-slice products on the tcgen05 tensor cores (Ozaki scheme):
//     Y_k = A_k X_k - X_k B_k      (Eq. (2) in the Fourier domain, Algorithm 1 step 2)
// from FP64 inputs, with a result at the accuracy level of an FP64 product, computed from BF16
// products that the tensor cores form and sum without rounding.  GB300 issues FP64 at ~1.26
// TFLOP/s but BF16 at ~2 PFLOP/s, so the ~21 digit-pair products cost far less than one DFMA GEMM.
//
// Method: Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix multiplication by
// using fast routines of matrix multiplication and its applications", Numer. Algorithms 59 (2012),
// arranged for tensor memory:
//  * Every FP64 slice Z (A_k and B_k share one exponent E_op[k]; X_k has E_x[k], both with
//    max |Re|, |Im| < 2^(E-1)) is written as Z = 2^E sum_{t=1..S} d_t 256^-t + r, |r| <= 2^E 256^-S / 2,
//    with integer digits |d_t| <= 128: the balanced base-256 expansion of round(Z 2^(8S-E)), taken
//    with integer arithmetic from the FP64 bit pattern.  Such digits are exact in BF16.
//  * A digit product is an integer of magnitude <= 2^14.  One accumulator run adds at most 2 x 512
//    of them into a TMEM FP32 accumulator (Re gets Ar Xr and -Ai Xi over 512 reduction indices);
//    every partial sum is an integer below 2^24, so the tensor core sums them exactly.
//  * Digit pairs (u, v) with u + v = g share the scale 2^(E_op + E_x - 8g); the pairs with
//    g <= S + 1 are kept (the dropped ones are below the truncation error of the digits).  Each
//    accumulator run ("unit": up to 8 k-blocks of 64 of one digit pair) is read from TMEM, converted to
//    int32 and added into per-thread int64 accumulators at the common fixed point
//    2^(E_op + E_x - F), F = 63 - ceil(log2(2 (n + s))), which keeps every partial sum below 2^62.
//    Units with 8g > F are added with a rounded right shift.
//  * Y = double(acc) 2^(E_op + E_x - F): one rounding.
//
// One CTA computes a 128 x 64 output tile of one slice; each MMA (N = 128) produces its Re and Im
// columns together from a B operand stored as three 64-row blocks (see the MMA warp).  Warp roles
// (320 threads):
//   warps 0-7  epilogue: warp w reads TMEM lanes 32 (w mod 4) .. +31 (output rows) and columns
//              32 (w div 4) .. +31 of the tile; holds 2 x 32 int64 accumulators per thread
//   warp 8     TMA producer (A-operand Re/Im tiles 128 x 64, three B-operand blocks 64 x 64)
//   warp 9     TMEM allocator and MMA issuer (one elected lane)
// Two TMEM accumulator buffers (Re 64 + Im 64 columns each) alternate between units, so the MMAs
// of one unit overlap the epilogue of the previous one.  Every wait is bounded.
#include <cuda_bf16.h>
#include <climits>
#include <cfloat>
#include "internal.cuh"
#include "apply.cuh"
#include "tcgen05.cuh"
#include "oz.cuh"

namespace ts {
namespace {
using namespace tcg;

constexpr int kOzM = 128;                               // tile rows (TMEM lanes)
constexpr int kOzN = 64;                                // tile columns
constexpr int kOzKB = 64;                               // k-block: BF16 elements per 128-byte row
constexpr int kOzStages = 4;
constexpr int kOzTileA = kOzM * 128;                    // bytes of one A-operand plane tile
constexpr int kOzTileB = kOzN * 128;                    // bytes of one 64-row B-operand block
constexpr int kOzStage = 2 * kOzTileA + 3 * kOzTileB;   // A Re, A Im; B blocks [P; Q; R]
constexpr int kOzSmem = kOzStages * kOzStage + 1024 + 256;
constexpr int kOzUnitBlocks = 8;                        // k-blocks per exact accumulator run
constexpr int kOzTmemCols = 256;                        // 2 buffers x (Re 64 + Im 64)
constexpr int kOzThreads = 320;
constexpr int kOzBadExp = INT_MAX;                      // slice with a non-finite entry

struct OzMaps {
  CUtensorMap a_re, a_im;     // A digits  [S*K][n][ldn]  row-major A_k         (A operand of A X)
  CUtensorMap xc_re, xc_im;   // X digits  [S*K][s][ldn]  column-major X_k      (B operand of A X)
  CUtensorMap xc_nim;         //   and the digits of -Im X_k
  CUtensorMap xr_re, xr_im;   // X digits  [S*K][n][lds]  row-major X_k         (A operand of X B)
  CUtensorMap b_re, b_im;     // B digits  [S*K][s][lds]  column-major B_k      (B operand of X B)
  CUtensorMap b_nre;          //   and the digits of -Re B_k
};

// The work of one tile as a list of units, each an exact accumulator run over at most
// kOzUnitBlocks k-blocks of one digit pair: the A X part, then the X B part; within a part, for
// each chunk of kOzUnitBlocks k-blocks, every kept digit pair (u, v), u + v <= S + 1, in the order
// (1,1) .. (1,S), (2,1) .. (2,S-1), ...  Consecutive units therefore reuse one chunk of every
// operand, which keeps the operands in flight across the grid small enough for L2.
struct OzSeq {
  int S, kbA, kbB;
  __device__ __forceinline__ int npairs() const { return S * (S + 1) / 2; }
  __device__ __forceinline__ int chunks(int kb) const { return (kb + kOzUnitBlocks - 1) / kOzUnitBlocks; }
  __device__ __forceinline__ int units() const { return npairs() * (chunks(kbA) + chunks(kbB)); }
  // Unit q -> (A X or X B, digit u of the A operand, digit v of the B operand, first k-block, count).
  __device__ __forceinline__ void unit(int q, bool& ax, int& u, int& v, int& lb0, int& nb) const {
    const int P = npairs(), qa = P * chunks(kbA);
    ax = q < qa;
    const int r = ax ? q : q - qa;
    int p = r % P;
    u = 1;
    while (u < S && p >= S + 1 - u) {
      p -= S + 1 - u;
      ++u;
    }
    v = p + 1;
    const int kb = ax ? kbA : kbB;
    lb0 = (r / P) * kOzUnitBlocks;
    nb = kb - lb0 < kOzUnitBlocks ? kb - lb0 : kOzUnitBlocks;
  }
};

// 16 consecutive TMEM columns of this warp's 32 lanes (one value per column per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// acc[c0 + c] += value of TMEM column (taddr + c) at the fixed point: shifted left by `shift`, or
// right with rounding when shift < 0.  The FP32 values are integers below 2^24 in magnitude.
template <int C0>
__device__ __forceinline__ void acc_add16(long long (&acc)[32], uint32_t taddr, int shift) {
  uint32_t r[16];
  tmem_ld16(taddr, r);
  if (shift >= 0) {
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[C0 + c] += (long long)__float2int_rn(__uint_as_float(r[c])) << shift;
  } else {
    const int rs = -shift;
    const long long half = 1ll << (rs - 1);
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[C0 + c] += ((long long)__float2int_rn(__uint_as_float(r[c])) + half) >> rs;
  }
}

__global__ void __launch_bounds__(kOzThreads, 1)
    k_oz_sylv(const __grid_constant__ OzMaps maps, double2* __restrict__ Y, int n, int s, int K, int nyq, int S,
              int F, const int* __restrict__ Eop, const int* __restrict__ Ex, const int* __restrict__ gate, int* err) {
  if (gate && *gate == 0) return;   // instance of a batch that has left the current cycle
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* smem = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kOzStages * kOzStage);
  // bars: full[kOzStages], empty[kOzStages], acc[2], free[2], done; then the TMEM address slot
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kOzStages + 5);
  const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + kOzStages);
  const uint32_t bar_acc = smem_u32(bars + 2 * kOzStages), bar_free = smem_u32(bars + 2 * kOzStages + 2);
  const uint32_t bar_done = smem_u32(bars + 2 * kOzStages + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.x * kOzN, i0 = blockIdx.y * kOzM, k = blockIdx.z;
  const bool real = (k == 0) || (k == nyq);
  const OzSeq seq{S, (n + kOzKB - 1) / kOzKB, (s + kOzKB - 1) / kOzKB};

  if (threadIdx.x == 0) {
    for (int q = 0; q < kOzStages; ++q) {
      mbar_init(bar_full + 8 * q, 1);
      mbar_init(bar_empty + 8 * q, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_acc + 8 * b, 1);
      mbar_init(bar_free + 8 * b, 8);   // one arrival per epilogue warp
    }
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kOzTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 8) {
    if (lane == 0) {
      int it = 0, issued = 0;   // stages visited / stages whose loads were issued
      bool ok = true;
      const int U = seq.units();
      for (int q = 0; q < U && ok; ++q) {
        bool ax;
        int u, v, lb0, nb;
        seq.unit(q, ax, u, v, lb0, nb);
        const int pa = (u - 1) * K + k, pb = (v - 1) * K + k;
        for (int t = 0; t < nb; ++t, ++it) {
          const int slot = it % kOzStages;
          const uint32_t phase = (uint32_t)(it / kOzStages) & 1u;
          if (!mbar_wait(bar_empty + 8 * slot, phase ^ 1u, err, 11)) {
            ok = false;
            break;
          }
          const uint32_t full = bar_full + 8 * slot;
          // a real slice (k = 0 or p/2) uses the real A tile and one B block (Q = Xr, or P = Br) only
          mbar_expect_tx(full, real ? kOzTileA + kOzTileB : kOzStage);
          const uint32_t sA = base + slot * kOzStage;
          const uint32_t sAi = sA + kOzTileA, sP = sA + 2 * kOzTileA, sQ = sP + kOzTileB, sR = sQ + kOzTileB;
          const int l0 = (lb0 + t) * kOzKB;
          if (ax) {
            tma_load_3d(sA, &maps.a_re, l0, i0, pa, full);
            tma_load_3d(sQ, &maps.xc_re, l0, j0, pb, full);    // [P; Q; R] = [-Xi; Xr; Xi]
            if (!real) {
              tma_load_3d(sAi, &maps.a_im, l0, i0, pa, full);
              tma_load_3d(sP, &maps.xc_nim, l0, j0, pb, full);
              tma_load_3d(sR, &maps.xc_im, l0, j0, pb, full);
            }
          } else {
            tma_load_3d(sA, &maps.xr_re, l0, i0, pa, full);
            tma_load_3d(sP, &maps.b_re, l0, j0, pb, full);     // [P; Q; R] = [Br; Bi; -Br]
            if (!real) {
              tma_load_3d(sAi, &maps.xr_im, l0, i0, pa, full);
              tma_load_3d(sQ, &maps.b_im, l0, j0, pb, full);
              tma_load_3d(sR, &maps.b_nre, l0, j0, pb, full);
            }
          }
          issued = it + 1;
        }
      }
      // Every stage this warp loaded lands before the CTA exits, also when an error stopped the MMA
      // warp from consuming it: bounded waits on the last kOzStages loads (immediate when all were used).
      for (int i = issued > kOzStages ? issued - kOzStages : 0; i < issued; ++i)
        mbar_wait(bar_full + 8 * (i % kOzStages), (uint32_t)(i / kOzStages) & 1u, err, 15);
    }
  } else if (warp == 9) {
    if (lane == 0) {
      // One accumulator covers [Re | Im] (N = 128): with the B blocks [P; Q; R] of a stage,
      //   A X:  D += Ar [Xr | Xi] + Ai [-Xi | Xr]        (blocks Q-R, then P-Q)
      //   X B:  D += -Xr [Br | Bi] + Xi [Bi | -Br]       (blocks P-Q, then Q-R)
      // Real slices use the Re half only (N = 64).
      constexpr uint32_t idp = make_idesc(1, kOzM, 2 * kOzN, false);
      constexpr uint32_t idn = make_idesc(1, kOzM, 2 * kOzN, true);
      constexpr uint32_t idp1 = make_idesc(1, kOzM, kOzN, false);
      constexpr uint32_t idn1 = make_idesc(1, kOzM, kOzN, true);
      int it = 0;
      bool ok = true;
      const int U = seq.units();
      for (int q = 0; q < U && ok; ++q) {
        bool ax;
        int u, v, lb0, nb;
        seq.unit(q, ax, u, v, lb0, nb);
        const int b = q & 1;
        if (q >= 2 && !mbar_wait(bar_free + 8 * b, (uint32_t)((q >> 1) - 1) & 1u, err, 12)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * 2 * kOzN);
        for (int t = 0; t < nb; ++t, ++it) {
          const int slot = it % kOzStages;
          const uint32_t phase = (uint32_t)(it / kOzStages) & 1u;
          if (!mbar_wait(bar_full + 8 * slot, phase, err, 13)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sA = base + slot * kOzStage;
          const uint64_t dAr = smem_desc_sw128(sA), dAi = smem_desc_sw128(sA + kOzTileA);
          const uint64_t dP = smem_desc_sw128(sA + 2 * kOzTileA);
          const uint64_t dQ = smem_desc_sw128(sA + 2 * kOzTileA + kOzTileB);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t o = (uint64_t)(kk * 2);   // 32 bytes >> 4
            const uint32_t acc = (t == 0 && kk == 0) ? 0u : 1u;
            if (ax) {
              if (real) {
                mma_issue(d, dAr + o, dQ + o, idp1, acc, 0);
              } else {
                mma_issue(d, dAr + o, dQ + o, idp, acc, 0);
                mma_issue(d, dAi + o, dP + o, idp, 1u, 0);
              }
            } else {
              if (real) {
                mma_issue(d, dAr + o, dP + o, idn1, acc, 0);
              } else {
                mma_issue(d, dAr + o, dP + o, idn, acc, 0);
                mma_issue(d, dAi + o, dQ + o, idp, 1u, 0);
              }
            }
          }
          mma_commit(bar_empty + 8 * slot);
        }
        if (ok) mma_commit(bar_acc + 8 * b);
      }
      if (!ok) {   // after an error the MMAs already issued still complete before TMEM is freed
        mma_commit(bar_done);
        mbar_wait(bar_done, 0u, err, 16);
      }
    }
  } else {
    // Epilogue: rows i0 + 32 (warp mod 4) + lane, columns j0 + 32 (warp div 4) + c.
    const int quad = warp & 3, half = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 32);
    long long ar[32], ai[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) ar[c] = ai[c] = 0;
    bool ok = true;
    const int U = seq.units();
    for (int q = 0; q < U; ++q) {
      bool ax;
      int u, v, lb0, nb;
      seq.unit(q, ax, u, v, lb0, nb);
      const int shift = F - 8 * (u + v);
      const int b = q & 1;
      if (!mbar_wait(bar_acc + 8 * b, (uint32_t)(q >> 1) & 1u, err, 14)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t tre = lane_base + (uint32_t)(b * 2 * kOzN);
      acc_add16<0>(ar, tre, shift);
      acc_add16<16>(ar, tre + 16, shift);
      if (!real) {
        acc_add16<0>(ai, tre + kOzN, shift);
        acc_add16<16>(ai, tre + kOzN + 16, shift);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_free + 8 * b);
    }
    const int row = i0 + quad * 32 + lane;
    if (ok && row < n) {
      const int ea = Eop[k], ex = Ex[k];
      const bool bad = ea == kOzBadExp || ex == kOzBadExp;
      const double scale = bad ? __longlong_as_double(0x7ff8000000000000ll) : ldexp(1.0, ea + ex - F);
      const long long T = (long long)n * s;
      double2* Yk = Y + (long long)k * T;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int j = j0 + half * 32 + c;
        if (j < s) {
          double2 y;
          y.x = (double)ar[c] * scale;
          y.y = real ? (bad ? scale : 0.0) : (double)ai[c] * scale;
          Yk[(long long)j * n + row] = y;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 9) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kOzTmemCols));
  }
}

// ------------------------------------------------------------------------------------------------
// Exponents and digits
// ------------------------------------------------------------------------------------------------
// Per-slice max(|Re|, |Im|) of K complex slices of T entries, as FP64 bit patterns (monotone for
// non-negative values) combined with atomicMax; a non-finite entry makes the slice's value +inf.
__global__ void k_oz_maxabs(const double2* __restrict__ Z, long long T, unsigned long long* __restrict__ out,
                            const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  const int k = blockIdx.y;
  const double2* Zk = Z + (long long)k * T;
  // Non-negative doubles order like their bit patterns read as unsigned integers (and every
  // non-finite pattern lies above that of +Inf), so the maximum is taken on integer ALUs: FP64
  // compares would make this pass FP64-pipe bound on GB300.
  constexpr unsigned long long kAbs = 0x7FFFFFFFFFFFFFFFull, kInf = 0x7FF0000000000000ull;
  unsigned long long m = 0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < T; e += (long long)gridDim.x * blockDim.x) {
    const double2 v = Zk[e];
    const unsigned long long a = (unsigned long long)__double_as_longlong(v.x) & kAbs;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v.y) & kAbs;
    m = max(m, max(a, b));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ unsigned long long wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = max(t, wm[w]);
    atomicMax(out + k, t >= kInf ? kInf : t);   // any non-finite entry reads as +Inf
  }
}

// E[k] with max|slice k| < 2^(E-1): ilogb(max) + 2 (0 for an all-zero slice, kOzBadExp if not finite).
__global__ void k_oz_exponents(const unsigned long long* __restrict__ mx, int K, int* __restrict__ E) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double m = __longlong_as_double((long long)mx[k]);
  E[k] = !(m <= DBL_MAX) ? kOzBadExp : (m == 0.0 ? 0 : ilogb(m) + 2);
}

// round(v 2^(8S - E)) as an integer from the FP64 bit pattern (|v| < 2^(E-1), so |q| < 2^(8S-1)).
__device__ __forceinline__ long long oz_fixed(double v, int E, int S) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long m = (long long)(bits & 0xFFFFFFFFFFFFFull);
  int e2;
  if (ex == 0) {
    e2 = 1 - 1075;            // subnormal: no implicit bit
  } else {
    m |= 1ll << 52;
    e2 = ex - 1075;
  }
  const int sh = e2 + 8 * S - E;
  long long q;
  if (m == 0 || sh <= -54) q = 0;
  else if (sh >= 0) q = m << sh;
  else q = (m + (1ll << (-sh - 1))) >> (-sh);
  return (bits >> 63) ? -q : q;
}

// Digit planes of K complex slices.  Slice k of src is a column-major R x C matrix (entry (r, c) at
// src[k*sstride + c*R + r]).  TRANS = false: output rows c, contiguous index r; TRANS = true: output
// rows r, contiguous index c.  Digit t (0 = most significant) of slice k lands in plane t*K + k of
// plane_elems entries with row pitch ld.  nre / nim (optional) receive the digits of -Re / -Im.
// Entries beyond R or C are not written (the tensor maps read them as zero).
template <bool TRANS>
__global__ void k_oz_split(const double2* __restrict__ src, long long sstride, int R, int C, int K,
                           const int* __restrict__ E, int S, __nv_bfloat16* __restrict__ re,
                           __nv_bfloat16* __restrict__ im, __nv_bfloat16* __restrict__ nre,
                           __nv_bfloat16* __restrict__ nim, int ld, long long plane_elems, const int* __restrict__ gate) {
  if (gate && *gate == 0) return;
  __shared__ double2 tile[32][33];
  const int k = blockIdx.z, r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const double2* Sk = src + (long long)k * sstride;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int r = r0 + threadIdx.x, c = c0 + q;
    tile[q][threadIdx.x] = (r < R && c < C) ? Sk[(long long)c * R + r] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int Ek = E[k] == kOzBadExp ? 0 : E[k];
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    int r, c;
    double2 v;
    long long o;
    if (TRANS) {
      r = r0 + q;
      c = c0 + threadIdx.x;
      v = tile[threadIdx.x][q];
      o = (long long)r * ld + c;
    } else {
      r = r0 + threadIdx.x;
      c = c0 + q;
      v = tile[q][threadIdx.x];
      o = (long long)c * ld + r;
    }
    if (r >= R || c >= C) continue;
    long long qr = oz_fixed(v.x, Ek, S), qi = oz_fixed(v.y, Ek, S);
    for (int t = S - 1; t >= 1; --t) {
      int dr = (int)(qr & 255), di = (int)(qi & 255);
      if (dr >= 128) dr -= 256;
      if (di >= 128) di -= 256;
      qr = (qr - dr) >> 8;
      qi = (qi - di) >> 8;
      const long long po = ((long long)t * K + k) * plane_elems + o;
      re[po] = __int2bfloat16_rn(dr);
      im[po] = __int2bfloat16_rn(di);
      if (nre) nre[po] = __int2bfloat16_rn(-dr);
      if (nim) nim[po] = __int2bfloat16_rn(-di);
    }
    const long long po = (long long)k * plane_elems + o;
    re[po] = __int2bfloat16_rn((int)qr);
    im[po] = __int2bfloat16_rn((int)qi);
    if (nre) nre[po] = __int2bfloat16_rn(-(int)qr);
    if (nim) nim[po] = __int2bfloat16_rn(-(int)qi);
  }
}

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

void slice_maxabs(const double2* Z, long long T, int K, unsigned long long* out, cudaStream_t st,
                  const int* gate = nullptr) {
  long long b = (T + 255) / 256;
  if (b > 64) b = 64;
  k_oz_maxabs<<<dim3((unsigned)b, K), 256, 0, st>>>(Z, T, out, gate);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

void exponents(const unsigned long long* mx, int K, int* E, cudaStream_t st) {
  k_oz_exponents<<<(K + 127) / 128, 128, 0, st>>>(mx, K, E);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

template <bool TRANS>
void split(const double2* src, long long sstride, int R, int C, int K, const int* E, int S, void* re, void* im,
           void* nre, void* nim, int ld, long long plane_elems, cudaStream_t st, const int* gate = nullptr) {
  k_oz_split<TRANS><<<dim3((R + 31) / 32, (C + 31) / 32, K), dim3(32, 8), 0, st>>>(
      src, sstride, R, C, K, E, S, static_cast<__nv_bfloat16*>(re), static_cast<__nv_bfloat16*>(im),
      static_cast<__nv_bfloat16*>(nre), static_cast<__nv_bfloat16*>(nim), ld, plane_elems, gate);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

}  // namespace

void OzOperands::release() {
  op_free(a_re);
  op_free(a_im);
  op_free(b_re);
  op_free(b_im);
  op_free(b_nre);
  op_free(Eop);
  op_free(mx);
  a_re = a_im = b_re = b_im = b_nre = nullptr;
  Eop = nullptr;
  mx = nullptr;
  S = 0;
}

void oz_prepare(ts_op* op, int S, cudaStream_t st) {
  if (op->oz && op->oz->S == S) return;
  OzOperands* t = op->oz ? op->oz : new OzOperands();
  op->oz = t;
  t->release();
  const int n = op->n, s = op->s, K = op->K;
  t->ldn = round_up(n, 64);
  t->lds = round_up(s, 64);
  const size_t na = (size_t)S * K * n * t->ldn * 2, nb = (size_t)S * K * s * t->lds * 2;
  op_alloc_on(t->a_re, na, st);
  op_alloc_on(t->a_im, na, st);
  op_alloc_on(t->b_re, nb, st);
  op_alloc_on(t->b_im, nb, st);
  op_alloc_on(t->b_nre, nb, st);
  op_alloc_on(t->Eop, sizeof(int) * K, st);
  op_alloc_on(t->mx, sizeof(unsigned long long) * K, st);
  // A_k and B_k share one exponent per slice, so both products of Eq. (2) land on one fixed point.
  unsigned long long* mxb = t->mx;
  TS_CUDA(cudaMemsetAsync(mxb, 0, sizeof(unsigned long long) * K, st));
  slice_maxabs(op->Ah, (long long)n * n, K, mxb, st);
  slice_maxabs(op->Bh, (long long)s * s, K, mxb, st);
  exponents(mxb, K, t->Eop, st);
  split<true>(op->Ah, (long long)n * n, n, n, K, t->Eop, S, t->a_re, t->a_im, nullptr, nullptr, t->ldn,
              (long long)n * t->ldn, st);
  split<false>(op->Bh, (long long)s * s, s, s, K, t->Eop, S, t->b_re, t->b_im, t->b_nre, nullptr, t->lds,
               (long long)s * t->lds, st);
  t->S = S;
}

double oz_bf16_flops(int n, int s, int K, int nyq, int S) {
  const int nreal = 1 + (nyq >= 0 ? 1 : 0);
  const double pairs = 0.5 * S * (S + 1);
  const double per = (double)n * s * ((double)n + s);
  return pairs * per * (8.0 * (K - nreal) + 2.0 * nreal);
}

void oz_preload() {
  const void* fns[] = {(const void*)k_oz_maxabs, (const void*)k_oz_exponents, (const void*)k_oz_split<false>,
                       (const void*)k_oz_split<true>, (const void*)k_oz_sylv};
  for (const void* f : fns) {
    cudaFuncAttributes fa;
    TS_CUDA(cudaFuncGetAttributes(&fa, f));
  }
  set_max_dynamic_smem((const void*)k_oz_sylv, kOzSmem);
}

OzBufferSizes oz_buffer_sizes(int n, int s, int K, int S) {
  OzBufferSizes z;
  z.xc = (size_t)S * K * s * round_up(n, 64) * 2;
  z.xr = (size_t)S * K * n * round_up(s, 64) * 2;
  z.K = K;
  return z;
}

void oz_products(const ts_op* cop, const double2* Xh, double2* Yh, int S, const OzBuffers& b, const int* gate,
                 int* err, cudaStream_t st) {
  const OzOperands& t = *cop->oz;
  TS_REQUIRE(S >= 1 && t.S >= S, "oz_products: operator digits not prepared");
  const int n = cop->n, s = cop->s, p = cop->p, K = cop->K;
  const long long T = (long long)n * s;
  TS_CUDA(cudaMemsetAsync(b.mx, 0, sizeof(unsigned long long) * K, st));
  slice_maxabs(Xh, T, K, b.mx, st, gate);
  exponents(b.mx, K, b.Ex, st);
  split<false>(Xh, T, n, s, K, b.Ex, S, b.xc_re, b.xc_im, nullptr, b.xc_nim, t.ldn, (long long)s * t.ldn, st, gate);
  split<true>(Xh, T, n, s, K, b.Ex, S, b.xr_re, b.xr_im, nullptr, nullptr, t.lds, (long long)n * t.lds, st, gate);
  OzMaps maps;
  // operator planes: all t.S digits exist (digit u of slice k is plane u K + k), the kernel reads u < S
  make_map(&maps.a_re, t.a_re, 2, t.ldn, n, n, t.S * K, kOzM);
  make_map(&maps.a_im, t.a_im, 2, t.ldn, n, n, t.S * K, kOzM);
  make_map(&maps.xc_nim, b.xc_nim, 2, t.ldn, n, s, S * K, kOzN);
  make_map(&maps.xc_re, b.xc_re, 2, t.ldn, n, s, S * K, kOzN);
  make_map(&maps.xc_im, b.xc_im, 2, t.ldn, n, s, S * K, kOzN);
  make_map(&maps.xr_re, b.xr_re, 2, t.lds, s, n, S * K, kOzM);
  make_map(&maps.xr_im, b.xr_im, 2, t.lds, s, n, S * K, kOzM);
  make_map(&maps.b_re, t.b_re, 2, t.lds, s, s, t.S * K, kOzN);
  make_map(&maps.b_im, t.b_im, 2, t.lds, s, s, t.S * K, kOzN);
  make_map(&maps.b_nre, t.b_nre, 2, t.lds, s, s, t.S * K, kOzN);
  // Fixed point 2^(E_op + E_x - F): |partial sums| < 2 (n + s) 2^(E_op + E_x - 2) <= 2^(E_op + E_x + 62 - F).
  int lg = 0;
  while ((1ll << lg) < 2ll * (n + s)) ++lg;
  const int F = 63 - lg;
  dim3 grid((s + kOzN - 1) / kOzN, (n + kOzM - 1) / kOzM, K);
  k_oz_sylv<<<grid, kOzThreads, kOzSmem, st>>>(maps, Yh, n, s, K, nyquist_index(p), S, F, t.Eop, b.Ex, gate, err);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

// The emulated products on spectral tensors: Yh = A_k Xh_k - Xh_k B_k (workspace digit planes of Xh).
void oz_apply_spectral(ts_ctx* ctx, const ts_op* cop, const double2* Xh, double2* Yh, int S, int S_op,
                       cudaStream_t st) {
  ts_op* op = const_cast<ts_op*>(cop);   // the digit planes are cached on first use
  oz_prepare(op, S_op, st);
  oz_preload();
  const int n = op->n, s = op->s, p = op->p, K = op->K;
  const OzBufferSizes z = oz_buffer_sizes(n, s, K, S);
  OzBuffers b;
  b.xc_re = ctx->ws.get("oz_xc_re", z.xc);
  b.xc_im = ctx->ws.get("oz_xc_im", z.xc);
  b.xc_nim = ctx->ws.get("oz_xc_nim", z.xc);
  b.xr_re = ctx->ws.get("oz_xr_re", z.xr);
  b.xr_im = ctx->ws.get("oz_xr_im", z.xr);
  b.mx = static_cast<unsigned long long*>(ctx->ws.get("oz_mx", sizeof(unsigned long long) * K));
  b.Ex = static_cast<int*>(ctx->ws.get("oz_Ex", sizeof(int) * K));
  int* err = static_cast<int*>(ctx->ws.get("tc_err", sizeof(int) * 4));
  KernelTimer& tm = ctx->timer;
  tm.begin(st, 3, gemm_flops(n, s, n, s, K, nyquist_index(p)));
  if (tm.enabled) tm.oz_pair_flops += oz_bf16_flops(n, s, K, nyquist_index(p), S);
  oz_products(op, Xh, Yh, S, b, nullptr, err, st);
  tm.end(st);
}

void apply_f64_oz(ts_ctx* ctx, const ts_op* cop, const double* X, double* Y, int mode, const double* C,
                  double* partials, int S, int S_op, cudaStream_t st) {
  ts_op* op = const_cast<ts_op*>(cop);   // the digit planes are cached on first use
  oz_prepare(op, S_op, st);
  oz_preload();
  const int n = op->n, s = op->s, p = op->p, K = op->K;
  const long long T = (long long)n * s;
  double2* Xh = static_cast<double2*>(ctx->ws.get("apply_Xh", sizeof(double2) * (size_t)K * T));
  double2* Yh = static_cast<double2*>(ctx->ws.get("apply_Yh", sizeof(double2) * (size_t)K * T));
  const OzBufferSizes z = oz_buffer_sizes(n, s, K, S);
  OzBuffers b;
  b.xc_re = ctx->ws.get("oz_xc_re", z.xc);
  b.xc_im = ctx->ws.get("oz_xc_im", z.xc);
  b.xc_nim = ctx->ws.get("oz_xc_nim", z.xc);
  b.xr_re = ctx->ws.get("oz_xr_re", z.xr);
  b.xr_im = ctx->ws.get("oz_xr_im", z.xr);
  b.mx = static_cast<unsigned long long*>(ctx->ws.get("oz_mx", sizeof(unsigned long long) * K));
  b.Ex = static_cast<int*>(ctx->ws.get("oz_Ex", sizeof(int) * K));
  int* err = static_cast<int*>(ctx->ws.get("tc_err", sizeof(int) * 4));
  KernelTimer& tm = ctx->timer;
  tm.begin(st, 1, 8.0 * T * p + 16.0 * K * T);
  rfft_tube<double, double2>(X, Xh, T, p, st);
  tm.end(st);
  tm.begin(st, 3, gemm_flops(n, s, n, s, K, nyquist_index(p)));
  if (tm.enabled) tm.oz_pair_flops += oz_bf16_flops(n, s, K, nyquist_index(p), S);
  oz_products(op, Xh, Yh, S, b, nullptr, err, st);
  tm.end(st);
  tm.begin(st, 1, 16.0 * K * T + 8.0 * T * p * (mode == IRFFT_RESIDUAL ? 2 : 1));
  irfft_tube<double, double2>(Yh, Y, T, p, mode, C, partials, st);
  tm.end(st);
}

}  // namespace ts
