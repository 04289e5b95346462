// Complex Schur form B_k = Q T Q^H of the small s x s Fourier slices of B (t-Bartels-Stewart,
// Algorithm 4 read with a complex Schur form per slice; and the projected equation of TBAS): one
// warp per slice, Givens reduction to upper Hessenberg form, then implicitly shifted single-shift
// QR with Wilkinson shifts and deflation.
//
// The Wilkinson shift takes the principal square root with the smaller component formed as
// Im z / (2 larger): the first version formed both components from (|z| +- Re z) / 2, lost the small
// one to cancellation when Im z was tiny, and its shift then missed the trailing window's eigenvalue
// by that much; some 64 x 64 and 96 x 96 slices of the dense test family never deflated their last
// 2 x 2 window and ran into the iteration limit (TS_SINGULAR).  With the stable root the same
// matrices converge in 220-348 iterations, as in a host emulation of the same steps.
#include "internal.cuh"
#include "complex_ops.cuh"
#include "tba.cuh"

namespace ts {
namespace {

// Givens rotation G = [[c, s], [-conj(s), c]] (c real) with G [a; b] = [r; 0].
__device__ __forceinline__ void givens(double2 a, double2 b, double& c, double2& s) {
  const double na = cabs2(a), nb = cabs2(b);
  if (nb == 0.0) {
    c = 1.0;
    s = make_double2(0.0, 0.0);
    return;
  }
  if (na == 0.0) {
    c = 0.0;
    s = cscale(cconj(b), 1.0 / nb);   // G [0; b] = [s b; c b] = [|b|; 0]
    return;
  }
  const double nr = hypot(na, nb);
  c = na / nr;
  const double2 ua = cscale(a, 1.0 / na);  // a / |a|
  s = cscale(cmul(ua, cconj(b)), 1.0 / nr);
}

// Rows (i, i+1), columns [c0, s):  row_i' = c row_i + s row_{i+1};  row_{i+1}' = -conj(s) row_i + c row_{i+1}
__device__ void rot_rows(double2* T, int ld, int i, int c0, int c1, double c, double2 s) {
  for (int q = c0 + (int)(threadIdx.x & 31); q < c1; q += 32) {
    const double2 a = T[i + (long long)ld * q], b = T[i + 1 + (long long)ld * q];
    T[i + (long long)ld * q] = cadd(cscale(a, c), cmul(s, b));
    T[i + 1 + (long long)ld * q] = csub(cscale(b, c), cmul(cconj(s), a));
  }
  __syncwarp();
}
// Columns (i, i+1), rows [r0, r1): multiply on the right by G^H:
//   col_i' = c col_i + conj(s) col_{i+1};  col_{i+1}' = -s col_i + c col_{i+1}
__device__ void rot_cols(double2* T, int ld, int i, int r0, int r1, double c, double2 s) {
  for (int r = r0 + (int)(threadIdx.x & 31); r < r1; r += 32) {
    const double2 a = T[r + (long long)ld * i], b = T[r + (long long)ld * (i + 1)];
    T[r + (long long)ld * i] = cadd(cscale(a, c), cmul(cconj(s), b));
    T[r + (long long)ld * (i + 1)] = csub(cscale(b, c), cmul(s, a));
  }
  __syncwarp();
}

// Complex Schur form, one warp per matrix: B (s x s) = Q T Q^H, T upper triangular.
// In: T holds B.  Out: T, Q.  err bit 1 on failure to converge.
__global__ void k_schur_small(double2* __restrict__ Tall, double2* __restrict__ Qall, int s, int* err) {
  double2* T = Tall + (long long)blockIdx.x * s * s;
  double2* Q = Qall + (long long)blockIdx.x * s * s;
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < s * s; e += 32) Q[e] = make_double2((e % s) == (e / s) ? 1.0 : 0.0, 0.0);
  __syncwarp();
  // Hessenberg reduction by Givens rotations.
  for (int c = 0; c + 2 < s; ++c) {
    for (int r = s - 1; r >= c + 2; --r) {
      double cs;
      double2 sn;
      givens(T[r - 1 + (long long)s * c], T[r + (long long)s * c], cs, sn);
      rot_rows(T, s, r - 1, c, s, cs, sn);
      rot_cols(T, s, r - 1, 0, s, cs, sn);
      rot_cols(Q, s, r - 1, 0, s, cs, sn);
      if (lane == 0) T[r + (long long)s * c] = make_double2(0.0, 0.0);
      __syncwarp();
    }
  }
  // Shifted QR on the active window [lo, hi].
  const double eps = 2.220446049250313e-16;
  int hi = s - 1, iter = 0, since = 0;
  const int max_iter = 60 * s + 60;
  while (hi > 0) {
    if (iter++ > max_iter) {
      if (lane == 0) atomicOr(err, 1);
      break;
    }
    int lo = hi;
    while (lo > 0) {
      const double2 sub = T[lo + (long long)s * (lo - 1)];
      double scale = cabs2(T[lo + (long long)s * lo]) + cabs2(T[lo - 1 + (long long)s * (lo - 1)]);
      if (scale == 0.0) scale = 1.0;
      if (cabs2(sub) <= eps * scale) {
        if (lane == 0) T[lo + (long long)s * (lo - 1)] = make_double2(0.0, 0.0);
        __syncwarp();
        break;
      }
      --lo;
    }
    if (lo == hi) {
      --hi;
      since = 0;
      continue;
    }
    // Wilkinson shift from the trailing 2 x 2 block of the window.
    const double2 a = T[hi - 1 + (long long)s * (hi - 1)], b = T[hi - 1 + (long long)s * hi];
    const double2 cc = T[hi + (long long)s * (hi - 1)], d = T[hi + (long long)s * hi];
    double2 mu;
    ++since;
    if (since % 11 == 10) {
      // exceptional shift
      mu = cadd(d, make_double2(cabs2(cc), 0.0));
    } else {
      const double2 half = cscale(csub(a, d), 0.5);
      const double2 disc2 = cadd(cmul(half, half), cmul(b, cc));
      // principal square root of disc2: the larger component from (|z| +- Re z) / 2, the other as
      // Im z / (2 larger), which avoids the cancellation in |z| - |Re z| (taking both components from
      // those formulas lost the small one entirely when Im z was tiny, and the shift then missed the
      // window's eigenvalue by that much: a 96 x 96 slice never deflated its last 2 x 2 window)
      const double r = cabs2(disc2);
      double2 sq = make_double2(0.0, 0.0);
      if (r > 0.0) {
        if (disc2.x >= 0.0) {
          const double t = sqrt(0.5 * (r + disc2.x));
          sq = make_double2(t, disc2.y / (2.0 * t));
        } else {
          const double t = sqrt(0.5 * (r - disc2.x));
          sq = make_double2(fabs(disc2.y) / (2.0 * t), disc2.y < 0.0 ? -t : t);
        }
      }
      const double2 m1 = cadd(cadd(d, half), sq), m2 = csub(cadd(d, half), sq);
      mu = cabs2(csub(m1, d)) <= cabs2(csub(m2, d)) ? m1 : m2;
    }
    double2 x = csub(T[lo + (long long)s * lo], mu), y = T[lo + 1 + (long long)s * lo];
    for (int i = lo; i < hi; ++i) {
      double cs;
      double2 sn;
      givens(x, y, cs, sn);
      const int c0 = i > lo ? i - 1 : lo;
      rot_rows(T, s, i, c0, s, cs, sn);
      const int r1 = (i + 3 <= hi + 1) ? i + 3 : hi + 1;
      rot_cols(T, s, i, 0, r1, cs, sn);
      rot_cols(Q, s, i, 0, s, cs, sn);
      if (i > lo) {
        if (lane == 0) T[i + 1 + (long long)s * (i - 1)] = make_double2(0.0, 0.0);
        __syncwarp();
      }
      if (i + 1 < hi) {
        x = T[i + 1 + (long long)s * i];
        y = T[i + 2 + (long long)s * i];
      }
    }
  }
  for (int e = lane; e < s * s; e += 32)
    if ((e % s) > (e / s)) T[e] = make_double2(0.0, 0.0);
}

}  // namespace

void schur_small(double2* T, double2* Q, int s, int count, int* err, cudaStream_t st) {
  k_schur_small<<<count, 32, 0, st>>>(T, Q, s, err);
  count_launch();
  TS_CUDA(cudaGetLastError());
}

}  // namespace ts
