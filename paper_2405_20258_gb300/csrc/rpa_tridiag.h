// FP64 eigenpairs of a real symmetric tridiagonal matrix T (diagonal d[0..n-1],
// off-diagonal e[0..n-2]): the start of the mixed-precision subspace of chi~(0).
//
// The FP32 Householder reduction of chi~ to T keeps the graded structure of chi~
// (large entries first) well enough for an N_eig + p subspace accurate to ~1e-5,
// but an FP32 solve of T itself resolves eigenvalues only to ~1e-7 of the largest,
// which near the cut (~1e-5 of the largest) mixes the subspace to ~0.1.  So T's
// eigenpairs are computed in FP64:
//   * eigenvalue j (ascending) by bisection on the Sturm count of T - x I (the
//     number of negative pivots of its LDL^T factorisation, Sylvester's law of
//     inertia), each eigenvalue independently: in FP32 first, then, from the
//     FP32 bracket once two FP64 counts confirm it, in FP64;
//   * its eigenvector by inverse iteration with T - lambda_j I factored by
//     Gaussian elimination with partial pivoting (three iterations from a fixed
//     pseudo-random start), re-orthogonalised (modified Gram-Schmidt) against the
//     earlier vectors of its cluster: consecutive eigenvalues closer than
//     cluster_tol apart, whose inverse-iteration vectors are not reliably
//     orthogonal by themselves.
// Every routine here is plain scalar code, compiled both for the device (one
// thread per eigenvalue or per cluster) and for the host (tests).
#pragma once

#include <math.h>
#include <float.h>
#include <stdint.h>

#ifndef RPA_HD
#ifdef __CUDACC__
#define RPA_HD __host__ __device__ __forceinline__
#else
#define RPA_HD inline
#endif
#endif

namespace rpa {
namespace tri {

// Gershgorin interval [*lo, *hi] of T and a pivot floor (the smallest magnitude a
// Sturm pivot may take before it is replaced, to keep the recurrence finite).
RPA_HD void bounds(const double* d, const double* e, int n, double* lo, double* hi,
                   double* pivmin) {
  double l = d[0], h = d[0], emax2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
    l = fmin(l, d[i] - r);
    h = fmax(h, d[i] + r);
    if (i + 1 < n) emax2 = fmax(emax2, e[i] * e[i]);
  }
  const double w = fmax(h - l, DBL_MIN);
  // widen by a little more than the rounding of the Gershgorin sums
  *lo = l - 2.0 * DBL_EPSILON * w * n - DBL_MIN;
  *hi = h + 2.0 * DBL_EPSILON * w * n + DBL_MIN;
  *pivmin = DBL_MIN * fmax(1.0, emax2);
}

// Number of eigenvalues of T below x: the negative pivots q_i of T - x I = L D L^T,
// q_0 = d_0 - x, q_i = d_i - x - e_{i-1}^2 / q_{i-1}.  A pivot at or below pivmin
// counts as negative and is clamped to -pivmin (the standard safeguard; the count
// stays that of a matrix within a few ulps of T).
RPA_HD int sturm_count(const double* d, const double* e2, int n, double x, double pivmin) {
  int c = 0;
  double q = d[0] - x;
  if (q <= pivmin) {
    ++c;
    q = fmin(q, -pivmin);
  }
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (q <= pivmin) {
      ++c;
      q = fmin(q, -pivmin);
    }
  }
  return c;
}

// Eigenvalue j (0-based, ascending) of T by bisection of [lo, hi] (the Gershgorin
// interval), to the larger of 2 ulps of the eigenvalue and abstol.  At most 160
// halvings: from any finite interval this reaches the tolerance.
RPA_HD double bisect(const double* d, const double* e2, int n, int j, double lo, double hi,
                     double pivmin, double abstol) {
  for (int it = 0; it < 160; ++it) {
    const double tol = fmax(abstol, 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)));
    if (hi - lo <= tol) break;
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(d, e2, n, mid, pivmin) <= j)
      lo = mid;  // at most j eigenvalues below mid: lambda_j >= mid
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

// The Sturm count in FP32 (T's FP32 diagonal d and squared off-diagonal e2):
// exact for a matrix within a few FP32 ulps of T, so an FP32 bisection places
// each eigenvalue of the graded T to ~1e-7 of itself at FP32 cost.
RPA_HD int sturm_count_f(const float* d, const float* e2, int n, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (q <= pivmin) {
    ++c;
    q = fminf(q, -pivmin);
  }
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (q <= pivmin) {
      ++c;
      q = fminf(q, -pivmin);
    }
  }
  return c;
}

// FP32 bisection of [*lo, *hi] for eigenvalue j, to 4 FP32 ulps of the eigenvalue
// (at most 64 halvings).  d32, e2_32: T's diagonal and squared off-diagonal in FP32.
RPA_HD void bisect_f(const float* d32, const float* e2_32, int n, int j, float* lo, float* hi) {
  float flo = *lo, fhi = *hi;
  const float fpiv = 1.1754944e-38f;  // FLT_MIN
  for (int it = 0; it < 64; ++it) {
    if (fhi - flo <= 4.0f * 1.1920929e-7f * fmaxf(fabsf(flo), fabsf(fhi))) break;
    const float mid = 0.5f * (flo + fhi);
    if (mid <= flo || mid >= fhi) break;
    if (sturm_count_f(d32, e2_32, n, mid, fpiv) <= j)
      flo = mid;
    else
      fhi = mid;
  }
  *lo = flo;
  *hi = fhi;
}

// Eigenvalue j of T: the FP32 bracket of bisect_f, widened by twice its width,
// checked with two FP64 Sturm counts and bisected on in FP64 to the tolerance of
// bisect().  A bracket that the FP64 counts reject (the FP32 counts disagreed with
// FP64 near the eigenvalue) falls back to FP64 bisection of [lo, hi], so the FP32
// phase only ever saves FP64 counts.
RPA_HD double bisect_mixed(const double* d, const double* e2, const float* d32,
                           const float* e2_32, int n, int j, double lo, double hi,
                           double pivmin, double abstol) {
  float flo = (float)lo, fhi = (float)hi;
  bisect_f(d32, e2_32, n, j, &flo, &fhi);
  const double w = (double)fhi - (double)flo;
  const double blo = fmax(lo, (double)flo - 2.0 * w - abstol);
  const double bhi = fmin(hi, (double)fhi + 2.0 * w + abstol);
  if (blo < bhi && sturm_count(d, e2, n, blo, pivmin) <= j &&
      sturm_count(d, e2, n, bhi, pivmin) > j)
    return bisect(d, e2, n, j, blo, bhi, pivmin, abstol);
  return bisect(d, e2, n, j, lo, hi, pivmin, abstol);
}

// Cluster starts of the ascending eigenvalues w[0..k-1]: a new cluster begins at j
// when w[j] - w[j-1] > cluster_tol.  first[c] is the first index of cluster c,
// first[n_clusters] = k.  Returns the number of clusters.
inline int clusters(const double* w, int k, double cluster_tol, int* first) {
  int nc = 0;
  for (int j = 0; j < k; ++j)
    if (j == 0 || w[j] - w[j - 1] > cluster_tol) first[nc++] = j;
  first[nc] = k;
  return nc;
}

// Strided view of one thread's scratch: element i lives at p[i * stride], so that
// the threads of a warp, each at the same i, touch consecutive addresses.
template <typename R>
struct LaneT {
  R* p;
  long stride;
  RPA_HD R& operator[](long i) const { return p[i * stride]; }
};
using Lane = LaneT<double>;

template <typename R>
RPA_HD R rabs(R x) {
  return x < R(0) ? -x : x;
}

// Gaussian elimination with partial pivoting of M = T - lambda I.  U (upper, two
// super-diagonals) in u0 (diagonal), u1, u2; multipliers in l; piv[i] = 1 when
// rows i and i+1 were exchanged at step i.  Pivots smaller than tiny are replaced
// by +-tiny, so that the solve stays finite at an exact eigenvalue.
template <typename R>
RPA_HD void lu_factor(const R* d, const R* e, int n, R lambda, R tiny, LaneT<R> u0, LaneT<R> u1,
                      LaneT<R> u2, LaneT<R> l, LaneT<R> piv) {
  // current row k: a at column k, b at column k+1
  R a = d[0] - lambda, b = n > 1 ? e[0] : R(0);
  for (int k = 0; k + 1 < n; ++k) {
    const R g = e[k];                          // M[k+1][k]
    const R al = d[k + 1] - lambda;            // M[k+1][k+1]
    const R be = k + 2 < n ? e[k + 1] : R(0);  // M[k+1][k+2]
    if (rabs(a) >= rabs(g)) {
      if (rabs(a) < tiny) a = a < R(0) ? -tiny : tiny;
      const R m = g / a;
      u0[k] = a;
      u1[k] = b;
      u2[k] = R(0);
      l[k] = m;
      piv[k] = R(0);
      a = al - m * b;
      b = be;
    } else {
      const R m = a / g;
      u0[k] = g;
      u1[k] = al;
      u2[k] = be;
      l[k] = m;
      piv[k] = R(1);
      a = b - m * al;
      b = -m * be;
    }
  }
  if (rabs(a) < tiny) a = a < R(0) ? -tiny : tiny;
  u0[n - 1] = a;
}

// Solve M x = y in place (y becomes x) with the factors of lu_factor.  Returns the
// factor by which the result was scaled down to stay finite (1 if none).  Both
// sweeps are recurrences; their operands are fetched PF steps ahead (the lanes
// live in global memory on the device, where a fetch takes hundreds of cycles),
// with the arithmetic in the same order as one step at a time.
constexpr int PF = 8;
template <typename R>
RPA_HD R lu_solve(int n, LaneT<R> u0, LaneT<R> u1, LaneT<R> u2, LaneT<R> l, LaneT<R> piv,
                  LaneT<R> y) {
  // forward: row exchanges and multipliers; cur = y[k] as updated so far
  R cur = n > 0 ? y[0] : R(0);
  for (int k0 = 0; k0 + 1 < n; k0 += PF) {
    const int cnt = (n - 1 - k0) < PF ? (n - 1 - k0) : PF;
    R bp[PF], bl[PF], by[PF];
    for (int t = 0; t < cnt; ++t) {
      bp[t] = piv[k0 + t];
      bl[t] = l[k0 + t];
      by[t] = y[k0 + t + 1];
    }
    for (int t = 0; t < cnt; ++t) {
      const int k = k0 + t;
      if (bp[t] != R(0)) {
        const R yk = cur, yk1 = by[t];
        y[k] = yk1;
        cur = yk - bl[t] * yk1;
      } else {
        y[k] = cur;
        cur = by[t] - bl[t] * cur;
      }
    }
  }
  if (n > 0) y[n - 1] = cur;
  R scale = R(1);
  const R big = sizeof(R) == 4 ? R(1e30) : R(1e150);
  // backward: s_k = (y_k - u1_k s_{k+1} - u2_k s_{k+2}) / u0_k
  R s1 = R(0), s2 = R(0);  // s_{k+1}, s_{k+2}
  for (int k0 = n - 1; k0 >= 0; k0 -= PF) {
    const int cnt = (k0 + 1) < PF ? (k0 + 1) : PF;
    R by[PF], b0[PF], b1[PF], b2[PF];
    for (int t = 0; t < cnt; ++t) {
      const int k = k0 - t;
      by[t] = y[k];
      b0[t] = u0[k];
      b1[t] = u1[k];
      b2[t] = u2[k];
    }
    for (int t = 0; t < cnt; ++t) {
      const int k = k0 - t;
      R s = by[t];
      if (k + 1 < n) s -= b1[t] * s1;
      if (k + 2 < n) s -= b2[t] * s2;
      s /= b0[t];
      if (rabs(s) > big) {
        // rescale the solved tail (and the rest of the right-hand side) by 1/big
        for (int i = 0; i < n; ++i) y[i] *= R(1) / big;
        for (int t2 = t + 1; t2 < cnt; ++t2) by[t2] *= R(1) / big;
        s1 *= R(1) / big;
        s2 *= R(1) / big;
        s *= R(1) / big;
        scale *= R(1) / big;
      }
      y[k] = s;
      s2 = s1;
      s1 = s;
    }
  }
  return scale;
}

// A fixed pseudo-random start in [-1, 1) for component i of vector j (splitmix64 of
// the pair; any start with a component along the eigenvector serves).
RPA_HD double start_component(int j, long i) {
  uint64_t x = ((uint64_t)(uint32_t)j << 32) ^ (uint64_t)i;
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Eigenvectors of the cluster w[j0..j1-1] by inverse iteration.  Column j of Z is
// z[i * ldz + j] (row-major, i the row).  The scratch lanes hold n elements each.
// R: the arithmetic and scratch type (double, or float for a T that is itself an FP32
// object); w and z are FP64 either way.
template <typename R>
RPA_HD void cluster_vectors(const R* d, const R* e, int n, const double* w, int j0, int j1,
                            R tiny, double* z, long ldz, LaneT<R> u0, LaneT<R> u1, LaneT<R> u2,
                            LaneT<R> l, LaneT<R> piv, LaneT<R> y) {
  for (int j = j0; j < j1; ++j) {
    lu_factor(d, e, n, (R)w[j], tiny, u0, u1, u2, l, piv);
    R nrm2 = R(0);
    for (long i = 0; i < n; ++i) {
      y[i] = (R)start_component(j, i);
      nrm2 += y[i] * y[i];
    }
    for (int it = 0; it < 3; ++it) {
      const R s = R(1) / sqrt(nrm2);
      for (long i = 0; i < n; ++i) y[i] *= s;
      lu_solve(n, u0, u1, u2, l, piv, y);
      // modified Gram-Schmidt against the cluster's earlier (unit) vectors
      for (int jj = j0; jj < j; ++jj) {
        R dot = R(0);
        for (long i = 0; i < n; ++i) dot += (R)z[i * ldz + jj] * y[i];
        for (long i = 0; i < n; ++i) y[i] -= dot * (R)z[i * ldz + jj];
      }
      nrm2 = R(0);
      for (long i = 0; i < n; ++i) nrm2 += y[i] * y[i];
      if (!(nrm2 > R(0))) {
        // the solve returned nothing outside the earlier vectors: restart from a
        // different pseudo-random vector
        nrm2 = R(0);
        for (long i = 0; i < n; ++i) {
          y[i] = (R)start_component(j + 7919 * (it + 1), i);
          nrm2 += y[i] * y[i];
        }
      }
    }
    const R s = R(1) / sqrt(nrm2);
    for (long i = 0; i < n; ++i) z[i * ldz + j] = (double)(y[i] * s);
  }
}

}  // namespace tri
}  // namespace rpa
