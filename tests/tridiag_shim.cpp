// Host build of the FP64 tridiagonal eigensolver (paper_2405_20258_gb300/csrc/rpa_tridiag.h)
// for the CPU tests: the same scalar routines the device kernels run, one
// eigenvalue or cluster at a time.
#include <stdlib.h>

#include "rpa_tridiag.h"

extern "C" {

// The k smallest eigenvalues of T, ascending.
int tri_eigvals(const double* d, const double* e, int n, int k, double* w) {
  if (n < 1 || k < 0 || k > n) return 1;
  double* e2 = (double*)malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
  for (int i = 0; i + 1 < n; ++i) e2[i] = e[i] * e[i];
  double lo, hi, pivmin;
  rpa::tri::bounds(d, e, n, &lo, &hi, &pivmin);
  const double abstol = 1e-8 * DBL_EPSILON * fmax(fabs(lo), fabs(hi));
  for (int j = 0; j < k; ++j) w[j] = rpa::tri::bisect(d, e2, n, j, lo, hi, pivmin, abstol);
  free(e2);
  return 0;
}

// The same k eigenvalues by FP32 bisection finished in FP64 (the device's default);
// lo32/hi32 (may be NULL) receive each eigenvalue's FP32 bracket.
int tri_eigvals_mixed(const double* d, const double* e, int n, int k, double* w, float* lo32,
                      float* hi32) {
  if (n < 1 || k < 0 || k > n) return 1;
  double* e2 = (double*)malloc(sizeof(double) * (n > 1 ? n - 1 : 1));
  float* d32 = (float*)malloc(sizeof(float) * n);
  float* e2f = (float*)malloc(sizeof(float) * (n > 1 ? n - 1 : 1));
  for (int i = 0; i < n; ++i) d32[i] = (float)d[i];
  for (int i = 0; i + 1 < n; ++i) {
    e2[i] = e[i] * e[i];
    const float ef = (float)e[i];
    e2f[i] = ef * ef;
  }
  double lo, hi, pivmin;
  rpa::tri::bounds(d, e, n, &lo, &hi, &pivmin);
  const double abstol = 1e-8 * DBL_EPSILON * fmax(fabs(lo), fabs(hi));
  for (int j = 0; j < k; ++j) {
    w[j] = rpa::tri::bisect_mixed(d, e2, d32, e2f, n, j, lo, hi, pivmin, abstol);
    if (lo32 && hi32) {
      float a = (float)lo, b = (float)hi;
      rpa::tri::bisect_f(d32, e2f, n, j, &a, &b);
      lo32[j] = a;
      hi32[j] = b;
    }
  }
  free(e2);
  free(d32);
  free(e2f);
  return 0;
}

int tri_clusters(const double* w, int k, double tol, int* first) {
  return rpa::tri::clusters(w, k, tol, first);
}

// Eigenvectors of the given ascending eigenvalues, z row-major [n][k].  The
// scratch lanes are laid out as the device kernel lays them out (lane q of
// cluster c, element i at q n nc + i nc + c), and the clusters run in turn.
int tri_vectors(const double* d, const double* e, int n, const double* w, int k,
                double cluster_tol, double* z) {
  int* first = (int*)malloc(sizeof(int) * (k + 1));
  const int nc = rpa::tri::clusters(w, k, cluster_tol, first);
  const long plane = (long)n * nc;
  double* lanes = (double*)malloc(sizeof(double) * 6 * (size_t)plane);
  double lo, hi, pivmin;
  rpa::tri::bounds(d, e, n, &lo, &hi, &pivmin);
  const double tiny = DBL_EPSILON * fmax(fabs(lo), fabs(hi));
  for (int c = 0; c < nc; ++c) {
    double* b = lanes + c;
    rpa::tri::cluster_vectors(d, e, n, w, first[c], first[c + 1], tiny, z, k,
                              rpa::tri::Lane{b, nc}, rpa::tri::Lane{b + plane, nc},
                              rpa::tri::Lane{b + 2 * plane, nc}, rpa::tri::Lane{b + 3 * plane, nc},
                              rpa::tri::Lane{b + 4 * plane, nc}, rpa::tri::Lane{b + 5 * plane, nc});
  }
  free(lanes);
  free(first);
  return nc;
}

}  // extern "C"
