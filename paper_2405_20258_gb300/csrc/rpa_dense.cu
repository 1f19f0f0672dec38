// Dense Hermitian eigensolver building blocks (declarations and the algorithms
// they follow in rpa_dense.h).
//
// Persistent kernels (hetrd, jacobi) are launched cooperatively, one CTA per SM
// at most, so that every CTA is resident; their grid-wide barriers are an
// arrival counter and a generation word in global memory.  Every barrier wait
// is bounded (about 2 s of SM clock): on expiry the CTA raises the abort word
// and a status bit and the kernel returns at its next barrier, so a stalled
// launch ends with an error the host reads instead of hanging.  Data that
// other CTAs wrote during the launch is read with ld.global.cg (L2, not the
// per-SM L1, which is not coherent across SMs).
#include "rpa_dense.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

namespace rpa {
namespace dense {
namespace {

template <typename T>
struct CxT;
template <>
struct CxT<float> {
  using C = float2;
};
template <>
struct CxT<double> {
  using C = double2;
};

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  return C{a.x + b.x, a.y + b.y};
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  return C{a.x - b.x, a.y - b.y};
}
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// conj(a) b
template <typename C>
__device__ __forceinline__ C cmul_ca(C a, C b) {
  return C{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
// a conj(b)
template <typename C>
__device__ __forceinline__ C cmul_cb(C a, C b) {
  return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// acc + a b with four FMAs
template <typename C>
__device__ __forceinline__ C cfma(C acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
template <typename C>
__device__ __forceinline__ C cconj(C a) {
  return C{a.x, -a.y};
}
template <typename C>
__device__ __forceinline__ C warp_csum(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

// A complex128 element through L2 (written by another CTA of the same launch).
__device__ __forceinline__ cplx ldcg_c(const cplx* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return cplx{v.x, v.y};
}

// Grid-wide barrier: bar[0] arrivals, bar[1] generation, bar[2] abort.  gen is the
// generation this CTA last passed (kept by thread 0).  false: a wait ran out here
// or in another CTA; the caller returns.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned& gen, int* status,
                             int code) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned target = gen + 1;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], target);
    } else {
      const long long t0 = clock64();
      while (true) {
        if (*(volatile unsigned*)&bar[1] == target) break;
        if (*(volatile unsigned*)&bar[2]) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > kWaitCycles) {
          atomicExch(&bar[2], 1u);
          atomicOr(status, code);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    gen = target;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Words of barrier state for a grid of `grid` CTAs (arrivals, generation, abort).
size_t bar_words(int) { return 4; }

// ---------------------------------------------------------------------------
// Householder tridiagonalisation (lower), blocked, persistent.
//
// CTA b owns the rows and columns i = b + G r.  Per column k, with c earlier
// columns of the current panel whose updates are deferred (A_eff = A - V W^H -
// W V^H over the panel's V, W):
//   A  each CTA forms its rows of x = A_eff(k:n, k) and partial sums of
//      ||x(k+2:)||^2, W^H x and V^H x over them;                     barrier
//   B  every CTA completes the sums (fixed order), forms the reflector
//      (beta, tau; v = [1, x(k+2:) / (alpha - beta)]) and, for its columns i,
//      y_i = (A_eff v)_i = conj(A(:, i)) . v - V(i,:) (W^H v) - W(i,:) (V^H v),
//      and a partial sum of y^H v;                                   barrier
//   C  w = tau y - (1/2) |tau|^2 (y^H v) v for its rows: the panel's next W
//      column.  Row k+1 of W, which the next column's step A needs in every CTA,
//      is recomputed by each CTA from y_{k+1} (the same arithmetic, so the same
//      value).
// After 32 columns (or the last): barrier, A(k+1:, k+1:) -= V W^H + W V^H over the
// CTA's columns (register-tiled: a lane updates up to four rows of four columns per
// pass over the panel), barrier.  Each step issues its global loads in one round:
// what a step needs from other CTAs was written before the barrier that opens it.
// ---------------------------------------------------------------------------
constexpr int PNB = 32;             // panel width
constexpr int HT = 512;             // threads per CTA
constexpr int HW = HT / 32;         // warps per CTA
constexpr int PL = 2 * PNB + 1;     // partial sums per CTA
constexpr int MAXG = 160;           // largest persistent grid (the sums' staging)
constexpr int MAXOWN = 128;         // rows a CTA may own (n <= MAXOWN * grid)

// Rows per chunk of the trailing update staged in shared memory: 128 (FP32) or 32
// (FP64); a lane updates up to RJ/32 rows of four columns per pass.
template <typename T>
__host__ __device__ constexpr int rj_rows() {
  return sizeof(T) == 4 ? 128 : 32;
}

template <typename T>
struct HetrdArgs {
  using C = typename CxT<T>::C;
  C* a;
  int n;
  T* d;
  T* e;
  C* tau;
  C *vp, *wp, *xcol, *ycol, *part, *part2;
  unsigned* bar;
  int* status;
};

// The reflector v of the current column is staged in shared memory when it has at
// most VCAP elements (96 KB); longer ones are read from L2.  During a trailing
// update the same space holds conj W(i, :) and conj V(i, :) of the CTA's columns.
template <typename T>
__host__ __device__ constexpr int vcap() {
  return (int)(96 * 1024 / sizeof(typename CxT<T>::C));
}

// Shared memory of hetrd_kernel in complex elements: y and v of the CTA's columns
// (2 MAXOWN), partial sums (PL MAXG/4), their totals (PL), W^H v and V^H v (2 PNB),
// the staged panel rows of a trailing-update chunk (2 RJ (PNB + 1)), scalars (8),
// the staged reflector (vcap).
template <typename T>
size_t hetrd_smem() {
  using C = typename CxT<T>::C;
  return sizeof(C) * (2 * MAXOWN + PL * (MAXG / 4) + PL + 2 * PNB +
                      2 * rj_rows<T>() * (PNB + 1) + 8 + vcap<T>());
}

template <typename T>
__global__ void __launch_bounds__(HT, 1) hetrd_kernel(HetrdArgs<T> p) {
  using C = typename CxT<T>::C;
  constexpr int RJT = rj_rows<T>();
  constexpr int RL = RJT / 32;                // rows per lane of a whole chunk
  constexpr int NCB = vcap<T>() / (2 * PNB);  // columns staged per trailing-update batch
  static_assert(NCB % 4 == 0, "column batches of whole quads");
  extern __shared__ __align__(16) unsigned char smraw[];
  C* ys = (C*)smraw;               // [MAXOWN] y_i of this CTA's columns (step B to C)
  C* vsv = ys + MAXOWN;            // [MAXOWN] v_i of this CTA's columns
  C* red = vsv + MAXOWN;           // [PL * MAXG/4] (>= HW * PL)
  C* tot = red + PL * (MAXG / 4);  // [PL]
  C* s1 = tot + PL;                // [PNB] W^H v
  C* s2 = s1 + PNB;                // [PNB] V^H v
  C* Vs = s2 + PNB;                // [RJT][PNB + 1]
  C* Ws = Vs + RJT * (PNB + 1);    // [RJT][PNB + 1]
  C* scal = Ws + RJT * (PNB + 1);  // tau, sc, alpha2, W(k+1, c), alpha
  C* vsm = scal + 8;               // [vcap] v(k+1 : n) when it fits
  const int n = p.n, G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, warp = tid >> 5,
            lane = tid & 31;
  const int rend = n > b ? (n - b + G - 1) / G : 0;  // local r < rend: i = b + G r < n
  unsigned gen = 0;
  int c = 0;
  if (tid == 0) scal[3] = C{0, 0};
  for (int k = 0; k < n; ++k) {
    // W(i, c-1) of this CTA's rows, written by other threads of the CTA in step C of
    // the previous column, is read below
    __syncthreads();
    // ---- A: this CTA's rows of the updated column k and their partial sums, one
    // round of loads per row.  Row k of the panel is held by lane q < c of every
    // warp: V(k, c-1) = 1, W(k, c-1) as recomputed in step C of the previous column.
    const int rbeg = k > b ? (k - b + G - 1) / G : 0;
    const int nown = max(0, rend - rbeg);
    C vkl = {0, 0}, wkl = {0, 0};
    if (lane < c) {
      vkl = lane == c - 1 ? C{1, 0} : __ldcg(&p.vp[(size_t)k * PNB + lane]);
      wkl = lane == c - 1 ? scal[3] : __ldcg(&p.wp[(size_t)k * PNB + lane]);
    }
    C a1 = {0, 0}, a2 = {0, 0};
    T nrm = T(0);
    // a warp per owned row, lanes over the panel's columns; partial sums over the
    // rows >= k+2 (per warp in row order, then warps in order): ||x||^2, W^H x, V^H x
    for (int q = warp; q < nown; q += HW) {
      const int i = b + G * (rbeg + q);
      C vil = {0, 0}, wil = {0, 0};
      if (lane < c) {
        vil = __ldcg(&p.vp[(size_t)i * PNB + lane]);
        wil = __ldcg(&p.wp[(size_t)i * PNB + lane]);
      }
      const C aik = __ldcg(&p.a[(size_t)k * n + i]);
      const C x = csub(aik, warp_csum(cadd(cmul_cb(vil, wkl), cmul_cb(wil, vkl))));
      if (lane == 0) {
        if (i == k)
          p.d[k] = x.x;
        else
          p.xcol[i] = x;
      }
      if (i >= k + 2) {
        nrm += x.x * x.x + x.y * x.y;
        a1 = cadd(a1, cmul_ca(wil, x));
        a2 = cadd(a2, cmul_ca(vil, x));
      }
    }
    if (k == n - 1) break;
    if (lane == 0) red[warp * PL] = C{nrm, T(0)};
    if (lane < c) {
      red[warp * PL + 1 + lane] = a1;
      red[warp * PL + 1 + c + lane] = a2;
    }
    __syncthreads();
    if (tid <= 2 * c) {
      C acc = {0, 0};
      for (int w = 0; w < HW; ++w) acc = cadd(acc, red[w * PL + tid]);
      p.part[(size_t)tid * G + b] = acc;  // entry-major: one entry's G partials adjacent
    }
    if (!grid_barrier(p.bar, G, gen, p.status, 1)) return;

    // ---- B: reflector and A_eff v over this CTA's columns.  One round of
    // independent loads: every CTA's partial sums (entry q by the 8 lanes of group
    // tid / 8, each summing G/8 partials in order, then a fixed tree over the group:
    // the same order in every CTA), alpha = x(k+1), row k+1 of the panel, and
    // x(k+2:) staged unscaled.
    const int L = 2 * c + 1;  // <= 63: c <= 31 here
    const int j0 = k + 1, len = n - j0;
    const bool staged = len <= vcap<T>();
    {
      const int q = tid >> 3, sub = tid & 7;
      C acc = {0, 0};
      if (q < L) {
        C v[MAXG / 8];
#pragma unroll
        for (int u = 0; u < MAXG / 8; ++u) {
          const int g = sub + 8 * u;
          v[u] = g < G ? __ldcg(&p.part[(size_t)q * G + g]) : C{0, 0};
        }
#pragma unroll
        for (int u = 0; u < MAXG / 8; ++u) acc = cadd(acc, v[u]);
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (sub == 0 && q < L) tot[q] = acc;
    }
    C wr1 = {0, 0}, vr1 = {0, 0};
    if (tid < c) {
      wr1 = __ldcg(&p.wp[(size_t)(k + 1) * PNB + tid]);
      vr1 = __ldcg(&p.vp[(size_t)(k + 1) * PNB + tid]);
    }
    if (tid == HT - 1) scal[4] = __ldcg(&p.xcol[k + 1]);
    if (staged)
      for (int t = tid; t < len; t += HT) vsm[t] = t == 0 ? C{1, 0} : __ldcg(&p.xcol[j0 + t]);
    __syncthreads();
    if (tid == 0) {
      const C alpha = scal[4];
      const T xn2 = tot[0].x;
      C tau, sc;
      T beta;
      if (xn2 == T(0) && alpha.y == T(0)) {
        tau = C{0, 0};
        sc = C{0, 0};
        beta = alpha.x;
      } else {
        const T nrm2 = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
        beta = alpha.x >= T(0) ? -nrm2 : nrm2;
        tau = C{(beta - alpha.x) / beta, -alpha.y / beta};
        const T dx = alpha.x - beta, dy = alpha.y, dd = dx * dx + dy * dy;
        sc = C{dx / dd, -dy / dd};
      }
      scal[0] = tau;
      scal[1] = sc;
      if (b == 0) {
        p.e[k] = beta;
        p.tau[k] = tau;
      }
    }
    __syncthreads();
    const C tau = scal[0], sc = scal[1];
    if (tid < c) {
      s1[tid] = cadd(cconj(wr1), cmul(sc, tot[1 + tid]));
      s2[tid] = cadd(cconj(vr1), cmul(sc, tot[1 + c + tid]));
    }
    if (staged)
      for (int t = 1 + tid; t < len; t += HT) vsm[t] = cmul(vsm[t], sc);
    __syncthreads();
    const int cbeg = k + 1 > b ? (k + 1 - b + G - 1) / G : 0;
    const int ncol = max(0, rend - cbeg);
    C yvp = {0, 0};
    // Work items (column q, segment sg): when a CTA has fewer columns than warps,
    // each column's dot product is cut into nseg segments so that every warp streams
    // A; eight loads in flight per lane; segment sums are added in segment order.
    const int nseg = ncol > 0 ? max(1, HW / ncol) : 1;
    const int seglen = ((len + nseg - 1) / nseg + 31) / 32 * 32;
    auto finish = [&](int q, C acc) {
      const int i = b + G * (cbeg + q);
      C corr = {0, 0};
      if (lane < c)
        corr = cadd(cmul(__ldcg(&p.vp[(size_t)i * PNB + lane]), s1[lane]),
                    cmul(__ldcg(&p.wp[(size_t)i * PNB + lane]), s2[lane]));
      corr = warp_csum(corr);
      if (lane == 0) {
        const C y = csub(acc, corr);
        const C vi = i == k + 1 ? C{1, 0} : cmul(__ldcg(&p.xcol[i]), sc);
        p.ycol[i] = y;
        p.vp[(size_t)i * PNB + c] = vi;
        p.a[(size_t)k * n + i] = vi;
        ys[q] = y;
        vsv[q] = vi;
        yvp = cadd(yvp, cmul_ca(y, vi));
      }
    };
    for (int it = warp; it < ncol * nseg; it += HW) {
      const int q = it / nseg, sg = it % nseg;
      const int i = b + G * (cbeg + q);
      const C* col = p.a + (size_t)i * n + j0;
      const int t0 = sg * seglen, t1 = min(len, t0 + seglen);
      C acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = C{0, 0};
      int t = t0 + lane;
      if (staged) {
        for (; t + 224 < t1; t += 256) {
          C av[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) av[u] = __ldcg(&col[t + 32 * u]);
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] = cadd(acc[u], cmul_ca(av[u], vsm[t + 32 * u]));
        }
        for (; t < t1; t += 32) acc[0] = cadd(acc[0], cmul_ca(__ldcg(&col[t]), vsm[t]));
      } else {
        for (; t < t1; t += 32) {
          const C vj = t == 0 ? C{1, 0} : cmul(__ldcg(&p.xcol[j0 + t]), sc);
          acc[0] = cadd(acc[0], cmul_ca(__ldcg(&col[t]), vj));
        }
      }
      const C sum = warp_csum(cadd(cadd(cadd(acc[0], acc[1]), cadd(acc[2], acc[3])),
                                   cadd(cadd(acc[4], acc[5]), cadd(acc[6], acc[7]))));
      if (nseg == 1)
        finish(q, sum);
      else if (lane == 0)
        red[it] = sum;
    }
    if (nseg > 1) {
      __syncthreads();
      for (int q = warp; q < ncol; q += HW) {
        C sum = {0, 0};
        for (int sg = 0; sg < nseg; ++sg) sum = cadd(sum, red[q * nseg + sg]);
        finish(q, sum);
      }
    }
    __syncthreads();
    if (lane == 0) red[warp] = yvp;
    __syncthreads();
    if (tid == 0) {
      C t = {0, 0};
      for (int w = 0; w < HW; ++w) t = cadd(t, red[w]);
      p.part2[b] = t;
    }
    if (!grid_barrier(p.bar, G, gen, p.status, 1)) return;

    // ---- C: the panel's W column (y and v of the CTA's columns from shared memory)
    if (warp == 0) {
      const C y1 = lane == 0 ? __ldcg(&p.ycol[k + 1]) : C{0, 0};
      C t = {0, 0};
      for (int g = lane; g < G; g += 32) t = cadd(t, __ldcg(&p.part2[g]));
      t = warp_csum(t);
      if (lane == 0) {
        const T t2 = tau.x * tau.x + tau.y * tau.y;
        const C alpha2 = C{T(-0.5) * t2 * t.x, T(-0.5) * t2 * t.y};
        scal[2] = alpha2;
        scal[3] = cadd(cmul(tau, y1), alpha2);
      }
    }
    __syncthreads();
    const C alpha2 = scal[2];
    for (int q = tid; q < ncol; q += HT) {
      const int i = b + G * (cbeg + q);
      p.wp[(size_t)i * PNB + c] = cadd(cmul(tau, ys[q]), cmul(alpha2, vsv[q]));
    }
    ++c;
    if (c == PNB || k == n - 2) {
      if (!grid_barrier(p.bar, G, gen, p.status, 1)) return;
      // trailing update of this CTA's columns i >= k+1, rows j >= k+1:
      // A(j, i) -= sum_q V(j, q) conj(W(i, q)) + W(j, q) conj(V(i, q)).  The columns'
      // conj W(i, :), conj V(i, :) are staged in batches of NCB (in the reflector's
      // space), the rows in chunks of RJT; a warp takes a quad of columns and a
      // slice of the chunk's rows, a lane up to RL rows of the quad.
      const int kn = k + 1;
      const int cb2 = kn > b ? (kn - b + G - 1) / G : 0;
      const int nc2 = max(0, rend - cb2);
      C* wcs = vsm;              // [NCB][PNB]
      C* vcs = vsm + NCB * PNB;  // [NCB][PNB]
      for (int cb0 = 0; cb0 < nc2; cb0 += NCB) {
        const int ncb = min(NCB, nc2 - cb0);
        __syncthreads();
        for (int e = tid; e < ncb * PNB; e += HT) {
          const int q = e / PNB, qq = e % PNB, i = b + G * (cb2 + cb0 + q);
          const bool in = qq < c;
          wcs[e] = in ? cconj(__ldcg(&p.wp[(size_t)i * PNB + qq])) : C{0, 0};
          vcs[e] = in ? cconj(__ldcg(&p.vp[(size_t)i * PNB + qq])) : C{0, 0};
        }
        // row slices per chunk: the fewest passes x rows per lane, ties to fewer slices
        const int nquad = (ncb + 3) / 4;
        int rs = 1, best = 1 << 30;
        for (int r = 1; r <= RL; r *= 2) {
          const int cost = ((nquad * r + HW - 1) / HW) * (RL / r);
          if (cost < best) {
            best = cost;
            rs = r;
          }
        }
        const int nr = RL / rs;
        for (int r0 = kn; r0 < n; r0 += RJT) {
          __syncthreads();
          for (int e = tid; e < RJT * PNB; e += HT) {
            const int r = e / PNB, qq = e % PNB, j = r0 + r;
            const bool in = j < n && qq < c;
            Vs[r * (PNB + 1) + qq] = in ? __ldcg(&p.vp[(size_t)j * PNB + qq]) : C{0, 0};
            Ws[r * (PNB + 1) + qq] = in ? __ldcg(&p.wp[(size_t)j * PNB + qq]) : C{0, 0};
          }
          __syncthreads();
          for (int it = warp; it < nquad * rs; it += HW) {
            const int quad = it / rs, sl = it % rs;
            const int rb = sl * (RJT / rs) + lane;  // this lane's rows: rb + 32 u, u < nr
            const C* wq = wcs + quad * 4 * PNB;
            const C* vq = vcs + quad * 4 * PNB;
            C acc[RL][4];
#pragma unroll
            for (int u = 0; u < RL; ++u)
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) acc[u][cc] = C{0, 0};
            for (int qq = 0; qq < c; ++qq) {
              C vr[RL], wr[RL];
#pragma unroll
              for (int u = 0; u < RL; ++u)
                if (u < nr) {
                  vr[u] = Vs[(rb + 32 * u) * (PNB + 1) + qq];
                  wr[u] = Ws[(rb + 32 * u) * (PNB + 1) + qq];
                }
#pragma unroll
              for (int cc = 0; cc < 4; ++cc) {
                const C wcv = wq[cc * PNB + qq], vcv = vq[cc * PNB + qq];
#pragma unroll
                for (int u = 0; u < RL; ++u)
                  if (u < nr) acc[u][cc] = cfma(cfma(acc[u][cc], vr[u], wcv), wr[u], vcv);
              }
            }
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              const int q = quad * 4 + cc;
              if (q < ncb) {
                const int i = b + G * (cb2 + cb0 + q);
#pragma unroll
                for (int u = 0; u < RL; ++u) {
                  const int j = r0 + rb + 32 * u;
                  if (u < nr && j < n) {
                    C* aji = &p.a[(size_t)i * n + j];
                    *aji = csub(__ldcg(aji), acc[u][cc]);
                  }
                }
              }
            }
          }
        }
      }
      if (!grid_barrier(p.bar, G, gen, p.status, 1)) return;
      c = 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Compact WY factors and X <- Q X.
// ---------------------------------------------------------------------------

// T factor of reflector block blockIdx.x (reflectors b0 .. b0 + nb - 1, nb <= 32):
// H_b0 ... H_{b0+nb-1} = I - V T V^H, T upper triangular (forward, columnwise):
// T[r][r] = tau_r, T[0:s, s] = -tau_s T[0:s, 0:s] (V[:, 0:s]^H v_s).
template <typename T>
__global__ void __launch_bounds__(256) wy_t_kernel(const typename CxT<T>::C* a,
                                                   const typename CxT<T>::C* tau, int n,
                                                   typename CxT<T>::C* tfac) {
  using C = typename CxT<T>::C;
  __shared__ C S[PNB][PNB + 1];
  __shared__ C Tt[PNB][PNB + 1];
  __shared__ C Vc[32][PNB + 1];
  const int blk = blockIdx.x, b0 = blk * PNB, nr = n - 1, tid = threadIdx.x;
  const int nb = min(PNB, nr - b0);
  C acc[4] = {};
  for (int j0 = b0 + 1; j0 < n; j0 += 32) {
    __syncthreads();
    for (int e = tid; e < 32 * PNB; e += 256) {
      const int r = e / 32, jj = e % 32, j = j0 + jj;
      Vc[jj][r] = (r < nb && j < n && j >= b0 + r + 1) ? a[(size_t)(b0 + r) * n + j] : C{0, 0};
    }
    __syncthreads();
    for (int u = 0; u < 4; ++u) {
      const int e = tid + 256 * u, r = e / PNB, s = e % PNB;
      for (int jj = 0; jj < 32; ++jj) acc[u] = cadd(acc[u], cmul_ca(Vc[jj][r], Vc[jj][s]));
    }
  }
  for (int u = 0; u < 4; ++u) {
    const int e = tid + 256 * u;
    S[e / PNB][e % PNB] = acc[u];
    Tt[e / PNB][e % PNB] = C{0, 0};
  }
  __syncthreads();
  if (tid == 0)
    for (int r = 0; r < nb; ++r) Tt[r][r] = tau[b0 + r];
  __syncthreads();
  for (int s = 1; s < nb; ++s) {
    if (tid < s) {
      const int r = tid;
      C t = {0, 0};
      for (int q = r; q < s; ++q) t = cadd(t, cmul(Tt[r][q], S[q][s]));
      const C ts = tau[b0 + s];
      const C v = cmul(ts, t);
      Tt[r][s] = C{-v.x, -v.y};
    }
    __syncthreads();
  }
  for (int e = tid; e < PNB * PNB; e += 256) tfac[(size_t)blk * PNB * PNB + e] = Tt[e / PNB][e % PNB];
}

// X <- Q X: CTA owns CT columns of X (n x m, column-major) and applies the blocks
// from the last to the first: X -= V (T (V^H X)), 512 threads.  The CTA's n x CT tile
// of X stays in shared memory for the whole product when it fits (`resident`), so
// only the reflectors stream from L2.  V is staged in chunks of AR rows, double
// buffered: each thread loads its part of chunk c+1 into registers while chunk c is
// used.  V^H X: thread (part, r, cc) sums the rows part, part + AQP, ... of a chunk;
// the AQP parts are added at the end of the block.  X -= V W: an element per thread.
constexpr int CT = 4;
constexpr int AQ_THREADS = 512;
constexpr int AQP = AQ_THREADS / (PNB * CT);  // row parts of the V^H X sums

template <typename T>
__host__ __device__ constexpr int aq_rows() {
  return sizeof(T) == 4 ? 128 : 64;
}

template <typename T>
size_t aq_smem(int n, bool resident) {
  using C = typename CxT<T>::C;
  return sizeof(C) * (2 * (size_t)aq_rows<T>() * (PNB + 1) + PNB * (PNB + 1) +
                      (size_t)AQP * PNB * CT + PNB * CT + (resident ? (size_t)n * CT : 0));
}

template <typename T>
__global__ void __launch_bounds__(AQ_THREADS) apply_q_kernel(const typename CxT<T>::C* a, int n,
                                                             const typename CxT<T>::C* tfac,
                                                             typename CxT<T>::C* x, int m,
                                                             int resident) {
  using C = typename CxT<T>::C;
  constexpr int AR = aq_rows<T>();
  constexpr int PER = AR * PNB / AQ_THREADS;  // staged V elements per thread and chunk
  extern __shared__ __align__(16) unsigned char aq_raw[];
  C* Vb = (C*)aq_raw;               // [2][AR][PNB + 1]
  C* Tt = Vb + 2 * AR * (PNB + 1);  // [PNB][PNB + 1]
  C* Wp = Tt + PNB * (PNB + 1);     // [AQP][PNB][CT]
  C* W2 = Wp + AQP * PNB * CT;      // [PNB][CT]
  C* xr = W2 + PNB * CT;            // [n][CT] when resident
  const int tid = threadIdx.x, c0 = blockIdx.x * CT;
  const int nr = n - 1, nblk = (nr + PNB - 1) / PNB;
  const int cc1 = tid % CT, r1 = (tid / CT) % PNB, part1 = tid / (CT * PNB);
  const bool in1 = c0 + cc1 < m;
  auto xat = [&](int j, int cc) -> C& { return resident ? xr[(size_t)j * CT + cc]
                                                        : x[(size_t)(c0 + cc) * n + j]; };
  if (resident)
    for (int e = tid; e < n * CT; e += AQ_THREADS) {
      const int cc = e / n, j = e % n;
      xr[(size_t)j * CT + cc] = c0 + cc < m ? x[(size_t)(c0 + cc) * n + j] : C{0, 0};
    }
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int b0 = blk * PNB, nb = min(PNB, nr - b0);
    const int jb = b0 + 1, nch = (n - jb + AR - 1) / AR;
    // V(j, r) of chunk ch for this thread's element u (r = e / AR, jj = e % AR)
    auto vload = [&](int ch, int u) -> C {
      const int e = tid + AQ_THREADS * u, r = e / AR, j = jb + ch * AR + e % AR;
      return (r < nb && j < n && j >= b0 + r + 1) ? a[(size_t)(b0 + r) * n + j] : C{0, 0};
    };
    auto vstore = [&](int buf, int u, C v) {
      const int e = tid + AQ_THREADS * u;
      Vb[((size_t)buf * AR + e % AR) * (PNB + 1) + e / AR] = v;
    };
    __syncthreads();
    for (int e = tid; e < PNB * PNB; e += AQ_THREADS)
      Tt[(e / PNB) * (PNB + 1) + e % PNB] = tfac[(size_t)blk * PNB * PNB + e];
    // ---- W = V^H X
    C acc = {0, 0};
    C pf[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) vstore(0, u, vload(0, u));
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      if (ch + 1 < nch) {
#pragma unroll
        for (int u = 0; u < PER; ++u) pf[u] = vload(ch + 1, u);
      }
      __syncthreads();
      const C* V = Vb + (size_t)buf * AR * (PNB + 1);
      const int j0 = jb + ch * AR, jmax = min(AR, n - j0);
      if (in1)
        for (int jj = part1; jj < jmax; jj += AQP)
          acc = cadd(acc, cmul_ca(V[jj * (PNB + 1) + r1], xat(j0 + jj, cc1)));
      if (ch + 1 < nch) {
#pragma unroll
        for (int u = 0; u < PER; ++u) vstore(buf ^ 1, u, pf[u]);
      }
    }
    Wp[(part1 * PNB + r1) * CT + cc1] = acc;
    __syncthreads();
    if (tid < PNB * CT) {
      C t = Wp[tid];
      for (int q = 1; q < AQP; ++q) t = cadd(t, Wp[q * PNB * CT + tid]);
      W2[tid] = t;  // V^H X, replaced by T (V^H X) below
    }
    __syncthreads();
    C tw = {0, 0};
    if (tid < PNB * CT) {
      const int r = tid / CT, cc = tid % CT;
      for (int q = r; q < PNB; ++q) tw = cadd(tw, cmul(Tt[r * (PNB + 1) + q], W2[q * CT + cc]));
    }
    __syncthreads();
    if (tid < PNB * CT) W2[tid] = tw;
    // ---- X -= V (T W)
#pragma unroll
    for (int u = 0; u < PER; ++u) vstore(0, u, vload(0, u));
    for (int ch = 0; ch < nch; ++ch) {
      const int buf = ch & 1;
      if (ch + 1 < nch) {
#pragma unroll
        for (int u = 0; u < PER; ++u) pf[u] = vload(ch + 1, u);
      }
      __syncthreads();
      const C* V = Vb + (size_t)buf * AR * (PNB + 1);
      const int j0 = jb + ch * AR;
      for (int e = tid; e < AR * CT; e += AQ_THREADS) {
        const int jj = e % AR, cc = e / AR, j = j0 + jj;
        if (j < n && c0 + cc < m) {
          C t = {0, 0};
#pragma unroll 8
          for (int r = 0; r < PNB; ++r) t = cadd(t, cmul(V[jj * (PNB + 1) + r], W2[r * CT + cc]));
          C& xv = xat(j, cc);
          xv = csub(xv, t);
        }
      }
      if (ch + 1 < nch) {
#pragma unroll
        for (int u = 0; u < PER; ++u) vstore(buf ^ 1, u, pf[u]);
      }
    }
  }
  __syncthreads();
  if (resident)
    for (int e = tid; e < n * CT; e += AQ_THREADS) {
      const int cc = e / n, j = e % n;
      if (c0 + cc < m) x[(size_t)(c0 + cc) * n + j] = xr[(size_t)j * CT + cc];
    }
}

// ---------------------------------------------------------------------------
// Cyclic two-sided Jacobi (FP64) with round-robin pairs of M = m + (m & 1)
// players: round r pairs (M-1, r) and ((r + k) mod (M-1), (r - k) mod (M-1)),
// k = 1 .. M/2 - 1.  With m odd, the player paired with the padding index m takes
// no rotation that round (its column still takes the other pairs' row rotations).
// Per round:
//   1. the CTA owning pair k (k = b, b + G, ...) computes its rotation from
//      a = G_pp, c = G_qq, g = G_pq = |g| e^{i phi}: zeta = (c - a) / (2 |g|),
//      t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), cs = 1/sqrt(1 + t^2),
//      sn = t cs; J = diag(1, e^{-i phi}) [[cs, sn], [-sn, cs]];      barrier
//   2. it rotates its columns p, q of G and Y (G J, Y J), then applies every
//      pair's row rotation (J^H) to those two columns, and zeroes G_pq;  barrier
//   (Every CTA computing every pair's rotation from double-buffered inputs, one
//   barrier per round, measured slower: the rotations' FP64 square roots and
//   divisions then run G times over.)
// Rotations with |g| <= 1e-300 or |g| <= eps sqrt(|a c|) are skipped.  A sweep
// is M - 1 rounds; sweeps stop when no pair of a sweep needed a rotation.
// ---------------------------------------------------------------------------
constexpr int JT = 512;
constexpr int MAX_JM = 4096;  // largest m (rotation parameters are staged in shared memory)

__device__ __forceinline__ void pair_of(int M, int r, int k, int& p, int& q) {
  int a, b;
  if (k == 0) {
    a = M - 1;
    b = r;
  } else {
    a = (r + k) % (M - 1);
    b = (r - k + (M - 1)) % (M - 1);
  }
  p = min(a, b);
  q = max(a, b);
}

struct JacArgs {
  cplx* g;
  int m;
  cplx* y;
  double* prm;   // [M/2][4]: cs, sn, Re e^{-i phi}, Im e^{-i phi}
  double* part;  // [grid]: rotations needed in the sweep
  unsigned* bar;
  int* status;
  int max_sweeps;
};

__global__ void __launch_bounds__(JT, 1) jacobi_kernel(JacArgs p) {
  extern __shared__ double jsm[];  // [M/2][4]
  __shared__ int stop_s;
  const int m = p.m, M = m + (m & 1), np = M / 2, G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x;
  unsigned gen = 0;
  const double eps = 2.220446049250313e-16;
  // largest relative off-diagonal |g_pq| / sqrt(|g_pp g_qq|) this thread rotated away in
  // the current sweep: Jacobi converges quadratically, so once a whole sweep needed
  // only rotations below kConverged the matrix it leaves is diagonal to ~kConverged^2
  double offmax = 0.0;
  constexpr double kConverged = 1e-8;
  for (int sweep = 0; sweep < p.max_sweeps; ++sweep) {
    for (int r = 0; r < M - 1; ++r) {
      // 1. rotation parameters of this CTA's pairs (the FP64 pipe is narrow: each pair's
      //    are computed once, by its owner, and published)
      for (int k = b + G * tid; k < np; k += G * JT) {
        int pp, qq;
        pair_of(M, r, k, pp, qq);
        double cs = 1.0, sn = 0.0, er = 1.0, ei = 0.0;
        if (qq < m) {
          const double a = ldcg_c(&p.g[(size_t)pp * m + pp]).re;
          const double c = ldcg_c(&p.g[(size_t)qq * m + qq]).re;
          const cplx gpq = ldcg_c(&p.g[(size_t)qq * m + pp]);
          const double beta = hypot(gpq.re, gpq.im);
          const double ref = sqrt(fabs(a * c));
          if (beta > 1e-300 && beta > eps * ref) {
            offmax = fmax(offmax, ref > 0.0 ? beta / ref : 1.0);
            const double zeta = (c - a) / (2.0 * beta);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            cs = 1.0 / sqrt(1.0 + t * t);
            sn = t * cs;
            er = gpq.re / beta;
            ei = -gpq.im / beta;
          }
        }
        double* o = p.prm + 4 * (size_t)k;
        o[0] = cs;
        o[1] = sn;
        o[2] = er;
        o[3] = ei;
      }
      if (!grid_barrier(p.bar, G, gen, p.status, 2)) return;
      for (int e = tid; e < 4 * np; e += JT) jsm[e] = __ldcg(&p.prm[e]);
      __syncthreads();
      // 2. columns p, q of this CTA's pairs: G J and Y J, then J^H on those columns
      for (int k = b; k < np; k += G) {
        int pp, qq;
        pair_of(M, r, k, pp, qq);
        // with m odd, the player paired with the padding index m idles this round: its
        // column takes no column rotation but still every pair's row rotation
        const bool idle = qq >= m;
        const double cs = jsm[4 * k], sn = jsm[4 * k + 1], er = jsm[4 * k + 2], ei = jsm[4 * k + 3];
        if (idle || (sn == 0.0 && er == 1.0 && ei == 0.0)) {
          // no rotation of these columns; their rows still rotate below
        } else {
          for (int mat = 0; mat < 2; ++mat) {
            cplx* X = mat == 0 ? p.g : p.y;
            for (int i = tid; i < m; i += JT) {
              const cplx xp = ldcg_c(&X[(size_t)pp * m + i]), xq = ldcg_c(&X[(size_t)qq * m + i]);
              // e^{-i phi} xq
              const cplx eq = {er * xq.re - ei * xq.im, er * xq.im + ei * xq.re};
              X[(size_t)pp * m + i] = cplx{cs * xp.re - sn * eq.re, cs * xp.im - sn * eq.im};
              X[(size_t)qq * m + i] = cplx{sn * xp.re + cs * eq.re, sn * xp.im + cs * eq.im};
            }
          }
        }
        __syncthreads();
        // rows: (J^H X)[p'] = cs X[p'] - sn e^{i phi'} X[q'], (J^H X)[q'] = sn X[p'] + cs e^{i phi'} X[q']
        for (int col = 0; col < (idle ? 1 : 2); ++col) {
          cplx* X = p.g + (size_t)(col == 0 ? pp : qq) * m;
          for (int k2 = tid; k2 < np; k2 += JT) {
            int p2, q2;
            pair_of(M, r, k2, p2, q2);
            if (q2 >= m) continue;
            const double c2 = jsm[4 * k2], s2 = jsm[4 * k2 + 1], er2 = jsm[4 * k2 + 2],
                         ei2 = -jsm[4 * k2 + 3];  // e^{+i phi'}
            if (s2 == 0.0 && er2 == 1.0 && ei2 == 0.0) continue;
            const cplx xp = ldcg_c(&X[p2]), xq = ldcg_c(&X[q2]);
            const cplx eq = {er2 * xq.re - ei2 * xq.im, er2 * xq.im + ei2 * xq.re};
            X[p2] = cplx{c2 * xp.re - s2 * eq.re, c2 * xp.im - s2 * eq.im};
            X[q2] = cplx{s2 * xp.re + c2 * eq.re, s2 * xp.im + c2 * eq.im};
          }
        }
        __syncthreads();
        if (tid == 0 && !idle && !(sn == 0.0 && er == 1.0 && ei == 0.0)) {
          p.g[(size_t)qq * m + pp] = cplx{0.0, 0.0};
          p.g[(size_t)pp * m + qq] = cplx{0.0, 0.0};
          p.g[(size_t)pp * m + pp].im = 0.0;
          p.g[(size_t)qq * m + qq].im = 0.0;
        }
      }
      if (!grid_barrier(p.bar, G, gen, p.status, 2)) return;
    }
    // stop once the sweep needed no rotation above kConverged (in any CTA)
    __syncthreads();
    {
      __shared__ double cmax[JT / 32];
      double v = offmax;
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      if ((tid & 31) == 0) cmax[tid >> 5] = v;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < JT / 32; ++w) s = fmax(s, cmax[w]);
        p.part[b] = s;
      }
    }
    offmax = 0.0;
    if (!grid_barrier(p.bar, G, gen, p.status, 2)) return;
    if (tid == 0) {
      double s = 0.0;
      for (int g = 0; g < G; ++g) s = fmax(s, __ldcg(&p.part[g]));
      stop_s = s < kConverged;
    }
    __syncthreads();
    if (stop_s) break;
    if (!grid_barrier(p.bar, G, gen, p.status, 2)) return;
  }
}

// rank of each diagonal entry (ascending, ties by index), theta, and Y's columns
// permuted into that order (one CTA per output column for the copy)
__global__ void jacobi_rank_kernel(const cplx* g, int m, int* rank, double* theta) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const double v = g[(size_t)i * m + i].re;
    int r = 0;
    for (int j = 0; j < m; ++j) {
      const double u = g[(size_t)j * m + j].re;
      r += (u < v) || (u == v && j < i);
    }
    rank[i] = r;
    theta[r] = v;
  }
}

__global__ void permute_cols_kernel(const cplx* src, int m, const int* rank, cplx* dst) {
  const int i = blockIdx.x;  // source column
  const int r = rank[i];
  for (int e = threadIdx.x; e < m; e += blockDim.x) dst[(size_t)r * m + e] = src[(size_t)i * m + e];
}

__global__ void identity_kernel(cplx* y, int m) {
  const long tot = (long)m * m;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < tot;
       e += (long)gridDim.x * blockDim.x)
    y[e] = cplx{e / m == e % m ? 1.0 : 0.0, 0.0};
}

// ---------------------------------------------------------------------------
// FP64 complex GEMM: 32 x 32 output tile per CTA, 2 x 2 per thread, K in chunks of 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ cplx load_op(const cplx* a, int lda, char op, int i, int k, int rows,
                                        int cols) {
  // element (i, k) of op(A), op(A) rows x cols
  if (i >= rows || k >= cols) return cplx{0.0, 0.0};
  if (op == 'N') return a[(size_t)k * lda + i];
  const cplx v = a[(size_t)i * lda + k];
  return op == 'C' ? cplx{v.re, -v.im} : v;
}

// C tile (TILE x TILE; TILE = 32: 2 x 2 outputs per thread, 16: one) of
// alpha op(A) op(B) + beta C.  tri bit 0: op(B) upper triangular (its rows k > j are
// zero), bit 1: op(A) upper triangular (its columns k < i are zero); the K range of a
// tile is cut to where both are nonzero.
template <int TILE>
__global__ void __launch_bounds__(256) gemm_z_kernel(char opa, char opb, int m, int n, int k,
                                                     cplx alpha, const cplx* a, int lda,
                                                     const cplx* b, int ldb, cplx beta, cplx* c,
                                                     int ldc, int tri) {
  constexpr int R = TILE / 16;
  __shared__ cplx As[TILE][17];      // As[i][kk]
  __shared__ cplx Bs[16][TILE + 1];  // Bs[kk][j]
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int i0 = blockIdx.x * TILE, j0 = blockIdx.y * TILE;
  const int kbeg = (tri & 2) ? (i0 / 16) * 16 : 0;
  const int kend = (tri & 1) ? min(k, j0 + TILE) : k;
  cplx acc[R][R] = {};
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = tid; e < TILE * 16; e += 256) {
      const int ii = e % TILE, kk = e / TILE;
      As[ii][kk] = load_op(a, lda, opa, i0 + ii, k0 + kk, m, k);
    }
    for (int e = tid; e < 16 * TILE; e += 256) {
      const int kk = e % 16, jj = e / 16;
      Bs[kk][jj] = load_op(b, ldb, opb, k0 + kk, j0 + jj, k, n);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
#pragma unroll
      for (int y = 0; y < R; ++y) {
        const cplx av = As[R * ty + y][kk];
#pragma unroll
        for (int x = 0; x < R; ++x) {
          const cplx bv = Bs[kk][R * tx + x];
          acc[y][x].re = fma(av.re, bv.re, fma(-av.im, bv.im, acc[y][x].re));
          acc[y][x].im = fma(av.re, bv.im, fma(av.im, bv.re, acc[y][x].im));
        }
      }
    }
    __syncthreads();
  }
  for (int y = 0; y < R; ++y)
    for (int x = 0; x < R; ++x) {
      const int i = i0 + R * ty + y, j = j0 + R * tx + x;
      if (i >= m || j >= n) continue;
      const cplx v = acc[y][x];
      cplx out = {alpha.re * v.re - alpha.im * v.im, alpha.re * v.im + alpha.im * v.re};
      if (beta.re != 0.0 || beta.im != 0.0) {
        const cplx o = c[(size_t)j * ldc + i];
        out.re += beta.re * o.re - beta.im * o.im;
        out.im += beta.re * o.im + beta.im * o.re;
      }
      c[(size_t)j * ldc + i] = out;
    }
}

// Inverse of each 32 x 32 diagonal tile (the last one ragged) of the upper-triangular
// n x n R (column-major, leading dimension ld), in place, zero below the diagonal:
// blockIdx.x = tile.  Backward elimination of the identity: for j from the last row
// up, row j of X = R^-1 is scaled by 1 / R_jj and eliminated from the rows above.
__global__ void __launch_bounds__(256) trinv_tiles_kernel(cplx* r, int n, int ld) {
  __shared__ cplx t[32][33];
  __shared__ cplx u[32][33];
  __shared__ cplx rd;
  const int tid = threadIdx.x, o = 32 * blockIdx.x, kb = min(32, n - o);
  for (int e = tid; e < 32 * 32; e += blockDim.x) {
    const int i = e % 32, j = e / 32;
    t[i][j] = (i < kb && j < kb && i <= j) ? r[(size_t)(o + j) * ld + o + i] : cplx{0.0, 0.0};
    u[i][j] = cplx{(i == j && i < kb) ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  for (int j = kb - 1; j >= 0; --j) {
    if (tid == 0) {
      const cplx d = t[j][j];
      const double dd = d.re * d.re + d.im * d.im;
      rd = cplx{d.re / dd, -d.im / dd};
    }
    __syncthreads();
    if (tid >= j && tid < kb) {
      const cplx x = u[j][tid], q = rd;
      u[j][tid] = cplx{x.re * q.re - x.im * q.im, x.re * q.im + x.im * q.re};
    }
    __syncthreads();
    const int w = kb - j;  // columns c = j .. kb-1 of the rows i < j
    for (int e = tid; e < j * w; e += blockDim.x) {
      const int i = e / w, c = j + e % w;
      const cplx a = t[i][j], x = u[j][c];
      u[i][c].re -= a.re * x.re - a.im * x.im;
      u[i][c].im -= a.re * x.im + a.im * x.re;
    }
    __syncthreads();
  }
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e % kb, j = e / kb;
    r[(size_t)(o + j) * ld + o + i] = i <= j ? u[i][j] : cplx{0.0, 0.0};
  }
}

// Per-device cooperative-launch limits.
struct CoopLimits {
  int sms = 0;
  bool hetrd_f = false, hetrd_d = false, jac = false;
};
constexpr int kMaxDev = 64;
CoopLimits g_coop[kMaxDev];
std::mutex g_coop_mutex;

rpa_status coop_setup(int& sms, std::string& err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    err = "no CUDA device";
    return RPA_ECUDA;
  }
  std::lock_guard<std::mutex> lk(g_coop_mutex);
  CoopLimits& L = g_coop[dev];
  if (L.sms == 0) {
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&L.sms, cudaDevAttrMultiProcessorCount, dev);
    if (!coop || L.sms <= 0) {
      err = "device without cooperative launch";
      L.sms = 0;
      return RPA_ECUDA;
    }
    if (cudaFuncSetAttribute(hetrd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hetrd_smem<float>()) != cudaSuccess ||
        cudaFuncSetAttribute(hetrd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hetrd_smem<double>()) != cudaSuccess ||
        cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(double) * 4 * (MAX_JM / 2))) != cudaSuccess) {
      (void)cudaGetLastError();
      err = "cudaFuncSetAttribute for the dense eigensolver kernels failed";
      L.sms = 0;
      return RPA_ECUDA;
    }
  }
  sms = L.sms;
  return RPA_OK;
}

template <typename T>
int hetrd_grid(int n, int sms) {
  const int need = (n + MAXOWN - 1) / MAXOWN;
  const int want = std::max(need, std::min(sms, std::max(1, n / 16)));
  return std::min(sms, want);
}

}  // namespace

rpa_status hetrd_alloc(HetrdWork& w, int n_max, size_t elem, std::string& err) {
  int sms = 0;
  rpa_status s = coop_setup(sms, err);
  if (s != RPA_OK) return s;
  w.n_max = n_max;
  w.elem = elem;
  w.grid = std::min(sms, MAXG);
  if ((long)MAXOWN * w.grid < n_max) {
    err = "dense eigensolver: matrix too large for the persistent grid";
    return RPA_EINVAL;
  }
  auto al = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    return true;
  };
  const size_t n = n_max;
  if (!al(&w.vp, n * PNB * elem) || !al(&w.wp, n * PNB * elem) || !al(&w.xcol, n * elem) ||
      !al(&w.ycol, n * elem) || !al(&w.part, (size_t)sms * PL * elem) ||
      !al(&w.part2, (size_t)sms * elem) ||
      !al((void**)&w.bar, bar_words(w.grid) * sizeof(unsigned)) ||
      !al((void**)&w.status, sizeof(int))) {
    hetrd_free(w);
    err = "dense eigensolver: cudaMalloc failed";
    return RPA_ENOMEM;
  }
  if (cudaMemset(w.status, 0, sizeof(int)) != cudaSuccess) {
    hetrd_free(w);
    err = "dense eigensolver: cudaMemset failed";
    return RPA_ECUDA;
  }
  return RPA_OK;
}

void hetrd_free(HetrdWork& w) {
  void* b[] = {w.vp, w.wp, w.xcol, w.ycol, w.part, w.part2, w.bar, w.status};
  for (void* p : b)
    if (p) cudaFree(p);
  w = HetrdWork{};
}

template <typename T>
rpa_status hetrd(HetrdWork& w, void* a, int n, T* d, T* e, void* tau, cudaStream_t st,
                 std::string& err, int* launches) {
  using C = typename CxT<T>::C;
  if (n < 1) return RPA_OK;
  if (n > w.n_max || sizeof(C) != w.elem) {
    err = "dense eigensolver: matrix outside the workspace";
    return RPA_EINVAL;
  }
  int sms = 0;
  rpa_status s = coop_setup(sms, err);
  if (s != RPA_OK) return s;
  const int G = hetrd_grid<T>(n, std::min(std::min(sms, w.grid), MAXG));
  if (cudaMemsetAsync(w.bar, 0, bar_words(w.grid) * sizeof(unsigned), st) != cudaSuccess) {
    err = "dense eigensolver: barrier reset failed";
    return RPA_ECUDA;
  }
  HetrdArgs<T> args{(C*)a, n, d, e, (C*)tau, (C*)w.vp, (C*)w.wp, (C*)w.xcol, (C*)w.ycol,
                    (C*)w.part, (C*)w.part2, w.bar, w.status};
  void* kargs[] = {&args};
  const cudaError_t ce = cudaLaunchCooperativeKernel((const void*)hetrd_kernel<T>, dim3(G),
                                                     dim3(HT), kargs, hetrd_smem<T>(), st);
  if (ce != cudaSuccess) {
    (void)cudaGetLastError();
    err = std::string("hetrd launch: ") + cudaGetErrorString(ce);
    return RPA_ECUDA;
  }
  if (launches) *launches += 1;
  return RPA_OK;
}

template rpa_status hetrd<float>(HetrdWork&, void*, int, float*, float*, void*, cudaStream_t,
                                 std::string&, int*);
template rpa_status hetrd<double>(HetrdWork&, void*, int, double*, double*, void*, cudaStream_t,
                                  std::string&, int*);

template <typename T>
rpa_status apply_q(const void* a, const void* tau, int n, void* x, int m, void* tfac,
                   cudaStream_t st, std::string& err, int* launches) {
  using C = typename CxT<T>::C;
  if (n < 2 || m < 1) return RPA_OK;
  const int nblk = (n - 1 + PNB - 1) / PNB;
  wy_t_kernel<T><<<nblk, 256, 0, st>>>((const C*)a, (const C*)tau, n, (C*)tfac);
  // the X tile resident in shared memory when everything fits in 227 KB
  const bool resident = aq_smem<T>(n, true) <= 227 * 1024;
  const size_t smem = aq_smem<T>(n, resident);
  if (cudaFuncSetAttribute(apply_q_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    (void)cudaGetLastError();
    err = "apply_q: shared memory attribute";
    return RPA_ECUDA;
  }
  apply_q_kernel<T><<<(m + CT - 1) / CT, AQ_THREADS, smem, st>>>(
      (const C*)a, n, (const C*)tfac, (C*)x, m, resident ? 1 : 0);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("apply_q launch: ") + cudaGetErrorString(ce);
    return RPA_ECUDA;
  }
  if (launches) *launches += 2;
  return RPA_OK;
}

template rpa_status apply_q<float>(const void*, const void*, int, void*, int, void*,
                                   cudaStream_t, std::string&, int*);
template rpa_status apply_q<double>(const void*, const void*, int, void*, int, void*,
                                    cudaStream_t, std::string&, int*);

rpa_status jacobi_alloc(JacobiWork& w, int m_max, std::string& err) {
  int sms = 0;
  rpa_status s = coop_setup(sms, err);
  if (s != RPA_OK) return s;
  if (m_max > MAX_JM) {
    err = "Jacobi eigensolver: matrix larger than " + std::to_string(MAX_JM);
    return RPA_EINVAL;
  }
  w.m_max = m_max;
  w.grid = sms;
  const size_t M = (size_t)m_max + 1;
  if (cudaMalloc(&w.prm, 8 * (M / 2 + 1) * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&w.part, (size_t)sms * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&w.bar, bar_words(w.grid) * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&w.status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&w.perm, M * sizeof(int)) != cudaSuccess ||
      cudaMemset(w.status, 0, sizeof(int)) != cudaSuccess) {
    (void)cudaGetLastError();
    jacobi_free(w);
    err = "Jacobi eigensolver: cudaMalloc failed";
    return RPA_ENOMEM;
  }
  return RPA_OK;
}

void jacobi_free(JacobiWork& w) {
  void* b[] = {w.prm, w.part, w.bar, w.status, w.perm};
  for (void* p : b)
    if (p) cudaFree(p);
  w = JacobiWork{};
}

rpa_status jacobi(JacobiWork& w, cplx* g, int m, double* theta, cplx* y, cplx* ywork,
                  cudaStream_t st, std::string& err, int* launches) {
  if (m < 1) return RPA_OK;
  if (m > w.m_max) {
    err = "Jacobi eigensolver: matrix outside the workspace";
    return RPA_EINVAL;
  }
  int sms = 0;
  rpa_status s = coop_setup(sms, err);
  if (s != RPA_OK) return s;
  const int M = m + (m & 1), np = M / 2;
  const int G = std::max(1, std::min(std::min(sms, w.grid), np / 2));
  identity_kernel<<<std::min(4096, (m * m + 255) / 256), 256, 0, st>>>(ywork, m);
  if (cudaMemsetAsync(w.bar, 0, bar_words(w.grid) * sizeof(unsigned), st) != cudaSuccess) {
    err = "Jacobi eigensolver: barrier reset failed";
    return RPA_ECUDA;
  }
  JacArgs args{g, m, ywork, w.prm, w.part, w.bar, w.status, 12};
  void* kargs[] = {&args};
  cudaError_t ce = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(G), dim3(JT),
                                               kargs, sizeof(double) * 4 * np, st);
  if (ce != cudaSuccess) {
    (void)cudaGetLastError();
    err = std::string("Jacobi launch: ") + cudaGetErrorString(ce);
    return RPA_ECUDA;
  }
  jacobi_rank_kernel<<<(m + 127) / 128, 128, 0, st>>>(g, m, w.perm, theta);
  permute_cols_kernel<<<m, 256, 0, st>>>(ywork, m, w.perm, y);
  ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("Jacobi sort: ") + cudaGetErrorString(ce);
    return RPA_ECUDA;
  }
  if (launches) *launches += 4;
  return RPA_OK;
}

static rpa_status gemm_z_tri(char opa, char opb, int m, int n, int k, cplx alpha,
                             const cplx* a, int lda, const cplx* b, int ldb, cplx beta, cplx* c,
                             int ldc, int tri, cudaStream_t st, std::string& err,
                             int* launches) {
  if (m < 1 || n < 1) return RPA_OK;
  // 16 x 16 tiles when 32 x 32 ones would leave SMs idle (the FP64 pipe is narrow)
  const bool small = (long)((m + 31) / 32) * ((n + 31) / 32) < 152;
  const int tile = small ? 16 : 32;
  const dim3 grid((m + tile - 1) / tile, (n + tile - 1) / tile);
  if (grid.y > 65535) {
    err = "gemm_z: n too large";
    return RPA_EINVAL;
  }
  if (small)
    gemm_z_kernel<16><<<grid, 256, 0, st>>>(opa, opb, m, n, k, alpha, a, lda, b, ldb, beta, c,
                                            ldc, tri);
  else
    gemm_z_kernel<32><<<grid, 256, 0, st>>>(opa, opb, m, n, k, alpha, a, lda, b, ldb, beta, c,
                                            ldc, tri);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("gemm_z launch: ") + cudaGetErrorString(ce);
    return RPA_ECUDA;
  }
  if (launches) *launches += 1;
  return RPA_OK;
}

rpa_status gemm_z(char opa, char opb, int m, int n, int k, cplx alpha, const cplx* a, int lda,
                  const cplx* b, int ldb, cplx beta, cplx* c, int ldc, cudaStream_t st,
                  std::string& err, int* launches) {
  return gemm_z_tri(opa, opb, m, n, k, alpha, a, lda, b, ldb, beta, c, ldc, 0, st, err,
                    launches);
}

// Off-diagonal blocks of R^-1 by recursive doubling, the diagonal 32 x 32 tiles
// already inverted: [R11 R12; 0 R22]^-1 = [X11, -X11 R12 X22; 0, X22].  Splits fall
// on multiples of 32, so the leaves are the inverted tiles.
static rpa_status trinv_blocks(cplx* r, int n, int ld, cplx* work, cudaStream_t st,
                               std::string& err, int* launches) {
  if (n <= 32) return RPA_OK;
  const int n1 = ((n / 2 + 31) / 32) * 32, n2 = n - n1;
  rpa_status s;
  if ((s = trinv_blocks(r, n1, ld, work, st, err, launches)) != RPA_OK) return s;
  if ((s = trinv_blocks(r + (size_t)n1 * ld + n1, n2, ld, work, st, err, launches)) != RPA_OK)
    return s;
  // work (n1 x n2) = R12 X22 (X22 upper triangular); X12 = -X11 work (X11 upper)
  cplx* r12 = r + (size_t)n1 * ld;
  if ((s = gemm_z_tri('N', 'N', n1, n2, n2, cplx{1.0, 0.0}, r12, ld, r + (size_t)n1 * ld + n1,
                      ld, cplx{0.0, 0.0}, work, n1, 1, st, err, launches)) != RPA_OK)
    return s;
  return gemm_z_tri('N', 'N', n1, n2, n1, cplx{-1.0, 0.0}, r, ld, work, n1, cplx{0.0, 0.0}, r12,
                    ld, 2, st, err, launches);
}

rpa_status trinv_upper(cplx* r, int n, int ld, cplx* work, cudaStream_t st, std::string& err,
                       int* launches) {
  if (n < 1) return RPA_OK;
  trinv_tiles_kernel<<<(n + 31) / 32, 256, 0, st>>>(r, n, ld);
  const cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) {
    err = std::string("trinv launch: ") + cudaGetErrorString(ce);
    return RPA_ECUDA;
  }
  if (launches) *launches += 1;
  return trinv_blocks(r, n, ld, work, st, err, launches);
}

}  // namespace dense
}  // namespace rpa
