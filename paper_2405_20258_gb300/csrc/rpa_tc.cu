// Tensor-core (tcgen05) contractions of the mixed-precision path: exact
// digit-sliced BF16 GEMM with TMEM accumulation and a double-float epilogue,
// plus the HBM-bound kernels that cut FP64 operands into digit planes.
//
// GEMM kernel roles (320 threads, one output tile of 128 x 64 per CTA):
//   warp 0      TMA producer: per 64-wide K-tile, all S digit planes of the B
//               tile (double-buffered) and the S digit planes of the A tile
//               through a 4-stage ring;
//   warp 1      TMEM allocation and the single MMA-issuing thread: for every
//               slice pair (s, t) with s + t <= S-1, four kind::f16 MMAs
//               (K = 16 each) into the level accumulator L = s + t;
//   warps 2..9  epilogue: at the end of each drain interval, read the S level
//               accumulators (exact integers) from TMEM, scale by 2^-8L and add
//               them into per-thread double-float registers (one TMEM lane and
//               32 columns per thread); finally apply the row scales and write
//               complex FP64 results.
// Every mbarrier wait is bounded (about 2 s of SM clock): on expiry the CTA
// raises a flag in the status word, stops issuing, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "rpa_tc.h"

namespace rpa {
namespace tc {
namespace {

constexpr int BM = 128;  // A rows per tile = TMEM lanes = MMA M
constexpr int BN = 64;   // B rows per tile = MMA N
constexpr int BK = 64;   // K elements per tile: 128 bytes of BF16, one 128B swizzle row
constexpr int NA = 4;    // A ring depth
constexpr int THREADS = 320;  // producer, MMA, 8 epilogue warps
constexpr uint32_t A_TILE = BM * BK * 2;  // 16 KB
constexpr uint32_t B_TILE = BN * BK * 2;  // 8 KB
constexpr long long WAIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz

// kind::f16 instruction descriptor: D = F32 (bits 4-5), A = B = BF16 (bits 7-9,
// 10-12), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

enum : int {
  ERR_WAIT_PRODUCER = 1,
  ERR_WAIT_MMA = 2,
  ERR_WAIT_EPILOGUE = 4,
};

struct GemmArgs {
  int S;              // digit slices per operand
  int K;              // padded K (multiple of BK)
  int kd_tiles;       // K-tiles per drain interval
  int k_per_split;    // K elements per split (multiple of BK)
  const int4* work;   // (tile_m, tile_n, batch, k_split)
  const int* ea;      // exponent per A row
  const int* eb;      // exponent per complex B row pair, [batch][eb_stride]
  int eb_stride;
  int a_rows, b_rows; // valid rows of A and B (B rows = 2 x complex columns)
  double alpha;
  double2* out;       // complex output
  long out_bstride, ld_row, ld_col;
  int conj, atomic;
  int stall;          // test hook: the producer issues nothing
  int* status;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on one phase of an mbarrier.  false: timed out (flag raised) or
// another role of this CTA aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* status,
                          int code) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_CYCLES) {
      *abort_flag = 1;
      atomicOr(status, code);
      return false;
    }
    __nanosleep(64);
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes with the
// 128-byte swizzle, 8-row groups 1024 bytes apart (SBO), version bits 46-48 = 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32; // stride byte offset
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;           // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 32 consecutive columns of FP32 from TMEM.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 2^k as a double (exact; ldexp outside the normal range).
__device__ __forceinline__ double pow2(int k) {
  if (k >= -1022 && k <= 1023) return __longlong_as_double((long long)(1023 + k) << 52);
  return ldexp(1.0, k);
}

// Knuth's two-sum: (hi, lo) += x with the rounding error of hi + x kept in lo.
__device__ __forceinline__ void dfloat_add(float& hi, float& lo, float x) {
  float s = __fadd_rn(hi, x);
  float bp = __fsub_rn(s, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__global__ void __launch_bounds__(THREADS, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const GemmArgs p) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_a[NA], empty_a[NA], full_b[2], empty_b[2];
  __shared__ __align__(8) uint64_t acc_full, acc_empty;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                         // NA x 16 KB
  uint8_t* sB = smem + NA * A_TILE;           // 2 x S x 8 KB
  const int S = p.S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 wk = p.work[blockIdx.x];
  const int tm = wk.x, tn = wk.y, batch = wk.z, ks = wk.w;
  const int k_begin = ks * p.k_per_split;
  const int k_end = min(p.K, k_begin + p.k_per_split);
  const int nkt = (k_end - k_begin) / BK;
  const int kdt = p.kd_tiles;
  const int niv = (nkt + kdt - 1) / kdt;
  const uint32_t ncols = S * BN <= 32 ? 32 : (S * BN <= 64 ? 64 : (S * BN <= 128 ? 128 : (S * BN <= 256 ? 256 : 512)));

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < NA; ++i) {
      mbar_init(&full_a[i], 1);
      mbar_init(&empty_a[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full_b[i], 1);
      mbar_init(&empty_b[i], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 8);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0 && !p.stall) {
      int ia = 0;
      for (int kt = 0; kt < nkt && !abort_flag; ++kt) {
        const int k0 = k_begin + kt * BK;
        const int bb = kt & 1;
        if (!mbar_wait(&empty_b[bb], ((kt >> 1) & 1) ^ 1, &abort_flag, p.status, ERR_WAIT_PRODUCER))
          break;
        mbar_expect_tx(&full_b[bb], S * B_TILE);
        for (int t = 0; t < S; ++t)
          tma_load_3d(sB + (bb * S + t) * B_TILE, &tmB, &full_b[bb], k0, tn * BN, batch * S + t);
        bool ok = true;
        for (int s = 0; s < S; ++s, ++ia) {
          const int slot = ia % NA;
          if (!mbar_wait(&empty_a[slot], ((ia / NA) & 1) ^ 1, &abort_flag, p.status,
                         ERR_WAIT_PRODUCER)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full_a[slot], A_TILE);
          tma_load_3d(sA + slot * A_TILE, &tmA, &full_a[slot], k0, tm * BM, s);
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int ia = 0;
      unsigned first = 0;
      for (int kt = 0; kt < nkt; ++kt) {
        if (kt % kdt == 0) {
          const int iv = kt / kdt;
          if (!mbar_wait(&acc_empty, (iv & 1) ^ 1, &abort_flag, p.status, ERR_WAIT_MMA)) break;
          tc_fence_after();
          first = (1u << S) - 1;
        }
        const int bb = kt & 1;
        if (!mbar_wait(&full_b[bb], (kt >> 1) & 1, &abort_flag, p.status, ERR_WAIT_MMA)) break;
        bool ok = true;
        for (int s = 0; s < S; ++s, ++ia) {
          const int slot = ia % NA;
          if (!mbar_wait(&full_a[slot], (ia / NA) & 1, &abort_flag, p.status, ERR_WAIT_MMA)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint64_t ad = smem_desc(smem_u32(sA + slot * A_TILE));
          for (int t = 0; t + s < S; ++t) {
            const int L = s + t;
            const uint64_t bd = smem_desc(smem_u32(sB + (bb * S + t) * B_TILE));
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t acc = (kk > 0 || !(first & (1u << L))) ? 1u : 0u;
              mma_bf16(tmem + L * BN, ad + 2 * kk, bd + 2 * kk, acc);
            }
            first &= ~(1u << L);
          }
          mma_commit(&empty_a[slot]);
        }
        if (!ok) break;
        mma_commit(&empty_b[bb]);
        if (kt % kdt == kdt - 1 || kt == nkt - 1) mma_commit(&acc_full);
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int q = warp & 3;              // TMEM lane quadrant of this warp
    const int h = (warp - 2) >> 2;       // which 32 of the 64 columns
    float hi[32], lo[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0.f;
    bool ok = true;
    for (int iv = 0; iv < niv; ++iv) {
      if (!mbar_wait(&acc_full, iv & 1, &abort_flag, p.status, ERR_WAIT_EPILOGUE)) {
        ok = false;
        break;
      }
      tc_fence_after();
      for (int L = 0; L < S; ++L) {
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + L * BN + 32 * h;
        const float sc = __int_as_float((127 - 8 * L) << 23);  // 2^-8L, exact
        uint32_t r[32];
        tmem_ld32(ta, r);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 32; ++c) dfloat_add(hi[c], lo[c], __uint_as_float(r[c]) * sc);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty);
    }
    if (ok) {
      const int row = tm * BM + q * 32 + lane;
      if (row < p.a_rows) {
        const int ea = p.ea[row];
        double2* out = p.out + (long)batch * p.out_bstride + (long)row * p.ld_row;
        const int* eb = p.eb + (long)batch * p.eb_stride;
#pragma unroll
        for (int c = 0; c < 32; c += 2) {
          const int col = tn * BN + 32 * h + c;
          if (col < p.b_rows) {
            const int j = col >> 1;
            const double sc = p.alpha * pow2(ea + eb[j] - 14);
            double re = ((double)hi[c] + (double)lo[c]) * sc;
            double im = ((double)hi[c + 1] + (double)lo[c + 1]) * sc;
            if (p.conj) im = -im;
            double2* o = out + (long)j * p.ld_col;
            if (p.atomic) {
              atomicAdd(&o->x, re);
              atomicAdd(&o->y, im);
            } else {
              *o = make_double2(re, im);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

// ---------------------------------------------------------------------------
// digit slicing (HBM-bound)
// ---------------------------------------------------------------------------

// Signed base-256 digits of Y = round(x 2^(7 + 8(S-1) - e)) for |x| < 2^e:
// x ~= 2^(e-7) sum_s d_s 2^(-8s), integer |d_s| <= 128 (exact in BF16).
// Pure integer arithmetic on the IEEE fields (GB300's FP64 pipe is narrow).
__device__ __forceinline__ void cut_digits(double x, int e, int S, float* d) {
  const long long bits = __double_as_longlong(x);
  const int bexp = (int)((bits >> 52) & 0x7FF);
  long long Y = 0;
  if (bexp != 0) {  // zero and subnormals give zero digits
    const long long mant = (bits & ((1LL << 52) - 1)) | (1LL << 52);
    const int sh = bexp - 1075 + 7 + 8 * (S - 1) - e;  // Y = mant 2^sh
    if (sh >= 0)
      Y = mant << sh;  // < 2^(7 + 8(S-1)) <= 2^63 since |x| < 2^e
    else if (sh > -63)
      Y = (mant + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) Y = -Y;
  }
  for (int s = S - 1; s >= 1; --s) {
    const int dd = (int)((Y + 128) & 255) - 128;
    d[s] = (float)dd;
    Y = (Y - dd) >> 8;
  }
  d[0] = (float)Y;
}

// e with m < 2^e (frexp exponent) for m > 0; 0 for m == 0.
__device__ __forceinline__ int row_exponent(double m) {
  const long long bits = __double_as_longlong(m);
  const int bexp = (int)((bits >> 52) & 0x7FF);
  if (bexp == 0) return m > 0.0 ? -1022 : 0;
  return bexp - 1022;
}

__device__ __forceinline__ double2 load_any(const void* p, int dtype, long idx) {
  if (dtype == RPA_C64) {
    float2 v = reinterpret_cast<const float2*>(p)[idx];
    return make_double2(v.x, v.y);
  }
  return reinterpret_cast<const double2*>(p)[idx];
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// chi0 operand X[vc][g] = sf[vc] sv[g] A[vc][g]: row maxima over vc per g.
__global__ void chi0_rowmax_kernel(const void* A, int dtype, int n_vc, int n_g, const double* sf,
                                   const double* sv, unsigned long long* rowmax) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_g) return;
  const double w = sv[g];
  double m = 0.0;
  for (int vc = blockIdx.y; vc < n_vc; vc += gridDim.y) {
    double2 a = load_any(A, dtype, (long)vc * n_g + g);
    double s = sf[vc] * w;
    m = fmax(m, fmax(fabs(a.x * s), fabs(a.y * s)));
  }
  atomic_max_pos(rowmax + g, m);
}

// chi0 operand planes, [S][2 n_g_pad][K], K index 2 vc + part: row 2g holds
// (x_r, x_i), row 2g+1 holds (x_i, -x_r), so that Re chi = X_g . X_h and
// Im chi = X_g . Y_h.  One 32 x 32 (vc, g) tile per block, transposed through
// shared memory so that the plane rows are written contiguously.
__global__ void chi0_slice_kernel(const void* A, int dtype, int n_vc, int n_g, int n_g_pad,
                                  long K, const double* sf, const double* sv,
                                  const unsigned long long* rowmax, int S,
                                  __nv_bfloat162* planes, int* exps) {
  __shared__ double2 t[32][33];
  __shared__ int es[32];
  const int vc0 = blockIdx.x * 32, g0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (ty == 0) {
    int g = g0 + tx;
    int e = g < n_g ? row_exponent(__longlong_as_double((long long)rowmax[g])) : 0;
    es[tx] = e;
    if (blockIdx.x == 0 && g < n_g_pad) exps[g] = e;
  }
  for (int r = ty; r < 32; r += 8) {
    int vc = vc0 + r, g = g0 + tx;
    double2 x = make_double2(0.0, 0.0);
    if (vc < n_vc && g < n_g) {
      x = load_any(A, dtype, (long)vc * n_g + g);
      double s = sf[vc] * sv[g];
      x.x *= s;
      x.y *= s;
    }
    t[r][tx] = x;
  }
  __syncthreads();
  const long plane = (long)2 * n_g_pad * (K / 2);  // in bf162 units
  for (int r = ty; r < 32; r += 8) {
    const int g = g0 + r;
    if (g >= n_g_pad) continue;
    const int vc = vc0 + tx;  // K pair index
    if ((long)2 * vc >= K) continue;
    double2 x = t[tx][r];
    float dr[MAX_SLICES], di[MAX_SLICES];
    cut_digits(x.x, es[r], S, dr);
    cut_digits(x.y, es[r], S, di);
    for (int s = 0; s < S; ++s) {
      __nv_bfloat162* p0 = planes + s * plane + (long)(2 * g) * (K / 2) + vc;
      p0[0] = __floats2bfloat162_rn(dr[s], di[s]);
      p0[K / 2] = __floats2bfloat162_rn(di[s], -dr[s]);
    }
  }
}

// Generic row slicing: row r of a complex matrix (row stride `ld` complex
// elements, n_cplx valid elements) scaled by `scale` (may be NULL), planes
// [S][rows_pad][K] with K index 2 k + part.  One block per row.
__global__ void slice_rows_kernel(const void* src, int dtype, long ld, int n_rows, int n_cplx,
                                  int rows_pad, long K, int S, __nv_bfloat162* planes, int* exps) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  if (r >= rows_pad) return;
  double m = 0.0;
  if (r < n_rows)
    for (int k = threadIdx.x; k < n_cplx; k += blockDim.x) {
      double2 x = load_any(src, dtype, (long)r * ld + k);
      m = fmax(m, fmax(fabs(x.x), fabs(x.y)));
    }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmax(mm, red[i]);
    red[0] = mm;
  }
  __syncthreads();
  const int e = row_exponent(red[0]);
  if (threadIdx.x == 0) exps[r] = e;
  const long plane = (long)rows_pad * (K / 2);
  for (long k = threadIdx.x; k < K / 2; k += blockDim.x) {
    double2 x = make_double2(0.0, 0.0);
    if (r < n_rows && k < n_cplx) x = load_any(src, dtype, (long)r * ld + k);
    float dr[MAX_SLICES], di[MAX_SLICES];
    cut_digits(x.x, e, S, dr);
    cut_digits(x.y, e, S, di);
    for (int s = 0; s < S; ++s)
      planes[s * plane + (long)r * (K / 2) + k] = __floats2bfloat162_rn(dr[s], di[s]);
  }
}

// Projection B operand from B[g][i] (= v^1/2 C): rows 2i = (b_r, -b_i) and
// 2i+1 = (b_i, b_r) along K index 2g + part; one block per i.
__global__ void proj_b_slice_kernel(const double2* B, int n_g, int n_eig, int n_eig_pad, long K,
                                    int S, __nv_bfloat162* planes, int* exps) {
  __shared__ double red[32];
  const int i = blockIdx.x;
  double m = 0.0;
  if (i < n_eig)
    for (int g = threadIdx.x; g < n_g; g += blockDim.x) {
      double2 b = B[(long)g * n_eig + i];
      m = fmax(m, fmax(fabs(b.x), fabs(b.y)));
    }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[w]);
    red[0] = mm;
  }
  __syncthreads();
  const int e = row_exponent(red[0]);
  if (threadIdx.x == 0) exps[i] = e;
  const long plane = (long)2 * n_eig_pad * (K / 2);
  for (long g = threadIdx.x; g < K / 2; g += blockDim.x) {
    double2 b = make_double2(0.0, 0.0);
    if (i < n_eig && g < n_g) b = B[g * n_eig + i];
    float dr[MAX_SLICES], di[MAX_SLICES];
    cut_digits(b.x, e, S, dr);
    cut_digits(b.y, e, S, di);
    for (int s = 0; s < S; ++s) {
      __nv_bfloat162* p0 = planes + s * plane + (long)(2 * i) * (K / 2) + g;
      p0[0] = __floats2bfloat162_rn(dr[s], -di[s]);
      p0[K / 2] = __floats2bfloat162_rn(di[s], dr[s]);
    }
  }
}

// f[b][vc] = 4 D / (D^2 + w_{k0+b}^2) for the frequencies of one group.
__global__ void freq_weights_kernel(const double* delta, const double* omega, int n_vc, int k0,
                                    int nb, double* f) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= (long)nb * n_vc) return;
  const int b = (int)(i / n_vc), vc = (int)(i % n_vc);
  const double d = delta[vc], w = omega[k0 + b];
  f[i] = 4.0 * d / (d * d + w * w);
}

// chi_s B operand of frequencies k0 .. k0+nb-1: for row j, f_k(vc) M~[j][vc]
// as rows 2j = (f m_r, f m_i) and 2j+1 = (-f m_i, f m_r); one block per j.
constexpr int MAX_GROUP = 8;
__global__ void chis_b_slice_kernel(const double2* mt, int n_eig, int n_eig_pad, int n_vc,
                                    long K, const double* f, int nb, int S,
                                    __nv_bfloat162* planes, int* exps, int eb_stride) {
  __shared__ double red[MAX_GROUP][32];
  const int j = blockIdx.x;
  double m[MAX_GROUP];
#pragma unroll
  for (int b = 0; b < MAX_GROUP; ++b) m[b] = 0.0;
  if (j < n_eig)
    for (int vc = threadIdx.x; vc < n_vc; vc += blockDim.x) {
      const double2 x = mt[(long)j * n_vc + vc];
      const double a = fmax(fabs(x.x), fabs(x.y));
#pragma unroll
      for (int b = 0; b < MAX_GROUP; ++b)
        if (b < nb) m[b] = fmax(m[b], f[(long)b * n_vc + vc] * a);
    }
#pragma unroll
  for (int b = 0; b < MAX_GROUP; ++b) {
    double v = m[b];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[b][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  int e[MAX_GROUP];
#pragma unroll
  for (int b = 0; b < MAX_GROUP; ++b) {
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[b][w]);
    e[b] = row_exponent(mm);
    if (threadIdx.x == 0 && b < nb) exps[b * eb_stride + j] = e[b];
  }
  const long plane = (long)2 * n_eig_pad * (K / 2);
  for (long vc = threadIdx.x; vc < K / 2; vc += blockDim.x) {
    double2 x = make_double2(0.0, 0.0);
    const bool in = j < n_eig && vc < n_vc;
    if (in) x = mt[(long)j * n_vc + vc];
#pragma unroll
    for (int b = 0; b < MAX_GROUP; ++b) {
      if (b >= nb) break;
      const double fv = in ? f[(long)b * n_vc + vc] : 0.0;
      float dr[MAX_SLICES], di[MAX_SLICES];
      cut_digits(fv * x.x, e[b], S, dr);
      cut_digits(fv * x.y, e[b], S, di);
      for (int s = 0; s < S; ++s) {
        __nv_bfloat162* p0 = planes + (long)(b * S + s) * plane + (long)(2 * j) * (K / 2) + vc;
        p0[0] = __floats2bfloat162_rn(dr[s], di[s]);
        p0[K / 2] = __floats2bfloat162_rn(-di[s], dr[s]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

inline long rup(long a, long b) { return (a + b - 1) / b * b; }
inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

int drain_tiles(int S) {
  // exact FP32 sums need K_d * (L+1) * 2^14 <= 2^24 for every level L <= S-1
  int kd = (1024 / S) / BK * BK;
  return std::max(1, kd / BK);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 3-D map over BF16 planes: dim0 = K (contiguous), dim1 = rows (row_bytes apart),
// dim2 = plane (plane_bytes apart); box K 64 x box_rows x 1, 128-byte swizzle.
bool make_map(CUtensorMap* m, void* base, long K, long rows, long planes, long row_bytes,
              long plane_bytes, int box_rows, std::string& err) {
  auto fn = encode_fn();
  if (!fn) {
    err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)plane_bytes};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char b[160];
    snprintf(b, sizeof b, "cuTensorMapEncodeTiled failed (%d): K=%ld rows=%ld planes=%ld", (int)r,
             K, rows, planes);
    err = b;
    return false;
  }
  return true;
}

size_t gemm_smem(int S) { return 1024 + NA * A_TILE + 2 * S * B_TILE; }

// Build the work list (upper block triangle when `upper`), choose split-K, launch.
rpa_status run_gemm(Workspace& w, const CUtensorMap& ta, const CUtensorMap& tb, GemmArgs a,
                    int tiles_m, int tiles_n, int batches, bool upper, void* zero_ptr,
                    size_t zero_bytes, cudaStream_t st, std::string& err, int* launches) {
  std::vector<int4> work;
  const int kdt = drain_tiles(a.S);
  const int kd = kdt * BK;
  int tiles = 0;
  for (int b = 0; b < batches; ++b)
    for (int m = 0; m < tiles_m; ++m)
      for (int n = 0; n < tiles_n; ++n)
        if (!upper || (long)n * BN / 2 + BN / 2 - 1 >= (long)m * BM) ++tiles;
  int split = 1;
  const int want = 2 * 148;
  if (tiles < want) split = std::min(cdiv(want, tiles), std::max(1, a.K / kd));
  long kps = rup(cdiv(a.K, split), kd);
  split = cdiv(a.K, kps);
  a.k_per_split = (int)kps;
  a.kd_tiles = kdt;
  a.atomic = 0;
  if (split > 1) {
    // split-K partial tiles are summed with FP64 atomics into a zeroed output
    cudaError_t ez = cudaMemsetAsync(zero_ptr, 0, zero_bytes, st);
    if (ez != cudaSuccess) {
      err = cudaGetErrorString(ez);
      return RPA_ECUDA;
    }
    a.atomic = 1;
  }
  for (int b = 0; b < batches; ++b)
    for (int m = 0; m < tiles_m; ++m)
      for (int n = 0; n < tiles_n; ++n)
        if (!upper || (long)n * BN / 2 + BN / 2 - 1 >= (long)m * BM)
          for (int s = 0; s < split; ++s) work.push_back(make_int4(m, n, b, s));
  if (work.size() > w.work_count) {
    err = "work list exceeds workspace";
    return RPA_ENOMEM;
  }
  if (work.empty()) return RPA_OK;
  cudaError_t e = cudaMemcpyAsync(w.work, work.data(), work.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return RPA_ECUDA;
  }
  a.work = w.work;
  a.status = w.status;
  a.stall = w.debug_stall;
  const size_t smem = gemm_smem(a.S);
  static size_t configured = 0;
  if (smem > configured) {
    e = cudaFuncSetAttribute(slice_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gemm_smem(MAX_SLICES));
    if (e != cudaSuccess) {
      err = cudaGetErrorString(e);
      return RPA_ECUDA;
    }
    configured = gemm_smem(MAX_SLICES);
  }
  slice_gemm_kernel<<<(unsigned)work.size(), THREADS, smem, st>>>(ta, tb, a);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = cudaGetErrorString(e);
    return RPA_ECUDA;
  }
  if (launches) *launches += 1;
  return RPA_OK;
}

#define CK(call)                                    \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      err = std::string(#call ": ") + cudaGetErrorString(e_); \
      return RPA_ECUDA;                             \
    }                                               \
  } while (0)

}  // namespace

rpa_status alloc_workspace(Workspace& w, size_t max_g, size_t max_eig, size_t max_vc,
                           size_t max_freq, const Slices& s, std::string& err) {
  w = Workspace{};
  w.slices = s;
  const long g_pad = rup(max_g, BM), e_pad = rup(max_eig, BM), vc_pad = rup(max_vc, BM);
  const long k_vc = rup(2 * max_vc, BK), k_g = rup(2 * max_g, BK);
  const int grp = (int)std::min<size_t>(MAX_GROUP, max_freq);
  w.freq_group = grp;
  size_t p1 = std::max({(size_t)s.chi0 * 2 * g_pad * k_vc, (size_t)s.proj * vc_pad * k_g,
                        (size_t)grp * s.chis * 2 * e_pad * k_vc});
  size_t p2 = std::max((size_t)s.proj * 2 * e_pad * k_g, (size_t)s.chis * e_pad * k_vc);
  w.plane_bytes = p1 * 2;
  w.plane2_bytes = p2 * 2;
  w.exp_count = std::max({(size_t)g_pad, (size_t)vc_pad, (size_t)e_pad}) +
                std::max((size_t)g_pad, (size_t)grp * e_pad);
  w.rowmax_count = g_pad;
  w.work_count = 1 << 20;
  w.fweight_count = (size_t)grp * max_vc;
  auto al = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      char b[128];
      snprintf(b, sizeof b, "tensor-core workspace: cudaMalloc of %zu bytes failed", bytes);
      err = b;
      return false;
    }
    return true;
  };
  if (!al(&w.planes, w.plane_bytes) || !al(&w.planes2, w.plane2_bytes) ||
      !al((void**)&w.exps, w.exp_count * sizeof(int)) ||
      !al((void**)&w.rowmax, w.rowmax_count * sizeof(unsigned long long)) ||
      !al((void**)&w.work, w.work_count * sizeof(int4)) || !al((void**)&w.status, sizeof(int)) ||
      !al((void**)&w.fweights, w.fweight_count * sizeof(double))) {
    free_workspace(w);
    return RPA_ENOMEM;
  }
  cudaMemset(w.status, 0, sizeof(int));
  return RPA_OK;
}

void free_workspace(Workspace& w) {
  void* b[] = {w.planes, w.planes2, w.exps, w.rowmax, w.work, w.status, w.fweights};
  for (void* p : b)
    if (p) cudaFree(p);
  w = Workspace{};
}

rpa_status chi0(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const double* sf,
                const double* sv, double scale, cplx* chi, cudaStream_t st, std::string& err,
                int* launches) {
  const int S = w.slices.chi0;
  const long g_pad = rup(n_g, BM), K = rup(2L * n_vc, BK);
  w.hook(RPA_T_SLICE, 1);
  CK(cudaMemsetAsync(w.rowmax, 0, g_pad * sizeof(unsigned long long), st));
  {
    dim3 grid(cdiv(n_g, 128), std::min(cdiv(n_vc, 64), 512));
    chi0_rowmax_kernel<<<grid, 128, 0, st>>>(A, dtype, n_vc, n_g, sf, sv, w.rowmax);
    CK(cudaGetLastError());
  }
  __nv_bfloat162* planes = (__nv_bfloat162*)w.planes;
  {
    dim3 grid(cdiv(K / 2, 32), cdiv(g_pad, 32));
    chi0_slice_kernel<<<grid, dim3(32, 8), 0, st>>>(A, dtype, n_vc, n_g, (int)g_pad, K, sf, sv,
                                                    w.rowmax, S, planes, w.exps);
    CK(cudaGetLastError());
  }
  if (launches) *launches += 2;
  w.hook(RPA_T_SLICE, 0);
  CUtensorMap ta, tb;
  const long plane_bytes = 2 * g_pad * K * 2;
  // A view: even rows of the planes (X_g); B: all rows (X_h, Y_h interleaved)
  if (!make_map(&ta, w.planes, K, g_pad, S, 2 * K * 2, plane_bytes, BM, err)) return RPA_ECUDA;
  if (!make_map(&tb, w.planes, K, 2 * g_pad, S, K * 2, plane_bytes, BN, err)) return RPA_ECUDA;
  GemmArgs a{};
  a.S = S;
  a.K = (int)K;
  a.ea = w.exps;
  a.eb = w.exps;
  a.eb_stride = 0;
  a.a_rows = n_g;
  a.b_rows = 2 * n_g;
  a.alpha = scale;
  a.out = (double2*)chi;
  a.out_bstride = 0;
  a.ld_row = n_g;
  a.ld_col = 1;
  a.conj = 0;
  a.atomic = 0;
  const int tiles_m = cdiv(n_g, BM), tiles_n = cdiv(2L * n_g, BN);
  w.hook(RPA_T_CHI0, 1);
  rpa_status r = run_gemm(w, ta, tb, a, tiles_m, tiles_n, 1, true, chi,
                          sizeof(cplx) * (size_t)n_g * n_g, st, err, launches);
  w.hook(RPA_T_CHI0, 0);
  return r;
}

rpa_status project(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const cplx* B,
                   int n_eig, cplx* mt, cudaStream_t st, std::string& err, int* launches) {
  const int S = w.slices.proj;
  const long vc_pad = rup(n_vc, BM), e_pad = rup(n_eig, BM), K = rup(2L * n_g, BK);
  __nv_bfloat162* pa = (__nv_bfloat162*)w.planes;
  __nv_bfloat162* pb = (__nv_bfloat162*)w.planes2;
  int* ea = w.exps;
  int* eb = w.exps + std::max({rup(n_g, BM), vc_pad, e_pad});
  w.hook(RPA_T_SLICE, 1);
  slice_rows_kernel<<<(unsigned)vc_pad, 256, 0, st>>>(A, dtype, n_g, n_vc, n_g, (int)vc_pad, K, S,
                                                      pa, ea);
  CK(cudaGetLastError());
  proj_b_slice_kernel<<<(unsigned)e_pad, 256, 0, st>>>((const double2*)B, n_g, n_eig, (int)e_pad,
                                                       K, S, pb, eb);
  CK(cudaGetLastError());
  if (launches) *launches += 2;
  w.hook(RPA_T_SLICE, 0);
  CUtensorMap ta, tb;
  if (!make_map(&ta, w.planes, K, vc_pad, S, K * 2, vc_pad * K * 2, BM, err)) return RPA_ECUDA;
  if (!make_map(&tb, w.planes2, K, 2 * e_pad, S, K * 2, 2 * e_pad * K * 2, BN, err))
    return RPA_ECUDA;
  GemmArgs a{};
  a.S = S;
  a.K = (int)K;
  a.ea = ea;
  a.eb = eb;
  a.eb_stride = 0;
  a.a_rows = n_vc;
  a.b_rows = 2 * n_eig;
  a.alpha = 1.0;
  a.out = (double2*)mt;
  a.out_bstride = 0;
  a.ld_row = 1;
  a.ld_col = n_vc;
  a.conj = 1;
  a.atomic = 0;
  const int tiles_m = cdiv(n_vc, BM), tiles_n = cdiv(2L * n_eig, BN);
  w.hook(RPA_T_PROJ, 1);
  rpa_status r = run_gemm(w, ta, tb, a, tiles_m, tiles_n, 1, false, mt,
                          sizeof(cplx) * (size_t)n_eig * n_vc, st, err, launches);
  w.hook(RPA_T_PROJ, 0);
  return r;
}

rpa_status chis(Workspace& w, const cplx* mt, int n_eig, int n_vc, const double* delta,
                const double* omega, int n_freq, double scale, cplx* out, cudaStream_t st,
                std::string& err, int* launches) {
  const int S = w.slices.chis;
  const long e_pad = rup(n_eig, BM), K = rup(2L * n_vc, BK);
  __nv_bfloat162* pa = (__nv_bfloat162*)w.planes2;
  __nv_bfloat162* pb = (__nv_bfloat162*)w.planes;
  int* ea = w.exps;
  int* eb = w.exps + e_pad;
  w.hook(RPA_T_SLICE, 1);
  slice_rows_kernel<<<(unsigned)e_pad, 256, 0, st>>>(mt, RPA_C128, n_vc, n_eig, n_vc, (int)e_pad,
                                                     K, S, pa, ea);
  CK(cudaGetLastError());
  if (launches) *launches += 1;
  w.hook(RPA_T_SLICE, 0);
  CUtensorMap ta;
  if (!make_map(&ta, w.planes2, K, e_pad, S, K * 2, e_pad * K * 2, BM, err)) return RPA_ECUDA;
  const int tiles_m = cdiv(n_eig, BM), tiles_n = cdiv(2L * n_eig, BN);
  for (int k0 = 0; k0 < n_freq; k0 += w.freq_group) {
    const int nb = std::min(w.freq_group, n_freq - k0);
    w.hook(RPA_T_SLICE, 1);
    freq_weights_kernel<<<cdiv((long)nb * n_vc, 256), 256, 0, st>>>(delta, omega, n_vc, k0, nb,
                                                                    w.fweights);
    CK(cudaGetLastError());
    chis_b_slice_kernel<<<(unsigned)e_pad, 256, 0, st>>>((const double2*)mt, n_eig, (int)e_pad,
                                                         n_vc, K, w.fweights, nb, S, pb, eb,
                                                         (int)e_pad);
    CK(cudaGetLastError());
    if (launches) *launches += 2;
    w.hook(RPA_T_SLICE, 0);
    CUtensorMap tb;
    if (!make_map(&tb, w.planes, K, 2 * e_pad, (long)nb * S, K * 2, 2 * e_pad * K * 2, BN, err))
      return RPA_ECUDA;
    GemmArgs a{};
    a.S = S;
    a.K = (int)K;
    a.ea = ea;
    a.eb = eb;
    a.eb_stride = (int)e_pad;
    a.a_rows = n_eig;
    a.b_rows = 2 * n_eig;
    a.alpha = scale;
    a.out = (double2*)(out + (size_t)k0 * n_eig * n_eig);
    a.out_bstride = (long)n_eig * n_eig;
    a.ld_row = n_eig;
    a.ld_col = 1;
    a.conj = 0;
    w.hook(RPA_T_CHIS, 1);
    rpa_status s = run_gemm(w, ta, tb, a, tiles_m, tiles_n, nb, true, a.out,
                            sizeof(cplx) * (size_t)nb * n_eig * n_eig, st, err, launches);
    w.hook(RPA_T_CHIS, 0);
    if (s != RPA_OK) return s;
  }
  return RPA_OK;
}

}  // namespace tc
}  // namespace rpa
