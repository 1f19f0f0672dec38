// Tensor-core (tcgen05) contractions of the mixed-precision path: exact
// digit-sliced BF16 GEMM with TMEM accumulation and a double-float epilogue,
// plus the HBM-bound kernels that cut FP64 operands into digit planes.
//
// GEMM kernel: persistent, one CTA per SM walking every grid-th output tile of
// 128 x BN (BN = 64 or 128) of a rasterised work list; its roles:
//   warp 0      TMA producer: per 64-wide K-tile, all S digit planes of the B
//               tile (double- or triple-buffered) and the S digit planes of the
//               A tile through a ring of slots in groups of G = min(S, NA/2);
//               each group has one full and one empty barrier, so the MMA
//               thread waits and commits once per group rather than per plane
//               (G <= S keeps a group within two K-tiles, which the B buffers
//               always cover, so the producer can fill it);
//   warp 1      TMEM allocation and the single MMA-issuing thread: per A digit
//               plane s, kind::f16 MMAs (K = 16 each) against the B planes
//               t = 0 .. Le-1-s taken together as one operand of BN (Le - s)
//               rows, whose output columns land in the exact level accumulators
//               L = s + t (levels sit BN columns apart in TMEM), and one MMA per
//               remaining pair (s, t) into the tail accumulator;
//   BN/8 epilogue warps (4 lane quadrants x BN/32 column blocks): at the end
//               of each drain interval, read the level accumulators from TMEM
//               and add them into per-thread double-float accumulators (one
//               TMEM lane and 32 columns per thread); at the end of a tile apply
//               the row scales and write complex FP64 results while the MMA
//               thread already works on the next tile.
// Digit planes are stored pre-scaled (plane s holds d_s 2^-8s), so level L
// sums integers times 2^-8L.  Levels L < Le (p.nexact) have accumulators of
// their own and stay exact (integer sums below 2^24 over a drain interval);
// levels Le .. S-1, which weigh at most 2^-8Le of the leading one, share one
// FP32 "tail" accumulator whose rounding stays far below the truncation.
// Every mbarrier wait is bounded (about 2 s of SM clock): on expiry the CTA
// raises a flag in the status word, stops issuing, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <vector>

#include "rpa_tc.h"

namespace rpa {
namespace tc {
namespace {

constexpr int BM = 128;  // A rows per tile = TMEM lanes = MMA M
constexpr int BK = 64;   // K elements per tile: 128 bytes of BF16, one 128B swizzle row
// B rows per tile (= MMA N) is a template parameter: 128 when the level
// accumulators (at most 3) and the low halves fit in TMEM, else 64 (pick_bn).
constexpr int MAX_NA = 8;   // A ring depth (runtime, <= MAX_NA), in groups of G slots
constexpr int MAX_NB = 3;   // B buffers (runtime, <= MAX_NB)
// Per-device launch limits of the GEMM, set up once per device (the dynamic
// shared-memory attribute of a kernel is a per-device setting).
struct DeviceLimits {
  size_t smem = 0;  // dynamic shared memory a CTA of the GEMM may use
  int sms = 0;      // streaming multiprocessors
};
constexpr int kMaxDevices = 64;
DeviceLimits g_limits[kMaxDevices];
std::mutex g_limits_mutex;
// producer warp, MMA warp, and 4 x BN/32 epilogue warps (4 lane quadrants x
// BN/32 column blocks of 32 accumulator columns)
template <int BN>
constexpr int threads_for() {
  return 64 + 4 * BN;
}

// TMEM columns between level accumulators: BN, so that the columns of B plane
// t in an MMA that covers planes 0 .. S-1-s fall into level s + t.
template <int BN>
constexpr int tmem_stride() {
  static_assert(BN % 64 == 0, "level accumulators start at multiples of 64 TMEM columns");
  return BN;
}
constexpr int MMA_N_MAX = 256;  // largest N of a cta_group::1 kind::f16 MMA with M = 128
constexpr uint32_t A_TILE = BM * BK * 2;  // 16 KB
constexpr long long WAIT_CYCLES = 4000000000LL;  // about 2 s at 2 GHz

// Instruction descriptor of kind::f16 (A = B = BF16, code 1) or kind::tf32 (A = B =
// TF32, code 2): D = F32 (bits 4-5), A and B formats at bits 7-9 and 10-12, both K-major
// (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t idesc_n(int n, bool tf32 = false) {
  return (1u << 4) | ((tf32 ? 2u : 1u) << 7) | ((tf32 ? 2u : 1u) << 10) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// K elements per 128-byte row of a tile: 64 BF16 or 32 TF32 (FP32 storage).
__host__ __device__ constexpr int bk_elems(bool tf32) { return tf32 ? 32 : 64; }
constexpr int ROWB = 128;   // bytes per K-major tile row (one 128-byte swizzle row)
constexpr int KSTEPS = 4;   // MMAs per K-tile: 32 bytes of K each (16 BF16 or 8 TF32)

enum : int {
  ERR_WAIT_PRODUCER = 1,
  ERR_WAIT_MMA = 2,
  ERR_WAIT_EPILOGUE = 4,
};

struct GemmArgs {
  int S;              // digit slices per operand
  int na, nb;         // A ring depth, B buffers
  int nacc;           // level-accumulator buffers in TMEM (1 or 2)
  int K;              // padded K (multiple of BK)
  int kd_tiles;       // K-tiles per drain interval
  int k_per_split;    // K elements per split (multiple of BK)
  const int4* work;   // (tile_m, tile_n, batch, k_split)
  int n_work;         // tiles in the list; CTA b takes tiles b, b + gridDim.x, ...
  const int* ea;      // exponent per A row
  const int* eb;      // exponent per complex B row pair, [batch][eb_stride]
  int eb_stride;
  int a_rows, b_rows; // valid rows of A and B (B rows = 2 x complex columns)
  double alpha;
  double2* out;       // complex output
  long out_bstride, ld_row, ld_col;
  int conj, atomic;
  int accumulate;     // add into the output with FP64 atomics, never zero it
  const double* rsa;  // optional FP64 factor per A row (NULL: 1)
  const double* rsb;  // optional FP64 factor per complex B column (NULL: 1)
  int nexact;         // levels with exact accumulators (Le); the rest share a tail
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
// another role of this CTA aborted.  The latency-critical producer and MMA
// threads spin on try_wait (which suspends in hardware); epilogue warps also
// back off with a short sleep.
template <bool kSleep>
__device__ __forceinline__ bool mbar_wait_t(uint64_t* bar, uint32_t parity,
                                            volatile int* abort_flag, int* status, int code) {
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
    if (kSleep) __nanosleep(64);
  }
}
#define mbar_wait mbar_wait_t<false>
#define mbar_wait_sleep mbar_wait_t<true>

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

template <bool TF>
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  if constexpr (TF)
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  else
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 lanes x 8 consecutive columns of FP32 from TMEM.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]),
               "r"(r[7])
               : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
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

template <int BN, bool TF>
__global__ void __launch_bounds__(threads_for<BN>(), 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const GemmArgs p) {
  constexpr uint32_t B_TILE = BN * ROWB;
  constexpr int BKE = bk_elems(TF);  // K elements per tile
  constexpr int CPT = 32;           // accumulator columns per epilogue thread
  constexpr int EPI = BN / 8;       // epilogue warps: 4 lane quadrants x BN/32 column blocks
  constexpr int TS = tmem_stride<BN>();
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_a[MAX_NA], empty_a[MAX_NA], full_b[MAX_NB], empty_b[MAX_NB];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = p.S, NA = p.na, NB = p.nb, NACC = p.nacc;
  const int Le = min(p.nexact, S);            // exact levels
  const int NL = Le < S ? Le + 1 : S;         // accumulators: exact levels (+ tail)
  const int G = min(S, NA / 2);               // A slots per barrier group
  const int NG = NA / G;                      // barrier groups in the ring (>= 2)
  uint8_t* sA = smem;                         // NA x 16 KB
  uint8_t* sB = smem + NA * A_TILE;           // NB x S x 8 KB
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kdt = p.kd_tiles;
  const int used = NACC * NL * TS + (BN == 128 ? BN : 0);  // + low halves for BN = 128
  const uint32_t ncols = used <= 32 ? 32 : (used <= 64 ? 64 : (used <= 128 ? 128 : (used <= 256 ? 256 : 512)));

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int i = 0; i < NG; ++i) {
      mbar_init(&full_a[i], 1);
      mbar_init(&empty_a[i], 1);
    }
    for (int i = 0; i < NB; ++i) {
      mbar_init(&full_b[i], 1);
      mbar_init(&empty_b[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&acc_full[i], 1);
      mbar_init(&acc_empty[i], EPI);
    }
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
      // A planes of a tile in K order i = kt S + s fill groups of G slots of the
      // ring; a group ends after G planes or at the tile's last plane
      int pos = 0, h = 0, aphase = 0, bb = 0, bphase = 0;
      bool ok = true;
      for (int wi = blockIdx.x; wi < p.n_work && ok; wi += gridDim.x) {
      const int4 wk = p.work[wi];
      const int tm = wk.x, tn = wk.y, batch = wk.z;
      const int k_begin = wk.w * p.k_per_split;
      const int nkt = (min(p.K, k_begin + p.k_per_split) - k_begin) / BKE;
      const int total = nkt * S;
      int i = 0;
      for (int kt = 0; kt < nkt && !abort_flag; ++kt) {
        const int k0 = k_begin + kt * BKE;
        if (!mbar_wait(&empty_b[bb], bphase ^ 1, &abort_flag, p.status, ERR_WAIT_PRODUCER)) {
          ok = false;
          break;
        }
        mbar_expect_tx(&full_b[bb], S * B_TILE);
        for (int t = 0; t < S; ++t)
          tma_load_3d(sB + (bb * S + t) * B_TILE, &tmB, &full_b[bb], k0, tn * BN, batch * S + t);
        if (++bb == NB) {
          bb = 0;
          bphase ^= 1;
        }
        for (int s = 0; s < S; ++s, ++i) {
          if (pos == 0) {
            if (!mbar_wait(&empty_a[h], aphase ^ 1, &abort_flag, p.status, ERR_WAIT_PRODUCER)) {
              ok = false;
              break;
            }
            mbar_expect_tx(&full_a[h], (uint32_t)min(G, total - i) * A_TILE);
          }
          tma_load_3d(sA + (h * G + pos) * A_TILE, &tmA, &full_a[h], k0, tm * BM, s);
          if (++pos == G || i == total - 1) {
            pos = 0;
            if (++h == NG) {
              h = 0;
              aphase ^= 1;
            }
          }
        }
        if (!ok) break;
      }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      unsigned first = 0;
      int pos = 0, h = 0, aphase = 0, bb = 0, bphase = 0, ab = 0, accphase = 0;
      uint32_t acc_base = tmem;
      const uint32_t sA0 = smem_u32(sA), sB0 = smem_u32(sB);
      bool alive = true;
      for (int wi = blockIdx.x; wi < p.n_work && alive; wi += gridDim.x) {
      const int k_begin = p.work[wi].w * p.k_per_split;
      const int nkt = (min(p.K, k_begin + p.k_per_split) - k_begin) / BKE;
      const int total = nkt * S;
      int i = 0, kin = 0;
      alive = false;
      for (int kt = 0; kt < nkt; ++kt) {
        if (kin == 0) {
          if (!mbar_wait(&acc_empty[ab], accphase ^ 1, &abort_flag, p.status, ERR_WAIT_MMA)) break;
          tc_fence_after();
          first = 1;
          acc_base = tmem + ab * NL * TS;
        }
        if (!mbar_wait(&full_b[bb], bphase, &abort_flag, p.status, ERR_WAIT_MMA)) break;
        tc_fence_after();
        bool ok = true;
        // The B planes of this stage are contiguous (plane t at rows t BN ..), so
        // the rows of planes 0 .. Le-1-s form one K-major operand; its output
        // column t BN + j goes to TMEM column (s + t) BN + j = exact level s + t.
        // Pairs with s + t >= Le go one plane at a time into the tail.  The
        // first MMAs of an interval into a column range overwrite it: plane
        // s = 0 covers every exact level, and its first tail MMA the tail.
        const uint64_t bd0 = smem_desc(sB0 + bb * S * B_TILE);
        // with a single tail level (S = Le + 1) the tail accumulator sits where level Le
        // would, so every plane's pairs form one contiguous run
        const int Lr = S - Le == 1 ? S : min(S, Le);
        bool tail_first = first;
        for (int s = 0; s < S; ++s, ++i) {
          if (pos == 0) {
            if (!mbar_wait(&full_a[h], aphase, &abort_flag, p.status, ERR_WAIT_MMA)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const uint64_t ad = smem_desc(sA0 + (h * G + pos) * A_TILE);
          const int rows = s < Lr ? BN * (Lr - s) : 0;
          for (int c0 = 0; c0 < rows; c0 += MMA_N_MAX) {
            const int n = min(MMA_N_MAX, rows - c0);
            const uint32_t id = idesc_n(n, TF);
            const uint64_t bd = bd0 + (uint64_t)((c0 * ROWB) >> 4);
            const uint32_t d = acc_base + s * TS + c0;
            mma_issue<TF>(d, ad, bd, id, (s == 0 && first) ? 0u : 1u);
#pragma unroll
            for (int kk = 1; kk < KSTEPS; ++kk) mma_issue<TF>(d, ad + 2 * kk, bd + 2 * kk, id, 1u);
          }
          for (int t = max(0, Lr - s); t <= S - 1 - s; ++t) {
            const uint32_t id = idesc_n(BN, TF);
            const uint64_t bd = bd0 + (uint64_t)((t * BN * ROWB) >> 4);
            const uint32_t d = acc_base + Le * TS;
            mma_issue<TF>(d, ad, bd, id, tail_first ? 0u : 1u);
#pragma unroll
            for (int kk = 1; kk < KSTEPS; ++kk) mma_issue<TF>(d, ad + 2 * kk, bd + 2 * kk, id, 1u);
            tail_first = false;
          }
          if (s == 0) first = 0;
          if (++pos == G || i == total - 1) {
            mma_commit(&empty_a[h]);  // frees the group once its MMAs complete
            pos = 0;
            if (++h == NG) {
              h = 0;
              aphase ^= 1;
            }
          }
        }
        if (!ok) break;
        mma_commit(&empty_b[bb]);
        if (++bb == NB) {
          bb = 0;
          bphase ^= 1;
        }
        if (++kin == kdt || kt == nkt - 1) {
          mma_commit(&acc_full[ab]);
          kin = 0;
          if (++ab == NACC) {
            ab = 0;
            accphase ^= 1;
          }
        }
        if (kt == nkt - 1) alive = true;  // the tile completed
      }
      if (nkt == 0) alive = true;
      }
    }
  } else {
    // ---------------- epilogue (warps 2 .. 1 + BN/8) ----------------
    // BN = 128 keeps the low halves of the double-float accumulators in the TMEM
    // columns after the S level accumulators (registers are scarce with 576
    // threads); BN = 64 keeps both halves in registers.  TMEM loads and stores
    // are warp-collective, so every branch around them is warp-uniform.
    constexpr bool kLoTmem = BN == 128;
    constexpr int NLO = kLoTmem ? 1 : CPT;
    const int q = warp & 3;              // TMEM lane quadrant of this warp
    const int h = (warp - 2) >> 2;       // which 32-column block of the BN columns
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    const uint32_t lo_base = lane_base + NACC * NL * TS + CPT * h;  // used when kLoTmem
    int ivg = 0;  // drain intervals consumed so far (all tiles of this CTA)
    bool ok = true;
    for (int wi = blockIdx.x; wi < p.n_work && ok; wi += gridDim.x) {
    const int4 wk = p.work[wi];
    const int tm = wk.x, tn = wk.y, batch = wk.z;
    const int k_begin = wk.w * p.k_per_split;
    const int nkt = (min(p.K, k_begin + p.k_per_split) - k_begin) / BKE;
    const int niv = (nkt + kdt - 1) / kdt;
    float hi[CPT], lo[NLO];
#pragma unroll
    for (int c = 0; c < CPT; ++c) hi[c] = 0.f;
#pragma unroll
    for (int c = 0; c < NLO; ++c) lo[c] = 0.f;
    if (kLoTmem) {
      const uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
      for (int c0 = 0; c0 < CPT; c0 += 8) tmem_st8(lo_base + c0, z);
      tmem_wait_st();
    }
    for (int iv = 0; iv < niv; ++iv, ++ivg) {
      const int ab = ivg % NACC;
      const bool got = mbar_wait_sleep(&acc_full[ab], (ivg / NACC) & 1, &abort_flag, p.status,
                                       ERR_WAIT_EPILOGUE);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
      if constexpr (kLoTmem) {
        // per 8 columns: the low halves and the first two levels issued together, one
        // wait (a third level, where there is one, after them)
#pragma unroll
        for (int c0 = 0; c0 < CPT; c0 += 8) {
          uint32_t lr[8], r[2][8];
          tmem_ld8(lo_base + c0, lr);
          tmem_ld8(lane_base + (ab * NL) * TS + CPT * h + c0, r[0]);
          if (NL > 1) tmem_ld8(lane_base + (ab * NL + 1) * TS + CPT * h + c0, r[1]);
          tmem_wait_ld();
#pragma unroll
          for (int L = 0; L < 2; ++L)
            if (L < NL) {
#pragma unroll
              for (int c = 0; c < 8; ++c) {
                float l = __uint_as_float(lr[c]);
                dfloat_add(hi[c0 + c], l, __uint_as_float(r[L][c]));
                lr[c] = __float_as_uint(l);
              }
            }
          for (int L = 2; L < NL; ++L) {
            tmem_ld8(lane_base + (ab * NL + L) * TS + CPT * h + c0, r[0]);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              float l = __uint_as_float(lr[c]);
              dfloat_add(hi[c0 + c], l, __uint_as_float(r[0][c]));
              lr[c] = __float_as_uint(l);
            }
          }
          tmem_st8(lo_base + c0, lr);
        }
        tmem_wait_st();
      } else {
        for (int L = 0; L < NL; ++L) {
          const uint32_t ta = lane_base + (ab * NL + L) * TS + CPT * h;
#pragma unroll
          for (int c0 = 0; c0 < CPT; c0 += 8) {
            uint32_t r[8];
            tmem_ld8(ta + c0, r);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 8; ++c)
              dfloat_add(hi[c0 + c], lo[(c0 + c) % NLO], __uint_as_float(r[c]));
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
    }
    if (ok) {
      const int row = tm * BM + q * 32 + lane;
      const bool row_ok = row < p.a_rows;
      const int ea = row_ok ? p.ea[row] : 0;
      const double ra = (row_ok && p.rsa) ? p.rsa[row] : 1.0;
      double2* out = p.out + (long)batch * p.out_bstride + (long)(row_ok ? row : 0) * p.ld_row;
      const int* eb = p.eb + (long)batch * p.eb_stride;
#pragma unroll
      for (int c0 = 0; c0 < CPT; c0 += 8) {
        uint32_t lr[8];
        if (kLoTmem) {
          tmem_ld8(lo_base + c0, lr);  // warp-collective: before any per-row branch
          tmem_wait_ld();
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) lr[c] = __float_as_uint(lo[kLoTmem ? 0 : c0 + c]);
        }
#pragma unroll
        for (int c = 0; c < 8; c += 2) {
          const int col = tn * BN + CPT * h + c0 + c;
          if (row_ok && col < p.b_rows) {
            const int j = col >> 1;
            double sc = p.alpha * pow2(ea + eb[j] - 14) * ra;
            if (p.rsb) sc *= p.rsb[j];
            double re = ((double)hi[c0 + c] + (double)__uint_as_float(lr[c])) * sc;
            double im = ((double)hi[c0 + c + 1] + (double)__uint_as_float(lr[c + 1])) * sc;
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

// Y = round(x 2^(7 + 8(S-1) - e)) for |x| < 2^e, whose signed base-256 digits
// give x ~= 2^(e-7) sum_s d_s 2^(-8s), integer |d_s| <= 128 (exact in BF16).
// Pure integer arithmetic on the IEEE fields (GB300's FP64 pipe is narrow).
__device__ __forceinline__ long long digits_y(double x, int e, int S) {
  const long long bits = __double_as_longlong(x);
  const int bexp = (int)((bits >> 52) & 0x7FF);
  const int F = 7 + 8 * (S - 1);
  long long Y = 0;
  if (bexp != 0) {  // zero and subnormals give zero digits
    const long long mant = (bits & ((1LL << 52) - 1)) | (1LL << 52);
    const int sh = bexp - 1075 + F - e;  // Y = mant 2^sh
    if (sh >= 0)
      Y = mant << sh;  // < 2^(7 + 8(S-1)) <= 2^63 since |x| < 2^e
    else if (sh > -63)
      Y = (mant + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) Y = -Y;
  }
  return Y;
}

// The signed base-256 digits of Y = sum_s d_s 256^(S-1-s) for a complex value
// (yr, yi), |d_s| <= 128 for s >= 1 (and for s = 0 when |Y| < 2^(7 + 8(S-1))),
// least significant first, handed to put(s, d_s^r 2^-8s, d_s^i 2^-8s) one plane at
// a time.  The pre-scaled digit d_s 2^-8s is exact in BF16, and the product of
// digits s and t then carries its level's weight 2^-8(s+t) by itself.
template <class Put>
__device__ __forceinline__ void emit_digits(long long yr, long long yi, int S, Put put) {
#pragma unroll 1
  for (int s = S - 1; s >= 0; --s) {
    int dr, di;
    if (s > 0) {
      dr = (int)((yr + 128) & 255) - 128;
      di = (int)((yi + 128) & 255) - 128;
      yr = (yr - dr) >> 8;
      yi = (yi - di) >> 8;
    } else {
      dr = (int)yr;
      di = (int)yi;
    }
    const float sc = __int_as_float((127 - 8 * s) << 23);
    put(s, (float)dr * sc, (float)di * sc);
  }
}

// Digit planes hold (re, im) pairs of BF16 (kind::f16) or of TF32 values in FP32
// storage (kind::tf32, the split precision RPA_MIXED_TF32X3).
template <typename P>
struct PlaneT;
template <>
struct PlaneT<__nv_bfloat162> {
  __device__ static void put(__nv_bfloat162* p, float a, float b) {
    *p = __floats2bfloat162_rn(a, b);
  }
  // round-to-nearest BF16
  __device__ static float round(double y) { return __bfloat162float(__double2bfloat16(y)); }
};
template <>
struct PlaneT<float2> {
  __device__ static void put(float2* p, float a, float b) { *p = make_float2(a, b); }
  // round to nearest FP32, then to TF32 (10 stored mantissa bits, ties away)
  __device__ static float round(double y) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)y));
    return __uint_as_float(r);
  }
};

// Round-to-nearest split of the row-scaled value y = x 2^(7 - e), |y| < 128: the first
// plane the plane type's rounding of y, each further plane the rounding of what the
// earlier planes leave (the classic hi/lo split).  Used by the split precisions
// (RPA_MIXED_BF16X3 / X6, RPA_MIXED_TF32X3), whose products are summed in FP32 over
// the whole K.
template <typename P, class Put>
__device__ __forceinline__ void emit_split(double xr, double xi, int e, int S, Put put) {
  const double sc = ldexp(1.0, 7 - e);
  double yr = xr * sc, yi = xi * sc;
#pragma unroll 1
  for (int s = 0; s < S; ++s) {
    const float hr = PlaneT<P>::round(yr);
    const float hi = PlaneT<P>::round(yi);
    put(s, hr, hi);
    yr -= (double)hr;
    yi -= (double)hi;
  }
}

// Y = round(x f 2^(7 + 8(S-1) - e)) for |x f| < 2^e and S <= 3 without an FP64
// multiply: the product of the leading 31 bits of both
// significands (relative error below 2^-29) is rounded to the at most 23-bit Y,
// so Y can differ from the digits of the FP64 product only where x f 2^(F-e)
// lies within 2^-6 of a rounding tie, by one unit of the last digit.
constexpr int PROD_DIGITS_MAX_S = 3;
__device__ __forceinline__ long long digits_y_prod(double x, double f, int e, int S) {
  const long long bx = __double_as_longlong(x), bf = __double_as_longlong(f);
  const int ex = (int)((bx >> 52) & 0x7FF), ef = (int)((bf >> 52) & 0x7FF);
  long long Y = 0;
  if (ex != 0 && ef != 0) {  // zero and subnormal factors give zero digits
    const unsigned long long mx = ((bx & ((1LL << 52) - 1)) | (1LL << 52)) >> 22;  // [2^30, 2^31)
    const unsigned long long mf = ((bf & ((1LL << 52) - 1)) | (1LL << 52)) >> 22;
    const unsigned long long m = mx * mf;  // x f ~= m 2^(ex + ef - 2106), m < 2^62
    const int sh = ex + ef - 2106 + 7 + 8 * (S - 1) - e;  // Y = m 2^sh, sh < -36
    if (sh > -63) Y = (long long)((m + (1ULL << (-sh - 1))) >> (-sh));
    if ((bx ^ bf) < 0) Y = -Y;
  }
  return Y;
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

// chi0 operand X[r][g] = sf[vc] A[vc][g] for the transitions vc = order[r],
// r < n_rows, of one K-block (v^1/2 is applied per output row in the GEMM
// epilogue): row maxima over the block per g.
__global__ void chi0_rowmax_kernel(const void* A, int dtype, const int* order, int n_rows,
                                   int n_g, const double* sf, unsigned long long* rowmax) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_g) return;
  double m = 0.0;
  for (int r = blockIdx.y; r < n_rows; r += gridDim.y) {
    const int vc = order[r];
    double2 a = load_any(A, dtype, (long)vc * n_g + g);
    double s = sf[vc];
    m = fmax(m, fmax(fabs(a.x * s), fabs(a.y * s)));
  }
  atomic_max_pos(rowmax + g, m);
}

// chi0 operand planes, [S][2 n_g_pad][K], K index 2 vc + part: row 2g holds
// (x_r, x_i), row 2g+1 holds (x_i, -x_r), so that Re chi = X_g . X_h and
// Im chi = X_g . Y_h.  One 32 x 32 (vc, g) tile per block, transposed through
// shared memory so that the plane rows are written contiguously.
template <typename P>
__global__ void chi0_slice_kernel(const void* A, int dtype, const int* order, int n_vc, int n_g,
                                  int n_g_pad, long K, const double* sf,
                                  const unsigned long long* rowmax, int S, P* planes, int* exps,
                                  int split) {
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
    int vr = vc0 + r, g = g0 + tx;
    double2 x = make_double2(0.0, 0.0);
    if (vr < n_vc && g < n_g) {
      const int vc = order[vr];
      x = load_any(A, dtype, (long)vc * n_g + g);
      double s = sf[vc];
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
    P* p = planes + (long)(2 * g) * (K / 2) + vc;
    auto put = [&](int s, float fr, float fi) {
      P* p0 = p + s * plane;
      PlaneT<P>::put(p0, fr, fi);
      PlaneT<P>::put(p0 + K / 2, fi, -fr);
    };
    if (split)
      emit_split<P>(x.x, x.y, es[r], S, put);
    else
      emit_digits(digits_y(x.x, es[r], S), digits_y(x.y, es[r], S), S, put);
  }
}

constexpr int CHUNK = 2048;  // complex elements of one row handled by one block

// Row maxima max_k max(|Re x|, |Im x|) of a complex matrix (row stride `ld`
// complex elements, n_cplx valid columns); grid (rows, column chunks).
__global__ void row_max_kernel(const void* src, int dtype, long ld, int n_rows, int n_cplx,
                               unsigned long long* rowmax) {
  __shared__ double red[32];
  const int r = blockIdx.x;
  const long k0 = (long)blockIdx.y * CHUNK, k1 = min((long)n_cplx, k0 + CHUNK);
  double m = 0.0;
  if (r < n_rows)
    for (long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
      double2 x = load_any(src, dtype, (long)r * ld + k);
      m = fmax(m, fmax(fabs(x.x), fabs(x.y)));
    }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) mm = fmax(mm, red[i]);
    if (r < n_rows && mm > 0.0) atomic_max_pos(rowmax + r, mm);
  }
}

// Row slicing: planes [S][rows_pad][K] with K index 2 k + part, from the row
// maxima; grid (rows_pad, K/2 chunks).
template <typename P>
__global__ void slice_rows_kernel(const void* src, int dtype, long ld, int n_rows, int n_cplx,
                                  int rows_pad, long K, int S,
                                  const unsigned long long* rowmax, P* planes, int* exps,
                                  int split) {
  const int r = blockIdx.x;
  const int e = r < n_rows ? row_exponent(__longlong_as_double((long long)rowmax[r])) : 0;
  if (blockIdx.y == 0 && threadIdx.x == 0) exps[r] = e;
  const long plane = (long)rows_pad * (K / 2);
  const long k0 = (long)blockIdx.y * CHUNK, k1 = min(K / 2, k0 + CHUNK);
  for (long k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    double2 x = make_double2(0.0, 0.0);
    if (r < n_rows && k < n_cplx) x = load_any(src, dtype, (long)r * ld + k);
    P* p = planes + (long)r * (K / 2) + k;
    auto put = [&](int s, float fr, float fi) { PlaneT<P>::put(p + s * plane, fr, fi); };
    if (split)
      emit_split<P>(x.x, x.y, e, S, put);
    else
      emit_digits(digits_y(x.x, e, S), digits_y(x.y, e, S), S, put);
  }
}

// Projection B operand from B[g][i] (= v^1/2 C): rows 2i = (b_r, -b_i) and
// 2i+1 = (b_i, b_r) along K index 2g + part; one block per i.
template <typename P>
__global__ void proj_b_slice_kernel(const double2* B, int n_g, int n_eig, int n_eig_pad, long K,
                                    int S, P* planes, int* exps, int split) {
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
    P* p = planes + (long)(2 * i) * (K / 2) + g;
    auto put = [&](int s, float fr, float fi) {
      P* p0 = p + s * plane;
      PlaneT<P>::put(p0, fr, -fi);
      PlaneT<P>::put(p0 + K / 2, fi, fr);
    };
    if (split)
      emit_split<P>(b.x, b.y, e, S, put);
    else
      emit_digits(digits_y(b.x, e, S), digits_y(b.y, e, S), S, put);
  }
}

// f[b][vc] = ow[vc] 4 D / (D^2 + w_{k0+b}^2) for the frequencies of one group.
// Row maxima of f_b(vc) |M~[j][vc]| for the nb frequencies of a group;
// grid (n_eig, vc chunks); rowmax[b * stride + j].  The products are formed in
// FP32 from copies of f and |M~| rounded up and are rounded up themselves, so
// each maximum bounds the FP64 one from above (a row exponent may come out one
// larger, never smaller); a product above the FP32 range is taken in FP64.
constexpr int MAX_GROUP = 8;   // frequencies per chis_b kernel launch (upper bound)
constexpr int RMR = 4;         // rows of M~ per block of the chi_s operand kernels
constexpr int CHIS_PLANE_GB = 64;  // default budget of the two chi_s B plane buffers
constexpr int PROJ_PLANE_GB = 48;  // default budget of the projection's A planes
__global__ void chis_b_rowmax_kernel(const double2* mt, int n_eig, int n_vc, const float* f_up,
                                     const double* f, int nb, unsigned long long* rowmax,
                                     int stride) {
  // RMR rows of M~ per block, so that each f value read serves RMR rows
  __shared__ double red[RMR][MAX_GROUP][8];
  __shared__ int ovf_s;
  const int j0 = blockIdx.x * RMR;
  const long v0 = (long)blockIdx.y * CHUNK, v1 = min((long)n_vc, v0 + CHUNK);
  if (threadIdx.x == 0) ovf_s = 0;
  __syncthreads();
  float m[RMR][MAX_GROUP];
#pragma unroll
  for (int r = 0; r < RMR; ++r)
#pragma unroll
    for (int b = 0; b < MAX_GROUP; ++b) m[r][b] = 0.f;
  bool ovf = false;
  for (long vc = v0 + threadIdx.x; vc < v1; vc += blockDim.x) {
    float a[RMR];
#pragma unroll
    for (int r = 0; r < RMR; ++r) {
      const double2 x = j0 + r < n_eig ? mt[(long)(j0 + r) * n_vc + vc] : make_double2(0.0, 0.0);
      a[r] = __double2float_ru(fmax(fabs(x.x), fabs(x.y)));
    }
#pragma unroll
    for (int b = 0; b < MAX_GROUP; ++b)
      if (b < nb) {
        const float fu = f_up[(long)b * n_vc + vc];
#pragma unroll
        for (int r = 0; r < RMR; ++r) {
          const float pr = __fmul_ru(fu, a[r]);
          if (pr <= 3.0e38f)
            m[r][b] = fmaxf(m[r][b], pr);
          else
            ovf = true;
        }
      }
  }
  if (ovf) ovf_s = 1;
#pragma unroll
  for (int r = 0; r < RMR; ++r)
#pragma unroll
    for (int b = 0; b < MAX_GROUP; ++b) {
      float v = m[r][b];
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if ((threadIdx.x & 31) == 0) red[r][b][threadIdx.x >> 5] = (double)v;
    }
  __syncthreads();
  if (ovf_s) {
    // a product beyond the FP32 range (rare): this block's maxima in FP64 instead
    for (int q = 0; q < RMR * nb; ++q) {
      const int r = q / nb, b = q % nb;
      double v = 0.0;
      if (j0 + r < n_eig)
        for (long vc = v0 + threadIdx.x; vc < v1; vc += blockDim.x) {
          const double2 x = mt[(long)(j0 + r) * n_vc + vc];
          v = fmax(v, f[(long)b * n_vc + vc] * fmax(fabs(x.x), fabs(x.y)));
        }
      for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[r][b][threadIdx.x >> 5] = v;
      __syncthreads();
    }
  }
  if (threadIdx.x < RMR * nb) {
    const int r = threadIdx.x / nb, b = threadIdx.x % nb, j = j0 + r;
    double mm = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, red[r][b][w]);
    if (j < n_eig && mm > 0.0) atomic_max_pos(rowmax + (long)b * stride + j, mm);
  }
}

// f rounded up to FP32 (finite f >= 0)
__global__ void float_up_kernel(const double* f, long n, float* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = __double2float_ru(f[i]);
}

// chi_s B operand of the group's frequencies: for row j, f_b(vc) M~[j][vc] as
// rows 2j = (f m_r, f m_i) and 2j+1 = (-f m_i, f m_r); RMR rows j per block (each f
// value read serves all of them), grid (ceil(n_eig_pad / RMR), chunks).
template <typename P>
__global__ void chis_b_slice_kernel(const double2* mt, int n_eig, int n_eig_pad, int n_vc,
                                    long K, const double* f, int nb, int S,
                                    const unsigned long long* rowmax, P* planes, int* exps,
                                    int eb_stride, int split) {
  const int j0 = blockIdx.x * RMR;
  __shared__ int e[RMR][MAX_GROUP];
  if (threadIdx.x < RMR * MAX_GROUP) {
    const int r = threadIdx.x / MAX_GROUP, b = threadIdx.x % MAX_GROUP, j = j0 + r;
    e[r][b] = (b < nb && j < n_eig)
                  ? row_exponent(__longlong_as_double((long long)rowmax[(long)b * eb_stride + j]))
                  : 0;
    if (blockIdx.y == 0 && b < nb && j < n_eig_pad) exps[b * eb_stride + j] = e[r][b];
  }
  __syncthreads();
  const long plane = (long)2 * n_eig_pad * (K / 2);
  const long v0 = (long)blockIdx.y * CHUNK, v1 = min(K / 2, v0 + CHUNK);
  for (long vc = v0 + threadIdx.x; vc < v1; vc += blockDim.x) {
    double2 x[RMR];
#pragma unroll
    for (int r = 0; r < RMR; ++r)
      x[r] = (j0 + r < n_eig && vc < n_vc) ? mt[(long)(j0 + r) * n_vc + vc]
                                           : make_double2(0.0, 0.0);
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
      const double fv = vc < n_vc ? f[(long)b * n_vc + vc] : 0.0;
#pragma unroll
      for (int r = 0; r < RMR; ++r) {
        const int j = j0 + r;
        if (j >= n_eig_pad) break;
        P* p = planes + (long)(b * S) * plane + (long)(2 * j) * (K / 2) + vc;
        if (split) {
          emit_split<P>(fv * x[r].x, fv * x[r].y, e[r][b], S, [&](int s, float fr, float fi) {
            P* p0 = p + s * plane;
            PlaneT<P>::put(p0, fr, fi);
            PlaneT<P>::put(p0 + K / 2, -fi, fr);
          });
          continue;
        }
        long long yr, yi;
        if (S <= PROD_DIGITS_MAX_S) {
          yr = digits_y_prod(x[r].x, fv, e[r][b], S);
          yi = digits_y_prod(x[r].y, fv, e[r][b], S);
        } else {
          yr = digits_y(fv * x[r].x, e[r][b], S);
          yi = digits_y(fv * x[r].y, e[r][b], S);
        }
        emit_digits(yr, yi, S, [&](int s, float fr, float fi) {
          P* p0 = p + s * plane;
          PlaneT<P>::put(p0, fr, fi);
          PlaneT<P>::put(p0 + K / 2, -fi, fr);
        });
      }
    }
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

inline long rup(long a, long b) { return (a + b - 1) / b * b; }
inline int cdiv(long a, long b) { return (int)((a + b - 1) / b); }

int env_int(const char* name, int dflt);

int drain_tiles(int Le) {
  // exact FP32 sums need K_d * (L+1) * 2^14 <= 2^24 for every exact level L <= Le-1
  int kd = (1024 / Le) / BK * BK;
  return std::max(1, kd / BK);
}

// Level accumulators for S slices of which Le are exact: Le, plus one tail.
int n_levels(int S, int Le) { return Le < S ? Le + 1 : S; }

// Exact levels per stage: chi~(0) and chi_s with S >= 3 slices keep their two
// lowest-weight levels in the tail (weights 2^-8(S-2) and below relative to the
// leading level; the FP32 rounding of their sum stays below the truncation of
// the digit expansion); the projection, whose accuracy the whole subspace rests on
// and whose sums cancel strongly, keeps all but its last level exact: the tail then
// holds level S-1 alone (weight 2^-8(S-1)), whose FP32 rounding lies ~2^-9 below the
// truncation, it occupies level S-1's own columns (the MMAs are those of all-exact
// levels), and the drain interval grows from 2 to 3 K-tiles at S = 6.  chi~(0) at S = 4 keeps only level 0 exact:
// the tail's FP32 rounding (~2^-32 of the leading level per interval) then matches
// the truncation (2^-31), the drain interval doubles to 16 K-tiles and one
// accumulator fewer is drained (measured at N_G = 4000: |dE_c| 1.2e-7 / 1.0e-8 /
// 4.5e-8 Ha at N_eig = 200 / 400 / 800 against the FP64 path, chi~ 9% faster).
// RPA_TC_LE_<STAGE> overrides (tuning).
int clamp_levels(int Le, int S) { return std::max(1, std::min(S, Le)); }
int exact_levels_chi0(int S) {
  return clamp_levels(env_int("RPA_TC_LE_CHI0", S == 4 ? 1 : (S >= 3 ? S - 2 : S)), S);
}
int exact_levels_proj(int S) {
  return clamp_levels(env_int("RPA_TC_LE_PROJ", S >= 2 ? S - 1 : S), S);
}
int exact_levels_chis(int S) {
  return clamp_levels(env_int("RPA_TC_LE_CHIS", S >= 3 ? S - 2 : S), S);
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

// 3-D map over digit planes (BF16, or TF32 in FP32 storage when tf32): dim0 = K
// (contiguous), dim1 = rows (row_bytes apart), dim2 = plane (plane_bytes apart); box
// 128 bytes of K x box_rows x 1, 128-byte swizzle.
bool make_map(CUtensorMap* m, void* base, long K, long rows, long planes, long row_bytes,
              long plane_bytes, int box_rows, std::string& err, bool tf32 = false) {
  auto fn = encode_fn();
  if (!fn) {
    err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)plane_bytes};
  cuuint32_t box[3] = {(cuuint32_t)bk_elems(tf32), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char b[160];
    snprintf(b, sizeof b, "cuTensorMapEncodeTiled failed (%d): K=%ld rows=%ld planes=%ld", (int)r,
             K, rows, planes);
    err = b;
    return false;
  }
  return true;
}

// Tuning knobs of the GEMM pipeline (environment overrides for autotuning):
// RPA_TC_NA (A ring depth), RPA_TC_NB (B buffers), RPA_TC_NACC (TMEM level
// accumulator sets), RPA_TC_GROUP (tile rows per rasterisation group).
int env_int(const char* name, int dflt) {
  const char* v = getenv(name);
  return v && *v ? atoi(v) : dflt;
}

// B rows per tile: 128 when the level accumulators of 128 columns and the 128
// columns of double-float low halves fit in TMEM (at most 3 accumulators),
// else 64.  Level accumulators start at multiples of 64 TMEM columns.
int pick_bn(int S, int Le) {
  const int cap = env_int("RPA_TC_BN", 128);
  if (cap >= 128 && (n_levels(S, Le) + 1) * 128 <= 512) return 128;
  return 64;
}

// Pipeline shape for S slices: the deepest A ring and B buffering that fit in
// shared memory (up to the knobs), two TMEM accumulator sets when they fit.
void gemm_shape(int S, int Le, size_t smem_limit, int* na, int* nb, int* nacc) {
  const int BN = pick_bn(S, Le), NL = n_levels(S, Le);
  const size_t B_TILE = (size_t)BN * BK * 2;
  const int want_na = std::min(MAX_NA, std::max(2, env_int("RPA_TC_NA", MAX_NA)));
  const int want_nb = std::min(MAX_NB, std::max(2, env_int("RPA_TC_NB", 2)));
  const int want_acc = std::min(2, std::max(1, env_int("RPA_TC_NACC", 2)));
  *nacc = (want_acc == 2 && BN == 64 && 2 * NL * BN <= 512) ? 2 : 1;  // BN 128: one set
  for (int b = want_nb; b >= 2; --b)
    for (int a = want_na; a >= 2; --a)
      if (1024 + (size_t)a * A_TILE + (size_t)b * S * B_TILE <= smem_limit) {
        *na = a;
        *nb = b;
        return;
      }
  *na = 2;
  *nb = 2;
}

size_t gemm_smem(int S, int Le, size_t smem_limit) {
  int na, nb, nacc;
  gemm_shape(S, Le, smem_limit, &na, &nb, &nacc);
  return 1024 + (size_t)na * A_TILE + (size_t)nb * S * ((size_t)pick_bn(S, Le) * BK * 2);
}

// Build the work list (upper block triangle when `upper`), choose split-K, launch.
rpa_status run_gemm(Workspace& w, const CUtensorMap& ta, const CUtensorMap& tb, GemmArgs a,
                    int tiles_m, int batches, bool upper, void* zero_ptr,
                    size_t zero_bytes, cudaStream_t st, std::string& err, int* launches) {
  std::vector<int4> work;
  const int BN = pick_bn(a.S, a.nexact);
  const int tiles_n = cdiv(a.b_rows, BN);
  // split precisions sum in FP32 over the whole K (one drain at the end)
  const int bke = bk_elems(w.tf32 != 0);
  const int kdt = w.split ? std::max(1, a.K / bke) : drain_tiles(std::min(a.nexact, a.S));
  const int kd = kdt * bke;
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
  if (a.accumulate) {
    a.atomic = 1;  // the caller zeroed the output and adds several K-blocks
  } else if (split > 1) {
    // split-K partial tiles are summed with FP64 atomics into a zeroed output
    cudaError_t ez = cudaMemsetAsync(zero_ptr, 0, zero_bytes, st);
    if (ez != cudaSuccess) {
      err = cudaGetErrorString(ez);
      return RPA_ECUDA;
    }
    a.atomic = 1;
  }
  // Rasterised order: groups of `grp` tile rows are walked column by column, so
  // the CTAs resident at one time share a few A row-tiles and a few B row-tiles
  // and the operands stream from HBM about once per group instead of per row.
  const int grp = std::max(1, env_int("RPA_TC_GROUP", 8));
  for (int b = 0; b < batches; ++b)
    for (int m0 = 0; m0 < tiles_m; m0 += grp)
      for (int n = 0; n < tiles_n; ++n)
        for (int m = m0; m < std::min(tiles_m, m0 + grp); ++m)
          if (!upper || (long)n * BN / 2 + BN / 2 - 1 >= (long)m * BM)
            for (int s = 0; s < split; ++s) work.push_back(make_int4(m, n, b, s));
  if (work.size() > w.work_count) {
    err = "work list exceeds workspace";
    return RPA_ENOMEM;
  }
  if (work.empty()) return RPA_OK;
  // Work lists repeat from call to call (the 32 chi~ K-blocks, every step of a
  // q-point), so each distinct list is uploaded once and kept in the device work
  // buffer: no host-to-device copy (which could queue behind a large input copy
  // on the copy engine) in the steady state.
  cudaError_t e = cudaSuccess;
  size_t at = SIZE_MAX;
  for (const auto& c : w.work_cache)
    if (c.first.size() == work.size() &&
        std::equal(work.begin(), work.end(), c.first.begin(), [](const int4& x, const int4& y) {
          return x.x == y.x && x.y == y.y && x.z == y.z && x.w == y.w;
        })) {
      at = c.second;
      break;
    }
  if (at == SIZE_MAX) {
    if (w.work_used + work.size() > w.work_count) {
      w.work_cache.clear();  // start over; earlier launches are ordered before the copy
      w.work_used = 0;
    }
    at = w.work_used;
    e = cudaMemcpyAsync(w.work + at, work.data(), work.size() * sizeof(int4),
                        cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      err = cudaGetErrorString(e);
      return RPA_ECUDA;
    }
    w.work_cache.emplace_back(work, at);
    w.work_used += work.size();
  }
  a.work = w.work + at;
  a.status = w.status;
  a.stall = w.debug_stall;
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    err = std::string("slice GEMM: no usable current device: ") + cudaGetErrorString(e);
    return RPA_ECUDA;
  }
  std::unique_lock<std::mutex> lock(g_limits_mutex);
  DeviceLimits& lim_dev = g_limits[dev];
  if (!lim_dev.smem) {
    // opt-in shared memory per block minus the kernels' static shared memory
    int optin = 0, sms = 0;
    cudaFuncAttributes fa[4]{};
    const void* kern[4] = {(const void*)slice_gemm_kernel<64, false>,
                           (const void*)slice_gemm_kernel<128, false>,
                           (const void*)slice_gemm_kernel<64, true>,
                           (const void*)slice_gemm_kernel<128, true>};
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
        cudaSuccess) {
      err = std::string("querying shared memory limits: ") + cudaGetErrorString(e);
      return RPA_ECUDA;
    }
    size_t stat = 0;
    for (int i = 0; i < 4; ++i) {
      if ((e = cudaFuncGetAttributes(&fa[i], kern[i])) != cudaSuccess) {
        err = std::string("querying shared memory limits: ") + cudaGetErrorString(e);
        return RPA_ECUDA;
      }
      stat = std::max(stat, fa[i].sharedSizeBytes);
    }
    size_t lim = (size_t)optin - stat;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i)
      e = cudaFuncSetAttribute(kern[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
    if (e != cudaSuccess) {
      err = std::string("cudaFuncSetAttribute(max dynamic smem): ") + cudaGetErrorString(e);
      return RPA_ECUDA;
    }
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
      err = std::string("querying the SM count: ") + cudaGetErrorString(e);
      return RPA_ECUDA;
    }
    lim_dev.sms = sms;
    lim_dev.smem = lim;
  }
  const DeviceLimits limits = lim_dev;
  lock.unlock();
  gemm_shape(a.S, a.nexact, limits.smem, &a.na, &a.nb, &a.nacc);
  const size_t smem = gemm_smem(a.S, a.nexact, limits.smem);
  if (smem > limits.smem) {
    err = "slice GEMM: shared memory of the pipeline exceeds the device limit";
    return RPA_EINVAL;
  }
  // persistent: one CTA per SM (the pipeline fills the shared memory), each taking every
  // grid-th tile of the rasterised list, so a tile's epilogue overlaps the next tile's MMAs
  a.n_work = (int)work.size();
  const unsigned grid = (unsigned)std::min<long>(
      a.n_work, std::max(1, env_int("RPA_TC_GRID", limits.sms > 0 ? limits.sms : a.n_work)));
  if (w.tf32) {
    if (BN == 128)
      slice_gemm_kernel<128, true><<<grid, threads_for<128>(), smem, st>>>(ta, tb, a);
    else
      slice_gemm_kernel<64, true><<<grid, threads_for<64>(), smem, st>>>(ta, tb, a);
  } else {
    if (BN == 128)
      slice_gemm_kernel<128, false><<<grid, threads_for<128>(), smem, st>>>(ta, tb, a);
    else
      slice_gemm_kernel<64, false><<<grid, threads_for<64>(), smem, st>>>(ta, tb, a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("slice GEMM launch: ") + cudaGetErrorString(e);
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
  // chi_s: two alternating buffers of the B planes of up to MAX_GROUP frequencies,
  // as many as fit in a budget (RPA_TC_CHIS_GB, default 64 GB) for both buffers
  const double per_freq = (double)s.chis * 2 * e_pad * k_vc * 2;
  const long budget = (long)std::max(1, env_int("RPA_TC_CHIS_GB", CHIS_PLANE_GB)) << 30;
  const int fit = (int)std::max(1.0, std::floor(budget / (2.0 * per_freq)));
  const int grp = (int)std::min<size_t>(
      std::max(1, std::min({MAX_GROUP, fit, env_int("RPA_TC_CHIS_GROUP", MAX_GROUP)})), max_freq);
  w.freq_group = grp;
  w.chis_overlap = env_int("RPA_TC_CHIS_OVERLAP", 1) != 0;
  w.chi0_blocks = std::max(1, env_int("RPA_TC_CHI0_BLOCKS", 32));
  const long k_blk = rup(2 * rup(cdiv(max_vc, w.chi0_blocks), 32), BK);
  // projection: the A planes of all rows if they fit in the budget (RPA_TC_PROJ_GB,
  // default 48 GB), else chunks of rows (tile-height multiples) one after another
  const long proj_budget = (long)std::max(1, env_int("RPA_TC_PROJ_GB", PROJ_PLANE_GB)) << 30;
  const long proj_row_bytes = (long)s.proj * k_g * 2;
  w.proj_chunk = std::max<long>(BM, std::min<long>(vc_pad, proj_budget / proj_row_bytes / BM * BM));
  if (env_int("RPA_TC_PROJ_CHUNK", 0) > 0)  // test hook: force small chunks
    w.proj_chunk = std::max<long>(BM, rup(env_int("RPA_TC_PROJ_CHUNK", 0), BM));
  // chi~(0) double-buffers the planes of its K-blocks (one cut while the other multiplies)
  size_t p1 = std::max({(size_t)2 * s.chi0 * 2 * g_pad * k_blk,
                        (size_t)s.proj * std::min<long>(vc_pad, w.proj_chunk) * k_g,
                        (size_t)2 * grp * s.chis * 2 * e_pad * k_vc});
  size_t p2 = std::max((size_t)s.proj * 2 * e_pad * k_g, (size_t)s.chis * e_pad * k_vc);
  // the eigensolver's block products (chi~ times N_eig + p columns and smaller) run on
  // the projection GEMM with EIG_SLICES planes
  p1 = std::max(p1, (size_t)EIG_SLICES * g_pad * k_g);
  p2 = std::max(p2, (size_t)EIG_SLICES * 2 * e_pad * k_g);
  w.plane_bytes = p1 * 2;
  w.plane2_bytes = p2 * 2;
  w.exp_count = std::max({(size_t)g_pad, (size_t)vc_pad, (size_t)e_pad}) +
                std::max((size_t)g_pad, (size_t)2 * grp * e_pad);
  // chi_s: the A operand's row maxima (e_pad) beside the B operand's two groups
  w.rowmax_count = std::max({(size_t)2 * g_pad, (size_t)vc_pad, (size_t)(2 * grp + 1) * e_pad});
  w.work_count = 1 << 20;
  w.fweight_count = max_freq * max_vc;
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
      !al((void**)&w.fweights, w.fweight_count * sizeof(float))) {
    free_workspace(w);
    return RPA_ENOMEM;
  }
  cudaError_t e = cudaMemset(w.status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking);
  cudaEvent_t* evs[] = {&w.ev_in, &w.ev_side_last, &w.ev_sliced[0], &w.ev_sliced[1],
                        &w.ev_gemm[0], &w.ev_gemm[1]};
  for (cudaEvent_t* ev : evs)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  // a completed marker: the first join waits for nothing
  if (e == cudaSuccess) e = cudaEventRecord(w.ev_side_last, w.side);
  if (e != cudaSuccess) {
    err = std::string("tensor-core workspace streams and events: ") + cudaGetErrorString(e);
    free_workspace(w);
    return RPA_ECUDA;
  }
  return RPA_OK;
}

void free_workspace(Workspace& w) {
  if (w.side) cudaStreamSynchronize(w.side);
  void* b[] = {w.planes, w.planes2, w.exps, w.rowmax, w.work, w.status, w.fweights};
  for (void* p : b)
    if (p) cudaFree(p);
  cudaEvent_t evs[] = {w.ev_in, w.ev_side_last, w.ev_sliced[0], w.ev_sliced[1], w.ev_gemm[0],
                       w.ev_gemm[1]};
  for (cudaEvent_t ev : evs)
    if (ev) cudaEventDestroy(ev);
  if (w.side) cudaStreamDestroy(w.side);
  w = Workspace{};
}

rpa_status join_side(Workspace& w, cudaStream_t st, std::string& err) {
  CK(cudaStreamWaitEvent(st, w.ev_side_last, 0));
  return RPA_OK;
}

// The side stream waits for the work queued so far on the caller's stream.
static rpa_status side_fork(Workspace& w, cudaStream_t st, std::string& err) {
  CK(cudaEventRecord(w.ev_in, st));
  CK(cudaStreamWaitEvent(w.side, w.ev_in, 0));
  return RPA_OK;
}

template <typename P>
rpa_status chi0_t(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const double* sf,
                const int* order, const double* sv, double scale, cplx* chi, cudaStream_t st,
                std::string& err, int* launches, bool zero, int blocks) {
  constexpr int EB = (int)sizeof(P) / 2;  // bytes of one plane element
  constexpr bool TFP = sizeof(P) == 8;
  const int S = w.slices.chi0, Le = w.split ? 1 : exact_levels_chi0(S);
  const long g_pad = rup(n_g, BM);
  // K-blocks of the transitions in `order` (sorted by sqrt f(0)): each block has
  // its own per-row digit exponents, so rows keep more significant bits where
  // the transition weights of the block are smaller than the overall maximum.
  const int nblk =
      std::max(1, std::min(blocks > 0 ? blocks : w.chi0_blocks, cdiv(n_vc, 32)));
  const long per = rup(cdiv(n_vc, nblk), 32);
  // Two plane buffers: block b is cut on the side stream while block b-1 is
  // multiplied on `st`; buffer b % 2 is reused once the GEMM of block b-2 is done.
  const size_t buf_elems = (size_t)S * 2 * g_pad * rup(2 * per, BK);  // BF16 pairs / 2
  w.proj_a.valid = false;
  if (zero) CK(cudaMemsetAsync(chi, 0, sizeof(cplx) * (size_t)n_g * n_g, st));
  if (side_fork(w, st, err) != RPA_OK) return RPA_ECUDA;
  int b = 0;
  for (long r0 = 0; r0 < n_vc; r0 += per, ++b) {
    const int buf = b & 1;
    const int nr = (int)std::min<long>(per, n_vc - r0);
    const long K = rup(2L * nr, BK);
    P* planes = (P*)w.planes + buf * (buf_elems / 2);
    int* exps = w.exps + buf * g_pad;
    unsigned long long* rowmax = w.rowmax + buf * g_pad;
    if (b >= 2) CK(cudaStreamWaitEvent(w.side, w.ev_gemm[buf], 0));
    CK(cudaMemsetAsync(rowmax, 0, g_pad * sizeof(unsigned long long), w.side));
    {
      dim3 grid(cdiv(n_g, 128), std::min(cdiv(nr, 64), 512));
      chi0_rowmax_kernel<<<grid, 128, 0, w.side>>>(A, dtype, order + r0, nr, n_g, sf, rowmax);
      CK(cudaGetLastError());
    }
    {
      dim3 grid(cdiv(K / 2, 32), cdiv(g_pad, 32));
      chi0_slice_kernel<P><<<grid, dim3(32, 8), 0, w.side>>>(A, dtype, order + r0, nr, n_g,
                                                          (int)g_pad, K, sf, rowmax, S, planes,
                                                          exps, w.split);
      CK(cudaGetLastError());
    }
    CK(cudaEventRecord(w.ev_sliced[buf], w.side));
    CK(cudaEventRecord(w.ev_side_last, w.side));
    if (launches) *launches += 2;
    // the slice timer measures how long `st` waits for the cut planes
    w.hook(RPA_T_SLICE, 1);
    CK(cudaStreamWaitEvent(st, w.ev_sliced[buf], 0));
    w.hook(RPA_T_SLICE, 0);
    CUtensorMap ta, tb;
    const long plane_bytes = 2 * g_pad * K * EB;
    // A view: even rows of the planes (X_g); B: all rows (X_h, Y_h interleaved)
    if (!make_map(&ta, planes, K, g_pad, S, 2 * K * EB, plane_bytes, BM, err, TFP)) return RPA_ECUDA;
    if (!make_map(&tb, planes, K, 2 * g_pad, S, K * EB, plane_bytes, pick_bn(S, Le), err, TFP))
      return RPA_ECUDA;
    GemmArgs a{};
    a.S = S;
    a.nexact = Le;
    a.K = (int)K;
    a.ea = exps;
    a.eb = exps;
    a.eb_stride = 0;
    a.a_rows = n_g;
    a.b_rows = 2 * n_g;
    a.alpha = scale;
    a.rsa = sv;  // chi~ = v^1/2 chi0 v^1/2: the v^1/2 factors scale rows and columns
    a.rsb = sv;
    a.out = (double2*)chi;
    a.out_bstride = 0;
    a.ld_row = n_g;
    a.ld_col = 1;
    a.conj = 0;
    a.accumulate = 1;
    const int tiles_m = cdiv(n_g, BM);
    w.hook(RPA_T_CHI0, 1);
    rpa_status r = run_gemm(w, ta, tb, a, tiles_m, 1, true, chi, 0, st, err, launches);
    w.hook(RPA_T_CHI0, 0);
    if (r != RPA_OK) return r;
    CK(cudaEventRecord(w.ev_gemm[buf], st));
  }
  return RPA_OK;
}

// rows of A -> S digit planes of the projection's A operand and exponents ea
// Rows of A per projection chunk: all of them when their digit planes fit in the
// plane budget, else a multiple of the tile height (the planes of one chunk at a time).
static long proj_chunk_rows(const Workspace& w, int n_vc) {
  return std::min<long>(rup(n_vc, BM), w.proj_chunk);
}

// A byte offset of `rows` rows of A (n_g complex elements each, complex128 or complex64).
static const void* a_rows_at(const void* A, int dtype, long row, int n_g) {
  return (const char*)A + row * n_g * (dtype == RPA_C64 ? 8 : 16);
}

// rows [r0, r0 + nr) of A -> S digit planes of the projection's A operand and exponents ea
template <typename P>
static rpa_status slice_proj_a(Workspace& w, const void* A, int dtype, long r0, int nr, int n_g,
                               cudaStream_t s, std::string& err, int* launches) {
  const int S = w.proj_slices_override > 0 ? w.proj_slices_override : w.slices.proj;
  const long rpad = rup(nr, BM), K = rup(2L * n_g, BK);
  const void* a0 = a_rows_at(A, dtype, r0, n_g);
  CK(cudaMemsetAsync(w.rowmax, 0, rpad * sizeof(unsigned long long), s));
  row_max_kernel<<<dim3((unsigned)nr, cdiv(n_g, CHUNK)), 256, 0, s>>>(a0, dtype, n_g, nr, n_g,
                                                                      w.rowmax);
  CK(cudaGetLastError());
  slice_rows_kernel<P><<<dim3((unsigned)rpad, cdiv(K / 2, CHUNK)), 256, 0, s>>>(
      a0, dtype, n_g, nr, n_g, (int)rpad, K, S, w.rowmax, (P*)w.planes, w.exps,
      w.split);
  CK(cudaGetLastError());
  if (launches) *launches += 2;
  return RPA_OK;
}

template <typename P>
rpa_status project_prepare_t(Workspace& w, const void* A, int dtype, int n_vc, int n_g,
                           cudaStream_t st, std::string& err, int* launches) {
  w.proj_a.valid = false;
  if (side_fork(w, st, err) != RPA_OK) return RPA_ECUDA;
  const int nr = (int)std::min<long>(n_vc, proj_chunk_rows(w, n_vc));  // the first chunk
  rpa_status r = slice_proj_a<P>(w, A, dtype, 0, nr, n_g, w.side, err, launches);
  if (r != RPA_OK) return r;
  CK(cudaEventRecord(w.ev_side_last, w.side));
  w.proj_a.valid = true;
  w.proj_a.a = A;
  w.proj_a.dtype = dtype;
  w.proj_a.n_vc = n_vc;
  w.proj_a.n_g = n_g;
  w.proj_a.S = w.slices.proj;
  return RPA_OK;
}

template <typename P>
rpa_status project_t(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const cplx* B,
                   int n_eig, cplx* mt, cudaStream_t st, std::string& err, int* launches,
                   long ld_out) {
  constexpr int EB = (int)sizeof(P) / 2;  // bytes of one plane element
  constexpr bool TFP = sizeof(P) == 8;
  if (ld_out <= 0) ld_out = n_vc;
  const int S = w.proj_slices_override > 0 ? w.proj_slices_override : w.slices.proj;
  const long e_pad = rup(n_eig, BM), K = rup(2L * n_g, BK);
  // rows of A cut at a time: the budgeted chunk, and no more than the plane buffer
  // holds at this slice count
  const long fit = (long)(w.plane_bytes / ((size_t)S * K * EB)) / BM * BM;
  const long chunk = std::min(proj_chunk_rows(w, n_vc), fit);
  if (chunk < BM || (size_t)S * 2 * e_pad * K * EB > w.plane2_bytes) {
    err = "projection: operand planes exceed the workspace";
    return RPA_EINVAL;
  }
  const bool chunked = chunk < n_vc;
  P* pb = (P*)w.planes2;
  int* ea = w.exps;
  int* eb = w.exps + std::max({rup(n_g, BM), rup(std::min<long>(chunk, n_vc), BM), e_pad});
  const bool ready = w.proj_a.valid && w.proj_a.a == A && w.proj_a.dtype == dtype &&
                     w.proj_a.n_vc == n_vc && w.proj_a.n_g == n_g && w.proj_a.S == S;
  w.proj_a.valid = false;  // the chi_s stage reuses the planes next
  w.hook(RPA_T_SLICE, 1);
  if (join_side(w, st, err) != RPA_OK) return RPA_ECUDA;
  proj_b_slice_kernel<P><<<(unsigned)e_pad, 256, 0, st>>>((const double2*)B, n_g, n_eig, (int)e_pad,
                                                       K, S, pb, eb, w.split);
  CK(cudaGetLastError());
  if (launches) *launches += 1;
  // chunks of the output's columns, and a strided output (ld_out != n_vc, whose
  // split-K tiles must not zero a contiguous range), are added with FP64 atomics
  // into a zeroed M~
  const bool strided = ld_out != n_vc;
  if (chunked || strided)
    CK(cudaMemset2DAsync(mt, sizeof(cplx) * (size_t)ld_out, 0, sizeof(cplx) * (size_t)n_vc,
                         (size_t)n_eig, st));
  w.hook(RPA_T_SLICE, 0);
  const int Le = w.split ? 1 : exact_levels_proj(S);
  CUtensorMap tb;
  if (!make_map(&tb, w.planes2, K, 2 * e_pad, S, K * EB, 2 * e_pad * K * EB, pick_bn(S, Le), err,
                TFP))
    return RPA_ECUDA;
  for (long r0 = 0; r0 < n_vc; r0 += chunk) {
    const int nr = (int)std::min<long>(chunk, n_vc - r0);
    const long rpad = rup(nr, BM);
    if (r0 > 0 || !ready) {
      w.hook(RPA_T_SLICE, 1);
      rpa_status r = slice_proj_a<P>(w, A, dtype, r0, nr, n_g, st, err, launches);
      w.hook(RPA_T_SLICE, 0);
      if (r != RPA_OK) return r;
    }
    CUtensorMap ta;
    if (!make_map(&ta, w.planes, K, rpad, S, K * EB, rpad * K * EB, BM, err, TFP)) return RPA_ECUDA;
    GemmArgs a{};
    a.S = S;
    a.nexact = Le;
    a.K = (int)K;
    a.ea = ea;
    a.eb = eb;
    a.eb_stride = 0;
    a.a_rows = nr;
    a.b_rows = 2 * n_eig;
    a.alpha = 1.0;
    a.out = (double2*)(mt + r0);
    a.out_bstride = 0;
    a.ld_row = 1;
    a.ld_col = ld_out;
    a.conj = 1;
    a.atomic = 0;
    a.accumulate = (chunked || strided) ? 1 : 0;
    w.hook(RPA_T_PROJ, 1);
    rpa_status r = run_gemm(w, ta, tb, a, cdiv(nr, BM), 1, false, mt,
                            sizeof(cplx) * (size_t)n_eig * n_vc, st, err, launches);
    w.hook(RPA_T_PROJ, 0);
    if (r != RPA_OK) return r;
  }
  return RPA_OK;
}

template <typename P>
rpa_status chis_t(Workspace& w, const cplx* mt, int n_eig, int n_vc, const double* f,
                int n_freq, double scale, cplx* out, cudaStream_t st, std::string& err,
                int* launches) {
  constexpr int EB = (int)sizeof(P) / 2;  // bytes of one plane element
  constexpr bool TFP = sizeof(P) == 8;
  const int S = w.slices.chis, Le = w.split ? 1 : exact_levels_chis(S);
  const long e_pad = rup(n_eig, BM), K = rup(2L * n_vc, BK);
  const int grp = w.freq_group;
  P* pa = (P*)w.planes2;
  int* ea = w.exps;
  w.proj_a.valid = false;
  w.hook(RPA_T_SLICE, 1);
  if (join_side(w, st, err) != RPA_OK) return RPA_ECUDA;
  float_up_kernel<<<std::min(cdiv((long)n_freq * n_vc, 256), 4096), 256, 0, st>>>(
      f, (long)n_freq * n_vc, w.fweights);
  CK(cudaGetLastError());
  // the first frequency group's B planes are cut on the side stream while the A planes
  // of M~ are cut here
  if (side_fork(w, st, err) != RPA_OK) return RPA_ECUDA;
  CK(cudaMemsetAsync(w.rowmax, 0, e_pad * sizeof(unsigned long long), st));
  row_max_kernel<<<dim3((unsigned)n_eig, cdiv(n_vc, CHUNK)), 256, 0, st>>>(mt, RPA_C128, n_vc,
                                                                            n_eig, n_vc, w.rowmax);
  CK(cudaGetLastError());
  slice_rows_kernel<P><<<dim3((unsigned)e_pad, cdiv(K / 2, CHUNK)), 256, 0, st>>>(
      mt, RPA_C128, n_vc, n_eig, n_vc, (int)e_pad, K, S, w.rowmax, pa, ea, w.split);
  CK(cudaGetLastError());
  if (launches) *launches += 3;
  w.hook(RPA_T_SLICE, 0);
  CUtensorMap ta;
  if (!make_map(&ta, w.planes2, K, e_pad, S, K * EB, e_pad * K * EB, BM, err, TFP)) return RPA_ECUDA;
  const int tiles_m = cdiv(n_eig, BM);
  // B planes of frequency groups in two alternating buffers: group g + 1 is cut
  // on the side stream while group g is multiplied on `st`.
  const size_t buf_pairs = (size_t)grp * S * 2 * e_pad * (K / 2);  // BF16 pairs per buffer
  cudaStream_t cut = w.chis_overlap ? w.side : st;
  int g = 0;
  for (int k0 = 0; k0 < n_freq; k0 += grp, ++g) {
    const int nb = std::min(grp, n_freq - k0), buf = g & 1;
    P* pb = (P*)w.planes + buf * buf_pairs;
    int* eb = w.exps + e_pad + (size_t)buf * grp * e_pad;
    unsigned long long* rowmax = w.rowmax + e_pad + (size_t)buf * grp * e_pad;
    if (g >= 2) CK(cudaStreamWaitEvent(cut, w.ev_gemm[buf], 0));
    if (cut == st) w.hook(RPA_T_SLICE, 1);
    CK(cudaMemsetAsync(rowmax, 0, (size_t)nb * e_pad * sizeof(unsigned long long), cut));
    chis_b_rowmax_kernel<<<dim3((unsigned)cdiv(n_eig, RMR), cdiv(n_vc, CHUNK)), 256, 0, cut>>>(
        (const double2*)mt, n_eig, n_vc, w.fweights + (size_t)k0 * n_vc, f + (size_t)k0 * n_vc,
        nb, rowmax, (int)e_pad);
    CK(cudaGetLastError());
    chis_b_slice_kernel<P><<<dim3((unsigned)cdiv(e_pad, RMR), cdiv(K / 2, CHUNK)), 256, 0, cut>>>(
        (const double2*)mt, n_eig, (int)e_pad, n_vc, K, f + (size_t)k0 * n_vc, nb, S, rowmax, pb,
        eb, (int)e_pad, w.split);
    CK(cudaGetLastError());
    CK(cudaEventRecord(w.ev_sliced[buf], cut));
    CK(cudaEventRecord(w.ev_side_last, cut));
    if (launches) *launches += 2;
    if (cut != st) w.hook(RPA_T_SLICE, 1);
    CK(cudaStreamWaitEvent(st, w.ev_sliced[buf], 0));
    w.hook(RPA_T_SLICE, 0);
    CUtensorMap tb;
    if (!make_map(&tb, pb, K, 2 * e_pad, (long)nb * S, K * EB, 2 * e_pad * K * EB, pick_bn(S, Le),
                  err, TFP))
      return RPA_ECUDA;
    GemmArgs a{};
    a.S = S;
    a.nexact = Le;
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
    rpa_status r = run_gemm(w, ta, tb, a, tiles_m, nb, true, a.out,
                            sizeof(cplx) * (size_t)nb * n_eig * n_eig, st, err, launches);
    w.hook(RPA_T_CHIS, 0);
    if (r != RPA_OK) return r;
    CK(cudaEventRecord(w.ev_gemm[buf], st));
  }
  return RPA_OK;
}


rpa_status chi0(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const double* sf,
                const int* order, const double* sv, double scale, cplx* chi, cudaStream_t st,
                std::string& err, int* launches, bool zero, int blocks) {
  return w.tf32 ? chi0_t<float2>(w, A, dtype, n_vc, n_g, sf, order, sv, scale, chi, st, err,
                                 launches, zero, blocks)
                : chi0_t<__nv_bfloat162>(w, A, dtype, n_vc, n_g, sf, order, sv, scale, chi, st,
                                         err, launches, zero, blocks);
}

rpa_status project_prepare(Workspace& w, const void* A, int dtype, int n_vc, int n_g,
                           cudaStream_t st, std::string& err, int* launches) {
  return w.tf32 ? project_prepare_t<float2>(w, A, dtype, n_vc, n_g, st, err, launches)
                : project_prepare_t<__nv_bfloat162>(w, A, dtype, n_vc, n_g, st, err, launches);
}

rpa_status project(Workspace& w, const void* A, int dtype, int n_vc, int n_g, const cplx* B,
                   int n_eig, cplx* mt, cudaStream_t st, std::string& err, int* launches,
                   long ld_out) {
  return w.tf32 ? project_t<float2>(w, A, dtype, n_vc, n_g, B, n_eig, mt, st, err, launches,
                                    ld_out)
                : project_t<__nv_bfloat162>(w, A, dtype, n_vc, n_g, B, n_eig, mt, st, err,
                                            launches, ld_out);
}

rpa_status chis(Workspace& w, const cplx* mt, int n_eig, int n_vc, const double* f,
                int n_freq, double scale, cplx* out, cudaStream_t st, std::string& err,
                int* launches) {
  return w.tf32 ? chis_t<float2>(w, mt, n_eig, n_vc, f, n_freq, scale, out, st, err, launches)
                : chis_t<__nv_bfloat162>(w, mt, n_eig, n_vc, f, n_freq, scale, out, st, err,
                                         launches);
}

}  // namespace tc
}  // namespace rpa
