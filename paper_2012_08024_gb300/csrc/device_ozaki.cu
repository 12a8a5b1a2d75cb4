// FP64 level-0 apply of the many-right-hand-side CG, Y = A_0 X for R columns,
// on the tcgen05 tensor cores by exact splitting (Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", 2012).
//
// Every row (K, i) of A_0 is scaled by a power of two 2^{E_A(K,i)} above its
// largest entry and every column r of X by 2^{E_X(r)}; the scaled values, in
// (-1, 1), are cut into S = 8 signed 7-bit integer slices,
//   a = 2^{E_A} sum_s a_s 2^{-7(s+1)},   x = 2^{E_X} sum_t x_t 2^{-7(t+1)},
// each exact in BF16.  A BF16 x BF16 product is exact in FP32, and so is a sum
// of them while it stays an integer below 2^24 (checked on the host, with one
// bit of headroom: blocks per row x n_p x S x 127^2 < 2^23).  The slice products of one diagonal d = s + t share the
// scale 2^{-7(d+2)}, so they go to one FP32 accumulator: the MMA of slice t of
// X against the stacked slices [A_0; ...; A_{S-1-t}] (N = 16 (S - t) rows)
// writes at TMEM column 16 t, i.e. onto the accumulators d = t .. S-1.  The
// pairs s + t >= S are left out (relative truncation below 2^-56 of the row
// and column scales).  The epilogue converts the eight integer-valued
// accumulators to integers, combines them exactly in 64-bit integers and
// rounds once to FP64.
//
// Layout: the slices of one block are stored as the 4 KB shared-memory image
// of the MMA B operand (128 rows s * 16 + i, K = 16 columns j, canonical
// K-major SWIZZLE_NONE core matrices: 8 rows x 16 bytes, LBO = 128 bytes
// along K, SBO = 256 bytes between 8-row groups); X is sliced once per apply
// into the same images, 4 KB per (element, column tile, slice), and staged per
// block as S operands A = X_J^T (128 columns x 16).  A CTA owns a tile of 128
// columns: one thread copies the operands of each block into a ring of three
// shared-memory stages with bulk copies and issues its MMAs, so the copies of
// the next blocks overlap the MMAs of the current one, and four epilogue warps
// read finished rows from one of two TMEM accumulator sets while the MMAs of
// the next row fill the other.  Every wait has an iteration limit; on expiry
// the kernel sets the error flag, drains its copies and MMAs (default limit),
// frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "device_state.h"
#include "host_setup.h"

namespace {

constexpr int kS = 8;                         // slices per operand
constexpr int kTile = 128;                    // columns per tile (MMA M, TMEM lanes)
constexpr int kBRows = 16 * kS;               // B operand rows: slice s, row i
constexpr uint32_t kLBO = 128, kSBO = 256;    // bytes (BF16, K = 16)
constexpr int kXBytes = kTile * 16 * 2;       // one X slice operand: 4 KB
constexpr int kABytes = kBRows * 16 * 2;      // all A slices of one block: 4 KB
constexpr int kStageBytes = kS * kXBytes + kABytes;
constexpr int kStages = 3;
constexpr int kWaitLimit = 1 << 22;
constexpr int kAccSets = 2;                   // accumulator sets: rows in flight between MMAs and epilogue
constexpr int kTmemCols = 16 * kS * kAccSets;  // per set, accumulators d = 0 .. S-1, 16 columns each
constexpr int kEpiThreads = kTile;            // epilogue warps 0-3: one column of the tile per thread
constexpr int kOzThreads = kEpiThreads + 32;    // and warp 4, whose lane 0 copies and issues the MMAs

__host__ __device__ __forceinline__ int kmaj16(int row, int k) {
  return (row >> 3) * (int)kSBO + (k >> 3) * (int)kLBO + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(kLBO >> 4) << 16;
  d |= (uint64_t)(kSBO >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the tcgen05 family; base offset 0, no swizzle
  return d;
}

// instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, N rows of B, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTile >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
  return done != 0;
}

// BF16 bits of a signed integer |k| <= 127 (exact): 2^23 + k as FP32 bits minus 2^23
__device__ __forceinline__ uint32_t bf16_small(uint32_t mag, bool neg) {
  const float f = __uint_as_float(0x4B000000u | mag) - 8388608.0f;
  return ((__float_as_uint(f) >> 16) & 0x7FFFu) | (neg ? 0x8000u : 0u);
}

// 2^k * v for an integer |v| < 2^53, built from its bits (exact); ldexp outside the normal range
__device__ __forceinline__ double i64_scaled(long long v, int k) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int e = 63 - __clzll((long long)a);
  const int be = e + 1023 + k;
  if (be <= 0 || be >= 2047) return ldexp((double)v, k);
  const unsigned long long mant = (a << (52 - e)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | mant));
}

// per column r: the largest biased FP64 exponent of x[.][r] (0 for a zero column)
__global__ void oz_colexp_kernel(size_t nrows, int R, const double* __restrict__ x, int* __restrict__ maxb) {
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const size_t lo = nrows * blockIdx.x / gridDim.x, hi = nrows * (blockIdx.x + 1) / gridDim.x;
  int m = 0;
  for (size_t row = lo; row < hi; ++row) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x[row * R + r]);
    m = max(m, (int)((b >> 52) & 0x7FF));
  }
  atomicMax(maxb + r, m);
}

// Slices of x as MMA operand images: for element J, column tile c and slice t,
// the 4 KB image of X_J^T (rows = the tile's 128 columns, K = 16 coefficients
// j, zero beyond n_p and beyond R) at xs + ((J * tiles + c) * S + t) * 4 KB.
// One thread per (J, column); the column is scaled by 2^{-(maxb - 1022)}.
template <int NP>
__global__ void oz_slice_kernel(int n, int R, int tiles, const double* __restrict__ x,
                                const int* __restrict__ maxb, unsigned char* __restrict__ xs) {
  const size_t tot = (size_t)n * tiles * kTile;
  for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < tot; u += (size_t)gridDim.x * blockDim.x) {
    const size_t J = u / ((size_t)tiles * kTile);
    const int rr = (int)(u - J * tiles * kTile);
    const int c = rr / kTile, row = rr - c * kTile;
    const int r = rr;
    uint32_t w[kS][8];
#pragma unroll
    for (int t = 0; t < kS; ++t)
#pragma unroll
      for (int q = 0; q < 8; ++q) w[t][q] = 0u;
    if (r < R) {
      const int mb = maxb[r];
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(x[(J * NP + j) * (size_t)R + r]);
        const bool neg = (bits >> 63) != 0;
        const int b = (int)((bits >> 52) & 0x7FF);
        unsigned long long F = 0;   // |x| 2^{56 - E_X}, truncated: < 2^56
        if (b != 0) {
          const unsigned long long M = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
          const int sh = b - mb + 3;   // <= 3
          if (sh >= 0) F = M << sh;
          else if (sh > -64) F = M >> (-sh);
        }
#pragma unroll
        for (int t = 0; t < kS; ++t)
          w[t][j >> 1] |= bf16_small((uint32_t)((F >> (49 - 7 * t)) & 127u), neg) << ((j & 1) * 16);
      }
    }
    unsigned char* img = xs + ((J * tiles + c) * kS) * (size_t)kXBytes;
#pragma unroll
    for (int t = 0; t < kS; ++t) {
      unsigned char* dst = img + t * kXBytes;
      *reinterpret_cast<uint4*>(dst + kmaj16(row, 0)) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
      *reinterpret_cast<uint4*>(dst + kmaj16(row, 8)) = make_uint4(w[t][4], w[t][5], w[t][6], w[t][7]);
    }
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void arrive_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// A bounded wait that also gives up once another role of the CTA has failed
__device__ __forceinline__ bool wait_or_fail(uint32_t mbar, uint32_t parity, int limit, const volatile int* fail) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (!done && *fail) return false;
  }
  return done != 0;
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// CTA (x, c) owns the block rows K = x, x + gridDim.x, ... and column tile c
// (strided, so that the CTAs working at the same time cover neighbouring rows
// and share the X images of their neighbours in L2; contiguous row ranges per
// CTA measured a 25% instead of 46% L2 hit rate and 1.8x the DRAM reads),
// with two roles that run concurrently:
//  - lane 0 of warp 4 streams the blocks of those rows through a ring of
//    kStages shared-memory stages (a stage is free once the MMAs that read it
//    completed: empty[]; its bulk copies complete full[]) and issues each
//    block's S MMAs into accumulator set a = (row index) mod 2 of TMEM, then
//    commits the row to accf[a].  Before the first MMA of a row it waits on
//    acce[a], until the epilogue has read that set's previous row.
//  - warps 0-3 (lane = column of the tile) wait on accf[a], read the row's S
//    accumulators, release the set (acce[a], one arrive per warp), combine
//    them exactly and write y.  With pq_partial they also sum x . y over the
//    CTA's rows, in row order, into pq_partial[blockIdx.x][column] (the CG's
//    p . A p, without a separate pass over both vectors).
// So the MMAs of row k + 1 run while the epilogue of row k converts and
// stores.  Every wait is bounded; a role that gives up sets the shared fail
// flag, on which the other role's waits give up too.  Before the CTA ends the
// issuing thread waits (default limit) for its copies in flight and for all of
// its MMAs (a final commit), and warp 0 frees the tensor memory.
template <int NP>
__global__ void __launch_bounds__(kOzThreads, 2) oz_apply_kernel(int n, int R, int tiles,
                                                               const int* __restrict__ rowptr,
                                                               const int* __restrict__ col,
                                                               const unsigned char* __restrict__ Aimg,
                                                               const int* __restrict__ eA,
                                                               const unsigned char* __restrict__ xs,
                                                               const int* __restrict__ maxb, double* __restrict__ y,
                                                               const double* __restrict__ xdot,
                                                               double* __restrict__ pq_partial, int* __restrict__ err,
                                                               int wait_limit) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf[kAccSets], acce[kAccSets], fin;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c = blockIdx.y;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
    }
    for (int a = 0; a < kAccSets; ++a) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf[a])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&acce[a])), "n"(kEpiThreads / 32));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&fin)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    fail_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "n"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  if (warp == kEpiThreads / 32) {
    if (lane == 0) {
      // ---- copies and MMAs
      int pk = blockIdx.x, pb = pk < n ? rowptr[pk] : 0;   // the next block to copy, as (row, block)
      long long issued = 0, consumed = 0;                 // blocks copied / blocks whose MMAs are issued
      bool ok = true;
      auto advance = [&]() {
        while (pk < n && pb >= rowptr[pk + 1]) {
          pk += gridDim.x;
          pb = pk < n ? rowptr[pk] : 0;
        }
      };
      auto issue = [&]() -> bool {   // copies of the block at the cursor into stage issued % kStages
        advance();
        if (pk >= n) return true;
        const int st = (int)(issued % kStages);
        if (issued >= kStages &&
            !wait_or_fail(smem_u32(&empty[st]), (uint32_t)(((issued / kStages) - 1) & 1), wait_limit, &fail_s))
          return false;
        unsigned char* sx = smem + st * kStageBytes;
        const uint32_t fb = smem_u32(&full[st]);
        arrive_expect(fb, (uint32_t)kStageBytes);
        bulk_g2s(sx, xs + ((size_t)col[pb] * tiles + c) * kS * (size_t)kXBytes, (uint32_t)(kS * kXBytes), fb);
        bulk_g2s(sx + kS * kXBytes, Aimg + (size_t)pb * kABytes, (uint32_t)kABytes, fb);
        ++issued;
        ++pb;
        return true;
      };
      int rowi = 0;   // rows of this CTA with blocks, so far
      for (int K = blockIdx.x; K < n && ok; K += gridDim.x) {
        const int b0 = rowptr[K], b1 = rowptr[K + 1];
        if (b1 == b0) continue;
        const int a = rowi % kAccSets;
        if (rowi >= kAccSets &&
            !wait_or_fail(smem_u32(&acce[a]), (uint32_t)(((rowi / kAccSets) - 1) & 1), wait_limit, &fail_s)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t dacc = tmem + (uint32_t)(a * 16 * kS);
        for (int bb = b0; bb < b1 && ok; ++bb) {
          while (ok && issued < consumed + kStages) {
            const long long before = issued;
            ok = issue();
            if (issued == before) break;   // no block left to copy
          }
          if (!ok) break;
          const int st = (int)(consumed % kStages);
          if (!wait_or_fail(smem_u32(&full[st]), (uint32_t)((consumed / kStages) & 1), wait_limit, &fail_s)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;");
          unsigned char* sx = smem + st * kStageBytes;
          const uint64_t bdesc = smem_desc(smem_u32(sx + kS * kXBytes));
#pragma unroll
          for (int t = 0; t < kS; ++t)
            mma_bf16(dacc + (uint32_t)(16 * t), smem_desc(smem_u32(sx + t * kXBytes)), bdesc,
                     idesc_bf16(16 * (kS - t)), (bb > b0 || t > 0) ? 1u : 0u);
          mma_commit(smem_u32(&empty[st]));
          ++consumed;
        }
        if (!ok) break;
        mma_commit(smem_u32(&accf[a]));
        ++rowi;
      }
      if (!ok) {
        fail_s = 1;
        atomicExch(err, 1);
      }
      // copies in flight land and issued MMAs finish before the CTA ends: every
      // unconsumed stage phase in order (at most one per stage), then one commit
      // that completes after all earlier MMAs of this thread
      for (long long u = consumed; u < issued; ++u)
        wait_phase(smem_u32(&full[u % kStages]), (uint32_t)((u / kStages) & 1), kWaitLimit);
      mma_commit(smem_u32(&fin));
      wait_phase(smem_u32(&fin), 0u, kWaitLimit);
    }
  } else {
    // ---- epilogue: y[K][i][r] = 2^{E_A + E_X - 63} sum_d acc_d 2^{7 (S - 1 - d)}
    const int r = c * kTile + tid;   // this thread's column
    const int ex = r < R ? maxb[r] - 1022 : 0;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    const bool dot = pq_partial != nullptr && r < R;
    double dsum = 0.0;   // with pq_partial: sum over this CTA's rows of x . y for column r
    int rowi = 0;
    for (int K = blockIdx.x; K < n; K += gridDim.x) {
      const int b0 = rowptr[K], b1 = rowptr[K + 1];
      if (b1 == b0) {
        if (r < R)
          for (int i = 0; i < NP; ++i) y[((size_t)K * NP + i) * R + r] = 0.0;
        continue;
      }
      const int a = rowi % kAccSets;
      int kexp[NP];   // the row's scale exponents (and x, for the dot), loaded before the wait
      double xd[NP];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        kexp[i] = eA[(size_t)K * 16 + i] + ex - 63;
        xd[i] = dot ? xdot[((size_t)K * NP + i) * R + r] : 0.0;
      }
      const bool got = wait_or_fail(smem_u32(&accf[a]), (uint32_t)((rowi / kAccSets) & 1), wait_limit, &fail_s);
      if (!__all_sync(0xffffffffu, got ? 1 : 0)) {   // the warp leaves together (tcgen05.ld is warp-wide)
        if (lane == 0) {
          fail_s = 1;
          atomicExch(err, 1);
        }
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t taddr = tmem + lanes + (uint32_t)(a * 16 * kS);
      long long vh[NP], vl[NP];
#pragma unroll
      for (int h = 0; h < (NP + 7) / 8; ++h) {
        uint32_t v[kS][8];
#pragma unroll
        for (int d = 0; d < kS; ++d)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(v[d][0]), "=r"(v[d][1]), "=r"(v[d][2]), "=r"(v[d][3]), "=r"(v[d][4]), "=r"(v[d][5]),
                         "=r"(v[d][6]), "=r"(v[d][7])
                       : "r"(taddr + (uint32_t)(16 * d + 8 * h)));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = 8 * h + q;
          if (i >= NP) break;
          int s[kS];
#pragma unroll
          for (int d = 0; d < kS; ++d) s[d] = __float2int_rz(__uint_as_float(v[d][q]));
          const int p0 = s[0] * 128 + s[1], p1 = s[2] * 128 + s[3];
          const int p2 = s[4] * 128 + s[5], p3 = s[6] * 128 + s[7];
          vh[i] = (long long)p0 * 16384 + p1;
          vl[i] = (long long)p2 * 16384 + p3;
        }
      }
      // the set is read: the issuing thread may start the row after next in it
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[a])) : "memory");
      if (r < R) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
          const double v = i64_scaled(vh[i], kexp[i] + 28) + i64_scaled(vl[i], kexp[i]);
          y[((size_t)K * NP + i) * R + r] = v;
          if (dot) dsum = fma(xd[i], v, dsum);
        }
      }
      ++rowi;
    }
    if (dot) pq_partial[(size_t)blockIdx.x * R + r] = dsum;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols));
}

// S signed 7-bit slices of a, scaled by 2^{-E} (|a| < 2^E): a = 2^E sum_s out[s] 2^{-7(s+1)} + rest
void host_slices(double a, int E, int out[kS]) {
  const double v = std::ldexp(std::fabs(a), 56 - E);   // < 2^56, exact
  const uint64_t F = (uint64_t)v;                      // floor
  const int sg = a < 0 ? -1 : 1;
  for (int s = 0; s < kS; ++s) out[s] = sg * (int)((F >> (49 - 7 * s)) & 127u);
}

uint16_t host_bf16_int(int k) {
  const float f = (float)k;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

}  // namespace

size_t oz_image_bytes(const cdg::BSR& A) { return (size_t)A.nnzb() * kABytes; }
size_t oz_xslice_bytes(int64_t n, int np, int R) {
  (void)np;
  return (size_t)n * ((R + kTile - 1) / kTile) * kS * kXBytes;
}

// The split is exact when every FP32 accumulator stays an integer below 2^23
// (below 2^24 for exact FP32 sums, one bit more of headroom for the int32
// combination of the epilogue): blocks per row x n_p x S pairs x 127^2 < 2^23.
bool oz_feasible(const cdg::BSR& A, int np) {
  if (np > 16) return false;
  int64_t maxblk = 0;
  for (int64_t K = 0; K < A.nrows; ++K) maxblk = std::max<int64_t>(maxblk, A.rowptr[K + 1] - A.rowptr[K]);
  return (double)maxblk * np * kS * 127.0 * 127.0 < 8388608.0;
}

// Host preparation of the slices of A_0: the B operand image of every block and
// the row exponents eA[K * 16 + i].  False when the split would not be exact.
bool oz_prepare(const cdg::BSR& A, int np, std::vector<uint16_t>& img, std::vector<int32_t>& eA) {
  if (!oz_feasible(A, np)) return false;
  const int64_t n = A.nrows;
  img.assign((size_t)A.nnzb() * (kABytes / 2), 0);
  eA.assign((size_t)n * 16, 0);
  for (int64_t K = 0; K < n; ++K) {
    for (int i = 0; i < np; ++i) {
      double m = 0.0;
      for (int64_t b = A.rowptr[K]; b < A.rowptr[K + 1]; ++b)
        for (int j = 0; j < np; ++j) m = std::max(m, std::fabs(A.block(b)[i * np + j]));
      int e = 0;
      if (m > 0.0) std::frexp(m, &e);   // m < 2^e
      eA[(size_t)K * 16 + i] = e;
    }
    for (int64_t b = A.rowptr[K]; b < A.rowptr[K + 1]; ++b) {
      uint16_t* o = img.data() + (size_t)b * (kABytes / 2);
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < np; ++j) {
          int sl[kS];
          host_slices(A.block(b)[i * np + j], eA[(size_t)K * 16 + i], sl);
          for (int s = 0; s < kS; ++s) o[kmaj16(s * 16 + i, j) / 2] = host_bf16_int(sl[s]);
        }
    }
  }
  return true;
}

// y = A_0 x for R columns ([n][np][R] FP64 vectors): column exponents, slices of x, tensor-core products.
bool oz_apply(int np, int n, int R, const int* rowptr, const int* col, const void* img, const int* eA, void* xs,
              int* maxb, bool maxb_ready, const double* x, double* y, double* pq_partial, int* pq_groups, int* err,
              int wait_limit, cudaStream_t s) {
  const size_t nrows = (size_t)n * np;
  if (!maxb_ready) {
    cudaMemsetAsync(maxb, 0, sizeof(int) * R, s);
    const unsigned ty = (unsigned)((R + 255) / 256);
    oz_colexp_kernel<<<dim3(2 * 152, ty), 256, 0, s>>>(nrows, R, x, maxb);
    count_launch();
  }
  const int tiles = (R + kTile - 1) / kTile;
  const int lim = wait_limit < 0 ? kWaitLimit : std::min(wait_limit, kWaitLimit);
  // two CTAs per SM (108 KB of shared memory, 256 TMEM columns each): the whole grid is resident
  const dim3 grid((unsigned)std::max(1, std::min(n, 152 * 2 / tiles)), (unsigned)tiles);
  const int smem = kStages * kStageBytes;
  auto go = [&](auto slice, auto kern) {
    slice<<<4 * 152 * 4, 256, 0, s>>>(n, R, tiles, x, maxb, (unsigned char*)xs);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    kern<<<grid, kOzThreads, smem, s>>>(n, R, tiles, rowptr, col, (const unsigned char*)img, eA,
                                        (const unsigned char*)xs, maxb, y, x, pq_partial, err, lim);
  };
  switch (np) {
    case 3: go(oz_slice_kernel<3>, oz_apply_kernel<3>); break;
    case 4: go(oz_slice_kernel<4>, oz_apply_kernel<4>); break;
    case 6: go(oz_slice_kernel<6>, oz_apply_kernel<6>); break;
    case 10: go(oz_slice_kernel<10>, oz_apply_kernel<10>); break;
    default: return false;
  }
  count_launch(2);
  if (pq_groups) *pq_groups = (int)grid.x;
  return true;
}
