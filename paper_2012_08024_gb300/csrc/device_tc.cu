// Block-Jacobi smoother sweep of the many-right-hand-side V-cycle on the 5th
// generation tensor cores (tcgen05): y = x + omega (bh - x - Ahat x) for R
// columns, Ahat the BF16 row-scaled off-diagonal blocks (precision mode 2).
//
// A CTA of 128 threads owns a tile of 128 columns and walks block rows K.  For
// every block (K, J) of Ahat the contraction Y_K^T += X_J^T Ahat_KJ^T is one
// 128 x 16 x 16 MMA (n_p padded to 16): the A operand is X_J^T (128 columns x
// n_p coefficients, staged K-major in shared memory), the B operand the block
// (n_p rows x n_p coefficients, K-major as stored), the accumulator 128 TMEM
// lanes x 16 FP32 columns.  kind::tf32 reads FP32 operands with 10-bit
// significands; a BF16 block is exact there, and x is split into a TF32 part
// and its remainder, two MMAs per K step, so the product keeps FP32 accuracy.
//
// Shared-memory operands use the canonical SWIZZLE_NONE K-major layout: core
// matrices of 8 rows x 16 bytes (4 TF32), 128 bytes each; LBO = 128 bytes
// between neighbouring core matrices along K, SBO = 512 bytes between groups
// of 8 rows (4 core matrices cover the padded K = 16).  One thread issues the
// MMAs and commits them to an mbarrier; every wait has an iteration limit,
// after which the kernel sets the error flag, waits once more (bounded by the
// default limit) for its MMAs and frees its tensor memory.  The limit of the
// waits inside the loop is a kernel argument: a caller can lower it (0 makes
// the first wait give up at once) to exercise that path without a fault.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "device_state.h"

namespace {

constexpr int kTcRows = 128;          // columns per tile = MMA M = TMEM lanes
constexpr int kTcK = 16;              // padded n_p (MMA N and total K)
constexpr uint32_t kLBO = 128, kSBO = 512;
constexpr int kWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of (row, k) in a K-major FP32 operand
__device__ __forceinline__ int kmaj(int row, int k) {
  return (row >> 3) * kSBO + (k >> 2) * kLBO + (row & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(kLBO >> 4) << 16;
  d |= (uint64_t)(kSBO >> 4) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version of the tcgen05 family; base offset 0, no swizzle
  return d;
}

// instruction descriptor: FP32 accumulate, TF32 A and B, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcK >> 3) << 17) |
                            ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t parity, int limit = kWaitLimit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
  return done != 0;
}

__device__ __forceinline__ float tf32_round(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

template <int NP>
__global__ void __launch_bounds__(kTcRows) mr_tc_smooth_kernel(int n, int R, const int* __restrict__ rowptr,
                                                               const int* __restrict__ col,
                                                               const __nv_bfloat16* __restrict__ Ahat,
                                                               const float* __restrict__ x,
                                                               const float* __restrict__ bh, float* __restrict__ y,
                                                               float omega, int* __restrict__ err, int wait_limit) {
  __shared__ __align__(1024) unsigned char sXhi[kTcRows * kTcK * 4];
  __shared__ __align__(1024) unsigned char sXlo[kTcRows * kTcK * 4];
  __shared__ __align__(1024) unsigned char sB[kTcK * kTcK * 4];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int r = blockIdx.y * kTcRows + tid;   // this thread's right-hand side
  // padding (k >= NP, rows >= NP of the block) stays zero
  for (int e = tid; e < kTcRows * kTcK; e += kTcRows) {
    reinterpret_cast<float*>(sXhi)[e] = 0.f;
    reinterpret_cast<float*>(sXlo)[e] = 0.f;
  }
  for (int e = tid; e < kTcK * kTcK; e += kTcRows) reinterpret_cast<float*>(sB)[e] = 0.f;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t mb = smem_u32(&mbar);
  const uint32_t aHi = smem_u32(sXhi), aLo = smem_u32(sXlo), bB = smem_u32(sB);
  uint32_t parity = 0;
  bool ok = true;
  for (int K = blockIdx.x; K < n && ok; K += gridDim.x) {
    const int b0 = rowptr[K], b1 = rowptr[K + 1];
    for (int t = b0; t < b1 && ok; ++t) {
      const int J = col[t];
      if (r < R) {
        // this column's n_p coefficients of x_J, written one core-matrix row (4 values) at a time
        const float* xj = x + (size_t)J * NP * R + r;
        float hv[(NP + 3) / 4 * 4], lv[(NP + 3) / 4 * 4];
#pragma unroll
        for (int k = 0; k < (NP + 3) / 4 * 4; ++k) {
          const float v = k < NP ? xj[(size_t)k * R] : 0.f;
          hv[k] = tf32_round(v);
          lv[k] = v - hv[k];
        }
#pragma unroll
        for (int c = 0; c < (NP + 3) / 4; ++c) {
          *reinterpret_cast<float4*>(sXhi + kmaj(tid, 4 * c)) =
              make_float4(hv[4 * c], hv[4 * c + 1], hv[4 * c + 2], hv[4 * c + 3]);
          *reinterpret_cast<float4*>(sXlo + kmaj(tid, 4 * c)) =
              make_float4(lv[4 * c], lv[4 * c + 1], lv[4 * c + 2], lv[4 * c + 3]);
        }
      }
      const __nv_bfloat16* blk = Ahat + (size_t)t * NP * NP;
      for (int e = tid; e < NP * NP; e += kTcRows) {
        const int i = e / NP, k = e - i * NP;
        *reinterpret_cast<float*>(sB + kmaj(i, k)) = __bfloat162float(blk[e]);
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
#pragma unroll
        for (int ks = 0; ks < (NP + 7) / 8; ++ks) {   // K = 8 TF32 values = two core matrices per MMA
          const uint32_t off = (uint32_t)ks * 2 * kLBO;
          mma_tf32(tmem, smem_desc(aHi + off), smem_desc(bB + off), (t > b0 || ks > 0) ? 1u : 0u);
          mma_tf32(tmem, smem_desc(aLo + off), smem_desc(bB + off), 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
      }
      ok = __syncthreads_and(wait_phase(mb, parity, wait_limit) ? 1 : 0) != 0;   // the same decision in every thread
      parity ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!ok) break;
    float acc[kTcK];
    if (b1 > b0) {
      uint32_t v[kTcK];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int i = 0; i < kTcK; ++i) acc[i] = __uint_as_float(v[i]);
    } else {
#pragma unroll
      for (int i = 0; i < kTcK; ++i) acc[i] = 0.f;
    }
    if (r < R) {
      const size_t base = (size_t)K * NP * R + r;
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const size_t o = base + (size_t)i * R;
        const float xv = x[o];
        y[o] = xv + omega * (bh[o] - xv - acc[i]);
      }
    }
    // the next row's MMAs overwrite the accumulator: every lane has read it
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
    wait_phase(mb, parity ^ 1u);   // the commit of the last issued MMAs, if they are still running
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

}  // namespace

bool mr_tc_smooth(int np, int n, int R, const int* rowptr, const int* col, const void* Ahat_bf16, const float* x,
                  const float* bh, float* y, float omega, int* err, int wait_limit, cudaStream_t s) {
  const unsigned gy = (unsigned)((R + kTcRows - 1) / kTcRows);
  const unsigned gx = (unsigned)std::min(n, 152 * 8);
  const __nv_bfloat16* A = (const __nv_bfloat16*)Ahat_bf16;
  const int lim = wait_limit < 0 ? kWaitLimit : std::min(wait_limit, kWaitLimit);
  switch (np) {
    case 3: mr_tc_smooth_kernel<3><<<dim3(gx, gy), kTcRows, 0, s>>>(n, R, rowptr, col, A, x, bh, y, omega, err, lim); break;
    case 4: mr_tc_smooth_kernel<4><<<dim3(gx, gy), kTcRows, 0, s>>>(n, R, rowptr, col, A, x, bh, y, omega, err, lim); break;
    case 6: mr_tc_smooth_kernel<6><<<dim3(gx, gy), kTcRows, 0, s>>>(n, R, rowptr, col, A, x, bh, y, omega, err, lim); break;
    case 10: mr_tc_smooth_kernel<10><<<dim3(gx, gy), kTcRows, 0, s>>>(n, R, rowptr, col, A, x, bh, y, omega, err, lim); break;
    default: return false;
  }
  count_launch();
  return true;
}
