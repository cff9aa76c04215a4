// Tensor-core (tcgen05) gather GEMM for the mixed-precision chain.
//
// Same tasks and items as the SIMT gather kernels (R^T / R sweep blocks, both
// far-field stages), on complex64 matrices and panels.  One CTA computes one
// task for a tile of 128 right-hand sides:
//
//   D (128 RHS x 2m) = X' (128 x 2K) * B'^T,   B' row 2i   = [a_re, -a_im] (interleaved over k)
//                                              B' row 2i+1 = [a_im,  a_re]
//   so D[r][2i] = Re(sum_k a_ik x_kr), D[r][2i+1] = Im(...)   (complex product as one real GEMM)
//
// Both operands are split into three bf16 slices (v = s0 + s1 + s2, about 24
// significant bits) and the six slice products with s_p * s_q, p + q <= 2,
// accumulate in FP32 in tensor memory: products carry FP32-level accuracy.
//
// Mechanics: operands are staged by all threads into shared memory in the
// K-major no-swizzle canonical layout (8-row x 16-byte core matrices); one
// thread issues tcgen05.mma (kind::f16, bf16 inputs, f32 accumulate, M = 128,
// N = 2m rounded up to 16, K = 16 per instruction) and tcgen05.commit to an
// mbarrier; every wait on the mbarrier is bounded (spin_limit), after which the
// CTA records a timeout in *err and returns after releasing its tensor memory.
// The accumulator is read back with tcgen05.ld (32 lanes x 32-bit per warp).
#include <cuda_bf16.h>

#include "hm_internal.h"

namespace hm {

namespace {

constexpr int TC_M = 128;        // RHS per CTA (MMA M)
constexpr int TC_KC = 16;        // complex inner rows per stage (K = 32 real)
constexpr int TC_KR = 2 * TC_KC;
constexpr int TC_NS = 3;         // bf16 slices per operand
constexpr int TC_NMAX = 256;     // max MMA N (2 * 128 complex rows)
constexpr int TC_THREADS = 256;     // two halves share the staging; warps 0-3 own TMEM rows
constexpr int A_SLICE_BYTES = TC_M * TC_KR * 2;       // 8 KB
constexpr int B_SLICE_BYTES = TC_NMAX * TC_KR * 2;    // 16 KB
constexpr int TC_SMEM = TC_NS * (A_SLICE_BYTES + B_SLICE_BYTES) + 1024;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of (row, k) in a K-major tile with TC_KR elements along K
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return ((row >> 3) * (TC_KR >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;                   // K-adjacent core matrices
  d |= (uint64_t)(((TC_KR / 8) * 128u >> 4) & 0x3FFF) << 32;      // next 8-row group
  d |= (uint64_t)1 << 46;                                          // descriptor version
  return d;
}

__device__ __forceinline__ void split3(float v, __nv_bfloat16* s) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);
  float r = v - __bfloat162float(h);
  __nv_bfloat16 m = __float2bfloat16_rn(r);
  float r2 = r - __bfloat162float(m);
  s[0] = h;
  s[1] = m;
  s[2] = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (done) return true;
  }
  return false;
}

__global__ void __launch_bounds__(TC_THREADS) k_tc_gather(const GTask* __restrict__ tasks,
                                                          const GItem* __restrict__ items,
                                                          VBufs vb, ABufs ab, int nrhs,
                                                          long long spin_limit, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;                                  // TC_NS x (128 x 32) bf16
  unsigned char* sB = smem + TC_NS * A_SLICE_BYTES;          // TC_NS x (N x 32) bf16
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const GTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (TC_M - 1), half = tid >> 7;
  const int r0 = blockIdx.y * TC_M;
  const int n_real = ((2 * t.m + 15) / 16) * 16;             // MMA N
  const uint32_t ncols = n_real <= 32 ? 32 : (n_real <= 64 ? 64 : (n_real <= 128 ? 128 : 256));
  const uint32_t bar = smem_u32(&mbar);
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n_real >> 3) << 17) |
                         ((uint32_t)(TC_M >> 4) << 24);
  uint32_t phase = 0;
  bool first = true, ok = true;
  for (int it = t.it0; it < t.it1 && ok; ++it) {
    const GItem I = items[it];
    const float2* A = (const float2*)ab.p[I.a_buf] + I.a_off;
    const float2* X = (const float2*)vb.p[I.in_buf] + (long long)I.in_row * nrhs;
    for (int k0 = 0; k0 < I.k && ok; k0 += TC_KC) {
      const int kc = min(TC_KC, I.k - k0);
      // ---- stage X' (128 RHS x 32): thread = RHS row, halves split the inner rows;
      // all loads of the thread are issued before any use (one memory latency)
      {
        const int r = row;
        const int col = r0 + r;
        constexpr int KH = TC_KC / 2;
        float2 xv[KH];
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int kk = half * KH + j;
          xv[j] = (kk < kc && col < nrhs) ? X[(long long)(k0 + kk) * nrhs + col]
                                          : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int kk = half * KH + j;
          __nv_bfloat16 sr[TC_NS], si[TC_NS];
          split3(xv[j].x, sr);
          split3(xv[j].y, si);
#pragma unroll
          for (int s = 0; s < TC_NS; ++s) {
            *(__nv_bfloat16*)(sA + s * A_SLICE_BYTES + kmaj(r, 2 * kk)) = sr[s];
            *(__nv_bfloat16*)(sA + s * A_SLICE_BYTES + kmaj(r, 2 * kk + 1)) = si[s];
          }
        }
      }
      // ---- stage B' (n_real rows x 32): element (i, kk) of op(A); loads first
      {
        constexpr int EMAX = (TC_NMAX / 2) * TC_KC / TC_THREADS;   // 8
        const int ne = (n_real / 2) * TC_KC;
        float2 av[EMAX];
#pragma unroll
        for (int q = 0; q < EMAX; ++q) {
          const int e = tid + q * TC_THREADS;
          int i, kk;
          if (I.trans) {
            kk = e / (n_real / 2);
            i = e % (n_real / 2);
          } else {
            i = e / TC_KC;
            kk = e % TC_KC;
          }
          av[q] = make_float2(0.f, 0.f);
          if (e < ne && i < t.m && kk < kc)
            av[q] = I.trans ? A[(long long)(k0 + kk) * I.lda + i]
                            : A[(long long)i * I.lda + k0 + kk];
        }
#pragma unroll
        for (int q = 0; q < EMAX; ++q) {
          const int e = tid + q * TC_THREADS;
          if (e >= ne) break;
          int i, kk;
          if (I.trans) {
            kk = e / (n_real / 2);
            i = e % (n_real / 2);
          } else {
            i = e / TC_KC;
            kk = e % TC_KC;
          }
          __nv_bfloat16 ar[TC_NS], ai[TC_NS];
          split3(av[q].x, ar);
          split3(av[q].y, ai);
#pragma unroll
          for (int s = 0; s < TC_NS; ++s) {
            unsigned char* b = sB + s * B_SLICE_BYTES;
            *(__nv_bfloat16*)(b + kmaj(2 * i, 2 * kk)) = ar[s];
            *(__nv_bfloat16*)(b + kmaj(2 * i, 2 * kk + 1)) = __hneg(ai[s]);
            *(__nv_bfloat16*)(b + kmaj(2 * i + 1, 2 * kk)) = ai[s];
            *(__nv_bfloat16*)(b + kmaj(2 * i + 1, 2 * kk + 1)) = ar[s];
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        for (int p = 0; p < TC_NS; ++p)
          for (int q = 0; p + q < TC_NS; ++q)
            for (int kh = 0; kh < TC_KR / 16; ++kh) {
              uint64_t da = sdesc(smem_u32(sA + p * A_SLICE_BYTES) + kh * 256);
              uint64_t db = sdesc(smem_u32(sB + q * B_SLICE_BYTES) + kh * 256);
              uint32_t acc = first ? 0u : 1u;
              first = false;
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                  :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
            :: "r"(bar));
      }
      first = false;
      // shared memory is reused by the next stage: wait for the MMAs
      if (!mbar_wait(bar, phase, spin_limit)) {
        ok = false;
        if (tid == 0) atomicExch(err, 1);
      }
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;");
    }
  }
  // ---- epilogue: thread (warp w < 4, lane l) owns TMEM lane 32w + l = RHS row
  if (ok && half == 0) {
    const int r = tid;
    const int col = r0 + r;
    float2* out = (float2*)vb.p[t.out_buf] + (long long)t.out_row * nrhs;
    const float2* base = (t.mode == 1) ? (const float2*)vb.p[t.base_buf] + (long long)t.base_row * nrhs
                                       : nullptr;
    for (int c0 = 0; c0 < n_real; c0 += 16) {
      uint32_t v[16];
      uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      if (first) {
        for (int j = 0; j < 16; ++j) v[j] = 0u;     // no inner rows: acc = 0
      } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
      }
      if (col < nrhs) {
        for (int j = 0; j < 16; j += 2) {
          int i = (c0 + j) / 2;
          if (i >= t.m) break;
          float2 y = make_float2(__uint_as_float(v[j]), __uint_as_float(v[j + 1]));
          if (base) {
            float2 b = base[(long long)i * nrhs + col];
            y.x += b.x;
            y.y += b.y;
          }
          out[(long long)i * nrhs + col] = y;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(ncols));
}

}  // namespace

bool tc_ok_for(const TaskList& tl) {
  for (const GTask& t : tl.tasks)
    if (2 * t.m > TC_NMAX) return false;
  return true;
}

hm_status launch_tasks_tc(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, long long spin_limit, int* err) {
  if (tl.tasks.empty()) return HM_OK;
  static bool attr = false;
  if (!attr) {
    HM_CUDA(cudaFuncSetAttribute(k_tc_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_SMEM));
    attr = true;
  }
  dim3 grid((unsigned)tl.tasks.size(), (unsigned)((nrhs + TC_M - 1) / TC_M));
  k_tc_gather<<<grid, TC_THREADS, TC_SMEM, s>>>(tl.d_tasks, tl.d_items, vb, ab, nrhs, spin_limit,
                                                err);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

}  // namespace hm
