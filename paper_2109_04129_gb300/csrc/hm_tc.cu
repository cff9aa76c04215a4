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
// Mechanics: the matrix operand never changes between solves, so its three
// bf16 slices are computed once at set-up (build_tc_tiles) and stored tile by
// tile in the K-major no-swizzle canonical layout (8-row x 16-byte core
// matrices) that the MMA reads; a stage fetches its tile with three bulk
// copies (cp.async.bulk, completion on an mbarrier).  The right-hand sides
// change between launches and are split on the fly, their loads issued one
// stage ahead.  Two shared-memory stages alternate; one thread issues
// tcgen05.mma (kind::f16, bf16 inputs, f32 accumulate, M = 128, N = 2m
// rounded up to 16, K = 16 per instruction) and tcgen05.commit to an mbarrier
// per stage; every wait is bounded (spin_limit), a failed wait is made
// uniform over the CTA, recorded in *err, and the CTA returns after letting
// its copies land and releasing its tensor memory.  The accumulator is read
// back with tcgen05.ld (32 lanes x 32-bit per warp).
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

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
constexpr int TC_STAGE = TC_NS * (A_SLICE_BYTES + B_SLICE_BYTES);   // 72 KB
constexpr int TC_SMEM = 2 * TC_STAGE + 1024;                       // double buffered

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

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__host__ __device__ __forceinline__ int tc_nreal(int m) { return ((2 * m + 15) / 16) * 16; }

// Matrix tiles of one task: for each item and each 16-row inner stage, three
// bf16 slice planes of B' (n_real rows x 32 real inner columns, plane stride
// n_real x 64 bytes) in the canonical layout.
__global__ void __launch_bounds__(TC_THREADS) k_tc_tiles(const GTask* __restrict__ tasks,
                                                         const GItem* __restrict__ items,
                                                         ABufs ab, unsigned char* __restrict__ tiles,
                                                         const long long* __restrict__ toff) {
  const GTask t = tasks[blockIdx.x];
  const int n_real = tc_nreal(t.m);
  const long long plane = (long long)n_real * 64;
  unsigned char* dst = tiles + toff[blockIdx.x];
  const int ne = (n_real / 2) * TC_KC;
  for (int it = t.it0; it < t.it1; ++it) {
    const GItem I = items[it];
    const float2* A = (const float2*)ab.p[I.a_buf] + I.a_off;
    for (int k0 = 0; k0 < I.k; k0 += TC_KC) {
      const int kc = min(TC_KC, I.k - k0);
      for (int e = threadIdx.x; e < ne; e += TC_THREADS) {
        int i, kk;
        if (I.trans) {
          kk = e / (n_real / 2);
          i = e % (n_real / 2);
        } else {
          i = e / TC_KC;
          kk = e % TC_KC;
        }
        float2 a = make_float2(0.f, 0.f);
        if (i < t.m && kk < kc)
          a = I.trans ? A[(long long)(k0 + kk) * I.lda + i] : A[(long long)i * I.lda + k0 + kk];
        __nv_bfloat16 ar[TC_NS], ai[TC_NS];
        split3(a.x, ar);
        split3(a.y, ai);
        for (int q = 0; q < TC_NS; ++q) {
          unsigned char* b = dst + q * plane;
          *(uint32_t*)(b + kmaj(2 * i, 2 * kk)) = pack2(ar[q], __hneg(ai[q]));
          *(uint32_t*)(b + kmaj(2 * i + 1, 2 * kk)) = pack2(ai[q], ar[q]);
        }
      }
      dst += TC_NS * plane;
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_tc_gather(
    const GTask* __restrict__ tasks, const GItem* __restrict__ items, VBufs vb,
    const unsigned char* __restrict__ tiles, const long long* __restrict__ toff, int nrhs,
    long long spin_limit, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[4];   // [b]: MMAs of buffer b done; [2 + b]: its tile landed
  __shared__ uint32_t tmem_base;
  const GTask t = tasks[blockIdx.x];
  if (t.m <= 0) return;                                      // whole CTA: uniform
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (TC_M - 1), half = tid >> 7;
  const int r0 = blockIdx.y * TC_M;
  const int col = r0 + row;
  const int n_real = tc_nreal(t.m);                          // MMA N
  const uint32_t ncols = n_real <= 32 ? 32 : (n_real <= 64 ? 64 : (n_real <= 128 ? 128 : 256));
  const uint32_t plane = (uint32_t)n_real * 64;              // bytes of one slice plane of a tile
  const uint32_t bar_done = smem_u32(&mbar[0]);
  const uint32_t bar_full = smem_u32(&mbar[2]);
  if (tid == 0) {
    for (int b = 0; b < 4; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_done + 8u * b));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
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
  uint32_t ph_done[2] = {0u, 0u}, ph_full[2] = {0u, 0u};
  bool outstanding[2] = {false, false};
  bool landing[2] = {false, false};       // (thread 0) copies issued into b, not yet seen landed
  uint32_t land_ph[2] = {0u, 0u};          // (thread 0) the phase they complete
  bool fail = false, ok = true, first = true;
  int sidx = 0;
  const unsigned char* tile = tiles + toff[blockIdx.x];

  auto wait_buf = [&](int b) {
    if (!outstanding[b]) return;
    if (!mbar_wait(bar_done + 8u * b, ph_done[b], spin_limit)) {
      fail = true;
      if (tid == 0) atomicExch(err, 1);
    }
    ph_done[b] ^= 1u;
    outstanding[b] = false;
  };
  // this thread's right-hand-side values of stage k0 of item it
  constexpr int KH = TC_KC / 2;
  auto load_x = [&](int it, int k0, float2* xv) {
    const GItem I = items[it];
    const float2* X = (const float2*)vb.p[I.in_buf] + (long long)I.in_row * nrhs;
    const int kc = min(TC_KC, I.k - k0);
#pragma unroll
    for (int j = 0; j < KH; ++j) {
      const int kk = half * KH + j;
      xv[j] = (kk < kc && col < nrhs) ? X[(long long)(k0 + kk) * nrhs + col]
                                      : make_float2(0.f, 0.f);
    }
  };

  // stages in the order of the tiles: items in order, 16 inner rows at a time
  // (items without inner rows have no stage)
  int it = t.it0, k0 = 0;
  while (it < t.it1 && items[it].k <= 0) ++it;
  float2 xv[KH];
  if (it < t.it1) load_x(it, 0, xv);
  while (it < t.it1 && ok) {
    const int kI = items[it].k;
    const int sb = sidx & 1;
    wait_buf(sb);
    unsigned char* sA = smem + sb * TC_STAGE;                  // X' slices
    unsigned char* sB = sA + TC_NS * A_SLICE_BYTES;            // B' slices
    // ---- matrix tile: three bulk copies (thread 0)
    if (tid == 0) {
      const uint32_t fb = bar_full + 8u * sb;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(fb), "r"(TC_NS * plane) : "memory");
      for (int q = 0; q < TC_NS; ++q)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            :: "r"(smem_u32(sB + q * B_SLICE_BYTES)), "l"(tile + (size_t)q * plane), "r"(plane),
               "r"(fb) : "memory");
    }
    landing[sb] = true;
    land_ph[sb] = ph_full[sb];
    tile += (size_t)TC_NS * plane;
    // ---- X' slices of the prefetched values (thread = RHS row, halves split the rows)
#pragma unroll
    for (int j = 0; j < KH; ++j) {
      const int kk = half * KH + j;
      __nv_bfloat16 sr[TC_NS], si[TC_NS];
      split3(xv[j].x, sr);
      split3(xv[j].y, si);
#pragma unroll
      for (int q = 0; q < TC_NS; ++q)
        *(uint32_t*)(sA + q * A_SLICE_BYTES + kmaj(row, 2 * kk)) = pack2(sr[q], si[q]);
    }
    // ---- next stage and its loads (in flight during this stage's MMAs)
    int it2 = it, k2 = k0 + TC_KC;
    if (k2 >= kI) {
      it2 = it + 1;
      k2 = 0;
      while (it2 < t.it1 && items[it2].k <= 0) ++it2;
    }
    if (it2 < t.it1) load_x(it2, k2, xv);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = !__syncthreads_or(fail);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) break;
    if (tid == 0) {
      if (!mbar_wait(bar_full + 8u * sb, ph_full[sb], spin_limit)) {
        fail = true;                  // the copies may still land: waited for at the end
        atomicExch(err, 1);
      } else {
        landing[sb] = false;
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
      }
      // always committed: a stage whose MMAs were skipped completes at once
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
          :: "r"(bar_done + 8u * sb));
    }
    first = false;
    if (tid != 0) landing[sb] = false;
    ph_full[sb] ^= 1u;
    outstanding[sb] = true;
    ++sidx;
    it = it2;
    k0 = k2;
  }
  // MMAs and copies in flight complete before the memory is released (a
  // limit of its own, so that a CTA that gave up still waits for them)
  const long long lim = spin_limit > (1LL << 24) ? spin_limit : (1LL << 24);
  for (int b = 0; b < 2; ++b) {
    if (outstanding[b] && !mbar_wait(bar_done + 8u * b, ph_done[b], lim)) {
      fail = true;
      if (tid == 0) atomicExch(err, 1);
    }
    outstanding[b] = false;
  }
  if (tid == 0) {
    for (int b = 0; b < 2; ++b)
      if (landing[b] && !mbar_wait(bar_full + 8u * b, land_ph[b], lim)) atomicExch(err, 1);
  }
  ok = !__syncthreads_or(fail);
  asm volatile("tcgen05.fence::after_thread_sync;");
  // ---- epilogue: thread (warp w < 4, lane l) owns TMEM lane 32w + l = RHS row
  if (ok && half == 0) {
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

hm_status build_tc_tiles(TaskList& tl, const ABufs& ab, size_t* dev_bytes) {
  cudaFree(tl.d_tiles);
  cudaFree(tl.d_toff);
  tl.d_tiles = nullptr;
  tl.d_toff = nullptr;
  tl.tile_bytes = 0;
  if (tl.tasks.empty() || !tc_ok_for(tl)) return HM_OK;
  std::vector<long long> off(tl.tasks.size());
  long long total = 0;
  for (size_t q = 0; q < tl.tasks.size(); ++q) {
    const GTask& t = tl.tasks[q];
    long long stages = 0;
    for (int it = t.it0; it < t.it1; ++it) stages += (tl.items[it].k + TC_KC - 1) / TC_KC;
    off[q] = total;
    total += stages * TC_NS * (long long)tc_nreal(t.m) * 64;
  }
  HM_CUDA(cudaMalloc((void**)&tl.d_toff, off.size() * sizeof(long long)));
  HM_CUDA(cudaMemcpy(tl.d_toff, off.data(), off.size() * sizeof(long long),
                     cudaMemcpyHostToDevice));
  HM_CUDA(cudaMalloc((void**)&tl.d_tiles, std::max<long long>(total, 16)));
  k_tc_tiles<<<(unsigned)tl.tasks.size(), TC_THREADS>>>(tl.d_tasks, tl.d_items, ab, tl.d_tiles,
                                                        tl.d_toff);
  HM_CUDA(cudaGetLastError());
  HM_CUDA(cudaDeviceSynchronize());
  tl.tile_bytes = (size_t)total;
  if (dev_bytes) *dev_bytes += (size_t)total + off.size() * sizeof(long long);
  return HM_OK;
}

hm_status launch_tasks_tc(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, long long spin_limit, int* err) {
  if (tl.tasks.empty()) return HM_OK;
  if (!tl.d_tiles || !tl.d_toff) return HM_ERR_STATE;
  (void)ab;
  static bool attr = false;
  if (!attr) {
    HM_CUDA(cudaFuncSetAttribute(k_tc_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_SMEM));
    attr = true;
  }
  dim3 grid((unsigned)tl.tasks.size(), (unsigned)((nrhs + TC_M - 1) / TC_M));
  k_tc_gather<<<grid, TC_THREADS, TC_SMEM, s>>>(tl.d_tasks, tl.d_items, vb, tl.d_tiles,
                                                tl.d_toff, nrhs, spin_limit, err);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

}  // namespace hm
