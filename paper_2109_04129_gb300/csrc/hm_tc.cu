// Tensor-core (tcgen05) gather GEMM for the mixed-precision chain.
//
// Same tasks and items as the SIMT gather kernels (R^T / R sweep blocks, both
// far-field stages; far stage 1 in its stacked form), on complex64 matrices
// and panels.  For each task and tile of 128 right-hand sides:
//
//   D (128 RHS x 2m) = X' (128 x 2K) * B'^T,   B' row 2i   = [a_re, -a_im] (interleaved over k)
//                                              B' row 2i+1 = [a_im,  a_re]
//   so D[r][2i] = Re(sum_k a_ik x_kr), D[r][2i+1] = Im(...)   (complex product as one real GEMM)
//
// Both operands are split into three bf16 slices (v = s0 + s1 + s2, about 24
// significant bits) and the six slice products with s_p * s_q, p + q <= 2,
// accumulate in FP32 in tensor memory (s0 * s0 and the rest in two separate
// accumulators, added in the epilogue): products carry FP32-level accuracy.
//
// Operands: the matrix never changes between solves, so its three slices are
// computed once at set-up (build_tc_tiles) and stored tile by tile in the
// K-major no-swizzle canonical layout (8-row x 16-byte core matrices) that the
// MMA reads.  The right-hand sides come from split panels (k_split for the
// far-field inputs, and for the sweep buffer at the start of a sweep, kept
// current by k_finalize_split).  A stage of both operands arrives by bulk
// copies (cp.async.bulk, completion on an mbarrier).  The kernel is persistent and warp-specialised; the roles,
// barriers and bounded waits are described at k_tc_gather.
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
constexpr int TC_THREADS = 256;  // threads of the set-up tile builder
constexpr int A_SLICE_BYTES = TC_M * TC_KR * 2;       // 8 KB
constexpr int B_SLICE_BYTES = TC_NMAX * TC_KR * 2;    // 16 KB
constexpr int TC_STAGE = TC_NS * (A_SLICE_BYTES + B_SLICE_BYTES);   // 72 KB

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


__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__host__ __device__ __forceinline__ int tc_nreal(int m) { return ((2 * m + 15) / 16) * 16; }

// Matrix tiles of one task: for each item and each 16-row inner stage, three
// bf16 slice planes of B' (n_real rows x 32 real inner columns, plane stride
// n_real x 64 bytes) in the canonical layout.  The stages of an item start on
// the 4-row boundary of the input below its first row (the inputs come from
// split panels tiled in 4-row groups); the rows the shift adds get zeros.
__global__ void __launch_bounds__(TC_THREADS) k_tc_tiles(const GTask* __restrict__ tasks,
                                                         const GItem* __restrict__ items,
                                                         ABufs ab, unsigned char* __restrict__ tiles,
                                                         const long long* __restrict__ toff) {
  const GTask t = tasks[blockIdx.x];
  const int n_real = tc_nreal(t.m);
  const long long plane = (long long)n_real * 64;
  unsigned char* dst = tiles + toff[blockIdx.x];
  const int ne = (n_real / 2) * TC_KC;
  for (int it = t.it0; it < task_it_end(t); ++it) {
    const GItem I = items[it];
    const int dl = I.in_row & 3;
    const int nst = (I.k + dl + TC_KC - 1) / TC_KC;
    for (int st = 0; st < nst; ++st) {
      for (int e = threadIdx.x; e < ne; e += TC_THREADS) {
        int i, kk;
        if (I.trans) {
          kk = e / (n_real / 2);
          i = e % (n_real / 2);
        } else {
          i = e / TC_KC;
          kk = e % TC_KC;
        }
        const int kr = st * TC_KC + kk - dl;
        // the item holding row i: this one, or the row segment of a stacked task
        GItem S = I;
        int li = i;
        if (t.mode == 2) {
          S.nrow = 0;
          for (int q = t.it0; q < t.it1; ++q) {
            const GItem Q = items[q];
            if (i >= Q.r0 && i < Q.r0 + Q.nrow) {
              S = Q;
              li = i - Q.r0;
            }
          }
          if (S.nrow == 0) li = -1;
        }
        const float2* A = (const float2*)ab.p[S.a_buf] + S.a_off;
        float2 a = make_float2(0.f, 0.f);
        if (i < t.m && li >= 0 && kr >= 0 && kr < I.k)
          a = S.trans ? A[(long long)kr * S.lda + li] : A[(long long)li * S.lda + kr];
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

// byte offset of the 16-byte row (slice p, 128-RHS tile y, 4-row group j,
// 8-RHS group gl, RHS r8 within it) of a split panel with Y tiles, J groups
__host__ __device__ __forceinline__ long long xs_off(int p, int Y, int y, long long J, long long j,
                                                     int gl, int r8) {
  return ((((long long)p * Y + y) * J + j) * 16 + gl) * 128 + r8 * 16;
}

// Split panel of V (rows x nrhs complex64, RHS fastest): thread = (4-row
// group j, RHS r); for every slice it writes the 16-byte core-matrix row
// (re, im) of rows 4j..4j+3.  Rows >= rows and RHS >= nrhs are zero.
__global__ void k_split(const float2* __restrict__ V, int rows, int nrhs,
                        unsigned char* __restrict__ out, long long J, int G) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int R8 = G * 8;
  if (idx >= J * R8) return;
  const int r = (int)(idx % R8);
  const long long j = idx / R8;
  __nv_bfloat16 d[8][TC_NS];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const long long row = 4 * j + c;
    const float2 v = (row < rows && r < nrhs) ? V[row * nrhs + r] : make_float2(0.f, 0.f);
    split3(v.x, d[2 * c]);
    split3(v.y, d[2 * c + 1]);
  }
  const int Y = G / 16;
#pragma unroll
  for (int p = 0; p < TC_NS; ++p) {
    uint4 w;
    w.x = pack2(d[0][p], d[1][p]);
    w.y = pack2(d[2][p], d[3][p]);
    w.z = pack2(d[4][p], d[5][p]);
    w.w = pack2(d[6][p], d[7][p]);
    *(uint4*)(out + xs_off(p, Y, r >> 7, J, j, (r >> 3) & 15, r & 7)) = w;
  }
}

// Sweep finalize (complex64) that also keeps the split panel of the sweep
// buffer current: out = base + sum of the task's partial panels, and the
// three bf16 slices of every finalized element go to its place in the split
// panel (4-byte (re, im) pairs).
// Each thread finalizes FIN_EPT elements of the target, FIN_EPT apart by the
// grid stride, and issues the loads of all of them before it adds: the
// partials of one element are summed in slot order, as a plain loop would.
constexpr int FIN_EPT = 4;
__global__ void k_finalize_split(const FTask* __restrict__ tasks, const int* __restrict__ slots,
                                 VBufs vb, int nrhs, unsigned char* __restrict__ xs, long long J,
                                 int G) {
  const FTask t = tasks[blockIdx.x];
  const long long n = (long long)t.m * nrhs;
  const long long e0 = threadIdx.x + (long long)blockIdx.y * blockDim.x;
  if (e0 >= n) return;
  const long long stride = (long long)blockDim.x * gridDim.y;
  float2* out = (float2*)vb.p[t.out_buf] + (long long)t.out_row * nrhs;
  const float2* base = (const float2*)vb.p[t.base_buf] + (long long)t.base_row * nrhs;
  const float2* scr = (const float2*)vb.p[VB_SCR];
  const int Y = G / 16;
  for (long long ea = e0; ea < n; ea += FIN_EPT * stride) {
    float2 v[FIN_EPT];
#pragma unroll
    for (int k = 0; k < FIN_EPT; ++k) {
      const long long e = ea + k * stride;
      v[k] = e < n ? base[e] : make_float2(0.f, 0.f);
    }
    for (int s = t.s0; s < t.s1; ++s) {
      const float2* P = scr + (long long)slots[s] * nrhs;
      float2 p[FIN_EPT];
#pragma unroll
      for (int k = 0; k < FIN_EPT; ++k) {
        const long long e = ea + k * stride;
        p[k] = e < n ? P[e] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < FIN_EPT; ++k) {
        v[k].x += p[k].x;
        v[k].y += p[k].y;
      }
    }
#pragma unroll
    for (int k = 0; k < FIN_EPT; ++k) {
      const long long e = ea + k * stride;
      if (e >= n) break;
      out[e] = v[k];
      const long long row = t.out_row + e / nrhs;
      const int r = (int)(e % nrhs);
      __nv_bfloat16 sr[TC_NS], si[TC_NS];
      split3(v[k].x, sr);
      split3(v[k].y, si);
#pragma unroll
      for (int q = 0; q < TC_NS; ++q)
        *(uint32_t*)(xs + xs_off(q, Y, r >> 7, J, row >> 2, (r >> 3) & 15, r & 7) +
                     (row & 3) * 4) = pack2(sr[q], si[q]);
    }
  }
}

// shared-memory descriptor with explicit strides (no swizzle)
__device__ __forceinline__ uint64_t sdesc_g(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

constexpr int TC_RING = 3;                 // shared-memory stages of the gather
constexpr int TC_WTHREADS = 192;           // 6 warps
constexpr int TC_GSMEM = TC_RING * TC_STAGE + 1024;

// bounded wait that also gives up when another role has aborted the CTA
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t phase, long long limit,
                                        volatile int* abort_flag, int* err) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (done) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ void tc_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(bar));
}
// the 16-row stages of an item: from the 4-row boundary of the input panel
// below its first row (split-panel blocks start on 4-row groups)
__device__ __forceinline__ int tc_nst(const GItem& I) {
  return (I.k + (I.in_row & 3) + TC_KC - 1) / TC_KC;
}

// Persistent, warp-specialised gather GEMM on complex64 lists.  Each CTA
// walks its share of the tasks (costliest first) for one tile of 128 RHS:
//   warp 0 (one thread) issues the 12 MMAs of a stage (6 slice products x 2 K
//     steps) into the task's two accumulators: s0 x s0 into the main one, the
//     five smaller slice products into a correction accumulator.  A narrow
//     task (n_real <= 128) keeps both in tensor-memory half j & 1 for the
//     CTA's j-th task, so the epilogue of one task overlaps the next task; a
//     wide one (n_real <= 256) takes all 512 columns, and before task j the
//     MMAs wait for the drain of task j - 2, or of j - 1 when j or j - 1 is
//     wide;
//   warp 1 (one thread) fetches the stage: the pre-split matrix tile and the
//     16 input rows of every slice of the split panel (six bulk copies,
//     completion on the stage's "tile" mbarrier);
//   warps 2-5 read both accumulators (thread = TMEM lane = RHS row), add them
//     and the base rows in FP32 and store complex64 outputs.
// Why two accumulators: every MMA rounds the running FP32 sum it adds into
// toward zero, and these sums cancel heavily, so the rounding error of a
// chain grows with the number of MMAs that add into the same accumulator.
// Five of the six products are 2^8 to 2^16 times smaller than s0 x s0: added
// into the main sum they cost five roundings of it each for bits it barely
// needs.  In a separate accumulator their roundings scale with their own
// size, and the main sum takes one sixth of the MMAs (measured on the 2
// lambda sphere: the mixed chain's error is unchanged by 16x shorter split-K
// chains, so it is the count of MMAs per target, not the chain length).
// Stage buffers form a ring of TC_RING: tile[b] full -> MMAs -> empty[b];
// accumulators: tfull[h] (MMAs of a task done) -> epilogue -> tempty[h].
// Every wait is bounded and watches a CTA-wide abort flag.
__global__ void __launch_bounds__(TC_WTHREADS, 1) k_tc_gather(
    const GTask* __restrict__ tasks, const GItem* __restrict__ items,
    const int* __restrict__ order, int n_tasks, VBufs vb, XSplit xsp,
    const unsigned char* __restrict__ tiles, const long long* __restrict__ toff, int nrhs,
    long long spin_limit, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[2 * TC_RING + 5];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int armed_s, consumed_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_tile = __cvta_generic_to_shared(&bars[0]);               // + 8 b
  const uint32_t b_empty = __cvta_generic_to_shared(&bars[TC_RING]);        // + 8 b
  const uint32_t b_tfull = __cvta_generic_to_shared(&bars[2 * TC_RING]);    // + 8 h
  const uint32_t b_tempty = b_tfull + 16;                                    // + 8 h
  const uint32_t b_fin = b_tfull + 32;
  volatile int* abortp = &abort_flag;
  const int y = blockIdx.y;
  if (tid == 0) {
    for (int b = 0; b < TC_RING; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_tile + 8u * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_empty + 8u * b));
    }
    for (int h = 0; h < 2; ++h) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_tfull + 8u * h));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(b_tempty + 8u * h),
                   "r"(TC_M));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_fin));
    abort_flag = 0;
    armed_s = 0;
    consumed_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------ MMA issuer (one thread)
    if (lane == 0) {
      int g = 0, j = 0;
      bool stop = false, prev_wide = false;
      for (int u = blockIdx.x; u < n_tasks && !stop; u += gridDim.x) {
        const GTask t = tasks[order[u]];
        if (t.m <= 0) continue;
        const int n_real = tc_nreal(t.m);
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) |
                               ((uint32_t)(n_real >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
        const bool wide = n_real > 128;
        const uint32_t dmain = tmem + (wide ? 0u : (uint32_t)(j & 1) * 256u);
        const uint32_t dcorr = dmain + (wide ? 256u : 128u);
        bool first_m = true, first_c = true;
        for (int it = t.it0; it < task_it_end(t) && !stop; ++it) {
          const int nst = tc_nst(items[it]);
          for (int st = 0; st < nst; ++st) {
            // the columns of task j were last used by task j - 2 (both
            // narrow), or by task j - 1 as well when either of the two is wide
            const int need = (wide || prev_wide) ? j - 1 : j - 2;
            if (first_m && need >= 0 &&
                !tc_wait(b_tempty + 8u * (need & 1), (uint32_t)((need >> 1) & 1), spin_limit,
                         abortp, err)) {
              stop = true;
              break;
            }
            const int b = g % TC_RING;
            const uint32_t ph = (uint32_t)((g / TC_RING) & 1);
            if (!tc_wait(b_tile + 8u * b, ph, spin_limit, abortp, err)) {
              stop = true;
              break;
            }
            consumed_s = g + 1;
            asm volatile("tcgen05.fence::after_thread_sync;");
            unsigned char* sA = smem + b * TC_STAGE;
            // X' slices: split-panel blocks (K-adjacent core matrices 2 KB
            // apart, 8-row groups 128 B apart)
            const uint64_t da0 = sdesc_g(smem_u32(sA), 2048, 128);
            constexpr int kstep = 4096;             // bytes per 16 real inner columns
            const uint64_t db0 = sdesc(smem_u32(sA + TC_NS * A_SLICE_BYTES));
#pragma unroll
            for (int p = 0; p < TC_NS; ++p)
#pragma unroll
              for (int q = 0; p + q < TC_NS; ++q)
#pragma unroll
                for (int kh = 0; kh < TC_KR / 16; ++kh) {
                  const uint64_t da = da0 + (uint64_t)((p * A_SLICE_BYTES + kh * kstep) >> 4);
                  const uint64_t db = db0 + (uint64_t)((q * B_SLICE_BYTES + kh * 256) >> 4);
                  // s0 x s0 into the main accumulator, the five smaller
                  // products into a second one (see the note above)
                  const bool mainp = p + q == 0;
                  const uint32_t acc = (mainp ? first_m : first_c) ? 0u : 1u;
                  if (mainp)
                    first_m = false;
                  else
                    first_c = false;
                  asm volatile(
                      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                      :: "r"(mainp ? dmain : dcorr), "l"(da), "l"(db), "r"(idesc), "r"(acc));
                }
            tc_commit(b_empty + 8u * b);
            ++g;
          }
        }
        if (!first_m && !stop) {
          tc_commit(b_tfull + 8u * (j & 1));
          prev_wide = wide;
          ++j;
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ matrix tiles (one thread)
    if (lane == 0) {
      int g = 0;
      bool stop = false;
      for (int u = blockIdx.x; u < n_tasks && !stop; u += gridDim.x) {
        const GTask t = tasks[order[u]];
        if (t.m <= 0) continue;
        const uint32_t plane = (uint32_t)tc_nreal(t.m) * 64;
        const unsigned char* tile = tiles + toff[order[u]];
        for (int it = t.it0; it < task_it_end(t) && !stop; ++it) {
          const GItem I = items[it];
          const int nst = tc_nst(I);
          const int xb = (I.in_buf == VB_FAR) ? 1 : 0;
          const long long j00 = (long long)((I.in_row - (I.in_row & 3)) >> 2);
          for (int st = 0; st < nst; ++st) {
            const int b = g % TC_RING;
            if (g >= TC_RING &&
                !tc_wait(b_empty + 8u * b, (uint32_t)(((g - TC_RING) / TC_RING) & 1),
                         spin_limit, abortp, err)) {
              stop = true;
              break;
            }
            const uint32_t fb = b_tile + 8u * b;
            unsigned char* sB = smem + b * TC_STAGE + TC_NS * A_SLICE_BYTES;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(fb), "r"(TC_NS * (plane + A_SLICE_BYTES)) : "memory");
            for (int q = 0; q < TC_NS; ++q)
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                  :: "r"(smem_u32(sB + q * B_SLICE_BYTES)), "l"(tile + (size_t)q * plane),
                     "r"(plane), "r"(fb) : "memory");
            {
              // the stage's 16 input rows of each slice: one 8 KB block
              const long long j0 = j00 + 4LL * st;
              unsigned char* sA = smem + b * TC_STAGE;
              for (int q = 0; q < TC_NS; ++q)
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    :: "r"(smem_u32(sA + q * A_SLICE_BYTES)),
                       "l"(xsp.xs[xb] + xs_off(q, xsp.G / 16, y, xsp.J[xb], j0, 0, 0)),
                       "r"(A_SLICE_BYTES), "r"(fb) : "memory");
            }
            tile += (size_t)TC_NS * plane;
            ++g;
            armed_s = g;
          }
        }
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 2-5)
    const int q4 = warp & 3;                   // TMEM lane quarter of this warp
    const int r = q4 * 32 + lane;              // RHS row of the tile
    const int col = y * TC_M + r;
    const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
    int j = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < n_tasks && !stop; u += gridDim.x) {
      const GTask t = tasks[order[u]];
      if (t.m <= 0) continue;
      bool has = false;
      for (int it = t.it0; it < task_it_end(t) && !has; ++it) has = tc_nst(items[it]) > 0;
      const int n_real = tc_nreal(t.m);
      float2* out = (float2*)vb.p[t.out_buf] + (long long)t.out_row * nrhs;
      const float2* base = (t.mode == 1) ? (const float2*)vb.p[t.base_buf] + (long long)t.base_row * nrhs
                                         : nullptr;
      if (!has) {                              // no inner rows: out = base (or 0)
        if (col < nrhs)
          for (int i = 0; i < t.m; ++i)
            out[(long long)i * nrhs + col] = base ? base[(long long)i * nrhs + col]
                                                  : make_float2(0.f, 0.f);
        continue;
      }
      // tcgen05.ld is warp-collective: the warp takes one decision
      const bool okw = tc_wait(b_tfull + 8u * (j & 1), (uint32_t)((j >> 1) & 1), spin_limit,
                               abortp, err);
      if (!__all_sync(0xffffffffu, okw)) {
        stop = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      // main and correction sums: half j & 1 (at 0 and 128) for a narrow
      // task, all of tensor memory (at 0 and 256) for a wide one
      const bool wide = n_real > 128;
      const uint32_t cm = wide ? 0u : (uint32_t)(j & 1) * 256u;
      const uint32_t cc = cm + (wide ? 256u : 128u);
      for (int c0 = 0; c0 < n_real; c0 += 16) {
        uint32_t v[16], w[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(lane_base + cm + (uint32_t)c0));
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]),
              "=r"(w[6]), "=r"(w[7]), "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]),
              "=r"(w[12]), "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
            : "r"(lane_base + cc + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (col < nrhs) {
#pragma unroll
          for (int jj = 0; jj < 16; jj += 2) {
            const int i = (c0 + jj) / 2;
            if (i < t.m) {
              float2 yv = make_float2(__uint_as_float(v[jj]) + __uint_as_float(w[jj]),
                                      __uint_as_float(v[jj + 1]) + __uint_as_float(w[jj + 1]));
              if (base) {
                const float2 bv = base[(long long)i * nrhs + col];
                yv.x += bv.x;
                yv.y += bv.y;
              }
              out[(long long)i * nrhs + col] = yv;
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      tc_arrive(b_tempty + 8u * (j & 1));
      ++j;
    }
  }
  __syncthreads();
  if (abort_flag && tid == 0) {
    // a CTA that gave up: its MMAs and copies complete before tensor memory
    // and shared memory are released (bounded waits, abort flag ignored)
    volatile int never = 0;
    const long long lim = spin_limit > (1LL << 24) ? spin_limit : (1LL << 24);
    tc_commit(b_fin);
    tc_wait(b_fin, 0u, lim, &never, err);
    for (int g = consumed_s; g < armed_s; ++g)
      tc_wait(b_tile + 8u * (g % TC_RING), (uint32_t)((g / TC_RING) & 1), lim, &never, err);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
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
  cudaFree(tl.d_torder);
  tl.d_tiles = nullptr;
  tl.d_toff = nullptr;
  tl.d_torder = nullptr;
  tl.tile_bytes = 0;
  if (tl.tasks.empty() || !tc_ok_for(tl)) return HM_OK;
  std::vector<long long> off(tl.tasks.size());
  long long total = 0;
  for (size_t q = 0; q < tl.tasks.size(); ++q) {
    const GTask& t = tl.tasks[q];
    long long stages = 0;
    for (int it = t.it0; it < task_it_end(t); ++it) {
      const GItem& I = tl.items[it];
      stages += (I.k + (I.in_row & 3) + TC_KC - 1) / TC_KC;
    }
    off[q] = total;
    total += stages * TC_NS * (long long)tc_nreal(t.m) * 64;
  }
  HM_CUDA(cudaMalloc((void**)&tl.d_toff, off.size() * sizeof(long long)));
  HM_CUDA(cudaMemcpy(tl.d_toff, off.data(), off.size() * sizeof(long long),
                     cudaMemcpyHostToDevice));
  HM_CUDA(cudaMalloc((void**)&tl.d_tiles, std::max<long long>(total, 16)));
  // persistent CTAs walk the tasks costliest first
  std::vector<long long> cost(tl.tasks.size());
  std::vector<int> ord(tl.tasks.size());
  for (size_t q = 0; q < tl.tasks.size(); ++q) {
    cost[q] = (q + 1 < off.size() ? off[q + 1] : total) - off[q];
    ord[q] = (int)q;
  }
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  HM_CUDA(cudaMalloc((void**)&tl.d_torder, ord.size() * sizeof(int)));
  HM_CUDA(cudaMemcpy(tl.d_torder, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice));
  k_tc_tiles<<<(unsigned)tl.tasks.size(), TC_THREADS>>>(tl.d_tasks, tl.d_items, ab, tl.d_tiles,
                                                        tl.d_toff);
  HM_LAUNCHED();
  HM_CUDA(cudaDeviceSynchronize());
  tl.tile_bytes = (size_t)total;
  if (dev_bytes) *dev_bytes += (size_t)total + off.size() * sizeof(long long);
  return HM_OK;
}

size_t tc_split_bytes(int rows, int nrhs) {
  return (size_t)TC_NS * oz_rhs_groups(nrhs) * oz_row_groups(rows) * 128;
}

hm_status launch_split(const float2* V, int rows, int nrhs, unsigned char* out, long long J, int G,
                       cudaStream_t s) {
  const long long n = J * G * 8;
  k_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, rows, nrhs, out, J, G);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_fin_split(const FinList& fl, const VBufs& vb, int nrhs, unsigned char* xs,
                           long long J, int G, cudaStream_t s) {
  if (fl.tasks.empty()) return HM_OK;
  int mmax = 1;
  for (const FTask& f : fl.tasks) mmax = std::max(mmax, f.m);
  const long long per_task = (long long)mmax * nrhs;
  const long long per_block = 256LL * FIN_EPT;
  const int ny = (int)std::min<long long>(512, std::max<long long>(1, (per_task + per_block - 1) /
                                                                          per_block));
  k_finalize_split<<<dim3((unsigned)fl.tasks.size(), ny), 256, 0, s>>>(fl.d_tasks, fl.d_slots, vb,
                                                                       nrhs, xs, J, G);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_tasks_tc(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, long long spin_limit, int* err, const XSplit* xsp) {
  if (tl.tasks.empty()) return HM_OK;
  if (!tl.d_tiles || !tl.d_toff || !tl.d_torder) return HM_ERR_STATE;
  // the right-hand sides come from split panels
  if (!xsp || xsp->G * 8 < nrhs || xsp->G % 16 != 0 || !xsp->xs[0]) return HM_ERR_INVALID;
  (void)ab;
  static bool attr = false;
  static int nsm = 0;
  if (!attr) {
    HM_CUDA(cudaFuncSetAttribute(k_tc_gather, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_GSMEM));
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    attr = true;
  }
  // one resident CTA per SM: the tiles of 128 RHS share the SMs
  const int nt = (int)tl.tasks.size();
  const int ytiles = (nrhs + TC_M - 1) / TC_M;
  const int gx = std::max(1, std::min(nt, std::max(1, nsm / ytiles)));
  dim3 grid((unsigned)gx, (unsigned)ytiles);
  k_tc_gather<<<grid, TC_WTHREADS, TC_GSMEM, s>>>(tl.d_tasks, tl.d_items, tl.d_torder, nt, vb,
                                                  *xsp, tl.d_tiles, tl.d_toff, nrhs, spin_limit,
                                                  err);
  HM_LAUNCHED();
  return HM_OK;
}

}  // namespace hm
