// FP64 kernels of the power-series solve: one generic "gather GEMM" that
// carries every block product of the chain (R^T and R sweeps of Eq. 25-26,
// the block-diagonal Z~_N^-1 of Eq. 32, both stages of the low-rank far-field
// product U (V^T y) of Eq. 11/13 and the near-field product), the split-K
// finalize, permutations, an axpby and per-RHS column norms (Eq. 45).
//
// Layout: vector panels are row-major (row stride nrhs, RHS fastest), so a
// row of a panel is one contiguous run of complex values.  Matrix blocks are
// row-major complex128.
#include <type_traits>

#include "hm_internal.h"

namespace hm {

namespace {

constexpr int MT = 64;    // output rows per tile
constexpr int KT = 32;    // inner-dimension tile
constexpr int NTHR = 256;

template <class T> struct Cx;
template <> struct Cx<double2> { typedef double R; };
template <> struct Cx<float2> { typedef float R; };

template <class A, class B> __device__ __forceinline__ A cvt(B v);
template <> __device__ __forceinline__ double2 cvt<double2, double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 cvt<double2, float2>(float2 v) {
  return make_double2(v.x, v.y);
}
template <> __device__ __forceinline__ float2 cvt<float2, double2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

template <class T>
__device__ __forceinline__ void cmac(T& acc, T a, T x) {
  acc.x = fma(a.x, x.x, acc.x);
  acc.x = fma(-a.y, x.y, acc.x);
  acc.y = fma(a.x, x.y, acc.y);
  acc.y = fma(a.y, x.x, acc.y);
}

template <class T> __device__ __forceinline__ T czero() { T z; z.x = 0; z.y = 0; return z; }

// Stage the (MT x KT) tile of op(A) rows [r0, r0+MT) x cols [k0, k0+KT) into
// shared memory (converted to the accumulation type), zero outside (m, k).
// Both orientations read along the contiguous direction of A, so global loads
// are coalesced.
template <class TA, class TC>
__device__ __forceinline__ void load_a_tile(TC (*As)[KT + 1], const TA* A, int lda, int trans,
                                            int r0, int m, int k0, int k) {
  if (!trans) {
    for (int e = threadIdx.x; e < MT * KT; e += NTHR) {
      int rr = e / KT, cc = e % KT;
      int r = r0 + rr, c = k0 + cc;
      As[rr][cc] = (r < m && c < k) ? cvt<TC, TA>(A[(long long)r * lda + c]) : czero<TC>();
    }
  } else {
    for (int e = threadIdx.x; e < MT * KT; e += NTHR) {
      int cc = e / MT, rr = e % MT;
      int r = r0 + rr, c = k0 + cc;
      As[rr][cc] = (r < m && c < k) ? cvt<TC, TA>(A[(long long)c * lda + r]) : czero<TC>();
    }
  }
}

// NT = RHS columns per CTA.  NT == 1: 64 rows x 4 k-lanes, shuffle reduce.
// NT >= 4: each thread owns RPT rows x CPT columns.
// TA: matrix element, TV: vector element, TC: accumulation (complex).
template <int NT, class TA, class TV, class TC>
__global__ void __launch_bounds__(NTHR) k_gather_gemm(const GTask* __restrict__ tasks,
                                                       const GItem* __restrict__ items,
                                                       VBufs vb, ABufs ab, int nrhs) {
  const GTask t = tasks[blockIdx.x];
  const int c0 = blockIdx.y * NT;
  __shared__ TC As[MT][KT + 1];
  __shared__ TC Xs[KT][NT];
  constexpr int CPT = (NT >= 16) ? 4 : (NT >= 4 ? NT / 4 : 1);
  constexpr int RPT = (NT >= 4) ? NT / (4 * CPT) : 1;
  constexpr int CG = (NT >= 4) ? NT / CPT : 1;        // column groups
  const int tid = threadIdx.x;
  int trow, tcol, klane;
  if (NT == 1) {
    trow = tid >> 2;
    klane = tid & 3;
    tcol = 0;
  } else {
    trow = (tid / CG) * RPT;
    tcol = (tid % CG) * CPT;
    klane = 0;
  }
  for (int r0 = 0; r0 < t.m; r0 += MT) {
    TC acc[RPT][CPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) acc[i][j] = czero<TC>();
    for (int it = t.it0; it < t.it1; ++it) {
      const GItem I = items[it];
      const TA* A = (const TA*)ab.p[I.a_buf] + I.a_off;
      const TV* X = (const TV*)vb.p[I.in_buf] + (long long)I.in_row * nrhs;
      for (int k0 = 0; k0 < I.k; k0 += KT) {
        load_a_tile<TA, TC>(As, A, I.lda, I.trans, r0, t.m, k0, I.k);
        for (int e = tid; e < KT * NT; e += NTHR) {
          int kk = e / NT, cc = e % NT;
          int kr = k0 + kk, col = c0 + cc;
          Xs[kk][cc] = (kr < I.k && col < nrhs) ? cvt<TC, TV>(X[(long long)kr * nrhs + col])
                                                : czero<TC>();
        }
        __syncthreads();
        if (NT == 1) {
#pragma unroll 8
          for (int kk = klane; kk < KT; kk += 4) cmac(acc[0][0], As[trow][kk], Xs[kk][0]);
        } else {
#pragma unroll 4
          for (int kk = 0; kk < KT; ++kk) {
            TC a[RPT], x[CPT];
#pragma unroll
            for (int i = 0; i < RPT; ++i) a[i] = As[trow + i][kk];
#pragma unroll
            for (int j = 0; j < CPT; ++j) x[j] = Xs[kk][tcol + j];
#pragma unroll
            for (int i = 0; i < RPT; ++i)
#pragma unroll
              for (int j = 0; j < CPT; ++j) cmac(acc[i][j], a[i], x[j]);
          }
        }
        __syncthreads();
      }
    }
    if (NT == 1) {
      // lanes 4q..4q+3 hold partial sums of the same row
      TC v = acc[0][0];
      v.x += __shfl_xor_sync(0xffffffffu, v.x, 1);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, 1);
      v.x += __shfl_xor_sync(0xffffffffu, v.x, 2);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, 2);
      acc[0][0] = v;
      if (klane != 0) continue;
    }
    TV* out = (TV*)vb.p[t.out_buf] + (long long)t.out_row * nrhs;
    const TV* base = (t.mode == 1) ? (const TV*)vb.p[t.base_buf] + (long long)t.base_row * nrhs
                                   : nullptr;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      int r = r0 + trow + i;
      if (r >= t.m) continue;
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        int col = c0 + tcol + j;
        if (col >= nrhs) continue;
        TC v = acc[i][j];
        if (base) {
          TC b = cvt<TC, TV>(base[(long long)r * nrhs + col]);
          v.x += b.x;
          v.y += b.y;
        }
        out[(long long)r * nrhs + col] = cvt<TV, TC>(v);
      }
    }
  }
}

// One-RHS variant (nrhs == 1), bound by HBM bandwidth: every matrix entry is
// read once and used once, so the kernel streams op(A) with coalesced loads
// and keeps several loads in flight per thread.  One CTA (8 warps) per task,
// output rows in chunks of 64:
//   trans = 1 (op(A)[i][k] = A[k lda + i]): lane = output rows (lane and
//     lane + 32), warp w takes the inner rows k = w, w + 8, ...: a warp reads
//     consecutive entries of one stored row, and x[k] is one broadcast load;
//   trans = 0 (op(A)[i][k] = A[i lda + k]): warp w owns rows w, w + 8, ...,
//     w + 56 of the chunk and its lanes walk k (coalesced along the stored
//     rows, the eight rows' loads issued together); each row's lane partials
//     meet in a warp-shuffle reduction.
// The next item's descriptor is fetched while the current one streams.  The
// eight warps' partials of a row are added in shared memory in warp order
// (deterministic, no atomics).
constexpr int GV_WARPS = 8;
constexpr int GV_UNROLL = 4;
constexpr int GV_ROWS = 64;               // output rows per chunk
constexpr int GV_RPW = GV_ROWS / GV_WARPS;  // trans = 0 rows per warp
template <class TA, class TV, class TC>
__global__ void __launch_bounds__(256) k_gemv(const GTask* __restrict__ tasks,
                                              const GItem* __restrict__ items, VBufs vb,
                                              ABufs ab) {
  const GTask t = tasks[blockIdx.x];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __shared__ TC part[GV_WARPS][GV_ROWS];
  typedef typename Cx<TC>::R R;
  for (int r0 = 0; r0 < t.m; r0 += GV_ROWS) {
    const int mr = min(GV_ROWS, t.m - r0);
    TC a1[2];                       // trans = 1: rows r0 + lane, r0 + 32 + lane
    TC a0[GV_RPW];                  // trans = 0: rows r0 + w + 8q, this lane's share of k
#pragma unroll
    for (int q = 0; q < 2; ++q) a1[q] = czero<TC>();
#pragma unroll
    for (int q = 0; q < GV_RPW; ++q) a0[q] = czero<TC>();
    GItem In;
    if (t.it0 < t.it1) In = items[t.it0];
    for (int it = t.it0; it < t.it1; ++it) {
      const GItem I = In;
      if (it + 1 < t.it1) In = items[it + 1];
      const TA* A = (const TA*)ab.p[I.a_buf] + I.a_off;
      const TV* X = (const TV*)vb.p[I.in_buf] + I.in_row;
      if (I.trans) {
        const bool v0 = lane < mr, v1 = lane + 32 < mr;
        const TA* Ai = A + r0 + lane;
        int k = w;
        for (; k + (GV_UNROLL - 1) * GV_WARPS < I.k; k += GV_UNROLL * GV_WARPS) {
          TA av0[GV_UNROLL], av1[GV_UNROLL];
          TV xv[GV_UNROLL];
#pragma unroll
          for (int u = 0; u < GV_UNROLL; ++u) {
            const long long o = (long long)(k + u * GV_WARPS) * I.lda;
            av0[u] = v0 ? Ai[o] : TA{};
            av1[u] = v1 ? Ai[o + 32] : TA{};
            xv[u] = X[k + u * GV_WARPS];
          }
#pragma unroll
          for (int u = 0; u < GV_UNROLL; ++u) {
            cmac(a1[0], cvt<TC, TA>(av0[u]), cvt<TC, TV>(xv[u]));
            cmac(a1[1], cvt<TC, TA>(av1[u]), cvt<TC, TV>(xv[u]));
          }
        }
        for (; k < I.k; k += GV_WARPS) {
          const long long o = (long long)k * I.lda;
          const TC xk = cvt<TC, TV>(X[k]);
          if (v0) cmac(a1[0], cvt<TC, TA>(Ai[o]), xk);
          if (v1) cmac(a1[1], cvt<TC, TA>(Ai[o + 32]), xk);
        }
      } else {
        // the warp's rows, their loads issued together
        for (int k0 = 0; k0 < I.k; k0 += 32) {
          const int k = k0 + lane;
          TA av[GV_RPW];
          TV xv = k < I.k ? X[k] : TV{};
#pragma unroll
          for (int q = 0; q < GV_RPW; ++q) {
            const int i = w + 8 * q;
            av[q] = (i < mr && k < I.k) ? A[(long long)(r0 + i) * I.lda + k] : TA{};
          }
#pragma unroll
          for (int q = 0; q < GV_RPW; ++q) cmac(a0[q], cvt<TC, TA>(av[q]), cvt<TC, TV>(xv));
        }
      }
    }
    // shuffle-reduce the trans = 0 partials of the warp's rows
#pragma unroll
    for (int q = 0; q < GV_RPW; ++q) {
      R re = a0[q].x, im = a0[q].y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      a0[q].x = re;
      a0[q].y = im;
    }
    // this warp's partials of rows r0 + lane and r0 + 32 + lane
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      TC mine = a1[h];
#pragma unroll
      for (int q = 0; q < GV_RPW; ++q)
        if (lane + 32 * h == w + 8 * q) {
          mine.x += a0[q].x;
          mine.y += a0[q].y;
        }
      part[w][lane + 32 * h] = mine;
    }
    __syncthreads();
    if (threadIdx.x < mr) {
      const int i = threadIdx.x;
      TC v = part[0][i];
#pragma unroll
      for (int q = 1; q < GV_WARPS; ++q) {
        v.x += part[q][i].x;
        v.y += part[q][i].y;
      }
      if (t.mode == 1) {
        const TC b = cvt<TC, TV>(((const TV*)vb.p[t.base_buf])[t.base_row + r0 + i]);
        v.x += b.x;
        v.y += b.y;
      }
      ((TV*)vb.p[t.out_buf])[t.out_row + r0 + i] = cvt<TV, TC>(v);
    }
    __syncthreads();
  }
}

// One-RHS variant for complex128 matrices with the blocks staged by bulk
// copies.  Every item of a task is a set of stored rows of one matrix block:
// trans = 0: rows i < m, each k entries (op(A)[i][kk] = A[i lda + kk]);
// trans = 1: rows kk < k, each m entries (op(A)[i][kk] = A[kk lda + i]).
// A piece is a run of whole stored rows of one item, at most GB_CHUNK bytes;
// warp 8 (one thread) copies the pieces in order into a ring of GB_STAGES
// shared-memory stages (cp.async.bulk, completion on the stage's "full"
// mbarrier: one copy when the rows are contiguous, else one per row), and the
// eight consumer warps multiply them as they land ("empty" mbarrier, eight
// arrivals, hands the stage back), so several pieces are in flight per CTA.
//   trans = 1: thread c is row i = c % m of group c / m; group g takes the
//     stored rows kk = g, g + G, ... of each piece (G = 256 / m groups);
//   trans = 0: warp w takes the rows i = w mod 8 of each piece, lanes along
//     kk, one warp-shuffle reduction per row into a shared row sum.
// Rows are added in a fixed order (deterministic).  Every wait is bounded: a
// CTA that gives up records it in *err, waits (bounded) for its own copies in
// flight and leaves its outputs unwritten.  Tasks of at most 256 rows and
// stored rows of at most GB_CHUNK bytes (checked on the host per list).
constexpr int GB_STAGES = 4;
constexpr int GB_CHUNK = 16384;
constexpr int GB_THREADS = 288;           // 8 consumer warps + 1 copy warp
constexpr int GB_SMEM = GB_STAGES * GB_CHUNK + 1024;

__device__ __forceinline__ bool gb_wait(uint32_t bar, uint32_t phase, long long limit,
                                        volatile int* abort_flag, int* err) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (done) return true;
    if (abort_flag && *abort_flag) return false;
  }
  if (abort_flag) *abort_flag = 1;
  if (err) atomicExch(err, 1);
  return false;
}

// stored rows of item I and the entries of each (see k_gemv_bulk)
__device__ __forceinline__ void gb_rows(const GItem& I, int m, int& nrow, int& len) {
  nrow = I.trans ? I.k : m;
  len = I.trans ? m : I.k;
}

template <class TV>
__global__ void __launch_bounds__(GB_THREADS) k_gemv_bulk(const GTask* __restrict__ tasks,
                                                          const GItem* __restrict__ items,
                                                          VBufs vb, ABufs ab,
                                                          long long spin_limit, int* err) {
  extern __shared__ __align__(128) unsigned char gb_smem[];
  __shared__ __align__(8) uint64_t bars[2 * GB_STAGES];
  __shared__ double2 part[256];            // trans = 1 partials [group][row]
  __shared__ double2 rowsum[256];          // trans = 0 row sums
  __shared__ int abort_flag, issued_s;
  const GTask t = tasks[blockIdx.x];
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const uint32_t b_full = (uint32_t)__cvta_generic_to_shared(&bars[0]);
  const uint32_t b_empty = (uint32_t)__cvta_generic_to_shared(&bars[GB_STAGES]);
  volatile int* abortp = &abort_flag;
  const int m = t.m;
  if (tid == 0) {
    for (int b = 0; b < GB_STAGES; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_full + 8u * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" :: "r"(b_empty + 8u * b));
    }
    abort_flag = 0;
    issued_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int e = tid; e < 256; e += GB_THREADS) {
    part[e] = make_double2(0.0, 0.0);
    rowsum[e] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (w == 8) {
    // ------------------------------------------------ copies (one thread)
    if (lane == 0) {
      int g = 0;
      bool stop = false;
      for (int it = t.it0; it < t.it1 && !stop; ++it) {
        const GItem I = items[it];
        int nrow, len;
        gb_rows(I, m, nrow, len);
        const int rb = len * 16;
        const int per = max(1, GB_CHUNK / rb);
        const unsigned char* A = (const unsigned char*)((const double2*)ab.p[I.a_buf] + I.a_off);
        const bool contig = I.lda == len;
        for (int r = 0; r < nrow; r += per) {
          const int nr = min(per, nrow - r);
          const int b = g % GB_STAGES;
          if (g >= GB_STAGES &&
              !gb_wait(b_empty + 8u * b, (uint32_t)(((g - GB_STAGES) / GB_STAGES) & 1), spin_limit,
                       abortp, err)) {
            stop = true;
            break;
          }
          const uint32_t fb = b_full + 8u * b;
          const uint32_t dst = (uint32_t)__cvta_generic_to_shared(gb_smem + b * GB_CHUNK);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                       :: "r"(fb), "r"(nr * rb) : "memory");
          if (contig) {
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                :: "r"(dst), "l"(A + (long long)r * rb), "r"(nr * rb), "r"(fb) : "memory");
          } else {
            for (int q = 0; q < nr; ++q)
              asm volatile(
                  "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                  :: "r"(dst + (uint32_t)(q * rb)), "l"(A + (long long)(r + q) * I.lda * 16),
                     "r"(rb), "r"(fb) : "memory");
          }
          ++g;
          issued_s = g;
        }
      }
    }
  } else {
    // ------------------------------------------------ consumers (8 warps)
    const int G = m > 0 ? max(1, 256 / m) : 1;
    const int grp = tid / max(1, m), row = tid % max(1, m);
    const bool t1 = m > 0 && grp < G;       // this thread owns (group, row) for trans = 1
    double2 acc1 = make_double2(0.0, 0.0);
    int g = 0;
    bool stop = false;
    for (int it = t.it0; it < t.it1 && !stop; ++it) {
      const GItem I = items[it];
      int nrow, len;
      gb_rows(I, m, nrow, len);
      const int per = max(1, GB_CHUNK / (len * 16));
      const TV* X = (const TV*)vb.p[I.in_buf] + I.in_row;
      for (int r = 0; r < nrow; r += per) {
        const int nr = min(per, nrow - r);
        const int b = g % GB_STAGES;
        // one decision per warp
        bool ok = true;
        if (lane == 0) ok = gb_wait(b_full + 8u * b, (uint32_t)((g / GB_STAGES) & 1), spin_limit,
                                    abortp, err);
        if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) {
          stop = true;
          break;
        }
        const double2* S = (const double2*)(gb_smem + b * GB_CHUNK);
        if (I.trans) {
          if (t1)
            for (int q = grp; q < nr; q += G) {
              const double2 a = S[q * len + row];
              cmac(acc1, a, cvt<double2, TV>(X[r + q]));
            }
        } else {
          for (int q = (w - r % 8 + 8) % 8; q < nr; q += 8) {   // rows i = r + q with i % 8 == w
            double2 v = make_double2(0.0, 0.0);
            for (int kk = lane; kk < len; kk += 32)
              cmac(v, S[q * len + kk], cvt<double2, TV>(X[kk]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
              v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (lane == 0) {
              double2& rs = rowsum[r + q];
              rs.x += v.x;
              rs.y += v.y;
            }
          }
        }
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b_empty + 8u * b) : "memory");
        ++g;
      }
    }
    if (t1) part[tid] = acc1;
  }
  __syncthreads();
  if (abort_flag) {
    // the copies still in flight (at most the last GB_STAGES issued, the
    // latest phase of each stage barrier) land before the CTA leaves
    if (tid == 0) {
      volatile int never = 0;
      const long long lim = spin_limit > (1LL << 24) ? spin_limit : (1LL << 24);
      for (int g = max(0, issued_s - GB_STAGES); g < issued_s; ++g)
        gb_wait(b_full + 8u * (g % GB_STAGES), (uint32_t)((g / GB_STAGES) & 1), lim, &never,
                nullptr);
    }
    __syncthreads();
    return;
  }
  if (tid < m) {
    const int G = max(1, 256 / m);
    double2 v = rowsum[tid];
    for (int q = 0; q < G; ++q) {
      const double2 p = part[q * m + tid];
      v.x += p.x;
      v.y += p.y;
    }
    if (t.mode == 1) {
      const double2 bv = cvt<double2, TV>(((const TV*)vb.p[t.base_buf])[t.base_row + tid]);
      v.x += bv.x;
      v.y += bv.y;
    }
    ((TV*)vb.p[t.out_buf])[t.out_row + tid] = cvt<TV, double2>(v);
  }
}

// Many-RHS variant: one CTA owns up to 128 rows of a target panel and a
// 32-column RHS slice.  Lane = RHS column, warp = row group (rows g, g+8, ...),
// so the inner dimension streams without row-tile padding: per inner index a
// column of op(A) (broadcast from shared memory) meets one row of the input
// panel (one value per lane).
constexpr int RK = 16;     // inner rows per staged chunk
constexpr int RR = 128;    // rows per pass
template <class TA, class TV, class TC>
__global__ void __launch_bounds__(256) k_gather_rows(const GTask* __restrict__ tasks,
                                                     const GItem* __restrict__ items, VBufs vb,
                                                     ABufs ab, int nrhs) {
  const GTask t = tasks[blockIdx.x];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int col = blockIdx.y * 32 + lane;
  __shared__ TC As[RK][RR + 1];
  __shared__ TC Xs[RK][32];
  constexpr int RPT = RR / 8;
  for (int r0 = 0; r0 < t.m; r0 += RR) {
    const int mr = min(RR, t.m - r0);
    TC acc[RPT];
#pragma unroll
    for (int i = 0; i < RPT; ++i) acc[i] = czero<TC>();
    for (int it = t.it0; it < t.it1; ++it) {
      const GItem I = items[it];
      const TA* A = (const TA*)ab.p[I.a_buf] + I.a_off;
      const TV* X = (const TV*)vb.p[I.in_buf] + (long long)I.in_row * nrhs;
      for (int k0 = 0; k0 < I.k; k0 += RK) {
        const int kc = min(RK, I.k - k0);
        // only the block's mr rows are staged (rows >= mr are never read); every
        // thread issues all of its loads before storing (one memory latency)
        {
          constexpr int EA = RR * RK / 256;     // 8
          TC av[EA];
#pragma unroll
          for (int q = 0; q < EA; ++q) {
            const int e = threadIdx.x + q * 256;
            int r, kk;
            if (!I.trans) { r = e / RK; kk = e % RK; } else { kk = e / mr; r = e % mr; }
            av[q] = (e < mr * RK && kk < kc)
                        ? cvt<TC, TA>(I.trans ? A[(long long)(k0 + kk) * I.lda + r0 + r]
                                              : A[(long long)(r0 + r) * I.lda + k0 + kk])
                        : czero<TC>();
          }
          constexpr int EX = RK * 32 / 256;     // 2
          TC xv[EX];
#pragma unroll
          for (int q = 0; q < EX; ++q) {
            const int e = threadIdx.x + q * 256;
            const int kk = e >> 5, c = e & 31;
            const int cc = blockIdx.y * 32 + c;
            xv[q] = (kk < kc && cc < nrhs) ? cvt<TC, TV>(X[(long long)(k0 + kk) * nrhs + cc])
                                           : czero<TC>();
          }
#pragma unroll
          for (int q = 0; q < EA; ++q) {
            const int e = threadIdx.x + q * 256;
            if (e < mr * RK) {
              int r, kk;
              if (!I.trans) { r = e / RK; kk = e % RK; } else { kk = e / mr; r = e % mr; }
              As[kk][r] = av[q];
            }
          }
#pragma unroll
          for (int q = 0; q < EX; ++q) {
            const int e = threadIdx.x + q * 256;
            Xs[e >> 5][e & 31] = xv[q];
          }
        }
        __syncthreads();
        // rows g, g+8, ... below mr only (warp-uniform bound: no divergence)
        const int nri = (mr - g + 7) >> 3;
        for (int kk = 0; kk < kc; ++kk) {
          TC x = Xs[kk][lane];
#pragma unroll
          for (int i = 0; i < RPT; ++i)
            if (i < nri) cmac(acc[i], As[kk][g + 8 * i], x);
        }
        __syncthreads();
      }
    }
    if (col < nrhs) {
      TV* out = (TV*)vb.p[t.out_buf] + (long long)(t.out_row + r0) * nrhs;
      const TV* base = (t.mode == 1)
                           ? (const TV*)vb.p[t.base_buf] + (long long)(t.base_row + r0) * nrhs
                           : nullptr;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        int r = g + 8 * i;
        if (r >= mr) continue;
        TC v = acc[i];
        if (base) {
          TC b = cvt<TC, TV>(base[(long long)r * nrhs + col]);
          v.x += b.x;
          v.y += b.y;
        }
        out[(long long)r * nrhs + col] = cvt<TV, TC>(v);
      }
    }
  }
}

template <class TV>
__global__ void k_finalize(const FTask* __restrict__ tasks, const int* __restrict__ slots,
                           VBufs vb, int nrhs) {
  const FTask t = tasks[blockIdx.x];
  const long long n = (long long)t.m * nrhs;
  TV* out = (TV*)vb.p[t.out_buf] + (long long)t.out_row * nrhs;
  const TV* base = (const TV*)vb.p[t.base_buf] + (long long)t.base_row * nrhs;
  const TV* scr = (const TV*)vb.p[VB_SCR];
  for (long long e = threadIdx.x + (long long)blockIdx.y * blockDim.x; e < n;
       e += (long long)blockDim.x * gridDim.y) {
    TV v = base[e];
    for (int s = t.s0; s < t.s1; ++s) {
      TV p = scr[(long long)slots[s] * nrhs + e];
      v.x += p.x;
      v.y += p.y;
    }
    out[e] = v;
  }
}

__global__ void k_gather_perm32(const cplx* __restrict__ B, float2* __restrict__ V,
                                const int* __restrict__ perm, int N, int nrhs) {
  long long n = (long long)N * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / nrhs), r = (int)(e % nrhs);
    cplx b = B[(long long)r * N + perm[i]];
    V[e] = make_float2((float)b.x, (float)b.y);
  }
}

__global__ void k_to32(const cplx* __restrict__ a, float2* __restrict__ o, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x)
    o[e] = make_float2((float)a[e].x, (float)a[e].y);
}

// o (FP64) = sa * o + sb * b (FP32 panel widened)
__global__ void k_axpby64_32(cplx* o, double sa, const float2* b, double sb, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    cplx x = o[e];
    float2 y = b[e];
    o[e] = make_double2(sa * x.x + sb * (double)y.x, sa * x.y + sb * (double)y.y);
  }
}

__global__ void k_axpby32(float2* out, const float2* a, float sa, const float2* b, float sb,
                          size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    float2 x = a[e], y = b[e];
    out[e] = make_float2(sa * x.x + sb * y.x, sa * x.y + sb * y.y);
  }
}

__global__ void k_col_norms2_32(const float2* __restrict__ V, int N, int nrhs, double* out) {
  __shared__ double red[256];
  int r = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    float2 v = V[(long long)i * nrhs + r];
    s += (double)v.x * v.x + (double)v.y * v.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[r] = red[0];
}

__global__ void k_gather_perm(const cplx* __restrict__ B, cplx* __restrict__ V,
                              const int* __restrict__ perm, int N, int nrhs) {
  long long n = (long long)N * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / nrhs), r = (int)(e % nrhs);
    V[e] = B[(long long)r * N + perm[i]];
  }
}

__global__ void k_scatter_perm(const cplx* __restrict__ V, cplx* __restrict__ X,
                               const int* __restrict__ perm, int N, int nrhs) {
  long long n = (long long)N * nrhs;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    int i = (int)(e / nrhs), r = (int)(e % nrhs);
    X[(long long)r * N + perm[i]] = V[e];
  }
}

__global__ void k_axpby(cplx* out, const cplx* a, double sa, const cplx* b, double sb, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    cplx x = a[e], y = b[e];
    out[e] = make_double2(sa * x.x + sb * y.x, sa * x.y + sb * y.y);
  }
}

// Squared 2-norm of each RHS column; one CTA per column, fixed-order tree
// reduction (deterministic).
__global__ void k_col_norms2(const cplx* __restrict__ V, int N, int nrhs, double* out) {
  __shared__ double red[256];
  int r = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    cplx v = V[(long long)i * nrhs + r];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[r] = red[0];
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

// The bulk-copy kernel takes a list whose items are all transposed blocks
// stored as whole contiguous rows (lda equal to the task's rows): every piece
// is then one copy of whole stored rows, and each thread walks its own row
// through shared memory.  Tasks of at most 256 rows, stored rows of at most
// GB_CHUNK bytes, no stacked tasks.  (Measured on the 2-lambda sphere: 1.2 to
// 1.6 TB/s on such launches, against 0.5 to 0.9 TB/s for k_gemv; lists with
// untransposed blocks ran faster on k_gemv, whose lanes read along the rows.)
static bool bulk_ok_for(const TaskList& tl) {
  if (tl.bulk_ok < 0) {
    bool ok = !tl.tasks.empty();
    for (const GTask& t : tl.tasks) {
      if (t.mode == 2 || t.m > 256 || t.m <= 0) { ok = false; break; }
      for (int q = t.it0; q < t.it1 && ok; ++q) {
        const GItem& I = tl.items[q];
        if (!I.trans || I.lda != t.m || t.m * 16 > GB_CHUNK) ok = false;
      }
      if (!ok) break;
    }
    tl.bulk_ok = ok ? 1 : 0;
  }
  return tl.bulk_ok == 1;
}

template <class TA, class TV, class TC>
static void launch_tl(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                      cudaStream_t s, long long spin_limit, int* err) {
  int nt = (int)tl.tasks.size();
  if (nrhs == 1) {
    if (std::is_same<TA, double2>::value && err && bulk_ok_for(tl))
      k_gemv_bulk<TV><<<nt, GB_THREADS, GB_SMEM, s>>>(tl.d_tasks, tl.d_items, vb, ab,
                                                       spin_limit, err);
    else
      k_gemv<TA, TV, TC><<<nt, 256, 0, s>>>(tl.d_tasks, tl.d_items, vb, ab);
  } else if (nrhs <= 4) {
    k_gather_gemm<4, TA, TV, TC><<<dim3(nt, 1), NTHR, 0, s>>>(tl.d_tasks, tl.d_items, vb, ab, nrhs);
  } else if (nrhs <= 8) {
    k_gather_gemm<8, TA, TV, TC><<<dim3(nt, 1), NTHR, 0, s>>>(tl.d_tasks, tl.d_items, vb, ab, nrhs);
  } else {
    k_gather_rows<TA, TV, TC><<<dim3(nt, (nrhs + 31) / 32), 256, 0, s>>>(tl.d_tasks, tl.d_items,
                                                                         vb, ab, nrhs);
  }
}

hm_status launch_tasks(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                       cudaStream_t s, int prec, long long spin_limit, int* err) {
  if (tl.tasks.empty()) return HM_OK;
  if (!abufs_bound(tl, ab)) return HM_ERR_STATE;
  static bool attr = false;
  if (!attr) {
    HM_CUDA(cudaFuncSetAttribute(k_gemv_bulk<double2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, GB_SMEM));
    HM_CUDA(cudaFuncSetAttribute(k_gemv_bulk<float2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, GB_SMEM));
    attr = true;
  }
  if (prec == PREC_64)
    launch_tl<double2, double2, double2>(tl, vb, ab, nrhs, s, spin_limit, err);
  else if (prec == PREC_32)
    launch_tl<float2, float2, float2>(tl, vb, ab, nrhs, s, spin_limit, err);
  else
    launch_tl<double2, float2, double2>(tl, vb, ab, nrhs, s, spin_limit, err);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_fin(const FinList& fl, const VBufs& vb, int nrhs, cudaStream_t s, int prec) {
  if (fl.tasks.empty()) return HM_OK;
  // about one element per thread: the slot reads of different elements are
  // independent, so a wide grid hides their latency on narrow levels
  int mmax = 1;
  for (const FTask& f : fl.tasks) mmax = f.m > mmax ? f.m : mmax;
  long long per_task = (long long)mmax * nrhs;
  int ny = (int)((per_task + 255) / 256);
  if (ny > 512) ny = 512;
  if (ny < 1) ny = 1;
  if (prec == PREC_64)
    k_finalize<double2><<<dim3((unsigned)fl.tasks.size(), ny), 256, 0, s>>>(fl.d_tasks, fl.d_slots,
                                                                            vb, nrhs);
  else
    k_finalize<float2><<<dim3((unsigned)fl.tasks.size(), ny), 256, 0, s>>>(fl.d_tasks, fl.d_slots,
                                                                           vb, nrhs);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_gather_perm32(const cplx* B, float2* V, const int* perm, int N, int nrhs,
                               cudaStream_t s) {
  k_gather_perm32<<<grid_for((long long)N * nrhs), 256, 0, s>>>(B, V, perm, N, nrhs);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_to32(const cplx* a, float2* o, size_t n, cudaStream_t s) {
  k_to32<<<grid_for((long long)n), 256, 0, s>>>(a, o, n);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_axpby64_32(cplx* o, double sa, const float2* b, double sb, size_t n,
                            cudaStream_t s) {
  k_axpby64_32<<<grid_for((long long)n), 256, 0, s>>>(o, sa, b, sb, n);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_axpby32(float2* out, const float2* a, float sa, const float2* b, float sb,
                         size_t n, cudaStream_t s) {
  k_axpby32<<<grid_for((long long)n), 256, 0, s>>>(out, a, sa, b, sb, n);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_col_norms2_32(const float2* V, int N, int nrhs, double* out, cudaStream_t s) {
  k_col_norms2_32<<<nrhs, 256, 0, s>>>(V, N, nrhs, out);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_gather_perm(const cplx* B, cplx* V, const int* perm, int N, int nrhs,
                             cudaStream_t s) {
  k_gather_perm<<<grid_for((long long)N * nrhs), 256, 0, s>>>(B, V, perm, N, nrhs);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_scatter_perm(const cplx* V, cplx* X, const int* perm, int N, int nrhs,
                              cudaStream_t s) {
  k_scatter_perm<<<grid_for((long long)N * nrhs), 256, 0, s>>>(V, X, perm, N, nrhs);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_axpby(cplx* out, const cplx* a, double sa, const cplx* b, double sb, size_t n,
                       cudaStream_t s) {
  k_axpby<<<grid_for((long long)n), 256, 0, s>>>(out, a, sa, b, sb, n);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_col_norms2(const cplx* V, int N, int nrhs, double* out, cudaStream_t s) {
  k_col_norms2<<<nrhs, 256, 0, s>>>(V, N, nrhs, out);
  HM_LAUNCHED();
  return HM_OK;
}

}  // namespace hm
