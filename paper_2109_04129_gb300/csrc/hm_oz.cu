// FP64-accurate complex gather GEMM on bf16 tensor cores (tcgen05), used for
// the FP64 residual r = b - (Z_N + Z_F) x of the refinement step.
//
// GB300 executes FP64 at about 1.1 TFLOP/s; the same products with FP64
// accuracy run here on the bf16 tensor cores by exact integer slicing
// (the error-free splitting idea of Ozaki et al.):
//   * every matrix row i of a task has a power-of-two scale 2^E_i > max |a_ik|
//     (precomputed), every right-hand side r a scale 2^F_r > max |x_kr| over
//     its panel (computed on the device before the launch);
//   * a value v with scale 2^S becomes the integer T = trunc(v 2^(55-S)),
//     |T| < 2^55, written with eight balanced base-128 digits
//     T = sum_p d_p 2^(7(7-p)), d_1..d_7 in [-64, 63] and d_0 in [-64, 64]
//     (sign of v applied): every digit is exact in bf16 and |d_p| <= 2^6;
//   * the slice products d^a_p d^x_q with level L = p + q <= 7 accumulate in
//     FP32 per level in tensor memory; a level holds at most 8 digit pairs of
//     magnitude <= 2^12, so over a window of at most 512 real inner terms
//     (256 complex rows) every partial sum is an integer of magnitude <= 2^24
//     and the FP32 accumulation is exact;
//   * after each window the levels are combined exactly in int64 (levels 0-3
//     and 4-7 in two words) and added to FP64 accumulators with the factor
//     2^(E_i + F_r - 110 + 7 (14 - L)).
// Dropped terms (L >= 8) and the truncated bits are below 2^-55 of the
// row/column scales times the inner length: FP64-class accuracy.
//
// Complex products use the real-expanded block (rows [a_re, -a_im] and
// [a_im, a_re] over interleaved inner k) as in the mixed-precision engine.
//
// The input panel is sliced once per product by k_digitize into eight digit
// planes that are already tiled like the MMA's shared-memory operand (8 RHS x
// 8 real inner core matrices of 128 bytes, 4-row groups contiguous), so a
// pipeline stage fetches its 128 RHS x 16 complex rows with 128 bulk copies
// of 512 bytes (cp.async.bulk, completion on an mbarrier) and no arithmetic.
// The matrix side (32 complex output rows x 16 inner rows per stage) is
// sliced on the fly from FP64, its loads issued one stage ahead.  A stage
// starts on a 4-row boundary of the panel (bulk copies need 16-byte aligned
// sources): the inner rows that the shift brings in before or after an item
// meet zero matrix digits and add exact zeros.
//
// One CTA = one task x 128 right-hand sides x 32 complex output rows; one
// thread issues the MMAs; every mbarrier wait is bounded and a failed wait is
// made uniform across the CTA before any decision that depends on it.  Two
// shared-memory stages alternate; a stage buffer is refilled only after the
// MMAs that read it have committed.
#include <cuda_bf16.h>

#include "hm_internal.h"

namespace hm {

namespace {

constexpr int OZ_M = 128;                 // RHS per CTA
constexpr int OZ_KC = 16;                 // complex inner rows per stage
constexpr int OZ_KR = 32;                 // real inner columns per stage
constexpr int OZ_NS = 8;                  // digits per value
constexpr int OZ_LV = 8;                  // levels kept (p + q <= 7)
constexpr int OZ_RC = 32;                 // complex output rows per CTA
constexpr int OZ_N = 64;                  // MMA N (2 * OZ_RC)
constexpr int OZ_WIN = 256;               // complex inner rows per exact window
constexpr int OZ_THREADS = 256;
constexpr int OZ_A_BYTES = OZ_M * OZ_KR * 2;      // one digit plane of X' (8 KB)
constexpr int OZ_B_BYTES = OZ_N * OZ_KR * 2;      // one digit plane of B' (4 KB)
constexpr int OZ_STAGE = OZ_NS * (OZ_A_BYTES + OZ_B_BYTES);   // one pipeline stage (96 KB)
constexpr int OZ_SMEM = 2 * OZ_STAGE + 1024;                      // double buffered
constexpr int OZ_COPY = 512;              // one bulk copy: 8 RHS x 16 complex rows, one plane
constexpr int OZ_COPIES = OZ_NS * (OZ_M / 8);                     // 128 per stage

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return ((row >> 3) * (OZ_KR >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(((OZ_KR / 8) * 128u >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
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

// Eight balanced base-128 digits of trunc(v 2^(55 - S)) for |v| < 2^S
// (integer operations only): d_1..d_7 in [-64, 63], d_0 in [0, 64], then the
// sign of v.
__device__ __forceinline__ void digits(double v, int S, __nv_bfloat16* d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  int e = (int)((b >> 52) & 0x7FF);
  unsigned long long U = 0;
  if (e != 0) {
    unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    int sh = e - 1020 - S;               // U = M 2^(e - 1075 + 55 - S)
    if (sh >= 0)
      U = (sh < 3) ? (M << sh) : 0ull;   // |v| < 2^S keeps sh < 3, U < 2^55
    else
      U = (-sh < 64) ? (M >> (-sh)) : 0ull;
  }
  const bool neg = (b >> 63) != 0;
  int carry = 0;
#pragma unroll
  for (int p = OZ_NS - 1; p >= 0; --p) {
    int s = (int)((U >> (49 - 7 * p)) & 0x7F) + carry;
    carry = 0;
    if (p > 0 && s >= 64) {
      s -= 128;
      carry = 1;
    }
    d[p] = __int2bfloat16_rn(neg ? -s : s);
  }
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ void put(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void put(float2* p, double2 v) {
  *p = make_float2((float)v.x, (float)v.y);
}

// byte offset of core matrix (plane p, RHS group g, 4-row group j) in a panel
__host__ __device__ __forceinline__ long long xd_off(int p, int G, long long g, long long J,
                                                     long long j) {
  return (((long long)p * G + g) * J + j) * 128;
}

// Digit panel of V (rows x nrhs, RHS fastest; complex128 or complex64 widened
// exactly): thread = (4-row group j, RHS r); for every plane it writes the
// 16-byte core-matrix row (re, im) of rows 4j..4j+3.  Rows >= rows and RHS >=
// nrhs get zero digits.
template <class TV>
__global__ void k_digitize(const TV* __restrict__ V, int rows, int nrhs,
                           const int* __restrict__ fexp, unsigned char* __restrict__ out,
                           long long J, int G) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int R8 = G * 8;
  if (idx >= J * R8) return;
  const int r = (int)(idx % R8);
  const long long j = idx / R8;
  const int F = r < nrhs ? fexp[r] : 0;
  double2 v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const long long row = 4 * j + c;
    v[c] = (row < rows && r < nrhs) ? to_d2(V[row * nrhs + r]) : make_double2(0.0, 0.0);
  }
  __nv_bfloat16 d[8][OZ_NS];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    digits(v[c].x, F, d[2 * c]);
    digits(v[c].y, F, d[2 * c + 1]);
  }
#pragma unroll
  for (int p = 0; p < OZ_NS; ++p) {
    uint4 w;
    w.x = pack2(d[0][p], d[1][p]);
    w.y = pack2(d[2][p], d[3][p]);
    w.z = pack2(d[4][p], d[5][p]);
    w.w = pack2(d[6][p], d[7][p]);
    *(uint4*)(out + xd_off(p, G, r >> 3, J, j) + (r & 7) * 16) = w;
  }
}

// TY: element type of the output (and base) panels
template <class TY>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gather(
    const GTask* __restrict__ tasks, const GItem* __restrict__ items, VBufs vb, ABufs ab,
    int nrhs, const int* __restrict__ task_row_exp, const long long* __restrict__ task_exp_off,
    const int* __restrict__ fexp_in, const int* __restrict__ fexp_far, OzPanels xp,
    long long spin_limit, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[4];   // [b]: MMAs of buffer b done; [2 + b]: its copies landed
  __shared__ uint32_t tmem_base;
  __shared__ int rexp[OZ_RC];
  const GTask t = tasks[blockIdx.x];
  const int rp = blockIdx.z * OZ_RC;                      // first complex row of this CTA
  if (rp >= t.m) return;                                  // whole CTA: uniform
  const int nr = min(OZ_RC, t.m - rp);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (OZ_M - 1);                       // RHS row (TMEM lane) of this thread
  const bool owner = tid < OZ_M;                          // warps 0-3 read TMEM, own acc
  const int col = blockIdx.y * OZ_M + row;                // this thread's RHS
  // MMA N: the rows of this CTA, rounded up to 16 (at least 32)
  const int n_real = max(32, ((2 * nr + 15) / 16) * 16);
  const uint32_t bar_done = smem_u32(&mbar[0]);
  const uint32_t bar_full = smem_u32(&mbar[2]);
  if (tid < OZ_RC) rexp[tid] = (tid < nr) ? task_row_exp[task_exp_off[blockIdx.x] + rp + tid] : 0;
  if (tid == 0) {
    for (int b = 0; b < 4; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_done + 8u * b));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n_real >> 3) << 17) |
                         ((uint32_t)(OZ_M >> 4) << 24);
  double acc[OZ_N];
#pragma unroll
  for (int c = 0; c < OZ_N; ++c) acc[c] = 0.0;
  uint32_t ph_done[2] = {0u, 0u}, ph_full[2] = {0u, 0u};
  bool outstanding[2] = {false, false};   // MMAs committed on buffer b, not yet waited for
  bool landing[2] = {false, false};       // copies issued into buffer b, not yet waited for
  int sidx = 0;                           // pipeline stage counter
  bool fail = false;        // this thread saw a wait run out (sticky)
  bool ok = true;           // no thread has: uniform, refreshed at every CTA barrier
  bool fresh = true;        // next MMA of each level starts a new window
  bool pending = false;     // the window holds products not yet added to acc
  int win = 0, cur_buf = -1, F = 0;

  // wait for the MMAs that read stage buffer b (bounded)
  auto wait_buf = [&](int b) {
    if (!outstanding[b]) return;
    if (!mbar_wait(bar_done + 8u * b, ph_done[b], spin_limit)) {
      fail = true;
      if (tid == 0) atomicExch(err, 1);
    }
    ph_done[b] ^= 1u;
    outstanding[b] = false;
  };

  auto flush = [&]() {
    wait_buf(0);              // every MMA of the window has completed
    wait_buf(1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    for (int c0 = 0; owner && c0 < n_real; c0 += 16) {
      long long hi[16], lo[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) { hi[j] = 0; lo[j] = 0; }
#pragma unroll
      for (int L = 0; L < OZ_LV; ++L) {
        uint32_t v[16];
        uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(L * OZ_N + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          long long iv = (long long)__float2int_rn(__uint_as_float(v[j]));   // exact integer
          if (L < 4)
            hi[j] += iv << (7 * (3 - L));
          else
            lo[j] += iv << (7 * (7 - L));
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int c = c0 + j;
        const int sc = rexp[c >> 1] + F - 14;
        acc[c] += ldexp((double)hi[j], sc - 19) + ldexp((double)lo[j], sc - 47);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = !__syncthreads_or(fail);   // TMEM reads done before the next window overwrites
    asm volatile("tcgen05.fence::after_thread_sync;");
    fresh = true;
    pending = false;
    win = 0;
  };

  // matrix values of stage st of item it (this thread's two elements)
  auto load_b = [&](int it, int st, double2* bv) {
    const GItem I = items[it];
    const double2* A = (const double2*)ab.p[I.a_buf] + I.a_off;
    const int dl = I.in_row & 3;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * OZ_THREADS;
      const int i = I.trans ? (e % OZ_RC) : (e / OZ_KC);
      const int kk = I.trans ? (e / OZ_RC) : (e % OZ_KC);
      const int kr = st * OZ_KC + kk - dl;                // inner row within the item
      bv[q] = make_double2(0.0, 0.0);
      if (i < nr && kr >= 0 && kr < I.k)
        bv[q] = I.trans ? A[(long long)kr * I.lda + rp + i] : A[(long long)(rp + i) * I.lda + kr];
    }
  };

  int it = t.it0, st = 0;
  double2 bv[2];
  if (it < t.it1) load_b(it, 0, bv);
  while (it < t.it1 && ok) {
    const GItem I = items[it];
    const int dl = I.in_row & 3;
    const int nst = (I.k + dl + OZ_KC - 1) / OZ_KC;
    const int xb = (I.in_buf == VB_FAR) ? 1 : 0;
    if (xb != cur_buf) {
      if (pending) flush();
      if (!ok) break;
      cur_buf = xb;
      const int* fe = xb ? fexp_far : fexp_in;
      F = (col < nrhs) ? fe[col] : 0;
    }
    if (pending && win + OZ_KC > OZ_WIN) {
      flush();
      if (!ok) break;
    }
    const int sb = sidx & 1;
    wait_buf(sb);             // the stage buffer is free once its previous MMAs committed
    unsigned char* sA = smem + sb * OZ_STAGE;                  // digit planes of X'
    unsigned char* sB = sA + OZ_NS * OZ_A_BYTES;               // digit planes of B'
    // ---- X' digits: bulk copies of the pre-sliced panel (warp 1)
    if (warp == 1) {
      const uint32_t fb = bar_full + 8u * sb;
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(fb), "r"(OZ_COPIES * OZ_COPY) : "memory");
      __syncwarp();
      const long long j0 = (long long)((I.in_row - dl) >> 2) + 4LL * st;
      const unsigned char* base = xp.xd[xb];
      for (int c = lane; c < OZ_COPIES; c += 32) {
        const int p = c >> 4, gl = c & 15;
        const unsigned char* src = base + xd_off(p, xp.G, (long long)blockIdx.y * 16 + gl,
                                                 xp.J[xb], j0);
        const uint32_t dst = smem_u32(sA + p * OZ_A_BYTES + gl * OZ_COPY);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            :: "r"(dst), "l"(src), "r"(OZ_COPY), "r"(fb) : "memory");
      }
    }
    landing[sb] = true;
    // ---- B' digits of the prefetched matrix values, packed (re, im) pairs
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int e = tid + q * OZ_THREADS;
      const int i = I.trans ? (e % OZ_RC) : (e / OZ_KC);
      const int kk = I.trans ? (e / OZ_RC) : (e % OZ_KC);
      __nv_bfloat16 ar[OZ_NS], ai[OZ_NS];
      digits(bv[q].x, rexp[i], ar);
      digits(bv[q].y, rexp[i], ai);
#pragma unroll
      for (int s = 0; s < OZ_NS; ++s) {
        unsigned char* bp = sB + s * OZ_B_BYTES;
        *(uint32_t*)(bp + kmaj(2 * i, 2 * kk)) = pack2(ar[s], __hneg(ai[s]));
        *(uint32_t*)(bp + kmaj(2 * i + 1, 2 * kk)) = pack2(ai[s], ar[s]);
      }
    }
    // ---- next stage and its matrix loads (in flight during this stage's MMAs)
    int it2 = it, st2 = st + 1;
    if (st2 >= nst) {
      it2 = it + 1;
      st2 = 0;
    }
    if (it2 < t.it1) load_b(it2, st2, bv);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = !__syncthreads_or(fail);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!ok) break;
    if (tid == 0) {
      if (!mbar_wait(bar_full + 8u * sb, ph_full[sb], spin_limit)) {
        fail = true;
        atomicExch(err, 1);
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        for (int p = 0; p < OZ_NS; ++p)
          for (int q = 0; p + q < OZ_LV; ++q) {
            const int L = p + q;
            for (int kh = 0; kh < OZ_KR / 16; ++kh) {
              uint64_t da = sdesc(smem_u32(sA + p * OZ_A_BYTES) + kh * 256);
              uint64_t db = sdesc(smem_u32(sB + q * OZ_B_BYTES) + kh * 256);
              // the first product of a level in a window overwrites the level
              // (levels are first reached in the p = 0 row of this loop)
              uint32_t accf = (fresh && p == 0 && kh == 0) ? 0u : 1u;
              asm volatile(
                  "{\n .reg .pred pp;\n setp.ne.b32 pp, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n"
                  :: "r"(tmem + (uint32_t)(L * OZ_N)), "l"(da), "l"(db), "r"(idesc), "r"(accf));
            }
          }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
            :: "r"(bar_done + 8u * sb));
      }
    }
    ph_full[sb] ^= 1u;
    landing[sb] = false;
    outstanding[sb] = true;
    ++sidx;
    fresh = false;
    pending = true;
    win += OZ_KC;
    it = it2;
    st = st2;
  }
  if (ok && pending) flush();
  wait_buf(0);                // nothing may still write tensor memory at release
  wait_buf(1);
  // copies issued but not consumed (a failed CTA): let them land (bounded)
  if (tid == 0 || warp == 1) {
    for (int b = 0; b < 2; ++b)
      if (landing[b] && !mbar_wait(bar_full + 8u * b, ph_full[b], spin_limit) && tid == 0)
        atomicExch(err, 1);
  }
  ok = !__syncthreads_or(fail);
  if (ok && owner && col < nrhs) {
    TY* out = (TY*)vb.p[t.out_buf] + (long long)(t.out_row + rp) * nrhs;
    const TY* base = (t.mode == 1) ? (const TY*)vb.p[t.base_buf] + (long long)(t.base_row + rp) * nrhs
                                   : nullptr;
    for (int i = 0; i < nr; ++i) {
      double2 y = make_double2(acc[2 * i], acc[2 * i + 1]);
      if (base) {
        double2 b = to_d2(base[(long long)i * nrhs + col]);
        y.x += b.x;
        y.y += b.y;
      }
      put(out + (long long)i * nrhs + col, y);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

__device__ __forceinline__ unsigned int bexp(double v) {
  return (unsigned int)((__double_as_longlong(v) >> 52) & 0x7FF);
}
// biased FP64 exponent of a float's value (0 for zero / subnormal floats)
__device__ __forceinline__ unsigned int bexp(float v) {
  unsigned int e = (__float_as_uint(v) >> 23) & 0xFF;
  return e == 0 ? 0u : e - 127u + 1023u;
}

// F_r = smallest S with max_k max(|re|, |im|) of panel column r < 2^S
template <class TV>
__global__ void k_col_exp(const TV* __restrict__ V, int rows, int nrhs, int* out) {
  __shared__ unsigned int red[256];
  const int r = blockIdx.x;
  unsigned int m = 0;      // max biased exponent seen
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    TV v = V[(long long)i * nrhs + r];
    m = max(m, max(bexp(v.x), bexp(v.y)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  // |v| < 2^(e - 1022) for biased exponent e (v = 1.f * 2^(e - 1023))
  if (threadIdx.x == 0) out[r] = red[0] == 0 ? -1022 : (int)red[0] - 1022;
}

}  // namespace

bool oz_ok_for(const TaskList& tl) { return !tl.tasks.empty(); }

int oz_max_passes(const TaskList& tl) {
  int mm = 1;
  for (const GTask& t : tl.tasks) mm = std::max(mm, t.m);
  return (mm + OZ_RC - 1) / OZ_RC;
}

hm_status launch_col_exp(const cplx* V, int rows, int nrhs, int* out, cudaStream_t s) {
  k_col_exp<double2><<<nrhs, 256, 0, s>>>(V, rows, nrhs, out);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

hm_status launch_col_exp32(const float2* V, int rows, int nrhs, int* out, cudaStream_t s) {
  k_col_exp<float2><<<nrhs, 256, 0, s>>>(V, rows, nrhs, out);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

long long oz_row_groups(int rows) { return (long long)rows / 4 + 5; }

int oz_rhs_groups(int nrhs) { return ((nrhs + OZ_M - 1) / OZ_M) * (OZ_M / 8); }

size_t oz_panel_bytes(int rows, int nrhs) {
  return (size_t)OZ_NS * oz_rhs_groups(nrhs) * oz_row_groups(rows) * 128;
}

hm_status launch_digitize(const void* V, bool f32, int rows, int nrhs, const int* fexp,
                          unsigned char* out, long long J, int G, cudaStream_t s) {
  const long long n = J * G * 8;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (f32)
    k_digitize<float2><<<blocks, 256, 0, s>>>((const float2*)V, rows, nrhs, fexp, out, J, G);
  else
    k_digitize<double2><<<blocks, 256, 0, s>>>((const double2*)V, rows, nrhs, fexp, out, J, G);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

hm_status launch_tasks_oz(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, const int* row_exp, const long long* exp_off,
                          const int* fexp_in, const int* fexp_far, const OzPanels& xp,
                          long long spin_limit, int* err, bool panels32) {
  if (tl.tasks.empty()) return HM_OK;
  if (xp.G * 8 < nrhs) return HM_ERR_INVALID;
  static bool attr = false;
  if (!attr) {
    HM_CUDA(cudaFuncSetAttribute(k_oz_gather<double2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    HM_CUDA(cudaFuncSetAttribute(k_oz_gather<float2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    attr = true;
  }
  dim3 grid((unsigned)tl.tasks.size(), (unsigned)((nrhs + OZ_M - 1) / OZ_M),
            (unsigned)oz_max_passes(tl));
  if (panels32)
    k_oz_gather<float2><<<grid, OZ_THREADS, OZ_SMEM, s>>>(
        tl.d_tasks, tl.d_items, vb, ab, nrhs, row_exp, exp_off, fexp_in, fexp_far, xp,
        spin_limit, err);
  else
    k_oz_gather<double2><<<grid, OZ_THREADS, OZ_SMEM, s>>>(
        tl.d_tasks, tl.d_items, vb, ab, nrhs, row_exp, exp_off, fexp_in, fexp_far, xp,
        spin_limit, err);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

}  // namespace hm
