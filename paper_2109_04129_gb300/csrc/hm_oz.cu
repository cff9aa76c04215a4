// FP64-accurate complex gather GEMM on bf16 tensor cores (tcgen05), used for
// the FP64 residual r = b - (Z_N + Z_F) x of the refinement step.
//
// GB300 executes FP64 at about 1.1 TFLOP/s; the same products with FP64
// accuracy run here on the bf16 tensor cores by exact integer slicing
// (the error-free splitting idea of Ozaki et al.):
//   * every matrix row i of a task has a power-of-two scale 2^E_i >= max |a_ik|
//     (precomputed), every right-hand side r a scale 2^F_r >= max |x_kr| over
//     its panel (computed on the device before the launch);
//   * a value v with scale 2^S becomes the integer T = trunc(v 2^(56-S)),
//     |T| < 2^56, cut into eight 7-bit digits s_0..s_7 (bits 55..49, ..., 6..0)
//     with the sign of v: every digit is an integer in [-127, 127], exact in
//     bf16, and v = sum_p s_p 2^(7(7-p)) 2^(S-56) up to the truncated bits;
//   * the slice products s^a_p s^x_q with level L = p + q <= 7 accumulate in
//     FP32 per level in tensor memory; each product is an integer below 2^14,
//     so a level sum over at most 1024 real inner terms is an integer below
//     2^24 and is exact in FP32;
//   * after each window of at most 512 complex inner terms the levels are
//     combined exactly in int64 (levels 0-3 and 4-7 in two words) and added to
//     FP64 accumulators with the factor 2^(E_i + F_r - 14 - 7L).
// Dropped terms (L >= 8) and the truncated bits are below 2^-56 of the
// row/column scales times the inner length: FP64-class accuracy.
//
// Complex products use the real-expanded block (rows [a_re, -a_im] and
// [a_im, a_re] over interleaved inner k) as in the mixed-precision engine.
// One CTA = one task x 128 right-hand sides x 32 complex output rows; one
// thread issues the MMAs; every mbarrier wait is bounded.  Two shared-memory
// stages alternate: the digits of stage s + 1 are computed while the tensor
// cores work on stage s; a stage buffer is refilled only after the MMAs that
// read it have committed.
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
constexpr int OZ_WIN = 512;               // complex inner rows per exact window
constexpr int OZ_THREADS = 256;          // two halves share the digit staging
constexpr int OZ_A_BYTES = OZ_M * OZ_KR * 2;      // one digit plane of X' (8 KB)
constexpr int OZ_B_BYTES = OZ_N * OZ_KR * 2;      // one digit plane of B' (4 KB)
constexpr int OZ_STAGE = OZ_NS * (OZ_A_BYTES + OZ_B_BYTES);   // one pipeline stage (96 KB)
constexpr int OZ_SMEM = 2 * OZ_STAGE + 1024;                      // double buffered

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

// Eight signed 7-bit digits of trunc(v 2^(56 - S)) (integer operations only).
__device__ __forceinline__ void digits(double v, int S, __nv_bfloat16* d) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  int e = (int)((b >> 52) & 0x7FF);
  unsigned long long T = 0;
  if (e != 0) {
    unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    int sh = e - 1019 - S;               // T = M 2^(e - 1075 + 56 - S)
    if (sh >= 0)
      T = (sh < 4) ? (M << sh) : 0ull;   // |v| < 2^S keeps sh < 4
    else
      T = (-sh < 64) ? (M >> (-sh)) : 0ull;
  }
  const bool neg = (b >> 63) != 0;
#pragma unroll
  for (int p = 0; p < OZ_NS; ++p) {
    int s = (int)((T >> (49 - 7 * p)) & 0x7F);
    d[p] = __int2bfloat16_rn(neg ? -s : s);
  }
}

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ void put(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void put(float2* p, double2 v) {
  *p = make_float2((float)v.x, (float)v.y);
}

// TX / TY: element type of the input / output panels (complex128 or complex64;
// complex64 inputs are widened exactly before slicing)
template <class TX, class TY>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gather(
    const GTask* __restrict__ tasks, const GItem* __restrict__ items, VBufs vb, ABufs ab,
    int nrhs, const int* __restrict__ task_row_exp, const long long* __restrict__ task_exp_off,
    const int* __restrict__ fexp_in, const int* __restrict__ fexp_far, long long spin_limit,
    int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int rexp[OZ_RC];
  const GTask t = tasks[blockIdx.x];
  const int rp = blockIdx.z * OZ_RC;                      // first complex row of this CTA
  if (rp >= t.m) return;                                  // whole CTA: uniform
  const int nr = min(OZ_RC, t.m - rp);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (OZ_M - 1);                       // RHS row (TMEM lane) of this thread
  const int half = tid >> 7;                              // staging half (inner rows)
  const bool owner = half == 0;                           // warps 0-3 read TMEM, own acc
  const int col = blockIdx.y * OZ_M + row;                // this thread's RHS
  // MMA N: the rows of this CTA, rounded up to 16 (at least 32)
  const int n_real = max(32, ((2 * nr + 15) / 16) * 16);
  const uint32_t bar0 = smem_u32(&mbar[0]);
  if (tid < OZ_RC) rexp[tid] = (tid < nr) ? task_row_exp[task_exp_off[blockIdx.x] + rp + tid] : 0;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar0));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar0 + 8));
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
  uint32_t ph[2] = {0u, 0u};
  bool outstanding[2] = {false, false};   // a committed stage not yet waited for
  int sidx = 0;                           // pipeline stage counter
  bool ok = true;
  bool fresh = true;        // next MMA of each level starts a new window
  bool pending = false;     // the window holds products not yet added to acc
  int win = 0, cur_buf = -1, F = 0;

  // wait for the MMAs that read stage buffer b (bounded)
  auto wait_buf = [&](int b) {
    if (!outstanding[b]) return;
    if (!mbar_wait(bar0 + 8u * b, ph[b], spin_limit)) {
      ok = false;
      if (tid == 0) atomicExch(err, 1);
    }
    ph[b] ^= 1u;
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
        acc[c] += ldexp((double)hi[j], sc - 21) + ldexp((double)lo[j], sc - 49);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();          // TMEM reads done before the next window overwrites
    asm volatile("tcgen05.fence::after_thread_sync;");
    fresh = true;
    pending = false;
    win = 0;
  };

  for (int it = t.it0; it < t.it1 && ok; ++it) {
    const GItem I = items[it];
    if (I.in_buf != cur_buf) {
      if (pending) flush();
      cur_buf = I.in_buf;
      const int* fe = (I.in_buf == VB_FAR) ? fexp_far : fexp_in;
      F = (col < nrhs) ? fe[col] : 0;
    }
    const double2* A = (const double2*)ab.p[I.a_buf] + I.a_off;
    const TX* X = (const TX*)vb.p[I.in_buf] + (long long)I.in_row * nrhs;
    for (int k0 = 0; k0 < I.k && ok; k0 += OZ_KC) {
      const int kc = min(OZ_KC, I.k - k0);
      if (pending && win + kc > OZ_WIN) flush();
      const int sb = sidx & 1;
      wait_buf(sb);           // the stage buffer is free once its previous MMAs committed
      unsigned char* sA = smem + sb * OZ_STAGE;                  // digit planes of X'
      unsigned char* sB = sA + OZ_NS * OZ_A_BYTES;               // digit planes of B'
      // ---- X' digits: thread = RHS row, the two halves split the inner rows;
      // all loads of the thread are issued before any use (one memory latency)
      {
        constexpr int KH = OZ_KC / 2;
        double2 xv[KH];
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int kk = half * KH + j;
          xv[j] = (kk < kc && col < nrhs) ? to_d2(X[(long long)(k0 + kk) * nrhs + col])
                                          : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int j = 0; j < KH; ++j) {
          const int kk = half * KH + j;
          __nv_bfloat16 dr[OZ_NS], di[OZ_NS];
          digits(xv[j].x, F, dr);
          digits(xv[j].y, F, di);
#pragma unroll
          for (int s = 0; s < OZ_NS; ++s) {
            *(__nv_bfloat16*)(sA + s * OZ_A_BYTES + kmaj(row, 2 * kk)) = dr[s];
            *(__nv_bfloat16*)(sA + s * OZ_A_BYTES + kmaj(row, 2 * kk + 1)) = di[s];
          }
        }
      }
      // ---- B' digits: element (i, kk) of op(A), rows rp + i; loads first
      {
        constexpr int EMAX = OZ_RC * OZ_KC / OZ_THREADS;     // 2
        double2 av[EMAX];
#pragma unroll
        for (int q = 0; q < EMAX; ++q) {
          const int e = tid + q * OZ_THREADS;
          int i, kk;
          if (I.trans) {
            kk = e / OZ_RC;
            i = e % OZ_RC;
          } else {
            i = e / OZ_KC;
            kk = e % OZ_KC;
          }
          av[q] = make_double2(0.0, 0.0);
          if (i < nr && kk < kc)
            av[q] = I.trans ? A[(long long)(k0 + kk) * I.lda + rp + i]
                            : A[(long long)(rp + i) * I.lda + k0 + kk];
        }
#pragma unroll
        for (int q = 0; q < EMAX; ++q) {
          const int e = tid + q * OZ_THREADS;
          int i, kk;
          if (I.trans) {
            kk = e / OZ_RC;
            i = e % OZ_RC;
          } else {
            i = e / OZ_KC;
            kk = e % OZ_KC;
          }
          __nv_bfloat16 ar[OZ_NS], ai[OZ_NS];
          digits(av[q].x, rexp[i], ar);
          digits(av[q].y, rexp[i], ai);
#pragma unroll
          for (int s = 0; s < OZ_NS; ++s) {
            unsigned char* bp = sB + s * OZ_B_BYTES;
            *(__nv_bfloat16*)(bp + kmaj(2 * i, 2 * kk)) = ar[s];
            *(__nv_bfloat16*)(bp + kmaj(2 * i, 2 * kk + 1)) = __hneg(ai[s]);
            *(__nv_bfloat16*)(bp + kmaj(2 * i + 1, 2 * kk)) = ai[s];
            *(__nv_bfloat16*)(bp + kmaj(2 * i + 1, 2 * kk + 1)) = ar[s];
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
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
            :: "r"(bar0 + 8u * sb));
      }
      outstanding[sb] = true;
      ++sidx;
      fresh = false;
      pending = true;
      win += kc;
    }
  }
  if (ok && pending) flush();
  wait_buf(0);                // nothing may still write tensor memory at release
  wait_buf(1);
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

hm_status launch_tasks_oz(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, const int* row_exp, const long long* exp_off,
                          const int* fexp_in, const int* fexp_far, long long spin_limit,
                          int* err, bool panels32) {
  if (tl.tasks.empty()) return HM_OK;
  static bool attr = false;
  if (!attr) {
    HM_CUDA(cudaFuncSetAttribute(k_oz_gather<double2, double2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    HM_CUDA(cudaFuncSetAttribute(k_oz_gather<float2, float2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    attr = true;
  }
  dim3 grid((unsigned)tl.tasks.size(), (unsigned)((nrhs + OZ_M - 1) / OZ_M),
            (unsigned)oz_max_passes(tl));
  if (panels32)
    k_oz_gather<float2, float2><<<grid, OZ_THREADS, OZ_SMEM, s>>>(
        tl.d_tasks, tl.d_items, vb, ab, nrhs, row_exp, exp_off, fexp_in, fexp_far, spin_limit, err);
  else
    k_oz_gather<double2, double2><<<grid, OZ_THREADS, OZ_SMEM, s>>>(
        tl.d_tasks, tl.d_items, vb, ab, nrhs, row_exp, exp_off, fexp_in, fexp_far, spin_limit, err);
  HM_CUDA(cudaGetLastError());
  return HM_OK;
}

}  // namespace hm
