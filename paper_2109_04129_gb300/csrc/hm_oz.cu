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
//     and 4-7 in two words, weights 2^(E_i + F_r - 110 + 7 (14 - L))), the two
//     words into one (bits below 2^-49 of the row and column scales dropped),
//     and that word is added to an FP64 accumulator with one fused
//     multiply-add.
// Dropped terms (L >= 8) and the truncated bits are below 2^-52.5 of the
// row/column scales per real product term (two per complex inner row), plus
// 2^-49 of the scales per window and the FP64 rounding of each window's sum:
// FP64-class accuracy.
//
// Complex products use the real-expanded block (rows [a_re, -a_im] and
// [a_im, a_re] over interleaved inner k) as in the mixed-precision engine.
//
// Data movement.  The input panel is sliced once per product by k_digitize
// into eight digit planes tiled so that the operand of one pipeline stage
// (128 right-hand sides x 8 complex inner rows of one plane) is one
// contiguous 4 KB block in the MMA's shared-memory layout: a stage arrives
// with eight bulk copies (cp.async.bulk, completion on an mbarrier).  The
// matrix side (32 complex output rows x 8 inner rows per stage) is sliced on
// the fly from FP64.  A stage starts on a 4-row boundary of the panel (bulk
// copies need 16-byte aligned sources): the inner rows the shift brings in
// meet zero matrix digits and add exact zeros.
//
// Kernel organisation (persistent, warp-specialised, one CTA per SM, 12
// warps).  A work unit is (task, 32-row pass); each CTA walks its share of the
// units (costliest first, or in list order for the leaf lists) for one tile of
// 128 right-hand sides.  Warp 1 issues the bulk copies; warps 2-3 and 8-11
// slice the matrix digits; warp 0 (one thread) issues the MMAs of a stage
// (the matrix digit planes are stacked along N and the levels spaced by the
// same width, so one MMA per input plane adds all of its digit products into
// their levels: 8 to 12 MMAs for the 36 products); warps 4-7 read the level
// accumulators out of tensor memory and keep the FP64 sums in shared memory.
// A stacked task (mode 2) is one operator made of row segments that share
// the input rows.  The roles hand over through mbarriers: a ring of
// three shared-memory stages (full: copies landed; digits: matrix digits
// written; empty: the MMAs that read it completed) and the tensor-memory
// window (full: the window's MMAs completed; empty: the epilogue has read it).
// Every wait is bounded and watches a CTA-wide abort flag; a CTA that gives up
// records it in *err, lets its copies and MMAs finish (bounded, with a limit
// of its own) and releases tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "hm_internal.h"

namespace hm {

namespace {

constexpr int OZ_M = 128;                 // RHS per CTA tile (MMA M)
constexpr int OZ_KC = 8;                  // complex inner rows per stage
constexpr int OZ_KR = 16;                 // real inner columns per stage (one MMA K)
constexpr int OZ_NS = 8;                  // digits per value
constexpr int OZ_LV = 8;                  // levels kept (p + q <= 7)
constexpr int OZ_RC = 32;                 // complex output rows per unit
constexpr int OZ_N = 64;                  // MMA N columns reserved per level (2 * OZ_RC)
constexpr int OZ_WIN = 256;               // complex inner rows per exact window
constexpr int OZ_THREADS = 384;          // 12 warps
constexpr int OZ_RING = 3;                // shared-memory stages
constexpr int OZ_BPROD = 192;             // matrix-digit producer threads (warps 2-3, 8-11)
constexpr int OZ_A_BYTES = OZ_M * OZ_KR * 2;      // one digit plane of X' (4 KB)
constexpr int OZ_B_BYTES = OZ_N * OZ_KR * 2;      // one digit plane of B' (2 KB)
constexpr int OZ_STAGE = OZ_NS * (OZ_A_BYTES + OZ_B_BYTES);   // 48 KB
constexpr int OZ_ACC_BYTES = OZ_N * OZ_M * 8;   // FP64 sums of the epilogue, [column][RHS row]
constexpr int OZ_SMEM = OZ_RING * OZ_STAGE + OZ_ACC_BYTES + 1024;
constexpr int OZ_GROUP = 16 * 128;       // one 4-row group of a 128-RHS tile, one plane (2 KB)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// B' (matrix) tile: canonical K-major, 8-row groups of (OZ_KR / 8) core matrices
__device__ __forceinline__ uint32_t kmaj_b(int row, int k) {
  return ((row >> 3) * (OZ_KR >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// element (i, kk) of the 32 x 8 matrix tile handled by producer slot e: a
// warp's 32 lanes cover 4 rows x 8 inner rows, so both the global loads
// (4 consecutive rows, or 8 consecutive inner rows) and the shared stores
// stay compact
__device__ __forceinline__ void oz_elem(int e, int trans, int& i, int& kk) {
  const int lane = e & 31, grp = e >> 5;
  if (trans) {
    i = 4 * grp + (lane & 3);
    kk = lane >> 2;
  } else {
    i = 4 * grp + (lane >> 3);
    kk = lane & 7;
  }
}
// shared-memory matrix descriptor (no swizzle): lbo = byte distance of
// K-adjacent core matrices, sbo = byte distance of adjacent 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// bounded wait that also gives up when another role has aborted the CTA
__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t phase, long long limit,
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
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

// Eight balanced base-128 digits of trunc(v 2^(55 - S)) for |v| < 2^S
// (integer operations only): d_1..d_7 in [-64, 63], d_0 in [0, 64], then the
// sign of v.  Adding 64 to each of the seven low base-128 positions turns the
// balanced digits into plain 7-bit fields (the additions carry exactly as the
// balanced representation needs): d_p = field_p - 64, d_0 = the bits above.
constexpr unsigned long long OZ_BIAS = 0x1020408102040ull;   // sum of 64 * 128^m, m = 0..6
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
  const unsigned long long V = U + OZ_BIAS;
  const int sg = (b >> 63) ? -1 : 1;
  d[0] = __int2bfloat16_rn(sg * (int)(V >> 49));
#pragma unroll
  for (int p = 1; p < OZ_NS; ++p)
    d[p] = __int2bfloat16_rn(sg * ((int)((V >> (49 - 7 * p)) & 0x7F) - 64));
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
// 2^e as a double (exact; ldexp outside the normal range)
__device__ __forceinline__ double pow2i(int e) {
  return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52)
                                   : ldexp(1.0, e);
}

// byte offset of the 16-byte row (plane p, 128-RHS tile y, 4-row group j,
// 8-RHS group gl, RHS r8 within it) of a digit panel with Y tiles and J groups
__host__ __device__ __forceinline__ long long xd_off(int p, int Y, int y, long long J, long long j,
                                                     int gl, int r8) {
  return ((((long long)p * Y + y) * J + j) * 16 + gl) * 128 + r8 * 16;
}

// stages of an item: 8-row stages from the 4-row boundary below its first row
__host__ __device__ __forceinline__ int oz_nst(const GItem& I) {
  return (I.k + (I.in_row & 3) + OZ_KC - 1) / OZ_KC;
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
  const int Y = G / 16;
#pragma unroll
  for (int p = 0; p < OZ_NS; ++p) {
    uint4 w;
    w.x = pack2(d[0][p], d[1][p]);
    w.y = pack2(d[2][p], d[3][p]);
    w.z = pack2(d[4][p], d[5][p]);
    w.w = pack2(d[6][p], d[7][p]);
    *(uint4*)(out + xd_off(p, Y, r >> 7, J, j, (r >> 3) & 15, r & 7)) = w;
  }
}

// TY: element type of the output (and base) panels
template <class TY>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gather(
    const GTask* __restrict__ tasks, const GItem* __restrict__ items,
    const int2* __restrict__ units, int n_units, VBufs vb, ABufs ab, int nrhs,
    const int* __restrict__ task_row_exp, const long long* __restrict__ task_exp_off,
    const int* __restrict__ fexp_in, const int* __restrict__ fexp_far, OzPanels xp,
    long long spin_limit, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t bars[3 * OZ_RING + 5];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int armed_s, consumed_s;     // stages armed by the copy warp / taken by the MMA warp
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b_full = smem_u32(&bars[0]);             // + 8 b: copies of stage b landed
  const uint32_t b_digs = smem_u32(&bars[OZ_RING]);       // + 8 b: matrix digits of b written
  const uint32_t b_empty = smem_u32(&bars[2 * OZ_RING]);  // + 8 b: MMAs reading b completed
  const uint32_t b_tfull = smem_u32(&bars[3 * OZ_RING]);
  const uint32_t b_tempty = b_tfull + 16;                 // + 8 (w & 1)
  const uint32_t b_fin = b_tfull + 32;
  volatile int* abortp = &abort_flag;
  const int y = blockIdx.y;
  const int Y = xp.G / 16;
  if (tid == 0) {
    for (int b = 0; b < OZ_RING; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_full + 8u * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(b_digs + 8u * b),
                   "r"(OZ_BPROD));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_empty + 8u * b));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_tfull + 8u * b));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(b_tempty + 8u * b), "r"(OZ_M));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b_fin));
    abort_flag = 0;
    armed_s = 0;
    consumed_s = 0;
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

  if (warp == 0) {
    // ------------------------------------------------ MMA issuer (one thread)
    // Tensor memory holds the 8 level accumulators of a window: a narrow unit
    // (N = 32 columns per level) uses one half (window w in half w & 1, so the
    // epilogue drains one window while the next one accumulates), a wide unit
    // (N = 64) uses all 512 columns.  Before window w the columns it writes
    // must have been drained: window w - 2 always, window w - 1 as well when
    // either of the two is wide.  Window w completes tfull[w & 1]; its drain
    // completes tempty[w & 1] (the waited window is always the latest one of
    // its parity, so a parity wait cannot alias).
    if (lane == 0) {
      int g = 0, w = 0;
      bool stop = false, prev_wide = false;
      for (int u = blockIdx.x; u < n_units && !stop; u += gridDim.x) {
        const int2 U = units[u];
        const GTask t = tasks[U.x];
        const int nr = min(OZ_RC, t.m - U.y * OZ_RC);
        const int n_real = max(32, ((2 * nr + 15) / 16) * 16);
        const bool wide = n_real > 32;
        // instruction descriptor without N (bf16 x bf16 -> f32, K-major, M = 128)
        const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_M >> 4) << 24);
        const int cmax = 256 / n_real;          // B' planes per MMA (N <= 256)
        const uint32_t pb = (uint32_t)n_real * (OZ_KR * 2);   // bytes of one B' plane
        bool open = false;
        int win = 0, cur = -1;
        uint32_t cbase = 0;
        for (int it = t.it0; it < task_it_end(t) && !stop; ++it) {
          const GItem I = items[it];
          const int nst = oz_nst(I);
          const int xb = (I.in_buf == VB_FAR) ? 1 : 0;
          for (int st = 0; st < nst && !stop; ++st) {
            const bool start = !open || xb != cur || win + OZ_KC > OZ_WIN;
            if (start) {
              if (open) {           // the previous window of this unit is complete
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                    :: "r"(b_tfull + 8u * (w & 1)));
                prev_wide = wide;
                ++w;
              }
              const int need = (wide || prev_wide) ? w - 1 : w - 2;   // drained before window w
              if (need >= 0 && !oz_wait(b_tempty + 8u * (need & 1), (uint32_t)((need >> 1) & 1),
                                        spin_limit, abortp, err)) {
                stop = true;
                break;
              }
              open = true;
              win = 0;
              cur = xb;
              cbase = wide ? 0u : (uint32_t)(w & 1) * 256u;
            }
            const int b = g % OZ_RING;
            if (!oz_wait(b_full + 8u * b, (uint32_t)((g / OZ_RING) & 1), spin_limit, abortp, err)) {
              stop = true;
              break;
            }
            consumed_s = g + 1;
            if (!oz_wait(b_digs + 8u * b, (uint32_t)((g / OZ_RING) & 1), spin_limit, abortp, err)) {
              stop = true;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            unsigned char* sA = smem + b * OZ_STAGE;
            // descriptors of plane 0; plane p is p * plane-bytes / 16 further in the
            // address field (all shared addresses stay below 256 KB: no carry)
            const uint64_t da0 = sdesc(smem_u32(sA), OZ_GROUP, 128);
            const uint64_t db0 = sdesc(smem_u32(sA + OZ_NS * OZ_A_BYTES), 128, (OZ_KR / 8) * 128);
            const uint32_t acc0 = start ? 0u : 1u;
            // The B' planes q = 0..7 are stacked along N and level L sits at
            // columns L * n_real, so one MMA of A' plane p against planes
            // q0 .. q0 + cnt - 1 (N = cnt * n_real) adds each product d_p d_q
            // into its level p + q: 8 to 12 MMAs per stage instead of 36.
#pragma unroll
            for (int p = 0; p < OZ_NS; ++p) {
              const uint64_t da = da0 + (uint64_t)(p * (OZ_A_BYTES >> 4));
              // every level is first reached by the p = 0 MMAs: they overwrite
              const uint32_t accf = p == 0 ? acc0 : 1u;
              for (int q0 = 0; q0 < OZ_LV - p; q0 += cmax) {
                const int cnt = min(cmax, OZ_LV - p - q0);
                const uint32_t idesc = idesc0 | ((uint32_t)((cnt * n_real) >> 3) << 17);
                const uint64_t db = db0 + (uint64_t)((q0 * pb) >> 4);
                asm volatile(
                    "{\n .reg .pred pp;\n setp.ne.b32 pp, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}\n"
                    :: "r"(tmem + cbase + (uint32_t)((p + q0) * n_real)), "l"(da), "l"(db),
                       "r"(idesc), "r"(accf));
              }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                :: "r"(b_empty + 8u * b));
            ++g;
            win += OZ_KC;
          }
        }
        if (open && !stop) {
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
              :: "r"(b_tfull + 8u * (w & 1)));
          prev_wide = wide;
          ++w;
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------ digit-panel copies
    int g = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < n_units && !stop; u += gridDim.x) {
      const GTask t = tasks[units[u].x];
      for (int it = t.it0; it < task_it_end(t) && !stop; ++it) {
        const GItem I = items[it];
        const int nst = oz_nst(I);
        const int xb = (I.in_buf == VB_FAR) ? 1 : 0;
        const long long j00 = (long long)((I.in_row - (I.in_row & 3)) >> 2);
        for (int st = 0; st < nst; ++st) {
          const int b = g % OZ_RING;
          // lane 0 waits for the stage buffer; the warp follows its decision
          bool okw = true;
          if (lane == 0 && g >= OZ_RING)
            okw = oz_wait(b_empty + 8u * b, (uint32_t)(((g - OZ_RING) / OZ_RING) & 1), spin_limit,
                          abortp, err);
          if (!__shfl_sync(0xffffffffu, okw ? 1 : 0, 0)) {
            stop = true;
            break;
          }
          const uint32_t fb = b_full + 8u * b;
          if (lane == 0)
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                         :: "r"(fb), "r"(OZ_NS * OZ_A_BYTES) : "memory");
          __syncwarp();
          if (lane < OZ_NS) {
            const long long j0 = j00 + 2LL * st;
            const unsigned char* src = xp.xd[xb] + xd_off(lane, Y, y, xp.J[xb], j0, 0, 0);
            const uint32_t dst = smem_u32(smem + b * OZ_STAGE + lane * OZ_A_BYTES);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                :: "r"(dst), "l"(src), "r"(OZ_A_BYTES), "r"(fb) : "memory");
          }
          ++g;
          if (lane == 0) armed_s = g;
        }
      }
    }
  } else if (warp < 4 || warp >= 8) {
    // ------------------------------------------------ matrix digits (192 threads)
    const int t2 = warp < 4 ? tid - 64 : tid - 192;      // 0..63, 64..191
    int g = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < n_units && !stop; u += gridDim.x) {
      const int2 U = units[u];
      const GTask t = tasks[U.x];
      const int rp = U.y * OZ_RC;
      const int nr = min(OZ_RC, t.m - rp);
      const int* rexp = task_row_exp + task_exp_off[U.x] + rp;
      // the unit's B' planes are n_real rows each, stacked back to back
      const int n_real = max(32, ((2 * nr + 15) / 16) * 16);
      const int ne = (n_real / 2) * OZ_KC;                 // elements of one plane
      const uint32_t pb = (uint32_t)n_real * (OZ_KR * 2);  // bytes of one plane
      constexpr int EQ = (OZ_RC * OZ_KC + OZ_BPROD - 1) / OZ_BPROD;   // up to 2 per thread
      // matrix values (and row exponents) of stage st of item it
      // a stacked task: the row segment (offset, lda, local row) that holds
      // each of this thread's element rows, looked up once per unit
      const bool stacked = t.mode == 2;
      long long soff[EQ];
      int slda[EQ], sli[EQ];
      if (stacked) {
        const int tr = items[t.it0].trans;
#pragma unroll
        for (int q = 0; q < EQ; ++q) {
          int i, kk;
          oz_elem(t2 + q * OZ_BPROD, tr, i, kk);
          const int row = rp + i;
          soff[q] = 0;
          slda[q] = 0;
          sli[q] = -1;
          for (int sq = t.it0; sq < t.it1; ++sq) {
            const GItem Q = items[sq];
            if (row >= Q.r0 && row < Q.r0 + Q.nrow) {
              soff[q] = Q.a_off;
              slda[q] = Q.lda;
              sli[q] = row - Q.r0;
            }
          }
        }
      }
      auto load = [&](int it, int st, double2* av, int* ex) {
        const GItem I = items[it];
        const double2* A = (const double2*)ab.p[I.a_buf] + I.a_off;
        const int dl = I.in_row & 3;
#pragma unroll
        for (int q = 0; q < EQ; ++q) {
          int i, kk;
          oz_elem(t2 + q * OZ_BPROD, I.trans, i, kk);
          const int kr = st * OZ_KC + kk - dl;
          av[q] = make_double2(0.0, 0.0);
          ex[q] = 0;
          if (t2 + q * OZ_BPROD < ne && i < nr && kr >= 0 && kr < I.k) {
            if (stacked) {
              if (sli[q] >= 0) {
                const double2* S = (const double2*)ab.p[I.a_buf] + soff[q];
                av[q] = I.trans ? S[(long long)kr * slda[q] + sli[q]]
                                : S[(long long)sli[q] * slda[q] + kr];
              }
            } else {
              av[q] = I.trans ? A[(long long)kr * I.lda + rp + i]
                              : A[(long long)(rp + i) * I.lda + kr];
            }
            ex[q] = rexp[i];
          }
        }
      };
      // the unit's stages in order (items without stages skipped)
      auto next = [&](int it, int st, int& it2, int& st2) {
        it2 = it;
        st2 = st + 1;
        if (st2 >= oz_nst(items[it])) {
          st2 = 0;
          ++it2;
          while (it2 < task_it_end(t) && oz_nst(items[it2]) == 0) ++it2;
        }
      };
      // slice and store the stage whose values are in (av, ex)
      auto put = [&](int it, const double2* av, const int* ex) -> bool {
        const int trans = items[it].trans;
        const int b = g % OZ_RING;
        if (g >= OZ_RING &&
            !oz_wait(b_empty + 8u * b, (uint32_t)(((g - OZ_RING) / OZ_RING) & 1), spin_limit,
                     abortp, err))
          return false;
        unsigned char* sB = smem + b * OZ_STAGE + OZ_NS * OZ_A_BYTES;
#pragma unroll
        for (int q = 0; q < EQ; ++q) {
          if (t2 + q * OZ_BPROD >= ne) continue;
          int i, kk;
          oz_elem(t2 + q * OZ_BPROD, trans, i, kk);
          __nv_bfloat16 ar[OZ_NS], ai[OZ_NS];
          digits(av[q].x, ex[q], ar);
          digits(av[q].y, ex[q], ai);
          // rows 2i and 2i+1 sit 16 bytes apart: lanes with kk >= 4 store
          // them in the other order, so each store instruction of the warp
          // hits 32 distinct banks
          const bool sw = (kk & 4) != 0;
          const uint32_t o0 = kmaj_b(2 * i + (sw ? 1 : 0), 2 * kk);
          const uint32_t o1 = kmaj_b(2 * i + (sw ? 0 : 1), 2 * kk);
#pragma unroll
          for (int s = 0; s < OZ_NS; ++s) {
            unsigned char* bp = sB + s * pb;
            const uint32_t w_re = pack2(ar[s], __hneg(ai[s]));   // row 2i:   [a_re, -a_im]
            const uint32_t w_im = pack2(ai[s], ar[s]);           // row 2i+1: [a_im,  a_re]
            *(uint32_t*)(bp + o0) = sw ? w_im : w_re;
            *(uint32_t*)(bp + o1) = sw ? w_re : w_im;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        mbar_arrive(b_digs + 8u * b);
        ++g;
        return true;
      };
      // loads of a stage are issued before the wait for its buffer
      int it = t.it0, st = 0;
      while (it < task_it_end(t) && oz_nst(items[it]) == 0) ++it;
      double2 av[EQ];
      int ex[EQ];
      while (it < task_it_end(t) && !stop) {
        load(it, st, av, ex);
        if (!put(it, av, ex)) {
          stop = true;
          break;
        }
        int it2, st2;
        next(it, st, it2, st2);
        it = it2;
        st = st2;
      }
    }
  } else {
    // ------------------------------------------------ epilogue (warps 4-7)
    const int row = tid - 128;                 // TMEM lane = RHS row of the tile
    const int col = y * OZ_M + row;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    // the FP64 sums of this thread's RHS row live in shared memory (column c
    // at acc_s[c * OZ_M + row]: a warp touches 32 consecutive doubles)
    double* acc_s = (double*)(smem + OZ_RING * OZ_STAGE);
    int w = 0;
    bool stop = false;
    for (int u = blockIdx.x; u < n_units && !stop; u += gridDim.x) {
      const int2 U = units[u];
      const GTask t = tasks[U.x];
      const int rp = U.y * OZ_RC;
      const int nr = min(OZ_RC, t.m - rp);
      const int* rexp = task_row_exp + task_exp_off[U.x] + rp;
#pragma unroll
      for (int c = 0; c < OZ_N; ++c) acc_s[c * OZ_M + row] = 0.0;
      bool open = false;
      int win = 0, cur = -1;
      // read one completed window out of tensor memory into acc (NC columns
      // per level, level stride NC)
      auto drain_nc = [&](auto ncc, int xb) {
        constexpr int NC = decltype(ncc)::value;
        // tcgen05.ld is warp-collective: the warp takes one decision
        const bool okw = oz_wait(b_tfull + 8u * (w & 1), (uint32_t)((w >> 1) & 1), spin_limit,
                                 abortp, err);
        if (!__all_sync(0xffffffffu, okw)) {
          stop = true;
          return;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int F = (col < nrhs) ? (xb ? fexp_far[col] : fexp_in[col]) : 0;
        // a narrow window lives in tensor-memory half w & 1, a wide one in all
        const uint32_t cb = (NC == 32) ? (uint32_t)(w & 1) * 256u : 0u;
#pragma unroll
        for (int c0 = 0; c0 < NC; c0 += 8) {
          int rx[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) rx[r] = rexp[(c0 / 2 + r) < nr ? (c0 / 2 + r) : 0];
          long long hi[8], lo[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) { hi[j] = 0; lo[j] = 0; }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t v[4][8];
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              const uint32_t ta = lane_base + cb + (uint32_t)((4 * h + l) * NC + c0);
              asm volatile(
                  "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                  : "=r"(v[l][0]), "=r"(v[l][1]), "=r"(v[l][2]), "=r"(v[l][3]), "=r"(v[l][4]),
                    "=r"(v[l][5]), "=r"(v[l][6]), "=r"(v[l][7])
                  : "r"(ta));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int l = 0; l < 4; ++l)
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const long long iv = (long long)__float2int_rn(__uint_as_float(v[l][j]));
                if (h == 0)
                  hi[j] += iv << (7 * (3 - l));
                else
                  lo[j] += iv << (7 * (3 - l));
              }
          }
          // one word hi 2^16 + lo / 2^12 (|hi|, |lo| < 2^45.1: no overflow; the
          // dropped bits are below 2^-49 of the row and column scales), in
          // units of 2^(E_i + F_r - 49), then one fused multiply-add
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const long long V = (hi[j] << 16) + (lo[j] >> 12);
            const int sc = rx[j >> 1] + F - 14;
            double* a = acc_s + (c0 + j) * OZ_M + row;
            *a = fma((double)V, pow2i(sc - 35), *a);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        mbar_arrive(b_tempty + 8u * (w & 1));
        ++w;
      };
      // level L of the unit sits at columns L * n_real (n_real = 32, 48 or 64)
      const int n_real = max(32, ((2 * nr + 15) / 16) * 16);
      auto drain = [&](int xb) {
        if (n_real == 32)
          drain_nc(std::integral_constant<int, 32>{}, xb);
        else if (n_real == 48)
          drain_nc(std::integral_constant<int, 48>{}, xb);
        else
          drain_nc(std::integral_constant<int, 64>{}, xb);
      };
      for (int it = t.it0; it < task_it_end(t) && !stop; ++it) {
        const GItem I = items[it];
        const int nst = oz_nst(I);
        const int xb = (I.in_buf == VB_FAR) ? 1 : 0;
        for (int st = 0; st < nst && !stop; ++st) {
          const bool start = !open || xb != cur || win + OZ_KC > OZ_WIN;
          if (start) {
            if (open) drain(cur);
            open = true;
            win = 0;
            cur = xb;
          }
          win += OZ_KC;
        }
      }
      if (open && !stop) drain(cur);
      if (stop || col >= nrhs) continue;
      TY* out = (TY*)vb.p[t.out_buf] + (long long)(t.out_row + rp) * nrhs;
      const TY* base = (t.mode == 1)
                           ? (const TY*)vb.p[t.base_buf] + (long long)(t.base_row + rp) * nrhs
                           : nullptr;
#pragma unroll
      for (int i = 0; i < OZ_RC; ++i) {
        if (i < nr) {
          double2 yv = make_double2(acc_s[(2 * i) * OZ_M + row], acc_s[(2 * i + 1) * OZ_M + row]);
          if (base) {
            const double2 bv = to_d2(base[(long long)i * nrhs + col]);
            yv.x += bv.x;
            yv.y += bv.y;
          }
          put(out + (long long)i * nrhs + col, yv);
        }
      }
    }
  }
  __syncthreads();
  if (abort_flag) {
    // a CTA that gave up: its MMAs and copies complete before tensor memory
    // and shared memory are released (bounded waits, abort flag ignored)
    if (tid == 0) {
      volatile int never = 0;
      const long long lim = spin_limit > (1LL << 24) ? spin_limit : (1LL << 24);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
          :: "r"(b_fin));
      oz_wait(b_fin, 0u, lim, &never, err);
      for (int g = consumed_s; g < armed_s; ++g)
        oz_wait(b_full + 8u * (g % OZ_RING), (uint32_t)((g / OZ_RING) & 1), lim, &never,
                err);
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

// F_r = smallest S with max_k max(|re|, |im|) of panel column r < 2^S.
// Thread = column r over a chunk of OZ_CE_ROWS rows (reads coalesced across
// the threads of a warp); chunks combine by an integer atomicMax on out[r],
// which the launcher first fills with a value below every candidate.
constexpr int OZ_CE_ROWS = 256;
template <class TV>
__global__ void k_col_exp(const TV* __restrict__ V, int rows, int nrhs, int* out) {
  const int r = blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  const long long i0 = (long long)blockIdx.x * OZ_CE_ROWS;
  const long long i1 = min((long long)rows, i0 + OZ_CE_ROWS);
  unsigned int m = 0;      // max biased exponent seen
  for (long long i = i0; i < i1; ++i) {
    const TV v = V[i * nrhs + r];
    m = max(m, max(bexp(v.x), bexp(v.y)));
  }
  // |v| < 2^(e - 1022) for biased exponent e (v = 1.f * 2^(e - 1023))
  atomicMax(out + r, m == 0 ? -1022 : (int)m - 1022);
}

}  // namespace

hm_status build_oz_units(TaskList& tl, size_t* dev_bytes, bool list_order) {
  cudaFree(tl.d_units);
  tl.d_units = nullptr;
  tl.n_units = 0;
  std::vector<std::pair<long long, int2>> u;
  for (size_t q = 0; q < tl.tasks.size(); ++q) {
    const GTask& t = tl.tasks[q];
    long long cost = 2;                       // set-up and output rows of a unit
    for (int it = t.it0; it < task_it_end(t); ++it) cost += oz_nst(tl.items[it]);
    for (int pass = 0; pass * OZ_RC < t.m; ++pass) u.push_back({cost, make_int2((int)q, pass)});
  }
  // costliest first (load balance), or in list order: neighbouring leaf tasks
  // read overlapping inputs, so walking them together keeps those in L2
  if (!list_order)
    std::stable_sort(u.begin(), u.end(), [](const std::pair<long long, int2>& a,
                                             const std::pair<long long, int2>& b) {
      return a.first > b.first;
    });
  if (u.empty()) return HM_OK;
  std::vector<int2> v(u.size());
  for (size_t q = 0; q < u.size(); ++q) v[q] = u[q].second;
  HM_CUDA(cudaMalloc((void**)&tl.d_units, v.size() * sizeof(int2)));
  HM_CUDA(cudaMemcpy(tl.d_units, v.data(), v.size() * sizeof(int2), cudaMemcpyHostToDevice));
  tl.n_units = (int)v.size();
  if (dev_bytes) *dev_bytes += v.size() * sizeof(int2);
  return HM_OK;
}

hm_status launch_col_exp(const cplx* V, int rows, int nrhs, int* out, cudaStream_t s) {
  HM_CUDA(cudaMemsetAsync(out, 0x80, sizeof(int) * nrhs, s));   // 0x80808080 < -1022
  const dim3 grid((unsigned)((rows + OZ_CE_ROWS - 1) / OZ_CE_ROWS), (unsigned)((nrhs + 127) / 128));
  k_col_exp<double2><<<grid, 128, 0, s>>>(V, rows, nrhs, out);
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_col_exp32(const float2* V, int rows, int nrhs, int* out, cudaStream_t s) {
  HM_CUDA(cudaMemsetAsync(out, 0x80, sizeof(int) * nrhs, s));   // 0x80808080 < -1022
  const dim3 grid((unsigned)((rows + OZ_CE_ROWS - 1) / OZ_CE_ROWS), (unsigned)((nrhs + 127) / 128));
  k_col_exp<float2><<<grid, 128, 0, s>>>(V, rows, nrhs, out);
  HM_LAUNCHED();
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
  HM_LAUNCHED();
  return HM_OK;
}

hm_status launch_tasks_oz(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, const int* row_exp, const long long* exp_off,
                          const int* fexp_in, const int* fexp_far, const OzPanels& xp,
                          long long spin_limit, int* err, bool panels32) {
  if (tl.tasks.empty() || tl.n_units == 0) return HM_OK;
  if (xp.G * 8 < nrhs || xp.G % 16 != 0 || !tl.d_units) return HM_ERR_INVALID;
  if (!abufs_bound(tl, ab)) return HM_ERR_STATE;
  static bool attr = false;
  static int nsm = 0;
  if (!attr) {
    HM_CUDA(cudaFuncSetAttribute(k_oz_gather<double2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    HM_CUDA(cudaFuncSetAttribute(k_oz_gather<float2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    int dev = 0;
    HM_CUDA(cudaGetDevice(&dev));
    HM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    attr = true;
  }
  // one resident CTA per SM: the tiles of 128 RHS share the SMs
  const int ytiles = (nrhs + OZ_M - 1) / OZ_M;
  const int gx = std::max(1, std::min(tl.n_units, std::max(1, nsm / ytiles)));
  dim3 grid((unsigned)gx, (unsigned)ytiles);
  if (panels32)
    k_oz_gather<float2><<<grid, OZ_THREADS, OZ_SMEM, s>>>(
        tl.d_tasks, tl.d_items, tl.d_units, tl.n_units, vb, ab, nrhs, row_exp, exp_off, fexp_in,
        fexp_far, xp, spin_limit, err);
  else
    k_oz_gather<double2><<<grid, OZ_THREADS, OZ_SMEM, s>>>(
        tl.d_tasks, tl.d_items, tl.d_units, tl.n_units, vb, ab, nrhs, row_exp, exp_off, fexp_in,
        fexp_far, xp, spin_limit, err);
  HM_LAUNCHED();
  return HM_OK;
}

}  // namespace hm
