// Far-field product Y = Z_F X that allocates no device memory.
//
// Why: some callers cannot allocate device memory at the time they need the
// product: code running inside a pre-sized memory pool or arena that owns all
// of the device memory, code under a framework allocator that forbids raw
// cudaMalloc, or a hot loop whose latency budget cannot absorb allocation.
// hm_apply (HM_OP_FAR) sizes its work panels on first use; this variant keeps
// its only scratch -- the stage-1 panels t_b = V_b^T x and U_b^T x of the
// low-rank far blocks -- in a fixed file-scope device array instead.
//
// The scratch array (HM_NOALLOC_SCRATCH_BYTES) is part of the library image:
// every GPU that loads the library holds it until the process exits.  All
// calls share it and it keeps the last call's contents; stage 1 overwrites
// every scratch row that stage 2 reads, so nothing needs clearing.  Two calls
// whose kernels overlap on the GPU (different streams, or different handles)
// race on the array.
#include <mutex>

#include "hm_internal.h"

using namespace hm;

namespace {

constexpr size_t NA_ELEMS = (size_t)HM_NOALLOC_SCRATCH_BYTES / sizeof(double2);
static __device__ __align__(256) double2 g_noalloc_scratch[NA_ELEMS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on device dev, which must be the
// current device: looked up with cudaGetSymbolAddress once per device (the
// name is only a host-side stand-in for the symbol and cannot be passed to a
// kernel).
hm_status scratch_ptr(int dev, double2** out) {
  if (dev < 0 || dev >= MAX_DEVICES) return HM_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return HM_ERR_CUDA;
    g_scr[dev] = p;
  }
  *out = (double2*)g_scr[dev];
  return HM_OK;
}

__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 x) {
  acc.x = fma(a.x, x.x, acc.x);
  acc.x = fma(-a.y, x.y, acc.x);
  acc.y = fma(a.x, x.y, acc.y);
  acc.y = fma(a.y, x.x, acc.y);
}

// Stage 1: T[(out_row + i) * nrhs + r] = sum_k op(A)[i][k] X[r * N + perm[in_row + k]]
// (tasks / items of the far stage-1 schedule; X column-major, original order).
__global__ void k_na_far1(const GTask* __restrict__ tasks, const GItem* __restrict__ items,
                          const double2* __restrict__ F, const double2* __restrict__ X,
                          const int* __restrict__ perm, int N, int nrhs, double2* T) {
  const GTask t = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < t.m * nrhs; e += blockDim.x) {
    int i = e / nrhs, r = e % nrhs;
    double2 acc = make_double2(0.0, 0.0);
    for (int q = t.it0; q < t.it1; ++q) {
      const GItem I = items[q];
      const double2* A = F + I.a_off;
      for (int k = 0; k < I.k; ++k) {
        double2 a = I.trans ? A[(long long)k * I.lda + i] : A[(long long)i * I.lda + k];
        cmac(acc, a, X[(long long)r * N + perm[I.in_row + k]]);
      }
    }
    T[(long long)(t.out_row + i) * nrhs + r] = acc;
  }
}

// Stage 2: Y[r * N + perm[out_row + i]] = sum over the leaf's items, reading
// T (low-rank items) or X (dense far blocks).
__global__ void k_na_far2(const GTask* __restrict__ tasks, const GItem* __restrict__ items,
                          const double2* __restrict__ F, const double2* __restrict__ X,
                          const int* __restrict__ perm, int N, int nrhs,
                          const double2* __restrict__ T, double2* __restrict__ Y) {
  const GTask t = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < t.m * nrhs; e += blockDim.x) {
    int i = e / nrhs, r = e % nrhs;
    double2 acc = make_double2(0.0, 0.0);
    for (int q = t.it0; q < t.it1; ++q) {
      const GItem I = items[q];
      const double2* A = F + I.a_off;
      for (int k = 0; k < I.k; ++k) {
        double2 a = I.trans ? A[(long long)k * I.lda + i] : A[(long long)i * I.lda + k];
        double2 x = (I.in_buf == VB_FAR) ? T[(long long)(I.in_row + k) * nrhs + r]
                                         : X[(long long)r * N + perm[I.in_row + k]];
        cmac(acc, a, x);
      }
    }
    Y[(long long)r * N + perm[t.out_row + i]] = acc;
  }
}

}  // namespace

extern "C" hm_status hm_apply_far_noalloc(hm_handle h, void* Y, const void* X, int nrhs) {
  if (!h || !Y || !X || nrhs <= 0) return HM_ERR_INVALID;
  if (!h->sched_ready) return HM_ERR_STATE;
  if ((size_t)h->far_t_rows * (size_t)nrhs > NA_ELEMS) return HM_ERR_INVALID;
  // the kernels run on the handle's stream, which belongs to the handle's
  // device: that device must be current
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return HM_ERR_CUDA;
  if (cur != h->dev) return HM_ERR_INVALID;
  double2* T = nullptr;
  hm_status s = scratch_ptr(h->dev, &T);
  if (s) return s;
  // a handle without far blocks (one leaf, or every pair near) has no stage-1
  // tasks; stage 2 still runs one task per leaf and writes Y = 0
  if (!h->far1_tl.tasks.empty())
    k_na_far1<<<(unsigned)h->far1_tl.tasks.size(), 256, 0, h->stream>>>(
        h->far1_tl.d_tasks, h->far1_tl.d_items, h->d_far, (const double2*)X, h->d_perm, h->N,
        nrhs, T);
  if (!h->far2_tl.tasks.empty())
    k_na_far2<<<(unsigned)h->far2_tl.tasks.size(), 256, 0, h->stream>>>(
        h->far2_tl.d_tasks, h->far2_tl.d_items, h->d_far, (const double2*)X, h->d_perm, h->N,
        nrhs, T, (double2*)Y);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HM_OK : cuda_status(e);
}
