// GPU Schur-complement scaling of the near field (Sec. III-A, Eq. 14-23) and
// the plane-wave excitation (Eq. 2 tested with RWG functions).
//
// For elimination rank k = 0..n-1 (leaf elim[k]):
//   D_k^-1   Gauss-Jordan with partial pivoting, FP64         (k_inverse)
//   alpha_kj = -D_k^-1 Z~_kj      for j in row k               (k_bgemm)
//   Z~_ij   += alpha_ki^T Z~_kj   for i <= j in row k          (k_bgemm)
// Row k holds every fill-in block (HM_FILL_FULL: symbolic block Cholesky
// pattern via the elimination tree) or only near blocks (HM_FILL_NEAR, where
// updates outside the pattern are dropped).
#include <algorithm>
#include <cmath>
#include <functional>
#include <new>
#include <numeric>
#include <set>

#include "hm_internal.h"
#include "hm_mixed.h"

using namespace hm;

namespace hm {
hm_status upload_values(hm_ctx* h);
hm_status rebuild_schedules(hm_ctx* h);
}

namespace {

struct BTask {
  const cplx* A;
  const cplx* B;
  cplx* C;
  int M, N, K, lda, ldb, ldc, transA, beta;   // C = beta*C + alpha op(A) B
  double alpha;
};

// C (M x N) = beta C + alpha op(A) B; op(A) = A (M x K, lda) or A^T with A
// K x M (lda).  One CTA per task, 32 x 32 output tiles, 256 threads.
__global__ void __launch_bounds__(256) k_bgemm(const BTask* tasks) {
  const BTask t = tasks[blockIdx.x];
  __shared__ cplx As[32][17];
  __shared__ cplx Bs[16][33];
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;   // 2 x 2 outputs each
  for (int m0 = 0; m0 < t.M; m0 += 32)
    for (int n0 = 0; n0 < t.N; n0 += 32) {
      cplx acc[2][2] = {{{0, 0}, {0, 0}}, {{0, 0}, {0, 0}}};
      for (int k0 = 0; k0 < t.K; k0 += 16) {
        for (int e = threadIdx.x; e < 32 * 16; e += 256) {
          int r, c;
          cplx v = make_double2(0.0, 0.0);
          if (!t.transA) {
            r = e / 16; c = e % 16;
            if (m0 + r < t.M && k0 + c < t.K) v = t.A[(long long)(m0 + r) * t.lda + k0 + c];
          } else {
            c = e / 32; r = e % 32;
            if (m0 + r < t.M && k0 + c < t.K) v = t.A[(long long)(k0 + c) * t.lda + m0 + r];
          }
          As[r][c] = v;
        }
        for (int e = threadIdx.x; e < 16 * 32; e += 256) {
          int r = e / 32, c = e % 32;
          Bs[r][c] = (k0 + r < t.K && n0 + c < t.N) ? t.B[(long long)(k0 + r) * t.ldb + n0 + c]
                                                     : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
          cplx a0 = As[tr * 2][kk], a1 = As[tr * 2 + 1][kk];
          cplx b0 = Bs[kk][tc * 2], b1 = Bs[kk][tc * 2 + 1];
          cplx a[2] = {a0, a1}, b[2] = {b0, b1};
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
              acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
              acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
              acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
            }
        }
        __syncthreads();
      }
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          int r = m0 + tr * 2 + i, c = n0 + tc * 2 + j;
          if (r >= t.M || c >= t.N) continue;
          cplx* p = t.C + (long long)r * t.ldc + c;
          cplx v = make_double2(t.alpha * acc[i][j].x, t.alpha * acc[i][j].y);
          if (t.beta) {
            v.x += p->x;
            v.y += p->y;
          }
          *p = v;
        }
    }
}

// In-place Gauss-Jordan inverse with partial pivoting of one m x m matrix
// (row-major) using the 2m-wide scratch W; writes the inverse to out and sets
// *flag = 1 if a pivot column is exactly zero.
__global__ void __launch_bounds__(512) k_inverse(const cplx* A, int m, cplx* W, cplx* out,
                                                 int* flag) {
  extern __shared__ double smem[];
  cplx* fac = (cplx*)smem;                       // m factors
  double* sv = smem + 2 * m;                     // 512 reduction values
  int* si = (int*)(sv + 512);
  const int w2 = 2 * m;
  for (int e = threadIdx.x; e < m * w2; e += blockDim.x) {
    int r = e / w2, c = e % w2;
    W[e] = (c < m) ? A[r * m + c] : make_double2(c - m == r ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    double best = -1.0;
    int bi = m;
    for (int r = c + threadIdx.x; r < m; r += blockDim.x) {
      cplx v = W[r * w2 + c];
      double a = v.x * v.x + v.y * v.y;
      if (a > best) { best = a; bi = r; }
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) {
        double b2 = sv[threadIdx.x + s];
        int i2 = si[threadIdx.x + s];
        if (b2 > sv[threadIdx.x] || (b2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
          sv[threadIdx.x] = b2;
          si[threadIdx.x] = i2;
        }
      }
      __syncthreads();
    }
    const int p = si[0];
    const double pv = sv[0];
    __syncthreads();
    if (!(pv > 0.0)) {
      if (threadIdx.x == 0) *flag = 1;
      return;
    }
    if (p != c)
      for (int e = threadIdx.x; e < w2; e += blockDim.x) {
        cplx t = W[c * w2 + e];
        W[c * w2 + e] = W[p * w2 + e];
        W[p * w2 + e] = t;
      }
    __syncthreads();
    cplx d = W[c * w2 + c];
    double dn = d.x * d.x + d.y * d.y;
    cplx di = make_double2(d.x / dn, -d.y / dn);
    __syncthreads();
    for (int e = threadIdx.x; e < w2; e += blockDim.x) {
      cplx v = W[c * w2 + e];
      W[c * w2 + e] = make_double2(v.x * di.x - v.y * di.y, v.x * di.y + v.y * di.x);
    }
    for (int r = threadIdx.x; r < m; r += blockDim.x) fac[r] = W[r * w2 + c];
    __syncthreads();
    for (int e = threadIdx.x; e < m * w2; e += blockDim.x) {
      int r = e / w2, col = e % w2;
      if (r == c) continue;
      cplx f = fac[r], v = W[c * w2 + col], x = W[e];
      x.x -= f.x * v.x - f.y * v.y;
      x.y -= f.x * v.y + f.y * v.x;
      W[e] = x;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int r = e / m, c = e % m;
    out[e] = W[r * w2 + m + c];
  }
}

struct CopyJob { long long src, dst; int rows, cols, trans; };

// identity diagonal blocks of every supernode matrix T_G (row-major n_G x n_G)
struct EyeJob { long long off; int nG; };
__global__ void k_eye_groups(const EyeJob* jobs, cplx* T) {
  EyeJob j = jobs[blockIdx.x];
  for (int i = threadIdx.x; i < j.nG; i += blockDim.x)
    T[j.off + (long long)i * j.nG + i] = make_double2(1.0, 0.0);
}

void k_eye_groups_launch(cplx* dT, const std::vector<long long>& tg_off,
                         const std::vector<int>& tg_n, const std::vector<int>&,
                         const std::vector<int>&, const std::vector<int>&) {
  std::vector<EyeJob> ej;
  for (size_t g = 0; g < tg_n.size(); ++g)
    if (tg_n[g]) ej.push_back(EyeJob{tg_off[g], tg_n[g]});
  if (ej.empty()) return;
  EyeJob* d = nullptr;
  if (cudaMalloc((void**)&d, ej.size() * sizeof(EyeJob)) != cudaSuccess) throw HM_ERR_OOM;
  cudaMemcpy(d, ej.data(), ej.size() * sizeof(EyeJob), cudaMemcpyHostToDevice);
  k_eye_groups<<<(unsigned)ej.size(), 256>>>(d, dT);
  cudaDeviceSynchronize();
  cudaFree(d);
}

// element offset of alpha_{l j} (ranks, l < j) or -1
long long zidx_alpha(const std::vector<std::vector<int>>& rows,
                     const std::vector<long long>& row_start, const std::vector<long long>& aoff,
                     int l, int j) {
  auto it = std::lower_bound(rows[l].begin(), rows[l].end(), j);
  if (it == rows[l].end() || *it != j) return -1;
  return aoff[row_start[l] + (it - rows[l].begin())];
}

__global__ void k_copy_blocks(const CopyJob* jobs, const cplx* src, cplx* dst) {
  CopyJob j = jobs[blockIdx.x];
  for (int e = threadIdx.x; e < j.rows * j.cols; e += blockDim.x) {
    int r = e / j.cols, c = e % j.cols;
    // destination r x c of a rows x cols block; source is cols x rows when transposed
    dst[j.dst + e] = j.trans ? src[j.src + (long long)c * j.rows + r] : src[j.src + e];
  }
}

// b_n = sum_{s in +-} s (l_n / 2) sum_q w_q ((r_q - v_s) . p) e^{-jk khat . r_q}
__global__ void k_plane_wave(const double* V, const int* T, const double* Q, const int* tp,
                             const int* tm, const int* fp, const int* fm, const double* len,
                             int N, double k, const double* dirs, int nrhs, cplx* B) {
  long long tot = (long long)N * nrhs;
  const double s15 = 3.872983346207417;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / N), n = (int)(e % N);
    const double* kh = dirs + 6 * r;
    const double* ph = kh + 3;
    double bx = 0.0, by = 0.0;
    for (int s = 0; s < 2; ++s) {
      int t = s ? tm[n] : tp[n];
      int f = s ? fm[n] : fp[n];
      const double* v = V + 3 * T[3 * t + f];
      double px = 0.0, py = 0.0;
      for (int q = 0; q < 7; ++q) {
        const double* rq = Q + (size_t)(7 * t + q) * 3;
        double w = q == 0 ? 9.0 / 40.0 : (q <= 3 ? (155.0 - s15) / 1200.0 : (155.0 + s15) / 1200.0);
        double proj = (rq[0] - v[0]) * ph[0] + (rq[1] - v[1]) * ph[1] + (rq[2] - v[2]) * ph[2];
        double arg = -k * (kh[0] * rq[0] + kh[1] * rq[1] + kh[2] * rq[2]);
        double sn, cs;
        sincos(arg, &sn, &cs);
        px += w * proj * cs;
        py += w * proj * sn;
      }
      double sc = (s ? -0.5 : 0.5) * len[n];
      bx += sc * px;
      by += sc * py;
    }
    B[(long long)r * N + n] = make_double2(bx, by);
  }
}

// Geometric nested dissection of the leaf graph (same rules as the CPU
// statement: median split of the widest axis of the cell centres, ties by
// leaf number; separator = the first half's leaves adjacent to the second).
void nd_order(const std::vector<double>& cen, int n, const std::vector<std::pair<int, int>>& near,
              std::vector<int>& order, std::vector<int>* groups = nullptr) {
  std::vector<std::vector<int>> adj(n);
  for (auto& e : near)
    if (e.first != e.second) {
      adj[e.first].push_back(e.second);
      adj[e.second].push_back(e.first);
    }
  std::vector<char> side(n, 0);
  std::function<void(std::vector<int>)> rec = [&](std::vector<int> ids) {
    if (ids.size() <= 4) {
      std::sort(ids.begin(), ids.end());
      if (groups && !ids.empty()) groups->push_back((int)order.size());
      order.insert(order.end(), ids.begin(), ids.end());
      return;
    }
    int ax = 0;
    double best = -1.0;
    for (int a = 0; a < 3; ++a) {
      double lo = 1e300, hi = -1e300;
      for (int i : ids) {
        lo = std::min(lo, cen[3 * i + a]);
        hi = std::max(hi, cen[3 * i + a]);
      }
      if (hi - lo > best) { best = hi - lo; ax = a; }
    }
    std::sort(ids.begin(), ids.end(), [&](int x, int y) {
      if (cen[3 * x + ax] != cen[3 * y + ax]) return cen[3 * x + ax] < cen[3 * y + ax];
      return x < y;
    });
    size_t h = ids.size() / 2;
    for (size_t q = 0; q < ids.size(); ++q) side[ids[q]] = q < h ? 1 : 2;
    std::vector<int> A, B, S;
    for (size_t q = 0; q < ids.size(); ++q) {
      int i = ids[q];
      if (q >= h) { B.push_back(i); continue; }
      bool sep = false;
      for (int j : adj[i]) sep |= (side[j] == 2);
      (sep ? S : A).push_back(i);
    }
    for (int i : ids) side[i] = 0;
    std::sort(A.begin(), A.end());
    std::sort(B.begin(), B.end());
    std::sort(S.begin(), S.end());
    rec(A);
    rec(B);
    if (groups && !S.empty()) groups->push_back((int)order.size());   // the separator
    order.insert(order.end(), S.begin(), S.end());
  };
  std::vector<int> all(n);
  std::iota(all.begin(), all.end(), 0);
  rec(all);
}

}  // namespace

extern "C" {

hm_status hm_compute_scaling(hm_handle h) {
  if (!h) return HM_ERR_INVALID;
  if (h->near.empty() || h->nonsym) return HM_ERR_STATE;   // symmetric elimination only
  cplx *dZ = nullptr, *dZd = nullptr, *dW = nullptr, *dA = nullptr, *dD = nullptr;
  BTask* dT = nullptr;
  CopyJob* dC = nullptr;
  int* dflag = nullptr;
  auto cleanup = [&]() {
    cudaFree(dZ); cudaFree(dZd); cudaFree(dW); cudaFree(dT); cudaFree(dC); cudaFree(dflag);
  };
  try {
    const int n = h->nl;
    // ---- elimination order
    std::vector<std::pair<int, int>> nearp;
    for (auto& d : h->near) nearp.push_back({d.i, d.j});
    std::vector<int> elim, groups;
    if (h->p.ordering == HM_ORDER_ND && (int)h->leaf_cen.size() == 3 * n) {
      nd_order(h->leaf_cen, n, nearp, elim, &groups);
    } else {
      elim.resize(n);
      std::iota(elim.begin(), elim.end(), 0);
    }
    groups.push_back(n);        // group g = ranks [groups[g], groups[g+1])
    std::vector<int> pos(n);
    for (int q = 0; q < n; ++q) pos[elim[q]] = q;
    // ---- symbolic pattern (ranks)
    std::vector<std::set<int>> rs(n);
    for (auto& e : nearp) {
      int a = pos[e.first], b = pos[e.second];
      if (a == b) continue;
      rs[std::min(a, b)].insert(std::max(a, b));
    }
    if (h->p.fill == HM_FILL_FULL)
      for (int k = 0; k < n; ++k)
        if (!rs[k].empty()) {
          int par = *rs[k].begin();
          for (int j : rs[k]) if (j != par) rs[par].insert(j);
        }
    std::vector<std::vector<int>> rows(n);
    for (int k = 0; k < n; ++k) rows[k].assign(rs[k].begin(), rs[k].end());
    std::vector<int> me(n);
    for (int q = 0; q < n; ++q) me[q] = h->m[elim[q]];
    std::vector<long long> row_start(n + 1, 0), aoff, doff(n);
    long long na = 0, nd = 0;
    for (int k = 0; k < n; ++k) {
      row_start[k] = (long long)aoff.size();
      for (int j : rows[k]) {
        aoff.push_back(na);
        na += (long long)me[k] * me[j];
      }
      doff[k] = nd;
      nd += (long long)me[k] * me[k];
    }
    row_start[n] = (long long)aoff.size();
    auto zidx = [&](int i, int j) -> long long {   // offset of Z~_ij (i < j), -1 if absent
      auto it = std::lower_bound(rows[i].begin(), rows[i].end(), j);
      if (it == rows[i].end() || *it != j) return -1;
      return aoff[row_start[i] + (it - rows[i].begin())];
    };
    HM_CUDA(cudaMalloc((void**)&dZ, std::max<long long>(1, na) * sizeof(cplx)));
    HM_CUDA(cudaMalloc((void**)&dZd, nd * sizeof(cplx)));
    HM_CUDA(cudaMemset(dZ, 0, std::max<long long>(1, na) * sizeof(cplx)));
    cplx* newA = nullptr;
    cplx* newD = nullptr;
    HM_CUDA(cudaMalloc((void**)&newA, std::max<long long>(1, na) * sizeof(cplx)));
    dA = newA;
    HM_CUDA(cudaMalloc((void**)&newD, nd * sizeof(cplx)));
    dD = newD;
    int mmax = *std::max_element(me.begin(), me.end());
    HM_CUDA(cudaMalloc((void**)&dW, (size_t)mmax * 2 * mmax * sizeof(cplx)));
    HM_CUDA(cudaMalloc((void**)&dflag, sizeof(int)));
    HM_CUDA(cudaMemset(dflag, 0, sizeof(int)));
    // ---- initial Z~ from the near blocks
    std::vector<CopyJob> cj;
    for (auto& d : h->near) {
      int a = pos[d.i], b = pos[d.j];
      if (a == b) {
        cj.push_back(CopyJob{d.off, doff[a], me[a], me[a], 0});
      } else if (a < b) {
        cj.push_back(CopyJob{d.off, zidx(a, b), me[a], me[b], 0});
      } else {
        cj.push_back(CopyJob{d.off, zidx(b, a), me[b], me[a], 1});
      }
    }
    {
      // diagonal jobs target dZd, others dZ
      std::vector<CopyJob> jd, jo;
      for (size_t q = 0; q < cj.size(); ++q) {
        const NearDesc& d = h->near[q];
        if (pos[d.i] == pos[d.j]) jd.push_back(cj[q]); else jo.push_back(cj[q]);
      }
      for (auto* lst : {&jd, &jo}) {
        if (lst->empty()) continue;
        HM_CUDA(cudaMalloc((void**)&dC, lst->size() * sizeof(CopyJob)));
        HM_CUDA(cudaMemcpy(dC, lst->data(), lst->size() * sizeof(CopyJob), cudaMemcpyHostToDevice));
        k_copy_blocks<<<(unsigned)lst->size(), 256>>>(dC, h->d_near, lst == &jd ? dZd : dZ);
        HM_LAUNCHED();
        HM_CUDA(cudaDeviceSynchronize());
        cudaFree(dC);
        dC = nullptr;
      }
    }
    // ---- numeric elimination
    std::vector<BTask> tasks;
    std::vector<std::pair<size_t, size_t>> step_alpha(n), step_schur(n);
    for (int k = 0; k < n; ++k) {
      size_t s0 = tasks.size();
      for (size_t q = 0; q < rows[k].size(); ++q) {
        int j = rows[k][q];
        long long ao = aoff[row_start[k] + q];
        tasks.push_back(BTask{dD + doff[k], dZ + ao, dA + ao, me[k], me[j], me[k], me[k], me[j],
                              me[j], 0, 0, -1.0});
      }
      step_alpha[k] = {s0, tasks.size()};
      s0 = tasks.size();
      for (size_t a = 0; a < rows[k].size(); ++a) {
        int i = rows[k][a];
        long long aki = aoff[row_start[k] + a];
        for (size_t b = a; b < rows[k].size(); ++b) {
          int j = rows[k][b];
          cplx* tgt;
          int ldc;
          if (i == j) {
            tgt = dZd + doff[i];
            ldc = me[i];
          } else {
            long long o = zidx(i, j);
            if (o < 0) continue;          // near-pattern fill: dropped
            tgt = dZ + o;
            ldc = me[j];
          }
          long long zkj = aoff[row_start[k] + b];
          tasks.push_back(BTask{dA + aki, dZ + zkj, tgt, me[i], me[j], me[k], me[i], me[j], ldc,
                                1, 1, 1.0});
        }
      }
      step_schur[k] = {s0, tasks.size()};
    }
    if (!tasks.empty()) {
      HM_CUDA(cudaMalloc((void**)&dT, tasks.size() * sizeof(BTask)));
      HM_CUDA(cudaMemcpy(dT, tasks.data(), tasks.size() * sizeof(BTask), cudaMemcpyHostToDevice));
    }
    size_t shm = 2 * (size_t)mmax * sizeof(double) + 512 * sizeof(double) + 512 * sizeof(int);
    if (shm > 48 * 1024)
      HM_CUDA(cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    for (int k = 0; k < n; ++k) {
      k_inverse<<<1, 512, shm>>>(dZd + doff[k], me[k], dW, dD + doff[k], dflag);
      auto sa = step_alpha[k];
      if (sa.second > sa.first) k_bgemm<<<(unsigned)(sa.second - sa.first), 256>>>(dT + sa.first);
      auto ss = step_schur[k];
      if (ss.second > ss.first) k_bgemm<<<(unsigned)(ss.second - ss.first), 256>>>(dT + ss.first);
    }
    HM_LAUNCHED();
    HM_CUDA(cudaDeviceSynchronize());
    int flag = 0;
    HM_CUDA(cudaMemcpy(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      cudaFree(dA);
      cudaFree(dD);
      cleanup();
      return HM_ERR_SINGULAR;
    }
    // ---- supernodes: T_G = (I - A_G^T)^-1 for every nested-dissection group G
    // with more than one leaf (A_G: the alpha blocks inside G), by the
    // row-block recurrence T_j,: = I_j,: + sum_{l<j in G} alpha_lj^T T_l,:
    std::vector<long long> tg_off;     // per group: element offset of T_G (n_G x n_G)
    std::vector<int> tg_n;             // n_G (0 for single-leaf groups)
    std::vector<int> rloc(n, 0);       // rank -> row offset inside its group
    long long nt_all = 0;
    const int ng = (int)groups.size() - 1;
    for (int g = 0; g < ng; ++g) {
      int nG = 0;
      for (int q = groups[g]; q < groups[g + 1]; ++q) { rloc[q] = nG; nG += me[q]; }
      bool multi = groups[g + 1] - groups[g] > 1;
      tg_off.push_back(nt_all);
      tg_n.push_back(multi ? nG : 0);
      if (multi) nt_all += (long long)nG * nG;
    }
    cplx* dT = nullptr;
    if (nt_all > 0) {
      HM_CUDA(cudaMalloc((void**)&dT, nt_all * sizeof(cplx)));
      HM_CUDA(cudaMemset(dT, 0, nt_all * sizeof(cplx)));
      std::vector<cplx> eye_dummy;
      // identity diagonal blocks
      std::vector<CopyJob> ij;
      int maxg = 0;
      for (int g = 0; g < ng; ++g) {
        if (!tg_n[g]) continue;
        maxg = std::max(maxg, groups[g + 1] - groups[g]);
      }
      k_eye_groups_launch(dT, tg_off, tg_n, groups, rloc, me);
      for (int pr = 1; pr < maxg; ++pr) {
        for (int qr = 0; qr < pr; ++qr) {
          std::vector<BTask> bt;
          for (int g = 0; g < ng; ++g) {
            if (!tg_n[g] || groups[g] + pr >= groups[g + 1]) continue;
            const int j = groups[g] + pr, l = groups[g] + qr;
            long long a = zidx_alpha(rows, row_start, aoff, l, j);
            if (a < 0) continue;
            const int nG = tg_n[g];
            const int w = rloc[l] + me[l];         // columns 0 .. (end of block l)
            cplx* base = dT + tg_off[g];
            bt.push_back(BTask{dA + a, base + (long long)rloc[l] * nG, base + (long long)rloc[j] * nG,
                               me[j], w, me[l], me[j], nG, nG, 1, 1, 1.0});
          }
          if (bt.empty()) continue;
          BTask* dbt = nullptr;
          HM_CUDA(cudaMalloc((void**)&dbt, bt.size() * sizeof(BTask)));
          HM_CUDA(cudaMemcpy(dbt, bt.data(), bt.size() * sizeof(BTask), cudaMemcpyHostToDevice));
          k_bgemm<<<(unsigned)bt.size(), 256>>>(dbt);
          cudaError_t ce = cudaDeviceSynchronize();
          cudaFree(dbt);
          if (ce != cudaSuccess) throw cuda_status(ce);
        }
      }
    }
    // ---- install
    cudaFree(h->d_tinv);
    h->d_tinv = dT;
    h->grp = groups;
    h->tg_off = tg_off;
    h->tg_n = tg_n;
    h->rloc = rloc;
    h->h_tinv.resize(nt_all);
    if (nt_all)
      HM_CUDA(cudaMemcpy(h->h_tinv.data(), dT, nt_all * sizeof(cplx), cudaMemcpyDeviceToHost));
    cudaFree(h->d_alpha);
    cudaFree(h->d_dinv);
    h->d_alpha = dA;
    h->d_dinv = dD;
    dA = dD = nullptr;
    h->elim = elim;
    h->rows = rows;
    h->alpha_off = aoff;
    h->alpha_row_start = row_start;
    h->dinv_off = doff;
    h->h_alpha.resize(na);
    h->h_dinv.resize(nd);
    if (na) HM_CUDA(cudaMemcpy(h->h_alpha.data(), h->d_alpha, na * sizeof(cplx), cudaMemcpyDeviceToHost));
    HM_CUDA(cudaMemcpy(h->h_dinv.data(), h->d_dinv, nd * sizeof(cplx), cudaMemcpyDeviceToHost));
    h->has_scaling = true;
    h->dev_bytes += (na + nd) * sizeof(cplx);
    cleanup();
    hm_status s = rebuild_schedules(h);
    if (s) return s;
    return hm_mixed_prepare(h);
  } catch (std::bad_alloc&) {
    cleanup();
    return HM_ERR_OOM;
  } catch (...) {
    cleanup();
    return HM_ERR_INVALID;
  }
}

hm_status hm_plane_wave_rhs(hm_handle h, const double* theta, const double* phi, const int* pol,
                            int nrhs, void* B) {
  if (!h || !theta || !phi || !pol || !B || nrhs <= 0) return HM_ERR_INVALID;
  if (!h->mesh_q) return HM_ERR_STATE;   // imported handles carry no mesh
  std::vector<double> dirs(6 * (size_t)nrhs);
  for (int r = 0; r < nrhs; ++r) {
    double st = std::sin(theta[r]), ct = std::cos(theta[r]);
    double sp = std::sin(phi[r]), cp = std::cos(phi[r]);
    double* d = dirs.data() + 6 * r;
    d[0] = -st * cp; d[1] = -st * sp; d[2] = -ct;
    if (pol[r] == 0) { d[3] = ct * cp; d[4] = ct * sp; d[5] = -st; }
    else if (pol[r] == 1) { d[3] = -sp; d[4] = cp; d[5] = 0.0; }
    else return HM_ERR_INVALID;
  }
  double* dd = nullptr;
  HM_CUDA(cudaMalloc((void**)&dd, dirs.size() * sizeof(double)));
  cudaError_t e = cudaMemcpyAsync(dd, dirs.data(), dirs.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    long long tot = (long long)h->N * nrhs;
    int grid = (int)std::min<long long>(152 * 16, (tot + 255) / 256);
    k_plane_wave<<<grid, 256, 0, h->stream>>>(h->d_verts, h->d_tris, h->mesh_q, h->mesh_tri[0],
                                               h->mesh_tri[1], h->mesh_fv[0], h->mesh_fv[1],
                                               h->mesh_len, h->N, h->k, dd, nrhs, (cplx*)B);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  cudaFree(dd);
  return e == cudaSuccess ? HM_OK : cuda_status(e);
}

}  // extern "C"
