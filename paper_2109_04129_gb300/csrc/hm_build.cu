// Native set-up: H-matrix build (Sec. II) and GPU Schur-complement scaling
// (Sec. III-A), plus the plane-wave excitation.
//
//  hm_build: RWG basis (one unknown per interior edge, sorted edge keys, T+
//    the lower triangle), octree over edge midpoints (split while > leaf_max,
//    upper half on >= centre, Morton child order, depth-first leaves),
//    non-touching admissibility on integer cell coordinates (Eq. 10 reading;
//    hm_params.eta > 0 adds the min(diam) <= eta dist form on the same integers),
//    dense near blocks filled on the GPU, far blocks by partially pivoted ACA
//    on the GPU (Eq. 11-12) and QR/SVD recompression on the host.
//  hm_compute_scaling: for k in elimination order D_k = Z~_kk, D_k^-1 by
//    Gauss-Jordan with partial pivoting, alpha_kj = -D_k^-1 Z~_kj,
//    Z~_ij += alpha_ki^T Z~_kj (Eq. 16, 21), all FP64 on the GPU; the block
//    pattern keeps every fill-in block (or only near blocks, HM_FILL_NEAR).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <numeric>
#include <stdexcept>
#include <thread>

#include "hm_efie.cuh"
#include "hm_internal.h"
#include "hm_mixed.h"

using namespace hm;

namespace hm {
hm_status upload_values(hm_ctx* h);
hm_status rebuild_schedules(hm_ctx* h);
}

namespace {

typedef std::complex<double> cd;
const int MAX_DEPTH = 21;
const int ACA_RCAP = 128;

// ------------------------------------------------------------------ mesh
struct Rwg {
  std::vector<int> tp, tm, fp, fm;
  std::vector<double> len, cen;   // cen: N x 3 midpoints
};

hm_status build_rwg(const double* V, int nv, const int* T, int nt, Rwg& r) {
  struct E { long long key; int t, k; };
  std::vector<E> es;
  es.reserve((size_t)nt * 3);
  for (int t = 0; t < nt; ++t) {
    for (int k = 0; k < 3; ++k) {
      int a = T[3 * t + (k + 1) % 3], b = T[3 * t + (k + 2) % 3];
      if (a < 0 || b < 0 || a >= nv || b >= nv || a == b) return HM_ERR_INVALID;
      int lo = std::min(a, b), hi = std::max(a, b);
      es.push_back(E{(long long)lo * nv + hi, t, k});
    }
  }
  std::sort(es.begin(), es.end(), [](const E& x, const E& y) {
    if (x.key != y.key) return x.key < y.key;
    if (x.t != y.t) return x.t < y.t;
    return x.k < y.k;
  });
  for (size_t i = 0; i < es.size();) {
    size_t j = i;
    while (j < es.size() && es[j].key == es[i].key) ++j;
    if (j - i > 2) return HM_ERR_INVALID;   // non-manifold edge
    if (j - i == 2) {
      int a = (int)(es[i].key / nv), b = (int)(es[i].key % nv);
      r.tp.push_back(es[i].t);
      r.fp.push_back(es[i].k);
      r.tm.push_back(es[i + 1].t);
      r.fm.push_back(es[i + 1].k);
      double dx = V[3 * a] - V[3 * b], dy = V[3 * a + 1] - V[3 * b + 1],
             dz = V[3 * a + 2] - V[3 * b + 2];
      r.len.push_back(std::sqrt(dx * dx + dy * dy + dz * dz));
      for (int c = 0; c < 3; ++c) r.cen.push_back(0.5 * (V[3 * a + c] + V[3 * b + c]));
    }
    i = j;
  }
  for (int t = 0; t < nt; ++t) {
    const double* a = V + 3 * T[3 * t];
    const double* b = V + 3 * T[3 * t + 1];
    const double* c = V + 3 * T[3 * t + 2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2],
           n2 = u[0] * w[1] - u[1] * w[0];
    double e2 = std::max(u[0] * u[0] + u[1] * u[1] + u[2] * u[2],
                         w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    // degenerate triangle: area below 1e-10 of its longest-edge square
    if (!(n0 * n0 + n1 * n1 + n2 * n2 > 1e-20 * e2 * e2)) return HM_ERR_INVALID;
  }
  return r.tp.empty() ? HM_ERR_INVALID : HM_OK;
}

// ------------------------------------------------------------------ octree
struct Node {
  int level, ijk[3];
  long long start, count;
  std::vector<int> children;
  int leaf = -1;
};

struct Octree {
  std::vector<Node> nodes;
  std::vector<long long> perm;
  std::vector<int> leaves;
  double origin[3], size;
  const double* pts;
  int leaf_max;
  double eta = 0.0;       // admissibility constant of Eq. 10 (0: non-touching)

  int build(std::vector<int>& idx, int level, const int ijk[3]) {
    int nid = (int)nodes.size();
    nodes.push_back(Node());
    nodes[nid].level = level;
    for (int a = 0; a < 3; ++a) nodes[nid].ijk[a] = ijk[a];
    nodes[nid].start = (long long)perm.size();
    nodes[nid].count = (long long)idx.size();
    if ((int)idx.size() <= leaf_max || level >= MAX_DEPTH) {
      nodes[nid].leaf = (int)leaves.size();
      leaves.push_back(nid);
      for (int i : idx) perm.push_back(i);
      return nid;
    }
    double cell = size / (double)(1LL << level);
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = origin[a] + ((double)ijk[a] + 0.5) * cell;
    std::vector<int> b[8];
    for (int i : idx) {
      const double* p = pts + 3 * (size_t)i;
      int q = (p[0] >= c[0] ? 1 : 0) | (p[1] >= c[1] ? 2 : 0) | (p[2] >= c[2] ? 4 : 0);
      b[q].push_back(i);
    }
    std::vector<int>().swap(idx);
    for (int q = 0; q < 8; ++q) {
      if (b[q].empty()) continue;
      int cijk[3] = {2 * ijk[0] + (q & 1), 2 * ijk[1] + ((q >> 1) & 1), 2 * ijk[2] + ((q >> 2) & 1)};
      int ch = build(b[q], level + 1, cijk);
      nodes[nid].children.push_back(ch);
    }
    return nid;
  }

  bool touching(int s, int t) const {
    const Node& a = nodes[s];
    const Node& b = nodes[t];
    long long sa = 1LL << (MAX_DEPTH - a.level), sb = 1LL << (MAX_DEPTH - b.level);
    for (int ax = 0; ax < 3; ++ax) {
      long long la = a.ijk[ax] * sa, ha = (a.ijk[ax] + 1) * sa;
      long long lb = b.ijk[ax] * sb, hb = (b.ijk[ax] + 1) * sb;
      if (la > hb || lb > ha) return false;
    }
    return true;
  }
  // far pair: the cells do not touch and, for eta > 0, min(diam) <= eta dist
  // (Eq. 10; diam = sqrt 3 edge, dist = distance between the cubes), tested
  // as 3 min(edge)^2 <= eta^2 sum(gap^2) in units of the finest cell (the
  // squares are exact integers, so ties such as a one-cell diagonal gap at
  // eta = 1 fall on the far side on every machine)
  bool admissible(int s, int t) const {
    if (touching(s, t)) return false;
    if (!(eta > 0.0)) return true;
    const Node& a = nodes[s];
    const Node& b = nodes[t];
    long long sa = 1LL << (MAX_DEPTH - a.level), sb = 1LL << (MAX_DEPTH - b.level);
    long long D = 0;
    for (int ax = 0; ax < 3; ++ax) {
      long long la = a.ijk[ax] * sa, ha = (a.ijk[ax] + 1) * sa;
      long long lb = b.ijk[ax] * sb, hb = (b.ijk[ax] + 1) * sb;
      long long g = std::max(0LL, std::max(lb - ha, la - hb));
      D += g * g;
    }
    const double m = (double)std::min(sa, sb);
    return 3.0 * m * m <= (eta * eta) * (double)D;
  }
};

void make_octree(const std::vector<double>& cen, int leaf_max, double eta, Octree& T) {
  int N = (int)(cen.size() / 3);
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    lo[a] = hi[a] = cen[a];
    for (int i = 1; i < N; ++i) {
      lo[a] = std::min(lo[a], cen[3 * i + a]);
      hi[a] = std::max(hi[a], cen[3 * i + a]);
    }
  }
  double half = 0.0;
  double ctr[3];
  for (int a = 0; a < 3; ++a) {
    ctr[a] = (lo[a] + hi[a]) / 2.0;
    half = std::max(half, hi[a] - lo[a]);
  }
  half = half / 2.0;
  if (half == 0.0) half = 1.0;
  for (int a = 0; a < 3; ++a) T.origin[a] = ctr[a] - half;
  T.size = 2.0 * half;
  T.pts = cen.data();
  T.leaf_max = leaf_max;
  T.eta = eta;
  std::vector<int> idx(N);
  std::iota(idx.begin(), idx.end(), 0);
  int z[3] = {0, 0, 0};
  T.build(idx, 0, z);
}

// ------------------------------------------------------------------ kernels
struct FillJob { int i, j; long long off; };   // near block (leaf i, leaf j) -> offset

__global__ void k_fill_near(MeshDev M, const FillJob* jobs, const long long* leaf_off,
                            const int* perm, cplx* out) {
  FillJob jb = jobs[blockIdx.x];
  int r0 = (int)leaf_off[jb.i], mi = (int)(leaf_off[jb.i + 1] - r0);
  int c0 = (int)leaf_off[jb.j], mj = (int)(leaf_off[jb.j + 1] - c0);
  for (int e = threadIdx.x; e < mi * mj; e += blockDim.x) {
    int r = e / mj, c = e % mj;
    out[jb.off + e] = efie_entry(M, perm[r0 + r], perm[c0 + c]);
  }
}

__global__ void k_symmetrize(const FillJob* jobs, const long long* leaf_off, cplx* out) {
  FillJob jb = jobs[blockIdx.x];
  if (jb.i != jb.j) return;
  int m = (int)(leaf_off[jb.i + 1] - leaf_off[jb.i]);
  cplx* B = out + jb.off;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    int r = e / m, c = e % m;
    if (r < c) {
      cplx a = B[r * m + c], b = B[c * m + r];
      cplx s = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y + b.y));
      B[r * m + c] = s;
      B[c * m + r] = s;
    }
  }
}

// Dense Z[rows][cols] for a far block kept dense.
__global__ void k_fill_dense(MeshDev M, const int* perm, int r0, int m, int c0, int n, cplx* out) {
  long long tot = (long long)m * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    int r = (int)(e / n), c = (int)(e % n);
    out[e] = efie_entry(M, perm[r0 + r], perm[c0 + c]);
  }
}

struct AcaJob {
  int r0, m, c0, n, maxr;
  long long u_off, v_off, flag_off;   // U: maxr x m (vector l contiguous), V: maxr x n
};

__device__ __forceinline__ double cabs2(cplx a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Block-wide argmax of val over index (ties -> lowest index); val < 0 = excluded.
__device__ void block_argmax(double val, int idx, double* sv, int* si, double* out_v, int* out_i) {
  int t = threadIdx.x;
  sv[t] = val;
  si[t] = idx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) {
      double a = sv[t], b = sv[t + w];
      int ia = si[t], ib = si[t + w];
      if (b > a || (b == a && ib < ia)) { sv[t] = b; si[t] = ib; }
    }
    __syncthreads();
  }
  *out_v = sv[0];
  *out_i = si[0];
  __syncthreads();
}

__device__ double block_sum(double v, double* sv) {
  int t = threadIdx.x;
  sv[t] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) sv[t] += sv[t + w];
    __syncthreads();
  }
  double r = sv[0];
  __syncthreads();
  return r;
}

// Partially pivoted ACA of one far block per CTA (same steps as the CPU
// statement: first row 0, pivot column = argmax |row residual|, next row =
// argmax |u| over unused rows, incremental Frobenius norm, stop when
// |u||v| <= eps ||S||).  Writes the rank (or -1 when the rank cap is reached
// unconverged) to ranks[b].
__global__ void __launch_bounds__(256) k_aca(MeshDev M, const AcaJob* jobs, const int* perm,
                                             cplx* U, cplx* Vv, char* used_all, double eps,
                                             int* ranks) {
  __shared__ double sv[256];
  __shared__ int si[256];
  const AcaJob jb = jobs[blockIdx.x];
  cplx* Ub = U + jb.u_off;
  cplx* Vb = Vv + jb.v_off;
  char* used = used_all + jb.flag_off;
  for (int i = threadIdx.x; i < jb.m; i += blockDim.x) used[i] = 0;
  __syncthreads();
  int rank = 0, i = 0;
  double norm2 = 0.0;
  bool converged = false;
  while (rank < jb.maxr) {
    if (threadIdx.x == 0) used[i] = 1;
    // residual row i -> tentative V[rank]
    double bv = -1.0;
    int bi = 0x7fffffff;
    for (int c = threadIdx.x; c < jb.n; c += blockDim.x) {
      cplx r = efie_entry(M, perm[jb.r0 + i], perm[jb.c0 + c]);
      for (int l = 0; l < rank; ++l) {
        cplx p = cmul(Ub[(long long)l * jb.m + i], Vb[(long long)l * jb.n + c]);
        r.x -= p.x;
        r.y -= p.y;
      }
      Vb[(long long)rank * jb.n + c] = r;
      double a = cabs2(r);
      if (a > bv) { bv = a; bi = c; }
    }
    double mv;
    int j;
    block_argmax(bv, bi, sv, si, &mv, &j);
    if (mv == 0.0) {
      // zero residual row: lowest unused row next
      int nx = 0x7fffffff;
      for (int q = threadIdx.x; q < jb.m; q += blockDim.x)
        if (!used[q]) nx = min(nx, q);
      double dummy;
      int lowest;
      block_argmax(nx == 0x7fffffff ? -1.0 : 1.0, nx, sv, si, &dummy, &lowest);
      if (dummy < 0.0) { converged = true; break; }
      i = lowest;
      continue;
    }
    cplx piv = Vb[(long long)rank * jb.n + j];
    double pn = cabs2(piv);
    cplx pinv = make_double2(piv.x / pn, -piv.y / pn);
    __syncthreads();
    double nv2p = 0.0;
    for (int c = threadIdx.x; c < jb.n; c += blockDim.x) {
      cplx v = cmul(Vb[(long long)rank * jb.n + c], pinv);
      Vb[(long long)rank * jb.n + c] = v;
      nv2p += cabs2(v);
    }
    __syncthreads();
    // residual column j -> U[rank]
    double nu2p = 0.0;
    for (int q = threadIdx.x; q < jb.m; q += blockDim.x) {
      cplx u = efie_entry(M, perm[jb.r0 + q], perm[jb.c0 + j]);
      for (int l = 0; l < rank; ++l) {
        cplx p = cmul(Vb[(long long)l * jb.n + j], Ub[(long long)l * jb.m + q]);
        u.x -= p.x;
        u.y -= p.y;
      }
      Ub[(long long)rank * jb.m + q] = u;
      nu2p += cabs2(u);
    }
    __syncthreads();
    double nu2 = block_sum(nu2p, sv);
    double nv2 = block_sum(nv2p, sv);
    double cross = 0.0;
    for (int l = 0; l < rank; ++l) {
      // (u_l^H u)(conj(v_l^H v))
      double ur = 0, ui = 0, vr = 0, vi = 0;
      for (int q = threadIdx.x; q < jb.m; q += blockDim.x) {
        cplx a = Ub[(long long)l * jb.m + q], b = Ub[(long long)rank * jb.m + q];
        ur += a.x * b.x + a.y * b.y;
        ui += a.x * b.y - a.y * b.x;
      }
      for (int c = threadIdx.x; c < jb.n; c += blockDim.x) {
        cplx a = Vb[(long long)l * jb.n + c], b = Vb[(long long)rank * jb.n + c];
        vr += a.x * b.x + a.y * b.y;
        vi += a.x * b.y - a.y * b.x;
      }
      ur = block_sum(ur, sv);
      ui = block_sum(ui, sv);
      vr = block_sum(vr, sv);
      vi = block_sum(vi, sv);
      // Re[(ur + i ui) * (vr - i vi)] = ur vr + ui vi
      cross += 2.0 * (ur * vr + ui * vi);
    }
    norm2 = norm2 + cross + nu2 * nv2;
    ++rank;
    if (sqrt(nu2 * nv2) <= eps * sqrt(fmax(norm2, 0.0))) { converged = true; break; }
    // next row: argmax |u| over unused rows
    double bu = -1.0;
    int bq = 0x7fffffff;
    for (int q = threadIdx.x; q < jb.m; q += blockDim.x) {
      if (used[q]) continue;
      double a = cabs2(Ub[(long long)(rank - 1) * jb.m + q]);
      if (a > bu) { bu = a; bq = q; }
    }
    double mu;
    int nq;
    block_argmax(bu, bq, sv, si, &mu, &nq);
    if (mu < 0.0) { converged = true; break; }
    i = nq;
  }
  if (threadIdx.x == 0) ranks[blockIdx.x] = (converged || rank == min(jb.m, jb.n)) ? rank : -1;
}

// ------------------------------------------------------------------ host linear algebra
// Householder QR of A (m x r, column-major): returns Q (m x r) and R (r x r).
void house_qr(int m, int r, std::vector<cd>& A, std::vector<cd>& Q, std::vector<cd>& R) {
  std::vector<std::vector<cd>> vs;
  std::vector<cd> taus;
  for (int c = 0; c < r; ++c) {
    double nrm = 0;
    for (int i = c; i < m; ++i) nrm += std::norm(A[(size_t)c * m + i]);
    nrm = std::sqrt(nrm);
    std::vector<cd> v(m, 0.0);
    cd x0 = A[(size_t)c * m + c];
    cd alpha = (std::abs(x0) > 0 ? -x0 / std::abs(x0) : cd(-1.0)) * nrm;
    for (int i = c; i < m; ++i) v[i] = A[(size_t)c * m + i];
    v[c] -= alpha;
    double vn = 0;
    for (int i = c; i < m; ++i) vn += std::norm(v[i]);
    if (vn > 0) {
      for (int cc = c; cc < r; ++cc) {
        cd s = 0;
        for (int i = c; i < m; ++i) s += std::conj(v[i]) * A[(size_t)cc * m + i];
        s *= 2.0 / vn;
        for (int i = c; i < m; ++i) A[(size_t)cc * m + i] -= s * v[i];
      }
    }
    vs.push_back(v);
    taus.push_back(vn > 0 ? cd(2.0 / vn) : cd(0.0));
  }
  R.assign((size_t)r * r, 0.0);
  for (int c = 0; c < r; ++c)
    for (int i = 0; i <= c; ++i) R[(size_t)c * r + i] = A[(size_t)c * m + i];
  Q.assign((size_t)m * r, 0.0);
  for (int c = 0; c < r; ++c) Q[(size_t)c * m + c] = 1.0;
  for (int c = r - 1; c >= 0; --c) {
    const std::vector<cd>& v = vs[c];
    for (int cc = 0; cc < r; ++cc) {
      cd s = 0;
      for (int i = c; i < m; ++i) s += std::conj(v[i]) * Q[(size_t)cc * m + i];
      s *= taus[c];
      for (int i = c; i < m; ++i) Q[(size_t)cc * m + i] -= s * v[i];
    }
  }
}

// One-sided Jacobi SVD of M (r x r, column-major): M = W diag(s) Y^H, s descending.
void jacobi_svd(int r, std::vector<cd> M, std::vector<cd>& W, std::vector<double>& s,
                std::vector<cd>& Y) {
  Y.assign((size_t)r * r, 0.0);
  for (int i = 0; i < r; ++i) Y[(size_t)i * r + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < r - 1; ++p)
      for (int q = p + 1; q < r; ++q) {
        double a = 0, b = 0;
        cd g = 0;
        for (int i = 0; i < r; ++i) {
          cd mp = M[(size_t)p * r + i], mq = M[(size_t)q * r + i];
          a += std::norm(mp);
          b += std::norm(mq);
          g += std::conj(mp) * mq;
        }
        double ag = std::abs(g);
        if (ag == 0.0 || ag <= 1e-15 * std::sqrt(a * b)) continue;
        off = std::max(off, ag / std::sqrt(a * b));
        double zeta = (b - a) / (2.0 * ag);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        cd e = g / ag;   // phase
        for (int i = 0; i < r; ++i) {
          cd mp = M[(size_t)p * r + i], mq = M[(size_t)q * r + i];
          M[(size_t)p * r + i] = c * mp - sn * std::conj(e) * mq;
          M[(size_t)q * r + i] = sn * e * mp + c * mq;
          cd yp = Y[(size_t)p * r + i], yq = Y[(size_t)q * r + i];
          Y[(size_t)p * r + i] = c * yp - sn * std::conj(e) * yq;
          Y[(size_t)q * r + i] = sn * e * yp + c * yq;
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<double> nrm(r);
  for (int c = 0; c < r; ++c) {
    double a = 0;
    for (int i = 0; i < r; ++i) a += std::norm(M[(size_t)c * r + i]);
    nrm[c] = std::sqrt(a);
  }
  std::vector<int> ord(r);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  W.assign((size_t)r * r, 0.0);
  s.assign(r, 0.0);
  std::vector<cd> Y2((size_t)r * r);
  for (int c = 0; c < r; ++c) {
    int o = ord[c];
    s[c] = nrm[o];
    for (int i = 0; i < r; ++i) {
      W[(size_t)c * r + i] = nrm[o] > 0 ? M[(size_t)o * r + i] / nrm[o] : cd(0.0);
      Y2[(size_t)c * r + i] = Y[(size_t)o * r + i];
    }
  }
  Y.swap(Y2);
}

// Recompress U (m x r) V (n x r) (column-major vectors) at eps; output row-major
// U' (m x r') and V' (n x r') with block = U' V'^T.
int recompress(int m, int n, int r, const cplx* Ucol, const cplx* Vcol, double eps,
               std::vector<cplx>& Uo, std::vector<cplx>& Vo) {
  if (r == 0) { Uo.clear(); Vo.clear(); return 0; }
  std::vector<cd> A((size_t)m * r), B((size_t)n * r);
  for (size_t e = 0; e < A.size(); ++e) A[e] = cd(Ucol[e].x, Ucol[e].y);
  for (size_t e = 0; e < B.size(); ++e) B[e] = cd(Vcol[e].x, Vcol[e].y);
  std::vector<cd> Qu, Ru, Qv, Rv;
  house_qr(m, r, A, Qu, Ru);
  house_qr(n, r, B, Qv, Rv);
  std::vector<cd> M((size_t)r * r, 0.0);   // Ru Rv^T
  for (int c = 0; c < r; ++c)
    for (int i = 0; i < r; ++i) {
      cd s = 0;
      for (int l = 0; l < r; ++l) s += Ru[(size_t)l * r + i] * Rv[(size_t)l * r + c];
      M[(size_t)c * r + i] = s;
    }
  std::vector<cd> W, Y;
  std::vector<double> sv;
  jacobi_svd(r, M, W, sv, Y);
  int keep = 0;
  if (sv[0] > 0)
    for (int c = 0; c < r; ++c) keep += (sv[c] >= eps * sv[0]) ? 1 : 0;
  Uo.assign((size_t)m * keep, make_double2(0, 0));
  Vo.assign((size_t)n * keep, make_double2(0, 0));
  for (int c = 0; c < keep; ++c) {
    for (int i = 0; i < m; ++i) {
      cd s = 0;
      for (int l = 0; l < r; ++l) s += Qu[(size_t)l * m + i] * W[(size_t)c * r + l];
      s *= sv[c];
      Uo[(size_t)i * keep + c] = make_double2(s.real(), s.imag());
    }
    for (int i = 0; i < n; ++i) {
      cd s = 0;   // V' = Q_V conj(Y)
      for (int l = 0; l < r; ++l) s += Qv[(size_t)l * n + i] * std::conj(Y[(size_t)c * r + l]);
      Vo[(size_t)i * keep + c] = make_double2(s.real(), s.imag());
    }
  }
  return keep;
}

template <class T>
hm_status dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  HM_CUDA(cudaMalloc((void**)p, n * sizeof(T)));
  return HM_OK;
}
template <class T>
hm_status h2d(T** p, const std::vector<T>& v) {
  hm_status s = dalloc(p, v.size());
  if (s) return s;
  if (!v.empty()) HM_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HM_OK;
}

struct MeshStore {
  double* V = nullptr;
  int* T = nullptr;
  double* Q = nullptr;
  double* area = nullptr;
  int* tri[2] = {nullptr, nullptr};
  int* fv[2] = {nullptr, nullptr};
  double* len = nullptr;
  int* perm = nullptr;
  long long* leaf_off = nullptr;
  void release() {
    cudaFree(V); cudaFree(T); cudaFree(Q); cudaFree(area);
    for (int i = 0; i < 2; ++i) { cudaFree(tri[i]); cudaFree(fv[i]); }
    cudaFree(len); cudaFree(perm); cudaFree(leaf_off);
  }
};

// quadrature points as (b0 v0 + b1 v1) + b2 v2 with the 7-point barycentric set
void quad_points(const std::vector<double>& V, const std::vector<int>& T, std::vector<double>& Q) {
  const double s15 = std::sqrt(15.0);
  const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
  double bary[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                       {a1, a1, 1 - 2 * a1}, {a1, 1 - 2 * a1, a1}, {1 - 2 * a1, a1, a1},
                       {a2, a2, 1 - 2 * a2}, {a2, 1 - 2 * a2, a2}, {1 - 2 * a2, a2, a2}};
  size_t nt = T.size() / 3;
  Q.resize(nt * 21);
  for (size_t t = 0; t < nt; ++t)
    for (int q = 0; q < 7; ++q)
      for (int c = 0; c < 3; ++c) {
        double v0 = V[3 * T[3 * t] + c], v1 = V[3 * T[3 * t + 1] + c], v2 = V[3 * T[3 * t + 2] + c];
        Q[t * 21 + q * 3 + c] = (bary[q][0] * v0 + bary[q][1] * v1) + bary[q][2] * v2;
      }
}

}  // namespace

// ====================================================================== API
extern "C" {

hm_status hm_build(const double* verts, int nv, const int* tris, int nt, const hm_params* p,
                   hm_handle* out) {
  if (!verts || !tris || !out || nv < 3 || nt < 2) return HM_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return HM_ERR_CUDA;
  hm_ctx* h = nullptr;
  MeshStore ms;
  try {
    h = new hm_ctx();
    if (p) h->p = *p; else hm_default_params(&h->p);
    if (h->p.freq_hz > 0) h->p.wavelength = 299792458.0 / h->p.freq_hz;
    if (h->p.leaf_max < 1 || !(h->p.wavelength > 0) || !(h->p.aca_tol > 0) ||
        !(h->p.eta >= 0) || !(h->p.freq_hz >= 0))
      throw HM_ERR_INVALID;
    cudaGetDevice(&h->dev);
    Rwg rw;
    hm_status s = build_rwg(verts, nv, tris, nt, rw);
    if (s) throw s;
    const int N = (int)rw.tp.size();
    h->N = N;
    h->wavelength = h->p.wavelength;
    h->k = 2.0 * 3.141592653589793 / h->p.wavelength;
    Octree T;
    make_octree(rw.cen, h->p.leaf_max, h->p.eta, T);
    // block partition from (root, root)
    std::vector<std::pair<int, int>> near, far;
    std::vector<std::pair<int, int>> st{{0, 0}};
    while (!st.empty()) {
      auto pr = st.back();
      st.pop_back();
      int a = pr.first, b = pr.second;
      if (T.admissible(a, b)) { far.push_back(pr); continue; }
      const Node& na = T.nodes[a];
      const Node& nb = T.nodes[b];
      if (na.leaf >= 0 && nb.leaf >= 0) near.push_back({na.leaf, nb.leaf});
      else if (na.leaf >= 0) for (int c : nb.children) st.push_back({a, c});
      else if (nb.leaf >= 0) for (int c : na.children) st.push_back({c, b});
      else for (int c : na.children) for (int d : nb.children) st.push_back({c, d});
    }
    // leaf storage order: depth first (every octree node a contiguous range)
    int nl = (int)T.leaves.size();
    h->leaf_off.assign(nl + 1, 0);
    for (int l = 0; l < nl; ++l) h->leaf_off[l] = T.nodes[T.leaves[l]].start;
    h->leaf_off[nl] = N;
    h->perm = T.perm;
    h->nl = nl;
    h->m.resize(nl);
    for (int q = 0; q < nl; ++q) h->m[q] = (int)(h->leaf_off[q + 1] - h->leaf_off[q]);
    h->leaf_cen.resize(3 * (size_t)nl);
    for (int l = 0; l < nl; ++l) {
      const Node& nd = T.nodes[T.leaves[l]];
      for (int a = 0; a < 3; ++a)
        h->leaf_cen[3 * l + a] = (nd.ijk[a] + 0.5) / (double)(1LL << nd.level);
    }
    struct FB { long long r0, m, c0, n; };
    std::vector<FB> fbs;
    for (auto& e : far) {
      const Node& a = T.nodes[e.first];
      const Node& b = T.nodes[e.second];
      if (a.start < b.start) fbs.push_back(FB{a.start, a.count, b.start, b.count});
    }
    std::sort(fbs.begin(), fbs.end(), [](const FB& x, const FB& y) {
      if (x.r0 != y.r0) return x.r0 < y.r0;
      if (x.c0 != y.c0) return x.c0 < y.c0;
      if (x.m != y.m) return x.m < y.m;
      return x.n < y.n;
    });
    std::vector<std::pair<int, int>> nu;
    for (auto& e : near)
      if (e.first <= e.second) nu.push_back(e);
    std::sort(nu.begin(), nu.end());
    nu.erase(std::unique(nu.begin(), nu.end()), nu.end());
    // ---- device mesh
    std::vector<double> Vh(verts, verts + 3 * (size_t)nv);
    std::vector<int> Th(tris, tris + 3 * (size_t)nt);
    std::vector<double> Qh, area(nt);
    quad_points(Vh, Th, Qh);
    for (int t = 0; t < nt; ++t) {
      const double* a = verts + 3 * tris[3 * t];
      const double* b = verts + 3 * tris[3 * t + 1];
      const double* c = verts + 3 * tris[3 * t + 2];
      double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
      double n0 = u[1] * w[2] - u[2] * w[1], n1 = u[2] * w[0] - u[0] * w[2],
             n2 = u[0] * w[1] - u[1] * w[0];
      area[t] = 0.5 * std::sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    }
    std::vector<int> perm32(h->perm.begin(), h->perm.end());
    if ((s = h2d(&ms.V, Vh)) || (s = h2d(&ms.T, Th)) || (s = h2d(&ms.Q, Qh)) ||
        (s = h2d(&ms.area, area)) || (s = h2d(&ms.tri[0], rw.tp)) || (s = h2d(&ms.tri[1], rw.tm)) ||
        (s = h2d(&ms.fv[0], rw.fp)) || (s = h2d(&ms.fv[1], rw.fm)) || (s = h2d(&ms.len, rw.len)) ||
        (s = h2d(&ms.perm, perm32)) || (s = h2d(&ms.leaf_off, h->leaf_off)))
      throw s;
    MeshDev M;
    M.V = ms.V; M.T = ms.T; M.Q = ms.Q; M.area = ms.area;
    M.tri[0] = ms.tri[0]; M.tri[1] = ms.tri[1]; M.fv[0] = ms.fv[0]; M.fv[1] = ms.fv[1];
    M.len = ms.len; M.k = h->k;
    M.eta = 4e-7 * 3.141592653589793 * 299792458.0;
    // ---- near blocks
    std::vector<FillJob> fj;
    long long ne = 0;
    for (auto& e : nu) {
      fj.push_back(FillJob{e.first, e.second, ne});
      h->near.push_back(NearDesc{e.first, e.second, ne});
      ne += (long long)h->m[e.first] * h->m[e.second];
    }
    FillJob* d_fj = nullptr;
    if ((s = h2d(&d_fj, fj))) throw s;
    if ((s = dalloc(&h->d_near, (size_t)ne))) { cudaFree(d_fj); throw s; }
    k_fill_near<<<(unsigned)fj.size(), 256>>>(M, d_fj, ms.leaf_off, ms.perm, h->d_near);
    k_symmetrize<<<(unsigned)fj.size(), 256>>>(d_fj, ms.leaf_off, h->d_near);
    cudaError_t ce = cudaDeviceSynchronize();
    cudaFree(d_fj);
    if (ce != cudaSuccess) throw cuda_status(ce);
    h->h_near.resize(ne);
    HM_CUDA(cudaMemcpy(h->h_near.data(), h->d_near, ne * sizeof(cplx), cudaMemcpyDeviceToHost));
    // ---- far blocks: ACA in batches that fit a scratch budget
    const size_t budget = (size_t)2 << 30;   // bytes of U/V scratch per batch
    std::vector<int> ranks(fbs.size(), 0);
    std::vector<std::vector<cplx>> fu(fbs.size()), fv(fbs.size());
    std::vector<int> fr(fbs.size(), 0), dense(fbs.size(), 0);
    size_t b0 = 0;
    while (b0 < fbs.size()) {
      std::vector<AcaJob> jobs;
      long long uo = 0, vo = 0, fo = 0;
      size_t b1 = b0;
      while (b1 < fbs.size()) {
        const FB& f = fbs[b1];
        int maxr = (int)std::min<long long>(std::min(f.m, f.n), ACA_RCAP);
        size_t need = (size_t)maxr * (f.m + f.n) * sizeof(cplx);
        if (!jobs.empty() && (size_t)(uo + vo) * sizeof(cplx) + need > budget) break;
        jobs.push_back(AcaJob{(int)f.r0, (int)f.m, (int)f.c0, (int)f.n, maxr, uo, vo, fo});
        uo += (long long)maxr * f.m;
        vo += (long long)maxr * f.n;
        fo += f.m;
        ++b1;
      }
      AcaJob* d_jobs = nullptr;
      cplx *dU = nullptr, *dV = nullptr;
      char* dflag = nullptr;
      int* d_rank = nullptr;
      if ((s = h2d(&d_jobs, jobs)) || (s = dalloc(&dU, (size_t)uo)) || (s = dalloc(&dV, (size_t)vo)) ||
          (s = dalloc(&dflag, (size_t)fo)) || (s = dalloc(&d_rank, jobs.size()))) {
        cudaFree(d_jobs); cudaFree(dU); cudaFree(dV); cudaFree(dflag); cudaFree(d_rank);
        throw s;
      }
      k_aca<<<(unsigned)jobs.size(), 256>>>(M, d_jobs, ms.perm, dU, dV, dflag, h->p.aca_tol, d_rank);
      ce = cudaDeviceSynchronize();
      std::vector<cplx> hU, hV;
      std::vector<int> hr(jobs.size());
      if (ce == cudaSuccess) {
        hU.resize(uo);
        hV.resize(vo);
        ce = cudaMemcpy(hU.data(), dU, uo * sizeof(cplx), cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess) ce = cudaMemcpy(hV.data(), dV, vo * sizeof(cplx), cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess)
          ce = cudaMemcpy(hr.data(), d_rank, hr.size() * sizeof(int), cudaMemcpyDeviceToHost);
      }
      cudaFree(d_jobs); cudaFree(dU); cudaFree(dV); cudaFree(dflag); cudaFree(d_rank);
      if (ce != cudaSuccess) throw cuda_status(ce);
      // host recompression in parallel
      unsigned nthr = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
      std::vector<std::thread> pool;
      for (unsigned w = 0; w < nthr; ++w)
        pool.emplace_back([&, w]() {
          for (size_t q = w; q < jobs.size(); q += nthr) {
            const AcaJob& jb = jobs[q];
            size_t bi = b0 + q;
            int r = hr[q];
            if (r < 0) { dense[bi] = 1; continue; }
            fr[bi] = recompress(jb.m, jb.n, r, hU.data() + jb.u_off, hV.data() + jb.v_off,
                                h->p.aca_tol, fu[bi], fv[bi]);
            if ((long long)fr[bi] * (jb.m + jb.n) >= (long long)jb.m * jb.n) dense[bi] = 1;
          }
        });
      for (auto& t : pool) t.join();
      b0 = b1;
    }
    for (size_t bi = 0; bi < fbs.size(); ++bi) {
      const FB& f = fbs[bi];
      FarDesc d{dense[bi], (int)f.r0, (int)f.m, (int)f.c0, (int)f.n, dense[bi] ? 0 : fr[bi], 0, 0};
      d.offU = (long long)h->h_far.size();
      if (!dense[bi]) {
        d.offV = d.offU + f.m * d.rank;
        h->h_far.insert(h->h_far.end(), fu[bi].begin(), fu[bi].end());
        h->h_far.insert(h->h_far.end(), fv[bi].begin(), fv[bi].end());
        std::vector<cplx>().swap(fu[bi]);
        std::vector<cplx>().swap(fv[bi]);
      } else {
        cplx* dB = nullptr;
        if ((s = dalloc(&dB, (size_t)(f.m * f.n)))) throw s;
        k_fill_dense<<<std::max<long long>(1, std::min<long long>(4096, (f.m * f.n + 255) / 256)), 256>>>(
            M, ms.perm, (int)f.r0, (int)f.m, (int)f.c0, (int)f.n, dB);
        h->h_far.resize(h->h_far.size() + f.m * f.n);
        ce = cudaMemcpy(h->h_far.data() + d.offU, dB, f.m * f.n * sizeof(cplx), cudaMemcpyDeviceToHost);
        cudaFree(dB);
        if (ce != cudaSuccess) throw cuda_status(ce);
      }
      h->far.push_back(d);
    }
    HM_CUDA(cudaMalloc((void**)&h->d_far, std::max<size_t>(1, h->h_far.size()) * sizeof(cplx)));
    if (!h->h_far.empty())
      HM_CUDA(cudaMemcpy(h->d_far, h->h_far.data(), h->h_far.size() * sizeof(cplx), cudaMemcpyHostToDevice));
    h->dev_bytes += (ne + h->h_far.size()) * sizeof(cplx);
    // keep the mesh for the plane-wave RHS
    h->d_verts = ms.V; ms.V = nullptr;
    h->d_tris = ms.T; ms.T = nullptr;
    h->verts = Vh;
    h->tris = Th;
    h->mesh_q = ms.Q; ms.Q = nullptr;
    h->mesh_area = ms.area; ms.area = nullptr;
    h->mesh_tri[0] = ms.tri[0]; h->mesh_tri[1] = ms.tri[1];
    h->mesh_fv[0] = ms.fv[0]; h->mesh_fv[1] = ms.fv[1];
    h->mesh_len = ms.len;
    ms.tri[0] = ms.tri[1] = ms.fv[0] = ms.fv[1] = nullptr;
    ms.len = nullptr;
    h->d_perm = ms.perm; ms.perm = nullptr;
    ms.release();
    if ((s = rebuild_schedules(h))) throw s;
    *out = h;
    return HM_OK;
  } catch (hm_status s) {
    ms.release();
    hm_destroy(h);
    return s;
  } catch (std::bad_alloc&) {
    ms.release();
    hm_destroy(h);
    return HM_ERR_OOM;
  } catch (...) {
    ms.release();
    hm_destroy(h);
    return HM_ERR_INVALID;
  }
}

}  // extern "C"
