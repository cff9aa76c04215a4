#include <atomic>
// C ABI of include/hm.h: handle life cycle, block-file import/export, the
// level schedules of the sweeps, and the power-series solve chain.
//
// The solve follows Eq. 25-36 of the paper with R = alpha_1 ... alpha_n:
//   b~ = R^T b  (forward block substitution, Eq. 25)
//   b_o = Z~_N^{-1} b~ (Eq. 32), it_1 = Z~_N^{-1} R^T Z_F R b_o (Eq. 31)
//   x = R (it_0 - it_1 + ...)  (Eq. 26, 36)
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <stdexcept>

#include "hm_internal.h"
#include "hm_mixed.h"

using namespace hm;

namespace hm {

static std::atomic<long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

hm_status cuda_status(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return HM_ERR_OOM;
  return HM_ERR_CUDA;
}

hm_status term_norms(hm_ctx* h, const void* v, bool f32, int nrhs, std::vector<double>& out) {
  double* d = h->d_norms + 4 * (size_t)nrhs;          // the fifth slot of the norm buffer
  hm_status s = f32 ? launch_col_norms2_32((const float2*)v, h->N, nrhs, d, h->stream)
                    : launch_col_norms2((const cplx*)v, h->N, nrhs, d, h->stream);
  if (s) return s;
  out.assign(nrhs, 0.0);
  HM_CUDA(cudaMemcpyAsync(out.data(), d, nrhs * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
  HM_CUDA(cudaStreamSynchronize(h->stream));
  return HM_OK;
}

// Adaptive term count (Sec. III-C, Eq. 44-45), on squared norms: stop after
// the latest term it_t when every RHS has ||it_t|| <= tol ||it_0||, or when
// some RHS has ||it_t|| >= ||it_(t-1)|| > 0 (no longer shrinking).
bool terms_stop(const std::vector<double>& n0, const std::vector<double>& nprev,
                const std::vector<double>& nt, double tol) {
  bool conv = true, grow = false;
  for (size_t r = 0; r < nt.size(); ++r) {
    if (nt[r] > tol * tol * n0[r]) conv = false;
    if (nt[r] > 0.0 && nt[r] >= nprev[r]) grow = true;
  }
  return conv || grow;
}

int prof_begin(hm_ctx* h) {
  if (!h->prof) return -1;
  while (h->evpool.size() < h->evused + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->evpool.push_back(e);
  }
  int ev = (int)h->evused;
  h->evused += 2;
  cudaEventRecord(h->evpool[ev], h->stream);
  return ev;
}

void prof_end(hm_ctx* h, int ev, int cat, double bytes, double flops) {
  if (ev < 0) return;
  cudaEventRecord(h->evpool[ev + 1], h->stream);
  h->recs.push_back(ProfRec{cat, ev, bytes, flops});
}

}  // namespace hm

namespace {

const long long KMAX = 128;   // inner rows per split-K task of a sweep (more CTAs on
                              // the narrow top levels of the elimination tree)
// largest split size of the tensor-core sweeps (the candidates the tuner
// times run from KMAX up to this size).  The split size hardly moves the mixed
// chain's error: on the 2-lambda sphere (one accumulator per task) it was
// 6.1e-5 with splits of at most 128 rows and 6.6e-5 with 2048, because each
// MMA's rounding scales with the partial sum, which is about as large in a
// split as in the whole sum; the error follows the number of MMAs adding into
// one accumulator, which the tensor-core kernel cuts with a separate
// accumulator for the small slice products.
const long long KMAX_TC = 2048;
long long split_cap(const hm_ctx* h) {
  long long c = KMAX_TC;
  if (h->p.tc_split_max >= (int)KMAX) {
    c = KMAX;
    while (c * 2 <= h->p.tc_split_max) c *= 2;
  }
  return c;
}

template <class T>
hm_status upload(T** dptr, const std::vector<T>& v, size_t* bytes) {
  if (*dptr) cudaFree(*dptr);
  *dptr = nullptr;
  if (v.empty()) return HM_OK;
  HM_CUDA(cudaMalloc((void**)dptr, v.size() * sizeof(T)));
  HM_CUDA(cudaMemcpy(*dptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  if (bytes) *bytes += v.size() * sizeof(T);
  return HM_OK;
}

hm_status upload_tasks(TaskList& tl, size_t* bytes) {
  tl.abuf_mask = 0;
  for (const GItem& it : tl.items) tl.abuf_mask |= 1u << it.a_buf;
  hm_status s = upload(&tl.d_tasks, tl.tasks, bytes);
  if (s != HM_OK) return s;
  return upload(&tl.d_items, tl.items, bytes);
}
hm_status upload_fin(FinList& fl, size_t* bytes) {
  hm_status s = upload(&fl.d_tasks, fl.tasks, bytes);
  if (s != HM_OK) return s;
  return upload(&fl.d_slots, fl.slots, bytes);
}
void free_tasks(TaskList& tl) {
  cudaFree(tl.d_tasks);
  cudaFree(tl.d_items);
  cudaFree(tl.d_tiles);
  cudaFree(tl.d_toff);
  cudaFree(tl.d_units);
  cudaFree(tl.d_torder);
  tl.d_torder = nullptr;
  tl.d_units = nullptr;
  tl.n_units = 0;
  tl.d_tasks = nullptr;
  tl.d_items = nullptr;
  tl.d_tiles = nullptr;
  tl.d_toff = nullptr;
  tl.tile_bytes = 0;
}
void free_sweep(Sweep& sw) {
  for (auto& t : sw.part) free_tasks(t);
  for (auto& f : sw.fin) {
    cudaFree(f.d_tasks);
    cudaFree(f.d_slots);
  }
  sw.part.clear();
  sw.fin.clear();
}

// One sweep over the alpha pattern.  forward: b~_j += sum_k alpha_kj^T b~_k
// (targets j, predecessors k < j); backward: x_k += sum_j alpha_kj x_j
// (targets k, successors j > k).  Levels: a target waits for all of its
// sources.  Each target's sources are split into tasks of <= KMAX inner rows
// writing scratch panels; the finalize adds them to the target in place.
void build_sweep(hm_ctx* h, bool forward, Sweep& sw) {
  const int n = h->nl;
  const std::vector<int>& L = h->elim;                          // rank -> leaf
  std::vector<std::vector<std::pair<int, long long>>> src(n);   // (source rank, alpha index)
  for (int k = 0; k < n; ++k) {
    long long base = h->alpha_row_start[k];
    for (size_t q = 0; q < h->rows[k].size(); ++q) {
      int j = h->rows[k][q];
      if (forward)
        src[j].push_back({k, base + (long long)q});
      else
        src[k].push_back({j, base + (long long)q});
    }
  }
  std::vector<int> lev(n, 0);
  int nlev = 0;
  if (forward) {
    for (int j = 0; j < n; ++j) {
      for (auto& s : src[j]) lev[j] = std::max(lev[j], lev[s.first] + 1);
      nlev = std::max(nlev, lev[j] + 1);
    }
  } else {
    for (int k = n - 1; k >= 0; --k) {
      for (auto& s : src[k]) lev[k] = std::max(lev[k], lev[s.first] + 1);
      nlev = std::max(nlev, lev[k] + 1);
    }
  }
  std::vector<std::vector<int>> bylev(nlev);
  for (int t = 0; t < n; ++t) bylev[lev[t]].push_back(t);
  sw.part.assign(nlev, TaskList());
  sw.fin.assign(nlev, FinList());
  int max_scr = 0;
  for (int l = 0; l < nlev; ++l) {
    TaskList& tl = sw.part[l];
    FinList& fl = sw.fin[l];
    int scr_row = 0;
    for (int t : bylev[l]) {
      if (src[t].empty()) continue;
      const int mt = h->m[L[t]];
      FTask ft{VB_OUT, (int)h->leaf_off[L[t]], mt, VB_OUT, (int)h->leaf_off[L[t]],
               (int)fl.slots.size(), 0};
      size_t q = 0;
      while (q < src[t].size()) {
        GTask task{VB_SCR, scr_row, mt, (int)tl.items.size(), 0, 0, 0, 0};
        long long kk = 0;
        while (q < src[t].size() && (kk == 0 || kk + h->m[L[src[t][q].first]] <= KMAX)) {
          int s = L[src[t][q].first];
          long long ai = src[t][q].second;
          GItem it{};
          it.a_off = h->alpha_off[ai];
          // forward over a non-symmetric system: the left coefficient
          // alphaL_st, stored as its transpose in alpha's layout
          it.a_buf = (forward && h->nonsym) ? AB_ALPHAL : AB_ALPHA;
          if (forward) {   // alpha_st is m_s x m_t; need alpha^T: trans read
            it.lda = mt;
            it.trans = 1;
          } else {         // alpha_ts is m_t x m_s
            it.lda = h->m[s];
            it.trans = 0;
          }
          it.k = h->m[s];
          it.in_buf = VB_OUT;
          it.in_row = (int)h->leaf_off[s];
          tl.items.push_back(it);
          tl.flops += (long long)mt * h->m[s];
          tl.a_bytes += (long long)mt * h->m[s] * 16;
          kk += h->m[s];
          ++q;
        }
        task.it1 = (int)tl.items.size();
        tl.tasks.push_back(task);
        fl.slots.push_back(scr_row);
        scr_row += mt;
      }
      ft.s1 = (int)fl.slots.size();
      fl.tasks.push_back(ft);
    }
    max_scr = std::max(max_scr, scr_row);
  }
  sw.scratch_rows = max_scr;
}

// For every task row i: E_i = max over the task's items and inner index of the
// frexp exponent of |re| and |im| of op(A)(i, k), so that |op(A)(i, k)| < 2^E_i.
hm_status row_exponents(hm_ctx* h, const TaskList& tl, RowExp& R) {
  cudaFree(R.d_e);
  cudaFree(R.d_off);
  R = RowExp();
  for (const GTask& t : tl.tasks) {
    R.off.push_back((long long)R.e.size());
    std::vector<int> ex(t.m, -1022);
    for (int q = t.it0; q < t.it1; ++q) {
      const GItem& it = tl.items[q];
      const std::vector<cplx>* src = it.a_buf == AB_NEAR ? &h->h_near
                                     : it.a_buf == AB_FAR ? &h->h_far
                                     : it.a_buf == AB_ALPHA ? &h->h_alpha
                                     : it.a_buf == AB_ALPHAL ? &h->h_alphaL : &h->h_dinv;
      const cplx* A = src->data() + it.a_off;
      // a row segment of a stacked task covers its rows only
      const int i0 = it.nrow > 0 ? it.r0 : 0, i1 = it.nrow > 0 ? it.r0 + it.nrow : t.m;
      for (int i = i0; i < i1; ++i)
        for (int k = 0; k < it.k; ++k) {
          const int li = i - i0;
          cplx a = it.trans ? A[(long long)k * it.lda + li] : A[(long long)li * it.lda + k];
          int e1 = 0, e2 = 0;
          if (a.x != 0.0) { std::frexp(a.x, &e1); ex[i] = std::max(ex[i], e1); }
          if (a.y != 0.0) { std::frexp(a.y, &e2); ex[i] = std::max(ex[i], e2); }
        }
    }
    R.e.insert(R.e.end(), ex.begin(), ex.end());
  }
  if (R.e.empty()) return HM_OK;
  hm_status s = upload(&R.d_e, R.e, &h->dev_bytes);
  if (s) return s;
  return upload(&R.d_off, R.off, &h->dev_bytes);
}

// Split the items of one target into split-K tasks (<= KMAX inner rows each),
// partials into scratch, and add the finalize entry (in place on the target).
void add_target(hm_ctx* h, TaskList& tl, FinList& fl, int& scr_row, int out_row, int mt,
                const std::vector<GItem>& its, long long kmax = KMAX) {
  if (its.empty()) return;
  FTask ft{VB_OUT, out_row, mt, VB_OUT, out_row, (int)fl.slots.size(), 0};
  size_t q = 0;
  while (q < its.size()) {
    GTask task{VB_SCR, scr_row, mt, (int)tl.items.size(), 0, 0, 0, 0};
    long long kk = 0;
    while (q < its.size() && (kk == 0 || kk + its[q].k <= kmax)) {
      tl.items.push_back(its[q]);
      tl.flops += (long long)mt * its[q].k;
      tl.a_bytes += (long long)mt * its[q].k * 16;
      kk += its[q].k;
      ++q;
    }
    task.it1 = (int)tl.items.size();
    tl.tasks.push_back(task);
    fl.slots.push_back(scr_row);
    scr_row += mt;
  }
  ft.s1 = (int)fl.slots.size();
  fl.tasks.push_back(ft);
}

// Sweep over supernodes: groups of consecutive ranks (nested-dissection
// separators and bottom groups).  Per group level: (1) every target adds its
// sources outside its group (alpha blocks, all final), then (2) a multi-leaf
// group G applies T_G = (I - A_G^T)^-1 (forward) or T_G^T (backward): the
// within-group substitution as one dense product.  Same result as the leaf
// substitution; 9 group levels instead of 151 leaf levels on the 2-lambda sphere.
void build_sweep_groups(hm_ctx* h, bool forward, Sweep& sw) {
  const int n = h->nl;
  const std::vector<int>& L = h->elim;
  const int ng = (int)h->grp.size() - 1;
  std::vector<int> gid(n);
  for (int g = 0; g < ng; ++g)
    for (int q = h->grp[g]; q < h->grp[g + 1]; ++q) gid[q] = g;
  std::vector<std::vector<std::pair<int, long long>>> src(n);
  for (int k = 0; k < n; ++k) {
    long long base = h->alpha_row_start[k];
    for (size_t q = 0; q < h->rows[k].size(); ++q) {
      int j = h->rows[k][q];
      if (forward) src[j].push_back({k, base + (long long)q});
      else src[k].push_back({j, base + (long long)q});
    }
  }
  std::vector<int> glev(ng, 0);
  int nlev = 0;
  auto visit = [&](int g) {
    for (int t = h->grp[g]; t < h->grp[g + 1]; ++t)
      for (auto& sp : src[t])
        if (gid[sp.first] != g) glev[g] = std::max(glev[g], glev[gid[sp.first]] + 1);
    nlev = std::max(nlev, glev[g] + 1);
  };
  if (forward) for (int g = 0; g < ng; ++g) visit(g);
  else for (int g = ng - 1; g >= 0; --g) visit(g);
  std::vector<std::vector<int>> bylev(nlev);
  for (int g = 0; g < ng; ++g) bylev[glev[g]].push_back(g);
  int max_scr = 0;
  for (int l = 0; l < nlev; ++l) {
    for (int phase = 0; phase < 2; ++phase) {
      TaskList tl;
      FinList fl;
      int scr_row = 0;
      struct Tgt { int out_row, mt; std::vector<GItem> its; };
      std::vector<Tgt> tgts;
      for (int g : bylev[l]) {
        if (phase == 1 && !h->tg_n[g]) continue;
        const int nG = h->tg_n[g];
        for (int t = h->grp[g]; t < h->grp[g + 1]; ++t) {
          const int mt = h->m[L[t]];
          std::vector<GItem> its;
          if (phase == 0) {
            for (auto& sp : src[t]) {
              if (gid[sp.first] == g) continue;
              const int s = L[sp.first];
              GItem it{};
              it.a_off = h->alpha_off[sp.second];
              it.a_buf = AB_ALPHA;
              it.lda = forward ? mt : h->m[s];
              it.trans = forward ? 1 : 0;
              it.k = h->m[s];
              it.in_buf = VB_OUT;
              it.in_row = (int)h->leaf_off[s];
              its.push_back(it);
            }
          } else {
            const long long T0 = h->tg_off[g];
            if (forward) {
              for (int k = h->grp[g]; k < t; ++k)        // T_G(t, k), k before t
                its.push_back(GItem{T0 + (long long)h->rloc[t] * nG + h->rloc[k], AB_TINV, nG, 0,
                                    h->m[L[k]], VB_OUT, (int)h->leaf_off[L[k]]});
            } else {
              for (int j = t + 1; j < h->grp[g + 1]; ++j)  // T_G(j, t)^T, j after t
                its.push_back(GItem{T0 + (long long)h->rloc[j] * nG + h->rloc[t], AB_TINV, nG, 1,
                                    h->m[L[j]], VB_OUT, (int)h->leaf_off[L[j]]});
            }
          }
          tgts.push_back(Tgt{(int)h->leaf_off[L[t]], mt, std::move(its)});
        }
      }
      // Split-K size of the phase.  The FP64 gather kernels want many small
      // tasks (KMAX); the persistent tensor-core kernel needs only enough tasks
      // to keep its CTAs busy, and every extra split is one more partial panel
      // for the finalize to read: take the largest size (up to KMAX_TC) that
      // keeps min(TC_TASK_GOAL, tasks at KMAX) tasks.
      long long kmax = KMAX;
      if (h->p.precision == HM_MIXED && h->p.tensor_cores) {
        auto count = [&](long long km) {
          long long c = 0;
          for (const Tgt& tg : tgts) {
            long long kk = 0;
            for (size_t q = 0; q < tg.its.size(); ++q) {
              if (kk == 0 || kk + tg.its[q].k > km) {
                ++c;
                kk = 0;
              }
              kk += tg.its[q].k;
            }
          }
          return c;
        };
        constexpr long long TC_TASK_GOAL = 300;
        const long long goal = std::min(TC_TASK_GOAL, count(KMAX));
        for (long long km = split_cap(h); km > KMAX; km /= 2)
          if (count(km) >= goal) {
            kmax = km;
            break;
          }
      }
      for (const Tgt& tg : tgts) add_target(h, tl, fl, scr_row, tg.out_row, tg.mt, tg.its, kmax);
      max_scr = std::max(max_scr, scr_row);
      if (tl.tasks.empty()) continue;
      if (kmax != KMAX) {
        // the partial panels of the smallest split size (the autotuner's
        // candidates all fit the scratch panel)
        TaskList t2;
        FinList f2;
        int r2 = 0;
        for (const Tgt& tg : tgts) add_target(h, t2, f2, r2, tg.out_row, tg.mt, tg.its, KMAX);
        max_scr = std::max(max_scr, r2);
      }
      PhaseTargets pt;
      for (const Tgt& tg : tgts) {
        if (tg.its.empty()) continue;
        pt.out_row.push_back(tg.out_row);
        pt.mt.push_back(tg.mt);
        pt.its.push_back(tg.its);
      }
      pt.kmax = kmax;
      sw.tgt.push_back(std::move(pt));
      sw.part.push_back(std::move(tl));
      sw.fin.push_back(std::move(fl));
    }
  }
  sw.scratch_rows = max_scr;
}

// Tasks of more than mmax output rows become row slices of at most mmax rows
// with the same items (matrix reads offset by the slice's first row; a
// split-K slice writes its rows of the target's partial panel).  The
// tensor-core engine takes at most 128 complex rows per task (MMA N = 256);
// leaves of up to 256 unknowns (leaf cap 256) would otherwise send a whole
// launch to the CUDA-core kernels.  Each output row keeps its items and inner
// order, so the arithmetic of every row is unchanged.
void split_wide_tasks(TaskList& tl, int mmax) {
  bool any = false;
  for (const GTask& t : tl.tasks) any |= (t.m > mmax && t.mode != 2);
  if (!any) return;
  std::vector<GTask> nt;
  std::vector<GItem> ni;
  for (const GTask& t : tl.tasks) {
    const int step = (t.mode == 2) ? std::max(1, t.m) : mmax;
    for (int r = 0; r < std::max(1, t.m); r += step) {
      GTask sl = t;
      if (t.mode != 2) {
        sl.m = std::min(step, t.m - r);
        sl.out_row = t.out_row + r;
        if (t.mode == 1) sl.base_row = t.base_row + r;
      }
      sl.it0 = (int)ni.size();
      for (int q = t.it0; q < t.it1; ++q) {
        GItem I = tl.items[q];
        if (t.mode != 2) I.a_off += I.trans ? (long long)r : (long long)r * I.lda;
        ni.push_back(I);
      }
      sl.it1 = (int)ni.size();
      nt.push_back(sl);
    }
  }
  tl.tasks.swap(nt);
  tl.items.swap(ni);
}

bool has_groups(hm_ctx* h) {
  for (int x : h->tg_n)
    if (x) return true;
  return false;
}

hm_status build_schedules(hm_ctx* h) {
  free_sweep(h->fwd);
  free_sweep(h->bwd);
  free_tasks(h->dinv_tl);
  free_tasks(h->far1_tl);
  free_tasks(h->far1s_tl);
  free_tasks(h->far2_tl);
  free_tasks(h->near_tl);
  h->fwd = Sweep();
  h->bwd = Sweep();
  h->dinv_tl = TaskList();
  h->far1_tl = TaskList();
  h->far1s_tl = TaskList();
  h->far2_tl = TaskList();
  h->near_tl = TaskList();
  const int n = h->nl;
  size_t* b = &h->dev_bytes;
  if (h->has_scaling) {
    if (has_groups(h)) {
      build_sweep_groups(h, true, h->fwd);
      build_sweep_groups(h, false, h->bwd);
    } else {
      build_sweep(h, true, h->fwd);
      build_sweep(h, false, h->bwd);
    }
    for (Sweep* sw : {&h->fwd, &h->bwd})
      for (TaskList& tl : sw->part) split_wide_tasks(tl, 128);
    for (int q = 0; q < n; ++q) {
      const int k = h->elim[q];
      GTask t{VB_OUT, (int)h->leaf_off[k], h->m[k], (int)h->dinv_tl.items.size(), 0, 0, 0, 0};
      GItem it{h->dinv_off[q], AB_DINV, h->m[k], 0, h->m[k], VB_IN, (int)h->leaf_off[k]};
      h->dinv_tl.items.push_back(it);
      t.it1 = (int)h->dinv_tl.items.size();
      h->dinv_tl.tasks.push_back(t);
      h->dinv_tl.flops += (long long)h->m[k] * h->m[k];
      h->dinv_tl.a_bytes += (long long)h->m[k] * h->m[k] * 16;
    }
    for (auto& tl : h->fwd.part) { hm_status s = upload_tasks(tl, b); if (s) return s; }
    for (auto& fl : h->fwd.fin) { hm_status s = upload_fin(fl, b); if (s) return s; }
    for (auto& tl : h->bwd.part) { hm_status s = upload_tasks(tl, b); if (s) return s; }
    for (auto& fl : h->bwd.fin) { hm_status s = upload_fin(fl, b); if (s) return s; }
    hm_status s = upload_tasks(h->dinv_tl, b);
    if (s) return s;
  }
  // far field: stage 1 per low-rank block, stage 2 per leaf.  The stage-1
  // panel holds, for every low-rank block, t = V^T x (rank rows) at tA and
  // t' = U^T x (rank rows) at tB; the rows of all blocks that read the same
  // input cluster are contiguous, so the tensor-core engines can treat them as
  // one stacked operator (far1s: up to 128 rows per task) and read the input
  // once per task instead of once per block.
  std::vector<int> tA(h->far.size(), -1), tB(h->far.size(), -1);
  struct Seg { int bi, side; };                    // side 0: V^T x_c, 1: U^T x_r
  std::map<std::pair<int, int>, std::vector<Seg>> by_input;   // (in_row, k) -> segments
  for (size_t bi = 0; bi < h->far.size(); ++bi) {
    const FarDesc& f = h->far[bi];
    if (f.kind != 0 || f.rank == 0) continue;
    by_input[{f.c0, f.n}].push_back(Seg{(int)bi, 0});
    if (!h->nonsym) by_input[{f.r0, f.m}].push_back(Seg{(int)bi, 1});
  }
  constexpr int SROWS = 128;                      // rows of a stacked task
  int nt = 0;
  for (auto& kv : by_input) {
    const int in_row = kv.first.first, k = kv.first.second;
    size_t q = 0;
    while (q < kv.second.size()) {
      GTask ts{VB_FAR, nt, 0, (int)h->far1s_tl.items.size(), 0, 0, 0, 2};
      while (q < kv.second.size() && (ts.m == 0 || ts.m + h->far[kv.second[q].bi].rank <= SROWS)) {
        const Seg sg = kv.second[q++];
        const FarDesc& f = h->far[sg.bi];
        const long long off = sg.side == 0 ? f.offV : f.offU;
        (sg.side == 0 ? tA : tB)[sg.bi] = nt + ts.m;
        // the unstacked task of the same rows (FP64 and SIMT paths)
        GTask t1{VB_FAR, nt + ts.m, f.rank, (int)h->far1_tl.items.size(), 0, 0, 0, 0};
        h->far1_tl.items.push_back(GItem{off, AB_FAR, f.rank, 1, k, VB_IN, in_row});
        t1.it1 = (int)h->far1_tl.items.size();
        h->far1_tl.tasks.push_back(t1);
        h->far1s_tl.items.push_back(GItem{off, AB_FAR, f.rank, 1, k, VB_IN, in_row, ts.m, f.rank});
        ts.m += f.rank;
        h->far1_tl.flops += (long long)f.rank * k;
        h->far1_tl.a_bytes += (long long)f.rank * k * 16;
      }
      ts.it1 = (int)h->far1s_tl.items.size();
      h->far1s_tl.tasks.push_back(ts);
      nt += ts.m;
    }
  }
  h->far1s_tl.flops = h->far1_tl.flops;
  h->far1s_tl.a_bytes = h->far1_tl.a_bytes;
  h->far_t_rows = nt;
  std::vector<std::vector<GItem>> per_leaf(n);
  std::vector<std::vector<int>> share(n);      // per item: unknowns of its cluster
  auto leaf_of = [&](long long row) {
    return (int)(std::upper_bound(h->leaf_off.begin(), h->leaf_off.end(), row) -
                 h->leaf_off.begin()) - 1;
  };
  for (size_t bi = 0; bi < h->far.size(); ++bi) {
    const FarDesc& f = h->far[bi];
    for (int l = leaf_of(f.r0); l < n && h->leaf_off[l] < f.r0 + f.m; ++l) {
      long long dr = h->leaf_off[l] - f.r0;
      if (f.kind == 0) {
        if (f.rank == 0) continue;
        per_leaf[l].push_back(GItem{f.offU + dr * f.rank, AB_FAR, f.rank, 0, f.rank, VB_FAR,
                                    tA[bi]});
      } else {
        per_leaf[l].push_back(GItem{f.offU + dr * f.n, AB_FAR, f.n, 0, f.n, VB_IN, f.c0});
      }
      share[l].push_back(f.m);
    }
    if (h->nonsym) continue;        // a block of its own order only: no V U^T side
    for (int l = leaf_of(f.c0); l < n && h->leaf_off[l] < f.c0 + f.n; ++l) {
      long long dc = h->leaf_off[l] - f.c0;
      if (f.kind == 0) {
        if (f.rank == 0) continue;
        per_leaf[l].push_back(GItem{f.offV + dc * f.rank, AB_FAR, f.rank, 0, f.rank, VB_FAR,
                                    tB[bi]});
      } else {
        per_leaf[l].push_back(GItem{f.offU + dc, AB_FAR, f.n, 1, f.m, VB_IN, f.r0});
      }
      share[l].push_back(f.n);
    }
  }
  for (int l = 0; l < n; ++l) {
    GTask t{VB_OUT, (int)h->leaf_off[l], h->m[l], (int)h->far2_tl.items.size(), 0, 0, 0, 0};
    // stage-1 panel items first, then the dense blocks on the input (the
    // FP64-accurate engine changes its input scale at most once per task);
    // the stage-1 items of the largest clusters lead, in stage-1 row order:
    // every leaf of a cluster reads those same rows, and the leaves that run
    // side by side (neighbouring work units) then reach them at about the same
    // time, while the rows are still in L2
    std::vector<int> ord(per_leaf[l].size());
    for (size_t q = 0; q < ord.size(); ++q) ord[q] = (int)q;
    const std::vector<GItem>& pl = per_leaf[l];
    const std::vector<int>& sh = share[l];
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      const bool fa = pl[a].in_buf == VB_FAR, fb = pl[b].in_buf == VB_FAR;
      if (fa != fb) return fa;
      if (!fa) return false;
      if (sh[a] != sh[b]) return sh[a] > sh[b];
      return pl[a].in_row < pl[b].in_row;
    });
    std::vector<GItem> sorted;
    for (int q : ord) sorted.push_back(pl[q]);
    per_leaf[l].swap(sorted);
    for (auto& it : per_leaf[l]) {
      h->far2_tl.items.push_back(it);
      h->far2_tl.flops += (long long)h->m[l] * it.k;
      h->far2_tl.a_bytes += (long long)h->m[l] * it.k * 16;
    }
    t.it1 = (int)h->far2_tl.items.size();
    h->far2_tl.tasks.push_back(t);
  }
  split_wide_tasks(h->far2_tl, 128);
  // near field Z_N (upper blocks + transposes; every ordered block once for a
  // non-symmetric system)
  std::vector<std::vector<GItem>> near_leaf(n);
  for (const NearDesc& d : h->near) {
    near_leaf[d.i].push_back(GItem{d.off, AB_NEAR, h->m[d.j], 0, h->m[d.j], VB_IN,
                                   (int)h->leaf_off[d.j]});
    if (d.i != d.j && !h->nonsym)
      near_leaf[d.j].push_back(GItem{d.off, AB_NEAR, h->m[d.j], 1, h->m[d.i], VB_IN,
                                     (int)h->leaf_off[d.i]});
  }
  for (int l = 0; l < n; ++l) {
    GTask t{VB_OUT, (int)h->leaf_off[l], h->m[l], (int)h->near_tl.items.size(), 0, 0, 0, 0};
    for (auto& it : near_leaf[l]) {
      h->near_tl.items.push_back(it);
      h->near_tl.flops += (long long)h->m[l] * it.k;
    }
    t.it1 = (int)h->near_tl.items.size();
    h->near_tl.tasks.push_back(t);
  }
  hm_status s = upload_tasks(h->far1_tl, b);
  if (!s) s = upload_tasks(h->far1s_tl, b);
  if (!s) s = upload_tasks(h->far2_tl, b);
  if (!s) s = upload_tasks(h->near_tl, b);
  if (!s) s = row_exponents(h, h->near_tl, h->rexp_near);
  if (!s) s = row_exponents(h, h->far1_tl, h->rexp_far1);
  if (!s) s = row_exponents(h, h->far1s_tl, h->rexp_far1s);
  if (!s) s = row_exponents(h, h->far2_tl, h->rexp_far2);
  if (!s && h->has_scaling) s = row_exponents(h, h->dinv_tl, h->rexp_dinv);
  for (TaskList* tl : {&h->near_tl, &h->far1_tl, &h->far1s_tl, &h->far2_tl, &h->dinv_tl})
    if (!s) s = build_oz_units(*tl, &h->dev_bytes, tl == &h->far2_tl || tl == &h->near_tl);
  if (s) return s;
  h->sched_ready = true;
  ++h->gen;
  return HM_OK;
}

hm_status ensure_buffers(hm_ctx* h, int nrhs) {
  if (nrhs <= h->cap_nrhs) return HM_OK;
  ++h->gen;
  for (int i = 0; i < NPHYS; ++i) {
    cudaFree(h->d_vec[i]);
    h->d_vec[i] = nullptr;
  }
  cudaFree(h->d_norms);
  h->d_norms = nullptr;
  h->cap_nrhs = 0;
  size_t rows[NPHYS];
  for (int i = 0; i < NPHYS; ++i) rows[i] = (size_t)h->N;
  rows[P_SCR] = std::max<size_t>(1, std::max(h->fwd.scratch_rows, h->bwd.scratch_rows));
  rows[P_FAR] = std::max<size_t>(1, h->far_t_rows);
  // the mixed-precision chain keeps its series panels in complex64: the FP64
  // series panels (and the FP64 refinement copies) are not needed there
  if (h->p.precision == HM_MIXED)
    for (int i : {(int)P_BO, (int)P_IT, (int)P_SCR, (int)P_X0, (int)P_B0}) rows[i] = 1;
  // the staging panels of host-buffer solves are sized by the first such solve
  rows[P_HB] = rows[P_HX] = 1;
  for (int i = 0; i < NPHYS; ++i) {
    HM_CUDA(cudaMalloc((void**)&h->d_vec[i], rows[i] * nrhs * sizeof(cplx)));
    h->vec_rows[i] = rows[i];
  }
  HM_CUDA(cudaMalloc((void**)&h->d_norms, 5 * sizeof(double) * nrhs));
  cudaFree(h->d_fexp);
  HM_CUDA(cudaMalloc((void**)&h->d_fexp, 2 * sizeof(int) * nrhs));
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->d_xdig[i]);
    h->d_xdig[i] = nullptr;
  }
  // scratch panels of the mixed chain: digit panels of the FP64-accurate
  // products and split panels of the tensor-core products share storage (every
  // phase writes its panel at its start and no two phases overlap in a solve)
  if (h->p.precision == HM_MIXED && (h->p.fp64_emulation || h->p.tensor_cores)) {
    const int rws[2] = {h->N, std::max(1, h->far_t_rows)};
    for (int i = 0; i < 2; ++i) {
      size_t bytes = 0;
      if (h->p.fp64_emulation) bytes = std::max(bytes, oz_panel_bytes(rws[i], nrhs));
      if (h->p.tensor_cores) bytes = std::max(bytes, tc_split_bytes(rws[i], nrhs));
      HM_CUDA(cudaMalloc((void**)&h->d_xdig[i], bytes));
    }
  }
  h->cap_nrhs = nrhs;
  return HM_OK;
}

ABufs abufs(hm_ctx* h) {
  ABufs a{};
  a.p[AB_NEAR] = h->d_near;
  a.p[AB_FAR] = h->d_far;
  a.p[AB_ALPHA] = h->d_alpha;
  a.p[AB_DINV] = h->d_dinv;
  a.p[AB_TINV] = h->d_tinv;
  a.p[AB_ALPHAL] = h->d_alphaL;
  return a;
}

VBufs vbufs(hm_ctx* h, cplx* in, cplx* out) {
  VBufs v{};
  v.p[VB_IN] = in;
  v.p[VB_OUT] = out;
  v.p[VB_SCR] = h->d_vec[P_SCR];
  v.p[VB_FAR] = h->d_vec[P_FAR];
  return v;
}

// algorithmic traffic of a task list: matrix bytes once, input and output
// panels once per launch (asz / vsz = bytes of a matrix / vector entry)
double tl_bytes(const TaskList& tl, int nrhs, double asz = 16, double vsz = 16) {
  double vec = 0;
  for (const GItem& it : tl.items) vec += (double)it.k * nrhs * vsz;
  for (const GTask& t : tl.tasks) vec += (double)t.m * nrhs * vsz;
  return (double)tl.a_bytes / 16.0 * asz + vec;
}

}  // namespace

namespace hm {
const void* mixed_alpha(hm_ctx* h);
const void* mixed_far_data(hm_ctx* h);
const void* mixed_tinv(hm_ctx* h);
void* mixed_scratch(hm_ctx* h);
void* mixed_fart(hm_ctx* h);

// Bind the logical buffers of a launch: FP64 tables, or (low) the complex64
// copies of alpha / far factors and the complex64 scratch panels.
static void tables(hm_ctx* h, void* in, void* out, bool low, VBufs& v, ABufs& a) {
  v = VBufs{};
  v.p[VB_IN] = in;
  v.p[VB_OUT] = out;
  v.p[VB_SCR] = low ? mixed_scratch(h) : (void*)h->d_vec[P_SCR];
  v.p[VB_FAR] = low ? mixed_fart(h) : (void*)h->d_vec[P_FAR];
  a = ABufs{};
  a.p[AB_NEAR] = h->d_near;
  a.p[AB_FAR] = low ? mixed_far_data(h) : h->d_far;
  a.p[AB_ALPHA] = low ? mixed_alpha(h) : h->d_alpha;
  a.p[AB_DINV] = h->d_dinv;
  a.p[AB_TINV] = low ? mixed_tinv(h) : h->d_tinv;
  a.p[AB_ALPHAL] = low ? nullptr : h->d_alphaL;   // FP64 only (non-symmetric handles)
}

hm_status ensure_err(hm_ctx* h) {
  if (h->d_err) return HM_OK;
  HM_CUDA(cudaMalloc((void**)&h->d_err, sizeof(int)));
  HM_CUDA(cudaMemset(h->d_err, 0, sizeof(int)));
  return HM_OK;
}

// CUDA-core gather in complex64 or complex128 (the tensor-core gather is
// launched by the callers that hold split panels of the inputs)
static hm_status launch_any(hm_ctx* h, const TaskList& tl, const VBufs& v, const ABufs& a,
                            int nrhs, int prec) {
  if (nrhs == 1) {                      // the one-RHS kernels wait on copy barriers
    hm_status s = ensure_err(h);
    if (s) return s;
  }
  return launch_tasks(tl, v, a, nrhs, h->stream, prec, h->p.spin_limit, h->d_err);
}

hm_status run_chain_list(hm_ctx* h, TaskList& tl, void* in, void* out, int nrhs, int cat,
                         int prec, bool low) {
  if (low && prec == PREC_32) {       // complex64 matrices on the CUDA cores
    hm_status s = mixed_ensure_c64(h);
    if (s) return s;
  }
  VBufs v;
  ABufs a;
  tables(h, in, out, low, v, a);
  int ev = prof_begin(h);
  hm_status s = launch_any(h, tl, v, a, nrhs, prec);
  double asz = prec == PREC_32 ? 8 : 16, vsz = prec == PREC_64 ? 16 : 8;
  prof_end(h, ev, cat, tl_bytes(tl, nrhs, asz, vsz), 8.0 * tl.flops * nrhs);
  return s;
}

hm_status run_chain_sweep(hm_ctx* h, Sweep& sw, void* buf, int nrhs, int cat, int prec,
                          bool low) {
  double asz = prec == PREC_32 ? 8 : 16, vsz = prec == PREC_64 ? 16 : 8;
  // complex64 sweeps on the tensor cores read the sweep buffer through its
  // split panel: split once here, then every finalize keeps it current
  XSplit xs;
  unsigned char* bufs[2];
  const bool split = prec == PREC_32 && low && h->p.tensor_cores && nrhs >= 32 &&
                     mixed_xsplit(h, &xs, bufs);
  hm_status s;
  if (low && prec == PREC_32) {
    // a phase on the CUDA cores reads the complex64 matrices
    bool simt = !split;
    for (const TaskList& tl : sw.part) simt |= !tc_ok_for(tl);
    if (simt && (s = mixed_ensure_c64(h))) return s;
  }
  VBufs v;
  ABufs a;
  tables(h, buf, buf, low, v, a);
  if (split) {
    s = ensure_err(h);
    if (s) return s;
    int ev = prof_begin(h);
    s = launch_split((const float2*)buf, h->N, nrhs, bufs[0], xs.J[0], xs.G, h->stream);
    prof_end(h, ev, PC_CONV, (double)h->N * nrhs * (8 + 12), 0.0);
    if (s) return s;
  }
  for (size_t l = 0; l < sw.part.size(); ++l) {
    int ev = prof_begin(h);
    TaskList& tl = sw.part[l];
    if (split && tc_ok_for(tl))
      s = launch_tasks_tc(tl, v, a, nrhs, h->stream, h->p.spin_limit, h->d_err, &xs);
    else
      s = launch_any(h, tl, v, a, nrhs, prec);
    if (s) return s;
    prof_end(h, ev, cat, tl_bytes(tl, nrhs, asz, vsz), 8.0 * tl.flops * nrhs);
    ev = prof_begin(h);
    s = split ? launch_fin_split(sw.fin[l], v, nrhs, bufs[0], xs.J[0], xs.G, h->stream)
              : launch_fin(sw.fin[l], v, nrhs, h->stream, prec);
    if (s) return s;
    double fb = 0;
    for (const FTask& f : sw.fin[l].tasks) fb += (double)f.m * nrhs * vsz * (2 + f.s1 - f.s0);
    prof_end(h, ev, PC_FIN, fb, 0.0);
  }
  return HM_OK;
}

// FP64-accurate product of a task list on tensor cores (refinement residual);
// fexp_in / fexp_far must hold the column exponents of the bound panels.
hm_status run_oz_list(hm_ctx* h, TaskList& tl, RowExp& R, void* in, void* out, int nrhs,
                      int cat, bool panels32) {
  hm_status s = ensure_err(h);
  if (s) return s;
  VBufs v;
  ABufs a;
  tables(h, in, out, false, v, a);
  int ev = prof_begin(h);
  OzPanels xp;
  xp.xd[0] = h->d_xdig[0];
  xp.xd[1] = h->d_xdig[1];
  xp.J[0] = oz_row_groups(h->N);
  xp.J[1] = oz_row_groups(std::max(1, h->far_t_rows));
  xp.G = oz_rhs_groups(h->cap_nrhs);
  if (!xp.xd[0] || !xp.xd[1]) return HM_ERR_STATE;
  s = launch_tasks_oz(tl, v, a, nrhs, h->stream, R.d_e, R.d_off, h->d_fexp,
                      h->d_fexp + h->cap_nrhs, xp, h->p.spin_limit, h->d_err, panels32);
  prof_end(h, ev, cat, tl_bytes(tl, nrhs, 16, panels32 ? 8 : 16), 8.0 * tl.flops * nrhs);
  return s;
}

// one far-field stage on the tensor cores with its input from a split panel
// (written first from the complex64 panel src of `rows` rows)
static hm_status far_stage_split(hm_ctx* h, TaskList& tl, void* in, void* out, int nrhs,
                                 const float2* src, int rows, unsigned char* dst, long long J,
                                 const XSplit& xs) {
  hm_status s = ensure_err(h);
  if (s) return s;
  int ev = prof_begin(h);
  s = launch_split(src, rows, nrhs, dst, J, xs.G, h->stream);
  prof_end(h, ev, PC_CONV, (double)rows * nrhs * (8 + 12), 0.0);
  if (s) return s;
  VBufs v;
  ABufs a;
  tables(h, in, out, true, v, a);
  ev = prof_begin(h);
  s = launch_tasks_tc(tl, v, a, nrhs, h->stream, h->p.spin_limit, h->d_err, &xs);
  prof_end(h, ev, PC_MX_FAR, tl_bytes(tl, nrhs, 8, 8), 8.0 * tl.flops * nrhs);
  return s;
}

// ------------------------------------------------------------ split-K autotuner
// For every supernode sweep phase of a mixed-precision handle on the tensor
// cores: rebuild the phase's lists for the candidate split sizes 128 ... 2048
// rows (each distinct decomposition once), time the phase (gather and
// finalize, best of three) on the handle's own buffers and keep the fastest.
// A choice is cached for the process under the phase's shape -- direction,
// kind (external gather or T_G product), and the powers of two of its target
// count, inner rows and widest target, and the 128-RHS tiles -- so handles
// with phases of the same shape (the scatterers of a batch) take it without
// timing.  It runs before the solve's data flow: its launches read and write
// a work panel that every solve fills first.
namespace {
std::mutex g_tune_mu;
std::map<std::array<int, 6>, long long> g_tune;

int lg2(long long v) {
  int r = 0;
  while (v > 1) {
    v >>= 1;
    ++r;
  }
  return r;
}

std::array<int, 6> phase_key(int dir, const PhaseTargets& pt, int ytiles) {
  long long kin = 0;
  int mmax = 0;
  bool tg = false;
  for (size_t q = 0; q < pt.its.size(); ++q) {
    mmax = std::max(mmax, pt.mt[q]);
    for (const GItem& it : pt.its[q]) {
      kin += it.k;
      tg |= it.a_buf == AB_TINV;
    }
  }
  return {dir, tg ? 1 : 0, lg2((long long)pt.its.size()), lg2(kin), lg2(mmax), ytiles};
}

void free_fin(FinList& fl) {
  cudaFree(fl.d_tasks);
  cudaFree(fl.d_slots);
  fl.d_tasks = nullptr;
  fl.d_slots = nullptr;
}

// the phase's lists for split size kmax on the device, with their tensor-core tiles
hm_status make_phase(hm_ctx* h, const PhaseTargets& pt, long long kmax, const ABufs& a,
                     TaskList& tl, FinList& fl, int& scr) {
  tl = TaskList();
  fl = FinList();
  scr = 0;
  for (size_t q = 0; q < pt.its.size(); ++q)
    add_target(h, tl, fl, scr, pt.out_row[q], pt.mt[q], pt.its[q], kmax);
  split_wide_tasks(tl, 128);
  hm_status s = upload_tasks(tl, nullptr);
  if (!s) s = upload_fin(fl, nullptr);
  if (!s) s = build_tc_tiles(tl, a, nullptr);
  return s;
}

// best of three device times of one phase (gather, then finalize)
hm_status time_phase(hm_ctx* h, const TaskList& tl, const FinList& fl, const VBufs& v,
                     const ABufs& a, int nrhs, const XSplit& xs, unsigned char* xs0,
                     float* best) {
  cudaEvent_t e0, e1;
  HM_CUDA(cudaEventCreate(&e0));
  HM_CUDA(cudaEventCreate(&e1));
  hm_status s = HM_OK;
  *best = 1e30f;
  for (int rep = 0; rep < 3 && !s; ++rep) {
    cudaEventRecord(e0, h->stream);
    s = launch_tasks_tc(tl, v, a, nrhs, h->stream, h->p.spin_limit, h->d_err, &xs);
    if (!s) s = launch_fin_split(fl, v, nrhs, xs0, xs.J[0], xs.G, h->stream);
    cudaEventRecord(e1, h->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess && !s) s = cuda_status(e);
    *best = std::min(*best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  // a bounded wait that ran out makes the timing meaningless: the caller stops
  // tuning (the error word stays set for hm_get_diagnostics)
  int e = 0;
  HM_CUDA(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  return e ? HM_ERR_TIMEOUT : HM_OK;
}
}  // namespace

hm_status tune_sweeps(hm_ctx* h, int nrhs) {
  if (h->p.precision != HM_MIXED || !h->p.tensor_cores || !h->p.autotune || nrhs < 32)
    return HM_OK;
  const int yt = (nrhs + 127) / 128;
  if (h->fwd.tuned_ytiles == yt && h->bwd.tuned_ytiles == yt) return HM_OK;
  XSplit xs;
  unsigned char* bufs[2];
  if (!mixed_xsplit(h, &xs, bufs)) return HM_OK;
  hm_status s = ensure_err(h);
  if (!s) s = mixed_ensure_c64(h);       // the candidates' tiles are cut from them
  if (s) return s;
  // a work panel of N x nrhs complex64 values (the complex128 panel P_Y, not
  // in use before the solve's residual) and its split panel
  void* buf = h->d_vec[P_Y];
  VBufs v;
  ABufs a;
  tables(h, buf, buf, true, v, a);
  s = launch_split((const float2*)buf, h->N, nrhs, bufs[0], xs.J[0], xs.G, h->stream);
  if (s) return s;
  const int scr_cap = std::max(h->fwd.scratch_rows, h->bwd.scratch_rows);
  int dir = 0;
  for (Sweep* sw : {&h->fwd, &h->bwd}) {
    if (sw->tuned_ytiles == yt || sw->tgt.size() != sw->part.size()) {
      ++dir;
      continue;
    }
    for (size_t l = 0; l < sw->part.size(); ++l) {
      PhaseTargets& pt = sw->tgt[l];
      if (!tc_ok_for(sw->part[l]) || !sw->part[l].d_tiles) continue;
      const auto key = phase_key(dir, pt, yt);
      long long want = -1;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) want = it->second;
      }
      if (want < 0) {
        float best_ms = 0.f;
        s = time_phase(h, sw->part[l], sw->fin[l], v, a, nrhs, xs, bufs[0], &best_ms);
        if (s == HM_ERR_TIMEOUT) return HM_OK;   // keep the built-in choices
        if (s) return s;
        long long best_k = pt.kmax;
        std::vector<std::pair<size_t, size_t>> seen{{sw->part[l].tasks.size(),
                                                     sw->fin[l].slots.size()}};
        for (long long km = KMAX; km <= split_cap(h); km *= 2) {
          if (km == pt.kmax) continue;
          TaskList tl;
          FinList fl;
          int scr = 0;
          s = make_phase(h, pt, km, a, tl, fl, scr);
          const std::pair<size_t, size_t> cnt{tl.tasks.size(), fl.slots.size()};
          const bool dup = std::find(seen.begin(), seen.end(), cnt) != seen.end();
          float ms = 1e30f;
          if (!s && !dup && scr <= scr_cap && tl.d_tiles) {
            seen.push_back(cnt);
            s = time_phase(h, tl, fl, v, a, nrhs, xs, bufs[0], &ms);
          }
          free_tasks(tl);
          free_fin(fl);
          if (s == HM_ERR_TIMEOUT) return HM_OK;
          if (s) return s;
          if (ms < best_ms) {
            best_ms = ms;
            best_k = km;
          }
        }
        want = best_k;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = want;
      }
      if (want != pt.kmax) {
        TaskList tl;
        FinList fl;
        int scr = 0;
        s = make_phase(h, pt, want, a, tl, fl, scr);
        if (s || scr > scr_cap || !tl.d_tiles) {
          free_tasks(tl);
          free_fin(fl);
          if (s) return s;
          continue;
        }
        h->dev_bytes += tl.tile_bytes;
        h->dev_bytes -= std::min(h->dev_bytes, sw->part[l].tile_bytes);
        free_tasks(sw->part[l]);
        free_fin(sw->fin[l]);
        sw->part[l] = tl;
        sw->fin[l] = fl;
        pt.kmax = want;
        ++h->gen;              // a graph recorded before refers to the old lists
      }
      ++h->tuned_phases;
    }
    sw->tuned_ytiles = yt;
    ++dir;
  }
  HM_CUDA(cudaStreamSynchronize(h->stream));
  mixed_drop_c64(h);                     // every tensor-core list has its tiles
  return HM_OK;
}

hm_status mixed_far(hm_ctx* h, void* in, void* out, int nrhs) {
  XSplit xs;
  unsigned char* bufs[2];
  const bool tc = h->p.tensor_cores && nrhs >= 32 && mixed_xsplit(h, &xs, bufs);
  hm_status s;
  if (tc && tc_ok_for(h->far1s_tl))
    s = far_stage_split(h, h->far1s_tl, in, out, nrhs, (const float2*)in, h->N, bufs[0], xs.J[0],
                        xs);
  else
    s = run_chain_list(h, h->far1_tl, in, out, nrhs, PC_MX_FAR, PREC_32, true);
  if (s) return s;
  if (tc && tc_ok_for(h->far2_tl)) {
    // far-2 items read both the stage-1 panel and (dense blocks) the input
    if (!tc_ok_for(h->far1s_tl)) {
      s = launch_split((const float2*)in, h->N, nrhs, bufs[0], xs.J[0], xs.G, h->stream);
      if (s) return s;
    }
    return far_stage_split(h, h->far2_tl, in, out, nrhs, (const float2*)mixed_fart(h),
                           std::max(1, h->far_t_rows), bufs[1], xs.J[1], xs);
  }
  return run_chain_list(h, h->far2_tl, in, out, nrhs, PC_MX_FAR, PREC_32, true);
}
}  // namespace hm

namespace {

hm_status run_sweep(hm_ctx* h, Sweep& sw, cplx* buf, int nrhs, int cat) {
  return run_chain_sweep(h, sw, buf, nrhs, cat, PREC_64, false);
}

hm_status run_list(hm_ctx* h, TaskList& tl, cplx* in, cplx* out, int nrhs, int cat) {
  return run_chain_list(h, tl, in, out, nrhs, cat, PREC_64, false);
}

hm_status copy_panel(hm_ctx* h, cplx* dst, const cplx* src, int nrhs) {
  HM_CUDA(cudaMemcpyAsync(dst, src, (size_t)h->N * nrhs * sizeof(cplx),
                          cudaMemcpyDeviceToDevice, h->stream));
  return HM_OK;
}

hm_status apply_far(hm_ctx* h, cplx* in, cplx* out, int nrhs) {
  hm_status s = run_list(h, h->far1_tl, in, out, nrhs, PC_FAR1);
  if (s) return s;
  return run_list(h, h->far2_tl, in, out, nrhs, PC_FAR2);
}

// x (leaf order, in-place in P_XT) from b (leaf order, P_B): FP64 chain.
hm_status series_fp64(hm_ctx* h, int nrhs, bool diag) {
  cplx** V = h->d_vec;
  hm_status s;
  // b~ = R^T b ; b_o = D^-1 b~
  if ((s = copy_panel(h, V[P_Y], V[P_B], nrhs))) return s;
  if ((s = run_sweep(h, h->fwd, V[P_Y], nrhs, PC_FWD))) return s;
  if ((s = run_list(h, h->dinv_tl, V[P_Y], V[P_BO], nrhs, PC_DINV))) return s;
  if ((s = copy_panel(h, V[P_XT], V[P_BO], nrhs))) return s;
  cplx* it = V[P_BO];
  const bool adapt = h->p.term_tol > 0.0;
  std::vector<double> n0, nprev, nt;
  if (adapt && h->p.n_terms > 1 && (s = term_norms(h, it, false, nrhs, n0))) return s;
  nprev = n0;
  int used = 1;
  for (int t = 1; t < h->p.n_terms; ++t) {
    // it_t = D^-1 R^T Z_F R it_{t-1}
    if ((s = copy_panel(h, V[P_Y], it, nrhs))) return s;
    if ((s = run_sweep(h, h->bwd, V[P_Y], nrhs, PC_BWD))) return s;
    if ((s = apply_far(h, V[P_Y], V[P_Z], nrhs))) return s;
    if ((s = run_sweep(h, h->fwd, V[P_Z], nrhs, PC_FWD))) return s;
    cplx* nxt = (it == V[P_IT]) ? V[P_R] : V[P_IT];
    if ((s = run_list(h, h->dinv_tl, V[P_Z], nxt, nrhs, PC_DINV))) return s;
    if (t == 1 && diag) {
      if ((s = launch_col_norms2(it, h->N, nrhs, h->d_norms, h->stream))) return s;
      if ((s = launch_col_norms2(nxt, h->N, nrhs, h->d_norms + nrhs, h->stream))) return s;
    }
    double sg = (t % 2) ? -1.0 : 1.0;
    if ((s = launch_axpby(V[P_XT], V[P_XT], 1.0, nxt, sg, (size_t)h->N * nrhs, h->stream)))
      return s;
    it = nxt;
    used = t + 1;
    if (adapt) {
      if ((s = term_norms(h, nxt, false, nrhs, nt))) return s;
      if (terms_stop(n0, nprev, nt, h->p.term_tol)) break;
      nprev.swap(nt);
    }
  }
  h->last_terms = std::max(h->last_terms, used);
  // x = R x~
  return run_sweep(h, h->bwd, V[P_XT], nrhs, PC_BWD);
}

hm_status check_ready(hm_ctx* h) {
  if (!h) return HM_ERR_INVALID;
  if (!h->has_scaling || !h->sched_ready) return HM_ERR_STATE;
  return HM_OK;
}

// ---------------------------------------------------------------- file IO
struct Reader {
  FILE* f;
  bool ok = true;
  template <class T>
  void get(T* p, size_t n) {
    if (ok && fread(p, sizeof(T), n, f) != n) ok = false;
  }
  long long q() {
    long long v = 0;
    get(&v, 1);
    return v;
  }
};

hm_status finish_structure(hm_ctx* h) {
  h->nl = (int)h->leaf_off.size() - 1;
  h->m.resize(h->nl);
  for (int i = 0; i < h->nl; ++i) h->m[i] = (int)(h->leaf_off[i + 1] - h->leaf_off[i]);
  std::vector<int> perm32(h->perm.begin(), h->perm.end());
  return upload(&h->d_perm, perm32, &h->dev_bytes);
}

}  // namespace

namespace hm {
hm_status upload_values(hm_ctx* h) {
  size_t* b = &h->dev_bytes;
  hm_status s = upload(&h->d_near, h->h_near, b);
  if (!s) s = upload(&h->d_far, h->h_far, b);
  if (!s) s = upload(&h->d_tinv, h->h_tinv, b);
  if (!s) s = upload(&h->d_alpha, h->h_alpha, b);
  if (!s) s = upload(&h->d_dinv, h->h_dinv, b);
  if (!s && !h->h_alphaL.empty()) s = upload(&h->d_alphaL, h->h_alphaL, b);
  return s;
}
hm_status rebuild_schedules(hm_ctx* h) { return build_schedules(h); }
}  // namespace hm

extern "C" {

void hm_default_params(hm_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->wavelength = 1.0;
  p->leaf_max = 64;
  p->ordering = HM_ORDER_DFS;
  p->aca_tol = 1e-4;
  p->fill = HM_FILL_FULL;
  p->n_terms = 2;
  p->precision = HM_FP64;
  p->refine_steps = 0;
  p->spin_limit = 1LL << 26;
  p->tensor_cores = 1;
  p->fp64_emulation = 1;
  p->autotune = 1;
}

const char* hm_status_string(hm_status s) {
  switch (s) {
    case HM_OK: return "ok";
    case HM_ERR_INVALID: return "invalid argument";
    case HM_ERR_CUDA: return "CUDA error";
    case HM_ERR_OOM: return "out of memory";
    case HM_ERR_SINGULAR: return "singular diagonal block";
    case HM_ERR_TIMEOUT: return "device wait timed out";
    case HM_ERR_STATE: return "call out of order";
    case HM_ERR_IO: return "file error";
    case HM_WARN_SERIES_RATIO: return "series ratio above 0.1 (Eq. 45)";
  }
  return "unknown status";
}

hm_status hm_import(const char* path, const hm_params* p, hm_handle* out) {
  if (!path || !out) return HM_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return HM_ERR_CUDA;
  FILE* f = fopen(path, "rb");
  if (!f) return HM_ERR_IO;
  hm_ctx* h = nullptr;
  try {
    h = new hm_ctx();
    if (p) h->p = *p; else hm_default_params(&h->p);
    cudaGetDevice(&h->dev);
    Reader r{f};
    char magic[8];
    r.get(magic, 8);
    if (!r.ok || memcmp(magic, "HMPSBLK1", 8) != 0) throw std::runtime_error("magic");
    long long N = r.q(), nl = r.q(), nn = r.q(), nf = r.q(), reading = r.q(), has_s = r.q();
    double wl = 0, kk = 0;
    r.get(&wl, 1);
    r.get(&kk, 1);
    if (!r.ok || N <= 0 || nl <= 0 || N > (1LL << 30) || nl > N) throw std::runtime_error("hdr");
    h->N = (int)N;
    h->wavelength = wl;
    h->k = kk;
    h->perm.resize(N);
    r.get(h->perm.data(), N);
    h->leaf_off.resize(nl + 1);
    r.get(h->leaf_off.data(), nl + 1);
    if (!r.ok || h->leaf_off[0] != 0 || h->leaf_off[nl] != N) throw std::runtime_error("off");
    for (long long i = 0; i < nl; ++i)
      if (h->leaf_off[i + 1] <= h->leaf_off[i]) throw std::runtime_error("off");
    std::vector<char> seen(N, 0);
    for (long long i = 0; i < N; ++i) {
      if (h->perm[i] < 0 || h->perm[i] >= N || seen[h->perm[i]]) throw std::runtime_error("perm");
      seen[h->perm[i]] = 1;
    }
    hm_status s = finish_structure(h);
    if (s) throw s;
    for (long long b = 0; b < nn; ++b) {
      long long i = r.q(), j = r.q();
      if (!r.ok || i < 0 || j < i || j >= nl) throw std::runtime_error("near");
      NearDesc d{(int)i, (int)j, (long long)h->h_near.size()};
      size_t cnt = (size_t)h->m[i] * h->m[j];
      h->h_near.resize(h->h_near.size() + cnt);
      r.get(h->h_near.data() + d.off, cnt);
      h->near.push_back(d);
    }
    auto read_far = [&]() {
      long long kind = r.q(), r0 = r.q(), m = r.q(), c0 = r.q(), n = r.q(), rank = r.q();
      if (!r.ok || kind < 0 || kind > 1 || r0 < 0 || c0 < 0 || m <= 0 || n <= 0 ||
          r0 + m > N || c0 + n > N || rank < 0 || rank > std::min(m, n))
        throw std::runtime_error("far");
      FarDesc d{(int)kind, (int)r0, (int)m, (int)c0, (int)n, (int)rank, 0, 0};
      d.offU = (long long)h->h_far.size();
      if (kind == 0) {
        d.offV = d.offU + m * rank;
        h->h_far.resize(h->h_far.size() + (m + n) * rank);
        r.get(h->h_far.data() + d.offU, (size_t)((m + n) * rank));
      } else {
        d.rank = 0;
        h->h_far.resize(h->h_far.size() + m * n);
        r.get(h->h_far.data() + d.offU, (size_t)(m * n));
      }
      h->far.push_back(d);
    };
    for (long long b = 0; b < nf; ++b) read_far();
    if (has_s) {
      long long na = r.q();
      h->elim.resize(nl);
      {
        std::vector<long long> el(nl);
        r.get(el.data(), nl);
        std::vector<char> hit(nl, 0);
        for (long long q = 0; q < nl; ++q) {
          if (el[q] < 0 || el[q] >= nl || hit[el[q]]) throw std::runtime_error("elim");
          hit[el[q]] = 1;
          h->elim[q] = (int)el[q];
        }
      }
      h->rows.assign(nl, {});
      h->alpha_row_start.assign(nl + 1, 0);
      long long cnt_all = 0;
      for (long long k = 0; k < nl; ++k) {
        long long c = r.q();
        if (!r.ok || c < 0 || c > nl) throw std::runtime_error("rows");
        std::vector<long long> js(c);
        r.get(js.data(), c);
        for (long long q = 0; q < c; ++q) {
          if (js[q] <= k || js[q] >= nl || (q && js[q] <= js[q - 1]))
            throw std::runtime_error("rows");
          h->rows[k].push_back((int)js[q]);
        }
        h->alpha_row_start[k] = cnt_all;
        cnt_all += c;
      }
      h->alpha_row_start[nl] = cnt_all;
      if (cnt_all != na) throw std::runtime_error("alpha count");
      for (long long k = 0; k < nl; ++k)
        for (int j : h->rows[k]) {
          h->alpha_off.push_back((long long)h->h_alpha.size());
          size_t cnt = (size_t)h->m[h->elim[k]] * h->m[h->elim[j]];
          h->h_alpha.resize(h->h_alpha.size() + cnt);
          r.get(h->h_alpha.data() + h->alpha_off.back(), cnt);
        }
      for (long long k = 0; k < nl; ++k) {
        h->dinv_off.push_back((long long)h->h_dinv.size());
        size_t cnt = (size_t)h->m[h->elim[k]] * h->m[h->elim[k]];
        h->h_dinv.resize(h->h_dinv.size() + cnt);
        r.get(h->h_dinv.data() + h->dinv_off.back(), cnt);
      }
      h->has_scaling = true;
      h->p.fill = (reading == 1) ? HM_FILL_NEAR : HM_FILL_FULL;
    }
    if (!r.ok) throw std::runtime_error("size");
    // optional trailing sections, each introduced by an 8-byte tag
    for (;;) {
      char tag[8];
      const size_t got = fread(tag, 1, 8, f);
      if (got == 0 && feof(f)) break;
      if (got != 8) throw std::runtime_error("tag");
      if (memcmp(tag, "LEAFCEN1", 8) == 0) {
        // leaf cell centres (input of the nested-dissection order)
        h->leaf_cen.resize(3 * (size_t)nl);
        r.get(h->leaf_cen.data(), h->leaf_cen.size());
        if (!r.ok) throw std::runtime_error("centres");
        for (double c : h->leaf_cen)
          if (!std::isfinite(c)) throw std::runtime_error("centres");
      } else if (memcmp(tag, "SUPERND1", 8) == 0) {
        // supernode groups of consecutive ranks and T_G = (I - A_G^T)^-1 of
        // every group with more than one leaf (row-major n_G x n_G)
        if (!h->has_scaling) throw std::runtime_error("groups without scaling");
        const long long ng = r.q();
        if (!r.ok || ng < 1 || ng > nl) throw std::runtime_error("groups");
        std::vector<long long> g(ng + 1);
        r.get(g.data(), g.size());
        if (!r.ok || g[0] != 0 || g[ng] != nl) throw std::runtime_error("groups");
        for (long long q = 0; q < ng; ++q)
          if (g[q + 1] <= g[q]) throw std::runtime_error("groups");
        h->grp.assign(g.begin(), g.end());
        h->tg_off.assign(ng, 0);
        h->tg_n.assign(ng, 0);
        h->rloc.assign(nl, 0);
        long long nt_all = 0;
        for (long long q = 0; q < ng; ++q) {
          int nG = 0;
          for (long long k = g[q]; k < g[q + 1]; ++k) {
            h->rloc[k] = nG;
            nG += h->m[h->elim[k]];
          }
          h->tg_off[q] = nt_all;
          if (g[q + 1] - g[q] > 1) {
            h->tg_n[q] = nG;
            nt_all += (long long)nG * nG;
          }
        }
        h->h_tinv.resize(nt_all);
        r.get(h->h_tinv.data(), h->h_tinv.size());
        if (!r.ok) throw std::runtime_error("supernodes");
      } else if (memcmp(tag, "NONSYM01", 8) == 0) {
        // non-symmetric system (the CFIE of Eq. 8): the near blocks below the
        // diagonal, the far blocks whose row cluster follows their column
        // cluster, and with the scaling the left coefficients alphaL_kj,
        // each stored as its transpose in alpha's order and shapes
        const long long nnl = r.q();
        if (!r.ok || nnl < 0 || nnl > nl * nl) throw std::runtime_error("nonsym");
        for (long long b = 0; b < nnl; ++b) {
          long long i = r.q(), j = r.q();
          if (!r.ok || j < 0 || i <= j || i >= nl) throw std::runtime_error("nonsym near");
          NearDesc d{(int)i, (int)j, (long long)h->h_near.size()};
          size_t cnt = (size_t)h->m[i] * h->m[j];
          h->h_near.resize(h->h_near.size() + cnt);
          r.get(h->h_near.data() + d.off, cnt);
          h->near.push_back(d);
        }
        const long long nfl = r.q();
        if (!r.ok || nfl < 0) throw std::runtime_error("nonsym far");
        for (long long b = 0; b < nfl; ++b) read_far();
        const long long has_l = r.q();
        if (!r.ok || has_l != (h->has_scaling ? 1 : 0)) throw std::runtime_error("nonsym alphaL");
        if (has_l) {
          h->h_alphaL.resize(h->h_alpha.size());
          r.get(h->h_alphaL.data(), h->h_alphaL.size());
        }
        if (!r.ok) throw std::runtime_error("nonsym");
        h->nonsym = true;
      } else {
        throw std::runtime_error("section");
      }
    }
    // a non-symmetric system runs the FP64 chain on the leaf-level sweeps (the
    // supernode products and the mixed engines are written for Z = Z^T)
    if (h->nonsym && (!h->grp.empty() || h->p.precision != HM_FP64)) throw HM_ERR_INVALID;
    fclose(f);
    f = nullptr;
    s = upload_values(h);
    if (s) throw s;
    s = build_schedules(h);
    if (s) throw s;
    s = hm_mixed_prepare(h);
    if (s) throw s;
    *out = h;
    return HM_OK;
  } catch (hm_status s) {
    if (f) fclose(f);
    hm_destroy(h);
    return s;
  } catch (std::bad_alloc&) {
    if (f) fclose(f);
    hm_destroy(h);
    return HM_ERR_OOM;
  } catch (...) {
    if (f) fclose(f);
    hm_destroy(h);
    return HM_ERR_IO;
  }
}

hm_status hm_save(hm_handle h, const char* path) {
  if (!h || !path) return HM_ERR_INVALID;
  if (h->nonsym) return HM_ERR_STATE;        // the file of a non-symmetric system is the input
  FILE* f = fopen(path, "wb");
  if (!f) return HM_ERR_IO;
  auto put = [&](const void* p, size_t sz) { return fwrite(p, 1, sz, f) == sz; };
  bool ok = put("HMPSBLK1", 8);
  long long reading = h->has_scaling ? (h->p.fill == HM_FILL_NEAR ? 1 : 0) : -1;
  long long hdr[6] = {h->N, h->nl, (long long)h->near.size(), (long long)h->far.size(), reading,
                      h->has_scaling ? 1 : 0};
  ok = ok && put(hdr, sizeof(hdr));
  double d2[2] = {h->wavelength, h->k};
  ok = ok && put(d2, sizeof(d2));
  ok = ok && put(h->perm.data(), h->perm.size() * 8);
  ok = ok && put(h->leaf_off.data(), h->leaf_off.size() * 8);
  for (auto& d : h->near) {
    long long ij[2] = {d.i, d.j};
    ok = ok && put(ij, 16) &&
         put(h->h_near.data() + d.off, (size_t)h->m[d.i] * h->m[d.j] * sizeof(cplx));
  }
  for (auto& d : h->far) {
    long long hd[6] = {d.kind, d.r0, d.m, d.c0, d.n, d.rank};
    ok = ok && put(hd, sizeof(hd));
    size_t cnt = d.kind == 0 ? (size_t)(d.m + d.n) * d.rank : (size_t)d.m * d.n;
    ok = ok && put(h->h_far.data() + d.offU, cnt * sizeof(cplx));
  }
  if (h->has_scaling) {
    long long na = (long long)h->alpha_off.size();
    ok = ok && put(&na, 8);
    for (int q = 0; q < h->nl; ++q) {
      long long e = h->elim[q];
      ok = ok && put(&e, 8);
    }
    for (int k = 0; k < h->nl; ++k) {
      long long c = (long long)h->rows[k].size();
      ok = ok && put(&c, 8);
      for (int j : h->rows[k]) {
        long long jj = j;
        ok = ok && put(&jj, 8);
      }
    }
    size_t q = 0;
    for (int k = 0; k < h->nl; ++k)
      for (int j : h->rows[k])
        ok = ok && put(h->h_alpha.data() + h->alpha_off[q++],
                       (size_t)h->m[h->elim[k]] * h->m[h->elim[j]] * sizeof(cplx));
    for (int k = 0; k < h->nl; ++k)
      ok = ok && put(h->h_dinv.data() + h->dinv_off[k],
                     (size_t)h->m[h->elim[k]] * h->m[h->elim[k]] * sizeof(cplx));
  }
  if ((long long)h->leaf_cen.size() == 3LL * h->nl) {
    ok = ok && put("LEAFCEN1", 8) && put(h->leaf_cen.data(), h->leaf_cen.size() * sizeof(double));
  }
  if (h->has_scaling && has_groups(h)) {
    const long long ng = (long long)h->grp.size() - 1;
    ok = ok && put("SUPERND1", 8) && put(&ng, 8);
    for (int g : h->grp) {
      long long gg = g;
      ok = ok && put(&gg, 8);
    }
    for (long long g = 0; g < ng; ++g)
      if (h->tg_n[g])
        ok = ok && put(h->h_tinv.data() + h->tg_off[g],
                       (size_t)h->tg_n[g] * h->tg_n[g] * sizeof(cplx));
  }
  ok = (fclose(f) == 0) && ok;
  return ok ? HM_OK : HM_ERR_IO;
}

hm_status hm_set_stream(hm_handle h, void* stream) {
  if (!h) return HM_ERR_INVALID;
  h->stream = (cudaStream_t)stream;
  return HM_OK;
}

hm_status hm_num_unknowns(hm_handle h, int* n) {
  if (!h || !n) return HM_ERR_INVALID;
  *n = h->N;
  return HM_OK;
}

hm_status hm_get_tree(hm_handle h, long long* perm, long long* off) {
  if (!h) return HM_ERR_INVALID;
  if (perm) memcpy(perm, h->perm.data(), h->perm.size() * 8);
  if (off) memcpy(off, h->leaf_off.data(), h->leaf_off.size() * 8);
  return HM_OK;
}

hm_status hm_apply(hm_handle h, int op, void* Y, const void* X, int nrhs) {
  if (!h || !Y || !X || nrhs <= 0) return HM_ERR_INVALID;
  if (op < HM_OP_RT || op > HM_OP_Z) return HM_ERR_INVALID;
  if ((op == HM_OP_RT || op == HM_OP_R || op == HM_OP_DINV) && !h->has_scaling)
    return HM_ERR_STATE;
  try {
    hm_status s = ensure_buffers(h, nrhs);
    if (s) return s;
    if (h->p.precision == HM_MIXED) return hm_mixed_apply(h, op, (cplx*)Y, (const cplx*)X, nrhs);
    cplx** V = h->d_vec;
    if ((s = launch_gather_perm((const cplx*)X, V[P_B], h->d_perm, h->N, nrhs, h->stream)))
      return s;
    cplx* res = V[P_Y];
    switch (op) {
      case HM_OP_RT:
        if ((s = copy_panel(h, V[P_Y], V[P_B], nrhs))) return s;
        s = run_sweep(h, h->fwd, V[P_Y], nrhs, PC_FWD);
        break;
      case HM_OP_R:
        if ((s = copy_panel(h, V[P_Y], V[P_B], nrhs))) return s;
        s = run_sweep(h, h->bwd, V[P_Y], nrhs, PC_BWD);
        break;
      case HM_OP_DINV: s = run_list(h, h->dinv_tl, V[P_B], V[P_Y], nrhs, PC_DINV); break;
      case HM_OP_FAR: s = apply_far(h, V[P_B], V[P_Y], nrhs); break;
      case HM_OP_NEAR: s = run_list(h, h->near_tl, V[P_B], V[P_Y], nrhs, PC_NEAR); break;
      case HM_OP_Z:
        s = run_list(h, h->near_tl, V[P_B], V[P_Y], nrhs, PC_NEAR);
        if (!s) s = apply_far(h, V[P_B], V[P_Z], nrhs);
        if (!s)
          s = launch_axpby(V[P_Y], V[P_Y], 1.0, V[P_Z], 1.0, (size_t)h->N * nrhs, h->stream);
        break;
    }
    if (s) return s;
    s = launch_scatter_perm(res, (cplx*)Y, h->d_perm, h->N, nrhs, h->stream);
    if (s) return s;
    HM_CUDA(cudaStreamSynchronize(h->stream));
    return HM_OK;
  } catch (std::bad_alloc&) {
    return HM_ERR_OOM;
  } catch (...) {
    return HM_ERR_INVALID;
  }
}

hm_status hm_power_series_solve(hm_handle h, void* X, const void* B, int nrhs) {
  hm_status s = check_ready(h);
  if (s) return s;
  if (!X || !B || nrhs <= 0) return HM_ERR_INVALID;
  if (h->p.n_terms < 1) return HM_ERR_INVALID;
  if (h->p.term_tol < 0.0) return HM_ERR_INVALID;
  try {
    if ((s = ensure_buffers(h, nrhs))) return s;
    h->last_terms = 0;
    if (h->p.precision == HM_MIXED) {
      s = hm_mixed_solve(h, (cplx*)X, (const cplx*)B, nrhs);
    } else {
      cplx** V = h->d_vec;
      if ((s = launch_gather_perm((const cplx*)B, V[P_B], h->d_perm, h->N, nrhs, h->stream)))
        return s;
      if ((s = series_fp64(h, nrhs, true))) return s;
      // optional refinement in FP64: r = b - (Z_N + Z_F) x, x += series(r)
      for (int step = 0; step < h->p.refine_steps; ++step) {
        const size_t n = (size_t)h->N * nrhs;
        // keep x (P_X0) and b (P_B0); the residual goes to P_B for the series
        HM_CUDA(cudaMemcpyAsync(V[P_X0], V[P_XT], n * sizeof(cplx), cudaMemcpyDeviceToDevice,
                                h->stream));
        HM_CUDA(cudaMemcpyAsync(V[P_B0], V[P_B], n * sizeof(cplx), cudaMemcpyDeviceToDevice,
                                h->stream));
        if ((s = run_list(h, h->near_tl, V[P_X0], V[P_Y], nrhs, PC_NEAR))) return s;
        if ((s = apply_far(h, V[P_X0], V[P_Z], nrhs))) return s;
        if ((s = launch_axpby(V[P_Y], V[P_Y], -1.0, V[P_Z], -1.0, n, h->stream))) return s;
        if ((s = launch_axpby(V[P_B], V[P_B0], 1.0, V[P_Y], 1.0, n, h->stream))) return s;
        if (step == h->p.refine_steps - 1) {
          if ((s = launch_col_norms2(V[P_B0], h->N, nrhs, h->d_norms + 2 * nrhs, h->stream)))
            return s;
          if ((s = launch_col_norms2(V[P_B], h->N, nrhs, h->d_norms + 3 * nrhs, h->stream)))
            return s;
        }
        if ((s = series_fp64(h, nrhs, false))) return s;       // P_XT = series(r)
        if ((s = launch_axpby(V[P_XT], V[P_XT], 1.0, V[P_X0], 1.0, n, h->stream))) return s;
        HM_CUDA(cudaMemcpyAsync(V[P_B], V[P_B0], n * sizeof(cplx), cudaMemcpyDeviceToDevice,
                                h->stream));
      }
      s = launch_scatter_perm(V[P_XT], (cplx*)X, h->d_perm, h->N, nrhs, h->stream);
      h->ratio.assign(nrhs, 0.0);
      h->resid.assign(nrhs, 0.0);
    }
    if (s) return s;
    h->last_nrhs = nrhs;
    return HM_OK;
  } catch (std::bad_alloc&) {
    return HM_ERR_OOM;
  } catch (...) {
    return HM_ERR_INVALID;
  }
}

hm_status hm_power_series_solve_host(hm_handle h, void* X_host, const void* B_host, int nrhs) {
  hm_status s = check_ready(h);
  if (s) return s;
  if (!X_host || !B_host || nrhs <= 0) return HM_ERR_INVALID;
  try {
    if ((s = ensure_buffers(h, nrhs))) return s;
    for (int i : {(int)P_HB, (int)P_HX})
      if (h->vec_rows[i] != (size_t)h->N) {
        cudaFree(h->d_vec[i]);
        h->d_vec[i] = nullptr;
        h->vec_rows[i] = 0;
        HM_CUDA(cudaMalloc((void**)&h->d_vec[i], (size_t)h->N * h->cap_nrhs * sizeof(cplx)));
        h->vec_rows[i] = (size_t)h->N;
      }
    size_t bytes = (size_t)h->N * nrhs * sizeof(cplx);
    cplx* dB = h->d_vec[P_HB];
    cplx* dX = h->d_vec[P_HX];
    HM_CUDA(cudaMemcpyAsync(dB, B_host, bytes, cudaMemcpyHostToDevice, h->stream));
    s = hm_power_series_solve(h, dX, dB, nrhs);
    if (s != HM_OK && s != HM_WARN_SERIES_RATIO) return s;
    HM_CUDA(cudaMemcpyAsync(X_host, dX, bytes, cudaMemcpyDeviceToHost, h->stream));
    HM_CUDA(cudaStreamSynchronize(h->stream));
    return s;
  } catch (...) {
    return HM_ERR_INVALID;
  }
}

hm_status hm_get_diagnostics(hm_handle h, double* ratio, double* resid, int nrhs) {
  if (!h || nrhs <= 0) return HM_ERR_INVALID;
  if (nrhs > h->last_nrhs || !h->d_norms) return HM_ERR_STATE;
  std::vector<double> nrm(4 * (size_t)h->cap_nrhs, 0.0);
  HM_CUDA(cudaStreamSynchronize(h->stream));
  if (h->d_err) {
    int e = 0;
    HM_CUDA(cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return HM_ERR_TIMEOUT;
  }
  HM_CUDA(cudaMemcpy(nrm.data(), h->d_norms, nrm.size() * sizeof(double),
                     cudaMemcpyDeviceToHost));
  bool warn = false;
  for (int r = 0; r < nrhs; ++r) {
    double a = std::sqrt(nrm[r]), b = std::sqrt(nrm[h->last_nrhs + r]);
    double q = (a > 0) ? b / a : 0.0;
    if (ratio) ratio[r] = h->p.n_terms >= 2 ? q : 0.0;
    if (q > 0.1 && h->p.n_terms >= 2) warn = true;
    if (resid) {
      double bb = nrm[2 * h->last_nrhs + r], rr = nrm[3 * h->last_nrhs + r];
      resid[r] = (h->p.refine_steps > 0 && bb > 0) ? std::sqrt(rr / bb) : 0.0;
    }
  }
  return warn ? HM_WARN_SERIES_RATIO : HM_OK;
}

hm_status hm_get_stats(hm_handle h, long long* out, int n) {
  if (!h || !out) return HM_ERR_INVALID;
  long long near_e = 0, far_e = 0, maxr = 0, a_e = 0, d_e = 0;
  for (auto& d : h->near) near_e += (long long)h->m[d.i] * h->m[d.j];
  for (auto& d : h->far) {
    far_e += d.kind == 0 ? (long long)(d.m + d.n) * d.rank : (long long)d.m * d.n;
    maxr = std::max<long long>(maxr, d.rank);
  }
  for (int k = 0; k < (int)h->rows.size(); ++k)
    for (int j : h->rows[k]) a_e += (long long)h->m[h->elim[k]] * h->m[h->elim[j]];
  for (int k = 0; k < h->nl; ++k) d_e += (long long)h->m[k] * h->m[k];
  long long v[15] = {h->N, h->nl, (long long)h->near.size(), (long long)h->far.size(), a_e, d_e,
                     near_e, far_e, maxr, (long long)h->fwd.part.size(),
                     (long long)h->bwd.part.size(), (long long)h->dev_bytes, hm::launch_count(),
                     h->last_terms, h->tuned_phases};
  for (int i = 0; i < n && i < 15; ++i) out[i] = v[i];
  return HM_OK;
}

hm_status hm_profile_enable(hm_handle h, int on) {
  if (!h) return HM_ERR_INVALID;
  h->prof = on != 0;
  return HM_OK;
}

hm_status hm_get_profile(hm_handle h, double* out, int ncat) {
  if (!h || !out || ncat <= 0) return HM_ERR_INVALID;
  HM_CUDA(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < 4 * ncat; ++i) out[i] = 0.0;
  for (const ProfRec& r : h->recs) {
    if (r.cat >= ncat) continue;
    float ms = 0.f;
    HM_CUDA(cudaEventElapsedTime(&ms, h->evpool[r.ev], h->evpool[r.ev + 1]));
    out[4 * r.cat] += 1.0;
    out[4 * r.cat + 1] += ms;
    out[4 * r.cat + 2] += r.bytes;
    out[4 * r.cat + 3] += r.flops;
  }
  h->recs.clear();
  h->evused = 0;
  return HM_OK;
}

hm_status hm_destroy(hm_handle h) {
  if (!h) return HM_OK;
  hm::hm_group_forget(h);
  for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
  free_sweep(h->fwd);
  free_sweep(h->bwd);
  free_tasks(h->dinv_tl);
  free_tasks(h->far1_tl);
  free_tasks(h->far1s_tl);
  free_tasks(h->far2_tl);
  free_tasks(h->near_tl);
  hm_mixed_release(h);
  cudaFree(h->d_perm);
  cudaFree(h->d_near);
  cudaFree(h->d_far);
  cudaFree(h->d_alpha);
  cudaFree(h->d_alphaL);
  cudaFree(h->d_dinv);
  cudaFree(h->d_tinv);
  for (int i = 0; i < NPHYS; ++i) cudaFree(h->d_vec[i]);
  cudaFree(h->d_norms);
  cudaFree(h->d_err);
  cudaFree(h->d_fexp);
  cudaFree(h->d_xdig[0]);
  cudaFree(h->d_xdig[1]);
  for (RowExp* R : {&h->rexp_near, &h->rexp_far1, &h->rexp_far2, &h->rexp_dinv, &h->rexp_far1s}) {
    cudaFree(R->d_e);
    cudaFree(R->d_off);
  }
  cudaFree(h->d_verts);
  cudaFree(h->d_tris);
  cudaFree(h->d_edge);
  cudaFree(h->mesh_q);
  cudaFree(h->mesh_area);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->mesh_tri[i]);
    cudaFree(h->mesh_fv[i]);
  }
  cudaFree(h->mesh_len);
  delete h;
  return HM_OK;
}

}  // extern "C"
