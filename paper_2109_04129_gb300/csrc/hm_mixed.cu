// Mixed-precision power-series solve.
//
// The chain of Eq. 25-36 runs with complex64 copies of the scaling
// coefficients alpha and of the far-field factors U, V (FP32 products, FP32
// accumulation) and complex64 vector panels; the scaled diagonal inverses
// D_k^-1 stay complex128 (FP64 products with FP64 accumulation on complex64
// panels).  Then refine_steps steps of iterative refinement against the FP64
// residual:  r = b - (Z_N + Z_F) x  (complex128 near blocks and far factors,
// FP64 products),  x += series(r)  in the same mixed precision.
#include <algorithm>
#include <vector>

#include "hm_mixed.h"

using namespace hm;

namespace hm {
hm_status run_chain_list(hm_ctx* h, TaskList& tl, void* in, void* out, int nrhs, int cat,
                         int prec, bool low);
hm_status run_chain_sweep(hm_ctx* h, Sweep& sw, void* buf, int nrhs, int cat, int prec,
                          bool low);
hm_status mixed_far(hm_ctx* h, void* in, void* out, int nrhs);
hm_status run_oz_list(hm_ctx* h, TaskList& tl, RowExp& R, void* in, void* out, int nrhs,
                      int cat, bool panels32 = false);
hm_status tune_sweeps(hm_ctx* h, int nrhs);
}

namespace {

enum { Q_B = 0, Q_BO, Q_Y, Q_Z, Q_IT, Q_R, Q_XT, Q_SCR, Q_FAR, NQ };

struct Mixed {
  float2* alpha = nullptr;
  float2* far = nullptr;
  float2* tinv = nullptr;
  float2* v[NQ] = {nullptr};
  int cap = 0;
  // the complex64 matrix copies are freed once every tensor-core list has its
  // bf16 tiles (the tensor-core kernels read only the tiles); a CUDA-core
  // launch (fewer than 32 RHS) or a new tiling rebuilds them from the host
  // copies first
  bool dropped = false;
};

template <class T>
void dfree(T*& p) {
  cudaFree(p);
  p = nullptr;
}

hm_status to32(const std::vector<cplx>& src, float2** dst) {
  dfree(*dst);
  if (src.empty()) return HM_OK;
  std::vector<float2> h(src.size());
  for (size_t i = 0; i < src.size(); ++i) h[i] = make_float2((float)src[i].x, (float)src[i].y);
  HM_CUDA(cudaMalloc((void**)dst, h.size() * sizeof(float2)));
  HM_CUDA(cudaMemcpy(*dst, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice));
  return HM_OK;
}

hm_status ensure32(hm_ctx* h, Mixed* M, int nrhs) {
  if (nrhs <= M->cap) return HM_OK;
  ++h->gen;
  for (int i = 0; i < NQ; ++i) dfree(M->v[i]);
  M->cap = 0;
  for (int i = 0; i < NQ; ++i) {
    size_t rows = (size_t)h->N;
    if (i == Q_SCR) rows = std::max<size_t>(1, std::max(h->fwd.scratch_rows, h->bwd.scratch_rows));
    if (i == Q_FAR) rows = std::max<size_t>(1, h->far_t_rows);
    HM_CUDA(cudaMalloc((void**)&M->v[i], rows * nrhs * sizeof(float2)));
  }
  M->cap = nrhs;
  return HM_OK;
}

hm_status copy32(hm_ctx* h, float2* d, const float2* s, int nrhs) {
  HM_CUDA(cudaMemcpyAsync(d, s, (size_t)h->N * nrhs * sizeof(float2), cudaMemcpyDeviceToDevice,
                          h->stream));
  return HM_OK;
}

// D^-1 (complex128) applied to a complex64 panel: FP64-accurate products on the
// tensor cores (exact integer slicing) for wide batches, else the FP64 units
hm_status dinv32(hm_ctx* h, float2* in, float2* out, int nrhs) {
  if (h->p.fp64_emulation && nrhs >= 32) {
    hm_status s = launch_col_exp32(in, h->N, nrhs, h->d_fexp, h->stream);
    if (!s) s = launch_digitize(in, true, h->N, nrhs, h->d_fexp, h->d_xdig[0],
                                oz_row_groups(h->N), oz_rhs_groups(h->cap_nrhs), h->stream);
    if (s) return s;
    return run_oz_list(h, h->dinv_tl, h->rexp_dinv, in, out, nrhs, PC_DINV, true);
  }
  return run_chain_list(h, h->dinv_tl, in, out, nrhs, PC_DINV, PREC_64x32, true);
}

// x32 (Q_XT) = series(b32 in Q_B); ratio norms when diag
hm_status series32(hm_ctx* h, Mixed* M, int nrhs, bool diag) {
  float2** V = M->v;
  hm_status s;
  if ((s = copy32(h, V[Q_Y], V[Q_B], nrhs))) return s;
  if ((s = run_chain_sweep(h, h->fwd, V[Q_Y], nrhs, PC_MX_SWEEP, PREC_32, true))) return s;
  if ((s = dinv32(h, V[Q_Y], V[Q_BO], nrhs))) return s;
  if ((s = copy32(h, V[Q_XT], V[Q_BO], nrhs))) return s;
  float2* it = V[Q_BO];
  // adaptive term count (hm_params.term_tol): the rule of the FP64 chain on
  // the complex64 terms
  const bool adapt = h->p.term_tol > 0.0;
  std::vector<double> n0, nprev, nt;
  if (adapt && h->p.n_terms > 1 && (s = term_norms(h, it, true, nrhs, n0))) return s;
  nprev = n0;
  int used = 1;
  for (int t = 1; t < h->p.n_terms; ++t) {
    if ((s = copy32(h, V[Q_Y], it, nrhs))) return s;
    if ((s = run_chain_sweep(h, h->bwd, V[Q_Y], nrhs, PC_MX_SWEEP, PREC_32, true))) return s;
    if ((s = mixed_far(h, V[Q_Y], V[Q_Z], nrhs))) return s;
    if ((s = run_chain_sweep(h, h->fwd, V[Q_Z], nrhs, PC_MX_SWEEP, PREC_32, true))) return s;
    float2* nxt = (it == V[Q_IT]) ? V[Q_R] : V[Q_IT];
    if ((s = dinv32(h, V[Q_Z], nxt, nrhs))) return s;
    if (t == 1 && diag) {
      if ((s = launch_col_norms2_32(it, h->N, nrhs, h->d_norms, h->stream))) return s;
      if ((s = launch_col_norms2_32(nxt, h->N, nrhs, h->d_norms + nrhs, h->stream))) return s;
    }
    float sg = (t % 2) ? -1.0f : 1.0f;
    if ((s = launch_axpby32(V[Q_XT], V[Q_XT], 1.0f, nxt, sg, (size_t)h->N * nrhs, h->stream)))
      return s;
    it = nxt;
    used = t + 1;
    if (adapt) {
      if ((s = term_norms(h, nxt, true, nrhs, nt))) return s;
      if (terms_stop(n0, nprev, nt, h->p.term_tol)) break;
      nprev.swap(nt);
    }
  }
  h->last_terms = std::max(h->last_terms, used);
  return run_chain_sweep(h, h->bwd, V[Q_XT], nrhs, PC_MX_SWEEP, PREC_32, true);
}

}  // namespace

hm_status hm_mixed_prepare(hm_ctx* h) {
  if (h->p.precision != HM_MIXED) return HM_OK;
  ++h->gen;
  Mixed* M = (Mixed*)h->mixed;
  if (!M) {
    M = new Mixed();
    h->mixed = M;
  }
  hm_status s = to32(h->h_far, &M->far);
  if (s) return s;
  if (h->has_scaling) s = to32(h->h_alpha, &M->alpha);
  if (!s && h->has_scaling) s = to32(h->h_tinv, &M->tinv);
  M->dropped = false;
  if (!s && h->has_scaling) {
    // a mixed-precision handle never runs the FP64 sweeps: their complex128
    // coefficients stay on the host only (hm_save writes the host copies)
    const size_t bytes = (h->h_alpha.size() + h->h_tinv.size()) * sizeof(cplx);
    if (h->d_alpha || h->d_tinv) h->dev_bytes -= std::min(h->dev_bytes, bytes);
    cudaFree(h->d_alpha);
    cudaFree(h->d_tinv);
    h->d_alpha = nullptr;
    h->d_tinv = nullptr;
  }
  if (s || !h->p.tensor_cores) return s;
  // bf16 slices of every complex64 matrix operand of the tensor-core lists
  ABufs a{};
  a.p[AB_FAR] = M->far;
  a.p[AB_ALPHA] = M->alpha;
  a.p[AB_TINV] = M->tinv;
  // sweep inputs come from the split panel of the sweep buffer
  for (Sweep* sw : {&h->fwd, &h->bwd})
    for (TaskList& tl : sw->part)
      if ((s = build_tc_tiles(tl, a, &h->dev_bytes))) return s;
  // the far-field inputs are fixed during a launch: they arrive as split
  // panels, and the tiles of the far lists are built for that
  if ((s = build_tc_tiles(h->far1s_tl, a, &h->dev_bytes))) return s;
  if ((s = build_tc_tiles(h->far2_tl, a, &h->dev_bytes))) return s;
  // with the autotuner on, the copies stay until the first tuning (it builds
  // tiles of its own from them)
  if (!h->p.autotune) mixed_drop_c64(h);
  return HM_OK;
}

void hm_mixed_release(hm_ctx* h) {
  Mixed* M = (Mixed*)h->mixed;
  if (!M) return;
  dfree(M->alpha);
  dfree(M->far);
  dfree(M->tinv);
  for (int i = 0; i < NQ; ++i) dfree(M->v[i]);
  delete M;
  h->mixed = nullptr;
}

namespace hm {
hm_status mixed_ensure_c64(hm_ctx* h) {
  Mixed* M = (Mixed*)h->mixed;
  if (!M || !M->dropped) return HM_OK;
  hm_status s = to32(h->h_far, &M->far);
  if (!s && h->has_scaling) s = to32(h->h_alpha, &M->alpha);
  if (!s && h->has_scaling) s = to32(h->h_tinv, &M->tinv);
  if (s) return s;
  M->dropped = false;
  ++h->gen;                 // a graph recorded before refers to other buffers
  return HM_OK;
}
void mixed_drop_c64(hm_ctx* h) {
  Mixed* M = (Mixed*)h->mixed;
  if (!M || M->dropped || !h->p.tensor_cores) return;
  dfree(M->far);
  dfree(M->alpha);
  dfree(M->tinv);
  M->dropped = true;
  ++h->gen;
}
const void* mixed_alpha(hm_ctx* h) { return h->mixed ? ((Mixed*)h->mixed)->alpha : nullptr; }
const void* mixed_far_data(hm_ctx* h) { return h->mixed ? ((Mixed*)h->mixed)->far : nullptr; }
const void* mixed_tinv(hm_ctx* h) { return h->mixed ? ((Mixed*)h->mixed)->tinv : nullptr; }
void* mixed_scratch(hm_ctx* h) { return h->mixed ? ((Mixed*)h->mixed)->v[Q_SCR] : nullptr; }
void* mixed_fart(hm_ctx* h) { return h->mixed ? ((Mixed*)h->mixed)->v[Q_FAR] : nullptr; }
// the split panels of the far-field inputs (false when not allocated)
// (the storage is the handle's scratch panel pair, shared with the digit panels)
bool mixed_xsplit(hm_ctx* h, XSplit* xs, unsigned char** bufs) {
  if (!h->mixed || !h->p.tensor_cores || !h->d_xdig[0] || !h->d_xdig[1]) return false;
  bufs[0] = h->d_xdig[0];
  bufs[1] = h->d_xdig[1];
  xs->xs[0] = h->d_xdig[0];
  xs->xs[1] = h->d_xdig[1];
  xs->J[0] = oz_row_groups(h->N);
  xs->J[1] = oz_row_groups(std::max(1, h->far_t_rows));
  xs->G = oz_rhs_groups(h->cap_nrhs);
  return true;
}
}  // namespace hm

// Y (P_Y) = Z_N x and Z (P_Z) = Z_F x for x in P_XT, FP64-accurate products:
// tensor cores with exact integer slicing, or the FP64 units.
static hm_status residual_products(hm_ctx* h, int nrhs, bool with_far) {
  cplx** V = h->d_vec;
  hm_status s;
  if (h->p.fp64_emulation && nrhs >= 32) {
    const int G = oz_rhs_groups(h->cap_nrhs);
    if ((s = launch_col_exp(V[P_XT], h->N, nrhs, h->d_fexp, h->stream))) return s;
    if ((s = launch_digitize(V[P_XT], false, h->N, nrhs, h->d_fexp, h->d_xdig[0],
                             oz_row_groups(h->N), G, h->stream)))
      return s;
    if ((s = run_oz_list(h, h->near_tl, h->rexp_near, V[P_XT], V[P_Y], nrhs, PC_NEAR)))
      return s;
    if (!with_far) return HM_OK;
    if ((s = run_oz_list(h, h->far1s_tl, h->rexp_far1s, V[P_XT], nullptr, nrhs, PC_FAR1)))
      return s;
    const int tr = std::max(1, h->far_t_rows);
    if ((s = launch_col_exp(h->d_vec[P_FAR], tr, nrhs, h->d_fexp + h->cap_nrhs, h->stream)))
      return s;
    if ((s = launch_digitize(h->d_vec[P_FAR], false, tr, nrhs, h->d_fexp + h->cap_nrhs,
                             h->d_xdig[1], oz_row_groups(tr), G, h->stream)))
      return s;
    return run_oz_list(h, h->far2_tl, h->rexp_far2, V[P_XT], V[P_Z], nrhs, PC_FAR2);
  }
  if ((s = run_chain_list(h, h->near_tl, V[P_XT], V[P_Y], nrhs, PC_NEAR, PREC_64, false)))
    return s;
  if (!with_far) return HM_OK;
  if ((s = run_chain_list(h, h->far1_tl, V[P_XT], nullptr, nrhs, PC_FAR1, PREC_64, false)))
    return s;
  return run_chain_list(h, h->far2_tl, V[P_XT], V[P_Z], nrhs, PC_FAR2, PREC_64, false);
}

hm_status hm_mixed_solve(hm_ctx* h, cplx* X, const cplx* B, int nrhs) {
  Mixed* M = (Mixed*)h->mixed;
  // (a handle with one leaf has scaling but no alpha blocks: M->alpha is null)
  if (!M || !h->has_scaling) return HM_ERR_STATE;
  hm_status s = ensure32(h, M, nrhs);
  if (s) return s;
  // split sizes of the tensor-core sweeps, timed once per number of RHS tiles
  if ((s = tune_sweeps(h, nrhs))) return s;
  cplx** V = h->d_vec;
  const size_t n = (size_t)h->N * nrhs;
  // b in leaf order: FP64 (for the residual) and FP32 (for the series)
  if ((s = launch_gather_perm(B, V[P_B], h->d_perm, h->N, nrhs, h->stream))) return s;
  if ((s = launch_to32(V[P_B], M->v[Q_B], n, h->stream))) return s;
  if ((s = series32(h, M, nrhs, true))) return s;
  // x (FP64, leaf order) in P_XT
  HM_CUDA(cudaMemsetAsync(V[P_XT], 0, n * sizeof(cplx), h->stream));
  if ((s = launch_axpby64_32(V[P_XT], 0.0, M->v[Q_XT], 1.0, n, h->stream))) return s;
  for (int step = 0; step < h->p.refine_steps; ++step) {
    // r = b - (Z_N + Z_F) x  with FP64-accurate products
    if ((s = residual_products(h, nrhs, true))) return s;
    if ((s = launch_axpby(V[P_Y], V[P_Y], -1.0, V[P_Z], -1.0, n, h->stream))) return s;
    if ((s = launch_axpby(V[P_R], V[P_B], 1.0, V[P_Y], 1.0, n, h->stream))) return s;
    if (step == h->p.refine_steps - 1) {
      if ((s = launch_col_norms2(V[P_B], h->N, nrhs, h->d_norms + 2 * nrhs, h->stream))) return s;
      if ((s = launch_col_norms2(V[P_R], h->N, nrhs, h->d_norms + 3 * nrhs, h->stream))) return s;
    }
    if ((s = launch_to32(V[P_R], M->v[Q_B], n, h->stream))) return s;
    if ((s = series32(h, M, nrhs, false))) return s;
    if ((s = launch_axpby64_32(V[P_XT], 1.0, M->v[Q_XT], 1.0, n, h->stream))) return s;
  }
  s = launch_scatter_perm(V[P_XT], X, h->d_perm, h->N, nrhs, h->stream);
  h->last_nrhs = nrhs;
  return s;
}

hm_status hm_mixed_apply(hm_ctx* h, int op, cplx* Y, const cplx* X, int nrhs) {
  Mixed* M = (Mixed*)h->mixed;
  if (!M) return HM_ERR_STATE;
  if ((op == HM_OP_RT || op == HM_OP_R) && !h->has_scaling) return HM_ERR_STATE;
  hm_status s = ensure32(h, M, nrhs);
  if (s) return s;
  cplx** V = h->d_vec;
  const size_t n = (size_t)h->N * nrhs;
  if (op == HM_OP_NEAR || op == HM_OP_Z) {
    // the refinement's FP64-accurate products
    if ((s = launch_gather_perm(X, V[P_XT], h->d_perm, h->N, nrhs, h->stream))) return s;
    if ((s = residual_products(h, nrhs, op == HM_OP_Z))) return s;
    if (op == HM_OP_Z &&
        (s = launch_axpby(V[P_Y], V[P_Y], 1.0, V[P_Z], 1.0, n, h->stream)))
      return s;
    if ((s = launch_scatter_perm(V[P_Y], Y, h->d_perm, h->N, nrhs, h->stream))) return s;
    HM_CUDA(cudaStreamSynchronize(h->stream));
    return HM_OK;
  }
  if ((s = launch_gather_perm(X, V[P_B], h->d_perm, h->N, nrhs, h->stream))) return s;
  if ((s = launch_to32(V[P_B], M->v[Q_B], n, h->stream))) return s;
  float2* res = M->v[Q_Y];
  switch (op) {
    case HM_OP_RT:
      if ((s = copy32(h, M->v[Q_Y], M->v[Q_B], nrhs))) return s;
      s = run_chain_sweep(h, h->fwd, M->v[Q_Y], nrhs, PC_MX_SWEEP, PREC_32, true);
      break;
    case HM_OP_R:
      if ((s = copy32(h, M->v[Q_Y], M->v[Q_B], nrhs))) return s;
      s = run_chain_sweep(h, h->bwd, M->v[Q_Y], nrhs, PC_MX_SWEEP, PREC_32, true);
      break;
    case HM_OP_DINV:
      s = dinv32(h, M->v[Q_B], M->v[Q_Y], nrhs);
      break;
    case HM_OP_FAR:
      s = mixed_far(h, M->v[Q_B], M->v[Q_Y], nrhs);
      break;
    default:
      return HM_ERR_INVALID;
  }
  if (s) return s;
  // widen to FP64 (the destination is read by axpby: clear it first)
  HM_CUDA(cudaMemsetAsync(V[P_Y], 0, n * sizeof(cplx), h->stream));
  if ((s = launch_axpby64_32(V[P_Y], 0.0, res, 1.0, n, h->stream))) return s;
  if ((s = launch_scatter_perm(V[P_Y], Y, h->d_perm, h->N, nrhs, h->stream))) return s;
  HM_CUDA(cudaStreamSynchronize(h->stream));
  return HM_OK;
}
