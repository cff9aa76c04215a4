// Internal declarations of the GB300 power-series H-matrix solver library.
// Everything here stays behind the C ABI of include/hm.h.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hm.h"

namespace hm {

typedef double2 cplx;   // complex128 as (re, im)

// ----------------------------------------------------------- gather GEMM
// A task computes one output panel of m rows x nrhs columns:
//   acc = sum over its items of op(A_item) * in_item
//   mode 0: out = acc        mode 1: out = base + acc
//   mode 2 (stacked, tensor-core engines only): the items are row segments
//     of one operator over the same input rows (those of item it0): out rows
//     [r0, r0 + nrow) = op(A_item) * in
// Panels live in "vector buffers" with row stride nrhs (RHS fastest).
struct GTask {
  int out_buf, out_row, m, it0, it1, base_buf, base_row, mode;
};
// op(A) is m x k: trans = 0 -> A[r * lda + c]; trans = 1 -> A[c * lda + r].
struct GItem {
  long long a_off;
  int a_buf, lda, trans, k, in_buf, in_row;
  // row segment of a stacked task (mode 2): this item supplies task rows
  // [r0, r0 + nrow); nrow = 0 elsewhere (the item covers every row)
  int r0, nrow;
};
// items whose inner rows a task walks: all of them, or only item it0 for a
// stacked task (its other items are row segments over the same inner rows)
__host__ __device__ inline int task_it_end(const GTask& t) {
  return t.mode == 2 ? t.it0 + 1 : t.it1;
}
// Finalize: out = base + sum of scratch panels (rows s of slot list).
struct FTask {
  int out_buf, out_row, m, base_buf, base_row, s0, s1;
};

// logical vector buffers named by tasks; bound to physical panels per launch
enum { VB_IN = 0, VB_OUT = 1, VB_SCR = 2, VB_FAR = 3, MAX_VBUF = 4 };
enum { MAX_ABUF = 6 };
struct VBufs { void* p[MAX_VBUF]; };
struct ABufs { const void* p[MAX_ABUF]; };
// element types of a launch: all FP64, all FP32, or FP64 matrix x FP32 vectors
enum { PREC_64 = 0, PREC_32 = 1, PREC_64x32 = 2 };
// physical panels of the solve (N x nrhs unless noted)
enum { P_B = 0, P_BO = 1, P_Y = 2, P_Z = 3, P_IT = 4, P_XT = 5, P_R = 6,
       P_SCR = 7,   // split-K scratch (sweep scratch rows)
       P_FAR = 8,   // far-field stage-1 panels (2 * sum of ranks rows)
       P_HB = 9, P_HX = 10,   // staging of host-buffer solves
       P_X0 = 11, P_B0 = 12,  // FP64 refinement: saved x and b
       NPHYS = 13 };
// matrix buffers
enum { AB_NEAR = 0, AB_FAR = 1, AB_ALPHA = 2, AB_DINV = 3, AB_TINV = 4, AB_ALPHAL = 5 };

// A launch-ready list of tasks (device copies of the host vectors).
struct TaskList {
  std::vector<GTask> tasks;
  std::vector<GItem> items;
  GTask* d_tasks = nullptr;
  GItem* d_items = nullptr;
  long long flops = 0;    // complex MACs per RHS
  long long a_bytes = 0;  // matrix bytes read per launch
  // tensor-core path: the complex64 matrix operand of every stage pre-split
  // into bf16 tiles (hm_tc.cu), task t's tiles from byte d_toff[t]
  unsigned char* d_tiles = nullptr;
  long long* d_toff = nullptr;
  int* d_torder = nullptr;   // task order of the persistent kernel, costliest first
  size_t tile_bytes = 0;
  // FP64-accurate path: work units (task, 32-row pass), costliest first
  int2* d_units = nullptr;
  int n_units = 0;
  // one-RHS bulk-copy kernel usable for this list (-1: not checked yet)
  mutable int bulk_ok = -1;
  // matrix buffers (bit AB_*) its items read, set at upload: a launch whose
  // table leaves one of them null returns an error instead of running
  unsigned abuf_mask = 0;
};
// every matrix buffer a list reads is bound (abuf_mask against the table)
inline bool abufs_bound(const TaskList& tl, const ABufs& ab) {
  for (int b = 0; b < MAX_ABUF; ++b)
    if (((tl.abuf_mask >> b) & 1u) && !ab.p[b]) return false;
  return true;
}
// per-task row scale exponents of a task list (FP64-accurate tensor products)
struct RowExp {
  std::vector<int> e;
  std::vector<long long> off;
  int* d_e = nullptr;
  long long* d_off = nullptr;
};
struct FinList {
  std::vector<FTask> tasks;
  std::vector<int> slots;
  FTask* d_tasks = nullptr;
  int* d_slots = nullptr;
};
// One sweep = a sequence of levels, each a partial launch and a finalize.
// The targets of one sweep phase (output rows, rows, items), kept so that the
// split-K autotuner can rebuild the phase's lists with another split size.
struct PhaseTargets {
  std::vector<int> out_row, mt;
  std::vector<std::vector<GItem>> its;
  long long kmax = 0;     // split size of the lists in use
};
struct Sweep {
  std::vector<TaskList> part;
  std::vector<FinList> fin;
  std::vector<PhaseTargets> tgt;   // per part (supernode sweeps only)
  int scratch_rows = 0;   // rows of VB_SCR needed
  int tuned_ytiles = 0;   // RHS tiles the split sizes were tuned for (0: not tuned)
};

enum { PC_FWD = 0, PC_BWD = 1, PC_FIN = 2, PC_DINV = 3, PC_FAR1 = 4, PC_FAR2 = 5,
       PC_NEAR = 6, PC_MISC = 7, PC_MX_SWEEP = 8, PC_MX_FAR = 9, PC_CONV = 10, PC_N = 11 };
struct ProfRec { int cat; int ev; double bytes, flops; };

struct FarDesc {
  int kind;               // 0 low rank U V^T, 1 dense
  int r0, m, c0, n, rank;
  long long offU, offV;   // element offsets in the far buffer (dense: offU)
};
struct NearDesc { int i, j; long long off; };

void hm_group_forget(hm_ctx* h);   // drops grouped-solve graphs that use h
}  // namespace hm

struct hm_ctx {
  hm_params p;
  int N = 0, nl = 0;
  int dev = 0;
  cudaStream_t stream = 0;
  std::vector<long long> perm, leaf_off;
  std::vector<int> m;                      // leaf sizes
  // host copies of the structure
  std::vector<hm::NearDesc> near;
  std::vector<hm::FarDesc> far;
  // scaling, indexed by elimination rank q (leaf elim[q] is eliminated q-th)
  std::vector<int> elim;                   // rank -> leaf
  std::vector<std::vector<int>> rows;      // alpha pattern, rows[q] = {ranks > q}
  std::vector<long long> alpha_off;        // per (k, j) in row order
  std::vector<long long> alpha_row_start;  // index of first (k, .) in alpha_off
  std::vector<long long> dinv_off;         // per rank
  std::vector<double> leaf_cen;            // leaf cell centres (built handles)
  // supernodes (nested-dissection groups of consecutive ranks)
  std::vector<int> grp;                    // group g = ranks [grp[g], grp[g+1])
  std::vector<long long> tg_off;           // T_G offset (elements) per group
  std::vector<int> tg_n;                   // n_G (0: single-leaf group, no T_G)
  std::vector<int> rloc;                   // rank -> row offset inside its group
  std::vector<hm::cplx> h_tinv;
  hm::cplx* d_tinv = nullptr;              // T_G = (I - A_G^T)^-1, row-major
  double wavelength = 1.0, k = 0.0;
  bool has_scaling = false;
  // non-symmetric system (imported CFIE): every near and far block is stored
  // for its own order and applied one way, and the forward sweep applies the
  // left coefficients (stored transposed, in alpha's layout and offsets)
  bool nonsym = false;
  std::vector<hm::cplx> h_alphaL;
  hm::cplx* d_alphaL = nullptr;
  // device data
  int* d_perm = nullptr;
  hm::cplx* d_near = nullptr;   long long near_elems = 0;
  hm::cplx* d_far = nullptr;    long long far_elems = 0;
  hm::cplx* d_alpha = nullptr;  long long alpha_elems = 0;
  hm::cplx* d_dinv = nullptr;   long long dinv_elems = 0;
  // host copies kept for save / rebuild (FP64 values)
  std::vector<hm::cplx> h_near, h_far, h_alpha, h_dinv;
  // schedules
  hm::Sweep fwd, bwd;
  hm::TaskList dinv_tl, far1_tl, far2_tl, near_tl;
  hm::TaskList far1s_tl;   // far stage 1 stacked by source cluster (tensor-core engines)
  int far_t_rows = 0;           // rows of VB_FAR (2 * sum rank)
  bool sched_ready = false;
  // work buffers sized for cap_nrhs
  int cap_nrhs = 0;
  hm::cplx* d_vec[hm::NPHYS] = {nullptr};
  size_t vec_rows[hm::NPHYS] = {0};
  int last_nrhs = 0;
  void* mixed = nullptr;        // low-precision copies (hm_mixed.cu)
  // mesh (hm_build handles only)
  double* d_verts = nullptr;
  int* d_tris = nullptr;
  int* d_edge = nullptr;
  double* mesh_q = nullptr;     // nt x 7 x 3 quadrature points
  double* mesh_area = nullptr;
  int* mesh_tri[2] = {nullptr, nullptr};
  int* mesh_fv[2] = {nullptr, nullptr};
  double* mesh_len = nullptr;
  std::vector<double> verts;
  std::vector<int> tris, edge;
  double* d_norms = nullptr;    // 4 * cap_nrhs
  int* d_err = nullptr;         // device status word (bounded waits that timed out)
  hm::RowExp rexp_near, rexp_far1, rexp_far2, rexp_dinv, rexp_far1s;
  int* d_fexp = nullptr;        // 2 * cap_nrhs column exponents
  unsigned char* d_xdig[2] = {nullptr, nullptr};   // digit / split panels (OzPanels, XSplit)
  // profiling (hm_profile_enable)
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  std::vector<hm::ProfRec> recs;
  size_t evused = 0;
  std::vector<double> ratio, resid;
  int last_terms = 0;           // series terms of the last solve (largest over its series)
  int tuned_phases = 0;         // sweep phases whose split size the autotuner set
  size_t dev_bytes = 0;
  // bumped whenever device buffers or task lists are replaced; a grouped-solve
  // graph captured under another value refers to freed memory and is rebuilt
  unsigned long long gen = 0;
};

namespace hm {
// kernels.cu
hm_status launch_tasks(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                       cudaStream_t s, int prec = PREC_64, long long spin_limit = 1LL << 26,
                       int* err = nullptr);
hm_status launch_fin(const FinList& fl, const VBufs& vb, int nrhs, cudaStream_t s,
                     int prec = PREC_64);
hm_status launch_gather_perm32(const cplx* B, float2* V, const int* perm, int N, int nrhs,
                               cudaStream_t s);
hm_status launch_to32(const cplx* a, float2* o, size_t n, cudaStream_t s);
hm_status launch_axpby64_32(cplx* o, double sa, const float2* b, double sb, size_t n,
                            cudaStream_t s);
hm_status launch_axpby32(float2* out, const float2* a, float sa, const float2* b, float sb,
                         size_t n, cudaStream_t s);
hm_status launch_col_norms2_32(const float2* V, int N, int nrhs, double* out, cudaStream_t s);
// hm_tc.cu: tensor-core gather for complex64 task lists (tasks with 2m <= 256)
bool tc_ok_for(const TaskList& tl);
// hm_oz.cu: FP64-accurate products on tensor cores
hm_status launch_col_exp(const cplx* V, int rows, int nrhs, int* out, cudaStream_t s);
hm_status launch_col_exp32(const float2* V, int rows, int nrhs, int* out, cudaStream_t s);
// Digit panels of the inputs of the FP64-accurate products: eight planes of
// signed 7-bit digits of a vector panel, tiled exactly as the MMA reads them
// from shared memory (xd[0]: the VB_IN input, xd[1]: the VB_FAR input).
struct OzPanels {
  const unsigned char* xd[2];
  long long J[2];   // 4-row groups of each panel
  int G;            // 8-RHS groups of both panels
};
hm_status build_oz_units(TaskList& tl, size_t* dev_bytes, bool list_order = false);
long long oz_row_groups(int rows);
int oz_rhs_groups(int nrhs);
size_t oz_panel_bytes(int rows, int nrhs);
hm_status launch_digitize(const void* V, bool f32, int rows, int nrhs, const int* fexp,
                          unsigned char* out, long long J, int G, cudaStream_t s);
hm_status launch_tasks_oz(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, const int* row_exp, const long long* exp_off,
                          const int* fexp_in, const int* fexp_far, const OzPanels& xp,
                          long long spin_limit, int* err, bool panels32 = false);
// Split panels of tensor-core inputs that stay fixed during a launch: the three
// bf16 slices of a complex64 panel, tiled so that a 16-row stage of one slice
// is one contiguous block in the MMA's shared-memory layout (xs[0]: the VB_IN
// input, xs[1]: the VB_FAR input; J and G as for OzPanels).
struct XSplit {
  const unsigned char* xs[2];
  long long J[2];
  int G;
};
size_t tc_split_bytes(int rows, int nrhs);
// the split panels of a mixed-precision handle (false when not allocated)
bool mixed_xsplit(hm_ctx* h, XSplit* xs, unsigned char** bufs);
hm_status launch_split(const float2* V, int rows, int nrhs, unsigned char* out, long long J, int G,
                       cudaStream_t s);
// complex64 sweep finalize that also writes the split panel of its rows
hm_status launch_fin_split(const FinList& fl, const VBufs& vb, int nrhs, unsigned char* xs,
                           long long J, int G, cudaStream_t s);
// tensor-core gather of a complex64 list whose inputs come from split panels
hm_status launch_tasks_tc(const TaskList& tl, const VBufs& vb, const ABufs& ab, int nrhs,
                          cudaStream_t s, long long spin_limit, int* err, const XSplit* xsp);
// pre-split the complex64 matrix operand of a tensor-core task list (set-up);
// its stages start on the 4-row boundaries of the split panels
hm_status build_tc_tiles(TaskList& tl, const ABufs& ab, size_t* dev_bytes);
hm_status launch_gather_perm(const cplx* B, cplx* V, const int* perm, int N, int nrhs,
                             cudaStream_t s);
hm_status launch_scatter_perm(const cplx* V, cplx* X, const int* perm, int N, int nrhs,
                              cudaStream_t s);
hm_status launch_axpby(cplx* out, const cplx* a, double sa, const cplx* b, double sb,
                       size_t n, cudaStream_t s);
hm_status launch_col_norms2(const cplx* V, int N, int nrhs, double* out, cudaStream_t s);
hm_status launch_plane_wave(const double* d_verts, const int* d_tris, const int* d_edge_tri,
                            int N, double k, const double* d_ang, int nrhs, cplx* B,
                            cudaStream_t s);
// api.cu helpers
hm_status cuda_status(cudaError_t e);
// adaptive term count: squared column norms of a leaf-order panel (complex128,
// or complex64 when f32) copied to the host (synchronises the stream), and the
// stopping rule of hm_params.term_tol on the squared norms of the first, the
// previous and the latest term
hm_status term_norms(hm_ctx* h, const void* v, bool f32, int nrhs, std::vector<double>& out);
bool terms_stop(const std::vector<double>& n0, const std::vector<double>& nprev,
                const std::vector<double>& nt, double tol);
int prof_begin(hm_ctx* h);                                   // -1 when disabled
void prof_end(hm_ctx* h, int ev, int cat, double bytes, double flops);
// kernels launched by the library in this process (hm_get_stats)
void note_launch();
long long launch_count();
}  // namespace hm

#define HM_LAUNCHED()              \
  do {                             \
    hm::note_launch();             \
    HM_CUDA(cudaGetLastError());   \
  } while (0)
#define HM_CUDA(x)                                       \
  do {                                                   \
    cudaError_t _e = (x);                                \
    if (_e != cudaSuccess) return hm::cuda_status(_e);   \
  } while (0)
