/*
 * hm.h -- C ABI of the GB300 power-series H-matrix EFIE solver.
 *
 * Method: Negi, Balakrishnan, Rao, "Fast Power Series Solution of Large 3-D
 * Electrodynamic Integral Equation for PEC Scatterers" (arXiv 2109.04129).
 * The system is the EFIE method-of-moments system [Z] x = b (Eq. 9) for a
 * perfectly conducting surface, Galerkin tested with RWG functions (Sec. II),
 * stored as an H-matrix Z = Z_N + Z_F (Eq. 13) and solved by the two-term
 * power series of the near-field-scaled system (Eq. 24-36).
 *
 * Conventions for every entry point:
 *  - No exception or C++ type crosses this boundary; every call returns an
 *    hm_status.  Pointers named *_host are host memory; X and B of
 *    hm_power_series_solve / hm_apply / hm_plane_wave_rhs are DEVICE memory
 *    owned by the caller (the library never frees them).
 *  - Complex vectors are complex128 interleaved (re, im), column-major
 *    N x nrhs (column r starts at element r*N), in ORIGINAL RWG order
 *    (unknown n = n-th interior edge in ascending (min vertex, max vertex)).
 *  - Device work is ordered on the stream given to hm_set_stream (default:
 *    the legacy default stream).  Calls that return values to the host
 *    synchronise that stream.  A device-side error (a bounded wait that timed
 *    out, a singular block) is reported by the next synchronising call.
 *  - Required order: hm_build or hm_import -> hm_compute_scaling (unless the
 *    imported file carries scaling) -> solves.  Otherwise HM_ERR_STATE.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns HM_ERR_CUDA.
 */
#ifndef HM_H
#define HM_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hm_ctx* hm_handle;   /* opaque; owns all device storage */

typedef enum {
  HM_OK = 0,
  HM_ERR_INVALID = 1,    /* bad argument, malformed mesh or file          */
  HM_ERR_CUDA = 2,       /* CUDA runtime error or no device               */
  HM_ERR_OOM = 3,        /* device or host allocation failed             */
  HM_ERR_SINGULAR = 4,   /* a scaled diagonal block has no usable pivot  */
  HM_ERR_TIMEOUT = 5,    /* a bounded device wait ran out                */
  HM_ERR_STATE = 6,      /* call out of order                            */
  HM_ERR_IO = 7,         /* file could not be read or written           */
  HM_WARN_SERIES_RATIO = 100 /* solve done; some ||it_1||/||it_0|| > 0.1 (Eq. 45) */
} hm_status;

enum { HM_FP64 = 0,        /* every product in complex FP64                   */
       HM_MIXED = 1,       /* scaling/far products in low precision with FP32
                              accumulation, D^-1 in FP64, FP64 refinement     */
       HM_MIXED_BF16 = 1 };/* the same mode by its operand type: the products
                              are three-way bf16 slice products (about 24
                              significant bits).  There is no TF32 mode: a
                              tf32 operand keeps 10 mantissa bits             */
enum { HM_ORDER_DFS = 0,   /* leaves in octree depth-first (Morton) order    */
       HM_ORDER_ND = 1 };  /* geometric nested dissection of the leaf graph  */
enum { HM_FILL_FULL = 0,   /* scaling keeps every fill-in block (Eq. 23 exact) */
       HM_FILL_NEAR = 1 }; /* fill restricted to the near-field pattern      */

typedef struct {
  double wavelength;     /* metres; k = 2 pi / wavelength (or see freq_hz)    */
  int leaf_max;          /* octree leaf cap in unknowns (Sec. II, V-A)         */
  int ordering;          /* HM_ORDER_*: elimination order of the leaves        */
  double aca_tol;        /* ACA / recompression tolerance eps of Eq. 12        */
  int fill;              /* HM_FILL_*                                          */
  int n_terms;           /* terms of Eq. 36 kept (paper: 2)                    */
  int precision;         /* HM_FP64 or HM_MIXED                                */
  int refine_steps;      /* refinement steps on the FP64 residual (mixed: 1)   */
  long long spin_limit;  /* iteration cap of every device-side wait           */
  int tensor_cores;      /* HM_MIXED products on tcgen05 tensor cores (three-way
                            bf16 split, FP32 accumulation) when nrhs >= 32:
                            1 (default) or 0 for the CUDA-core FP32 kernels    */
  int fp64_emulation;    /* HM_MIXED refinement residual (FP64-accurate products)
                            on tensor cores by exact 7-bit integer slicing of the
                            FP64 operands: 1 (default), or 0 for the FP64 units  */
  double term_tol;       /* 0 (default): exactly n_terms terms of Eq. 36.  > 0:
                            adaptive term count (Sec. III-C, Eq. 44-45): after
                            each term it_t, t >= 1, the series stops when every
                            RHS has ||it_t|| <= term_tol ||it_0|| (converged),
                            or when some RHS has ||it_t|| >= ||it_(t-1)|| (its
                            terms no longer shrink: the ratio of Eq. 45 is at
                            least one), and at n_terms terms in any case.  The
                            solve then synchronises its stream once per term.  */
  int autotune;          /* HM_MIXED with tensor cores: 1 (default) times the
                            candidate split-K sizes of every sweep phase on the
                            first solve with a new number of 128-RHS tiles and
                            keeps the fastest (cached per phase shape for the
                            process); that solve synchronises its stream, so
                            make it before any stream capture.  0 keeps the
                            built-in choice                                     */
  int tc_split_max;      /* largest split-K size (inner rows) of a tensor-core
                            sweep task, a power of two from 128; 0 (default):
                            2048.  Shorter tasks keep shorter FP32 sums in
                            tensor memory and hand more partial sums to the
                            (IEEE FP32) finalize; they change the mixed
                            chain's error little (its MMAs round each partial
                            sum, which is as large as the whole)                */
  double eta;            /* admissibility of two octree cells (Eq. 10) in
                            hm_build: 0 (default) = far exactly when the cells
                            do not touch (no shared face, edge or vertex); > 0 =
                            far when they do not touch and
                            min(diam) <= eta * dist, diam the cell diagonal and
                            dist the distance between the two cubes, evaluated
                            exactly on integer cell coordinates
                            (3 min(edge)^2 <= eta^2 sum(gap^2)).  eta >= sqrt 3
                            gives the non-touching partition; smaller eta moves
                            pairs from far to near.  hm_import takes the blocks
                            of its file and ignores it                          */
  double freq_hz;        /* > 0: the frequency in Hz; hm_build then uses
                            wavelength = 299 792 458 / freq_hz (metres) in place
                            of the wavelength field.  0 (default): wavelength  */
  int reserved[2];
} hm_params;

/* Fill *p with the defaults: wavelength 1, leaf_max 64, DFS order, eps 1e-4,
 * full fill, 2 terms, FP64, no refinement, spin_limit 1<<26, tensor_cores 1,
 * fp64_emulation 1, term_tol 0 (fixed term count), autotune 1, eta 0
 * (non-touching admissibility), freq_hz 0. */
void hm_default_params(hm_params* p);

/* Build the H-matrix of a closed or open triangulated PEC surface (Sec. II:
 * RWG basis, octree clusters, non-touching admissibility (Eq. 10), dense
 * near blocks, ACA + recompression far blocks (Eq. 11-12)).
 * verts_host: nv x 3 float64 metres; tris_host: nt x 3 int32, 0-based,
 * counter-clockwise seen from outside.  Both are copied.  Fails with
 * HM_ERR_INVALID for an empty mesh, an out-of-range index or an edge shared
 * by more than two triangles. */
hm_status hm_build(const double* verts_host, int nv, const int* tris_host, int nt,
                   const hm_params* p, hm_handle* out);

/* Load an H-matrix (and, if present, its scaling coefficients) from the
 * neutral block file: leaf order, near blocks, low-rank far blocks, alpha,
 * D^-1 (format in the package documentation).  p supplies the solve
 * options; its tree options are ignored.
 * A file with the non-symmetric section (the CFIE of Eq. 8, whose matrix is
 * not symmetric) gives a handle whose near and far blocks are stored for both
 * orders and applied one way, and whose forward sweep (HM_OP_RT) applies the
 * left scaling coefficients alphaL_kj = -Z~_jk D_k^-1 where the symmetric
 * system applies alpha^T (Sec. III-A without Z = Z^T): x = R sum (-1)^n it_n,
 * it_0 = D^-1 L b, it_n = D^-1 L Z_F R it_(n-1).  Such a handle runs the FP64
 * chain only: HM_MIXED in p, or a supernode section in the file, give
 * HM_ERR_INVALID; hm_compute_scaling and hm_save give HM_ERR_STATE. */
hm_status hm_import(const char* path, const hm_params* p, hm_handle* out);

/* Write the handle's H-matrix and scaling in the same file format
 * (checkpoint of the expensive set-up). */
hm_status hm_save(hm_handle h, const char* path);

/* Schur-complement scaling of the symmetric near field (Sec. III-A,
 * Eq. 14-23): for each leaf k in elimination order D_k = Z~_kk,
 * alpha_kj = -D_k^-1 Z~_kj, Z~_ij += alpha_ki^T Z~_kj; stores alpha and
 * D_k^-1 (FP64, LU with partial pivoting).  HM_ERR_SINGULAR if a pivot
 * vanishes. */
hm_status hm_compute_scaling(hm_handle h);

/* Power-series solve of Z X = B (Eq. 25-36):
 *   b~ = R^T b, b_o = D^-1 b~, w = D^-1 R^T Z_F R b_o, X = R (b_o - w)
 * (n_terms = 2; more terms continue the alternating series).  In HM_MIXED
 * the chain runs in low precision and refine_steps FP64 residual
 * corrections follow.  X, B: device, N x nrhs complex128, original order;
 * B is not modified; X is overwritten.  Asynchronous: the ratio check of
 * Eq. 45 is reported by hm_get_diagnostics. */
hm_status hm_power_series_solve(hm_handle h, void* X, const void* B, int nrhs);

/* Same solve for HOST buffers: copies B in, solves, copies X out (pinned or
 * pageable memory; synchronous). */
hm_status hm_power_series_solve_host(hm_handle h, void* X_host, const void* B_host,
                                     int nrhs);

/* One step of the chain, for per-kernel checks.  Y = op(X), original order,
 * device buffers, N x nrhs complex128:
 *   HM_OP_RT   Y = R^T X      (Eq. 25)       HM_OP_R    Y = R X   (Eq. 26)
 *   HM_OP_DINV Y = Z~_N^-1 X  (Eq. 32)       HM_OP_FAR  Y = Z_F X (Eq. 13)
 *   HM_OP_NEAR Y = Z_N X                      HM_OP_Z    Y = (Z_N + Z_F) X
 * op is applied in the handle's precision. */
enum { HM_OP_RT = 0, HM_OP_R = 1, HM_OP_DINV = 2, HM_OP_FAR = 3, HM_OP_NEAR = 4,
       HM_OP_Z = 5 };
hm_status hm_apply(hm_handle h, int op, void* Y, const void* X, int nrhs);

/* Plane-wave excitation b_m = <f_m, E_inc> (Eq. 2 tested), device output
 * B (N x nrhs complex128).  theta_host/phi_host: incidence angles in radians
 * (E_inc = p exp(-j k khat.r), khat = -(sin t cos p, sin t sin p, cos t));
 * pol_host: 0 = theta-hat, 1 = phi-hat. */
hm_status hm_plane_wave_rhs(hm_handle h, const double* theta_host, const double* phi_host,
                            const int* pol_host, int nrhs, void* B);

/* Grouped solve of many independent problems (a batch of scatterers, each
 * with its own handle, H-matrix and scaling): for every i < count,
 * X[i] = solve(hs[i], B[i], nrhs[i]) exactly as hm_power_series_solve does
 * (Eq. 25-36 per problem; the paper's method is per scatterer, and a batch is
 * a set of independent runs of it).  X[i], B[i]: device, N_i x nrhs[i]
 * complex128, original order, owned by the caller; the handles must be
 * distinct, scaled, and not profiling.  The first call for a given list of
 * (handle, X, B, nrhs) runs one ordinary solve per problem on the first
 * handle's stream and waits for it, then records all of them into one CUDA
 * graph with one branch per problem and keeps the instantiated graph; every
 * call, the first included, then launches that graph on the first handle's
 * stream (asynchronous).  Returns HM_ERR_INVALID for null or repeated handles
 * or non-positive counts, HM_ERR_STATE for a handle without scaling, with
 * profiling on or with an adaptive term count (term_tol > 0: its host-side
 * decisions cannot be recorded), and the first failing solve's status
 * otherwise.  A kept graph is
 * rebuilt when a handle's device buffers or schedules have been replaced
 * since it was recorded, and dropped when one of its handles is destroyed.
 * The call orders itself after the work already queued on every handle's own
 * stream, and later work queued on those streams runs after the graph: a
 * branch uses its handle's work panels.
 * Diagnostics per handle come from hm_get_diagnostics as usual. */
hm_status hm_solve_grouped(hm_handle* hs, void** X, const void** B, const int* nrhs,
                           int count);

hm_status hm_set_stream(hm_handle h, void* cuda_stream);
hm_status hm_num_unknowns(hm_handle h, int* n);

/* Per-RHS diagnostics of the last solve (host arrays of length nrhs, either
 * may be NULL): ratio_host[r] = ||it_1|| / ||it_0|| (Eq. 45); resid_host[r] =
 * ||B - Z X|| / ||B|| of the solution before its last refinement step (0 when
 * no refinement ran).  Synchronises; returns HM_WARN_SERIES_RATIO when some
 * ratio exceeds 0.1 (the paper's empirical convergence bound). */
hm_status hm_get_diagnostics(hm_handle h, double* ratio_host, double* resid_host, int nrhs);

/* Counts, as long long, in this order (up to n of them): N, leaves, near
 * blocks (upper), far blocks (upper), alpha entries, D entries, near entries
 * (upper), far factor entries, max rank, forward levels, backward levels,
 * device bytes held, the number of kernels the library has launched in
 * this process so far (all handles; read it before and after a region to
 * count that region's launches), the number of series terms of the last
 * solve (the largest over its series when refinement steps ran), and the
 * number of sweep phases whose split-K size the autotuner has set. */
hm_status hm_get_stats(hm_handle h, long long* out_host, int n);

/* Copy the leaf-order permutation (N int64, leaf position -> original index)
 * and leaf offsets (leaves + 1 int64) to host arrays. */
hm_status hm_get_tree(hm_handle h, long long* perm_host, long long* leaf_off_host);

/* Per-kernel timing of later device work: when enabled, every launch of the
 * chain is bracketed by CUDA events on the handle's stream.  hm_get_profile
 * synchronises, then writes for each category c < ncat four doubles
 * out_host[4c .. 4c+3] = {launches, total milliseconds, algorithmic bytes,
 * algorithmic real flops} accumulated since the last call (and resets them).
 * Categories: 0 R^T sweep blocks, 1 R sweep blocks, 2 sweep finalize,
 * 3 D^-1, 4 far stage 1 (V^T y), 5 far stage 2 (U t), 6 near product,
 * 7 permutations / axpby / norms, 8 mixed-precision sweep blocks,
 * 9 mixed-precision far field, 10 conversions. */
enum { HM_PROF_CATEGORIES = 11 };
hm_status hm_profile_enable(hm_handle h, int on);
hm_status hm_get_profile(hm_handle h, double* out_host, int ncat);

/* Far-field product that allocates no device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they need the product (code inside a pre-sized pool or
 * arena that owns the device memory, a framework allocator that forbids raw
 * cudaMalloc, latency-critical loops).  It computes Y = Z_F X like hm_apply
 * with HM_OP_FAR (FP64 factors, original RWG order, column-major N x nrhs
 * complex128 device buffers owned by the caller) but calls no cudaMalloc,
 * cudaFree or allocating library routine: its only scratch, 2 * (sum of the
 * far-block ranks) * nrhs complex128 values, lives in a fixed file-scope
 * device array of HM_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits.  Returns HM_ERR_INVALID when that scratch
 * would exceed the array (reduce nrhs), and also when the current device is
 * not the handle's.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress), so make that first call before any stream
 * capture.  Asynchronous on the handle's stream.  All calls share the array:
 * calls whose kernels overlap on the GPU race.  A handle without far blocks
 * gets Y = 0. */
#define HM_NOALLOC_SCRATCH_BYTES (32u << 20)
hm_status hm_apply_far_noalloc(hm_handle h, void* Y, const void* X, int nrhs);

hm_status hm_destroy(hm_handle h);
const char* hm_status_string(hm_status s);

#ifdef __cplusplus
}
#endif
#endif /* HM_H */
