/*
 * pmmm.h -- C ABI of the GB300 particle mesh multipole method library (libpmmm.so).
 *
 * The library computes, for N point charges (or masses) in a rectangular box
 * split into a uniform mesh of cells, the potential and force on every
 * particle with the particle mesh multipole method (PMMM) of K. Nitadori,
 * arXiv:1409.5981.  The problem statement follows Sec. 2.1 of the paper:
 * N particles in K uniform cells; multipole moments of (p+1)^2 real numbers per
 * cell (App. A.7); the cell convolution L_i = sum_j G_{i-j} M_j of Eq. pmmm done
 * with FFTs (Sec. 2.1), zero-padded to twice the mesh per axis for open
 * boundaries (App. C); the nearest (2c+1)^3 cells masked out of G and summed
 * directly as a pure 1/r near field (Sec. 2.1, Sec. 2.2); periodic boundaries
 * through the Ewald-split Green function of App. B with the corrections of
 * App. B.3.
 *
 * Conventions shared by every call:
 *   - Status: every function returning int returns PMMM_OK (0) or a negative
 *     PMMM_ERR_* code; no call aborts or prints.  pmmm_strerror() names a code.
 *   - Memory: pointers passed to pmmm_compute are DEVICE pointers of the
 *     current CUDA device, owned by the caller, and must stay valid until the
 *     work queued on the plan's stream has finished.  The plan owns its own
 *     workspace (allocated in pmmm_plan_create / pmmm_plan_reserve).
 *   - Element types: double for PMMM_FP64, float for the FP32 precisions.
 *   - Layout: positions and forces are array-of-structs, n x 3 (x, y, z);
 *     charges and potentials n.  Results are in the caller's particle order.
 *   - Streams: work is queued on the stream given at plan creation (NULL = the
 *     legacy default stream); calls return without waiting except where noted.
 *   - Physics: phi_i = sign * sum_{j != i} q_j / |r_i - r_j| (sign = +1 Coulomb,
 *     sign = -1 gravity with G = 1); force_i = -q_i grad phi_i.  Periodic
 *     results are those of the Ewald sum with tin-foil boundary conditions.
 */
#ifndef PMMM_H
#define PMMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMMM_ABI_VERSION 1

/* Boundary condition (abstract of the paper: open and periodic). */
typedef enum { PMMM_OPEN = 0, PMMM_PERIODIC = 1 } pmmm_boundary;

/* Arithmetic of the hot path.  FP64: everything in double.  FP32: binning,
 * Green-function set-up and global reductions in double, P2M / FFT / M2L /
 * L2P / near field in float.  FP32_SPLITBF16_M2L is reserved for the batched
 * tensor-core M2L and currently behaves as FP32. */
typedef enum { PMMM_FP64 = 0, PMMM_FP32 = 1, PMMM_FP32_SPLITBF16_M2L = 2 } pmmm_precision;

/* Near-field kernel (Sec. 2.2's direct sum over the (2c+1)^3 nearest cells; the
 * choice changes only the order of floating-point sums):
 *   PMMM_NEAR_CELL_ITEMS  one warp per work item (a cell and up to 32 of its
 *                         particles), sources staged per warp: for filled cells
 *   PMMM_NEAR_PER_TARGET  one thread per particle (FP32 precisions, c = 1 only):
 *                         for sparsely filled cells
 *   PMMM_NEAR_AUTO        per target when N < PMMM_NEAR_AUTO_OCCUPANCY x cells
 *                         (and it applies), else cell items
 *   PMMM_NEAR_CELL_ITEMS_SPLIT  cell items, with the far field on a second stream
 *                         beside them (FP32 precisions; see PMMM_INFO_SPLIT) */
typedef enum {
  PMMM_NEAR_AUTO = 0,
  PMMM_NEAR_CELL_ITEMS = 1,
  PMMM_NEAR_PER_TARGET = 2,
  PMMM_NEAR_CELL_ITEMS_SPLIT = 3
} pmmm_near_field;
#define PMMM_NEAR_AUTO_OCCUPANCY 8

enum {
  PMMM_OK = 0,
  PMMM_ERR_INVALID_ARG = -1,     /* NULL pointer, bad size, bad config field */
  PMMM_ERR_UNSUPPORTED = -2,     /* valid but not implemented (mesh not a power of two, p too high, ...) */
  PMMM_ERR_OUT_OF_BOX = -3,      /* open boundary: a particle outside [lo, lo + len) */
  PMMM_ERR_NONFINITE_INPUT = -4, /* a position is NaN or infinite */
  PMMM_ERR_CUDA = -5,            /* a CUDA runtime call or kernel launch failed */
  PMMM_ERR_TIMEOUT = -6,         /* a bounded device-side wait gave up */
  PMMM_ERR_OOM = -7              /* device allocation failed */
};

/* Problem configuration.  Initialise with pmmm_config_init() and set fields. */
typedef struct pmmm_config {
  double box_lo[3];    /* lower corner of the box */
  double box_len[3];   /* box side lengths b_x, b_y, b_z (> 0) */
  int32_t mesh[3];     /* cells per axis; powers of two, 1..256 (open) or 4..512 (periodic, >= 2c+1) */
  int32_t p;           /* expansion order 0..12 (gradients need p >= 1; at p = 0 only the near field has a gradient) */
  int32_t cutoff;      /* c: minimum cell separation of the far field; 1 -> 27 near cells, 2 -> 125 */
  int32_t boundary;    /* pmmm_boundary */
  int32_t precision;   /* pmmm_precision */
  int32_t near_field;  /* pmmm_near_field: near-field kernel (results agree to rounding) */
  double sign;         /* +1 Coulomb, -1 gravity */
  double ewald_alpha;  /* periodic splitting parameter; 0 -> 1.5 / min(box_len) (App. B.1 example) */
  int32_t ewald_nmax;  /* periodic lattice sums over |n|_2 <= nmax (both sums); 0 -> 5.  The
                        * M2L uses the parity of the converged kernel; a small nmax leaves an
                        * asymmetry of about erfc(alpha b nmax) (2e-10 at nmax = 3 with
                        * alpha b = 1.5, below 1e-25 at 5) */
  int32_t refine;      /* two-level PMMM (Sec. 5, hierarchical treatment): 0 or 1 -> one level;
                        * r = 2, 4, 8 or 16 -> mesh is the fine mesh, every r^3 block of fine cells
                        * one coarse cell (mesh divisible by r; the coarse mesh obeys the mesh rules
                        * above); single-system evaluations only (pmmm_compute, pmmm_compute_host) */
  int32_t reserved[6];
} pmmm_config;

typedef struct pmmm_plan pmmm_plan;

/* ABI version of the loaded library (PMMM_ABI_VERSION). */
int pmmm_abi_version(void);

/* Fills *cfg with defaults: unit box at the origin, mesh 8^3, p = 4, c = 1,
 * open boundary, FP64, sign +1, alpha and nmax automatic. */
void pmmm_config_init(pmmm_config* cfg);

/* Validates cfg, allocates the plan's workspace on the current device and
 * precomputes the Fourier spectra of the (2p+1)^2 Green-function components
 * (Sec. 2.1: "performed and saved at the beginning"; App. B for periodic).
 * Synchronises the stream before returning.  cuda_stream: a cudaStream_t or NULL.
 * On error *out is set to NULL and nothing is leaked. */
int pmmm_plan_create(const pmmm_config* cfg, void* cuda_stream, pmmm_plan** out);

/* Releases the plan and its device memory (synchronises its stream first).  NULL is accepted. */
int pmmm_plan_destroy(pmmm_plan* plan);

/* Pre-allocates particle workspace for up to n_max particles, so that later
 * pmmm_compute calls with n <= n_max allocate nothing. */
int pmmm_plan_reserve(pmmm_plan* plan, int64_t n_max);

/* One full force evaluation (all steps of the hot path on the plan's stream):
 * binning and stable counting sort by cell (Sec. 2.1), P2M (Eq. P2M), forward
 * FFTs of the (p+1)^2 channels, per-wavevector M2L (Eq. realmatrix), inverse
 * FFTs, periodic corrections (App. B.3), L2P with the order-one gradient
 * (Eqs. L2P, L2L, phigrad) and the (2c+1)^3-cell near field.
 * Two-level plans (cfg.refine = r >= 2, Sec. 5 hierarchical treatment): the
 * cell convolution becomes P2M about the coarse centres (Eq. P2M), the
 * one-level convolution on the coarse mesh (its (2c+1)^3 nearest
 * coarse cells masked, periodic corrections taken at the coarse level), the
 * free-space M2L between the fine cells of every masked coarse block (a
 * zero-padded block convolution, its (2c+1)^3 nearest fine cells masked) and L2L
 * of the coarse locals to the fine centres (Eq. L2L); the near field covers the
 * (2c+1)^3 nearest fine cells.
 *   n       number of particles (>= 0; n <= 2^31 - 1)
 *   pos     device, n x 3 positions (double for FP64, float otherwise)
 *   q       device, n charges / masses
 *   phi     device, n potentials (output; may be NULL)
 *   force   device, n x 3 forces (output; may be NULL)
 *   energy  HOST pointer or NULL; if given, receives U = 1/2 sum q_i phi_i
 *           (FP64 reduction) and the call synchronises the stream and also
 *           reports input errors (out-of-box, non-finite) detected on device.
 * Without `energy` the call is asynchronous: input errors detected on the device
 * are reported by the next pmmm_plan_status().  Invalid positions never cause an
 * out-of-bounds access: they are clamped into a cell and flagged.
 * Launch form: the first call with given n, pointers and plan workspace queues
 * the kernels one by one; from the second such call in a row on, the plan
 * launches a CUDA graph of the same sequence (captured once on a plan-owned
 * stream, launched on the plan's stream: same kernels, same results bit for
 * bit, one host call per evaluation).  Calls made while stage timing is on
 * (pmmm_plan_set_timing) or while the caller is capturing the plan's stream
 * queue the kernels one by one. */
int pmmm_compute(pmmm_plan* plan, int64_t n, const void* pos, const void* q, void* phi, void* force, double* energy);

/* Same as pmmm_compute with HOST arrays (pinned memory recommended): copies
 * the inputs to plan-owned device buffers, computes (with the launch form of
 * pmmm_compute), and copies phi / force back; synchronises the stream and
 * returns the device-side status.  */
int pmmm_compute_host(pmmm_plan* plan, int64_t n, const void* pos, const void* q, void* phi, void* force,
                      double* energy);

/* The batched form: nsys independent systems in one evaluation.  They share the
 * plan's box, mesh, p, cutoff, boundary and precision; system s holds the
 * particles offsets[s] ... offsets[s+1]-1 of the concatenated arrays, and its
 * results are those of pmmm_compute on its particles alone (up to rounding).
 * Every step runs once over all systems, laid side by side as nsys meshes of K
 * cells (system s owns cells s*K ... s*K + K-1 in the exports below).  The M2L
 * of Sec. 2.1 becomes, per wavevector k, one complex matrix product
 * L~(k) = A~(k) M~(k) with M~(k) a (p+1)^2 x nsys matrix and A~(k) the
 * real-matrix M2L of App. A.8 on the shared Green spectra.
 *   nsys      1 <= nsys <= PMMM_MAX_SYSTEMS, nsys * K <= 2^30 (else PMMM_ERR_UNSUPPORTED)
 *   offsets   HOST int64[nsys+1]: offsets[0] = 0, non-decreasing,
 *             n = offsets[nsys] <= 2^31 - 1; systems may be empty
 *   pos, q, phi, force  device arrays of the n particles, as in pmmm_compute
 *   energies  HOST double[nsys] or NULL: U of each system; if given, the call
 *             synchronises and returns the device-side status.
 * The plan grows its mesh workspace to nsys systems on first use (allocation,
 * stream synchronised).  New offsets are uploaded through a plan-owned staging
 * buffer after a stream synchronisation; offsets equal to the previous call's
 * are not uploaded again, so a call with unchanged offsets queues only kernels
 * (it can be captured into a CUDA graph once pmmm_plan_reserve_batched and one
 * uncaptured call with the same offsets and no larger n have been made). */
#define PMMM_MAX_SYSTEMS 65535
int pmmm_compute_batched(pmmm_plan* plan, int32_t nsys, const int64_t* offsets, const void* pos, const void* q,
                         void* phi, void* force, double* energies);

/* pmmm_compute_batched with HOST pos, q, phi, force (see pmmm_compute_host);
 * synchronises and returns the device-side status. */
int pmmm_compute_batched_host(pmmm_plan* plan, int32_t nsys, const int64_t* offsets, const void* pos, const void* q,
                              void* phi, void* force, double* energies);

/* pmmm_compute_batched replayed from a CUDA graph: the first call (and any call
 * whose offsets or array pointers differ from those of the graph, or made after
 * the plan's workspace was reallocated or re-tuned) uploads the offsets,
 * reserves the workspace, captures the whole evaluation into a graph on a
 * plan-owned stream and instantiates it; every call then launches the graph on
 * the plan's stream (any stream, the legacy default stream included), so one
 * host call queues every kernel of the evaluation.  The graph reads the arrays
 * at the pointers it was captured with: reuse the same buffers to avoid a new
 * capture.  Per-stage timing is not recorded. */
int pmmm_compute_batched_graph(pmmm_plan* plan, int32_t nsys, const int64_t* offsets, const void* pos,
                               const void* q, void* phi, void* force, double* energies);

/* Pre-allocates the workspace for nsys systems and n_max particles in total. */
int pmmm_plan_reserve_batched(pmmm_plan* plan, int32_t nsys, int64_t n_max);

/* Synchronises the plan's stream and returns (and clears) the first error
 * recorded on the device by earlier pmmm_compute calls. */
int pmmm_plan_status(pmmm_plan* plan);

/* Copies an internal result of the last evaluation to host memory, for tests
 * and diagnostics (synchronises).  bytes must equal the size stated; K below is
 * the cell count of all systems of that evaluation (nsys * cells per system),
 * and a cell id of system s is s * (cells per system) + its own id:
 *   PMMM_EXPORT_PERM        int32[n]     original index of each sorted slot
 *   PMMM_EXPORT_SORTED_CELL int32[n]     cell id (ix + nx (iy + ny iz)) of each sorted slot
 *   PMMM_EXPORT_CELL_START  int32[K+1]   first sorted slot of each cell; [K] = n
 *   PMMM_EXPORT_MULTIPOLE   double[C*K]  M in the real storage of App. A.7, channel-major
 *                                        ([c][cell]), physical units (C = (p+1)^2)
 *   PMMM_EXPORT_LOCAL       double[C*K]  L after the cell convolution, before the
 *                                        periodic corrections, same layout and units
 *   PMMM_EXPORT_CORR        double[8*nsys] per system: total charge Q, sum_cells M_1^0, Re
 *                                        and Im of sum_cells M_1^1, sum q |r_rel|^2, alpha, V, unused
 *   PMMM_EXPORT_FAR         double[4*n]  per sorted slot: far-field phi and grad phi
 *                                        (Coulomb sign, corrections included)
 */
enum {
  PMMM_EXPORT_PERM = 1,
  PMMM_EXPORT_SORTED_CELL = 2,
  PMMM_EXPORT_CELL_START = 3,
  PMMM_EXPORT_MULTIPOLE = 4,
  PMMM_EXPORT_LOCAL = 5,
  PMMM_EXPORT_CORR = 6,
  PMMM_EXPORT_FAR = 7
};
int pmmm_plan_export(pmmm_plan* plan, int what, void* host_dst, size_t bytes);

/* Integer facts about a plan: PMMM_INFO_K (cells), PMMM_INFO_C ((p+1)^2),
 * PMMM_INFO_CG ((2p+1)^2), PMMM_INFO_KH (stored wavevectors per channel),
 * PMMM_INFO_N (particles of the last compute), PMMM_INFO_WORKSPACE_BYTES,
 * PMMM_INFO_LAUNCHES (kernels launched by the last compute), PMMM_INFO_SYSTEMS
 * (systems of the last compute). */
enum {
  PMMM_INFO_K = 1,
  PMMM_INFO_C = 2,
  PMMM_INFO_CG = 3,
  PMMM_INFO_KH = 4,
  PMMM_INFO_N = 5,
  PMMM_INFO_WORKSPACE_BYTES = 6,
  PMMM_INFO_LAUNCHES = 7,
  PMMM_INFO_SYSTEMS = 8,
  PMMM_INFO_TUNED_NEAR = 9, /* near-field kernel chosen by pmmm_plan_autotune (0: none, from the config) */
  PMMM_INFO_M2L_TILE = 10,  /* systems per CTA of the tensor-core batched M2L (32 or 64; default 64) */
  PMMM_INFO_REFINE = 11,    /* refinement of a two-level plan (1: one level) */
  PMMM_INFO_M2L_ARITH = 12, /* arithmetic of the last compute's M2L: PMMM_M2L_ARITH_* (-1 before any) */
  PMMM_INFO_SPLIT = 13      /* 1 if the last compute ran the far field beside the near field (below) */
};
/* Split evaluation (near_field = PMMM_NEAR_CELL_ITEMS_SPLIT, set in the config or
 * chosen by pmmm_plan_autotune; FP32 plans): after the sort, the far field (P2M,
 * mesh stage, periodic corrections, L2P) runs on a second stream of the plan,
 * created with the highest priority, beside the cell-item near field, whose sums
 * go to a workspace buffer (16 bytes per particle, allocated on the first plain
 * call that needs it); one more launch adds the two.  The results equal those of
 * the one-stream sequence bit for bit.  One stream while stage timing is on, for
 * surrogate evaluations and inside a capture that would need the buffer first. */
/* The M2L arithmetic that actually ran.  PMMM_FP32_SPLITBF16_M2L asks for the
 * tensor cores, but they serve only where the per-wavevector M2L is a true matrix
 * product: batched evaluations of more than one system, and the fine-level block
 * M2L of two-level plans, both for p <= 7.  A single one-level system (each
 * wavevector its own matrix-vector product) and p > 7 run the FP32 SIMT M2L;
 * this key says which one a compute used. */
enum {
  PMMM_M2L_ARITH_FP64_SIMT = 0,
  PMMM_M2L_ARITH_FP32_SIMT = 1,
  PMMM_M2L_ARITH_SPLITBF16_TC = 2
};
int pmmm_plan_info(pmmm_plan* plan, int what, int64_t* value);

/* Autotuner: evaluates the given input (nsys systems; offsets as in
 * pmmm_compute_batched, or {0, n} for one system) once per candidate of each
 * tunable choice, timed over `reps` evaluations with CUDA events after one
 * warm-up, and keeps the fastest: the near-field schedule (cell items, cell items
 * with the far field beside them, or per target, where these apply) and, for
 * batched PMMM_FP32_SPLITBF16_M2L plans, the
 * systems per CTA of the tensor-core M2L (64 or 32).  The choice overrides the
 * config's near_field; results differ between choices only by the order of
 * floating-point sums.  Synchronous; reads back with PMMM_INFO_TUNED_NEAR and
 * PMMM_INFO_M2L_TILE. */
int pmmm_plan_autotune(pmmm_plan* plan, int32_t nsys, const int64_t* offsets, const void* pos, const void* q,
                       int32_t reps);

/* Per-stage timing with CUDA events on the plan's stream (off by default).
 * pmmm_plan_stage_times synchronises and writes up to max_stages values in
 * milliseconds for the last compute, in the order of pmmm_stage_name(i);
 * returns the number of stages written. */
int pmmm_plan_set_timing(pmmm_plan* plan, int enable);
int pmmm_plan_stage_times(pmmm_plan* plan, float* ms, int max_stages);
const char* pmmm_stage_name(int i);

/* Binning and stable sort by cell WITHOUT ANY DEVICE ALLOCATION.  The paper has
 * no counterpart: this is a service for callers that cannot call cudaMalloc --
 * a host framework or memory pool that owns all device memory and forbids
 * allocations behind its back, or a real-time loop that must never block in the
 * allocator (cudaMalloc may synchronise the device and take an unbounded
 * time).  It computes the first step of pmmm_compute
 * (same FP64 cell-index formula, same stable order) for the geometry of cfg
 * (box, mesh, boundary, precision; p and cutoff are ignored):
 *   n           number of particles, 0 <= n <= PMMM_STATIC_SORT_MAX_N
 *   pos         device, n x 3 positions (double for PMMM_FP64, float otherwise)
 *   perm        device int32[n] output: original index of each sorted slot
 *   cell_start  device int32[K+1] output: first sorted slot of each cell, [K] = n
 *   cuda_stream cudaStream_t or NULL; every call waits for this stream to
 *               finish (it reads the device-side status back) and returns that
 *               status (PMMM_ERR_OUT_OF_BOX / _NONFINITE_INPUT as in
 *               pmmm_compute).
 * All scratch lives in one file-scope device array of about 3 MiB that every
 * GPU loading this library keeps until the process exits; n above
 * PMMM_STATIC_SORT_MAX_N returns PMMM_ERR_UNSUPPORTED.  The first call on a
 * device looks up the array's device address (with that device current): make
 * it before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU (other streams or host threads) race and must not be made. */
#define PMMM_STATIC_SORT_MAX_N 65536
int pmmm_bin_sort_static(const pmmm_config* cfg, int64_t n, const void* pos, int32_t* perm, int32_t* cell_start,
                         void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Learned local-expansion correction.  The paper has no counterpart; this is an
 * added form of the method.  A multilayer perceptron 432 -> 256 -> 256 -> 121
 * (GELU; BF16 operands, FP32 accumulation on the tensor cores; FP32 master
 * parameters) maps, for every cell, the order-3 multipoles (16 real storage
 * channels, App. A.7) of its 27 nearest cells to the difference between the
 * cell's order-p_high local expansion and its order-3 one.  An evaluation then
 * runs the order-3 pipeline up to the cell convolution (Sec. 2.1), adds the
 * network's correction to the order-3 locals, and runs L2P (Eqs. L2P, phigrad)
 * at order p_high plus the usual near field.  The plain order-p_high
 * evaluation produces the training targets, and pmmm_surrogate_set_fallback
 * routes evaluations to it (used when the held-out error exceeds its bound).
 *
 * Units: features are M'_l = M_l / h^l times in_scale[channel]; targets and
 * outputs are (L'_l(p_high) - L'_l(3)) times out_scale[channel], L'_l = h^(l+1) L_l,
 * with h the cell size.  Parameter vector (FP32, PMMM_SUR_NPARAM values):
 * W1 [256 x 432], b1 [256], W2 [256 x 256], b2 [256], W3 [128 x 256], b3 [128]
 * (rows >= (p_high+1)^2 of W3 and b3 are padding).  Feature rows are ordered
 * neighbour-major ((dz, dy, dx) in {-1,0,1}^3, dx fastest) then channel.
 * Row counts passed to the calls below are multiples of 128.
 * ------------------------------------------------------------------------- */
typedef struct pmmm_surrogate pmmm_surrogate;
#define PMMM_SUR_IN 432
#define PMMM_SUR_OUT_ROWS 128
#define PMMM_SUR_NPARAM 209536
enum { PMMM_SUR_PARAMS = 1, PMMM_SUR_ADAM_M = 2, PMMM_SUR_ADAM_V = 3, PMMM_SUR_IN_SCALE = 4, PMMM_SUR_OUT_SCALE = 5 };
enum {
  PMMM_SUR_INFO_STEP = 1,     /* Adam steps taken */
  PMMM_SUR_INFO_FALLBACK = 2, /* 1 when evaluations run the plain order-p_high method */
  PMMM_SUR_INFO_CLOW = 3,     /* 16 */
  PMMM_SUR_INFO_CHIGH = 4,    /* (p_high + 1)^2 */
  PMMM_SUR_INFO_ROWS = 5      /* feature rows of one system: cells rounded up to 128 */
};

/* cfg: the order-3 configuration (p = 3, cutoff 1, PMMM_FP32); p_high in 4..10.
 * Creates both the order-3 and the order-p_high plans on the stream; parameters
 * and Adam state start at zero, scales at one. */
int pmmm_surrogate_create(const pmmm_config* cfg, int32_t p_high, void* cuda_stream, pmmm_surrogate** out);
int pmmm_surrogate_destroy(pmmm_surrogate* s);

/* Host copies of the parameters, Adam moments (PMMM_SUR_NPARAM each) and the
 * input (16) and output ((p_high+1)^2) scales; count must match.  Synchronous. */
int pmmm_surrogate_get(pmmm_surrogate* s, int what, float* host, int64_t count);
int pmmm_surrogate_set(pmmm_surrogate* s, int what, const float* host, int64_t count);
int pmmm_surrogate_info(pmmm_surrogate* s, int what, int64_t* value);
int pmmm_surrogate_set_step(pmmm_surrogate* s, int64_t step);
int pmmm_surrogate_set_fallback(pmmm_surrogate* s, int on);

/* One training example set from one system (device pos / q as in pmmm_compute):
 * runs the plain order-3 and order-p_high evaluations and writes the features
 * X (device, BF16 [rows][432]) and targets T (device, FP32 [rows][128]) of its
 * cells, rows = PMMM_SUR_INFO_ROWS (zero past the last cell).  stats: host
 * double[16 + (p_high+1)^2] or NULL; adds the sums over cells of the squared
 * raw multipole channels and raw target channels (for choosing the scales).
 * Synchronous. */
int pmmm_surrogate_training_pair(pmmm_surrogate* s, int64_t n, const void* pos, const void* q, void* X, float* T,
                                 double* stats);

/* Network output for rows of features: out (device, FP32 [rows][128]).  Synchronous. */
int pmmm_surrogate_forward(pmmm_surrogate* s, const void* X, int64_t rows, float* out);
/* Loss (mean over rows and the (p_high+1)^2 outputs of the squared error) and its
 * gradient with respect to the parameters (host, PMMM_SUR_NPARAM, may be NULL);
 * no update.  Synchronous. */
int pmmm_surrogate_gradients(pmmm_surrogate* s, const void* X, const float* T, int64_t rows, float* grad_host,
                             double* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch; loss (host) may be
 * NULL, in which case the call is asynchronous. */
int pmmm_surrogate_train_step(pmmm_surrogate* s, const void* X, const float* T, int64_t rows, float lr, double* loss);
/* Potential and force with the corrected locals (or the plain order-p_high
 * method in fallback); arguments as pmmm_compute. */
int pmmm_surrogate_compute(pmmm_surrogate* s, int64_t n, const void* pos, const void* q, void* phi, void* force,
                           double* energy);

/* Peak probes (measurement, the paper has no counterpart): the FMA rate of this
 * GPU, measured by a kernel of independent FMA chains (eight per thread, eight
 * resident blocks of 256 threads on every SM) timed with CUDA events, best of
 * five launches after a warm-up.  what: PMMM_PROBE_FP32_FMA (fma.rn.f32),
 * PMMM_PROBE_FP32X2_FMA (packed fma.rn.f32x2, two lanes per instruction) or
 * PMMM_PROBE_FP64_FMA.  *flops_per_s receives 2 x FMAs per second.  Allocates
 * and frees one small device buffer; synchronises the stream. */
enum { PMMM_PROBE_FP32_FMA = 0, PMMM_PROBE_FP32X2_FMA = 1, PMMM_PROBE_FP64_FMA = 2 };
int pmmm_probe_peak(int what, void* cuda_stream, double* flops_per_s);

/* Diagnostic of the failure detection (the paper has no counterpart): launches
 * one kernel that waits, with the same bounded mbarrier wait as the
 * tensor-core kernels (here at most `polls` polls, 1..2^24), on a barrier that
 * nothing arrives at.  The wait gives up, the kernel raises the device error
 * flag and returns, and the call returns PMMM_ERR_TIMEOUT with the CUDA context
 * still usable.  Synchronises the stream. */
int pmmm_selftest_wait_timeout(void* cuda_stream, int64_t polls);

/* Human-readable name of a status code (static string). */
const char* pmmm_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* PMMM_H */
