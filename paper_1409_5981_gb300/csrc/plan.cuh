// Private state of a PMMM plan (the opaque pmmm_plan of the C ABI), shared by
// the translation units that drive an evaluation (pmmm.cu, surrogate.cu).
#pragma once
#include <functional>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

enum Stage { ST_SORT = 0, ST_P2M, ST_FFT_FWD, ST_M2L, ST_FFT_INV, ST_L2P, ST_PP, ST_REDUCE, ST_COUNT };

namespace pmmm {
// Called after the cell convolution (locals L ready, before L2P): may replace
// the locals that L2P reads by an array of order p_l2p ([(p_l2p+1)^2][K], same
// device units and type as the plan's L).
struct FarHook {
  std::function<cudaError_t(cudaStream_t, int*)> fn;
  int p_l2p = -1;
  const void* L = nullptr;
};
}  // namespace pmmm

struct pmmm_plan {
  using Dims = pmmm::Dims;
  using Geo = pmmm::Geo;
  using SortWork = pmmm::SortWork;
  pmmm_config cfg;
  cudaStream_t stream = nullptr;
  int p = 0, C = 0, CG = 0;
  bool fp64 = true;
  Dims d{};
  Geo g{};
  int nmax = 5;
  size_t tsize = 8;  // sizeof(T)
  // mesh workspace
  void *M = nullptr, *L = nullptr, *specM = nullptr, *specL = nullptr, *G = nullptr;
  void* Gr = nullptr;  // parity-reduced kernel spectra [C_G][Kh]: one real number per value
  void *twx = nullptr, *twy = nullptr, *twz = nullptr;
  double* cellsum = nullptr;  // [5][K]: sum q, sum q u_x, sum q u_y, sum q u_z, sum q |u|^2
  int* cs = nullptr;          // [K+1]
  double* corr = nullptr;     // [16]
  double* partial = nullptr;  // [256 * 16]
  double* bpartial = nullptr;  // per-system reduction chunks: [5][bcap][bchunks]
  int bchunks = 0;
  double* epart = nullptr;    // [max items][4]
  uint32_t* item_start = nullptr;  // [K+1] near-field work items per cell (scanned)
  uint32_t* item_chunks = nullptr; // scan scratch
  uint32_t* item_cell = nullptr;   // [max items]
  int64_t max_items = 0;
  unsigned int* counter = nullptr; // near-field work counter
  uint32_t* pair_start = nullptr;  // [K+1] FP32 near-field source pairs per cell (scanned)
  void* src2 = nullptr;            // pair-interleaved FP32 sources
  int num_sms = 0;
  double* energy = nullptr;   // [4 * bcap]: energy and net force per system
  int* err = nullptr;
  // systems: the mesh workspace above holds bcap systems side by side
  int bcap = 0;
  int nsys_last = 1;
  int64_t* offsets_d = nullptr;       // [bcap + 1] particle offsets of the systems
  int64_t* offsets_pinned = nullptr;  // host staging of the offsets
  std::vector<int64_t> offsets_up;    // offsets of the last upload
  int* m2l_tab = nullptr;             // batched M2L entry table, 4 ints per entry
  uint32_t* m2l_tab_tc = nullptr;     // packed entry table of the tensor-core M2L
  bool m2l_tc = false;                // batched M2L on the tensor cores (split BF16)
  int m2l_arith = -1;                 // PMMM_M2L_ARITH_* of the last compute's M2L
  std::unordered_map<void*, size_t> sizes;
  // CUDA graph of one evaluation, and what it was captured for: the systems'
  // offsets, the caller's pointers, the workspace generation and the tuning
  // choices.  Captured on a private stream, launched on the plan's stream.
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t cstream = nullptr;
  std::vector<int64_t> gkey_off;
  const void* gkey_ptr[4] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t gkey_gen = 0;
  int gkey_tune[2] = {0, 0};
  bool capturing = false;
  // the last plain single-system call (pmmm_compute takes the graph from the
  // second identical call on)
  std::vector<int64_t> lkey_off;
  const void* lkey_ptr[4] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t lkey_gen = 0;
  uint64_t wgen = 0;  // bumped by every workspace allocation and release
  const pmmm::FarHook* hook = nullptr;  // set by the surrogate for one evaluation
  // choices of pmmm_plan_autotune: near-field kernel (0: from the config), tensor-core M2L system tile
  int tuned_near = 0;
  int m2l_tile = 64;
  // two-level evaluation (cfg.refine >= 2): the coarse level runs on a one-level
  // plan of the coarse mesh; the block convolution of the fine level takes its
  // free-space kernel spectra and twiddles from an open plan of (m/2)^3 fine cells
  bool hier = false;
  pmmm::HierGeo hg{};
  pmmm_plan* coarse = nullptr;
  pmmm_plan* block = nullptr;
  void *hspecM = nullptr, *hspecL = nullptr;  // block spectra, C * Kc * m^2 (m/2+1) complex
  void* hregion = nullptr;                    // kept block outputs, C * Kc * ((2c+1) r)^3
  void* hrtab = nullptr;                      // R(coarse centre - child centre), r^3 * C
  void* hum = nullptr;                        // L2L child matrices, r^3 * C * C (or none)
  // particle workspace
  int64_t cap = 0;
  SortWork sw{};
  void *part = nullptr, *far = nullptr;
  // staging for pmmm_compute_host
  int64_t hcap = 0;
  void *hpos = nullptr, *hq = nullptr, *hphi = nullptr, *hforce = nullptr;
  // last evaluation
  int64_t n_last = 0;
  uint32_t *keys_sorted = nullptr, *vals_sorted = nullptr;
  int launches = 0;
  size_t ws_bytes = 0;
  bool timing = false, timed = false;
  cudaEvent_t ev[ST_COUNT + 1] = {};
  // split evaluation (PMMM_NEAR_CELL_ITEMS_SPLIT, FP32): the far field (P2M .. L2P)
  // runs on `aux` beside the near field, which leaves its sums in `nearv` (float4
  // per sorted particle); fork / join order the two streams
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* nearv = nullptr;
  bool split_last = false;
};


namespace pmmm {
// One evaluation of B systems (pmmm.cu); B > 1 needs the offsets uploaded.
int plan_run(pmmm_plan* pl, int B, int64_t n, const void* pos, const void* q, void* phi, void* force);
int plan_read_energies(pmmm_plan* pl, int B, double* out);
int plan_map_cuda(cudaError_t e);
}  // namespace pmmm
