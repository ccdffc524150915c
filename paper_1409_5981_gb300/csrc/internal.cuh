// Internal declarations of the PMMM GPU library: plan state, geometry and the
// launchers of every kernel.  Not part of the C ABI.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "pmmm.h"

namespace pmmm {

// Mesh and transform geometry.  Physical cells nx*ny*nz; transforms of
// Lx*Ly*Lz points (L = n periodic, L = 2n open, App. C); r2c half spectrum
// along x with hx = Lx/2 + 1 points.
struct Dims {
  int nx, ny, nz;
  int Lx, Ly, Lz;
  int hx;
  int64_t K;   // nx*ny*nz
  int64_t Kt;  // Lx*Ly*Lz
  int64_t Kh;  // Lz*Ly*hx
};

// Physical constants of one plan, in the units the kernels use.  Lengths on
// the device are in units of hs (one scalar cell size); cs[a] = h_a / hs.
struct Geo {
  double lo[3], len[3], inv[3];  // binning: inv = n / len
  double h[3];                   // cell sizes
  double hh[3];                  // h / 2
  double hs;                     // length unit of the device arithmetic
  double ihs;                    // 1 / hs
  double cs[3];                  // h / hs
  double V;                      // box volume
  double alpha;                  // Ewald splitting parameter (physical)
  double sign;
  int n[3];
  int periodic;
  int c;
  // float splits for the FP32 binning path: lo = loh + lol, inv = invh + invl
  float loh[3], lol[3], invh[3], invl[3], csf[3];
};

// The binning geometry of a configuration (box, cells, cell-size units and the
// float splits of the FP32 binning path).  Plan creation and the allocation-free
// sort both take it from here, so their cell ids cannot drift apart.  V, alpha
// and sign are left for the caller.
inline Geo binning_geo(const pmmm_config& cfg) {
  Geo g{};
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = cfg.box_lo[a];
    g.len[a] = cfg.box_len[a];
    g.n[a] = cfg.mesh[a];
    g.inv[a] = (double)cfg.mesh[a] / cfg.box_len[a];
    g.h[a] = cfg.box_len[a] / cfg.mesh[a];
  }
  g.hs = (g.h[0] == g.h[1] && g.h[1] == g.h[2]) ? g.h[0] : cbrt(g.h[0] * g.h[1] * g.h[2]);
  g.ihs = 1.0 / g.hs;
  for (int a = 0; a < 3; ++a) {
    g.cs[a] = g.h[a] / g.hs;
    g.hh[a] = 0.5 * g.h[a];
    g.loh[a] = (float)g.lo[a];
    g.lol[a] = (float)(g.lo[a] - (double)g.loh[a]);
    g.invh[a] = (float)g.inv[a];
    g.invl[a] = (float)(g.inv[a] - (double)g.invh[a]);
    g.csf[a] = (float)g.cs[a];
  }
  g.periodic = cfg.boundary == PMMM_PERIODIC ? 1 : 0;
  g.c = cfg.cutoff;
  return g;
}

enum ErrBits { ERRBIT_OUT_OF_BOX = 1, ERRBIT_NONFINITE = 2, ERRBIT_TIMEOUT = 4 };

// Device error flag helpers
__device__ __forceinline__ void set_err(int* err, int bit) { atomicOr(err, bit); }

// ---------------------------------------------------------------- sort.cu
struct SortWork {
  uint32_t *keys0, *keys1, *vals0, *vals1;
  uint32_t* hist;    // [256 * ntiles_max]
  uint32_t* chunks;  // [scan chunk sums]
  int64_t cap;
};
int sort_tiles(int64_t n);
size_t sort_hist_entries(int64_t n);
size_t sort_chunk_entries(int64_t n);
// Bins the particles (FP64 formula) and writes their records (u, q) in input order.
cudaError_t launch_bin(const void* pos, const void* q, bool fp64, int64_t n, const Geo& g, uint32_t* keys, void* rec,
                       int* err, cudaStream_t s, int* nlaunch);
// Stable LSD radix sort of the cell ids; original indices in *vals_out.
cudaError_t launch_radix_sort(SortWork& w, int64_t n, int key_bits, uint32_t** keys_out, uint32_t** vals_out,
                              cudaStream_t s, int* nlaunch);
cudaError_t launch_cell_bounds(const uint32_t* keys, int64_t n, int64_t K, int* cell_start, cudaStream_t s,
                               int* nlaunch);
// In-place exclusive scan of n uint32 values (chunks: scratch of scan_chunk_count(n)).
int64_t scan_chunk_count(int64_t n);
cudaError_t launch_exclusive_scan(uint32_t* data, int64_t n, uint32_t* chunks, cudaStream_t s, int* nlaunch);

// ---------------------------------------------------------------- p2m_l2p.cu
// sparse (FP32, p <= 8): one thread per cell, crowded cells taken by the whole warp
cudaError_t launch_p2m(int p, bool fp64, const void* part, const int* cell_start, int64_t K, void* M,
                       double* cellq, double* celld, bool sparse, cudaStream_t s, int* nlaunch);
struct CorrParams {
  double hs, alpha, V;
  double ih, ih2;      // 1 / hs, 1 / hs^2
  double c_charged;    // 3 / (2 alpha^2)
  double c_self;       // 2 alpha / sqrt(pi)
  int periodic;
  int64_t ksys;        // cells per system (corrections corr[16 s ...] of system s = cell / ksys)
  // two-level plans: the corrections are those of the coarse level (positions
  // relative to the coarse centre, Q of the coarse cell in the self term)
  int refine;          // 0 / 1: one level; r >= 2: coarse cell = r^3 fine cells
  int nf[3], nc[3];    // fine and coarse cells per axis
  double cs[3];        // fine cell sides in units of hs
  // FP32 copies for the FP32 L2P, which then converts no FP64 value per particle
  // (GB300 converts from FP64 at a small fraction of its FP32 rate)
  float hs32, ih32, ih2_32, c_charged32, c_self32;
  float cshs32[3];     // two-level: fine cell sides in units of the coarse hs
};
// Per-system correction block corr[16 s ...]: FP64 terms corr[0..4] (App. B.3),
// their FP32 copies as five floats from byte offset 8 CORR_F32 (doubles 5..7),
// the FP64 sums corr[8..12].
constexpr int CORR_F32 = 5;
__device__ __forceinline__ void corr_store_f32(double* c) {
  float* f = reinterpret_cast<float*>(c + CORR_F32);
#pragma unroll
  for (int k = 0; k < 5; ++k) f[k] = (float)c[k];
}
// Two-level plans: multipoles of the coarse cells (r^3 fine cells each) from the
// particles sorted by fine cell, and the coarse per-cell sums [5][Kc].
struct CoarseGeo {
  int r;
  int nf[3], nc[3];
  int64_t Kc;
  double cs[3];  // fine cell sides in units of the fine hs
};
cudaError_t launch_p2m_coarse(int p, bool fp64, const void* part, const int* cell_start, const CoarseGeo& cg,
                              void* Mc, double* cellsum, cudaStream_t s, int* nlaunch);
cudaError_t launch_l2p(int p, bool fp64, const void* part, const uint32_t* keys, int64_t n, const void* L,
                       int64_t K, const double* corr, const double* cellq, CorrParams cp, void* far,
                       cudaStream_t s, int* nlaunch);

// ---------------------------------------------------------------- hier.cu
// Two-level PMMM (Sec. 5, hierarchical treatment): geometry of the levels.
struct HierGeo {
  int r, c, m;        // refinement per axis, cutoff, block transform length (>= 2 (c+1) r)
  int nf[3], nc[3];   // fine and coarse cells per axis
  int wavemajor;      // block spectra [k][channel][coarse cell] (else [channel][coarse cell][k])
};
bool hier_block_fits(const HierGeo& h, bool fp64, int C);
// R(coarse centre - child centre) in units of hs_f for the r^3 children, real storage, [r^3][C]
cudaError_t launch_hier_rtab(const HierGeo& h, int p, bool fp64, const double* cs, void* rtab, cudaStream_t s);
// whether the L2L child matrices (r^3 C^2 values) are built
bool hier_use_matrices(const HierGeo& h, int p);
// the L2L child matrices (coarse -> child), [r^3][C][C]
cudaError_t launch_hier_matrices(const HierGeo& h, int p, bool fp64, const void* rtab, void* um, cudaStream_t s);
// block spectra of the fine multipoles of every coarse cell (tw: exp(-2 pi i j / m), j < m)
cudaError_t launch_hier_forward(const HierGeo& h, int C, bool fp64, const void* Mf, void* spec, const void* tw,
                                cudaStream_t s, int* nlaunch);
// kept outputs [C][Kc][W^3] of the block convolution from the local block spectra
cudaError_t launch_hier_inverse(const HierGeo& h, int C, bool fp64, const void* spec, void* region, const void* tw,
                                cudaStream_t s, int* nlaunch);
// fine locals [C][Kf] = L2L(coarse locals [C][Kc]) + the kept block outputs (L2L through um when not null)
cudaError_t launch_hier_local(const HierGeo& h, int p, bool fp64, const void* Lc, const void* region,
                              const void* rtab, const void* um, void* Lf, int periodic, cudaStream_t s,
                              int* nlaunch);

// ---------------------------------------------------------------- fft.cu
struct FftTw {
  void* x;  // twiddles exp(-2 pi i t / L) for t < L, per axis
  void* y;
  void* z;
};
// Forward: real channels [C][nz][ny][nx] -> half spectra [C][Lz][Ly][hx].
cudaError_t launch_fft_forward(bool fp64, const void* in, void* spec, const Dims& d, int C, const FftTw& tw,
                               cudaStream_t s, int* nlaunch);
// Inverse (unnormalised): half spectra -> real channels [C][nz][ny][nx] (physical part).
cudaError_t launch_fft_inverse(bool fp64, void* spec, void* out, const Dims& d, int C, const FftTw& tw,
                               cudaStream_t s, int* nlaunch);
cudaError_t launch_twiddles(bool fp64, int L, void* tw, cudaStream_t s);
// One CTA per channel, whole 3-D transform in shared memory (fft_fused.cu): FP32,
// transform lengths <= 32, the physical planes' half spectrum <= 200 KB.
bool fft_fused_applies(bool fp64, const Dims& d);
cudaError_t launch_fft_fused_forward(const void* in, void* spec, const Dims& d, int C, const FftTw& tw, cudaStream_t s,
                                     int* nlaunch);
cudaError_t launch_fft_fused_inverse(const void* spec, void* out, const Dims& d, int C, const FftTw& tw, cudaStream_t s,
                                     int* nlaunch);

// ---------------------------------------------------------------- m2l.cu
cudaError_t launch_m2l(int p, bool fp64, const void* Mt, const void* Gt, const void* Gr, void* Lt, int64_t Kh,
                       cudaStream_t s,
                       int* nlaunch);
// nsys systems sharing Gt, spectra laid out [c][system][k] (thread per (k, l, system))
cudaError_t launch_m2l_systems(int p, bool fp64, const void* Mt, const void* Gt, const void* Gr, void* Lt, int64_t Kh,
                               int nsys,
                               cudaStream_t s, int* nlaunch);

// ---------------------------------------------------------------- batch.cu
// Many systems on one plan: system s owns cells s*Ksys ... s*Ksys + Ksys - 1 of
// a mesh of nsys*Ksys cells; the particles of system s are offsets[s] ...
// offsets[s+1]-1 (device array of nsys+1 entries).
cudaError_t launch_bin_batched(const void* pos, const void* q, bool fp64, int64_t n, const int64_t* offsets, int nsys,
                               const Geo& g, int64_t Ksys, uint32_t* keys, void* rec, int* err, cudaStream_t s,
                               int* nlaunch);
// Entry table of the real-matrix M2L as 4 ints per entry (i1, s1, i2, s2), C*C entries.
std::vector<int> build_m2l_table_int4(int p);
// out[k][r] = in[r][k] for complex R x Kh (channel-major <-> wavevector-major spectra)
cudaError_t launch_transpose(bool fp64, const void* in, void* out, int64_t R, int64_t Kh, cudaStream_t s,
                             int* nlaunch);
// Whether the SIMT matrix-product M2L fits (else launch_m2l_systems on channel-major spectra).
bool m2l_batched_gemm(bool fp64, int p, int nsys);
// L~(k) = A~(k) M~(k) for all systems at once on wavevector-major spectra
// ([k][c][system]); tab on the device.
cudaError_t launch_m2l_batched(bool fp64, const void* Mt, const void* Gt, void* Lt, const int* tab, int p, int nsys,
                               int64_t Kh, cudaStream_t s, int* nlaunch);
// The same product on the tensor cores (m2l_tc.cu): FP32 wavevector-major spectra,
// split-BF16 operands, FP32 accumulation; p <= 7.  tab: build_m2l_table_tc(p) on the device.
bool m2l_tc_supported(int p);
std::vector<uint32_t> build_m2l_table_tc(int p);
// tile: systems per CTA (32 or 64)
cudaError_t launch_m2l_tc(const void* Mt, const void* Gt, void* Lt, const uint32_t* tab, int p, int nsys, int64_t Kh,
                          int num_sms, int tile, int* err, cudaStream_t s, int* nlaunch);
// Chunks per system of the two-level batched reductions (partial: 5 * nsys * chunks doubles).
int reduce_batched_chunks(int64_t Ksys, int64_t max_items_per_sys);
// corr[16 s + ...] of every system (the single-system layout of launch_corrections)
cudaError_t launch_corrections_batched(const double* cellsum, int64_t Ktot, int64_t Ksys, int nsys, double hs,
                                       double V, double* partial, double* corr, cudaStream_t s, int* nlaunch);
// energies[4 s + ...] = energy and net force of system s from the near-field partials;
// nchunk >= ceil(items of any system / 4096)
cudaError_t launch_energy_batched(const double* epart, const uint32_t* item_start, int64_t Ksys, int nsys, int nchunk,
                                  double* partial, double* energies, cudaStream_t s, int* nlaunch);

// ---------------------------------------------------------------- mlp.cu
// D[M x N] = A[M x K] . B[N x K]^T on the tensor cores (BF16 in, FP32 accumulate);
// M % 128 == 0, N % 16 == 0, K % 16 == 0, row strides multiples of 8 elements.
enum GemmEpi {
  GEMM_EPI_LINEAR = 0,  // v = acc (+ bias): D32 and/or D16
  GEMM_EPI_GELU = 1,    // v = acc + bias: D32 = v (pre-activation), D16 = gelu(v)
  GEMM_EPI_DGELU = 2    // v = acc * gelu'(Zin): D32 and/or D16
};
struct GemmArgs {
  const __nv_bfloat16* A = nullptr;
  int64_t lda = 0;
  const __nv_bfloat16* B = nullptr;
  int64_t ldb = 0;
  int M = 0, N = 0, K = 0;
  const float* bias = nullptr;
  float* D32 = nullptr;
  int64_t ldd = 0;
  __nv_bfloat16* D16 = nullptr;
  int64_t ldd16 = 0;
  const float* Zin = nullptr;
  int64_t ldz = 0;
  int epi = GEMM_EPI_LINEAR;
  int* err = nullptr;
};
cudaError_t launch_gemm_tc(const GemmArgs& a, cudaStream_t s, int* nlaunch);
cudaError_t launch_transpose_bf16(const void* in, int64_t ld_in, void* out, int64_t ld_out, int R, int C,
                                  cudaStream_t s, int* nlaunch);
cudaError_t launch_colsum(const float* in, int64_t ld, int R, int C, float* out, cudaStream_t s, int* nlaunch);
// dO = 2 (O - T) / (rows nout) on columns < nout; *loss = mean square (device, FP64); part: nparts doubles
cudaError_t launch_mse_grad(const float* O, const float* T, int64_t rows, int ld, int nout, float* dO, void* dO16,
                            double* part, int nparts, double* loss, cudaStream_t s, int* nlaunch);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, int64_t step,
                        cudaStream_t s, int* nlaunch);
cudaError_t launch_to_bf16(const float* in, void* out, int64_t n, cudaStream_t s, int* nlaunch);
// X[cell][27 * 16]: the 16 multipole channels of the 27 neighbour cells, times in_scale
cudaError_t launch_gather_features(const float* M, int64_t K, const int n[3], int periodic, const float* in_scale,
                                   void* X, int64_t ldx, cudaStream_t s, int* nlaunch);
cudaError_t launch_build_targets(const float* Lhi, const float* Llo, int64_t K, int chi, int clow,
                                 const float* out_scale, float* T, int ldt, cudaStream_t s, int* nlaunch);
cudaError_t launch_combine_locals(const float* Llo, const float* O, int ldo, int64_t K, int chi, int clow,
                                  const float* out_scale, float* L, cudaStream_t s, int* nlaunch);
cudaError_t launch_channel_sumsq(const float* X, int C, int64_t K, double* out, cudaStream_t s, int* nlaunch);
cudaError_t launch_diff_sumsq(const float* Lhi, const float* Llo, int C, int clow, int64_t K, double* out,
                              cudaStream_t s, int* nlaunch);

// ---------------------------------------------------------------- green.cu
// Builds the real-space Green components G[s][Kt] (FP64, units of hs), s < (2p+1)^2.
cudaError_t launch_green_open(double* G, const Dims& d, int p, int c, const double cs[3], cudaStream_t st);
cudaError_t launch_green_periodic(double* G, const Dims& d, int p, int c, const double cs[3], double alpha_s,
                                  int nmax, cudaStream_t st);
// spectrum (FP64, [CG][Kh]) scaled by 1/Kt -> T
// Parity-reduced kernel spectra: one real number per component and wavevector
// (real part for even order, imaginary part for odd order), scaled.
cudaError_t launch_green_parity(const void* specd, void* outr, bool fp64, int CG, int64_t Kh, double scale,
                                cudaStream_t st);
cudaError_t launch_green_finish(const void* specd, void* out, bool fp64, int64_t count, int64_t Kh, double scale,
                                cudaStream_t st);

// ---------------------------------------------------------------- pp.cu
struct PPParams {
  int n[3];
  int c;
  int periodic;
  int ksys;  // cells per system: neighbours are taken within the target's own system
  // constants, rounded once on the host: cell size / hs per axis, 1 / hs,
  // 1 / hs^2, sign (+1 Coulomb, -1 gravity); FP64 and FP32 copies
  double csf[3], ihf, ih2f, signf;
  float cs32[3], ih32, ih2_32, sign32;
};
// Near-field work items, one per (cell, chunk of up to 32 target particles): at
// most pp_items_max of them; source pairs of the FP32 near field: at most
// (n + K) / 2 + 1.
int64_t pp_items_max(int64_t K, int64_t n);
int64_t pp_pairs_max(int64_t K, int64_t n);
// Near-field work lists: item_start / pair_start (exclusive scans of the per-cell
// item and source-pair counts, K + 1 entries; pair_start may be null) and the
// reset of the work counter; chunks: scratch of pp_lists_chunk_entries(K) entries.
int64_t pp_lists_chunk_entries(int64_t K);
cudaError_t launch_pp_lists(const int* cell_start, int64_t K, uint32_t* item_start, uint32_t* pair_start,
                            uint32_t* chunks, unsigned int* counter, cudaStream_t s, int* nlaunch);
// Sorted records part[s] = rec[vals[s]] (position relative to the cell centre in
// units of hs, and the charge), the cell of every work item (item_cell), the FP32
// pair-interleaved sources (src2 not null; 32 bytes per pair, layout in pp.cu) and
// zeroed energy partials of the unused item slots (of all of them with zero_all:
// the per-target kernel accumulates into them).
cudaError_t launch_gather_lists(const void* rec, bool fp64, const uint32_t* vals, const uint32_t* keys,
                                const int* cell_start, const uint32_t* item_start, const uint32_t* pair_start,
                                int64_t n, int64_t K, void* part, void* src2, uint32_t* item_cell, double* epart,
                                int64_t max_items, bool zero_all, cudaStream_t s, int* nlaunch);
// Near field over the (2c+1)^3 cells plus the far field from `far`, written in
// the caller's order to phi / force; energy and force partials per work item
// (epart[max_items][4]).  Persistent warps fetch items from *counter.  With
// FP32, c = 1 and src2 given, the packed-FP32 kernel on the pair layout is used.
// per_target (FP32, c = 1 only): one thread per sorted target (keys = sorted cell ids), for sparse cells.
// near_out (split evaluation; only where pp_tma_applies): the near sums of every
// sorted target go to near_out[s] = (phi, grad) / (hs, hs^2) instead of being
// combined, and launch_pp_combine adds the far field afterwards.
bool pp_per_target_applies(bool fp64, int c);
bool pp_tma_applies(bool fp64, int c, bool per_target);
cudaError_t launch_pp(bool fp64, const void* part, const void* src2, const uint32_t* pair_start, const uint32_t* vals,
                      const uint32_t* keys, int64_t n, bool per_target, const int* cell_start, int64_t K,
                      const uint32_t* item_start, const uint32_t* item_cell, unsigned int* counter, int num_sms,
                      const void* far, PPParams pp, void* phi, void* force, double* epart, int* err, void* near_out,
                      cudaStream_t s, int* nlaunch);
cudaError_t launch_pp_combine(const void* part, const uint32_t* vals, const int* cell_start, int64_t K,
                              const uint32_t* item_start, const uint32_t* item_cell, int64_t max_items,
                              const void* far, const void* nearv, PPParams pp, void* phi, void* force, double* epart,
                              int num_sms, cudaStream_t s, int* nlaunch);

// ---------------------------------------------------------------- reduce.cu
// Sums per-cell FP64 quantities and builds the periodic correction terms:
// corr[0] = c0 (potential constant), corr[1..3] = c1 (linear term), corr[4] = qfac,
// corr[8..12] = raw sums (Q, sum q u_x, sum q u_y, sum q u_z, sum q |u|^2) in hs units.
// One launch each: partial holds RD_BLOCKS (256) x 5 doubles, ticket one zeroed
// counter that the launch leaves zeroed again.
cudaError_t launch_corrections(const double* cellq, const double* celld, int64_t K, double hs, double V,
                               double* partial, unsigned int* ticket, double* corr, cudaStream_t s, int* nlaunch);
// energy[0] = sum of epart[i*4 + 0] over i < count, energy[1..3] = net force
cudaError_t launch_energy(const double* epart, int64_t count, double* partial, unsigned int* ticket, double* energy,
                          cudaStream_t s, int* nlaunch);
cudaError_t launch_to_physical(bool fp64, const void* X, double* out, int p, int64_t K, double hs, int power_shift,
                               cudaStream_t s);

}  // namespace pmmm
