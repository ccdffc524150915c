// C ABI of the PMMM GPU library (include/pmmm.h): plan life cycle, the full
// force evaluation and diagnostics.  Every step of the evaluation is a kernel
// of this library queued on the plan's stream; there is no host fallback.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "plan.cuh"

using namespace pmmm;

namespace {

const char* kStageNames[ST_COUNT] = {"bin_sort", "p2m", "fft_forward", "m2l", "fft_inverse", "l2p", "near_field",
                                     "reduce"};

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return PMMM_OK;
  if (e == cudaErrorMemoryAllocation) return PMMM_ERR_OOM;
  return PMMM_ERR_CUDA;
}

}  // namespace

namespace {

cudaError_t dalloc(pmmm_plan* pl, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e == cudaSuccess) {
    pl->ws_bytes += bytes;
    pl->sizes[*ptr] = bytes;
    ++pl->wgen;
  }
  return e;
}

template <typename P>
void dfree(pmmm_plan* pl, P*& p) {
  if (p) {
    auto it = pl->sizes.find((void*)p);
    if (it != pl->sizes.end()) {
      pl->ws_bytes -= it->second;
      pl->sizes.erase(it);
    }
    cudaFree((void*)p);
    ++pl->wgen;
  }
  p = nullptr;
}

void free_particles(pmmm_plan* pl) {
  dfree(pl, pl->sw.keys0);
  dfree(pl, pl->sw.keys1);
  dfree(pl, pl->sw.vals0);
  dfree(pl, pl->sw.vals1);
  dfree(pl, pl->sw.hist);
  dfree(pl, pl->sw.chunks);
  pl->sw = SortWork{};
  dfree(pl, pl->part);
  dfree(pl, pl->far);
  dfree(pl, pl->item_cell);
  dfree(pl, pl->src2);
  dfree(pl, pl->epart);
  dfree(pl, pl->bpartial);
  dfree(pl, pl->nearv);
  pl->bchunks = 0;
  pl->max_items = 0;
  pl->cap = 0;
}

// Buffers whose size scales with the number of systems.
void free_mesh(pmmm_plan* pl) {
  dfree(pl, pl->M); dfree(pl, pl->L); dfree(pl, pl->specM); dfree(pl, pl->specL);
  dfree(pl, pl->cellsum);
  dfree(pl, pl->cs);
  dfree(pl, pl->corr);
  dfree(pl, pl->item_start);
  dfree(pl, pl->item_chunks);
  dfree(pl, pl->pair_start);
  dfree(pl, pl->energy);
  dfree(pl, pl->offsets_d);
  if (pl->offsets_pinned) cudaFreeHost(pl->offsets_pinned);
  pl->offsets_pinned = nullptr;
  pl->offsets_up.clear();
  pl->bcap = 0;
}

void free_all(pmmm_plan* pl) {
  if (!pl) return;
  free_particles(pl);
  free_mesh(pl);
  dfree(pl, pl->G);
  dfree(pl, pl->Gr);
  dfree(pl, pl->twx); dfree(pl, pl->twy); dfree(pl, pl->twz);
  dfree(pl, pl->partial);
  dfree(pl, pl->counter);
  dfree(pl, pl->err);
  dfree(pl, pl->m2l_tab);
  dfree(pl, pl->m2l_tab_tc);
  dfree(pl, pl->hspecM); dfree(pl, pl->hspecL); dfree(pl, pl->hregion); dfree(pl, pl->hrtab);
  dfree(pl, pl->hum);
  if (pl->coarse) pmmm_plan_destroy(pl->coarse);
  if (pl->block) pmmm_plan_destroy(pl->block);
  pl->coarse = pl->block = nullptr;
  dfree(pl, pl->hpos); dfree(pl, pl->hq); dfree(pl, pl->hphi); dfree(pl, pl->hforce);
  if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
  pl->gexec = nullptr;
  if (pl->cstream) cudaStreamDestroy(pl->cstream);
  pl->cstream = nullptr;
  if (pl->aux) {
    cudaStreamSynchronize(pl->aux);
    cudaStreamDestroy(pl->aux);
  }
  pl->aux = nullptr;
  if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
  if (pl->ev_join) cudaEventDestroy(pl->ev_join);
  pl->ev_fork = pl->ev_join = nullptr;
  for (int i = 0; i <= ST_COUNT; ++i)
    if (pl->ev[i]) cudaEventDestroy(pl->ev[i]);
}

// Mesh workspace for B systems (B * K cells, C * B transform channels).
cudaError_t alloc_mesh(pmmm_plan* pl, int B) {
  const Dims& d = pl->d;
  const size_t T = pl->tsize;
  const int64_t Kb = d.K * B, Khb = d.Kh * B;
  void* v;
  cudaError_t e = dalloc(pl, &pl->M, T * pl->C * (size_t)Kb);
  if (e == cudaSuccess) e = dalloc(pl, &pl->L, T * pl->C * (size_t)Kb);
  if (e == cudaSuccess) e = dalloc(pl, &pl->specM, 2 * T * pl->C * (size_t)Khb);
  if (e == cudaSuccess) e = dalloc(pl, &pl->specL, 2 * T * pl->C * (size_t)Khb);
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(double) * 5 * (size_t)Kb); pl->cellsum = (double*)v; }
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(int) * (size_t)(Kb + 1)); pl->cs = (int*)v; }
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(double) * 16 * (size_t)B); pl->corr = (double*)v; }
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(uint32_t) * (size_t)(Kb + 1)); pl->item_start = (uint32_t*)v; }
  if (e == cudaSuccess) {
    e = dalloc(pl, &v, sizeof(uint32_t) * (size_t)pp_lists_chunk_entries(Kb));
    pl->item_chunks = (uint32_t*)v;
  }
  if (e == cudaSuccess && !pl->fp64) {
    e = dalloc(pl, &v, sizeof(uint32_t) * (size_t)(Kb + 1));
    pl->pair_start = (uint32_t*)v;
  }
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(double) * 4 * (size_t)B); pl->energy = (double*)v; }
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(int64_t) * (size_t)(B + 1)); pl->offsets_d = (int64_t*)v; }
  if (e == cudaSuccess) e = cudaMallocHost((void**)&pl->offsets_pinned, sizeof(int64_t) * (size_t)(B + 1));
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->corr, 0, sizeof(double) * 16 * (size_t)B, pl->stream);
  if (e == cudaSuccess) pl->bcap = B;
  return e;
}

int ensure_particles(pmmm_plan* pl, int64_t n);
int ensure_m2l_tables(pmmm_plan* pl);
void set_streams(pmmm_plan* pl, cudaStream_t s);
// the near sums' buffer of the split evaluation is kept once a choice asks for it
bool wants_split(const pmmm_plan* pl) {
  return !pl->fp64 && (pl->cfg.near_field == PMMM_NEAR_CELL_ITEMS_SPLIT || pl->tuned_near == PMMM_NEAR_CELL_ITEMS_SPLIT ||
                       pl->nearv != nullptr);
}

// Grows the mesh workspace to B systems (the particle workspace, sized by the
// cell count, is rebuilt with it).
int ensure_systems(pmmm_plan* pl, int B) {
  if (B <= pl->bcap) return PMMM_OK;
  cudaStreamSynchronize(pl->stream);
  const int64_t n = pl->cap;
  free_particles(pl);
  free_mesh(pl);
  cudaError_t e = alloc_mesh(pl, B);
  if (e != cudaSuccess) {
    free_mesh(pl);
    return map_cuda(e);
  }
  return ensure_particles(pl, n);
}

int validate(const pmmm_config* c) {
  if (!c) return PMMM_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a) {
    if (!(c->box_len[a] > 0.0) || !isfinite(c->box_len[a]) || !isfinite(c->box_lo[a])) return PMMM_ERR_INVALID_ARG;
    if (c->mesh[a] < 1) return PMMM_ERR_INVALID_ARG;
  }
  if (c->boundary != PMMM_OPEN && c->boundary != PMMM_PERIODIC) return PMMM_ERR_INVALID_ARG;
  if (c->precision < PMMM_FP64 || c->precision > PMMM_FP32_SPLITBF16_M2L) return PMMM_ERR_INVALID_ARG;
  if (c->p < 0 || c->cutoff < 1) return PMMM_ERR_INVALID_ARG;
  if (!(c->sign == 1.0 || c->sign == -1.0)) return PMMM_ERR_INVALID_ARG;
  if (c->ewald_alpha < 0.0 || !isfinite(c->ewald_alpha) || c->ewald_nmax < 0) return PMMM_ERR_INVALID_ARG;
  if (c->near_field < PMMM_NEAR_AUTO || c->near_field > PMMM_NEAR_CELL_ITEMS_SPLIT) return PMMM_ERR_INVALID_ARG;
  if (c->p > PMMM_PMAX || c->cutoff > 2) return PMMM_ERR_UNSUPPORTED;
  for (int a = 0; a < 3; ++a) {
    if (!pow2(c->mesh[a])) return PMMM_ERR_UNSUPPORTED;
    if (c->boundary == PMMM_PERIODIC) {
      if (c->mesh[a] < 2 * c->cutoff + 1 || c->mesh[a] > 512) return PMMM_ERR_UNSUPPORTED;
    } else if (c->mesh[a] > 256) {
      return PMMM_ERR_UNSUPPORTED;
    }
  }
  const int64_t K = (int64_t)c->mesh[0] * c->mesh[1] * c->mesh[2];
  if (K > (int64_t)1 << 28) return PMMM_ERR_UNSUPPORTED;
  if (c->refine < 0) return PMMM_ERR_INVALID_ARG;
  if (c->refine > 1) {
    if (!pow2(c->refine) || c->refine > 16) return PMMM_ERR_UNSUPPORTED;
    for (int a = 0; a < 3; ++a)
      if (c->mesh[a] % c->refine != 0 || c->mesh[a] / c->refine < 2) return PMMM_ERR_UNSUPPORTED;
  }
  return PMMM_OK;
}

// Particle workspace for n particles; allocated at least once (the near-field
// work items and energy partials exist even for n = 0).
int ensure_particles(pmmm_plan* pl, int64_t n) {
  if (pl->cap > 0 && n <= pl->cap) return PMMM_OK;
  cudaStreamSynchronize(pl->stream);
  free_particles(pl);
  const int64_t cap = n < 1024 ? 1024 : n;
  cudaError_t e = cudaSuccess;
  void* v;
#define ALLOC(field, type, count)                       \
  e = dalloc(pl, &v, sizeof(type) * (size_t)(count));   \
  if (e != cudaSuccess) {                               \
    free_particles(pl);                                 \
    return map_cuda(e);                                 \
  }                                                     \
  field = (type*)v;
  ALLOC(pl->sw.keys0, uint32_t, cap);
  ALLOC(pl->sw.keys1, uint32_t, cap);
  ALLOC(pl->sw.vals0, uint32_t, cap);
  ALLOC(pl->sw.vals1, uint32_t, cap);
  ALLOC(pl->sw.hist, uint32_t, sort_hist_entries(cap));
  ALLOC(pl->sw.chunks, uint32_t, sort_chunk_entries(cap));
#undef ALLOC
  e = dalloc(pl, &pl->part, 4 * pl->tsize * (size_t)cap);
  if (e == cudaSuccess) e = dalloc(pl, &pl->far, 4 * pl->tsize * (size_t)cap);
  const int64_t Kb = pl->d.K * pl->bcap;
  const int64_t mi = pp_items_max(Kb, cap);
  if (e == cudaSuccess) e = dalloc(pl, &v, sizeof(uint32_t) * (size_t)mi);
  if (e == cudaSuccess) pl->item_cell = (uint32_t*)v;
  if (e == cudaSuccess) e = dalloc(pl, &v, sizeof(double) * 4 * (size_t)mi);
  if (e == cudaSuccess) pl->epart = (double*)v;
  if (e == cudaSuccess && !pl->fp64) e = dalloc(pl, &pl->src2, 32 * (size_t)pp_pairs_max(Kb, cap));
  if (e == cudaSuccess && wants_split(pl)) e = dalloc(pl, &pl->nearv, 16 * (size_t)cap);
  // items of one system: at most its cells + cap / 32 + 1
  const int bch = reduce_batched_chunks(pl->d.K, pp_items_max(pl->d.K, cap));
  if (e == cudaSuccess) e = dalloc(pl, &v, sizeof(double) * 5 * (size_t)pl->bcap * bch);
  if (e == cudaSuccess) {
    pl->bpartial = (double*)v;
    pl->bchunks = bch;
  }
  if (e != cudaSuccess) {
    free_particles(pl);
    return map_cuda(e);
  }
  pl->sw.cap = cap;
  pl->cap = cap;
  pl->max_items = mi;
  return PMMM_OK;
}

int build_green(pmmm_plan* pl) {
  const Dims& d = pl->d;
  // full-grid geometry for the FFT of the kernel components
  Dims gd = d;
  gd.nx = d.Lx;
  gd.ny = d.Ly;
  gd.nz = d.Lz;
  gd.K = d.Kt;
  void *Gd = nullptr, *Sd = nullptr, *t64[3] = {nullptr, nullptr, nullptr};
  cudaError_t e = cudaMalloc(&Gd, sizeof(double) * (size_t)pl->CG * d.Kt);
  if (e == cudaSuccess) e = cudaMalloc(&Sd, sizeof(double) * 2 * (size_t)pl->CG * d.Kh);
  const int Ls[3] = {d.Lx, d.Ly, d.Lz};
  for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
    e = cudaMalloc(&t64[a], sizeof(double) * 2 * Ls[a]);
    if (e == cudaSuccess) e = launch_twiddles(true, Ls[a], t64[a], pl->stream);
  }
  if (e == cudaSuccess) {
    if (pl->g.periodic)
      e = launch_green_periodic((double*)Gd, d, pl->p, pl->g.c, pl->g.cs, pl->g.alpha * pl->g.hs, pl->nmax,
                                pl->stream);
    else
      e = launch_green_open((double*)Gd, d, pl->p, pl->g.c, pl->g.cs, pl->stream);
  }
  int nl = 0;
  if (e == cudaSuccess) {
    FftTw tw{t64[0], t64[1], t64[2]};
    e = launch_fft_forward(true, Gd, Sd, gd, pl->CG, tw, pl->stream, &nl);
  }
  if (e == cudaSuccess)
    e = launch_green_finish(Sd, pl->G, pl->fp64, (int64_t)pl->CG * d.Kh, d.Kh, 1.0 / (double)d.Kt, pl->stream);
  if (e == cudaSuccess) e = dalloc(pl, &pl->Gr, pl->tsize * pl->CG * (size_t)d.Kh);
  if (e == cudaSuccess) e = launch_green_parity(Sd, pl->Gr, pl->fp64, pl->CG, d.Kh, 1.0 / (double)d.Kt, pl->stream);
  cudaError_t e2 = cudaStreamSynchronize(pl->stream);
  if (e == cudaSuccess) e = e2;
  if (Gd) cudaFree(Gd);
  if (Sd) cudaFree(Sd);
  for (int a = 0; a < 3; ++a)
    if (t64[a]) cudaFree(t64[a]);
  return map_cuda(e);
}

// Two-level plan (Sec. 5, hierarchical treatment): the coarse one-level plan,
// the open plan of (m/2)^3 fine cells whose kernel spectra are those of the
// fine-level block convolution (free-space S(d h_fine), nearest (2c+1)^3 masked,
// offsets up to m/2 - 1 >= (c+1) r - 1), the block workspace and the child table.
int setup_hier(pmmm_plan* pl) {
  const pmmm_config& cf = pl->cfg;
  HierGeo& h = pl->hg;
  h.r = cf.refine;
  h.c = cf.cutoff;
  h.m = 1;
  while (h.m < 2 * (h.c + 1) * h.r) h.m <<= 1;
  pmmm_config cc = cf;
  cc.refine = 0;
  for (int a = 0; a < 3; ++a) {
    h.nf[a] = cf.mesh[a];
    h.nc[a] = cf.mesh[a] / h.r;
    cc.mesh[a] = h.nc[a];
  }
  int rc = pmmm_plan_create(&cc, pl->stream, &pl->coarse);
  if (rc != PMMM_OK) return rc;
  pmmm_config bc;
  pmmm_config_init(&bc);
  for (int a = 0; a < 3; ++a) {
    bc.box_lo[a] = 0.0;
    bc.mesh[a] = h.m / 2;
    bc.box_len[a] = (h.m / 2) * pl->g.h[a];
  }
  bc.p = cf.p;
  bc.cutoff = cf.cutoff;
  bc.boundary = PMMM_OPEN;
  bc.precision = cf.precision;
  rc = pmmm_plan_create(&bc, pl->stream, &pl->block);
  if (rc != PMMM_OK) return rc;
  const int64_t Kc = pl->coarse->d.K, Khh = pl->block->d.Kh;
  h.wavemajor = (pl->m2l_tc || m2l_batched_gemm(pl->fp64, pl->p, (int)Kc)) ? 1 : 0;
  if (!h.wavemajor && Kc > 65535) return PMMM_ERR_UNSUPPORTED;
  if (!hier_block_fits(h, pl->fp64, pl->C)) return PMMM_ERR_UNSUPPORTED;
  const size_t T = pl->tsize, W = (size_t)(2 * h.c + 1) * h.r;
  cudaError_t e = dalloc(pl, &pl->hspecM, 2 * T * pl->C * (size_t)Kc * Khh);
  if (e == cudaSuccess) e = dalloc(pl, &pl->hspecL, 2 * T * pl->C * (size_t)Kc * Khh);
  if (e == cudaSuccess) e = dalloc(pl, &pl->hregion, T * pl->C * (size_t)Kc * W * W * W);
  if (e == cudaSuccess) e = dalloc(pl, &pl->hrtab, T * pl->C * (size_t)h.r * h.r * h.r);
  if (e == cudaSuccess) e = launch_hier_rtab(h, pl->p, pl->fp64, pl->g.cs, pl->hrtab, pl->stream);
  if (e == cudaSuccess && hier_use_matrices(h, pl->p)) {
    e = dalloc(pl, &pl->hum, T * (size_t)h.r * h.r * h.r * pl->C * pl->C);
    if (e == cudaSuccess) e = launch_hier_matrices(h, pl->p, pl->fp64, pl->hrtab, pl->hum, pl->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
  if (e != cudaSuccess) return map_cuda(e);
  if (h.wavemajor) rc = ensure_m2l_tables(pl);
  if (rc == PMMM_OK) pl->hier = true;
  return rc;
}

int read_device_status(pmmm_plan* pl) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, pl->err, sizeof(int), cudaMemcpyDeviceToHost, pl->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(pl->stream);
  if (e != cudaSuccess) return map_cuda(e);
  if (h) cudaMemsetAsync(pl->err, 0, sizeof(int), pl->stream);
  if (h & ERRBIT_TIMEOUT) return PMMM_ERR_TIMEOUT;
  if (h & ERRBIT_NONFINITE) return PMMM_ERR_NONFINITE_INPUT;
  if (h & ERRBIT_OUT_OF_BOX) return PMMM_ERR_OUT_OF_BOX;
  return PMMM_OK;
}

// The two counters of the single-launch reductions (corrections, energy): the
// last doubles of partial, which the reductions (256 x 9 doubles) leave unused.
unsigned int* reduce_tickets(pmmm_plan* pl) { return reinterpret_cast<unsigned int*>(pl->partial + 256 * 15); }

void mark(pmmm_plan* pl, int st) {
  if (pl->timing && !pl->capturing) cudaEventRecord(pl->ev[st], pl->stream);
}

// The cell convolution of Sec. 2.1 for B systems: forward FFTs of the C
// channels, per-wavevector M2L, inverse FFTs (M -> L of the plan).
cudaError_t mesh_stage(pmmm_plan* pl, int B, int* nl) {
  cudaStream_t s = pl->stream;
  const bool fp64 = pl->fp64;
  cudaError_t e = cudaSuccess;
  FftTw tw{pl->twx, pl->twy, pl->twz};
  // one CTA per channel only when the channels fill the GPU; otherwise the plane
  // kernels (a CTA per channel and z plane) and the column pass
  const bool fused = fft_fused_applies(fp64, pl->d) && (int64_t)pl->C * B >= pl->num_sms;
  e = fused ? launch_fft_fused_forward(pl->M, pl->specM, pl->d, pl->C * B, tw, s, nl)
            : launch_fft_forward(fp64, pl->M, pl->specM, pl->d, pl->C * B, tw, s, nl);
  if (e != cudaSuccess) return e;
  mark(pl, ST_M2L);
  const int64_t R = (int64_t)pl->C * B;
  const int simt = fp64 ? PMMM_M2L_ARITH_FP64_SIMT : PMMM_M2L_ARITH_FP32_SIMT;
  pl->m2l_arith = (B > 1 && pl->m2l_tc) ? PMMM_M2L_ARITH_SPLITBF16_TC : simt;
  if (B == 1) {
    e = launch_m2l(pl->p, fp64, pl->specM, pl->G, pl->Gr, pl->specL, pl->d.Kh, s, nl);
  } else if (pl->m2l_tc || m2l_batched_gemm(fp64, pl->p, B)) {
    // matrix products per wavevector on wavevector-major spectra:
    // specM -> specL (transposed) -> M2L -> specM -> specL (channel-major)
    e = launch_transpose(fp64, pl->specM, pl->specL, R, pl->d.Kh, s, nl);
    if (e == cudaSuccess)
      e = pl->m2l_tc ? launch_m2l_tc(pl->specL, pl->G, pl->specM, pl->m2l_tab_tc, pl->p, B, pl->d.Kh, pl->num_sms,
                                     pl->m2l_tile, pl->err, s, nl)
                     : launch_m2l_batched(fp64, pl->specL, pl->G, pl->specM, pl->m2l_tab, pl->p, B, pl->d.Kh, s, nl);
    if (e == cudaSuccess) e = launch_transpose(fp64, pl->specM, pl->specL, pl->d.Kh, R, s, nl);
  } else {
    e = launch_m2l_systems(pl->p, fp64, pl->specM, pl->G, pl->Gr, pl->specL, pl->d.Kh, B, s, nl);
  }
  if (e != cudaSuccess) return e;
  mark(pl, ST_FFT_INV);
  return fused ? launch_fft_fused_inverse(pl->specL, pl->L, pl->d, pl->C * B, tw, s, nl)
               : launch_fft_inverse(fp64, pl->specL, pl->L, pl->d, pl->C * B, tw, s, nl);
}

// Two-level cell convolution (Sec. 5, hierarchical treatment): coarse
// multipoles by P2M about the coarse centres (with the coarse per-cell sums of
// the periodic corrections), the one-level convolution on the coarse mesh, the block
// convolution of the fine level, and the fine locals as L2L of the coarse ones
// plus the kept block outputs (M of the plan -> L of the plan).
cudaError_t hier_stage(pmmm_plan* pl, int* nl) {
  cudaStream_t s = pl->stream;
  const HierGeo& h = pl->hg;
  pmmm_plan* cp = pl->coarse;
  pmmm_plan* bp = pl->block;
  const bool fp64 = pl->fp64;
  const int64_t Kc = cp->d.K, Khh = bp->d.Kh;
  CoarseGeo cg;
  cg.r = h.r;
  cg.Kc = Kc;
  for (int a = 0; a < 3; ++a) {
    cg.nf[a] = h.nf[a];
    cg.nc[a] = h.nc[a];
    cg.cs[a] = pl->g.cs[a];
  }
  cudaError_t e = launch_p2m_coarse(pl->p, fp64, pl->part, pl->cs, cg, cp->M, cp->cellsum, s, nl);
  if (e == cudaSuccess) e = mesh_stage(cp, 1, nl);
  if (e == cudaSuccess) e = launch_hier_forward(h, pl->C, fp64, pl->M, pl->hspecM, bp->twx, s, nl);
  if (e != cudaSuccess) return e;
  mark(pl, ST_M2L);
  pl->m2l_arith = (h.wavemajor && pl->m2l_tc) ? PMMM_M2L_ARITH_SPLITBF16_TC
                                              : (fp64 ? PMMM_M2L_ARITH_FP64_SIMT : PMMM_M2L_ARITH_FP32_SIMT);
  if (!h.wavemajor)
    e = launch_m2l_systems(pl->p, fp64, pl->hspecM, bp->G, bp->Gr, pl->hspecL, Khh, (int)Kc, s, nl);
  else if (pl->m2l_tc)
    e = launch_m2l_tc(pl->hspecM, bp->G, pl->hspecL, pl->m2l_tab_tc, pl->p, (int)Kc, Khh, pl->num_sms, pl->m2l_tile,
                      pl->err, s, nl);
  else
    e = launch_m2l_batched(fp64, pl->hspecM, bp->G, pl->hspecL, pl->m2l_tab, pl->p, (int)Kc, Khh, s, nl);
  if (e != cudaSuccess) return e;
  mark(pl, ST_FFT_INV);
  e = launch_hier_inverse(h, pl->C, fp64, pl->hspecL, pl->hregion, bp->twx, s, nl);
  if (e == cudaSuccess)
    e = launch_hier_local(h, pl->p, fp64, cp->L, pl->hregion, pl->hrtab, pl->hum, pl->L, pl->g.periodic, s, nl);
  return e;
}

// One evaluation of B systems (B = 1: the single-system path; B > 1: the
// systems' particle offsets are already on the device in offsets_d).
int run(pmmm_plan* pl, int B, int64_t n, const void* pos, const void* q, void* phi, void* force) {
  int rc = ensure_systems(pl, B);
  if (rc == PMMM_OK) rc = ensure_particles(pl, n);
  if (rc != PMMM_OK) return rc;
  cudaStream_t s = pl->stream;
  int nl = 0;
  cudaError_t e = cudaSuccess;
  const bool fp64 = pl->fp64;
  const int64_t Ks = pl->d.K, K = Ks * B;  // cells per system, cells of all systems
  // near field: one thread per target when asked, or (automatic) when the cells
  // hold fewer than PMMM_NEAR_AUTO_OCCUPANCY particles on average
  const bool sparse = n < (int64_t)PMMM_NEAR_AUTO_OCCUPANCY * K;
  const int near = pl->tuned_near ? pl->tuned_near : pl->cfg.near_field;
  const bool per_target = pp_per_target_applies(fp64, pl->g.c) &&
                          (near == PMMM_NEAR_PER_TARGET || (near == PMMM_NEAR_AUTO && sparse));
  bool split = false;
  cudaStream_t fs = s;
#define CK(x)                    \
  do {                           \
    e = (x);                     \
    if (e != cudaSuccess) goto done; \
  } while (0)
  mark(pl, ST_SORT);
  {
    int key_bits = 0;
    while (((int64_t)1 << key_bits) < K) ++key_bits;
    // the unsorted records go to `far`, which L2P overwrites later
    if (B == 1)
      CK(launch_bin(pos, q, fp64, n, pl->g, pl->sw.keys0, pl->far, pl->err, s, &nl));
    else
      CK(launch_bin_batched(pos, q, fp64, n, pl->offsets_d, B, pl->g, Ks, pl->sw.keys0, pl->far, pl->err, s, &nl));
    CK(launch_radix_sort(pl->sw, n, key_bits, &pl->keys_sorted, &pl->vals_sorted, s, &nl));
    CK(launch_cell_bounds(pl->keys_sorted, n, K, pl->cs, s, &nl));
    CK(launch_pp_lists(pl->cs, K, pl->item_start, fp64 ? nullptr : pl->pair_start, pl->item_chunks, pl->counter, s,
                       &nl));
    CK(launch_gather_lists(pl->far, fp64, pl->vals_sorted, pl->keys_sorted, pl->cs, pl->item_start, pl->pair_start, n,
                           K, pl->part, fp64 ? nullptr : pl->src2, pl->item_cell, pl->epart, pp_items_max(K, n),
                           per_target, s, &nl));
  }
  // Split evaluation: the far field (P2M .. L2P) goes to the plan's second stream
  // and runs beside the near field, which then leaves its sums in nearv; a
  // combination launch follows both.  Not with stage timing (stages queued one
  // by one) nor with a far-field hook (the surrogate's own plans).
  split = near == PMMM_NEAR_CELL_ITEMS_SPLIT && pl->aux && !pl->timing && !pl->hook && pl->src2 &&
          pp_tma_applies(fp64, pl->g.c, per_target);
  if (split && !pl->nearv) {
    // the near sums' buffer, allocated outside a capture (the plan's or the
    // caller's; inside one the evaluation keeps one stream)
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    const cudaError_t qe = pl->capturing ? cudaSuccess : cudaStreamIsCapturing(s, &cst);
    if (qe != cudaSuccess) cudaGetLastError();  // only the answer matters here
    if (pl->capturing || pl->cap <= 0 || qe != cudaSuccess || cst != cudaStreamCaptureStatusNone)
      split = false;
    else
      CK(dalloc(pl, &pl->nearv, 16 * (size_t)pl->cap));
  }
  fs = s;
  if (split) {
    CK(cudaEventRecord(pl->ev_fork, s));
    CK(cudaStreamWaitEvent(pl->aux, pl->ev_fork, 0));
    fs = pl->aux;
    set_streams(pl, fs);
  }
  mark(pl, ST_P2M);
  CK(launch_p2m(pl->p, fp64, pl->part, pl->cs, K, pl->M, pl->cellsum, pl->cellsum + K, sparse, fs, &nl));
  mark(pl, ST_FFT_FWD);
  CK(pl->hier ? hier_stage(pl, &nl) : mesh_stage(pl, B, &nl));
  mark(pl, ST_L2P);
  if (pl->g.periodic) {
    if (pl->hier) {
      // the corrections belong to the coarse level (its Ewald split, its cells;
      // the coarse per-cell sums come from the coarse P2M)
      pmmm_plan* cp = pl->coarse;
      CK(launch_corrections(cp->cellsum, cp->cellsum + cp->d.K, cp->d.K, cp->g.hs, pl->g.V, pl->partial,
                            reduce_tickets(pl), pl->corr, fs, &nl));
    } else if (B == 1) {
      CK(launch_corrections(pl->cellsum, pl->cellsum + K, K, pl->g.hs, pl->g.V, pl->partial, reduce_tickets(pl),
                            pl->corr, fs, &nl));
    } else {
      CK(launch_corrections_batched(pl->cellsum, K, Ks, B, pl->g.hs, pl->g.V, pl->bpartial, pl->corr, fs, &nl));
    }
  }
  {
    CorrParams cp;
    cp.hs = pl->g.hs;
    cp.alpha = pl->g.alpha;
    cp.V = pl->g.V;
    cp.ih = 1.0 / pl->g.hs;
    cp.ih2 = cp.ih * cp.ih;
    cp.c_charged = 1.5 / (pl->g.alpha * pl->g.alpha);
    cp.c_self = 2.0 * pl->g.alpha * 0.56418958354775628695;  // 2 alpha / sqrt(pi)
    cp.periodic = pl->g.periodic;
    cp.ksys = Ks;
    cp.refine = pl->hier ? pl->hg.r : 0;
    for (int a = 0; a < 3; ++a) {
      cp.nf[a] = pl->g.n[a];
      cp.nc[a] = pl->hier ? pl->hg.nc[a] : pl->g.n[a];
      cp.cs[a] = pl->g.cs[a];
      cp.cshs32[a] = (float)(cp.cs[a] * cp.hs);
    }
    cp.hs32 = (float)cp.hs;
    cp.ih32 = (float)cp.ih;
    cp.ih2_32 = (float)cp.ih2;
    cp.c_charged32 = (float)cp.c_charged;
    cp.c_self32 = (float)cp.c_self;
    const double* cellq = pl->hier ? pl->coarse->cellsum : pl->cellsum;
    const void* Luse = pl->L;
    int puse = pl->p;
    if (pl->hook) {
      CK(pl->hook->fn(s, &nl));
      Luse = pl->hook->L;
      puse = pl->hook->p_l2p;
    }
    CK(launch_l2p(puse, fp64, pl->part, pl->keys_sorted, n, Luse, K, pl->corr, cellq, cp, pl->far, fs, &nl));
  }
  if (split) {
    set_streams(pl, s);
    CK(cudaEventRecord(pl->ev_join, fs));
  }
  mark(pl, ST_PP);
  {
    PPParams pp;
    for (int a = 0; a < 3; ++a) {
      pp.n[a] = pl->g.n[a];
      pp.csf[a] = pl->g.cs[a];
    }
    pp.c = pl->g.c;
    pp.periodic = pl->g.periodic;
    pp.ksys = (int)Ks;
    pp.ihf = 1.0 / pl->g.hs;
    pp.ih2f = pp.ihf * pp.ihf;
    pp.signf = pl->g.sign;
    for (int a = 0; a < 3; ++a) pp.cs32[a] = (float)pp.csf[a];
    pp.ih32 = (float)pp.ihf;
    pp.ih2_32 = (float)pp.ih2f;
    pp.sign32 = (float)pp.signf;
    const int64_t mi = pp_items_max(K, n);
    CK(launch_pp(fp64, pl->part, pl->src2, pl->pair_start, pl->vals_sorted, pl->keys_sorted, n, per_target, pl->cs, K,
                 pl->item_start, pl->item_cell, pl->counter, pl->num_sms, pl->far, pp, phi, force, pl->epart, pl->err,
                 split ? pl->nearv : nullptr, s, &nl));
    if (split) {
      CK(cudaStreamWaitEvent(s, pl->ev_join, 0));
      CK(launch_pp_combine(pl->part, pl->vals_sorted, pl->cs, K, pl->item_start, pl->item_cell, mi, pl->far,
                           pl->nearv, pp, phi, force, pl->epart, pl->num_sms, s, &nl));
    }
    mark(pl, ST_REDUCE);
    if (B == 1)
      CK(launch_energy(pl->epart, mi, pl->partial + 256 * 5, reduce_tickets(pl) + 1, pl->energy, s, &nl));
    else
      CK(launch_energy_batched(pl->epart, pl->item_start, Ks, B, pl->bchunks, pl->bpartial, pl->energy, s, &nl));
  }
  mark(pl, ST_COUNT);
#undef CK
done:
  if (split) set_streams(pl, s);
  pl->split_last = split && e == cudaSuccess;
  pl->launches = nl;
  pl->n_last = n;
  pl->nsys_last = B;
  pl->timed = pl->timing && !pl->capturing && e == cudaSuccess;
  return map_cuda(e);
}

// Validates host offsets of B systems and uploads them to offsets_d (skipped
// when they equal the last upload).  Returns the particle count in *n.
int upload_offsets(pmmm_plan* pl, int B, const int64_t* off, int64_t* n) {
  if (!off || off[0] != 0) return PMMM_ERR_INVALID_ARG;
  if (pl->hier && B > 1) return PMMM_ERR_UNSUPPORTED;  // two-level plans evaluate one system
  for (int s = 0; s < B; ++s)
    if (off[s + 1] < off[s]) return PMMM_ERR_INVALID_ARG;
  if (off[B] > INT32_MAX) return PMMM_ERR_INVALID_ARG;
  *n = off[B];
  int rc = ensure_systems(pl, B);
  if (rc == PMMM_OK) rc = ensure_m2l_tables(pl);
  if (rc != PMMM_OK) return rc;
  if (pl->offsets_up.size() == (size_t)B + 1 && memcmp(pl->offsets_up.data(), off, sizeof(int64_t) * (B + 1)) == 0)
    return PMMM_OK;
  // the staging buffer may still feed an earlier copy on the stream
  cudaError_t e = cudaStreamSynchronize(pl->stream);
  if (e == cudaSuccess) {
    memcpy(pl->offsets_pinned, off, sizeof(int64_t) * (B + 1));
    e = cudaMemcpyAsync(pl->offsets_d, pl->offsets_pinned, sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice,
                        pl->stream);
  }
  if (e != cudaSuccess) {
    pl->offsets_up.clear();
    return map_cuda(e);
  }
  pl->offsets_up.assign(off, off + B + 1);
  return PMMM_OK;
}

// Entry tables of the matrix-product M2L (SIMT and, for split-BF16 plans, tensor core).
int ensure_m2l_tables(pmmm_plan* pl) {
  if (!pl->m2l_tab) {
    std::vector<int> t = build_m2l_table_int4(pl->p);
    void* v = nullptr;
    cudaError_t e = dalloc(pl, &v, sizeof(int) * t.size());
    if (e == cudaSuccess) e = cudaMemcpy(v, t.data(), sizeof(int) * t.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      dfree(pl, v);
      return map_cuda(e);
    }
    pl->m2l_tab = (int*)v;
  }
  if (pl->m2l_tc && !pl->m2l_tab_tc) {
    std::vector<uint32_t> t = build_m2l_table_tc(pl->p);
    void* v = nullptr;
    cudaError_t e = dalloc(pl, &v, sizeof(uint32_t) * t.size());
    if (e == cudaSuccess) e = cudaMemcpy(v, t.data(), sizeof(uint32_t) * t.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      dfree(pl, v);
      return map_cuda(e);
    }
    pl->m2l_tab_tc = (uint32_t*)v;
  }
  return PMMM_OK;
}

// Device-to-host copy of the per-system energies (synchronises), then the device status.
int read_energies(pmmm_plan* pl, int B, double* out) {
  std::vector<double> h(4 * (size_t)B);
  cudaError_t e = cudaMemcpyAsync(h.data(), pl->energy, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, pl->stream);
  if (e != cudaSuccess) return map_cuda(e);
  const int rc = read_device_status(pl);
  for (int s = 0; s < B; ++s) out[s] = h[4 * (size_t)s];
  return rc;
}

// Workspace generation of a plan and its sub-plans (two-level plans): changes
// whenever any buffer that a captured graph may reference is allocated or freed.
uint64_t plan_gen(const pmmm_plan* pl) {
  uint64_t g = pl->wgen;
  if (pl->coarse) g += plan_gen(pl->coarse);
  if (pl->block) g += plan_gen(pl->block);
  return g;
}

void set_streams(pmmm_plan* pl, cudaStream_t s) {
  pl->stream = s;
  if (pl->coarse) set_streams(pl->coarse, s);
  if (pl->block) set_streams(pl->block, s);
}

// One evaluation of B systems as a CUDA graph launched on the plan's stream:
// replayed when it was captured for the same offsets, caller pointers,
// workspace and tuning choices, captured again otherwise.  The capture runs on a
// private stream, so any stream of the caller works (the legacy default stream
// included).  The workspace must already hold B systems and n particles:
// nothing is allocated while capturing.
int graph_eval(pmmm_plan* pl, int B, int64_t n, const int64_t* off, const void* pos, const void* q, void* phi,
               void* force) {
  const void* ptrs[4] = {pos, q, phi, force};
  const uint64_t gen = plan_gen(pl);
  const bool same = pl->gexec && pl->gkey_off.size() == (size_t)B + 1 &&
                    memcmp(pl->gkey_off.data(), off, sizeof(int64_t) * (B + 1)) == 0 &&
                    memcmp(pl->gkey_ptr, ptrs, sizeof(ptrs)) == 0 && pl->gkey_gen == gen &&
                    pl->gkey_tune[0] == pl->tuned_near && pl->gkey_tune[1] == pl->m2l_tile;
  cudaError_t e = cudaSuccess;
  if (!same) {
    if (pl->gexec) cudaGraphExecDestroy(pl->gexec);
    pl->gexec = nullptr;
    pl->gkey_off.clear();
    if (!pl->cstream) {
      e = cudaStreamCreateWithFlags(&pl->cstream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        pl->cstream = nullptr;
        return map_cuda(e);
      }
    }
    cudaStream_t user = pl->stream;
    set_streams(pl, pl->cstream);
    e = cudaStreamBeginCapture(pl->cstream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      set_streams(pl, user);
      return map_cuda(e);
    }
    pl->capturing = true;
    const int rc = run(pl, B, n, pos, q, phi, force);
    pl->capturing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(pl->cstream, &graph);
    set_streams(pl, user);
    // node priorities as captured (the far-field stream's launches first)
    if (e == cudaSuccess && rc == PMMM_OK)
      e = cudaGraphInstantiateWithFlags(&pl->gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
    if (graph) cudaGraphDestroy(graph);
    if (rc != PMMM_OK || e != cudaSuccess) {
      if (pl->gexec && e != cudaSuccess) cudaGraphExecDestroy(pl->gexec);
      pl->gexec = nullptr;
      return rc != PMMM_OK ? rc : map_cuda(e);
    }
    pl->gkey_off.assign(off, off + B + 1);
    memcpy(pl->gkey_ptr, ptrs, sizeof(ptrs));
    pl->gkey_gen = gen;
    pl->gkey_tune[0] = pl->tuned_near;
    pl->gkey_tune[1] = pl->m2l_tile;
  }
  e = cudaGraphLaunch(pl->gexec, pl->stream);
  if (e != cudaSuccess) return map_cuda(e);
  pl->n_last = n;
  pl->nsys_last = B;
  return PMMM_OK;
}

// A single-system evaluation: the plain launch sequence on the first call with
// given pointers and sizes, a CUDA graph of it from the second identical call in
// a row on (not while stage timing is on, nor while the caller captures the
// plan's stream into a graph of its own, which then records the plain launches).
int run_single(pmmm_plan* pl, int64_t n, const void* pos, const void* q, void* phi, void* force) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (pl->timing || cudaStreamIsCapturing(pl->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return run(pl, 1, n, pos, q, phi, force);
  int rc = ensure_systems(pl, 1);
  if (rc == PMMM_OK) rc = ensure_particles(pl, n);
  if (rc != PMMM_OK) return rc;
  const int64_t off[2] = {0, n};
  const void* ptrs[4] = {pos, q, phi, force};
  const uint64_t gen = plan_gen(pl);
  const bool repeat = pl->lkey_off.size() == 2 && pl->lkey_off[1] == n &&
                      memcmp(pl->lkey_ptr, ptrs, sizeof(ptrs)) == 0 && pl->lkey_gen == gen;
  pl->lkey_off.assign(off, off + 2);
  memcpy(pl->lkey_ptr, ptrs, sizeof(ptrs));
  pl->lkey_gen = gen;
  return repeat ? graph_eval(pl, 1, n, off, pos, q, phi, force) : run(pl, 1, n, pos, q, phi, force);
}

// Plan-owned device buffers for host-array calls of n particles.
int ensure_host_staging(pmmm_plan* pl, int64_t n) {
  if (n <= pl->hcap) return PMMM_OK;
  cudaStreamSynchronize(pl->stream);
  dfree(pl, pl->hpos); dfree(pl, pl->hq); dfree(pl, pl->hphi); dfree(pl, pl->hforce);
  pl->hcap = 0;
  const size_t T = pl->tsize;
  cudaError_t e = dalloc(pl, &pl->hpos, 3 * T * (size_t)n);
  if (e == cudaSuccess) e = dalloc(pl, &pl->hq, T * (size_t)n);
  if (e == cudaSuccess) e = dalloc(pl, &pl->hphi, T * (size_t)n);
  if (e == cudaSuccess) e = dalloc(pl, &pl->hforce, 3 * T * (size_t)n);
  if (e != cudaSuccess) return map_cuda(e);
  pl->hcap = n;
  return PMMM_OK;
}

// Host arrays in, B systems evaluated, host arrays out (energies: 4 doubles per system on the device).
int run_host(pmmm_plan* pl, int B, int64_t n, const void* pos, const void* q, void* phi, void* force) {
  int rc = ensure_host_staging(pl, n);
  if (rc != PMMM_OK) return rc;
  const size_t T = pl->tsize;
  cudaStream_t s = pl->stream;
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    e = cudaMemcpyAsync(pl->hpos, pos, 3 * T * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(pl->hq, q, T * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return map_cuda(e);
  }
  rc = B == 1 ? run_single(pl, n, pl->hpos, pl->hq, phi ? pl->hphi : nullptr, force ? pl->hforce : nullptr)
              : run(pl, B, n, pl->hpos, pl->hq, phi ? pl->hphi : nullptr, force ? pl->hforce : nullptr);
  if (rc != PMMM_OK) return rc;
  if (phi && n > 0) e = cudaMemcpyAsync(phi, pl->hphi, T * (size_t)n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && force && n > 0)
    e = cudaMemcpyAsync(force, pl->hforce, 3 * T * (size_t)n, cudaMemcpyDeviceToHost, s);
  return map_cuda(e);
}

}  // namespace

namespace pmmm {
int plan_run(pmmm_plan* pl, int B, int64_t n, const void* pos, const void* q, void* phi, void* force) {
  return run(pl, B, n, pos, q, phi, force);
}
int plan_read_energies(pmmm_plan* pl, int B, double* out) { return read_energies(pl, B, out); }
int plan_map_cuda(cudaError_t e) { return map_cuda(e); }
}  // namespace pmmm

extern "C" {

int pmmm_abi_version(void) { return PMMM_ABI_VERSION; }

void pmmm_config_init(pmmm_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  for (int a = 0; a < 3; ++a) {
    c->box_lo[a] = 0.0;
    c->box_len[a] = 1.0;
    c->mesh[a] = 8;
  }
  c->p = 4;
  c->cutoff = 1;
  c->boundary = PMMM_OPEN;
  c->precision = PMMM_FP64;
  c->sign = 1.0;
  c->ewald_alpha = 0.0;
  c->ewald_nmax = 0;
}

const char* pmmm_strerror(int s) {
  switch (s) {
    case PMMM_OK: return "ok";
    case PMMM_ERR_INVALID_ARG: return "invalid argument";
    case PMMM_ERR_UNSUPPORTED: return "unsupported configuration";
    case PMMM_ERR_OUT_OF_BOX: return "particle outside the open-boundary box";
    case PMMM_ERR_NONFINITE_INPUT: return "non-finite particle coordinate";
    case PMMM_ERR_CUDA: return "CUDA error";
    case PMMM_ERR_TIMEOUT: return "device-side wait timed out";
    case PMMM_ERR_OOM: return "device out of memory";
    default: return "unknown status";
  }
}

const char* pmmm_stage_name(int i) { return (i >= 0 && i < ST_COUNT) ? kStageNames[i] : nullptr; }

int pmmm_plan_create(const pmmm_config* cfg, void* stream, pmmm_plan** out) {
  if (!out) return PMMM_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = validate(cfg);
  if (rc != PMMM_OK) return rc;
  pmmm_plan* pl = new (std::nothrow) pmmm_plan();
  if (!pl) return PMMM_ERR_OOM;
  pl->cfg = *cfg;
  pl->stream = (cudaStream_t)stream;
  pl->p = cfg->p;
  pl->C = (cfg->p + 1) * (cfg->p + 1);
  pl->CG = (2 * cfg->p + 1) * (2 * cfg->p + 1);
  pl->fp64 = cfg->precision == PMMM_FP64;
  pl->m2l_tc = cfg->precision == PMMM_FP32_SPLITBF16_M2L && m2l_tc_supported(cfg->p);
  pl->tsize = pl->fp64 ? sizeof(double) : sizeof(float);
  const bool per = cfg->boundary == PMMM_PERIODIC;
  Dims& d = pl->d;
  d.nx = cfg->mesh[0];
  d.ny = cfg->mesh[1];
  d.nz = cfg->mesh[2];
  d.Lx = per ? d.nx : 2 * d.nx;
  d.Ly = per ? d.ny : 2 * d.ny;
  d.Lz = per ? d.nz : 2 * d.nz;
  d.hx = d.Lx / 2 + 1;
  d.K = (int64_t)d.nx * d.ny * d.nz;
  d.Kt = (int64_t)d.Lx * d.Ly * d.Lz;
  d.Kh = (int64_t)d.Lz * d.Ly * d.hx;
  Geo& g = pl->g;
  g = binning_geo(*cfg);
  g.V = cfg->box_len[0] * cfg->box_len[1] * cfg->box_len[2];
  g.alpha = cfg->ewald_alpha > 0.0 ? cfg->ewald_alpha
                                   : 1.5 / fmin(cfg->box_len[0], fmin(cfg->box_len[1], cfg->box_len[2]));
  g.sign = cfg->sign;
  pl->nmax = cfg->ewald_nmax > 0 ? cfg->ewald_nmax : 5;

  const size_t T = pl->tsize;
  void* v;
  cudaError_t e = alloc_mesh(pl, 1);
  if (e == cudaSuccess) e = dalloc(pl, &pl->G, 2 * T * pl->CG * (size_t)d.Kh);
  if (e == cudaSuccess) e = dalloc(pl, &pl->twx, 2 * T * d.Lx);
  if (e == cudaSuccess) e = dalloc(pl, &pl->twy, 2 * T * d.Ly);
  if (e == cudaSuccess) e = dalloc(pl, &pl->twz, 2 * T * d.Lz);
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(double) * 256 * 16); pl->partial = (double*)v; }
  // the reduction tickets at the end of partial start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->partial, 0, sizeof(double) * 256 * 16, pl->stream);
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(int)); pl->err = (int*)v; }
  if (e == cudaSuccess) { e = dalloc(pl, &v, sizeof(unsigned int)); pl->counter = (unsigned int*)v; }
  if (e == cudaSuccess) {
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pl->num_sms, cudaDevAttrMultiProcessorCount, dev);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(pl->err, 0, sizeof(int), pl->stream);
  if (e == cudaSuccess) e = launch_twiddles(pl->fp64, d.Lx, pl->twx, pl->stream);
  if (e == cudaSuccess) e = launch_twiddles(pl->fp64, d.Ly, pl->twy, pl->stream);
  if (e == cudaSuccess) e = launch_twiddles(pl->fp64, d.Lz, pl->twz, pl->stream);
  for (int i = 0; i <= ST_COUNT && e == cudaSuccess; ++i) e = cudaEventCreate(&pl->ev[i]);
  if (e == cudaSuccess && !pl->fp64) {
    // the far field's stream takes the highest priority, so that its blocks are
    // placed ahead of queued near-field blocks
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&pl->aux, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    rc = map_cuda(e);
    free_all(pl);
    delete pl;
    return rc;
  }
  rc = build_green(pl);
  if (rc == PMMM_OK && cfg->refine > 1) rc = setup_hier(pl);
  if (rc != PMMM_OK) {
    free_all(pl);
    delete pl;
    return rc;
  }
  *out = pl;
  return PMMM_OK;
}

int pmmm_plan_destroy(pmmm_plan* pl) {
  if (!pl) return PMMM_OK;
  cudaStreamSynchronize(pl->stream);
  free_all(pl);
  delete pl;
  return PMMM_OK;
}

int pmmm_plan_reserve(pmmm_plan* pl, int64_t n) {
  if (!pl || n < 0 || n > INT32_MAX) return PMMM_ERR_INVALID_ARG;
  return ensure_particles(pl, n);
}

int pmmm_plan_reserve_batched(pmmm_plan* pl, int32_t nsys, int64_t n) {
  if (!pl || nsys < 1 || nsys > PMMM_MAX_SYSTEMS || n < 0 || n > INT32_MAX) return PMMM_ERR_INVALID_ARG;
  if (pl->d.K * nsys > ((int64_t)1 << 30)) return PMMM_ERR_UNSUPPORTED;
  if (pl->hier && nsys > 1) return PMMM_ERR_UNSUPPORTED;
  int rc = ensure_systems(pl, nsys);
  if (rc == PMMM_OK) rc = ensure_particles(pl, n);
  return rc;
}

int pmmm_compute(pmmm_plan* pl, int64_t n, const void* pos, const void* q, void* phi, void* force, double* energy) {
  if (!pl || n < 0 || n > INT32_MAX) return PMMM_ERR_INVALID_ARG;
  if (n > 0 && (!pos || !q)) return PMMM_ERR_INVALID_ARG;
  int rc = run_single(pl, n, pos, q, phi, force);
  if (rc != PMMM_OK) return rc;
  return energy ? read_energies(pl, 1, energy) : PMMM_OK;
}

int pmmm_compute_host(pmmm_plan* pl, int64_t n, const void* pos, const void* q, void* phi, void* force,
                      double* energy) {
  if (!pl || n < 0 || n > INT32_MAX) return PMMM_ERR_INVALID_ARG;
  if (n > 0 && (!pos || !q)) return PMMM_ERR_INVALID_ARG;
  int rc = run_host(pl, 1, n, pos, q, phi, force);
  if (rc != PMMM_OK) return rc;
  double e = 0.0;
  rc = read_energies(pl, 1, &e);
  if (energy) *energy = e;
  return rc;
}

int pmmm_compute_batched(pmmm_plan* pl, int32_t nsys, const int64_t* offsets, const void* pos, const void* q,
                         void* phi, void* force, double* energies) {
  if (!pl || nsys < 1 || nsys > PMMM_MAX_SYSTEMS || !offsets) return PMMM_ERR_INVALID_ARG;
  if (pl->d.K * nsys > ((int64_t)1 << 30)) return PMMM_ERR_UNSUPPORTED;
  int64_t n = 0;
  int rc = upload_offsets(pl, nsys, offsets, &n);
  if (rc != PMMM_OK) return rc;
  if (n > 0 && (!pos || !q)) return PMMM_ERR_INVALID_ARG;
  rc = run(pl, nsys, n, pos, q, phi, force);
  if (rc != PMMM_OK) return rc;
  return energies ? read_energies(pl, nsys, energies) : PMMM_OK;
}

int pmmm_compute_batched_host(pmmm_plan* pl, int32_t nsys, const int64_t* offsets, const void* pos, const void* q,
                              void* phi, void* force, double* energies) {
  if (!pl || nsys < 1 || nsys > PMMM_MAX_SYSTEMS || !offsets) return PMMM_ERR_INVALID_ARG;
  if (pl->d.K * nsys > ((int64_t)1 << 30)) return PMMM_ERR_UNSUPPORTED;
  int64_t n = 0;
  int rc = upload_offsets(pl, nsys, offsets, &n);
  if (rc != PMMM_OK) return rc;
  if (n > 0 && (!pos || !q)) return PMMM_ERR_INVALID_ARG;
  rc = run_host(pl, nsys, n, pos, q, phi, force);
  if (rc != PMMM_OK) return rc;
  std::vector<double> e((size_t)nsys);
  rc = read_energies(pl, nsys, e.data());
  if (energies) memcpy(energies, e.data(), sizeof(double) * nsys);
  return rc;
}

int pmmm_compute_batched_graph(pmmm_plan* pl, int32_t nsys, const int64_t* offsets, const void* pos, const void* q,
                               void* phi, void* force, double* energies) {
  if (!pl || nsys < 1 || nsys > PMMM_MAX_SYSTEMS || !offsets) return PMMM_ERR_INVALID_ARG;
  if (pl->d.K * nsys > ((int64_t)1 << 30)) return PMMM_ERR_UNSUPPORTED;
  int64_t n = 0;
  int rc = upload_offsets(pl, nsys, offsets, &n);  // may synchronise: before any capture
  if (rc != PMMM_OK) return rc;
  if (n > 0 && (!pos || !q)) return PMMM_ERR_INVALID_ARG;
  rc = ensure_particles(pl, n);
  if (rc != PMMM_OK) return rc;
  rc = graph_eval(pl, nsys, n, offsets, pos, q, phi, force);
  if (rc != PMMM_OK) return rc;
  return energies ? read_energies(pl, nsys, energies) : PMMM_OK;
}

int pmmm_plan_autotune(pmmm_plan* pl, int32_t nsys, const int64_t* offsets, const void* pos, const void* q,
                       int32_t reps) {
  if (!pl || nsys < 1 || nsys > PMMM_MAX_SYSTEMS || reps < 1 || reps > 100) return PMMM_ERR_INVALID_ARG;
  int64_t n = 0;
  int rc = PMMM_OK;
  if (nsys > 1) {
    if (pl->d.K * nsys > ((int64_t)1 << 30)) return PMMM_ERR_UNSUPPORTED;
    rc = upload_offsets(pl, nsys, offsets, &n);
  } else {
    if (!offsets) return PMMM_ERR_INVALID_ARG;
    n = offsets[1] - offsets[0];
    if (offsets[0] != 0 || n < 0 || n > INT32_MAX) return PMMM_ERR_INVALID_ARG;
  }
  if (rc != PMMM_OK) return rc;
  if (n > 0 && (!pos || !q)) return PMMM_ERR_INVALID_ARG;
  std::vector<int> nears = {pl->tuned_near};
  if (pp_per_target_applies(pl->fp64, pl->g.c))
    nears = {PMMM_NEAR_CELL_ITEMS, PMMM_NEAR_PER_TARGET, PMMM_NEAR_CELL_ITEMS_SPLIT};
  std::vector<int> tiles = {pl->m2l_tile};
  if (pl->m2l_tc && nsys > 1) tiles = {64, 32};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return PMMM_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return PMMM_ERR_CUDA;
  }
  const bool timing = pl->timing;
  pl->timing = false;
  float best = 1e30f;
  int best_near = pl->tuned_near, best_tile = pl->m2l_tile;
  for (int nr : nears)
    for (int tl : tiles) {
      pl->tuned_near = nr;
      pl->m2l_tile = tl;
      rc = run(pl, nsys, n, pos, q, nullptr, nullptr);  // warm-up (allocates if needed)
      cudaError_t ce = cudaSuccess;
      if (rc == PMMM_OK) ce = cudaEventRecord(e0, pl->stream);
      for (int r = 0; r < reps && rc == PMMM_OK && ce == cudaSuccess; ++r) rc = run(pl, nsys, n, pos, q, nullptr, nullptr);
      if (rc == PMMM_OK && ce == cudaSuccess) ce = cudaEventRecord(e1, pl->stream);
      if (rc == PMMM_OK && ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (rc == PMMM_OK && ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (rc == PMMM_OK && ce != cudaSuccess) rc = map_cuda(ce);
      if (rc != PMMM_OK) break;
      if (ms < best) {
        best = ms;
        best_near = nr;
        best_tile = tl;
      }
    }
  pl->tuned_near = best_near;
  pl->m2l_tile = best_tile;
  pl->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PMMM_OK) return rc;
  return read_device_status(pl);
}

int pmmm_plan_status(pmmm_plan* pl) {
  if (!pl) return PMMM_ERR_INVALID_ARG;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return map_cuda(e);
  return read_device_status(pl);
}

int pmmm_plan_export(pmmm_plan* pl, int what, void* dst, size_t bytes) {
  if (!pl || !dst) return PMMM_ERR_INVALID_ARG;
  const int64_t n = pl->n_last, K = pl->d.K * pl->nsys_last;
  const int B = pl->nsys_last;
  cudaStream_t s = pl->stream;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_cuda(e);
  switch (what) {
    case PMMM_EXPORT_PERM:
    case PMMM_EXPORT_SORTED_CELL: {
      if (bytes != sizeof(int32_t) * (size_t)n) return PMMM_ERR_INVALID_ARG;
      if (n == 0) return PMMM_OK;
      const void* src = what == PMMM_EXPORT_PERM ? (const void*)pl->vals_sorted : (const void*)pl->keys_sorted;
      e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
      break;
    }
    case PMMM_EXPORT_CELL_START:
      if (bytes != sizeof(int32_t) * (size_t)(K + 1)) return PMMM_ERR_INVALID_ARG;
      e = cudaMemcpy(dst, pl->cs, bytes, cudaMemcpyDeviceToHost);
      break;
    case PMMM_EXPORT_MULTIPOLE:
    case PMMM_EXPORT_LOCAL: {
      if (bytes != sizeof(double) * (size_t)pl->C * K) return PMMM_ERR_INVALID_ARG;
      void* tmp = nullptr;
      e = cudaMalloc(&tmp, bytes);
      if (e != cudaSuccess) return map_cuda(e);
      e = launch_to_physical(pl->fp64, what == PMMM_EXPORT_MULTIPOLE ? pl->M : pl->L, (double*)tmp, pl->p, K,
                             pl->g.hs, what == PMMM_EXPORT_MULTIPOLE ? 0 : 1, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaMemcpy(dst, tmp, bytes, cudaMemcpyDeviceToHost);
      cudaFree(tmp);
      break;
    }
    case PMMM_EXPORT_CORR: {
      if (bytes != sizeof(double) * 8 * (size_t)B) return PMMM_ERR_INVALID_ARG;
      std::vector<double> c(16 * (size_t)B);
      e = cudaMemcpy(c.data(), pl->corr, sizeof(double) * c.size(), cudaMemcpyDeviceToHost);
      const double hs = pl->hier ? pl->coarse->g.hs : pl->g.hs;  // sums of the level that is corrected
      for (int b = 0; b < B; ++b) {
        const double* cb = c.data() + 16 * (size_t)b;
        double* o = (double*)dst + 8 * (size_t)b;
        o[0] = cb[8];                    // Q
        o[1] = -cb[11] * hs;             // sum M_1^0 = -sum q z_rel
        o[2] = 0.5 * cb[9] * hs;         // Re sum M_1^1 = sum q x_rel / 2
        o[3] = 0.5 * cb[10] * hs;        // Im sum M_1^1 = sum q y_rel / 2
        o[4] = cb[12] * hs * hs;         // sum q |r_rel|^2
        o[5] = pl->g.alpha;
        o[6] = pl->g.V;
        o[7] = 0.0;
      }
      break;
    }
    case PMMM_EXPORT_FAR: {
      if (bytes != sizeof(double) * 4 * (size_t)n) return PMMM_ERR_INVALID_ARG;
      if (n == 0) return PMMM_OK;
      if (pl->fp64) {
        e = cudaMemcpy(dst, pl->far, bytes, cudaMemcpyDeviceToHost);
      } else {
        std::vector<float> t((size_t)4 * n);
        e = cudaMemcpy(t.data(), pl->far, sizeof(float) * 4 * (size_t)n, cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < t.size(); ++i) ((double*)dst)[i] = t[i];
      }
      break;
    }
    default:
      return PMMM_ERR_INVALID_ARG;
  }
  return map_cuda(e);
}

int pmmm_plan_info(pmmm_plan* pl, int what, int64_t* value) {
  if (!pl || !value) return PMMM_ERR_INVALID_ARG;
  switch (what) {
    case PMMM_INFO_K: *value = pl->d.K; break;
    case PMMM_INFO_C: *value = pl->C; break;
    case PMMM_INFO_CG: *value = pl->CG; break;
    case PMMM_INFO_KH: *value = pl->d.Kh; break;
    case PMMM_INFO_N: *value = pl->n_last; break;
    case PMMM_INFO_WORKSPACE_BYTES:
      *value = (int64_t)pl->ws_bytes + (pl->coarse ? (int64_t)pl->coarse->ws_bytes : 0) +
               (pl->block ? (int64_t)pl->block->ws_bytes : 0);
      break;
    case PMMM_INFO_LAUNCHES: *value = pl->launches; break;
    case PMMM_INFO_SYSTEMS: *value = pl->nsys_last; break;
    case PMMM_INFO_TUNED_NEAR: *value = pl->tuned_near; break;
    case PMMM_INFO_M2L_TILE: *value = pl->m2l_tile; break;
    case PMMM_INFO_REFINE: *value = pl->hier ? pl->hg.r : 1; break;
    case PMMM_INFO_M2L_ARITH: *value = pl->m2l_arith; break;
    case PMMM_INFO_SPLIT: *value = pl->split_last ? 1 : 0; break;
    default: return PMMM_ERR_INVALID_ARG;
  }
  return PMMM_OK;
}

int pmmm_plan_set_timing(pmmm_plan* pl, int enable) {
  if (!pl) return PMMM_ERR_INVALID_ARG;
  pl->timing = enable != 0;
  pl->timed = false;
  return PMMM_OK;
}

int pmmm_plan_stage_times(pmmm_plan* pl, float* ms, int max_stages) {
  if (!pl || (!ms && max_stages > 0)) return PMMM_ERR_INVALID_ARG;
  if (!pl->timed) return 0;
  cudaError_t e = cudaEventSynchronize(pl->ev[ST_COUNT]);
  if (e != cudaSuccess) return map_cuda(e);
  int k = 0;
  for (int i = 0; i < ST_COUNT && k < max_stages; ++i, ++k) {
    float t = 0.f;
    cudaEventElapsedTime(&t, pl->ev[i], pl->ev[i + 1]);
    ms[k] = t;
  }
  return k;
}

}  // extern "C"
