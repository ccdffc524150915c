// Near field (Sec. 2.1, Sec. 2.2): the pure Newtonian 1/r interaction with every
// particle of the (2c+1)^3 masked cells, plus the combination with the far field
// and the scatter back to the caller's order:
//   phi_i   = sign * (phi_far + sum_j q_j / r_ij)
//   force_i = -q_i * sign * (grad_far + sum_j grad(q_j / r_ij))
//
// Work is split into items of (cell, chunk of up to 32 targets), numbered by an
// exclusive scan over the cells so that crowded cells spread over many warps.
// One warp per item: its R targets sit in registers, lane l owns target
// l mod TL and source phase l / TL (TL = R rounded up to a power of two, so a
// chunk of 8 targets still keeps 32 lanes busy on 4 source phases).  Sources
// are read with broadcast loads (all lanes of a phase read the same record):
// through L1 in the FP64 kernel, from shared memory staged by bulk asynchronous
// copies in the FP32 one.  Self pairs (r = 0) add zero.
#include "internal.cuh"
#include "tcgen05.cuh"

namespace pmmm {

namespace {

constexpr int PP_WARPS = 4;
constexpr int PP_BATCH = 1;  // work items taken per atomic by the FP32 near-field warps (one: the shortest tail)
constexpr int PP_BLOCKS_PER_SM = 6;  // resident blocks per SM (up to 80 registers per thread)
constexpr int CHUNK = 32;

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

// FP32 reciprocal square root: the hardware approximation (PTX rsqrt.approx,
// relative error below 2^-22.9) with subnormal inputs flushed to zero.  A pair
// distance is never subnormal (the self pair gives exactly zero and is masked),
// so the flush changes no result and spares the subnormal handling of rsqrtf.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrt_ftz(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }

// item counts per cell: ceil(count / CHUNK)
__global__ void item_count_kernel(const int* __restrict__ cs, int64_t K, uint32_t* __restrict__ item_start,
                                  uint32_t* __restrict__ pair_start, unsigned int* __restrict__ counter) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) *counter = 0u;
  if (c > K) return;
  const int cnt = (c < K) ? cs[c + 1] - cs[c] : 0;
  item_start[c] = (uint32_t)((cnt + CHUNK - 1) / CHUNK);
  if (pair_start) pair_start[c] = (uint32_t)((cnt + 1) / 2);
}

// Pair-interleaved source records for the FP32 near field: the particles of
// cell c occupy pairs pair_start[c] ... (a cell with an odd count ends with a
// dummy of zero charge far outside the box).  Pair j is two 16-byte words
// {x_a, x_b, y_a, y_b}, {z_a, z_b, q_a, q_b}, so that one 128-bit load yields
// the packed operands of two sources.

// Work lists: item and source-pair counts per cell from the cell offsets and
// their exclusive prefix sums, in two launches of LIST_BLK cells per block
// (lane = cell, loads and stores coalesced): list_local_kernel scans each block's
// cells (warp scans, then a scan of the 32 warp totals) and writes the block
// totals; list_fix_kernel adds to every cell the totals of the blocks before its
// own (a warp sums at most LIST_MAX_BLOCKS of them).
constexpr int LIST_BLK = 1024;
constexpr int64_t LIST_MAX_BLOCKS = 1024;

__device__ __forceinline__ void cell_counts(const int* __restrict__ cs, int64_t c, int64_t K, uint32_t& ni,
                                            uint32_t& np) {
  ni = np = 0u;
  if (c < K) {
    const int cnt = __ldg(cs + c + 1) - __ldg(cs + c);
    ni = (uint32_t)((cnt + CHUNK - 1) / CHUNK);
    np = (uint32_t)((cnt + 1) / 2);
  }
}

__global__ void __launch_bounds__(LIST_BLK) list_local_kernel(const int* __restrict__ cs, int64_t K,
                                                              uint32_t* __restrict__ item_start,
                                                              uint32_t* __restrict__ pair_start,
                                                              uint32_t* __restrict__ tot,
                                                              unsigned int* __restrict__ counter) {
  __shared__ uint32_t wi[32], wp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c = (int64_t)blockIdx.x * LIST_BLK + tid;
  uint32_t a, q;
  cell_counts(cs, c, K, a, q);
  uint32_t ii = a, ip = q;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, ii, o), y = __shfl_up_sync(0xffffffffu, ip, o);
    if (lane >= o) {
      ii += x;
      ip += y;
    }
  }
  if (lane == 31) {
    wi[warp] = ii;
    wp[warp] = ip;
  }
  __syncthreads();
  // exclusive offsets of the warps (every warp scans the 32 totals)
  uint32_t ti = wi[lane], tp = wp[lane];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, ti, o), y = __shfl_up_sync(0xffffffffu, tp, o);
    if (lane >= o) {
      ti += x;
      tp += y;
    }
  }
  const uint32_t oi = __shfl_sync(0xffffffffu, ti - wi[lane], warp);
  const uint32_t op = __shfl_sync(0xffffffffu, tp - wp[lane], warp);
  if (c <= K) {
    item_start[c] = oi + ii - a;
    if (pair_start) pair_start[c] = op + ip - q;
  }
  if (tid == LIST_BLK - 1) {
    tot[2 * blockIdx.x] = __shfl_sync(0xffffffffu, ti, 31);
    tot[2 * blockIdx.x + 1] = __shfl_sync(0xffffffffu, tp, 31);
  }
  if (c == 0) *counter = 0u;
}

__global__ void __launch_bounds__(LIST_BLK) list_fix_kernel(int64_t K, uint32_t* __restrict__ item_start,
                                                            uint32_t* __restrict__ pair_start,
                                                            const uint32_t* __restrict__ tot) {
  __shared__ uint32_t pre[2];
  const int b = blockIdx.x;
  if (b == 0) return;  // the first block's sums are complete
  if (threadIdx.x < 32) {
    uint32_t si = 0u, sp = 0u;
    for (int j = threadIdx.x; j < b; j += 32) {
      si += tot[2 * j];
      sp += tot[2 * j + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      si += __shfl_xor_sync(0xffffffffu, si, o);
      sp += __shfl_xor_sync(0xffffffffu, sp, o);
    }
    if (threadIdx.x == 0) {
      pre[0] = si;
      pre[1] = sp;
    }
  }
  __syncthreads();
  const int64_t c = (int64_t)b * LIST_BLK + threadIdx.x;
  if (c <= K) {
    item_start[c] += pre[0];
    if (pair_start) pair_start[c] += pre[1];
  }
}

// Sorted records part[s] = rec[vals[s]] (a pure permutation), and with them the
// near-field work lists: the cell of every work item (the first particle of each
// chunk of CHUNK writes it), the pair-interleaved FP32 sources (PACK, layout
// above) and zeroed energy partials of the unused item slots (of all
// slots when the near-field kernel accumulates into them).
template <typename V, bool PACK>
__global__ void gather_lists_kernel(const V* __restrict__ rec, const uint32_t* __restrict__ vals,
                                    const uint32_t* __restrict__ keys, const int* __restrict__ cs,
                                    const uint32_t* __restrict__ item_start, const uint32_t* __restrict__ pair_start,
                                    int64_t n, int64_t K, V* __restrict__ part, float* __restrict__ src2,
                                    uint32_t* __restrict__ item_cell, double* __restrict__ epart, int64_t max_items,
                                    int zero_all) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = (zero_all ? 0 : (int64_t)item_start[K]) + s; i < max_items; i += (int64_t)gridDim.x * blockDim.x)
    epart[4 * i] = epart[4 * i + 1] = epart[4 * i + 2] = epart[4 * i + 3] = 0.0;
  if (s - (int64_t)(threadIdx.x & 31) >= n) return;  // the whole warp lies past the particles
  const bool live = s < n;  // lanes past the particles stay for the shuffles below
  V r;
  r.x = r.y = r.z = r.w = 0;
  uint32_t cell = 0;
  int j = 0;
  if (live) {
    r = rec[vals[s]];
    part[s] = r;
    cell = keys[s];
    j = (int)(s - cs[cell]);
    if (j % CHUNK == 0) item_cell[item_start[cell] + j / CHUNK] = cell;
  }
  if constexpr (PACK) {
    // pair record of (a, b) = sorted particles (s, s + 1), j even: a writes
    // {x_a, x_b, y_a, y_b}, b writes {z_a, z_b, q_a, q_b}, each one 16-byte store; the
    // partner's values come from the neighbouring lane (a global load at the warp's edge)
    const int slot = j & 1;
    const int lane = threadIdx.x & 31;
    const int src_lane = (slot == 0 ? lane + 1 : lane - 1) & 31;
    float px = __shfl_sync(0xffffffffu, (float)r.x, src_lane), py = __shfl_sync(0xffffffffu, (float)r.y, src_lane);
    float pz = __shfl_sync(0xffffffffu, (float)r.z, src_lane), pw = __shfl_sync(0xffffffffu, (float)r.w, src_lane);
    if (!live) return;
    const int64_t pj = (int64_t)pair_start[cell] + j / 2;
    const bool alone = slot == 0 && s + 1 == (int64_t)cs[cell + 1];  // odd count: dummy partner
    const bool edge = slot == 0 ? lane == 31 : lane == 0;  // partner in the neighbouring warp
    if (alone) {
      px = py = pz = 1.0e4f;
      pw = 0.0f;
    } else if (edge) {
      const V pr = rec[vals[slot == 0 ? s + 1 : s - 1]];
      px = (float)pr.x;
      py = (float)pr.y;
      pz = (float)pr.z;
      pw = (float)pr.w;
    }
    float4* o = reinterpret_cast<float4*>(src2 + 8 * pj);
    if (slot == 0)
      o[0] = make_float4((float)r.x, px, (float)r.y, py);
    else
      o[1] = make_float4(pz, (float)r.z, pw, (float)r.w);
    if (alone) o[1] = make_float4((float)r.z, pz, (float)r.w, pw);
  }
}

// Accumulates the interactions of target (tx, ty, tz) with sources P[b + e],
// e = ph, ph + SP, ... < cnt.  SELF: the source set may contain the target
// itself (r = 0 contributes zero); other neighbour cells never contain a source
// at r = 0 (a point on a shared face belongs to one cell only), so their pairs
// skip the test.
template <typename T, typename V, bool SELF>
__device__ __forceinline__ void pp_pair(const V& r, T tx, T ty, T tz, T& pot, T& gx, T& gy, T& gz) {
  const T dx = tx - r.x, dy = ty - r.y, dz = tz - r.z;
  const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
  T ri = rsq<T>(r2);
  if (SELF) ri = r2 > T(0) ? ri : T(0);
  const T qr = r.w * ri;
  pot += qr;
  const T qr3 = qr * (ri * ri);
  gx = fma(-qr3, dx, gx);
  gy = fma(-qr3, dy, gy);
  gz = fma(-qr3, dz, gz);
}

// Accumulates the interactions of target (tx, ty, tz) with sources src[e],
// e = ph, ph + SP, ... < cnt.  SELF: the source set may contain the target
// itself (r = 0 contributes zero); other neighbour cells never contain a source
// at r = 0 (a point on a shared face belongs to one cell only), so their pairs
// skip the test.
template <typename T, typename V, bool SELF>
__device__ __forceinline__ void pp_sum(const V* __restrict__ src, int cnt, int ph, int SP, T tx, T ty, T tz, T& pot,
                                       T& gx, T& gy, T& gz) {
  if (SP == 1) {
    int e = 0;
    for (; e + 4 <= cnt; e += 4) {
      const V r0 = src[e], r1 = src[e + 1], r2 = src[e + 2], r3 = src[e + 3];
      pp_pair<T, V, SELF>(r0, tx, ty, tz, pot, gx, gy, gz);
      pp_pair<T, V, SELF>(r1, tx, ty, tz, pot, gx, gy, gz);
      pp_pair<T, V, SELF>(r2, tx, ty, tz, pot, gx, gy, gz);
      pp_pair<T, V, SELF>(r3, tx, ty, tz, pot, gx, gy, gz);
    }
    for (; e < cnt; ++e) pp_pair<T, V, SELF>(src[e], tx, ty, tz, pot, gx, gy, gz);
  } else {
    for (int e = ph; e < cnt; e += SP) pp_pair<T, V, SELF>(src[e], tx, ty, tz, pot, gx, gy, gz);
  }
}

template <typename T> struct PPConst;
template <> struct PPConst<float> {
  __device__ static void get(const PPParams& p, float* cs, float& ih, float& ih2, float& sg) {
    for (int a = 0; a < 3; ++a) cs[a] = p.cs32[a];
    ih = p.ih32; ih2 = p.ih2_32; sg = p.sign32;
  }
};
template <> struct PPConst<double> {
  __device__ static void get(const PPParams& p, double* cs, double& ih, double& ih2, double& sg) {
    for (int a = 0; a < 3; ++a) cs[a] = p.csf[a];
    ih = p.ihf; ih2 = p.ih2f; sg = p.signf;
  }
};

__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// Persistent warps: each takes work items from a global counter (reset to zero
// by the work-list kernels) until all are done.  Every item's results depend
// only on the item, so the assignment order does not change any output bit.
// NB_SLOTS: neighbour-table slots per lane, (2c+1)^3 <= 32 * NB_SLOTS (1 for c = 1, 4 for c = 2)
template <typename T, int NB_SLOTS>
__global__ void __launch_bounds__(PP_WARPS * 32, PP_BLOCKS_PER_SM) pp_kernel(const T* __restrict__ part, const uint32_t* __restrict__ vals,
                                                              const int* __restrict__ cs, int64_t K,
                                                              const uint32_t* __restrict__ item_start,
                                                              const uint32_t* __restrict__ item_cell,
                                                              unsigned int* __restrict__ counter, const T* __restrict__ far,
                                                              PPParams pp, T* __restrict__ phi, T* __restrict__ force,
                                                              double* __restrict__ epart) {
  using V = typename V4<T>::type;
  const V* P = reinterpret_cast<const V*>(part);
  const int lane = threadIdx.x & 31;
  const uint32_t nitems = item_start[K];
  const int nx = pp.n[0], ny = pp.n[1], nz = pp.n[2];
  const int c = pp.c, w = 2 * c + 1, NN = w * w * w;
  T csv[3], ih, ih2, sg;
  PPConst<T>::get(pp, csv, ih, ih2, sg);
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= nitems) break;  // warp-uniform
    const int cell = (int)item_cell[item];
    const int chunk = (int)(item - item_start[cell]);
    const int tbeg = cs[cell] + chunk * CHUNK;
    const int R = min(CHUNK, cs[cell + 1] - tbeg);
    int TL = 1;
    while (TL < R) TL <<= 1;
    const int SP = 32 / TL;
    const int tl = lane & (TL - 1), ph = lane / TL;
    const bool active = tl < R;
    V xi;
    xi.x = T(0); xi.y = T(0); xi.z = T(0); xi.w = T(0);
    if (active) xi = P[tbeg + tl];
    const int sbase = cell - cell % pp.ksys, lc = cell - sbase;  // system's first cell, local cell
    const int ix = lc % nx, iy = (lc / nx) % ny, iz = lc / (nx * ny);
    // neighbour table: entry k (x fastest) in lane k % 32, slot k / 32
    int nbb[NB_SLOTS], nbc[NB_SLOTS];
#pragma unroll
    for (int j = 0; j < NB_SLOTS; ++j) {
      const int k = lane + 32 * j;
      nbb[j] = 0;
      nbc[j] = 0;
      if (k < NN) {
        int jx = ix + k % w - c, jy = iy + (k / w) % w - c, jz = iz + k / (w * w) - c;
        bool ok = true;
        if (jx < 0 || jx >= nx) { ok = ok && pp.periodic; jx += (jx < 0) ? nx : -nx; }
        if (jy < 0 || jy >= ny) { ok = ok && pp.periodic; jy += (jy < 0) ? ny : -ny; }
        if (jz < 0 || jz >= nz) { ok = ok && pp.periodic; jz += (jz < 0) ? nz : -nz; }
        if (ok) {
          const int cj = sbase + jx + nx * (jy + ny * jz);
          nbb[j] = __ldg(cs + cj);
          nbc[j] = __ldg(cs + cj + 1) - nbb[j];
        }
      }
    }
    auto nb = [&](int k, int& b, int& n) {
      int bb = nbb[0], cc = nbc[0];
#pragma unroll
      for (int q = 1; q < NB_SLOTS; ++q)
        if ((k >> 5) == q) {
          bb = nbb[q];
          cc = nbc[q];
        }
      b = __shfl_sync(0xffffffffu, bb, k & 31);
      n = __shfl_sync(0xffffffffu, cc, k & 31);
    };
    int b, cnt;
    nb(0, b, cnt);
    if (lane < cnt) prefetch_l1(P + b + lane);
    T pot = T(0), gx = T(0), gy = T(0), gz = T(0);
    int k = 0;
    for (int ez = -c; ez <= c; ++ez) {
      const T tz = xi.z - (T)ez * csv[2];
      for (int ey = -c; ey <= c; ++ey) {
        const T ty = xi.y - (T)ey * csv[1];
        for (int ex = -c; ex <= c; ++ex, ++k) {
          int bn = 0, cn = 0;
          if (k + 1 < NN) {
            nb(k + 1, bn, cn);
            if (lane < cn) prefetch_l1(P + bn + lane);  // next neighbour cell into L1
          }
          const T tx = xi.x - (T)ex * csv[0];
          if (ex == 0 && ey == 0 && ez == 0)
            pp_sum<T, V, true>(P + b, cnt, ph, SP, tx, ty, tz, pot, gx, gy, gz);
          else
            pp_sum<T, V, false>(P + b, cnt, ph, SP, tx, ty, tz, pot, gx, gy, gz);
          b = bn;
          cnt = cn;
        }
      }
    }
    for (int o = TL; o < 32; o <<= 1) {
      pot += __shfl_xor_sync(0xffffffffu, pot, o);
      gx += __shfl_xor_sync(0xffffffffu, gx, o);
      gy += __shfl_xor_sync(0xffffffffu, gy, o);
      gz += __shfl_xor_sync(0xffffffffu, gz, o);
    }
    T e_t = T(0), f_t[3] = {T(0), T(0), T(0)};
    if (active && ph == 0) {
      const int s = tbeg + tl;
      const V fr = reinterpret_cast<const V*>(far)[s];
      const T pt = sg * (fr.x + pot * ih);
      const T g0 = sg * (fr.y + gx * ih2), g1 = sg * (fr.z + gy * ih2), g2 = sg * (fr.w + gz * ih2);
      const uint32_t o = vals[s];
      const T q = xi.w;
      if (phi) phi[o] = pt;
      if (force) {
        force[3 * (int64_t)o + 0] = -q * g0;
        force[3 * (int64_t)o + 1] = -q * g1;
        force[3 * (int64_t)o + 2] = -q * g2;
      }
      e_t = T(0.5) * q * pt;
      f_t[0] = -q * g0;
      f_t[1] = -q * g1;
      f_t[2] = -q * g2;
    }
    // deterministic warp reduction of this item's energy and net-force partials
    // (the <= 32 terms of one item in T; items are summed in FP64 afterwards)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e_t += __shfl_xor_sync(0xffffffffu, e_t, o);
      f_t[0] += __shfl_xor_sync(0xffffffffu, f_t[0], o);
      f_t[1] += __shfl_xor_sync(0xffffffffu, f_t[1], o);
      f_t[2] += __shfl_xor_sync(0xffffffffu, f_t[2], o);
    }
    if (lane == 0) {
      epart[(int64_t)item * 4 + 0] = (double)e_t;
      epart[(int64_t)item * 4 + 1] = (double)f_t[0];
      epart[(int64_t)item * 4 + 2] = (double)f_t[1];
      epart[(int64_t)item * 4 + 3] = (double)f_t[2];
    }
  }
}

typedef unsigned long long f2;  // two packed floats (low word = first)
__device__ __forceinline__ f2 pk2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(f2 r, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// A two-source step with the subtractions and r^2 packed (f32x2) and the
// arithmetic after the rsqrt in scalar FP32 (faster in the per-target kernel,
// whose lanes follow different neighbour lists).
template <bool SELF>
__device__ __forceinline__ void pp_pair2_mixed(const ulonglong2& A, const ulonglong2& B, f2 tx, f2 ty, f2 tz, f2& pot,
                                               f2& gx, f2& gy, f2& gz) {
  const f2 dx = sub2(tx, A.x), dy = sub2(ty, A.y), dz = sub2(tz, B.x);
  const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
  float a, b;
  up2(r2, a, b);
  float ra = rsqrt_ftz(a), rb = rsqrt_ftz(b);
  if (SELF) {
    ra = a > 0.f ? ra : 0.f;
    rb = b > 0.f ? rb : 0.f;
  }
  float qa, qb, dxa, dxb, dya, dyb, dza, dzb;
  up2(B.y, qa, qb);
  up2(dx, dxa, dxb);
  up2(dy, dya, dyb);
  up2(dz, dza, dzb);
  const float qra = qa * ra, qrb = qb * rb;
  float p0, p1, x0, x1, y0, y1, z0, z1;
  up2(pot, p0, p1);
  up2(gx, x0, x1);
  up2(gy, y0, y1);
  up2(gz, z0, z1);
  p0 += qra;
  p1 += qrb;
  const float ca = qra * (ra * ra), cb = qrb * (rb * rb);
  x0 = fmaf(ca, dxa, x0);
  y0 = fmaf(ca, dya, y0);
  z0 = fmaf(ca, dza, z0);
  x1 = fmaf(cb, dxb, x1);
  y1 = fmaf(cb, dyb, y1);
  z1 = fmaf(cb, dzb, z1);
  pot = pk2(p0, p1);
  gx = pk2(x0, x1);
  gy = pk2(y0, y1);
  gz = pk2(z0, z1);
}

// FP32 near field (c = 1 or 2) with the neighbour cells staged by the Tensor Memory
// Accelerator's bulk copies (cp.async.bulk, global -> shared, completion counted in
// bytes on an mbarrier).  Same work items, lane mapping, results and energy
// partials as the other cell-item kernels.  Per item the warp lists its (2c+1)^3 neighbour
// cells -- the target's own cell first, then the others in (z, y, x) order --
// numbers their source pairs consecutively and streams them through two
// shared-memory buffers of NT_CAP pairs: a buffer is filled by one bulk copy per
// cell piece (issued by the lane that owns the cell) and completes on its
// mbarrier; the warp waits for it (bounded), moves the staged sources of the
// neighbour cells into the target cell's frame (one packed add per coordinate),
// sweeps the whole chunk with the target fixed (the own cell's pairs, which hold
// the self pair, separately), and refills the buffer with the chunk after next
// while the other buffer's copies are in flight.  A wait that runs out
// raises the device error flag (PMMM_ERR_TIMEOUT), waits once more (bounded) for
// the copies it issued and leaves the kernel.
constexpr int NT_CAP = 128;                    // source pairs per buffer (4 KB), a multiple of 4
constexpr int NT_BLOCKS_PER_SM = 5;            // resident blocks per SM (up to 102 registers per thread)
constexpr long long NT_WAIT_POLLS = 1 << 20;  // polls of at most 1 us each

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One step of two sources (pair record A = {x_a, x_b, y_a, y_b}, B = {z_a, z_b,
// q_a, q_b}) for one target, on float2 values with the packed FP32 operations
// (each half an IEEE fp32 operation: t - s is formed as fma(s, -1, t), exactly
// the rounded difference).  The same 13 packed operations and 2 rsqrt for every
// two sources as the per-target kernel's step.
template <bool SELF>
__device__ __forceinline__ void pp_pair_v(const float4& A, const float4& B, float2 tx, float2 ty, float2 tz,
                                          float2& pot, float2& gx, float2& gy, float2& gz) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 dx = __ffma2_rn(make_float2(A.x, A.y), m1, tx);
  const float2 dy = __ffma2_rn(make_float2(A.z, A.w), m1, ty);
  const float2 dz = __ffma2_rn(make_float2(B.x, B.y), m1, tz);
  const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
  float ra = rsqrt_ftz(r2.x), rb = rsqrt_ftz(r2.y);
  if (SELF) {
    ra = r2.x > 0.f ? ra : 0.f;
    rb = r2.y > 0.f ? rb : 0.f;
  }
  const float2 ri = make_float2(ra, rb);
  const float2 qr = __fmul2_rn(make_float2(B.z, B.w), ri);
  pot = __fadd2_rn(pot, qr);
  const float2 qr3 = __fmul2_rn(qr, __fmul2_rn(ri, ri));
  gx = __ffma2_rn(qr3, dx, gx);
  gy = __ffma2_rn(qr3, dy, gy);
  gz = __ffma2_rn(qr3, dz, gz);
}

// Sweep of npair (a multiple of 4) staged source pairs: all of them for SP = 1, the
// pairs ph, ph + SP, ... of this lane's source phase otherwise.
template <bool SELF>
__device__ __forceinline__ void pp_sweep(const float4* __restrict__ src, int npair, int ph, int SP, float2 tx,
                                         float2 ty, float2 tz, float2& pot, float2& gx, float2& gy, float2& gz) {
  if (SP == 1) {
    int j = 0;
    for (; j + 8 <= npair; j += 8) {
      float4 A[8], B[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        A[u] = src[2 * (j + u)];
        B[u] = src[2 * (j + u) + 1];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) pp_pair_v<SELF>(A[u], B[u], tx, ty, tz, pot, gx, gy, gz);
    }
    for (; j < npair; j += 4) {
      const float4 A0 = src[2 * j], B0 = src[2 * j + 1], A1 = src[2 * j + 2], B1 = src[2 * j + 3];
      const float4 A2 = src[2 * j + 4], B2 = src[2 * j + 5], A3 = src[2 * j + 6], B3 = src[2 * j + 7];
      pp_pair_v<SELF>(A0, B0, tx, ty, tz, pot, gx, gy, gz);
      pp_pair_v<SELF>(A1, B1, tx, ty, tz, pot, gx, gy, gz);
      pp_pair_v<SELF>(A2, B2, tx, ty, tz, pot, gx, gy, gz);
      pp_pair_v<SELF>(A3, B3, tx, ty, tz, pot, gx, gy, gz);
    }
  } else {
    int j = ph;
    for (; j + 3 * SP < npair; j += 4 * SP) {
      float4 A[4], B[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        A[u] = src[2 * (j + u * SP)];
        B[u] = src[2 * (j + u * SP) + 1];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) pp_pair_v<SELF>(A[u], B[u], tx, ty, tz, pot, gx, gy, gz);
    }
    for (; j + SP < npair; j += 2 * SP) {
      const float4 A0 = src[2 * j], B0 = src[2 * j + 1], A1 = src[2 * (j + SP)], B1 = src[2 * (j + SP) + 1];
      pp_pair_v<SELF>(A0, B0, tx, ty, tz, pot, gx, gy, gz);
      pp_pair_v<SELF>(A1, B1, tx, ty, tz, pot, gx, gy, gz);
    }
    if (j < npair) pp_pair_v<SELF>(src[2 * j], src[2 * j + 1], tx, ty, tz, pot, gx, gy, gz);
  }
}

template <int CUT>
__global__ void __launch_bounds__(PP_WARPS * 32, NT_BLOCKS_PER_SM) pp_kernel_tma(
    const float* __restrict__ part, const float* __restrict__ src2f, const uint32_t* __restrict__ pair_start,
    const uint32_t* __restrict__ vals, const int* __restrict__ cs, int64_t K, const uint32_t* __restrict__ item_start,
    const uint32_t* __restrict__ item_cell, unsigned int* __restrict__ counter, const float* __restrict__ far,
    PPParams pp, float* __restrict__ phi, float* __restrict__ force, double* __restrict__ epart,
    int* __restrict__ err, float4* __restrict__ near_out) {
  constexpr int W = 2 * CUT + 1, NS = W * W * W, SL = (NS + 31) / 32, SELFK = (NS - 1) / 2;
  __shared__ __align__(128) float4 sbuf[PP_WARPS][2][2 * NT_CAP];
  __shared__ __align__(8) unsigned long long sbar[PP_WARPS][2];
  const float4* P = reinterpret_cast<const float4*>(part);
  const char* S2 = reinterpret_cast<const char*>(src2f);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t bar0 = tc::smem_u32(&sbar[warp][0]), bar1 = tc::smem_u32(&sbar[warp][1]);
  const uint32_t buf0 = tc::smem_u32(&sbuf[warp][0][0]), buf1 = tc::smem_u32(&sbuf[warp][1][0]);
  if (lane == 0) {
    tc::bar_init(bar0, 1);
    tc::bar_init(bar1, 1);
    tc::fence_proxy_async();
  }
  __syncwarp();
  uint32_t parity = 0;  // bit b: parity of the next phase of buffer b
  const uint32_t nitems = item_start[K];
  const int nx = pp.n[0], ny = pp.n[1], nz = pp.n[2];
  const float csx = pp.cs32[0], csy = pp.cs32[1], csz = pp.cs32[2];
  uint32_t item = 0, batch_end = 0;
  for (;;) {
    if (item >= batch_end) {
      if (lane == 0) item = atomicAdd(counter, (unsigned)PP_BATCH);
      item = __shfl_sync(0xffffffffu, item, 0);
      batch_end = item + PP_BATCH;
    }
    if (item >= nitems) break;  // warp-uniform
    const int cell = (int)item_cell[item];
    const int chunk = (int)(item - item_start[cell]);
    const int tbeg = cs[cell] + chunk * CHUNK;
    const int R = min(CHUNK, cs[cell + 1] - tbeg);
    int TL = 1;
    while (TL < R) TL <<= 1;
    const int SP = 32 / TL;
    const int tl = lane & (TL - 1), ph = lane / TL;
    const bool active = tl < R;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) xi = P[tbeg + tl];
    const int sbase = cell - cell % pp.ksys, lc = cell - sbase;
    const int ix = lc % nx, iy = (lc / nx) % ny, iz = lc / (nx * ny);
    // segment s (lane s % 32, slot s / 32): the own cell for s = 0, then the other
    // cells k = s - 1 (k >= SELFK: s) of the (2c+1)^3 block, x fastest: first pair
    // (global), pair count, first pair in the item's numbering, and the shift that
    // moves the cell's sources into the target cell's frame.  The numbering pads the
    // own cell and the whole list to multiples of 4 pairs with zero-charge dummies.
    int gb[SL], gn[SL], gf[SL];
    float gsx[SL], gsy[SL], gsz[SL];
#pragma unroll
    for (int j = 0; j < SL; ++j) {
      const int sg = lane + 32 * j;
      gb[j] = gn[j] = 0;
      gsx[j] = gsy[j] = gsz[j] = 0.f;
      if (sg < NS) {
        const int kk = sg == 0 ? SELFK : (sg - 1 >= SELFK ? sg : sg - 1);
        const int dx = kk % W - CUT, dy = (kk / W) % W - CUT, dz = kk / (W * W) - CUT;
        int jx = ix + dx, jy = iy + dy, jz = iz + dz;
        bool ok = true;
        if (jx < 0 || jx >= nx) { ok = ok && pp.periodic; jx += (jx < 0) ? nx : -nx; }
        if (jy < 0 || jy >= ny) { ok = ok && pp.periodic; jy += (jy < 0) ? ny : -ny; }
        if (jz < 0 || jz >= nz) { ok = ok && pp.periodic; jz += (jz < 0) ? nz : -nz; }
        if (ok) {
          const int cj = sbase + jx + nx * (jy + ny * jz);
          gb[j] = (int)__ldg(pair_start + cj);
          gn[j] = (int)__ldg(pair_start + cj + 1) - gb[j];
        }
        gsx[j] = (float)dx * csx;
        gsy[j] = (float)dy * csy;
        gsz[j] = (float)dz * csz;
      }
    }
    const int nself = __shfl_sync(0xffffffffu, gn[0], 0);
    const int nselfp = (nself + 3) & ~3;  // own cell, padded: [0, nselfp)
    int total = 0;
#pragma unroll
    for (int j = 0; j < SL; ++j) {
      const int w = (j == 0 && lane == 0) ? nselfp : gn[j];
      int v = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      gf[j] = total + v - w;
      total += __shfl_sync(0xffffffffu, v, 31);
    }
    const int real_end = total;        // dummies of the tail: [real_end, total)
    total = (total + 3) & ~3;
    const int nch = (total + NT_CAP - 1) / NT_CAP;
    // queues the copies of chunk ch into buffer b (real pairs only)
    auto issue = [&](int ch, int b) {
      const int base = ch * NT_CAP, end = min(base + NT_CAP, total);
      const int dummies = max(0, min(end, nselfp) - max(base, nself)) + max(0, end - max(base, real_end));
      const uint32_t bar = b ? bar1 : bar0, dst = b ? buf1 : buf0;
      if (lane == 0) bar_expect_tx(bar, (uint32_t)(end - base - dummies) * 32u);
      __syncwarp();
      tc::fence_proxy_async();
#pragma unroll
      for (int j = 0; j < SL; ++j) {
        const int lo = max(gf[j], base), hi = min(gf[j] + gn[j], end);
        if (hi > lo)
          bulk_g2s(dst + 32u * (uint32_t)(lo - base), S2 + 32 * ((int64_t)gb[j] + (lo - gf[j])),
                   32u * (uint32_t)(hi - lo), bar);
      }
    };
    for (int c0 = 0; c0 < 2 && c0 < nch; ++c0) issue(c0, c0);
    float2 pot = make_float2(0.f, 0.f), gx = pot, gy = pot, gz = pot;
    const float2 tx = make_float2(xi.x, xi.x), ty = make_float2(xi.y, xi.y), tz = make_float2(xi.z, xi.z);
    int sc = 1;  // first segment not yet moved into the target's frame
    bool ok = true;
    for (int ch = 0; ch < nch; ++ch) {
      const int b = ch & 1;
      const uint32_t bar = b ? bar1 : bar0;
      const bool done = tc::bar_wait(bar, (parity >> b) & 1u, NT_WAIT_POLLS);
      if (!__all_sync(0xffffffffu, done)) {
        if (lane == 0) set_err(err, ERRBIT_TIMEOUT);
        tc::bar_wait(bar, (parity >> b) & 1u, NT_WAIT_POLLS);
        if (ch + 1 < nch) tc::bar_wait(b ? bar0 : bar1, (parity >> (b ^ 1)) & 1u, NT_WAIT_POLLS);
        ok = false;
        break;
      }
      parity ^= 1u << b;
      float4* buf = &sbuf[warp][b][0];
      const int base = ch * NT_CAP, end = min(base + NT_CAP, total);
      // dummies: zero charge far outside every cell (they add exact zeros)
      const float4 far4 = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 1.0e4f), farq = make_float4(1.0e4f, 1.0e4f, 0.f, 0.f);
      for (int e = max(base, nself) + lane; e < min(end, nselfp); e += 32) {
        buf[2 * (e - base)] = far4;
        buf[2 * (e - base) + 1] = farq;
      }
      for (int e = max(base, real_end) + lane; e < end; e += 32) {
        buf[2 * (e - base)] = far4;
        buf[2 * (e - base) + 1] = farq;
      }
      // the neighbour cells' sources of this chunk moved into the target cell's frame
      while (sc < NS) {
        const int j = sc >> 5, src = sc & 31;
        int f = gf[0], n = gn[0];
        float sx = gsx[0], sy = gsy[0], sz = gsz[0];
#pragma unroll
        for (int q = 1; q < SL; ++q)
          if (j == q) {
            f = gf[q];
            n = gn[q];
            sx = gsx[q];
            sy = gsy[q];
            sz = gsz[q];
          }
        f = __shfl_sync(0xffffffffu, f, src);
        if (f >= end) break;  // the segment starts in a later chunk
        n = __shfl_sync(0xffffffffu, n, src);
        sx = __shfl_sync(0xffffffffu, sx, src);
        sy = __shfl_sync(0xffffffffu, sy, src);
        sz = __shfl_sync(0xffffffffu, sz, src);
        const int lo = max(f, base), hi = min(f + n, end);
        for (int e = lo + lane; e < hi; e += 32) {
          float4 A = buf[2 * (e - base)], B = buf[2 * (e - base) + 1];
          A.x += sx;
          A.y += sx;
          A.z += sy;
          A.w += sy;
          B.x += sz;
          B.y += sz;
          buf[2 * (e - base)] = A;
          buf[2 * (e - base) + 1] = B;
        }
        if (f + n > end) break;  // the segment continues in the next chunk
        ++sc;
      }
      __syncwarp();
      // own-cell pairs (self pair masked), then the rest of the chunk in one sweep
      const int s1 = min(max(nselfp - base, 0), end - base);
      if (s1 > 0) pp_sweep<true>(buf, s1, ph, SP, tx, ty, tz, pot, gx, gy, gz);
      if (end - base > s1) pp_sweep<false>(buf + 2 * s1, end - base - s1, ph, SP, tx, ty, tz, pot, gx, gy, gz);
      __syncwarp();  // every lane is done with buffer b
      if (ch + 2 < nch) issue(ch + 2, b);
    }
    if (!__all_sync(0xffffffffu, ok)) return;
    float ps = pot.x + pot.y, gxs = -(gx.x + gx.y), gys = -(gy.x + gy.y), gzs = -(gz.x + gz.y);
    for (int o = TL; o < 32; o <<= 1) {
      ps += __shfl_xor_sync(0xffffffffu, ps, o);
      gxs += __shfl_xor_sync(0xffffffffu, gxs, o);
      gys += __shfl_xor_sync(0xffffffffu, gys, o);
      gzs += __shfl_xor_sync(0xffffffffu, gzs, o);
    }
    // near sums in units of 1 / hs and 1 / hs^2, each product rounded on its own
    // (no contraction with the far-field addition), so that the split evaluation,
    // which stores them and adds the far field later, gives the same results
    const float np0 = __fmul_rn(ps, pp.ih32), np1 = __fmul_rn(gxs, pp.ih2_32), np2 = __fmul_rn(gys, pp.ih2_32),
                np3 = __fmul_rn(gzs, pp.ih2_32);
    if (near_out) {  // split evaluation: the near sums only, combined later by pp_combine_kernel
      if (active && ph == 0) near_out[tbeg + tl] = make_float4(np0, np1, np2, np3);
      ++item;
      continue;
    }
    float e_t = 0.f, f_t[3] = {0.f, 0.f, 0.f};
    if (active && ph == 0) {
      const int s = tbeg + tl;
      const float4 fr = reinterpret_cast<const float4*>(far)[s];
      const float sg = pp.sign32;
      const float pt = sg * (fr.x + np0);
      const float g0 = sg * (fr.y + np1), g1 = sg * (fr.z + np2), g2 = sg * (fr.w + np3);
      const uint32_t o = vals[s];
      const float q = xi.w;
      if (phi) phi[o] = pt;
      if (force) {
        force[3 * (int64_t)o + 0] = -q * g0;
        force[3 * (int64_t)o + 1] = -q * g1;
        force[3 * (int64_t)o + 2] = -q * g2;
      }
      e_t = 0.5f * q * pt;
      f_t[0] = -q * g0;
      f_t[1] = -q * g1;
      f_t[2] = -q * g2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e_t += __shfl_xor_sync(0xffffffffu, e_t, o);
      f_t[0] += __shfl_xor_sync(0xffffffffu, f_t[0], o);
      f_t[1] += __shfl_xor_sync(0xffffffffu, f_t[1], o);
      f_t[2] += __shfl_xor_sync(0xffffffffu, f_t[2], o);
    }
    if (lane == 0) {
      epart[(int64_t)item * 4 + 0] = (double)e_t;
      epart[(int64_t)item * 4 + 1] = (double)f_t[0];
      epart[(int64_t)item * 4 + 2] = (double)f_t[1];
      epart[(int64_t)item * 4 + 3] = (double)f_t[2];
    }
    ++item;
  }
}

// Combination of a split FP32 evaluation, where the near field ran beside the far
// field and left its sums (potential, gradient, in units of 1 / hs and 1 / hs^2)
// in near_out: one warp per work item, lane = target, the same combination,
// caller-order stores and per-item energy and net-force partials as the
// epilogue of pp_kernel_tma.
__global__ void __launch_bounds__(256) pp_combine_kernel(const float4* __restrict__ part,
                                                         const uint32_t* __restrict__ vals, const int* __restrict__ cs,
                                                         int64_t K, const uint32_t* __restrict__ item_start,
                                                         const uint32_t* __restrict__ item_cell,
                                                         const float4* __restrict__ far,
                                                         const float4* __restrict__ nearv, PPParams pp,
                                                         float* __restrict__ phi, float* __restrict__ force,
                                                         double* __restrict__ epart) {
  const int lane = threadIdx.x & 31;
  const uint32_t nitems = item_start[K];
  const uint32_t wstride = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < nitems; item += wstride) {
    const int cell = (int)item_cell[item];
    const int tbeg = cs[cell] + (int)(item - item_start[cell]) * CHUNK;
    const int R = min(CHUNK, cs[cell + 1] - tbeg);
    float e_t = 0.f, f_t[3] = {0.f, 0.f, 0.f};
    if (lane < R) {
      const int s = tbeg + lane;
      const float4 fr = far[s], nr = nearv[s];
      const float sg = pp.sign32;
      const float pt = sg * (fr.x + nr.x);
      const float g0 = sg * (fr.y + nr.y), g1 = sg * (fr.z + nr.z), g2 = sg * (fr.w + nr.w);
      const uint32_t o = vals[s];
      const float q = part[s].w;
      if (phi) phi[o] = pt;
      if (force) {
        force[3 * (int64_t)o + 0] = -q * g0;
        force[3 * (int64_t)o + 1] = -q * g1;
        force[3 * (int64_t)o + 2] = -q * g2;
      }
      e_t = 0.5f * q * pt;
      f_t[0] = -q * g0;
      f_t[1] = -q * g1;
      f_t[2] = -q * g2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      e_t += __shfl_xor_sync(0xffffffffu, e_t, o);
      f_t[0] += __shfl_xor_sync(0xffffffffu, f_t[0], o);
      f_t[1] += __shfl_xor_sync(0xffffffffu, f_t[1], o);
      f_t[2] += __shfl_xor_sync(0xffffffffu, f_t[2], o);
    }
    if (lane == 0) {
      epart[(int64_t)item * 4 + 0] = (double)e_t;
      epart[(int64_t)item * 4 + 1] = (double)f_t[0];
      epart[(int64_t)item * 4 + 2] = (double)f_t[1];
      epart[(int64_t)item * 4 + 3] = (double)f_t[2];
    }
  }
}

// FP32 near field (c = 1 or 2) with one thread per target: for sparsely filled cells,
// where the per-item set-up of the cell-item kernels costs more than the
// interactions.  Thread i takes sorted target i; it walks the 9 neighbour rows
// (dy, dz) and in each row the pairs of the cells x-1, x, x+1 of the pair layout
// (sources of neighbouring targets coincide, so loads are served by L1).  Energy
// and net-force terms are reduced per work item: a segmented warp scan over
// lanes of equal item, one store per item that lies inside the warp, and two
// double atomics (commutative, so deterministic) on a zeroed slot for an item
// split between two warps.
constexpr int PPS_THREADS = 256;

template <int CUT>
__global__ void __launch_bounds__(PPS_THREADS, 4) pp_target_kernel(
    const float4* __restrict__ P, const ulonglong2* __restrict__ S2, const uint32_t* __restrict__ pair_start,
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals, const int* __restrict__ cs,
    const uint32_t* __restrict__ item_start, int64_t n, const float4* __restrict__ far, PPParams pp,
    float* __restrict__ phi, float* __restrict__ force, double* __restrict__ epart) {
  const int64_t i = (int64_t)blockIdx.x * PPS_THREADS + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t wbase = i - lane;
  float e_t = 0.f, f_t0 = 0.f, f_t1 = 0.f, f_t2 = 0.f;
  uint32_t item = 0xffffffffu;
  int64_t tb = 0, te = 0;
  if (i < n) {
    const float4 xi = P[i];
    const int cell = (int)keys[i];
    const int c0 = cs[cell], c1 = cs[cell + 1];
    const int chunk = (int)((i - c0) / CHUNK);
    item = item_start[cell] + (uint32_t)chunk;
    tb = c0 + (int64_t)chunk * CHUNK;
    te = min(tb + CHUNK, (int64_t)c1);
    const int nx = pp.n[0], ny = pp.n[1], nz = pp.n[2];
    const int sbase = cell - cell % pp.ksys, lc = cell - sbase;
    const int ix = lc % nx, iy = (lc / nx) % ny, iz = lc / (nx * ny);
    const float csx = pp.cs32[0], csy = pp.cs32[1], csz = pp.cs32[2];
    f2 pot = pk2(0.f, 0.f), gx = pot, gy = pot, gz = pot;
    for (int dz = -CUT; dz <= CUT; ++dz) {
      int jz = iz + dz;
      if (jz < 0 || jz >= nz) {
        if (!pp.periodic) continue;
        jz += (jz < 0) ? nz : -nz;
      }
      const float tzs = xi.z - (float)dz * csz;
      const f2 tz = pk2(tzs, tzs);
      for (int dy = -CUT; dy <= CUT; ++dy) {
        int jy = iy + dy;
        if (jy < 0 || jy >= ny) {
          if (!pp.periodic) continue;
          jy += (jy < 0) ? ny : -ny;
        }
        const float tys = xi.y - (float)dy * csy;
        const f2 ty = pk2(tys, tys);
        const int row = sbase + nx * (jy + ny * jz);
#pragma unroll
        for (int d = 0; d < 2 * CUT + 1; ++d) {
          int jx = ix + d - CUT;
          if (jx < 0 || jx >= nx) {
            if (!pp.periodic) continue;
            jx += (jx < 0) ? nx : -nx;
          }
          const int pb = (int)__ldg(pair_start + row + jx), pe = (int)__ldg(pair_start + row + jx + 1);
          const float txs = xi.x - (float)(d - CUT) * csx;
          const f2 tx = pk2(txs, txs);
#pragma unroll 1
          for (int pr = pb; pr < pe; ++pr)
            pp_pair2_mixed<true>(S2[2 * pr], S2[2 * pr + 1], tx, ty, tz, pot, gx, gy, gz);
        }
      }
    }
    float pa, pbv, xa, xb, ya, yb, za, zb;
    up2(pot, pa, pbv);
    up2(gx, xa, xb);
    up2(gy, ya, yb);
    up2(gz, za, zb);
    const float ps = pa + pbv, gxs = -(xa + xb), gys = -(ya + yb), gzs = -(za + zb);
    const float4 fr = far[i];
    const float ih = pp.ih32, ih2 = pp.ih2_32, sg = pp.sign32;
    const float pt = sg * (fr.x + ps * ih);
    const float g0 = sg * (fr.y + gxs * ih2), g1 = sg * (fr.z + gys * ih2), g2 = sg * (fr.w + gzs * ih2);
    const uint32_t o = vals[i];
    const float q = xi.w;
    if (phi) phi[o] = pt;
    if (force) {
      force[3 * (int64_t)o + 0] = -q * g0;
      force[3 * (int64_t)o + 1] = -q * g1;
      force[3 * (int64_t)o + 2] = -q * g2;
    }
    e_t = 0.5f * q * pt;
    f_t0 = -q * g0;
    f_t1 = -q * g1;
    f_t2 = -q * g2;
  }
  // segmented inclusive scan over runs of lanes with the same item
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float ue = __shfl_up_sync(0xffffffffu, e_t, o), u0 = __shfl_up_sync(0xffffffffu, f_t0, o);
    const float u1 = __shfl_up_sync(0xffffffffu, f_t1, o), u2 = __shfl_up_sync(0xffffffffu, f_t2, o);
    const uint32_t uit = __shfl_up_sync(0xffffffffu, item, o);
    if (lane >= o && uit == item) {
      e_t += ue;
      f_t0 += u0;
      f_t1 += u1;
      f_t2 += u2;
    }
  }
  const uint32_t next = __shfl_down_sync(0xffffffffu, item, 1);
  if (i < n && (lane == 31 || next != item)) {
    double* ep = epart + 4 * (int64_t)item;
    if (tb >= wbase && te <= wbase + 32) {
      ep[0] = (double)e_t;
      ep[1] = (double)f_t0;
      ep[2] = (double)f_t1;
      ep[3] = (double)f_t2;
    } else {
      atomicAdd(ep + 0, (double)e_t);
      atomicAdd(ep + 1, (double)f_t0);
      atomicAdd(ep + 2, (double)f_t1);
      atomicAdd(ep + 3, (double)f_t2);
    }
  }
}

}  // namespace

int64_t pp_items_max(int64_t K, int64_t n) { return K + (n + CHUNK - 1) / CHUNK + 1; }

int64_t pp_pairs_max(int64_t K, int64_t n) { return (n + K) / 2 + 1; }

int64_t pp_lists_chunk_entries(int64_t K) {
  const int64_t a = scan_chunk_count(K + 1), b = 2 * ((K + 1 + LIST_BLK - 1) / LIST_BLK);
  return a > b ? a : b;
}

cudaError_t launch_pp_lists(const int* cell_start, int64_t K, uint32_t* item_start, uint32_t* pair_start,
                            uint32_t* chunks, unsigned int* counter, cudaStream_t s, int* nl) {
  const int64_t nb = (K + 1 + LIST_BLK - 1) / LIST_BLK;
  if (nb <= LIST_MAX_BLOCKS) {
    list_local_kernel<<<(unsigned)nb, LIST_BLK, 0, s>>>(cell_start, K, item_start, pair_start, chunks, counter);
    ++*nl;
    if (nb > 1) {
      list_fix_kernel<<<(unsigned)nb, LIST_BLK, 0, s>>>(K, item_start, pair_start, chunks);
      ++*nl;
    }
    return cudaGetLastError();
  }
  item_count_kernel<<<(unsigned)((K + 1 + 255) / 256), 256, 0, s>>>(cell_start, K, item_start, pair_start, counter);
  ++*nl;
  cudaError_t e = launch_exclusive_scan(item_start, K + 1, chunks, s, nl);
  if (e == cudaSuccess && pair_start) e = launch_exclusive_scan(pair_start, K + 1, chunks, s, nl);
  return e;
}

cudaError_t launch_gather_lists(const void* rec, bool fp64, const uint32_t* vals, const uint32_t* keys,
                                const int* cell_start, const uint32_t* item_start, const uint32_t* pair_start,
                                int64_t n, int64_t K, void* part, void* src2, uint32_t* item_cell, double* epart,
                                int64_t max_items, bool zero_all, cudaStream_t s, int* nl) {
  const int64_t work = n > max_items ? n : max_items;
  const unsigned blocks = (unsigned)((work + 255) / 256 > 0 ? (work + 255) / 256 : 1);
  if (fp64)
    gather_lists_kernel<double4, false><<<blocks, 256, 0, s>>>((const double4*)rec, vals, keys, cell_start, item_start,
                                                                 pair_start, n, K, (double4*)part, nullptr, item_cell,
                                                                 epart, max_items, zero_all ? 1 : 0);
  else if (src2)
    gather_lists_kernel<float4, true><<<blocks, 256, 0, s>>>((const float4*)rec, vals, keys, cell_start, item_start,
                                                               pair_start, n, K, (float4*)part, (float*)src2,
                                                               item_cell, epart, max_items, zero_all ? 1 : 0);
  else
    gather_lists_kernel<float4, false><<<blocks, 256, 0, s>>>((const float4*)rec, vals, keys, cell_start, item_start,
                                                                pair_start, n, K, (float4*)part, nullptr, item_cell,
                                                                epart, max_items, zero_all ? 1 : 0);
  ++*nl;
  return cudaGetLastError();
}

bool pp_per_target_applies(bool fp64, int c) { return !fp64 && c <= 2; }
bool pp_tma_applies(bool fp64, int c, bool per_target) { return !fp64 && c <= 2 && !per_target; }

cudaError_t launch_pp_combine(const void* part, const uint32_t* vals, const int* cell_start, int64_t K,
                              const uint32_t* item_start, const uint32_t* item_cell, int64_t max_items,
                              const void* far, const void* nearv, PPParams pp, void* phi, void* force, double* epart,
                              int num_sms, cudaStream_t s, int* nl) {
  if (max_items <= 0) return cudaSuccess;
  (void)num_sms;
  const int64_t blocks = (max_items + 7) / 8;  // 8 warps (items) per block, one item per warp
  pp_combine_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float4*)part, vals, cell_start, K, item_start, item_cell,
                                                     (const float4*)far, (const float4*)nearv, pp, (float*)phi,
                                                     (float*)force, epart);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_pp(bool fp64, const void* part, const void* src2, const uint32_t* pair_start, const uint32_t* vals,
                      const uint32_t* keys, int64_t n, bool per_target, const int* cell_start, int64_t K,
                      const uint32_t* item_start, const uint32_t* item_cell, unsigned int* counter, int num_sms,
                      const void* far, PPParams pp, void* phi, void* force, double* epart, int* err, void* near_out,
                      cudaStream_t s, int* nl) {
  // persistent launch: PP_BLOCKS_PER_SM resident blocks of PP_WARPS warps per SM
  const unsigned blocks = (unsigned)(PP_BLOCKS_PER_SM * (num_sms > 0 ? num_sms : 1));
  if (per_target && pp_per_target_applies(fp64, pp.c) && src2 != nullptr) {
    if (n <= 0) return cudaSuccess;
    const unsigned g = (unsigned)((n + PPS_THREADS - 1) / PPS_THREADS);
    if (pp.c <= 1)
      pp_target_kernel<1><<<g, PPS_THREADS, 0, s>>>((const float4*)part, (const ulonglong2*)src2, pair_start, keys,
                                                    vals, cell_start, item_start, n, (const float4*)far, pp,
                                                    (float*)phi, (float*)force, epart);
    else
      pp_target_kernel<2><<<g, PPS_THREADS, 0, s>>>((const float4*)part, (const ulonglong2*)src2, pair_start, keys,
                                                    vals, cell_start, item_start, n, (const float4*)far, pp,
                                                    (float*)phi, (float*)force, epart);
  } else if (pp_tma_applies(fp64, pp.c, false) && src2 != nullptr) {
    const unsigned tblocks = (unsigned)(NT_BLOCKS_PER_SM * (num_sms > 0 ? num_sms : 1));
    if (pp.c <= 1)
      pp_kernel_tma<1><<<tblocks, PP_WARPS * 32, 0, s>>>((const float*)part, (const float*)src2, pair_start, vals,
                                                         cell_start, K, item_start, item_cell, counter,
                                                         (const float*)far, pp, (float*)phi, (float*)force, epart, err,
                                                         (float4*)near_out);
    else
      pp_kernel_tma<2><<<tblocks, PP_WARPS * 32, 0, s>>>((const float*)part, (const float*)src2, pair_start, vals,
                                                         cell_start, K, item_start, item_cell, counter,
                                                         (const float*)far, pp, (float*)phi, (float*)force, epart, err,
                                                         (float4*)near_out);
  } else {
    if (near_out) return cudaErrorInvalidValue;  // only the cell-item FP32 kernel splits
#define PP_LAUNCH(T, S)                                                                                              \
  pp_kernel<T, S><<<blocks, PP_WARPS * 32, 0, s>>>((const T*)part, vals, cell_start, K, item_start, item_cell, counter, \
                                                   (const T*)far, pp, (T*)phi, (T*)force, epart)
    if (fp64) {
      if (pp.c <= 1) PP_LAUNCH(double, 1); else PP_LAUNCH(double, 4);
    } else {
      if (pp.c <= 1) PP_LAUNCH(float, 1); else PP_LAUNCH(float, 4);
    }
#undef PP_LAUNCH
  }
  ++*nl;
  return cudaGetLastError();
}

}  // namespace pmmm
