// P2M (Eq. P2M) and L2P with the order-one gradient (Eqs. L2P, L2L, phigrad).
//
// Device units: positions relative to the cell centre in units of hs, so the
// moments computed here are M'_l = M_l / hs^l and the locals read are
// L'_l = hs^(l+1) L_l; the physical potential is phi = phi' / hs and the
// gradient grad' / hs^2.
#include "harmonics.cuh"
#include "internal.cuh"
#include "translations.cuh"

namespace pmmm {

namespace {

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

// acc += q R(-u): the harmonics streamed column by column up to order 8 (fewer
// registers); above, the (p+1)^2 array form (measured faster there).
template <int P, typename T>
__device__ __forceinline__ void p2m_accumulate(T ux, T uy, T uz, T q, T* acc) {
  constexpr int C = (P + 1) * (P + 1);
  if constexpr (P <= 8) {
    regular_stream<P, T>(-ux, -uy, -uz, [&](int l, int m, T re, T im) {
      acc[sidx(l, m)] = fma(q, re, acc[sidx(l, m)]);
      if (m > 0) acc[sidx(l, -m)] = fma(q, im, acc[sidx(l, -m)]);
    });
  } else {
    T R[C];
    regular_real<P, T>(-ux, -uy, -uz, R);
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = fma(q, R[c], acc[c]);
  }
}

// Eight lanes per cell: each lane accumulates q R(r_M - r_i) = q R(-u) of every
// eighth particle of its cell into (p+1)^2 registers, a 3-step butterfly sums the
// eight lanes, and a shared-memory transpose writes the channel-major M of 16
// consecutive cells with coalesced stores.  Also the per-cell sums used by the
// periodic corrections: cellsum = (sum q, sum q u_x, sum q u_y, sum q u_z,
// sum q |u|^2), accumulated in T per lane and stored in FP64.
constexpr int P2M_LPC = 8;                  // lanes per cell
constexpr int P2M_THREADS = 128;            // (small blocks fit beside the near field of a split evaluation)
constexpr int P2M_CPB = P2M_THREADS / P2M_LPC;  // cells per block

template <int P, typename T>
__global__ void __launch_bounds__(P2M_THREADS) p2m_kernel(const T* __restrict__ part, const int* __restrict__ cs, int64_t K,
                                                  T* __restrict__ M, double* __restrict__ cellsum) {
  constexpr int C = (P + 1) * (P + 1);
  __shared__ T sh[C][P2M_CPB + 1];
  const int sub = threadIdx.x & (P2M_LPC - 1), cl = threadIdx.x / P2M_LPC;
  const int64_t cell = (int64_t)blockIdx.x * P2M_CPB + cl;
  T acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = T(0);
  T sq = 0, sx = 0, sy = 0, sz = 0, sr = 0;
  if (cell < K) {
    const int beg = cs[cell], end = cs[cell + 1];
    for (int i = beg + sub; i < end; i += P2M_LPC) {
      const typename V4<T>::type r = reinterpret_cast<const typename V4<T>::type*>(part)[i];
      p2m_accumulate<P, T>(r.x, r.y, r.z, r.w, acc);
      sq += r.w;
      sx = fma(r.w, r.x, sx);
      sy = fma(r.w, r.y, sy);
      sz = fma(r.w, r.z, sz);
      sr = fma(r.w, r.x * r.x + r.y * r.y + r.z * r.z, sr);
    }
  }
#pragma unroll
  for (int o = 1; o < P2M_LPC; o <<= 1) {
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
    sz += __shfl_xor_sync(0xffffffffu, sz, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
  }
#pragma unroll
  for (int c = 0; c < C; ++c)
    if ((c & (P2M_LPC - 1)) == sub) sh[c][cl] = acc[c];
  if (sub == 0 && cell < K) {
    cellsum[cell] = (double)sq;
    cellsum[K + cell] = (double)sx;
    cellsum[2 * K + cell] = (double)sy;
    cellsum[3 * K + cell] = (double)sz;
    cellsum[4 * K + cell] = (double)sr;
  }
  __syncthreads();
  const int64_t c0 = (int64_t)blockIdx.x * P2M_CPB;
  for (int idx = threadIdx.x; idx < C * P2M_CPB; idx += P2M_THREADS) {
    const int c = idx / P2M_CPB, l = idx - c * P2M_CPB;
    if (c0 + l < K) M[(int64_t)c * K + c0 + l] = sh[c][l];
  }
}

// Sparsely filled cells (FP32, p <= 8): one thread per cell accumulates its particles
// and writes its channels with coalesced stores (consecutive threads hold
// consecutive cells).  Cells with more than P2M_BIG particles are taken by the
// whole warp instead (lanes over particles, xor-butterfly sum), so that a
// crowded cell does not hold up the 31 other lanes.
constexpr int P2M_BIG = 16;

template <int P, typename T>
__global__ void __launch_bounds__(256) p2m_cell_kernel(const T* __restrict__ part, const int* __restrict__ cs,
                                                       int64_t K, T* __restrict__ M, double* __restrict__ cellsum) {
  constexpr int C = (P + 1) * (P + 1);
  const int lane = threadIdx.x & 31;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int beg = 0, end = 0;
  if (cell < K) {
    beg = cs[cell];
    end = cs[cell + 1];
  }
  const bool big = end - beg > P2M_BIG;
  T acc[C];
  T sq = 0, sx = 0, sy = 0, sz = 0, sr = 0;
  auto accumulate = [&](int i) {
    const typename V4<T>::type r = reinterpret_cast<const typename V4<T>::type*>(part)[i];
    p2m_accumulate<P, T>(r.x, r.y, r.z, r.w, acc);
    sq += r.w;
    sx = fma(r.w, r.x, sx);
    sy = fma(r.w, r.y, sy);
    sz = fma(r.w, r.z, sz);
    sr = fma(r.w, r.x * r.x + r.y * r.y + r.z * r.z, sr);
  };
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = T(0);
  if (cell < K && !big) {
    for (int i = beg; i < end; ++i) accumulate(i);
#pragma unroll
    for (int c = 0; c < C; ++c) M[(int64_t)c * K + cell] = acc[c];
    cellsum[cell] = (double)sq;
    cellsum[K + cell] = (double)sx;
    cellsum[2 * K + cell] = (double)sy;
    cellsum[3 * K + cell] = (double)sz;
    cellsum[4 * K + cell] = (double)sr;
  }
  unsigned todo = __ballot_sync(0xffffffffu, cell < K && big);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const int64_t bc = __shfl_sync(0xffffffffu, cell, src);
    const int bb = __shfl_sync(0xffffffffu, beg, src), be = __shfl_sync(0xffffffffu, end, src);
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = T(0);
    sq = sx = sy = sz = sr = T(0);
    for (int i = bb + lane; i < be; i += 32) accumulate(i);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
      sq += __shfl_xor_sync(0xffffffffu, sq, o);
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
    }
#pragma unroll
    for (int c = 0; c < C; ++c)
      if ((c & 31) == lane) M[(int64_t)c * K + bc] = acc[c];
    if (lane == 0) {
      cellsum[bc] = (double)sq;
      cellsum[K + bc] = (double)sx;
      cellsum[2 * K + bc] = (double)sy;
      cellsum[3 * K + bc] = (double)sz;
      cellsum[4 * K + bc] = (double)sr;
    }
  }
}

// Two-level plans (Sec. 5, hierarchical treatment): the multipoles of the coarse
// cells straight from the particles (Eq. P2M about the coarse centres), with the
// coarse per-cell sums of the periodic corrections.  One block per coarse cell;
// thread t takes the particles of the cell's r^3 fine cells whose running index
// is t modulo the block size (an even share whatever the fine occupancies);
// positions move to the coarse frame, u_c = (u_f + d_a) / r with d_a the fine
// centre minus the coarse centre in fine units; warp butterflies, then a
// fixed-order sum over the warps in shared memory.
constexpr int P2MC_THREADS = 256;

template <int P, typename T>
__global__ void __launch_bounds__(P2MC_THREADS) p2m_coarse_kernel(const T* __restrict__ part,
                                                                  const int* __restrict__ cs, CoarseGeo cg,
                                                                  T* __restrict__ Mc, double* __restrict__ cellsum) {
  constexpr int C = (P + 1) * (P + 1), NW = P2MC_THREADS / 32;
  __shared__ T red[NW][C + 5];
  const int64_t S = blockIdx.x;
  const int r = cg.r, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Sx = (int)(S % cg.nc[0]), Sy = (int)((S / cg.nc[0]) % cg.nc[1]), Sz = (int)(S / ((int64_t)cg.nc[0] * cg.nc[1]));
  const T ir = T(1) / T(r);
  T acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = T(0);
  T sq = 0, sx = 0, sy = 0, sz = 0, sr = 0;
  int run = 0;
  for (int az = 0; az < r; ++az)
    for (int ay = 0; ay < r; ++ay)
      for (int ax = 0; ax < r; ++ax) {
        const int64_t f = (int64_t)(Sx * r + ax) + (int64_t)cg.nf[0] * ((Sy * r + ay) + (int64_t)cg.nf[1] * (Sz * r + az));
        const int beg = cs[f], n = cs[f + 1] - beg;
        const T dx = (T)((ax + 0.5 - 0.5 * r) * cg.cs[0]), dy = (T)((ay + 0.5 - 0.5 * r) * cg.cs[1]),
                dz = (T)((az + 0.5 - 0.5 * r) * cg.cs[2]);
        for (int j = (tid - (run & (P2MC_THREADS - 1))) & (P2MC_THREADS - 1); j < n; j += P2MC_THREADS) {
          const typename V4<T>::type v = reinterpret_cast<const typename V4<T>::type*>(part)[beg + j];
          const T ux = (v.x + dx) * ir, uy = (v.y + dy) * ir, uz = (v.z + dz) * ir;
          p2m_accumulate<P, T>(ux, uy, uz, v.w, acc);
          sq += v.w;
          sx = fma(v.w, ux, sx);
          sy = fma(v.w, uy, sy);
          sz = fma(v.w, uz, sz);
          sr = fma(v.w, ux * ux + uy * uy + uz * uz, sr);
        }
        run += n;
      }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
    sq += __shfl_xor_sync(0xffffffffu, sq, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
    sz += __shfl_xor_sync(0xffffffffu, sz, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
  }
  if (lane == 0) {
#pragma unroll
    for (int c = 0; c < C; ++c) red[warp][c] = acc[c];
    red[warp][C] = sq;
    red[warp][C + 1] = sx;
    red[warp][C + 2] = sy;
    red[warp][C + 3] = sz;
    red[warp][C + 4] = sr;
  }
  __syncthreads();
  for (int c = tid; c < C + 5; c += P2MC_THREADS) {
    T v = red[0][c];
    for (int w = 1; w < NW; ++w) v += red[w][c];
    if (c < C)
      Mc[(int64_t)c * cg.Kc + S] = v;
    else
      cellsum[(int64_t)(c - C) * cg.Kc + S] = (double)v;
  }
}

// One thread per sorted particle.  Far-field potential and gradient in
// physical units, with the periodic corrections of App. B.3:
//   phi  += c0 + c1 . r_rel + qfac (|r_rel|^2 - 3/(2 alpha^2)) - 2 alpha/sqrt(pi) Q_cell
//   grad += c1 + 2 qfac r_rel
// (the c1 terms only for p >= 1: they are the correction of L_1)
// (c0 = 2pi/(3V) sum q|r_rel|^2, c1 = -4pi/(3V) sum q r_rel, qfac = 2pi/(3V) Q).
template <int P, typename T>
__global__ void __launch_bounds__(128) l2p_kernel(const T* __restrict__ part, const uint32_t* __restrict__ keys,
                                                  int64_t n, const T* __restrict__ L, int64_t K,
                                                  const double* __restrict__ corr_all, const double* __restrict__ cellq,
                                                  CorrParams cp, T* __restrict__ far) {
  constexpr int C = (P + 1) * (P + 1);
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const typename V4<T>::type r = reinterpret_cast<const typename V4<T>::type*>(part)[i];
  const uint32_t cell32 = keys[i];
  const int64_t cell = cell32;
  // this particle's system (one system: no division)
  const double* corr = corr_all + (cp.ksys >= K ? 0 : 16 * (int64_t)(cell32 / (uint32_t)cp.ksys));
  T f, gx, gy, gz;
  if constexpr (P >= 9) {
    // high orders: harmonics streamed column by column (no (p+1)^2 array)
    l2p_stream<P, T>([&](int c) { return __ldg(L + (int64_t)c * K + cell); }, r.x, r.y, r.z, f, gx, gy, gz);
  } else {
    T R[C];
    regular_real<P, T>(r.x, r.y, r.z, R);
    l2p_real<P, T>([&](int c) { return __ldg(L + (int64_t)c * K + cell); }, R, f, gx, gy, gz);
  }
  constexpr bool F32 = sizeof(T) == 4;
  const T ih = F32 ? (T)cp.ih32 : (T)cp.ih, ih2 = F32 ? (T)cp.ih2_32 : (T)cp.ih2;
  T phi = f * ih;
  T g[3] = {gx * ih2, gy * ih2, gz * ih2};
  if (cp.periodic) {
    // the correction terms: FP32 copies on the FP32 path (no FP64 conversion per particle)
    T cr[5];
    if constexpr (F32) {
      const float* cf = reinterpret_cast<const float*>(corr + CORR_F32);
#pragma unroll
      for (int k = 0; k < 5; ++k) cr[k] = cf[k];
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k) cr[k] = corr[k];
    }
    const T hs = F32 ? (T)cp.hs32 : (T)cp.hs;
    T rel[3] = {r.x * hs, r.y * hs, r.z * hs};
    int64_t qcell = cell;
    if (cp.refine > 1) {
      // two-level plan: position relative to the coarse centre, charge of the coarse cell
      const int R = cp.refine;
      const uint32_t nx = (uint32_t)cp.nf[0], ny = (uint32_t)cp.nf[1];
      const uint32_t ix = cell32 % nx, iy = (cell32 / nx) % ny, iz = cell32 / (nx * ny);
      const uint32_t ic[3] = {ix, iy, iz};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if constexpr (F32)
          rel[a] += ((float)(ic[a] % (uint32_t)R) + (0.5f - 0.5f * (float)R)) * cp.cshs32[a];
        else
          rel[a] += ((double)(ic[a] % (uint32_t)R) + 0.5 - 0.5 * R) * cp.cs[a] * cp.hs;
      }
      qcell = ix / R + (int64_t)cp.nc[0] * (iy / R + (int64_t)cp.nc[1] * (iz / R));
    }
    const T rr = rel[0] * rel[0] + rel[1] * rel[1] + rel[2] * rel[2];
    const T qf = cr[4];
    const T cch = F32 ? (T)cp.c_charged32 : (T)cp.c_charged, cself = F32 ? (T)cp.c_self32 : (T)cp.c_self;
    phi += cr[0] + qf * (rr - cch) - cself * (T)cellq[qcell];
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] += T(2) * qf * rel[a];
    // the dipole term corrects L_1 (App. B.3), which exists only for p >= 1
    if (P >= 1) {
      phi += cr[1] * rel[0] + cr[2] * rel[1] + cr[3] * rel[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) g[a] += cr[1 + a];
    }
  }
  typename V4<T>::type o;
  o.x = (T)phi;
  o.y = (T)g[0];
  o.z = (T)g[1];
  o.w = (T)g[2];
  reinterpret_cast<typename V4<T>::type*>(far)[i] = o;
}

template <int P, typename T>
cudaError_t p2m_run(const void* part, const int* cs, int64_t K, void* M, double* cq, double* cd, bool sparse,
                    cudaStream_t s) {
  (void)cd;  // the per-cell sums are laid out [5][K] starting at cq
  // one thread per cell keeps its (p+1)^2 sums in registers: FP32 and p <= 8 only
  if constexpr (sizeof(T) == 4 && P <= 8) {
    if (sparse) {
      p2m_cell_kernel<P, T><<<(unsigned)((K + 255) / 256), 256, 0, s>>>((const T*)part, cs, K, (T*)M, cq);
      return cudaGetLastError();
    }
  }
  const int blocks = (int)((K + P2M_CPB - 1) / P2M_CPB);
  p2m_kernel<P, T><<<blocks, P2M_THREADS, 0, s>>>((const T*)part, cs, K, (T*)M, cq);
  return cudaGetLastError();
}

template <int P, typename T>
cudaError_t l2p_run(const void* part, const uint32_t* keys, int64_t n, const void* L, int64_t K, const double* corr,
                    const double* cq, CorrParams cp, void* far, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  l2p_kernel<P, T><<<(int)((n + 127) / 128), 128, 0, s>>>((const T*)part, keys, n, (const T*)L, K, corr, cq, cp,
                                                          (T*)far);
  return cudaGetLastError();
}

template <int P>
cudaError_t p2m_dispatch(int p, bool fp64, const void* part, const int* cs, int64_t K, void* M, double* cq,
                         double* cd, bool sparse, cudaStream_t s) {
  if (p == P)
    return fp64 ? p2m_run<P, double>(part, cs, K, M, cq, cd, sparse, s)
                : p2m_run<P, float>(part, cs, K, M, cq, cd, sparse, s);
  if constexpr (P < PMMM_PMAX) return p2m_dispatch<P + 1>(p, fp64, part, cs, K, M, cq, cd, sparse, s);
  return cudaErrorInvalidValue;
}

template <int P>
cudaError_t l2p_dispatch(int p, bool fp64, const void* part, const uint32_t* keys, int64_t n, const void* L,
                         int64_t K, const double* corr, const double* cq, CorrParams cp, void* far, cudaStream_t s) {
  if (p == P)
    return fp64 ? l2p_run<P, double>(part, keys, n, L, K, corr, cq, cp, far, s)
                : l2p_run<P, float>(part, keys, n, L, K, corr, cq, cp, far, s);
  if constexpr (P < PMMM_PMAX) return l2p_dispatch<P + 1>(p, fp64, part, keys, n, L, K, corr, cq, cp, far, s);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_p2m(int p, bool fp64, const void* part, const int* cell_start, int64_t K, void* M, double* cellq,
                       double* celld, bool sparse, cudaStream_t s, int* nl) {
  ++*nl;
  return p2m_dispatch<0>(p, fp64, part, cell_start, K, M, cellq, celld, sparse, s);
}

namespace {
template <int P>
cudaError_t p2m_coarse_dispatch(int p, bool fp64, const void* part, const int* cs, const CoarseGeo& cg, void* Mc,
                                double* cellsum, cudaStream_t s) {
  if (p == P) {
    if (fp64)
      p2m_coarse_kernel<P, double><<<(unsigned)cg.Kc, P2MC_THREADS, 0, s>>>((const double*)part, cs, cg, (double*)Mc,
                                                                            cellsum);
    else
      p2m_coarse_kernel<P, float><<<(unsigned)cg.Kc, P2MC_THREADS, 0, s>>>((const float*)part, cs, cg, (float*)Mc,
                                                                           cellsum);
    return cudaGetLastError();
  }
  if constexpr (P < PMMM_PMAX) return p2m_coarse_dispatch<P + 1>(p, fp64, part, cs, cg, Mc, cellsum, s);
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_p2m_coarse(int p, bool fp64, const void* part, const int* cell_start, const CoarseGeo& cg,
                              void* Mc, double* cellsum, cudaStream_t s, int* nl) {
  if (cg.Kc < 1 || cg.Kc > 0x7fffffff) return cudaErrorInvalidValue;
  ++*nl;
  return p2m_coarse_dispatch<0>(p, fp64, part, cell_start, cg, Mc, cellsum, s);
}

cudaError_t launch_l2p(int p, bool fp64, const void* part, const uint32_t* keys, int64_t n, const void* L, int64_t K,
                       const double* corr, const double* cellq, CorrParams cp, void* far, cudaStream_t s, int* nl) {
  if (n > 0) ++*nl;
  return l2p_dispatch<0>(p, fp64, part, keys, n, L, K, corr, cellq, cp, far, s);
}

}  // namespace pmmm
