// Near field (Sec. 2.1, Sec. 2.2): the pure Newtonian 1/r interaction with every
// particle of the (2c+1)^3 masked cells, plus the combination with the far field
// and the scatter back to the caller's order:
//   phi_i   = sign * (phi_far + sum_j q_j / r_ij)
//   force_i = -q_i * sign * (grad_far + sum_j grad(q_j / r_ij))
// One block per target cell; the sources of the neighbour cells are staged in
// shared memory, shifted into the target cell's frame (periodic images included).
#include "internal.cuh"

namespace pmmm {

namespace {

constexpr int PP_THREADS = 128;
constexpr int PP_TILE = 1024;
constexpr int PP_MAXNB = 125;  // c <= 2

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; };
template <> struct V4<double> { using type = double4; };

template <typename T> __device__ __forceinline__ T rsq(T x);
template <> __device__ __forceinline__ float rsq<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsq<double>(double x) { return rsqrt(x); }

template <typename T>
__global__ void __launch_bounds__(PP_THREADS) pp_kernel(const T* __restrict__ part, const uint32_t* __restrict__ vals,
                                                        const int* __restrict__ cs, int64_t K,
                                                        const T* __restrict__ far, PPParams pp, T* __restrict__ phi,
                                                        T* __restrict__ force, double* __restrict__ epart) {
  using V = typename V4<T>::type;
  __shared__ V src[PP_TILE];
  __shared__ int nb_beg[PP_MAXNB], nb_off[PP_MAXNB + 1];
  __shared__ T nb_sh[PP_MAXNB][3];
  __shared__ int nb_n;
  __shared__ double red[PP_THREADS / 32][4];
  const int64_t cell = blockIdx.x;
  const int tid = threadIdx.x;
  const int ix = (int)(cell % pp.n[0]), iy = (int)((cell / pp.n[0]) % pp.n[1]),
            iz = (int)(cell / ((int64_t)pp.n[0] * pp.n[1]));
  const int tbeg = cs[cell], tcount = cs[cell + 1] - tbeg;
  if (tid == 0) {
    int k = 0, off = 0;
    const int c = pp.c;
    for (int ez = -c; ez <= c; ++ez)
      for (int ey = -c; ey <= c; ++ey)
        for (int ex = -c; ex <= c; ++ex) {
          int j[3] = {ix + ex, iy + ey, iz + ez};
          bool ok = true;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (j[a] < 0 || j[a] >= pp.n[a]) {
              if (pp.periodic)
                j[a] = (j[a] + pp.n[a]) % pp.n[a];
              else
                ok = false;
            }
          }
          if (!ok) continue;
          const int64_t cj = j[0] + (int64_t)pp.n[0] * (j[1] + (int64_t)pp.n[1] * j[2]);
          const int b = cs[cj], cnt = cs[cj + 1] - b;
          if (cnt == 0) continue;
          nb_beg[k] = b;
          nb_off[k] = off;
          // centre of the source cell relative to the target cell, units of hs
          nb_sh[k][0] = (T)(ex * pp.cs[0]);
          nb_sh[k][1] = (T)(ey * pp.cs[1]);
          nb_sh[k][2] = (T)(ez * pp.cs[2]);
          off += cnt;
          ++k;
        }
    nb_off[k] = off;
    nb_n = k;
  }
  __syncthreads();
  const int nn = nb_n;
  const int S = nb_off[nn];
  const int tpt = tcount <= 32 ? 4 : (tcount <= 64 ? 2 : 1);
  const int ntg = PP_THREADS / tpt;
  double e_acc = 0, f_acc[3] = {0, 0, 0};
  const double ih = 1.0 / pp.hs;
  for (int t0 = 0; t0 < tcount; t0 += ntg) {
    const int ti = t0 + tid / tpt, sub = tid % tpt;
    const bool active = ti < tcount;
    V xi;
    if (active) xi = reinterpret_cast<const V*>(part)[tbeg + ti];
    T ph = T(0), gx = T(0), gy = T(0), gz = T(0);
    for (int s0 = 0; s0 < S; s0 += PP_TILE) {
      __syncthreads();
      for (int k = 0; k < nn; ++k) {
        const int lo = max(nb_off[k], s0), hi = min(nb_off[k + 1], s0 + PP_TILE);
        const T sx = nb_sh[k][0], sy = nb_sh[k][1], sz = nb_sh[k][2];
        for (int e = lo + tid; e < hi; e += PP_THREADS) {
          V r = reinterpret_cast<const V*>(part)[nb_beg[k] + (e - nb_off[k])];
          r.x += sx;
          r.y += sy;
          r.z += sz;
          src[e - s0] = r;
        }
      }
      __syncthreads();
      if (active) {
        const int len = min(PP_TILE, S - s0);
        for (int e = sub; e < len; e += tpt) {
          const V r = src[e];
          const T dx = xi.x - r.x, dy = xi.y - r.y, dz = xi.z - r.z;
          const T r2 = dx * dx + dy * dy + dz * dz;
          const T ri = r2 > T(0) ? rsq<T>(r2) : T(0);
          const T qr = r.w * ri;
          ph += qr;
          const T qr3 = qr * ri * ri;
          gx -= qr3 * dx;
          gy -= qr3 * dy;
          gz -= qr3 * dz;
        }
      }
    }
    for (int o = 1; o < tpt; o <<= 1) {
      ph += __shfl_xor_sync(0xffffffffu, ph, o);
      gx += __shfl_xor_sync(0xffffffffu, gx, o);
      gy += __shfl_xor_sync(0xffffffffu, gy, o);
      gz += __shfl_xor_sync(0xffffffffu, gz, o);
    }
    if (active && sub == 0) {
      const int64_t s = tbeg + ti;
      const V fr = reinterpret_cast<const V*>(far)[s];
      const double q = (double)xi.w;
      const double pt = pp.sign * ((double)fr.x + (double)ph * ih);
      const double g[3] = {pp.sign * ((double)fr.y + (double)gx * ih * ih),
                           pp.sign * ((double)fr.z + (double)gy * ih * ih),
                           pp.sign * ((double)fr.w + (double)gz * ih * ih)};
      const uint32_t o = vals[s];
      if (phi) phi[o] = (T)pt;
      if (force) {
        force[3 * (int64_t)o + 0] = (T)(-q * g[0]);
        force[3 * (int64_t)o + 1] = (T)(-q * g[1]);
        force[3 * (int64_t)o + 2] = (T)(-q * g[2]);
      }
      e_acc += 0.5 * q * pt;
      f_acc[0] -= q * g[0];
      f_acc[1] -= q * g[1];
      f_acc[2] -= q * g[2];
    }
  }
  // deterministic block reduction of the energy and net-force partials
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
    f_acc[0] += __shfl_xor_sync(0xffffffffu, f_acc[0], o);
    f_acc[1] += __shfl_xor_sync(0xffffffffu, f_acc[1], o);
    f_acc[2] += __shfl_xor_sync(0xffffffffu, f_acc[2], o);
  }
  if ((tid & 31) == 0) {
    red[tid >> 5][0] = e_acc;
    red[tid >> 5][1] = f_acc[0];
    red[tid >> 5][2] = f_acc[1];
    red[tid >> 5][3] = f_acc[2];
  }
  __syncthreads();
  if (tid < 4) {
    double v = 0;
    for (int w = 0; w < PP_THREADS / 32; ++w) v += red[w][tid];
    epart[cell * 4 + tid] = v;
  }
}

}  // namespace

cudaError_t launch_pp(bool fp64, const void* part, const uint32_t* vals, const int* cell_start, int64_t K,
                      const void* far, PPParams pp, void* phi, void* force, double* epart, cudaStream_t s, int* nl) {
  if (K <= 0) return cudaSuccess;
  if (fp64)
    pp_kernel<double><<<(unsigned)K, PP_THREADS, 0, s>>>((const double*)part, vals, cell_start, K, (const double*)far,
                                                         pp, (double*)phi, (double*)force, epart);
  else
    pp_kernel<float><<<(unsigned)K, PP_THREADS, 0, s>>>((const float*)part, vals, cell_start, K, (const float*)far, pp,
                                                        (float*)phi, (float*)force, epart);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace pmmm
