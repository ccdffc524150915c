// Two-level PMMM (Sec. 5, hierarchical treatment; Fig. refine).
//
// The plan's mesh is the fine mesh; every r^3 block of fine cells is one coarse
// cell, and the same cutoff c masks (2c+1)^3 blocks at both levels.
//   coarse level   M2M of the fine multipoles to the coarse centres (Eq. M2M,
//                  exact), then the one-level mesh stage on the coarse mesh;
//   fine level     for every coarse source cell S, the free-space M2L from its
//                  r^3 fine multipoles to the fine cells of the (2c+1)^3 coarse
//                  cells around S, as a convolution over a zero-padded block of
//                  m^3 fine cells (m >= 2(c+1) r: no wrap-around reaches the
//                  kept outputs): pruned forward DFT of the r^3 inputs, the
//                  per-wavevector M2L of the plan's other kernels against the
//                  spectra of the masked kernel S(d h_fine), pruned inverse DFT
//                  to the ((2c+1) r)^3 kept outputs;
//   fine locals    L2L of the coarse locals to the fine centres (Eq. L2L, exact
//                  for the polynomial) plus the sum of the kept outputs of the
//                  (2c+1)^3 coarse source cells around the fine cell's own.
// Device units: lengths in units of the fine cell size hs_f, M_l in units of
// hs^-l, L_l in units of hs^(l+1) of its level (hs_c = r hs_f), hence the
// powers of r in the M2M and L2L below.
#include "harmonics.cuh"
#include "internal.cuh"

namespace pmmm {

namespace {

// Complex coefficient X_l^m for any sign of m from the real storage of App. A.7
// (X_l^{-m} = (-1)^m conj X_l^m).
template <typename T, class F>
__device__ __forceinline__ cpx<T> cget(F&& X, int l, int m) {
  const int am = m < 0 ? -m : m;
  T re = X(sidx(l, am));
  T im = am > 0 ? X(sidx(l, -am)) : T(0);
  if (m < 0) {
    if (am & 1)
      re = -re;
    else
      im = -im;
  }
  return mk(re, im);
}

__device__ __forceinline__ void decode_lm(int j, int& l, int& m) {
  l = 0;
  while ((l + 1) * (l + 2) / 2 <= j) ++l;
  m = j - l * (l + 1) / 2;
}

// Real storage of R(v_a) for every child a = ax + r (ay + r az) of a coarse
// cell, v_a = (coarse centre - child centre) / hs_f = (r/2 - (a + 1/2)) cs.
template <typename T>
__global__ void rtab_kernel(int p, int r, double csx, double csy, double csz, T* __restrict__ out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= r * r * r) return;
  const int ax = a % r, ay = (a / r) % r, az = a / (r * r);
  const double x = (0.5 * r - (ax + 0.5)) * csx, y = (0.5 * r - (ay + 0.5)) * csy, z = (0.5 * r - (az + 0.5)) * csz;
  const int C = nterms(p);
  regular_real_rt<double>(p, x, y, z, [&](int c, double v) { out[(int64_t)a * C + c] = (T)v; });
}

// Coarse multipoles: M'_c(l,m) = r^-l sum_a sum_{lam,mu} M'_f(a)(l-lam, m-mu) R_lam^mu(v_a).
// One thread per (coarse cell, complex coefficient l, m >= 0).
template <typename T>
__global__ void __launch_bounds__(128) m2m_kernel(const T* __restrict__ Mf, int64_t Kf, int nfx, int nfy,
                                                  T* __restrict__ Mc, int64_t Kc, int ncx, int ncy,
                                                  const T* __restrict__ Rtab, int p, int r) {
  int l, m;
  decode_lm(blockIdx.y, l, m);
  const int64_t S = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (S >= Kc) return;
  const int Sx = (int)(S % ncx), Sy = (int)((S / ncx) % ncy), Sz = (int)(S / ((int64_t)ncx * ncy));
  const int C = nterms(p);
  cpx<T> acc = mk(T(0), T(0));
  for (int az = 0; az < r; ++az)
    for (int ay = 0; ay < r; ++ay)
      for (int ax = 0; ax < r; ++ax) {
        const int a = ax + r * (ay + r * az);
        const int64_t f = (int64_t)(Sx * r + ax) + (int64_t)nfx * ((Sy * r + ay) + (int64_t)nfy * (Sz * r + az));
        const T* R = Rtab + (int64_t)a * C;
        auto Xm = [&](int c) { return __ldg(Mf + (int64_t)c * Kf + f); };
        auto Xr = [&](int c) { return __ldg(R + c); };
        for (int lam = 0; lam <= l; ++lam) {
          const int ls = l - lam;
          for (int mu = -lam; mu <= lam; ++mu) {
            const int ms = m - mu;
            if (ms < -ls || ms > ls) continue;
            cmac(acc, cget<T>(Xm, ls, ms), cget<T>(Xr, lam, mu));
          }
        }
      }
  T sc = T(1);
  for (int i = 0; i < l; ++i) sc /= T(r);
  Mc[(int64_t)sidx(l, m) * Kc + S] = acc.x * sc;
  if (m > 0) Mc[(int64_t)sidx(l, -m) * Kc + S] = acc.y * sc;
}

// Coarse per-cell sums for the periodic corrections from the fine ones:
// u_c = (u_f + d_a) / r with d_a = (child centre - coarse centre) / hs_f.
__global__ void cellsum_kernel(const double* __restrict__ fs, int64_t Kf, int nfx, int nfy, double* __restrict__ cs,
                               int64_t Kc, int ncx, int ncy, int r, double csx, double csy, double csz) {
  const int64_t S = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (S >= Kc) return;
  const int Sx = (int)(S % ncx), Sy = (int)((S / ncx) % ncy), Sz = (int)(S / ((int64_t)ncx * ncy));
  double q = 0, dx = 0, dy = 0, dz = 0, s2 = 0;
  for (int az = 0; az < r; ++az)
    for (int ay = 0; ay < r; ++ay)
      for (int ax = 0; ax < r; ++ax) {
        const int64_t f = (int64_t)(Sx * r + ax) + (int64_t)nfx * ((Sy * r + ay) + (int64_t)nfy * (Sz * r + az));
        const double qf = fs[f], fx = fs[Kf + f], fy = fs[2 * Kf + f], fz = fs[3 * Kf + f], f2 = fs[4 * Kf + f];
        const double ex = (ax + 0.5 - 0.5 * r) * csx, ey = (ay + 0.5 - 0.5 * r) * csy, ez = (az + 0.5 - 0.5 * r) * csz;
        q += qf;
        dx += fx + qf * ex;
        dy += fy + qf * ey;
        dz += fz + qf * ez;
        s2 += f2 + 2.0 * (ex * fx + ey * fy + ez * fz) + (ex * ex + ey * ey + ez * ez) * qf;
      }
  const double ir = 1.0 / r;
  cs[S] = q;
  cs[Kc + S] = dx * ir;
  cs[2 * Kc + S] = dy * ir;
  cs[3 * Kc + S] = dz * ir;
  cs[4 * Kc + S] = s2 * ir * ir;
}

struct BlockGeo {
  int r, c, m, hx, W;   // refinement, cutoff, transform length, m/2+1, kept outputs per axis
  int nf[3], nc[3];
  int64_t Kf, Kc, Khh;  // fine cells, coarse cells, m*m*hx
  int C;
  int wavemajor;        // spectra [k][c][cell] (else [c][cell][k])
};

__device__ __forceinline__ int64_t spec_index(const BlockGeo& g, int64_t k, int ch, int64_t S) {
  return g.wavemajor ? ((k * g.C + ch) * g.Kc + S) : (((int64_t)ch * g.Kc + S) * g.Khh + k);
}

// Forward DFT (exp(-2 pi i k.t / m)) of the r^3 fine multipoles of NS coarse
// cells (one channel) zero-padded to m^3, half spectrum in x, pruned to the
// nonzero inputs: x pass over r^2 rows, y pass over hx * r columns, z pass to
// every wavevector.
template <typename T>
__global__ void __launch_bounds__(256) block_forward_kernel(const T* __restrict__ Mf, cpx<T>* __restrict__ spec,
                                                            const cpx<T>* __restrict__ tw_g, BlockGeo g, int NS) {
  extern __shared__ unsigned char smem_raw[];
  const int r = g.r, m = g.m, hx = g.hx, r3 = r * r * r;
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* A = tw + m;                              // [NS][hx][r(b)][r(e)]
  cpx<T>* B = A + (size_t)NS * hx * r * r;         // [NS][hx][m(ky)][r(e)]
  T* x = reinterpret_cast<T*>(B + (size_t)NS * hx * m * r);  // [NS][r^3]
  const int ch = blockIdx.y;
  const int64_t S0 = (int64_t)blockIdx.x * NS;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m; i += nt) tw[i] = tw_g[i];
  for (int i = tid; i < NS * r3; i += nt) {
    const int s = i / r3, a = i % r3;
    const int ax = a % r, ay = (a / r) % r, az = a / (r * r);
    const int64_t S = S0 + s;
    T v = T(0);
    if (S < g.Kc) {
      const int Sx = (int)(S % g.nc[0]), Sy = (int)((S / g.nc[0]) % g.nc[1]), Sz = (int)(S / ((int64_t)g.nc[0] * g.nc[1]));
      const int64_t f = (int64_t)(Sx * r + ax) + (int64_t)g.nf[0] * ((Sy * r + ay) + (int64_t)g.nf[1] * (Sz * r + az));
      v = Mf[(int64_t)ch * g.Kf + f];
    }
    x[i] = v;
  }
  __syncthreads();
  // x pass: A[s][kx][b][e] = sum_a x[s][a,b,e] w^(kx a)
  for (int i = tid; i < NS * hx * r * r; i += nt) {
    const int e = i % r, b = (i / r) % r, kx = (i / (r * r)) % hx, s = i / (r * r * hx);
    cpx<T> acc = mk(T(0), T(0));
    for (int a = 0; a < r; ++a) {
      const T v = x[s * r3 + a + r * (b + r * e)];
      const cpx<T> w = tw[(kx * a) % m];
      acc.x += v * w.x;
      acc.y += v * w.y;
    }
    A[i] = acc;
  }
  __syncthreads();
  // y pass: B[s][kx][ky][e] = sum_b A[s][kx][b][e] w^(ky b)
  for (int i = tid; i < NS * hx * m * r; i += nt) {
    const int e = i % r, ky = (i / r) % m, kx = (i / (r * m)) % hx, s = i / (r * m * hx);
    const cpx<T>* Ar = A + ((size_t)(s * hx + kx) * r) * r;
    cpx<T> acc = mk(T(0), T(0));
    for (int b = 0; b < r; ++b) cmac(acc, Ar[b * r + e], tw[(ky * b) % m]);
    B[i] = acc;
  }
  __syncthreads();
  // z pass to every wavevector k = (kz m + ky) hx + kx; consecutive threads take consecutive cells
  const int64_t nout = g.Khh * NS;
  for (int64_t i = tid; i < nout; i += nt) {
    const int s = (int)(i % NS);
    const int64_t k = i / NS;
    const int64_t S = S0 + s;
    if (S >= g.Kc) continue;
    const int kx = (int)(k % hx), ky = (int)((k / hx) % m), kz = (int)(k / ((int64_t)hx * m));
    const cpx<T>* Br = B + ((size_t)(s * hx + kx) * m + ky) * r;
    cpx<T> acc = mk(T(0), T(0));
    for (int e = 0; e < r; ++e) cmac(acc, Br[e], tw[(kz * e) % m]);
    spec[spec_index(g, k, ch, S)] = acc;
  }
}

// Inverse DFT (exp(+2 pi i k.t / m), unnormalised: the 1/m^3 is in the kernel
// spectra) of NS coarse cells' local spectra (one channel), evaluated only at
// the kept outputs t = u - c r, u in [0, W)^3, one x-frequency plane at a time:
// z pass, y pass, then the Hermitian-weighted real part accumulated over kx.
template <typename T>
__global__ void __launch_bounds__(256) block_inverse_kernel(const cpx<T>* __restrict__ spec, T* __restrict__ region,
                                                            const cpx<T>* __restrict__ tw_g, BlockGeo g, int NS) {
  extern __shared__ unsigned char smem_raw[];
  const int m = g.m, hx = g.hx, W = g.W, W3 = W * W * W, cr = g.c * g.r;
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* X = tw + m;                        // [NS][m(kz)][m(ky)]
  cpx<T>* Z = X + (size_t)NS * m * m;        // [NS][m(ky)][W(tz)]
  cpx<T>* Y = Z + (size_t)NS * m * W;        // [NS][W(ty)][W(tz)]
  T* out = reinterpret_cast<T*>(Y + (size_t)NS * W * W);  // [NS][W^3], (tz, ty, tx) with tx fastest
  const int ch = blockIdx.y;
  const int64_t S0 = (int64_t)blockIdx.x * NS;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m; i += nt) tw[i] = tw_g[i];
  for (int i = tid; i < NS * W3; i += nt) out[i] = T(0);
  auto tt = [&](int u) { return ((u - cr) % m + m) % m; };
  for (int kx = 0; kx < hx; ++kx) {
    __syncthreads();
    for (int i = tid; i < NS * m * m; i += nt) {
      const int s = i % NS, ky = (i / NS) % m, kz = i / (NS * m);
      const int64_t S = S0 + s;
      const int64_t k = ((int64_t)kz * m + ky) * hx + kx;
      X[((size_t)s * m + kz) * m + ky] = S < g.Kc ? spec[spec_index(g, k, ch, S)] : mk(T(0), T(0));
    }
    __syncthreads();
    // z pass: Z[s][ky][tz] = sum_kz X[s][kz][ky] conj(w)^(kz t(tz))
    for (int i = tid; i < NS * m * W; i += nt) {
      const int tz = i % W, ky = (i / W) % m, s = i / (W * m);
      const int t = tt(tz);
      cpx<T> acc = mk(T(0), T(0));
      for (int kz = 0; kz < m; ++kz) cmac(acc, X[((size_t)s * m + kz) * m + ky], conjg(tw[(kz * t) % m]));
      Z[i] = acc;
    }
    __syncthreads();
    // y pass: Y[s][ty][tz] = sum_ky Z[s][ky][tz] conj(w)^(ky t(ty))
    for (int i = tid; i < NS * W * W; i += nt) {
      const int tz = i % W, ty = (i / W) % W, s = i / (W * W);
      const int t = tt(ty);
      cpx<T> acc = mk(T(0), T(0));
      for (int ky = 0; ky < m; ++ky) cmac(acc, Z[((size_t)s * m + ky) * W + tz], conjg(tw[(ky * t) % m]));
      Y[i] = acc;
    }
    __syncthreads();
    // x pass (real output): out += w_kx Re(Y conj(w)^(kx t(tx))), w_kx = 1 at kx = 0 and m/2, else 2
    const T wk = (kx == 0 || 2 * kx == m) ? T(1) : T(2);
    for (int i = tid; i < NS * W3; i += nt) {
      const int tx = i % W, ty = (i / W) % W, tz = (i / (W * W)) % W, s = i / W3;
      const cpx<T> y = Y[((size_t)s * W + ty) * W + tz];
      const cpx<T> w = tw[(kx * tt(tx)) % m];
      out[i] += wk * (y.x * w.x + y.y * w.y);  // Re(y conj(w))
    }
  }
  __syncthreads();
  for (int i = tid; i < NS * W3; i += nt) {
    const int s = i / W3;
    const int64_t S = S0 + s;
    if (S < g.Kc) region[((int64_t)ch * g.Kc + S) * W3 + (i % W3)] = out[i];
  }
}

// Fine locals: L2L of the coarse locals (L'_f(l,m) = sum_{lam >= l} r^-(lam+1)
// L'_c(lam,mu) R_{lam-l}^{mu-m}(-v_a)) plus the kept block outputs of the
// (2c+1)^3 coarse source cells around the fine cell's coarse cell.  One thread
// per (fine cell, complex coefficient l, m >= 0).
template <typename T>
__global__ void __launch_bounds__(128) local_kernel(const T* __restrict__ Lc, const T* __restrict__ region,
                                                    const T* __restrict__ Rtab, T* __restrict__ Lf, BlockGeo g, int p,
                                                    int periodic) {
  int l, m;
  decode_lm(blockIdx.y, l, m);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.Kf) return;
  const int r = g.r, c = g.c, W = g.W, W3 = W * W * W;
  const int tx = (int)(t % g.nf[0]), ty = (int)((t / g.nf[0]) % g.nf[1]), tz = (int)(t / ((int64_t)g.nf[0] * g.nf[1]));
  const int T3[3] = {tx / r, ty / r, tz / r}, A3[3] = {tx % r, ty % r, tz % r};
  const int64_t Tc = (int64_t)T3[0] + (int64_t)g.nc[0] * (T3[1] + (int64_t)g.nc[1] * T3[2]);
  const int a = A3[0] + r * (A3[1] + r * A3[2]);
  const int C = g.C;
  const T* R = Rtab + (int64_t)a * C;
  auto Xl = [&](int ch) { return __ldg(Lc + (int64_t)ch * g.Kc + Tc); };
  auto Xr = [&](int ch) { return __ldg(R + ch); };
  cpx<T> acc = mk(T(0), T(0));
  T sl = T(1);
  for (int i = 0; i <= l; ++i) sl /= T(r);  // r^-(l+1)
  for (int lam = l; lam <= p; ++lam) {
    const int lr = lam - l;
    const T s = (lr & 1) ? -sl : sl;  // R(-v) = (-1)^(lam-l) R(v)
    for (int mu = -lam; mu <= lam; ++mu) {
      const int mr = mu - m;
      if (mr < -lr || mr > lr) continue;
      const cpx<T> L = cget<T>(Xl, lam, mu);
      cmac(acc, mk(s * L.x, s * L.y), cget<T>(Xr, lr, mr));
    }
    sl /= T(r);
  }
  const int64_t cre = (int64_t)sidx(l, m) * g.Kc, cim = (int64_t)sidx(l, -m) * g.Kc;
  for (int dz = -c; dz <= c; ++dz)
    for (int dy = -c; dy <= c; ++dy)
      for (int dx = -c; dx <= c; ++dx) {
        const int D[3] = {dx, dy, dz};
        int S3[3];
        bool ok = true;
        for (int ax = 0; ax < 3; ++ax) {
          S3[ax] = T3[ax] - D[ax];
          if (S3[ax] < 0 || S3[ax] >= g.nc[ax]) {
            ok = ok && periodic;
            S3[ax] += S3[ax] < 0 ? g.nc[ax] : -g.nc[ax];
          }
        }
        if (!ok) continue;
        const int64_t S = (int64_t)S3[0] + (int64_t)g.nc[0] * (S3[1] + (int64_t)g.nc[1] * S3[2]);
        const int u = (dx * r + A3[0] + c * r) + W * ((dy * r + A3[1] + c * r) + W * (dz * r + A3[2] + c * r));
        acc.x += region[(cre + S) * W3 + u];
        if (m > 0) acc.y += region[(cim + S) * W3 + u];
      }
  Lf[(int64_t)sidx(l, m) * g.Kf + t] = acc.x;
  if (m > 0) Lf[(int64_t)sidx(l, -m) * g.Kf + t] = acc.y;
}

template <typename T>
size_t forward_smem(const BlockGeo& g, int NS) {
  return sizeof(cpx<T>) * ((size_t)g.m + (size_t)NS * g.hx * g.r * g.r + (size_t)NS * g.hx * g.m * g.r) +
         sizeof(T) * (size_t)NS * g.r * g.r * g.r;
}
template <typename T>
size_t inverse_smem(const BlockGeo& g, int NS) {
  return sizeof(cpx<T>) * ((size_t)g.m + (size_t)NS * g.m * g.m + (size_t)NS * g.m * g.W + (size_t)NS * g.W * g.W) +
         sizeof(T) * (size_t)NS * g.W * g.W * g.W;
}

constexpr size_t kBlockSmem = 100 * 1024;  // two blocks per SM

template <typename T>
int pick_ns(const BlockGeo& g, bool inverse) {
  int ns = 16;
  while (ns > 1 && (inverse ? inverse_smem<T>(g, ns) : forward_smem<T>(g, ns)) > kBlockSmem) ns /= 2;
  return ns;
}

BlockGeo make_geo(const HierGeo& h, int C) {
  BlockGeo g;
  g.r = h.r;
  g.c = h.c;
  g.m = h.m;
  g.hx = h.m / 2 + 1;
  g.W = (2 * h.c + 1) * h.r;
  for (int a = 0; a < 3; ++a) {
    g.nf[a] = h.nf[a];
    g.nc[a] = h.nc[a];
  }
  g.Kf = (int64_t)h.nf[0] * h.nf[1] * h.nf[2];
  g.Kc = (int64_t)h.nc[0] * h.nc[1] * h.nc[2];
  g.Khh = (int64_t)h.m * h.m * g.hx;
  g.C = C;
  g.wavemajor = h.wavemajor;
  return g;
}

template <typename T>
cudaError_t forward_run(const HierGeo& h, int C, const void* Mf, void* spec, const void* tw, cudaStream_t s) {
  const BlockGeo g = make_geo(h, C);
  const int NS = pick_ns<T>(g, false);
  const size_t smem = forward_smem<T>(g, NS);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(block_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.Kc + NS - 1) / NS), (unsigned)C);
  block_forward_kernel<T><<<grid, 256, smem, s>>>((const T*)Mf, (cpx<T>*)spec, (const cpx<T>*)tw, g, NS);
  return cudaGetLastError();
}

template <typename T>
cudaError_t inverse_run(const HierGeo& h, int C, const void* spec, void* region, const void* tw, cudaStream_t s) {
  const BlockGeo g = make_geo(h, C);
  const int NS = pick_ns<T>(g, true);
  const size_t smem = inverse_smem<T>(g, NS);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(block_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.Kc + NS - 1) / NS), (unsigned)C);
  block_inverse_kernel<T><<<grid, 256, smem, s>>>((const cpx<T>*)spec, (T*)region, (const cpx<T>*)tw, g, NS);
  return cudaGetLastError();
}

}  // namespace

bool hier_block_fits(const HierGeo& h, bool fp64, int C) {
  const BlockGeo g = make_geo(h, C);
  if (fp64)
    return forward_smem<double>(g, 1) <= 200 * 1024 && inverse_smem<double>(g, 1) <= 200 * 1024;
  return forward_smem<float>(g, 1) <= 200 * 1024 && inverse_smem<float>(g, 1) <= 200 * 1024;
}

cudaError_t launch_hier_rtab(const HierGeo& h, int p, bool fp64, const double* cs, void* rtab, cudaStream_t s) {
  const int n = h.r * h.r * h.r;
  if (fp64)
    rtab_kernel<double><<<(n + 63) / 64, 64, 0, s>>>(p, h.r, cs[0], cs[1], cs[2], (double*)rtab);
  else
    rtab_kernel<float><<<(n + 63) / 64, 64, 0, s>>>(p, h.r, cs[0], cs[1], cs[2], (float*)rtab);
  return cudaGetLastError();
}

cudaError_t launch_hier_m2m(const HierGeo& h, int p, bool fp64, const void* Mf, void* Mc, const void* rtab,
                            cudaStream_t s, int* nl) {
  const int64_t Kf = (int64_t)h.nf[0] * h.nf[1] * h.nf[2], Kc = (int64_t)h.nc[0] * h.nc[1] * h.nc[2];
  dim3 grid((unsigned)((Kc + 127) / 128), (unsigned)((p + 1) * (p + 2) / 2));
  if (fp64)
    m2m_kernel<double><<<grid, 128, 0, s>>>((const double*)Mf, Kf, h.nf[0], h.nf[1], (double*)Mc, Kc, h.nc[0],
                                            h.nc[1], (const double*)rtab, p, h.r);
  else
    m2m_kernel<float><<<grid, 128, 0, s>>>((const float*)Mf, Kf, h.nf[0], h.nf[1], (float*)Mc, Kc, h.nc[0], h.nc[1],
                                           (const float*)rtab, p, h.r);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_hier_cellsum(const HierGeo& h, const double* fine, double* coarse, const double* cs,
                                cudaStream_t s, int* nl) {
  const int64_t Kf = (int64_t)h.nf[0] * h.nf[1] * h.nf[2], Kc = (int64_t)h.nc[0] * h.nc[1] * h.nc[2];
  cellsum_kernel<<<(unsigned)((Kc + 127) / 128), 128, 0, s>>>(fine, Kf, h.nf[0], h.nf[1], coarse, Kc, h.nc[0],
                                                               h.nc[1], h.r, cs[0], cs[1], cs[2]);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_hier_forward(const HierGeo& h, int C, bool fp64, const void* Mf, void* spec, const void* tw,
                                cudaStream_t s, int* nl) {
  ++*nl;
  return fp64 ? forward_run<double>(h, C, Mf, spec, tw, s) : forward_run<float>(h, C, Mf, spec, tw, s);
}

cudaError_t launch_hier_inverse(const HierGeo& h, int C, bool fp64, const void* spec, void* region, const void* tw,
                                cudaStream_t s, int* nl) {
  ++*nl;
  return fp64 ? inverse_run<double>(h, C, spec, region, tw, s) : inverse_run<float>(h, C, spec, region, tw, s);
}

cudaError_t launch_hier_local(const HierGeo& h, int p, bool fp64, const void* Lc, const void* region,
                              const void* rtab, void* Lf, int periodic, cudaStream_t s, int* nl) {
  const BlockGeo g = make_geo(h, nterms(p));
  dim3 grid((unsigned)((g.Kf + 127) / 128), (unsigned)((p + 1) * (p + 2) / 2));
  if (fp64)
    local_kernel<double><<<grid, 128, 0, s>>>((const double*)Lc, (const double*)region, (const double*)rtab,
                                              (double*)Lf, g, p, periodic);
  else
    local_kernel<float><<<grid, 128, 0, s>>>((const float*)Lc, (const float*)region, (const float*)rtab, (float*)Lf,
                                             g, p, periodic);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace pmmm
