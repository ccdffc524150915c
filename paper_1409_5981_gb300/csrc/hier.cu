// Two-level PMMM (Sec. 5, hierarchical treatment; Fig. refine).
//
// The plan's mesh is the fine mesh; every r^3 block of fine cells is one coarse
// cell, and the same cutoff c masks (2c+1)^3 blocks at both levels.
//   coarse level   multipoles about the coarse centres straight from the
//                  particles (Eq. P2M, p2m_l2p.cu), then the one-level mesh stage
//                  on the coarse mesh;
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
// powers of r in the L2L below.
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

// The fine local (l, m) from one coarse local: sum_{lam >= l} r^-(lam+1) L'_c(lam,mu) R_{lam-l}^{mu-m}(-v_a)
// (Eq. L2L, R(-v) = (-1)^n R_n(v)).
template <typename T, class FL, class FR>
__device__ __forceinline__ void l2l_term(int l, int m, int p, int r, FL&& Xl, FR&& Xr, cpx<T>& acc) {
  T sl = T(1);
  for (int i = 0; i <= l; ++i) sl /= T(r);  // r^-(l+1)
  for (int lam = l; lam <= p; ++lam) {
    const int lr = lam - l;
    const T s = (lr & 1) ? -sl : sl;
    for (int mu = -lam; mu <= lam; ++mu) {
      const int mr = mu - m;
      if (mr < -lr || mr > lr) continue;
      const cpx<T> L = cget<T>(Xl, lam, mu);
      cmac(acc, mk(s * L.x, s * L.y), cget<T>(Xr, lr, mr));
    }
    sl /= T(r);
  }
}

// Real C x C matrices of the L2L to the r^3 children on the real storage,
// Um[a][co][ci], built by applying the complex translation to unit inputs.  One
// thread per (child a, input channel ci, output coefficient l, m >= 0).
template <typename T>
__global__ void translation_matrix_kernel(int p, int r, const T* __restrict__ Rtab, T* __restrict__ Um) {
  const int C = nterms(p), nj = (p + 1) * (p + 2) / 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)r * r * r * C * nj) return;
  const int j = (int)(idx % nj), ci = (int)((idx / nj) % C), a = (int)(idx / ((int64_t)nj * C));
  int l, m;
  decode_lm(j, l, m);
  const T* R = Rtab + (int64_t)a * C;
  cpx<T> u = mk(T(0), T(0));
  l2l_term<T>(l, m, p, r, [&](int c) { return c == ci ? T(1) : T(0); }, [&](int c) { return R[c]; }, u);
  const int64_t base = (int64_t)a * C * C;
  Um[base + (int64_t)sidx(l, m) * C + ci] = u.x;
  if (m > 0) Um[base + (int64_t)sidx(l, -m) * C + ci] = u.y;
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
// every wavevector.  Shared arrays keep the cell index fastest, so that the
// threads of a warp (consecutive cells) touch consecutive words.
template <typename T>
__global__ void __launch_bounds__(256) block_forward_kernel(const T* __restrict__ Mf, cpx<T>* __restrict__ spec,
                                                            const cpx<T>* __restrict__ tw_g, BlockGeo g, int NS) {
  extern __shared__ unsigned char smem_raw[];
  const int r = g.r, m = g.m, mm = g.m - 1, hx = g.hx, r3 = r * r * r;  // m is a power of two
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* A = tw + m;                              // [hx][r(b)][r(e)][NS]
  cpx<T>* B = A + (size_t)NS * hx * r * r;         // [hx][m(ky)][r(e)][NS]
  T* x = reinterpret_cast<T*>(B + (size_t)NS * hx * m * r);  // [r^3][NS]
  const int ch = blockIdx.y;
  const int64_t S0 = (int64_t)blockIdx.x * NS;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m; i += nt) tw[i] = tw_g[i];
  for (int i = tid; i < NS * r3; i += nt) {
    const int a = i / NS, s = i % NS;
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
  // x pass: A[kx][b][e][s] = sum_a x[a,b,e][s] w^(kx a)
  for (int i = tid; i < NS * hx * r * r; i += nt) {
    const int s = i % NS, be = i / NS, e = be % r, b = (be / r) % r, kx = be / (r * r);
    cpx<T> acc = mk(T(0), T(0));
    for (int a = 0; a < r; ++a) {
      const T v = x[(a + r * (b + r * e)) * NS + s];
      const cpx<T> w = tw[(kx * a) & mm];
      acc.x += v * w.x;
      acc.y += v * w.y;
    }
    A[i] = acc;
  }
  __syncthreads();
  // y pass: B[kx][ky][e][s] = sum_b A[kx][b][e][s] w^(ky b)
  for (int i = tid; i < NS * hx * m * r; i += nt) {
    const int s = i % NS, q = i / NS, e = q % r, ky = (q / r) & mm, kx = q / (r * m);
    const cpx<T>* Ar = A + ((size_t)kx * r * r + e) * NS + s;
    cpx<T> acc = mk(T(0), T(0));
    for (int b = 0; b < r; ++b) cmac(acc, Ar[(size_t)b * r * NS], tw[(ky * b) & mm]);
    B[i] = acc;
  }
  __syncthreads();
  // z pass to every wavevector k = (kz m + ky) hx + kx; consecutive threads take consecutive cells
  const int nout = (int)g.Khh * NS;
  for (int i = tid; i < nout; i += nt) {
    const int s = i % NS, k = i / NS;
    const int64_t S = S0 + s;
    if (S >= g.Kc) continue;
    const int kx = k % hx, kyz = k / hx, ky = kyz & mm, kz = kyz / m;
    const cpx<T>* Br = B + ((size_t)(kx * m + ky) * r) * NS + s;
    cpx<T> acc = mk(T(0), T(0));
    for (int e = 0; e < r; ++e) cmac(acc, Br[(size_t)e * NS], tw[(kz * e) & mm]);
    spec[spec_index(g, k, ch, S)] = acc;
  }
}

constexpr int fwd_ns(int M, int R, int esz) {
  // cells per block of the compile-time forward: the largest power of two <= 16 whose
  // shared arrays (twiddles, x-pass, y-pass, inputs) stay within 100 KB
  int ns = 16;
  while (ns > 1 && (size_t)(2 * esz) * (M + ns * (M / 2 + 1) * R * R + ns * (M / 2 + 1) * M * R) +
                           (size_t)esz * ns * R * R * R > 100 * 1024)
    ns /= 2;
  return ns;
}

// The forward of block_forward_kernel with the transform length M, the
// refinement R and the cells per block NS known at compile time (all index
// arithmetic by constants).
template <typename T, int M, int R>
__global__ void __launch_bounds__(256) block_forward_ct_kernel(const T* __restrict__ Mf, cpx<T>* __restrict__ spec,
                                                               const cpx<T>* __restrict__ tw_g, BlockGeo g) {
  constexpr int NS = fwd_ns(M, R, sizeof(T)), HX = M / 2 + 1, R3 = R * R * R, KHH = M * M * HX;
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* tw = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* A = tw + M;                          // [HX][R(b)][R(e)][NS]
  cpx<T>* B = A + NS * HX * R * R;             // [HX][M(ky)][R(e)][NS]
  T* x = reinterpret_cast<T*>(B + NS * HX * M * R);  // [R^3][NS]
  const int ch = blockIdx.y;
  const int64_t S0 = (int64_t)blockIdx.x * NS;
  const int tid = threadIdx.x;
  for (int i = tid; i < M; i += 256) tw[i] = tw_g[i];
  for (int i = tid; i < NS * R3; i += 256) {
    const int a = i / NS, s = i % NS;
    const int ax = a % R, ay = (a / R) % R, az = a / (R * R);
    const int64_t S = S0 + s;
    T v = T(0);
    if (S < g.Kc) {
      const int Sx = (int)(S % g.nc[0]), Sy = (int)((S / g.nc[0]) % g.nc[1]), Sz = (int)(S / ((int64_t)g.nc[0] * g.nc[1]));
      const int64_t f = (int64_t)(Sx * R + ax) + (int64_t)g.nf[0] * ((Sy * R + ay) + (int64_t)g.nf[1] * (Sz * R + az));
      v = Mf[(int64_t)ch * g.Kf + f];
    }
    x[i] = v;
  }
  __syncthreads();
  for (int i = tid; i < NS * HX * R * R; i += 256) {
    const int s = i % NS, be = i / NS, e = be % R, b = (be / R) % R, kx = be / (R * R);
    cpx<T> acc = mk(T(0), T(0));
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const T v = x[(a + R * (b + R * e)) * NS + s];
      const cpx<T> w = tw[(kx * a) & (M - 1)];
      acc.x += v * w.x;
      acc.y += v * w.y;
    }
    A[i] = acc;
  }
  __syncthreads();
  for (int i = tid; i < NS * HX * M * R; i += 256) {
    const int s = i % NS, q = i / NS, e = q % R, ky = (q / R) % M, kx = q / (R * M);
    const cpx<T>* Ar = A + (kx * R * R + e) * NS + s;
    cpx<T> acc = mk(T(0), T(0));
#pragma unroll
    for (int b = 0; b < R; ++b) cmac(acc, Ar[b * R * NS], tw[(ky * b) & (M - 1)]);
    B[i] = acc;
  }
  __syncthreads();
  const int64_t ncell = g.Kc - S0 < NS ? g.Kc - S0 : NS;
  const int64_t rowstride = g.wavemajor ? (int64_t)g.C * g.Kc : 1;
  cpx<T>* out = g.wavemajor ? spec + (int64_t)ch * g.Kc + S0 : spec + ((int64_t)ch * g.Kc + S0) * KHH;
  for (int i = tid; i < KHH * NS; i += 256) {
    const int s = i % NS, k = i / NS;
    if (s >= ncell) continue;
    const int kx = k % HX, kyz = k / HX, ky = kyz % M, kz = kyz / M;
    const cpx<T>* Br = B + ((kx * M + ky) * R) * NS + s;
    cpx<T> acc = mk(T(0), T(0));
#pragma unroll
    for (int e = 0; e < R; ++e) cmac(acc, Br[e * NS], tw[(kz * e) & (M - 1)]);
    if (g.wavemajor)
      out[k * rowstride + s] = acc;
    else
      out[(int64_t)s * KHH + k] = acc;
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
  const int m = g.m, mm = g.m - 1, hx = g.hx, W = g.W, W3 = W * W * W, cr = g.c * g.r;  // m a power of two
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
  auto tt = [&](int u) { return (u - cr) & mm; };
  for (int kx = 0; kx < hx; ++kx) {
    __syncthreads();
    for (int i = tid; i < NS * m * m; i += nt) {
      const int s = i % NS, ky = (i / NS) & mm, kz = i / (NS * m);
      const int64_t S = S0 + s;
      const int k = (kz * m + ky) * hx + kx;
      X[((size_t)s * m + kz) * m + ky] = S < g.Kc ? spec[spec_index(g, k, ch, S)] : mk(T(0), T(0));
    }
    __syncthreads();
    // z pass: Z[s][ky][tz] = sum_kz X[s][kz][ky] conj(w)^(kz t(tz))
    for (int i = tid; i < NS * m * W; i += nt) {
      const int tz = i % W, ky = (i / W) & mm, s = i / (W * m);
      const int t = tt(tz);
      cpx<T> acc = mk(T(0), T(0));
      for (int kz = 0; kz < m; ++kz) cmac(acc, X[((size_t)s * m + kz) * m + ky], conjg(tw[(kz * t) & mm]));
      Z[i] = acc;
    }
    __syncthreads();
    // y pass: Y[s][ty][tz] = sum_ky Z[s][ky][tz] conj(w)^(ky t(ty))
    for (int i = tid; i < NS * W * W; i += nt) {
      const int tz = i % W, ty = (i / W) % W, s = i / (W * W);
      const int t = tt(ty);
      cpx<T> acc = mk(T(0), T(0));
      for (int ky = 0; ky < m; ++ky) cmac(acc, Z[((size_t)s * m + ky) * W + tz], conjg(tw[(ky * t) & mm]));
      Y[i] = acc;
    }
    __syncthreads();
    // x pass (real output): out += w_kx Re(Y conj(w)^(kx t(tx))), w_kx = 1 at kx = 0 and m/2, else 2
    const T wk = (kx == 0 || 2 * kx == m) ? T(1) : T(2);
    for (int i = tid; i < NS * W3; i += nt) {
      const int tx = i % W, ty = (i / W) % W, tz = (i / (W * W)) % W, s = i / W3;
      const cpx<T> y = Y[((size_t)s * W + ty) * W + tz];
      const cpx<T> w = tw[(kx * tt(tx)) & mm];
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

// The same inverse with one thread per kept (ty, tz) column of each of NS cells:
// its W outputs along x stay in registers over the x-frequency planes, its y
// pass is private, and the inverse twiddles of the kept positions come from a
// table E[k][u] = exp(+2 pi i k t(u) / m) (t(u) = u - c r), so that a plane costs
// one shared-memory round trip (the z pass).
template <typename T, int W>
__global__ void __launch_bounds__(1024) block_inverse_reg_kernel(const cpx<T>* __restrict__ spec,
                                                                 T* __restrict__ region,
                                                                 const cpx<T>* __restrict__ tw_g, BlockGeo g, int NS) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int W2 = W * W, W3 = W * W * W;
  const int m = g.m, mm = g.m - 1, hx = g.hx, cr = g.c * g.r;
  cpx<T>* E = reinterpret_cast<cpx<T>*>(smem_raw);  // [m][W]
  cpx<T>* X = E + (size_t)m * W;                     // [NS][m(kz)][m(ky)]
  cpx<T>* Z = X + (size_t)NS * m * m;                // [NS][m(ky)][W(tz)]
  const int ch = blockIdx.y;
  const int64_t S0 = (int64_t)blockIdx.x * NS;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < m * W; i += nt) E[i] = conjg(tw_g[((i / W) * (i % W - cr)) & mm]);
  const bool own = tid < NS * W2;
  const int s = tid / W2, ty = (tid % W2) % W, tz = (tid % W2) / W;
  T out[W];
#pragma unroll
  for (int u = 0; u < W; ++u) out[u] = T(0);
  for (int kx = 0; kx < hx; ++kx) {
    __syncthreads();
    for (int i = tid; i < NS * m * m; i += nt) {
      const int si = i % NS, ky = (i / NS) & mm, kz = i / (NS * m);
      const int64_t S = S0 + si;
      const int k = (kz * m + ky) * hx + kx;
      X[((size_t)si * m + kz) * m + ky] = S < g.Kc ? spec[spec_index(g, k, ch, S)] : mk(T(0), T(0));
    }
    __syncthreads();
    // z pass: Z[s][ky][tz] = sum_kz X[s][kz][ky] E[kz][tz]
    for (int i = tid; i < NS * m * W; i += nt) {
      const int u = i % W, ky = (i / W) & mm, si = i / (W * m);
      const cpx<T>* xc = X + (size_t)si * m * m + ky;
      cpx<T> acc = mk(T(0), T(0));
      for (int kz = 0; kz < m; ++kz) cmac(acc, xc[kz * m], E[kz * W + u]);
      Z[i] = acc;
    }
    __syncthreads();
    if (own) {
      // y pass of this thread's (ty, tz): y = sum_ky Z[s][ky][tz] E[ky][ty]
      const cpx<T>* zc = Z + (size_t)s * m * W + tz;
      cpx<T> y = mk(T(0), T(0));
      for (int ky = 0; ky < m; ++ky) cmac(y, zc[ky * W], E[ky * W + ty]);
      // x pass (real output): out[tx] += w_kx Re(y E[kx][tx]), w_kx = 1 at kx = 0 and m/2, else 2
      const T wk = (kx == 0 || 2 * kx == m) ? T(1) : T(2);
      const T yr = wk * y.x, yi = wk * y.y;
      const cpx<T>* ex = E + kx * W;
#pragma unroll
      for (int u = 0; u < W; ++u) out[u] += yr * ex[u].x - yi * ex[u].y;
    }
  }
  const int64_t S = S0 + s;
  if (own && S < g.Kc) {
    T* o = region + ((int64_t)ch * g.Kc + S) * W3 + ((size_t)tz * W + ty) * W;
#pragma unroll
    for (int u = 0; u < W; ++u) o[u] = out[u];
  }
}

constexpr int bitrev(int v, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((v >> b) & 1) << (bits - 1 - b);
  return r;
}
constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// In-register radix-2 inverse DFT of length M (exp(+2 pi i j k / M), unnormalised):
// v holds the input in bit-reversed order and returns the output in natural order;
// wp[j] = exp(+2 pi i j / M).
template <typename T, int M>
__device__ __forceinline__ void ifft_reg(cpx<T>* v, const cpx<T>* wp) {
#pragma unroll
  for (int len = 2; len <= M; len <<= 1) {
    const int half = len / 2, step = M / len;
#pragma unroll
    for (int i = 0; i < M; i += len)
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const cpx<T> a = v[i + j], b = v[i + j + half] * wp[j * step];
        v[i + j] = a + b;
        v[i + j + half] = a - b;
      }
  }
}

// Inverse of the block convolution by FFTs along z and y (M-point, in
// registers, one thread per column) and a direct Hermitian-weighted real
// transform along x, for the kept outputs only (W per axis at t = u - CR).  The
// block's whole half spectrum sits in shared memory as F[kz][ky][kx][cell]
// (cell fastest, the order of the wavevector-major spectra), the z and y passes
// overwrite their own columns in place with the W kept values.
constexpr int inv_ns(int M, int esz) {
  // cells per block of the FFT inverse: the largest power of two <= 8 whose half
  // spectra stay within 100 KB (one cell when a single one needs more)
  int ns = 8;
  while (ns > 1 && (size_t)(2 * esz) * (M + ns * M * M * (M / 2 + 1)) > 100 * 1024) ns /= 2;
  return ns;
}

template <typename T, int M, int W, int CR>
__global__ void __launch_bounds__(256) block_inverse_fft_kernel(const cpx<T>* __restrict__ spec,
                                                                T* __restrict__ region,
                                                                const cpx<T>* __restrict__ tw_g, BlockGeo g) {
  extern __shared__ unsigned char smem_raw[];
  constexpr int NS = inv_ns(M, sizeof(T));
  constexpr int HX = M / 2 + 1, LB = ilog2(M), W3 = W * W * W;
  cpx<T>* wp = reinterpret_cast<cpx<T>*>(smem_raw);  // exp(+2 pi i j / M)
  cpx<T>* F = wp + M;                                 // [M(kz)][M(ky)][HX(kx)][NS]
  const int ch = blockIdx.y;
  const int64_t S0 = (int64_t)blockIdx.x * NS;
  const int tid = threadIdx.x, nt = blockDim.x;
  constexpr int NCOL = NS * HX * M;  // columns (ky, kx, cell) of the z pass
  for (int i = tid; i < M; i += nt) wp[i] = conjg(tw_g[i]);
  {
    const int64_t ncell = g.Kc - S0 < NS ? g.Kc - S0 : NS;
    const int64_t rowstride = g.wavemajor ? (int64_t)g.C * g.Kc : 1;
    const cpx<T>* in = g.wavemajor ? spec + (int64_t)ch * g.Kc + S0 : spec + ((int64_t)ch * g.Kc + S0) * (M * M * HX);
    for (int i = tid; i < M * NCOL; i += nt) {
      const int si = i % NS, k = i / NS;  // k = (kz M + ky) HX + kx
      F[i] = si < ncell ? (g.wavemajor ? in[k * rowstride + si] : in[(int64_t)si * (M * M * HX) + k])
                        : mk(T(0), T(0));
    }
  }
  __syncthreads();
  // z pass: column (ky, kx, cell) -> kept rows uz < W
  for (int col = tid; col < NCOL; col += nt) {
    cpx<T> v[M];
#pragma unroll
    for (int j = 0; j < M; ++j) v[j] = F[bitrev(j, LB) * NCOL + col];
    ifft_reg<T, M>(v, wp);
#pragma unroll
    for (int u = 0; u < W; ++u) F[u * NCOL + col] = v[(u - CR) & (M - 1)];
  }
  __syncthreads();
  // y pass: column (uz, kx, cell) over ky -> kept rows uy < W
  constexpr int NY = NS * HX * W;
  for (int yc = tid; yc < NY; yc += nt) {
    const int kxs = yc % (HX * NS), uz = yc / (HX * NS);
    cpx<T>* base = F + (size_t)uz * NCOL + kxs;
    cpx<T> v[M];
#pragma unroll
    for (int j = 0; j < M; ++j) v[j] = base[bitrev(j, LB) * HX * NS];
    ifft_reg<T, M>(v, wp);
#pragma unroll
    for (int u = 0; u < W; ++u) base[u * HX * NS] = v[(u - CR) & (M - 1)];
  }
  __syncthreads();
  // x pass (real output): row (uz, uy, cell): out[ux] = sum_kx w_kx Re(Y[kx] exp(+2 pi i kx t(ux) / M))
  constexpr int NX = NS * W * W;
  for (int xr = tid; xr < NX; xr += nt) {
    const int si = xr % NS, uy = (xr / NS) % W, uz = xr / (NS * W);
    const cpx<T>* Y = F + (size_t)uz * NCOL + (size_t)uy * HX * NS + si;
    T out[W];
#pragma unroll
    for (int u = 0; u < W; ++u) out[u] = T(0);
#pragma unroll
    for (int kx = 0; kx < HX; ++kx) {
      const T wk = (kx == 0 || 2 * kx == M) ? T(1) : T(2);
      const cpx<T> y = Y[kx * NS];
      const T yr = wk * y.x, yi = wk * y.y;
#pragma unroll
      for (int u = 0; u < W; ++u) {
        const cpx<T> w = wp[(kx * ((u - CR) & (M - 1))) & (M - 1)];
        out[u] += yr * w.x - yi * w.y;
      }
    }
    const int64_t S = S0 + si;
    if (S < g.Kc) {
      T* o = region + ((int64_t)ch * g.Kc + S) * W3 + ((size_t)uz * W + uy) * W;
#pragma unroll
      for (int u = 0; u < W; ++u) o[u] = out[u];
    }
  }
}

// Sum of the kept block outputs of the (2c+1)^3 coarse source cells around the
// coarse cell T3 of fine cell (A3 within it), for the real channel ch.
template <typename T>
__device__ __forceinline__ T gather_kept(const T* __restrict__ region, const BlockGeo& g, int ch, const int* T3,
                                         const int* A3, int periodic) {
  const int r = g.r, c = g.c, W = g.W, W3 = W * W * W;
  const int64_t cb = (int64_t)ch * g.Kc;
  T acc = T(0);
  for (int dz = -c; dz <= c; ++dz)
    for (int dy = -c; dy <= c; ++dy)
      for (int dx = -c; dx <= c; ++dx) {
        const int D[3] = {dx, dy, dz};
        int S3[3];
        bool ok = true;
#pragma unroll
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
        acc += region[(cb + S) * W3 + u];
      }
  return acc;
}

// Fine locals through the child matrices: L'_f[co][t] = sum_ci Um[a][co][ci] L'_c[ci][T]
// + the kept block outputs.  One thread per (fine cell, real output channel).
template <typename T>
__global__ void __launch_bounds__(128) local_matrix_kernel(const T* __restrict__ Lc, const T* __restrict__ region,
                                                           const T* __restrict__ Um, T* __restrict__ Lf, BlockGeo g,
                                                           int periodic) {
  const int co = blockIdx.y;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.Kf) return;
  const int r = g.r, C = g.C;
  const int tx = (int)(t % g.nf[0]), ty = (int)((t / g.nf[0]) % g.nf[1]), tz = (int)(t / ((int64_t)g.nf[0] * g.nf[1]));
  const int T3[3] = {tx / r, ty / r, tz / r}, A3[3] = {tx % r, ty % r, tz % r};
  const int64_t Tc = (int64_t)T3[0] + (int64_t)g.nc[0] * (T3[1] + (int64_t)g.nc[1] * T3[2]);
  const int a = A3[0] + r * (A3[1] + r * A3[2]);
  const T* row = Um + ((int64_t)a * C + co) * C;
  T acc = T(0);
  for (int ci = 0; ci < C; ++ci) acc += __ldg(row + ci) * __ldg(Lc + (int64_t)ci * g.Kc + Tc);
  acc += gather_kept<T>(region, g, co, T3, A3, periodic);
  Lf[(int64_t)co * g.Kf + t] = acc;
}

// Fine locals straight from the complex formula (child matrices too large): L2L
// of the coarse locals plus the kept block outputs.  One thread per (fine cell,
// complex coefficient l, m >= 0).
template <typename T>
__global__ void __launch_bounds__(128) local_kernel(const T* __restrict__ Lc, const T* __restrict__ region,
                                                    const T* __restrict__ Rtab, T* __restrict__ Lf, BlockGeo g, int p,
                                                    int periodic) {
  int l, m;
  decode_lm(blockIdx.y, l, m);
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.Kf) return;
  const int r = g.r;
  const int tx = (int)(t % g.nf[0]), ty = (int)((t / g.nf[0]) % g.nf[1]), tz = (int)(t / ((int64_t)g.nf[0] * g.nf[1]));
  const int T3[3] = {tx / r, ty / r, tz / r}, A3[3] = {tx % r, ty % r, tz % r};
  const int64_t Tc = (int64_t)T3[0] + (int64_t)g.nc[0] * (T3[1] + (int64_t)g.nc[1] * T3[2]);
  const int a = A3[0] + r * (A3[1] + r * A3[2]);
  const T* R = Rtab + (int64_t)a * g.C;
  cpx<T> acc = mk(T(0), T(0));
  l2l_term<T>(l, m, p, r, [&](int ch) { return __ldg(Lc + (int64_t)ch * g.Kc + Tc); },
              [&](int ch) { return __ldg(R + ch); }, acc);
  acc.x += gather_kept<T>(region, g, sidx(l, m), T3, A3, periodic);
  Lf[(int64_t)sidx(l, m) * g.Kf + t] = acc.x;
  if (m > 0) Lf[(int64_t)sidx(l, -m) * g.Kf + t] = acc.y + gather_kept<T>(region, g, sidx(l, -m), T3, A3, periodic);
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

template <typename T, int M, int R>
cudaError_t forward_ct_run(const BlockGeo& g, const void* Mf, void* spec, const void* tw, cudaStream_t s) {
  constexpr int NS = fwd_ns(M, R, sizeof(T)), HX = M / 2 + 1;
  const size_t smem = sizeof(cpx<T>) * (M + NS * HX * R * R + NS * HX * M * R) + sizeof(T) * NS * R * R * R;
  if (smem > 200 * 1024) return cudaErrorNotSupported;
  cudaError_t e =
      cudaFuncSetAttribute(block_forward_ct_kernel<T, M, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.Kc + NS - 1) / NS), (unsigned)g.C);
  block_forward_ct_kernel<T, M, R><<<grid, 256, smem, s>>>((const T*)Mf, (cpx<T>*)spec, (const cpx<T>*)tw, g);
  return cudaGetLastError();
}

template <typename T>
cudaError_t forward_run(const HierGeo& h, int C, const void* Mf, void* spec, const void* tw, cudaStream_t s) {
  const BlockGeo g = make_geo(h, C);
  cudaError_t ect = cudaErrorNotSupported;
  if (g.m == 8 && g.r == 2) ect = forward_ct_run<T, 8, 2>(g, Mf, spec, tw, s);
  if (g.m == 16 && g.r == 4) ect = forward_ct_run<T, 16, 4>(g, Mf, spec, tw, s);
  if (g.m == 16 && g.r == 2) ect = forward_ct_run<T, 16, 2>(g, Mf, spec, tw, s);
  if (g.m == 32 && g.r == 8) ect = forward_ct_run<T, 32, 8>(g, Mf, spec, tw, s);
  if (g.m == 32 && g.r == 4) ect = forward_ct_run<T, 32, 4>(g, Mf, spec, tw, s);
  if (ect != cudaErrorNotSupported) return ect;
  const int NS = pick_ns<T>(g, false);
  const size_t smem = forward_smem<T>(g, NS);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(block_forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.Kc + NS - 1) / NS), (unsigned)C);
  block_forward_kernel<T><<<grid, 256, smem, s>>>((const T*)Mf, (cpx<T>*)spec, (const cpx<T>*)tw, g, NS);
  return cudaGetLastError();
}

template <typename T, int W>
cudaError_t inverse_reg_run(const BlockGeo& g, const void* spec, void* region, const void* tw, cudaStream_t s) {
  int NS = 1;
  while (2 * NS * W * W <= 1024 && 2 * NS <= 8) NS *= 2;
  const int threads = (NS * W * W + 31) / 32 * 32;
  const size_t smem = sizeof(cpx<T>) * ((size_t)g.m * W + (size_t)NS * g.m * g.m + (size_t)NS * g.m * W);
  cudaError_t e =
      cudaFuncSetAttribute(block_inverse_reg_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.Kc + NS - 1) / NS), (unsigned)g.C);
  block_inverse_reg_kernel<T, W><<<grid, threads, smem, s>>>((const cpx<T>*)spec, (T*)region, (const cpx<T>*)tw, g,
                                                             NS);
  return cudaGetLastError();
}

template <typename T, int M, int W, int CR>
cudaError_t inverse_fft_run(const BlockGeo& g, const void* spec, void* region, const void* tw, cudaStream_t s) {
  constexpr int NS = inv_ns(M, sizeof(T));
  const size_t smem = sizeof(cpx<T>) * ((size_t)M + (size_t)NS * M * M * (M / 2 + 1));
  if (smem > 200 * 1024) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(block_inverse_fft_kernel<T, M, W, CR>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.Kc + NS - 1) / NS), (unsigned)g.C);
  block_inverse_fft_kernel<T, M, W, CR><<<grid, 256, smem, s>>>((const cpx<T>*)spec, (T*)region, (const cpx<T>*)tw, g);
  return cudaGetLastError();
}

template <typename T>
cudaError_t inverse_run(const HierGeo& h, int C, const void* spec, void* region, const void* tw, cudaStream_t s) {
  const BlockGeo g = make_geo(h, C);
  // (c, r) = (1, 2), (1, 4), (2, 2), (1, 8), (2, 4): FFT passes while a block's half spectrum fits
  cudaError_t e = cudaErrorNotSupported;
  if (g.m == 8 && g.W == 6) e = inverse_fft_run<T, 8, 6, 2>(g, spec, region, tw, s);
  if (g.m == 16 && g.W == 12) e = inverse_fft_run<T, 16, 12, 4>(g, spec, region, tw, s);
  if (g.m == 16 && g.W == 10) e = inverse_fft_run<T, 16, 10, 4>(g, spec, region, tw, s);
  if (g.m == 32 && g.W == 24) e = inverse_fft_run<T, 32, 24, 8>(g, spec, region, tw, s);
  if (g.m == 32 && g.W == 20) e = inverse_fft_run<T, 32, 20, 8>(g, spec, region, tw, s);
  if (e != cudaErrorNotSupported) return e;
  // kept widths (2c+1) r with (2c+1)^2 r^2 <= 1024: registers per thread column
  switch (g.W) {
    case 6: return inverse_reg_run<T, 6>(g, spec, region, tw, s);
    case 10: return inverse_reg_run<T, 10>(g, spec, region, tw, s);
    case 12: return inverse_reg_run<T, 12>(g, spec, region, tw, s);
    case 20: return inverse_reg_run<T, 20>(g, spec, region, tw, s);
    case 24: return inverse_reg_run<T, 24>(g, spec, region, tw, s);
    default: break;
  }
  const int NS = pick_ns<T>(g, true);
  const size_t smem = inverse_smem<T>(g, NS);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  e = cudaFuncSetAttribute(block_inverse_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

bool hier_use_matrices(const HierGeo& h, int p) {
  const int64_t C = nterms(p);
  return (int64_t)h.r * h.r * h.r * C * C <= ((int64_t)1 << 24);
}

cudaError_t launch_hier_matrices(const HierGeo& h, int p, bool fp64, const void* rtab, void* um, cudaStream_t s) {
  const int64_t n = (int64_t)h.r * h.r * h.r * nterms(p) * ((p + 1) * (p + 2) / 2);
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (fp64)
    translation_matrix_kernel<double><<<blocks, 128, 0, s>>>(p, h.r, (const double*)rtab, (double*)um);
  else
    translation_matrix_kernel<float><<<blocks, 128, 0, s>>>(p, h.r, (const float*)rtab, (float*)um);
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
                              const void* rtab, const void* um, void* Lf, int periodic, cudaStream_t s, int* nl) {
  const BlockGeo g = make_geo(h, nterms(p));
  if (um) {
    dim3 grid((unsigned)((g.Kf + 127) / 128), (unsigned)g.C);
    if (fp64)
      local_matrix_kernel<double><<<grid, 128, 0, s>>>((const double*)Lc, (const double*)region, (const double*)um,
                                                       (double*)Lf, g, periodic);
    else
      local_matrix_kernel<float><<<grid, 128, 0, s>>>((const float*)Lc, (const float*)region, (const float*)um,
                                                      (float*)Lf, g, periodic);
    ++*nl;
    return cudaGetLastError();
  }
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
