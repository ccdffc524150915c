// Green function components on the transform grid, FP64, lengths in units of hs
// ("performed and saved at the beginning of the simulation", Sec. 2.1).
// Component s = sidx(j, kap), j <= 2p, is the real storage (App. A.7) of the
// kernel entry S_j^kap, so that the M2L of cell j to cell i is
//   L_l^m = sum M_lam^mu G_{l+lam}^{-(m+mu)}(i - j)          (Eq. M2L, Eq. pmmm).
//
// Open boundary (Sec. 2.1, App. C): G(d) = S(d h) for cell offsets |d_a| < n_a
// with max |d_a| > c; zero for the (2c+1)^3 masked offsets and at index n_a of the
// 2n_a grid.
//
// Periodic boundary (App. B, Eqs. infsum, greenPBC): the Ewald split of the
// lattice sum over |n|_2 <= nmax in both spaces, at the minimum-image offset.
// The one image whose cell offset has max |D_a| <= c is masked: it enters as
// -P(j+1/2, (alpha r)^2) S_j instead of Q(j+1/2, (alpha r)^2) S_j, and is left
// out entirely at zero offset (its l = 0 limit, -2 alpha/sqrt(pi), is applied to
// the particles as the self term of App. B.3).
#include <vector>

#include "harmonics.cuh"
#include "internal.cuh"

namespace pmmm {

namespace {

constexpr double kPi = 3.14159265358979323846;

__global__ void green_open_kernel(double* __restrict__ G, Dims d, int J, int c, double csx, double csy, double csz) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d.Kt) return;
  const int x = (int)(g % d.Lx), y = (int)((g / d.Lx) % d.Ly), z = (int)(g / ((int64_t)d.Lx * d.Ly));
  const int dx = x < d.nx ? x : x - d.Lx;
  const int dy = y < d.ny ? y : y - d.Ly;
  const int dz = z < d.nz ? z : z - d.Lz;
  const int ng = (J + 1) * (J + 1);
  const bool outside = (dx <= -d.nx) || (dy <= -d.ny) || (dz <= -d.nz);
  const int am = max(abs(dx), max(abs(dy), abs(dz)));
  if (outside || am <= c) {
    for (int s = 0; s < ng; ++s) G[(int64_t)s * d.Kt + g] = 0.0;
    return;
  }
  const double rx = dx * csx, ry = dy * csy, rz = dz * csz;
  for (int m = 0; m <= J; ++m)
    singular_column<double>(m, J, rx, ry, rz, [&](int l, double re, double im) {
      G[(int64_t)sidx(l, m) * d.Kt + g] = re;
      if (m > 0) G[(int64_t)sidx(l, -m) * d.Kt + g] = im;
    });
}

// Regularised incomplete gamma functions of half-integer order a = l + 1/2,
// l = 0..J (App. B.1 split).  Upper: Q_0 = erfc(sqrt x), Q_l = Q_{l-1} + t_{l-1}
// with t_l = x^(l+1/2) e^-x / Gamma(l+3/2).  Lower: P_J by its power series, then
// P_l = P_{l+1} + t_l downward (no cancellation); 1 - Q where x is large.
template <int JMAX>
__device__ __forceinline__ void gamma_half(int J, double x, bool lower, double* out) {
  if (!lower || x > J + 1.5) {
    const double sx = sqrt(x);
    double q = erfc(sx);
    double t = 1.1283791670955125739 * sx * exp(-x);  // t_0 = x^(1/2) e^-x / Gamma(3/2)
#pragma unroll
    for (int l = 0; l <= JMAX; ++l) {
      if (l <= J) {
        out[l] = lower ? 1.0 - q : q;
        q += t;
        t *= x / (l + 1.5);
      }
    }
    return;
  }
  const double a = J + 0.5;
  const double tJ = exp(a * log(x) - x - lgamma(a + 1.0));  // x^(J+1/2) e^-x / Gamma(J+3/2)
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 400; ++k) {
    term *= x / (a + k);
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  double P = tJ * sum;
  double t = tJ;  // t_J
#pragma unroll
  for (int l = JMAX; l >= 0; --l) {
    if (l <= J) {
      if (l < J) {
        t = t * (l + 1.5) / x;  // t_l from t_{l+1}
        P += t;
      }
      out[l] = P;
    }
  }
}

template <int JMAX>
__global__ void __launch_bounds__(128) green_periodic_kernel(double* __restrict__ G, Dims d, int J, int c, double csx,
                                                             double csy, double csz, double alpha, int nmax,
                                                             const double2* __restrict__ rtab,
                                                             const int4* __restrict__ kvec, int nk) {
  const int64_t K = d.Kt;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * (J + 1)) return;
  const int m = (int)(t / K);
  const int64_t g = t - (int64_t)m * K;
  const int x = (int)(g % d.Lx), y = (int)((g / d.Lx) % d.Ly), z = (int)(g / ((int64_t)d.Lx * d.Ly));
  const int dm[3] = {2 * x <= d.Lx ? x : x - d.Lx, 2 * y <= d.Ly ? y : y - d.Ly, 2 * z <= d.Lz ? z : z - d.Lz};
  const double cs[3] = {csx, csy, csz};
  const int Ln[3] = {d.Lx, d.Ly, d.Lz};
  const double r0[3] = {dm[0] * csx, dm[1] * csy, dm[2] * csz};
  const double box[3] = {d.Lx * csx, d.Ly * csy, d.Lz * csz};
  double are[JMAX + 1], aim[JMAX + 1];
#pragma unroll
  for (int l = 0; l <= JMAX; ++l) are[l] = aim[l] = 0.0;

  // real-space part
  for (int a = -nmax; a <= nmax; ++a)
    for (int b = -nmax; b <= nmax; ++b)
      for (int e = -nmax; e <= nmax; ++e) {
        if (a * a + b * b + e * e > nmax * nmax) continue;
        const int nv[3] = {a, b, e};
        int D[3];
        bool near = true, zero = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          D[q] = dm[q] + nv[q] * Ln[q];
          near = near && (abs(D[q]) <= c);
          zero = zero && (D[q] == 0);
        }
        if (near && zero) continue;
        const double rx = r0[0] + a * box[0], ry = r0[1] + b * box[1], rz = r0[2] + e * box[2];
        const double r2 = rx * rx + ry * ry + rz * rz;
        double gam[JMAX + 1];
        gamma_half<JMAX>(J, alpha * alpha * r2, near, gam);
        const double ir2 = 1.0 / r2;
        double smr = 1.0 / sqrt(r2), smi = 0.0;  // S_0^0, then S_m^m
        for (int k = 1; k <= m; ++k) {
          const double s = -(2 * k - 1) * ir2;
          const double nr = s * (rx * smr - ry * smi);
          const double ni = s * (rx * smi + ry * smr);
          smr = nr;
          smi = ni;
        }
        double ar = 0, ai = 0, br = 0, bi = 0;
#pragma unroll
        for (int l = 0; l <= JMAX; ++l) {
          if (l >= m && l <= J) {
            double cr, ci;
            if (l == m) {
              cr = smr;
              ci = smi;
            } else {
              const double c1 = 2 * l - 1, c2 = (double)((l + m - 1) * (l - m - 1));
              cr = -(c1 * rz * br + c2 * ar) * ir2;
              ci = -(c1 * rz * bi + c2 * ai) * ir2;
            }
            ar = br;
            ai = bi;
            br = cr;
            bi = ci;
            const double w = near ? -gam[l] : gam[l];
            are[l] += w * cr;
            aim[l] += w * ci;
          }
        }
      }
  // reciprocal part: sum_n A_l^m(n) exp(2 pi i k_n . r), k_n . r = sum_a n_a dm_a / L_a
  const int ng = (J + 1) * (J + 1);
  for (int q = 0; q < nk; ++q) {
    const int4 kv = kvec[q];
    long long f[3] = {(long long)kv.x * dm[0], (long long)kv.y * dm[1], (long long)kv.z * dm[2]};
    double frac = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      long long v = f[a] % Ln[a];
      if (v < 0) v += Ln[a];
      frac += (double)v / (double)Ln[a];
    }
    double sp, cp;
    sincospi(2.0 * frac, &sp, &cp);
    const double2* A = rtab + (int64_t)q * ng;
#pragma unroll
    for (int l = 0; l <= JMAX; ++l) {
      if (l >= m && l <= J) {
        const double2 v = A[sidx(l, m)];
        are[l] += v.x * cp - v.y * sp;
        aim[l] += v.x * sp + v.y * cp;
      }
    }
  }
  (void)cs;
#pragma unroll
  for (int l = 0; l <= JMAX; ++l) {
    if (l >= m && l <= J) {
      G[(int64_t)sidx(l, m) * K + g] = are[l];
      if (m > 0) G[(int64_t)sidx(l, -m) * K + g] = aim[l];
    }
  }
}

// A_l^m(n) = (-i pi)^l / sqrt(pi) * exp(-(pi k / alpha)^2) / Gamma(l + 1/2) * k^(2l-1) / V * S_l^m(k_n)
// for the reciprocal vectors k_n = n / b (units of hs), m >= 0, at rtab[q][sidx(l, m)].
__global__ void green_recip_table_kernel(double2* __restrict__ rtab, const int4* __restrict__ kvec, int nk, int J,
                                         double bx, double by, double bz, double alpha, double V) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nk * (J + 1)) return;
  const int q = t / (J + 1), m = t - q * (J + 1);
  const int4 kv = kvec[q];
  const double kx = kv.x / bx, ky = kv.y / by, kz = kv.z / bz;
  const double k = sqrt(kx * kx + ky * ky + kz * kz);
  const double gauss = exp(-(kPi * k / alpha) * (kPi * k / alpha));
  const int ng = (J + 1) * (J + 1);
  singular_column<double>(m, J, kx, ky, kz, [&](int l, double re, double im) {
    // Gamma(l + 1/2) and pi^l by products (l <= 24)
    double gl = 1.7724538509055160273, pl = 1.0;
    for (int u = 1; u <= l; ++u) {
      gl *= (u - 0.5);
      pl *= kPi;
    }
    const double mag = pl / 1.7724538509055160273 * gauss / gl * pow(k, 2.0 * l - 1.0) / V;
    // (-i)^l
    double cr, ci;
    switch (l & 3) {
      case 0: cr = mag; ci = 0; break;
      case 1: cr = 0; ci = -mag; break;
      case 2: cr = -mag; ci = 0; break;
      default: cr = 0; ci = mag; break;
    }
    rtab[(int64_t)q * ng + sidx(l, m)] = make_double2(cr * re - ci * im, cr * im + ci * re);
  });
}

template <typename T>
__global__ void green_finish_kernel(const double2* __restrict__ in, cpx<T>* __restrict__ out, int64_t count,
                                    int64_t Kh, double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  // the spectrum of a component of order j is real (even j) or imaginary (odd j):
  // the other part, rounding noise of the transform (or the asymmetry of an
  // under-converged lattice sum), is set to zero
  const int s = (int)(i / Kh);
  int j = 0;
  while ((j + 1) * (j + 1) <= s) ++j;
  const double2 v = in[i];
  out[i] = (j & 1) ? mk((T)0, (T)(v.y * scale)) : mk((T)(v.x * scale), (T)0);
}

// The one real number per kernel spectrum value that the parity leaves (component
// s = sidx(j, a) of order j: the real part for even j, the imaginary part for odd
// j; the other part vanishes up to rounding), scaled as the complex spectra.
template <typename T>
__global__ void green_parity_kernel(const double2* __restrict__ in, T* __restrict__ out, int CG, int64_t Kh,
                                    double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)CG * Kh) return;
  const int s = (int)(i / Kh);
  int j = 0;
  while ((j + 1) * (j + 1) <= s) ++j;
  const double2 v = in[i];
  out[i] = (T)(((j & 1) ? v.y : v.x) * scale);
}

}  // namespace

cudaError_t launch_green_parity(const void* specd, void* outr, bool fp64, int CG, int64_t Kh, double scale,
                                cudaStream_t st) {
  const int64_t count = (int64_t)CG * Kh;
  const unsigned blocks = (unsigned)((count + 255) / 256);
  if (fp64)
    green_parity_kernel<double><<<blocks, 256, 0, st>>>((const double2*)specd, (double*)outr, CG, Kh, scale);
  else
    green_parity_kernel<float><<<blocks, 256, 0, st>>>((const double2*)specd, (float*)outr, CG, Kh, scale);
  return cudaGetLastError();
}

cudaError_t launch_green_open(double* G, const Dims& d, int p, int c, const double cs[3], cudaStream_t st) {
  green_open_kernel<<<(unsigned)((d.Kt + 127) / 128), 128, 0, st>>>(G, d, 2 * p, c, cs[0], cs[1], cs[2]);
  return cudaGetLastError();
}

cudaError_t launch_green_periodic(double* G, const Dims& d, int p, int c, const double cs[3], double alpha_s,
                                  int nmax, cudaStream_t st) {
  const int J = 2 * p;
  std::vector<int4> kv;
  for (int a = -nmax; a <= nmax; ++a)
    for (int b = -nmax; b <= nmax; ++b)
      for (int e = -nmax; e <= nmax; ++e) {
        const int nn = a * a + b * b + e * e;
        if (nn == 0 || nn > nmax * nmax) continue;
        kv.push_back(make_int4(a, b, e, 0));
      }
  const int nk = (int)kv.size();
  const int ng = (J + 1) * (J + 1);
  int4* dk = nullptr;
  double2* rt = nullptr;
  cudaError_t e = cudaMalloc(&dk, sizeof(int4) * (nk > 0 ? nk : 1));
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&rt, sizeof(double2) * (size_t)(nk > 0 ? nk : 1) * ng);
  if (e != cudaSuccess) {
    cudaFree(dk);
    return e;
  }
  cudaMemsetAsync(rt, 0, sizeof(double2) * (size_t)(nk > 0 ? nk : 1) * ng, st);
  if (nk > 0) cudaMemcpyAsync(dk, kv.data(), sizeof(int4) * nk, cudaMemcpyHostToDevice, st);
  const double bx = d.Lx * cs[0], by = d.Ly * cs[1], bz = d.Lz * cs[2];
  if (nk > 0)
    green_recip_table_kernel<<<(nk * (J + 1) + 127) / 128, 128, 0, st>>>(rt, dk, nk, J, bx, by, bz, alpha_s,
                                                                         bx * by * bz);
  const unsigned blocks = (unsigned)((d.Kt * (J + 1) + 127) / 128);
  if (J <= 8)
    green_periodic_kernel<8><<<blocks, 128, 0, st>>>(G, d, J, c, cs[0], cs[1], cs[2], alpha_s, nmax, rt, dk, nk);
  else if (J <= 16)
    green_periodic_kernel<16><<<blocks, 128, 0, st>>>(G, d, J, c, cs[0], cs[1], cs[2], alpha_s, nmax, rt, dk, nk);
  else
    green_periodic_kernel<24><<<blocks, 128, 0, st>>>(G, d, J, c, cs[0], cs[1], cs[2], alpha_s, nmax, rt, dk, nk);
  e = cudaGetLastError();
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFree(dk);
  cudaFree(rt);
  return e != cudaSuccess ? e : e2;
}

cudaError_t launch_green_finish(const void* specd, void* out, bool fp64, int64_t count, int64_t Kh, double scale,
                                cudaStream_t st) {
  const unsigned blocks = (unsigned)((count + 255) / 256);
  if (fp64)
    green_finish_kernel<double><<<blocks, 256, 0, st>>>((const double2*)specd, (cpx<double>*)out, count, Kh, scale);
  else
    green_finish_kernel<float><<<blocks, 256, 0, st>>>((const double2*)specd, (cpx<float>*)out, count, Kh, scale);
  return cudaGetLastError();
}

}  // namespace pmmm
