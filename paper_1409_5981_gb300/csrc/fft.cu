// Batched 3-D real FFTs of the (p+1)^2 moment channels (Sec. 2.1) on
// power-of-two meshes, with the zero padding of open boundaries (App. C) kept
// implicit: rows, columns and planes known to be zero are neither read nor
// transformed, and only the physical octant of the inverse is written.
//
//   forward:  x: real rows -> half spectra (two real rows per complex FFT)
//             y: columns of length Ly over z < nz planes (rows y >= ny are zero)
//             z: columns of length Lz (planes z >= nz are zero)
//   inverse:  z (only z < nz written), y (only y < ny), x: half -> real rows,
//             only x < nx written.
// Spectra are stored [C][Lz][Ly][hx], hx = Lx/2 + 1.  Every 1-D transform is a
// shared-memory Stockham FFT (fft.cuh).
#include "internal.cuh"

namespace pmmm {

namespace {

constexpr int FFT_THREADS = 256;

// Runs every Stockham stage of `ntrans` transforms held in shared memory.
// ROWS: transform tr occupies A[tr * L .. tr * L + L) (element stride 1) and the
// butterfly index varies fastest across threads.  Otherwise (columns) element t
// of transform tr sits at A[t * ntrans + tr] and the transform index varies
// fastest, so that neighbouring threads touch neighbouring words.
template <typename T, bool ROWS>
__device__ __forceinline__ void run_stages(cpx<T>*& A, cpx<T>*& B, const FftPlan1D& pl, int ntrans,
                                           const cpx<T>* tw, int sgn) {
  int Ns = 1;
  const int L = pl.L;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = pl.rad[st];
    const int nb = L / R;
    const int tasks = nb * ntrans;
    for (int t = threadIdx.x; t < tasks; t += blockDim.x) {
      if (ROWS) {
        const int tr = t / nb, j = t - tr * nb;
        stockham_bf_any<T>(R, A + tr * L, B + tr * L, L, Ns, j, 1, tw, sgn);
      } else {
        const int tr = t % ntrans, j = t / ntrans;
        stockham_bf_any<T>(R, A + tr, B + tr, L, Ns, j, ntrans, tw, sgn);
      }
    }
    __syncthreads();
    cpx<T>* tmp = A;
    A = B;
    B = tmp;
    Ns *= R;
  }
}

// Forward x pass: rows r = (c, z, y), z < nz, y < ny, real length nx inside Lx.
// Block handles `ppb` pairs of rows; pair (a, b) is packed as a + i b.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) r2c_rows_kernel(const T* __restrict__ in, cpx<T>* __restrict__ out,
                                                               Dims d, int C, FftPlan1D pl,
                                                               const cpx<T>* __restrict__ tw, int ppb) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* B = A + (size_t)ppb * d.Lx;
  const int64_t nrows = (int64_t)C * d.nz * d.ny;
  const int64_t pair0 = (int64_t)blockIdx.x * ppb;
  const int Lx = d.Lx;
  for (int e = threadIdx.x; e < ppb * Lx; e += blockDim.x) {
    const int pr = e / Lx, x = e - pr * Lx;
    const int64_t ra = 2 * (pair0 + pr), rb = ra + 1;
    T a = T(0), b = T(0);
    if (x < d.nx) {
      if (ra < nrows) a = in[ra * d.nx + x];
      if (rb < nrows) b = in[rb * d.nx + x];
    }
    A[e] = mk(a, b);
  }
  __syncthreads();
  run_stages<T, true>(A, B, pl, ppb, tw, -1);
  const int hx = d.hx;
  for (int e = threadIdx.x; e < ppb * hx; e += blockDim.x) {
    const int pr = e / hx, k = e - pr * hx;
    const int64_t ra = 2 * (pair0 + pr), rb = ra + 1;
    const cpx<T> Z = A[pr * Lx + k];
    const cpx<T> Zm = conjg(A[pr * Lx + ((Lx - k) & (Lx - 1))]);
    // X = (Z + conj Z_{-k}) / 2 ;  Y = (Z - conj Z_{-k}) / (2i)
    const cpx<T> X = mk((Z.x + Zm.x) * T(0.5), (Z.y + Zm.y) * T(0.5));
    const cpx<T> Dd = mk(Z.x - Zm.x, Z.y - Zm.y);
    const cpx<T> Y = mk(Dd.y * T(0.5), -Dd.x * T(0.5));
    if (ra < nrows) {
      const int64_t c = ra / ((int64_t)d.nz * d.ny), rem = ra - c * d.nz * d.ny;
      const int z = (int)(rem / d.ny), y = (int)(rem - (int64_t)z * d.ny);
      out[c * d.Kh + ((int64_t)z * d.Ly + y) * hx + k] = X;
    }
    if (rb < nrows) {
      const int64_t c = rb / ((int64_t)d.nz * d.ny), rem = rb - c * d.nz * d.ny;
      const int z = (int)(rem / d.ny), y = (int)(rem - (int64_t)z * d.ny);
      out[c * d.Kh + ((int64_t)z * d.Ly + y) * hx + k] = Y;
    }
  }
}

// Inverse x pass: half spectra of rows (c, z < nz, y < ny) -> real rows, x < nx written.
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) c2r_rows_kernel(const cpx<T>* __restrict__ in, T* __restrict__ out,
                                                               Dims d, int C, FftPlan1D pl,
                                                               const cpx<T>* __restrict__ tw, int ppb) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* B = A + (size_t)ppb * d.Lx;
  const int64_t nrows = (int64_t)C * d.nz * d.ny;
  const int64_t pair0 = (int64_t)blockIdx.x * ppb;
  const int Lx = d.Lx, hx = d.hx, half = Lx / 2;
  for (int e = threadIdx.x; e < ppb * Lx; e += blockDim.x) {
    const int pr = e / Lx, k = e - pr * Lx;
    const int64_t r2[2] = {2 * (pair0 + pr), 2 * (pair0 + pr) + 1};
    cpx<T> v[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      v[q] = mk(T(0), T(0));
      if (r2[q] < nrows) {
        const int64_t c = r2[q] / ((int64_t)d.nz * d.ny), rem = r2[q] - c * d.nz * d.ny;
        const int z = (int)(rem / d.ny), y = (int)(rem - (int64_t)z * d.ny);
        const cpx<T>* row = in + c * d.Kh + ((int64_t)z * d.Ly + y) * hx;
        if (k <= half) {
          v[q] = row[k];
          if (k == 0 || k == half) v[q].y = T(0);
        } else {
          v[q] = conjg(row[Lx - k]);
        }
      }
    }
    // Z = X + i Y
    A[e] = mk(v[0].x - v[1].y, v[0].y + v[1].x);
  }
  __syncthreads();
  run_stages<T, true>(A, B, pl, ppb, tw, +1);
  for (int e = threadIdx.x; e < ppb * d.nx; e += blockDim.x) {
    const int pr = e / d.nx, x = e - pr * d.nx;
    const int64_t ra = 2 * (pair0 + pr), rb = ra + 1;
    const cpx<T> z = A[pr * Lx + x];
    if (ra < nrows) out[ra * d.nx + x] = z.x;
    if (rb < nrows) out[rb * d.nx + x] = z.y;
  }
}

// Column FFTs along a strided axis: element (row, col) of batch b at
// base(b) + row * col_stride + col, col < inner.  Tile of TW columns per block;
// rows >= nin read as zero, only rows < nout written back (in place).
template <typename T>
__global__ void __launch_bounds__(FFT_THREADS) cols_kernel(cpx<T>* __restrict__ data, int64_t col_stride, int inner,
                                                           int64_t bstride1, int nb1, int64_t bstride2, int TW,
                                                           int nin, int nout, int sgn, FftPlan1D pl,
                                                           const cpx<T>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  const int L = pl.L;
  cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* B = A + (size_t)L * TW;
  const int col0 = blockIdx.y * TW;
  const int b1 = (int)(blockIdx.x % (unsigned)nb1), b2 = (int)(blockIdx.x / (unsigned)nb1);
  cpx<T>* base = data + (int64_t)b2 * bstride2 + (int64_t)b1 * bstride1 + col0;
  const int w = min(TW, inner - col0);
  for (int e = threadIdx.x; e < L * TW; e += blockDim.x) {
    const int row = e / TW, col = e - row * TW;
    A[e] = (row < nin && col < w) ? base[row * col_stride + col] : mk(T(0), T(0));
  }
  __syncthreads();
  run_stages<T, false>(A, B, pl, TW, tw, sgn);
  for (int e = threadIdx.x; e < L * TW; e += blockDim.x) {
    const int row = e / TW, col = e - row * TW;
    if (row < nout && col < w) base[row * col_stride + col] = A[e];
  }
}

// Block-wide copy of n complex values (plane of the spectrum <-> shared memory):
// 16-byte words (two FP32 complex values) when both ends are 16-byte aligned.
template <typename T>
__device__ __forceinline__ void copy_plane(cpx<T>* dst, const cpx<T>* src, int n) {
  if (sizeof(T) == 4 && ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll 4
    for (int e = threadIdx.x; e < n / 2; e += blockDim.x) d4[e] = s4[e];
    if ((n & 1) && threadIdx.x == 0) dst[n - 1] = src[n - 1];
  } else {
    for (int e = threadIdx.x; e < n; e += blockDim.x) dst[e] = src[e];
  }
}

// Forward x and y passes of one plane (c, z < nz) in one block: the real rows
// y < ny (two per complex transform) -> half-spectrum rows -> columns along y
// (rows y >= ny zero) -> the plane [Ly][hx] of the spectrum, written contiguously.
// One read of the moments and one write of the plane replace the separate x and
// y passes (each a read and a write of the spectrum).  LX, LY > 0: transform
// lengths known at compile time (indices fold; twiddles staged in shared memory);
// 0: taken from d.
template <typename T, int LX, int LY>
__global__ void __launch_bounds__(FFT_THREADS) plane_fwd_kernel(const T* __restrict__ in, cpx<T>* __restrict__ out,
                                                                Dims d, FftPlan1D plx, FftPlan1D ply,
                                                                const cpx<T>* __restrict__ twx,
                                                                const cpx<T>* __restrict__ twy, int64_t abuf) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* B = A + abuf;
  const int Lx = LX > 0 ? LX : d.Lx, Ly = LY > 0 ? LY : d.Ly, hx = Lx / 2 + 1;
  const cpx<T>* tx = twx;
  const cpx<T>* ty = twy;
  if constexpr (LX > 0) {
    cpx<T>* st = B + abuf;
    for (int t = threadIdx.x; t < LX; t += blockDim.x) st[t] = twx[t];
    for (int t = threadIdx.x; t < LY; t += blockDim.x) st[LX + t] = twy[t];
    tx = st;
    ty = st + LX;
  }
  const int64_t c = blockIdx.x / d.nz;
  const int z = (int)(blockIdx.x - c * d.nz);
  const int npairs = (d.ny + 1) / 2;
  const T* src = in + (c * d.nz + z) * (int64_t)d.ny * d.nx;
  // x pass: row pair pr packs rows 2 pr (real part) and 2 pr + 1 (imaginary part).
  // Compile-time lengths keep the pairs as columns (element x of pair pr at
  // A[x ES + pr], ES = npairs + 1 odd: bank-conflict-free butterflies); else rows.
  const int ES = LX > 0 ? npairs + 1 : 0;
  auto xat = [&](int pr, int x) { return LX > 0 ? x * ES + pr : pr * Lx + x; };
  if (sizeof(T) == 4 && (d.nx & 3) == 0) {
    // FP32 rows read as 16-byte vectors, four loads in flight per thread
    const int q4 = Lx / 4, nq = d.nx / 4;
#pragma unroll 4
    for (int v = threadIdx.x; v < npairs * q4; v += blockDim.x) {
      const int pr = v / q4, x4 = v - pr * q4;
      const int ya = 2 * pr, yb = ya + 1;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (x4 < nq) {
        a = reinterpret_cast<const float4*>(src + (int64_t)ya * d.nx)[x4];
        if (yb < d.ny) b = reinterpret_cast<const float4*>(src + (int64_t)yb * d.nx)[x4];
      }
      A[xat(pr, 4 * x4 + 0)] = mk((T)a.x, (T)b.x);
      A[xat(pr, 4 * x4 + 1)] = mk((T)a.y, (T)b.y);
      A[xat(pr, 4 * x4 + 2)] = mk((T)a.z, (T)b.z);
      A[xat(pr, 4 * x4 + 3)] = mk((T)a.w, (T)b.w);
    }
  } else {
    for (int e = threadIdx.x; e < npairs * Lx; e += blockDim.x) {
      const int pr = e / Lx, x = e - pr * Lx;
      const int ya = 2 * pr, yb = ya + 1;
      T a = T(0), b = T(0);
      if (x < d.nx) {
        a = src[(int64_t)ya * d.nx + x];
        if (yb < d.ny) b = src[(int64_t)yb * d.nx + x];
      }
      A[xat(pr, x)] = mk(a, b);
    }
  }
  __syncthreads();
  if constexpr (LX > 0)
    run_stages_ct<T, false, LX, -1>(A, B, npairs, tx, ES);
  else
    run_stages<T, true>(A, B, plx, npairs, tx, -1);
  // half spectra of the rows into B as the plane [Ly][hx] (rows y >= ny zero)
  for (int e = threadIdx.x; e < Ly * hx; e += blockDim.x) {
    const int y = e / hx, k = e - y * hx;
    cpx<T> v = mk(T(0), T(0));
    if (y < d.ny) {
      const int pr = y >> 1;
      const cpx<T> Z = A[xat(pr, k)];
      const cpx<T> Zm = conjg(A[xat(pr, (Lx - k) & (Lx - 1))]);
      v = (y & 1) ? mk((Z.y - Zm.y) * T(0.5), -(Z.x - Zm.x) * T(0.5)) : mk((Z.x + Zm.x) * T(0.5), (Z.y + Zm.y) * T(0.5));
    }
    B[e] = v;
  }
  __syncthreads();
  if constexpr (LY > 0)
    run_stages_ct<T, false, LY, -1>(B, A, hx, ty);
  else
    run_stages<T, false>(B, A, ply, hx, ty, -1);
  cpx<T>* dst = out + c * d.Kh + (int64_t)z * Ly * hx;
  copy_plane<T>(dst, B, Ly * hx);
}

// Inverse y and x passes of one plane (c, z < nz): the plane [Ly][hx] of the
// spectrum -> columns along y (only rows y < ny kept) -> row pairs -> real rows,
// x < nx written.
template <typename T, int LX, int LY>
__global__ void __launch_bounds__(FFT_THREADS) plane_inv_kernel(const cpx<T>* __restrict__ in, T* __restrict__ out,
                                                                Dims d, FftPlan1D plx, FftPlan1D ply,
                                                                const cpx<T>* __restrict__ twx,
                                                                const cpx<T>* __restrict__ twy, int64_t abuf) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* B = A + abuf;
  const int Lx = LX > 0 ? LX : d.Lx, Ly = LY > 0 ? LY : d.Ly, hx = Lx / 2 + 1, half = Lx / 2;
  const cpx<T>* tx = twx;
  const cpx<T>* ty = twy;
  if constexpr (LX > 0) {
    cpx<T>* st = B + abuf;
    for (int t = threadIdx.x; t < LX; t += blockDim.x) st[t] = twx[t];
    for (int t = threadIdx.x; t < LY; t += blockDim.x) st[LX + t] = twy[t];
    tx = st;
    ty = st + LX;
  }
  const int64_t c = blockIdx.x / d.nz;
  const int z = (int)(blockIdx.x - c * d.nz);
  const int npairs = (d.ny + 1) / 2;
  const cpx<T>* src = in + c * d.Kh + (int64_t)z * Ly * hx;
  copy_plane<T>(A, src, Ly * hx);
  __syncthreads();
  if constexpr (LY > 0)
    run_stages_ct<T, false, LY, +1>(A, B, hx, ty);
  else
    run_stages<T, false>(A, B, ply, hx, ty, +1);
  // rows y < ny of the plane -> row pairs Z = X + i Y over the full length Lx in B
  // (columns with the odd stride ES for compile-time lengths, as the forward pass)
  const int ES = LX > 0 ? npairs + 1 : 0;
  auto xat = [&](int pr, int x) { return LX > 0 ? x * ES + pr : pr * Lx + x; };
  for (int e = threadIdx.x; e < npairs * Lx; e += blockDim.x) {
    const int pr = e / Lx, k = e - pr * Lx;
    cpx<T> v[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int y = 2 * pr + q;
      v[q] = mk(T(0), T(0));
      if (y < d.ny) {
        const cpx<T>* row = A + y * hx;
        if (k <= half) {
          v[q] = row[k];
          if (k == 0 || k == half) v[q].y = T(0);
        } else {
          v[q] = conjg(row[Lx - k]);
        }
      }
    }
    B[xat(pr, k)] = mk(v[0].x - v[1].y, v[0].y + v[1].x);
  }
  __syncthreads();
  if constexpr (LX > 0)
    run_stages_ct<T, false, LX, +1>(B, A, npairs, tx, ES);
  else
    run_stages<T, true>(B, A, plx, npairs, tx, +1);
  T* dst = out + (c * d.nz + z) * (int64_t)d.ny * d.nx;
  if (sizeof(T) == 4 && (d.nx & 3) == 0) {
    const int nq = d.nx / 4;
#pragma unroll 4
    for (int v = threadIdx.x; v < d.ny * nq; v += blockDim.x) {
      const int y = v / nq, x = 4 * (v - y * nq), pr = y >> 1;
      const cpx<T> r0 = B[xat(pr, x)], r1 = B[xat(pr, x + 1)], r2 = B[xat(pr, x + 2)], r3 = B[xat(pr, x + 3)];
      float4 o;
      if (y & 1)
        o = make_float4((float)r0.y, (float)r1.y, (float)r2.y, (float)r3.y);
      else
        o = make_float4((float)r0.x, (float)r1.x, (float)r2.x, (float)r3.x);
      reinterpret_cast<float4*>(dst)[v] = o;
    }
  } else {
    for (int e = threadIdx.x; e < d.ny * d.nx; e += blockDim.x) {
      const int y = e / d.nx, x = e - y * d.nx;
      const cpx<T> v = B[xat(y >> 1, x)];
      dst[e] = (y & 1) ? v.y : v.x;
    }
  }
}

// Shared memory of the plane kernels: two buffers, each the larger of the row
// pairs (npairs x Lx) and the plane (Ly x hx).
template <typename T>
int64_t plane_buf(const Dims& d) {
  const int64_t a = (int64_t)((d.ny + 1) / 2 + 1) * d.Lx, b = (int64_t)d.Ly * d.hx;
  return a > b ? a : b;
}
template <typename T>
bool plane_applies(const Dims& d) {
  return (2 * plane_buf<T>(d) + d.Lx + d.Ly) * (int64_t)sizeof(cpx<T>) <= 200 * 1024;
}

template <typename T, bool FWD, int LX, int LY>
void launch_plane_l(const void* in, void* out, const Dims& d, int C, const FftTw& tw, cudaStream_t s) {
  const int64_t ab = plane_buf<T>(d);
  const size_t smem = (2 * (size_t)ab + (size_t)(LX + LY)) * sizeof(cpx<T>);
  const unsigned grid = (unsigned)((int64_t)C * d.nz);
  const FftPlan1D plx = make_fft_plan(d.Lx), ply = make_fft_plan(d.Ly);
  if constexpr (FWD) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(plane_fwd_kernel<T, LX, LY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    plane_fwd_kernel<T, LX, LY><<<grid, FFT_THREADS, smem, s>>>((const T*)in, (cpx<T>*)out, d, plx, ply,
                                                                (const cpx<T>*)tw.x, (const cpx<T>*)tw.y, ab);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(plane_inv_kernel<T, LX, LY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    plane_inv_kernel<T, LX, LY><<<grid, FFT_THREADS, smem, s>>>((const cpx<T>*)in, (T*)out, d, plx, ply,
                                                                (const cpx<T>*)tw.x, (const cpx<T>*)tw.y, ab);
  }
}

// Square planes of 32, 64 or 128 points take the compile-time-length kernels.
template <typename T, bool FWD>
void launch_plane(const void* in, void* out, const Dims& d, int C, const FftTw& tw, cudaStream_t s) {
  if (d.Lx == d.Ly && d.Lx == 32) return launch_plane_l<T, FWD, 32, 32>(in, out, d, C, tw, s);
  if (d.Lx == d.Ly && d.Lx == 64) return launch_plane_l<T, FWD, 64, 64>(in, out, d, C, tw, s);
  if (d.Lx == d.Ly && d.Lx == 128) return launch_plane_l<T, FWD, 128, 128>(in, out, d, C, tw, s);
  launch_plane_l<T, FWD, 0, 0>(in, out, d, C, tw, s);
}

// cols_kernel with the transform length L and the direction SGN known at compile
// time (twiddles staged in shared memory after the two buffers).
template <typename T, int L, int SGN>
__global__ void __launch_bounds__(FFT_THREADS) cols_ct_kernel(cpx<T>* __restrict__ data, int64_t col_stride,
                                                              int inner, int64_t bstride1, int nb1, int64_t bstride2,
                                                              int TW, int nin, int nout,
                                                              const cpx<T>* __restrict__ tw) {
  extern __shared__ unsigned char smem_raw[];
  cpx<T>* A = reinterpret_cast<cpx<T>*>(smem_raw);
  cpx<T>* B = A + (size_t)L * TW;
  cpx<T>* st = B + (size_t)L * TW;
  for (int t = threadIdx.x; t < L; t += blockDim.x) st[t] = tw[t];
  const int col0 = blockIdx.y * TW;
  const int b1 = (int)(blockIdx.x % (unsigned)nb1), b2 = (int)(blockIdx.x / (unsigned)nb1);
  cpx<T>* base = data + (int64_t)b2 * bstride2 + (int64_t)b1 * bstride1 + col0;
  const int w = min(TW, inner - col0);
  // FP32 full tiles with 16-byte aligned rows: two complex values per load / store
  const bool vec = sizeof(T) == 4 && w == TW && (TW & 1) == 0 && (col_stride & 1) == 0 &&
                   ((reinterpret_cast<uintptr_t>(base)) & 15) == 0;
  if (vec) {
    const int h = TW / 2;
#pragma unroll 4
    for (int e = threadIdx.x; e < L * h; e += blockDim.x) {
      const int row = e / h, c2 = e - row * h;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < nin) v = reinterpret_cast<const float4*>(base + row * col_stride)[c2];
      reinterpret_cast<float4*>(A)[e] = v;
    }
  } else {
    for (int e = threadIdx.x; e < L * TW; e += blockDim.x) {
      const int row = e / TW, col = e - row * TW;
      A[e] = (row < nin && col < w) ? base[row * col_stride + col] : mk(T(0), T(0));
    }
  }
  __syncthreads();
  run_stages_ct<T, false, L, SGN>(A, B, TW, st);
  if (vec) {
    const int h = TW / 2;
#pragma unroll 4
    for (int e = threadIdx.x; e < nout * h; e += blockDim.x) {
      const int row = e / h, c2 = e - row * h;
      reinterpret_cast<float4*>(base + row * col_stride)[c2] = reinterpret_cast<const float4*>(A)[e];
    }
  } else {
    for (int e = threadIdx.x; e < L * TW; e += blockDim.x) {
      const int row = e / TW, col = e - row * TW;
      if (row < nout && col < w) base[row * col_stride + col] = A[e];
    }
  }
}

template <typename T>
__global__ void twiddle_kernel(int L, cpx<T>* tw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L) return;
  double s, c;
  sincospi(-2.0 * (double)t / (double)L, &s, &c);
  tw[t] = mk((T)c, (T)s);
}

int pick_ppb(int L) {
  int ppb = 2048 / L;
  return ppb < 1 ? 1 : ppb;
}

int pick_tw(int inner, int L, size_t elem) {
  // whole rows of up to 40 columns (e.g. the 17 or 33 points of a half spectrum), else 32
  // (256-byte row segments of FP32 complex values)
  int TW = inner <= 40 ? inner : 32;
  while (TW > 1 && 2 * (size_t)L * TW * elem > 96 * 1024) TW /= 2;
  return TW;
}

template <typename T>
cudaError_t cols(cpx<T>* data, int64_t col_stride, int inner, int64_t bs1, int nb1, int64_t bs2, int nb2, int nin,
                 int nout, int sgn, int L, const cpx<T>* tw, cudaStream_t s) {
  const FftPlan1D pl = make_fft_plan(L);
  const int TW = pick_tw(inner, L, sizeof(cpx<T>));
  const size_t smem = 2 * (size_t)L * TW * sizeof(cpx<T>);
  // batches on x (up to 2^31 - 1), column tiles on y (inner / TW <= 65535 for L <= 512)
  dim3 grid((unsigned)(nb1 * nb2), (unsigned)((inner + TW - 1) / TW));
#define PMMM_COLS_CT(LL)                                                                                        \
  if (L == LL) {                                                                                              \
    const size_t sm2 = smem + LL * sizeof(cpx<T>);                                                            \
    if (sgn < 0) {                                                                                            \
      if (sm2 > 48 * 1024)                                                                                    \
        cudaFuncSetAttribute(cols_ct_kernel<T, LL, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2); \
      cols_ct_kernel<T, LL, -1><<<grid, FFT_THREADS, sm2, s>>>(data, col_stride, inner, bs1, nb1, bs2, TW, nin, nout, tw); \
    } else {                                                                                                  \
      if (sm2 > 48 * 1024)                                                                                    \
        cudaFuncSetAttribute(cols_ct_kernel<T, LL, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2); \
      cols_ct_kernel<T, LL, 1><<<grid, FFT_THREADS, sm2, s>>>(data, col_stride, inner, bs1, nb1, bs2, TW, nin, nout, tw); \
    }                                                                                                         \
    return cudaGetLastError();                                                                                \
  }
  PMMM_COLS_CT(32)
  PMMM_COLS_CT(64)
  PMMM_COLS_CT(128)
  PMMM_COLS_CT(256)
#undef PMMM_COLS_CT
  if (smem > 48 * 1024) cudaFuncSetAttribute(cols_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cols_kernel<T><<<grid, FFT_THREADS, smem, s>>>(data, col_stride, inner, bs1, nb1, bs2, TW, nin, nout, sgn, pl, tw);
  return cudaGetLastError();
}

template <typename T>
cudaError_t forward(const T* in, cpx<T>* spec, const Dims& d, int C, const FftTw& tw, cudaStream_t s, int* nl) {
  if (plane_applies<T>(d)) {
    // x and y passes together, one block per plane (c, z < nz)
    launch_plane<T, true>((const void*)in, (void*)spec, d, C, tw, s);
    ++*nl;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else {
    // x pass
    {
      const FftPlan1D pl = make_fft_plan(d.Lx);
      const int ppb = pick_ppb(d.Lx);
      const int64_t nrows = (int64_t)C * d.nz * d.ny;
      const int64_t npairs = (nrows + 1) / 2;
      const size_t smem = 2 * (size_t)ppb * d.Lx * sizeof(cpx<T>);
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(r2c_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      r2c_rows_kernel<T><<<(int)((npairs + ppb - 1) / ppb), FFT_THREADS, smem, s>>>(in, spec, d, C, pl,
                                                                                   (const cpx<T>*)tw.x, ppb);
      ++*nl;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    // y pass over (c, z < nz): rows y >= ny are zero
    cudaError_t e = cols<T>(spec, d.hx, d.hx, (int64_t)d.Ly * d.hx, d.nz, d.Kh, C, d.ny, d.Ly, -1, d.Ly,
                            (const cpx<T>*)tw.y, s);
    ++*nl;
    if (e != cudaSuccess) return e;
  }
  // z pass over c: planes z >= nz are zero
  cudaError_t e = cols<T>(spec, (int64_t)d.Ly * d.hx, (int)((int64_t)d.Ly * d.hx), 0, 1, d.Kh, C, d.nz, d.Lz, -1,
                          d.Lz, (const cpx<T>*)tw.z, s);
  ++*nl;
  return e;
}

template <typename T>
cudaError_t inverse(cpx<T>* spec, T* out, const Dims& d, int C, const FftTw& tw, cudaStream_t s, int* nl) {
  // z pass: only planes z < nz are needed afterwards
  cudaError_t e = cols<T>(spec, (int64_t)d.Ly * d.hx, (int)((int64_t)d.Ly * d.hx), 0, 1, d.Kh, C, d.Lz, d.nz, +1,
                          d.Lz, (const cpx<T>*)tw.z, s);
  ++*nl;
  if (e != cudaSuccess) return e;
  if (plane_applies<T>(d)) {
    // y and x passes together, one block per plane (c, z < nz)
    launch_plane<T, false>((const void*)spec, (void*)out, d, C, tw, s);
    ++*nl;
    return cudaGetLastError();
  }
  // y pass over (c, z < nz): only rows y < ny needed
  e = cols<T>(spec, d.hx, d.hx, (int64_t)d.Ly * d.hx, d.nz, d.Kh, C, d.Ly, d.ny, +1, d.Ly, (const cpx<T>*)tw.y, s);
  ++*nl;
  if (e != cudaSuccess) return e;
  const FftPlan1D pl = make_fft_plan(d.Lx);
  const int ppb = pick_ppb(d.Lx);
  const int64_t nrows = (int64_t)C * d.nz * d.ny;
  const int64_t npairs = (nrows + 1) / 2;
  const size_t smem = 2 * (size_t)ppb * d.Lx * sizeof(cpx<T>);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(c2r_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  c2r_rows_kernel<T><<<(int)((npairs + ppb - 1) / ppb), FFT_THREADS, smem, s>>>(spec, out, d, C, pl,
                                                                               (const cpx<T>*)tw.x, ppb);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fft_forward(bool fp64, const void* in, void* spec, const Dims& d, int C, const FftTw& tw,
                               cudaStream_t s, int* nl) {
  return fp64 ? forward<double>((const double*)in, (cpx<double>*)spec, d, C, tw, s, nl)
              : forward<float>((const float*)in, (cpx<float>*)spec, d, C, tw, s, nl);
}

cudaError_t launch_fft_inverse(bool fp64, void* spec, void* out, const Dims& d, int C, const FftTw& tw,
                               cudaStream_t s, int* nl) {
  return fp64 ? inverse<double>((cpx<double>*)spec, (double*)out, d, C, tw, s, nl)
              : inverse<float>((cpx<float>*)spec, (float*)out, d, C, tw, s, nl);
}

cudaError_t launch_twiddles(bool fp64, int L, void* tw, cudaStream_t s) {
  if (fp64)
    twiddle_kernel<double><<<(L + 255) / 256, 256, 0, s>>>(L, (cpx<double>*)tw);
  else
    twiddle_kernel<float><<<(L + 255) / 256, 256, 0, s>>>(L, (cpx<float>*)tw);
  return cudaGetLastError();
}

}  // namespace pmmm
