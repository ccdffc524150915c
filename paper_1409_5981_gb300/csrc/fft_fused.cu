// Whole 3-D real FFT of one channel per CTA, for FP32 meshes whose half
// spectrum of the physical z planes fits in shared memory and whose transform
// lengths are at most 32 (32^3 periodic, 16^3 open and smaller).  Same
// transforms, layout and conventions as fft.cu (Sec. 2.1, App. C): spectra
// [channel][Lz][Ly][hx], forward exp(-2 pi i jk/L), inverse unnormalised.
//
//   forward: x pass (two real rows per complex transform) from global memory
//            into shared memory, rows y >= ny and planes z >= nz never stored;
//            y pass in place; z pass from shared memory straight to the spectrum.
//   inverse: z pass from the spectrum into shared memory (planes z < nz), y pass
//            in place (rows y < ny kept), x pass to the real rows x < nx.
// Every 1-D transform is held by one thread in registers: a radix-2
// decimation-in-frequency FFT with all indices known at compile time, twiddles
// broadcast from shared memory, output in bit-reversed order (reindexed at the
// store).  Each channel is read and written once.
#include "internal.cuh"

namespace pmmm {

namespace {

constexpr int FF_MAX_L = 32;

template <int L>
__host__ __device__ constexpr int bitrev(int k) {
  int r = 0;
  for (int b = 1, m = L >> 1; b < L; b <<= 1, m >>= 1)
    if (k & b) r |= m;
  return r;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}

// In-register DIF FFT; on return v[bitrev(k)] holds X_k.  tw[t] = exp(-2 pi i t / L);
// the inverse uses the conjugates.
template <int L, bool INV>
__device__ __forceinline__ void fft_reg(float2 (&v)[L], const float2* __restrict__ tw) {
#pragma unroll
  for (int half = L / 2; half >= 1; half >>= 1) {
    const int ts = L / (2 * half);
#pragma unroll
    for (int b = 0; b < L; b += 2 * half) {
#pragma unroll
      for (int j = 0; j < half; ++j) {
        const float2 a = v[b + j], c = v[b + j + half];
        v[b + j] = make_float2(a.x + c.x, a.y + c.y);
        const float2 d = make_float2(a.x - c.x, a.y - c.y);
        if (j == 0) {
          v[b + j + half] = d;
        } else {
          float2 w = tw[j * ts];
          if (INV) w.y = -w.y;
          v[b + j + half] = cmul(d, w);
        }
      }
    }
  }
}

struct FFArgs {
  int nx, ny, nz, Lx, Ly, Lz, hx;
  int64_t Kh;
};

// ---------------------------------------------------------------- forward passes
template <int LX>
__device__ __forceinline__ void fwd_x(const float* __restrict__ src, float2* S, const FFArgs& a, int pr,
                                      const float2* tw) {
  const int nrows = a.nz * a.ny;
  const int r0 = 2 * pr, r1 = r0 + 1;
  const bool has1 = r1 < nrows;
  float2 v[LX];
#pragma unroll
  for (int t = 0; t < LX; ++t) v[t] = make_float2(0.f, 0.f);
  const float* p0 = src + (int64_t)r0 * a.nx;
  const float* p1 = src + (int64_t)r1 * a.nx;
  if ((a.nx & 3) == 0) {
#pragma unroll
    for (int t = 0; t < LX; t += 4) {
      if (t < a.nx) {
        const float4 x0 = *reinterpret_cast<const float4*>(p0 + t);
        const float4 x1 = has1 ? *reinterpret_cast<const float4*>(p1 + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[t] = make_float2(x0.x, x1.x);
        if (t + 1 < LX) v[t + 1] = make_float2(x0.y, x1.y);
        if (t + 2 < LX) v[t + 2] = make_float2(x0.z, x1.z);
        if (t + 3 < LX) v[t + 3] = make_float2(x0.w, x1.w);
      }
    }
  } else {
#pragma unroll
    for (int t = 0; t < LX; ++t)
      if (t < a.nx) v[t] = make_float2(p0[t], has1 ? p1[t] : 0.f);
  }
  fft_reg<LX, false>(v, tw);
  const int z0 = r0 / a.ny, y0 = r0 - z0 * a.ny, z1 = r1 / a.ny, y1 = r1 - z1 * a.ny;
  float2* o0 = S + ((int64_t)z0 * a.Ly + y0) * a.hx;
  float2* o1 = S + ((int64_t)z1 * a.Ly + y1) * a.hx;
#pragma unroll
  for (int k = 0; k <= LX / 2; ++k) {
    const float2 Z = v[bitrev<LX>(k)], Zm = v[bitrev<LX>((LX - k) & (LX - 1))];
    // X = (Z + conj Z_-k) / 2 ;  Y = (Z - conj Z_-k) / (2i)
    o0[k] = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
    if (has1) o1[k] = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
  }
}

template <int LY>
__device__ __forceinline__ void fwd_y(float2* S, const FFArgs& a, int col, const float2* tw) {
  const int z = col / a.hx, x = col - z * a.hx;
  float2* base = S + (int64_t)z * a.Ly * a.hx + x;
  float2 v[LY];
#pragma unroll
  for (int t = 0; t < LY; ++t) v[t] = t < a.ny ? base[t * a.hx] : make_float2(0.f, 0.f);
  fft_reg<LY, false>(v, tw);
#pragma unroll
  for (int t = 0; t < LY; ++t) base[t * a.hx] = v[bitrev<LY>(t)];
}

template <int LZ>
__device__ __forceinline__ void fwd_z(const float2* S, float2* __restrict__ dst, const FFArgs& a, int col,
                                      const float2* tw) {
  const int64_t plane = (int64_t)a.Ly * a.hx;
  float2 v[LZ];
#pragma unroll
  for (int t = 0; t < LZ; ++t) v[t] = t < a.nz ? S[t * plane + col] : make_float2(0.f, 0.f);
  fft_reg<LZ, false>(v, tw);
#pragma unroll
  for (int t = 0; t < LZ; ++t) dst[t * plane + col] = v[bitrev<LZ>(t)];
}

// ---------------------------------------------------------------- inverse passes
template <int LZ>
__device__ __forceinline__ void inv_z(const float2* __restrict__ src, float2* S, const FFArgs& a, int col,
                                      const float2* tw) {
  const int64_t plane = (int64_t)a.Ly * a.hx;
  float2 v[LZ];
#pragma unroll
  for (int t = 0; t < LZ; ++t) v[t] = src[t * plane + col];
  fft_reg<LZ, true>(v, tw);
#pragma unroll
  for (int t = 0; t < LZ; ++t)
    if (t < a.nz) S[t * plane + col] = v[bitrev<LZ>(t)];
}

template <int LY>
__device__ __forceinline__ void inv_y(float2* S, const FFArgs& a, int col, const float2* tw) {
  const int z = col / a.hx, x = col - z * a.hx;
  float2* base = S + (int64_t)z * a.Ly * a.hx + x;
  float2 v[LY];
#pragma unroll
  for (int t = 0; t < LY; ++t) v[t] = base[t * a.hx];
  fft_reg<LY, true>(v, tw);
#pragma unroll
  for (int t = 0; t < LY; ++t)
    if (t < a.ny) base[t * a.hx] = v[bitrev<LY>(t)];
}

// Writes the real rows into `rows` (shared memory, nz*ny*nx floats) after the
// caller's barrier; the rows reuse the spectrum's storage.
template <int LX>
__device__ __forceinline__ void inv_x(const float2* S, float* rows, const FFArgs& a, int pr, const float2* tw) {
  const int nrows = a.nz * a.ny;
  const bool mine = 2 * pr < nrows;  // threads past the last pair only join the barrier
  if (!mine) pr = 0;
  const int r0 = 2 * pr, r1 = r0 + 1;
  const bool has1 = mine && r1 < nrows;
  const int z0 = r0 / a.ny, y0 = r0 - z0 * a.ny, z1 = r1 / a.ny, y1 = r1 - z1 * a.ny;
  const float2* i0 = S + ((int64_t)z0 * a.Ly + y0) * a.hx;
  const float2* i1 = S + ((int64_t)z1 * a.Ly + y1) * a.hx;
  float2 v[LX];
#pragma unroll
  for (int k = 0; k <= LX / 2; ++k) {
    const float2 A = i0[k], B = has1 ? i1[k] : make_float2(0.f, 0.f);
    // Z_k = A_k + i B_k, and Z_{L-k} = conj(A_k) + i conj(B_k) (Hermitian rows)
    v[k] = make_float2(A.x - B.y, A.y + B.x);
    if (k > 0 && k < LX / 2) v[LX - k] = make_float2(A.x + B.y, -A.y + B.x);
  }
  fft_reg<LX, true>(v, tw);
  __syncthreads();  // every thread has read its half spectra before the rows overwrite them
  // element x of row r is staged at r*nx + ((x + r/2) mod nx): the row pairs of
  // neighbouring threads start on different banks
  float* p0 = rows + (int64_t)r0 * a.nx;
  float* p1 = rows + (int64_t)r1 * a.nx;
  const int rot = pr & (a.nx - 1);
#pragma unroll
  for (int t = 0; t < LX; ++t)
    if (mine && t < a.nx) {
      const float2 z = v[bitrev<LX>(t)];
      const int xs = (t + rot) & (a.nx - 1);
      p0[xs] = z.x;
      if (has1) p1[xs] = z.y;
    }
}

#define FF_DISPATCH(L, CALL)             \
  switch (L) {                           \
    case 2: { constexpr int LL = 2; CALL; } break;   \
    case 4: { constexpr int LL = 4; CALL; } break;   \
    case 8: { constexpr int LL = 8; CALL; } break;   \
    case 16: { constexpr int LL = 16; CALL; } break; \
    case 32: { constexpr int LL = 32; CALL; } break; \
    default: break;                      \
  }

constexpr int FF_THREADS = 512;  // 128 registers per thread: the 32-point transforms stay in registers

__global__ void __launch_bounds__(FF_THREADS, 1) fft3_fwd_kernel(const float* __restrict__ in, float2* __restrict__ spec,
                                                                FFArgs a, const float2* __restrict__ twx,
                                                                const float2* __restrict__ twy,
                                                                const float2* __restrict__ twz) {
  extern __shared__ __align__(16) unsigned char ff_smem[];
  float2* tx = reinterpret_cast<float2*>(ff_smem);
  float2* ty = tx + FF_MAX_L;
  float2* tz = ty + FF_MAX_L;
  float2* S = tz + FF_MAX_L;
  const int tid = threadIdx.x;
  for (int t = tid; t < FF_MAX_L; t += blockDim.x) {
    if (t < a.Lx) tx[t] = twx[t];
    if (t < a.Ly) ty[t] = twy[t];
    if (t < a.Lz) tz[t] = twz[t];
  }
  __syncthreads();
  const int64_t c = blockIdx.x;
  const float* src = in + c * a.nz * a.ny * a.nx;
  const int npairs = (a.nz * a.ny + 1) / 2;
  for (int pr = tid; pr < npairs; pr += blockDim.x) FF_DISPATCH(a.Lx, fwd_x<LL>(src, S, a, pr, tx));
  __syncthreads();
  for (int col = tid; col < a.nz * a.hx; col += blockDim.x) FF_DISPATCH(a.Ly, fwd_y<LL>(S, a, col, ty));
  __syncthreads();
  float2* dst = spec + c * a.Kh;
  for (int col = tid; col < a.Ly * a.hx; col += blockDim.x) FF_DISPATCH(a.Lz, fwd_z<LL>(S, dst, a, col, tz));
}

__global__ void __launch_bounds__(FF_THREADS, 1) fft3_inv_kernel(const float2* __restrict__ spec, float* __restrict__ out,
                                                                FFArgs a, const float2* __restrict__ twx,
                                                                const float2* __restrict__ twy,
                                                                const float2* __restrict__ twz) {
  extern __shared__ __align__(16) unsigned char ff_smem[];
  float2* tx = reinterpret_cast<float2*>(ff_smem);
  float2* ty = tx + FF_MAX_L;
  float2* tz = ty + FF_MAX_L;
  float2* S = tz + FF_MAX_L;
  const int tid = threadIdx.x;
  for (int t = tid; t < FF_MAX_L; t += blockDim.x) {
    if (t < a.Lx) tx[t] = twx[t];
    if (t < a.Ly) ty[t] = twy[t];
    if (t < a.Lz) tz[t] = twz[t];
  }
  __syncthreads();
  const int64_t c = blockIdx.x;
  const float2* src = spec + c * a.Kh;
  for (int col = tid; col < a.Ly * a.hx; col += blockDim.x) FF_DISPATCH(a.Lz, inv_z<LL>(src, S, a, col, tz));
  __syncthreads();
  for (int col = tid; col < a.nz * a.hx; col += blockDim.x) FF_DISPATCH(a.Ly, inv_y<LL>(S, a, col, ty));
  __syncthreads();
  // x pass: one row pair per thread (npairs <= blockDim, see fft_fused_applies);
  // the real rows go to shared memory, then out with coalesced 16-byte stores
  float* rows = reinterpret_cast<float*>(S);
  FF_DISPATCH(a.Lx, inv_x<LL>(S, rows, a, tid, tx));
  __syncthreads();
  const int64_t nreal = (int64_t)a.nz * a.ny * a.nx;
  float* dst = out + c * nreal;
  const int nxm = a.nx - 1;
  auto staged = [&](int64_t i) {
    const int64_t r = i / a.nx;
    const int x = (int)(i - r * a.nx);
    return rows[r * a.nx + ((x + (int)(r >> 1)) & nxm)];
  };
  if ((nreal & 3) == 0 && (a.nx & 3) == 0) {
    for (int64_t i = tid; i < nreal / 4; i += blockDim.x)
      reinterpret_cast<float4*>(dst)[i] = make_float4(staged(4 * i), staged(4 * i + 1), staged(4 * i + 2),
                                                       staged(4 * i + 3));
  } else {
    for (int64_t i = tid; i < nreal; i += blockDim.x) dst[i] = staged(i);
  }
}

size_t fused_smem(const Dims& d) { return sizeof(float2) * (3 * FF_MAX_L + (size_t)d.nz * d.Ly * d.hx); }

FFArgs ff_args(const Dims& d) {
  FFArgs a;
  a.nx = d.nx;
  a.ny = d.ny;
  a.nz = d.nz;
  a.Lx = d.Lx;
  a.Ly = d.Ly;
  a.Lz = d.Lz;
  a.hx = d.hx;
  a.Kh = d.Kh;
  return a;
}

}  // namespace

bool fft_fused_applies(bool fp64, const Dims& d) {
  return !fp64 && d.Lx <= FF_MAX_L && d.Ly <= FF_MAX_L && d.Lz <= FF_MAX_L && d.Lx >= 2 && d.Ly >= 2 &&
         d.Lz >= 2 && fused_smem(d) <= 200 * 1024 && (d.nz * d.ny + 1) / 2 <= FF_THREADS &&
         (int64_t)d.nz * d.Ly * d.hx * 2 >= (int64_t)d.nz * d.ny * d.nx;
}

cudaError_t launch_fft_fused_forward(const void* in, void* spec, const Dims& d, int C, const FftTw& tw, cudaStream_t s,
                                     int* nl) {
  if (C <= 0) return cudaSuccess;
  const size_t smem = fused_smem(d);
  cudaError_t e = cudaFuncSetAttribute(fft3_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fft3_fwd_kernel<<<(unsigned)C, FF_THREADS, smem, s>>>((const float*)in, (float2*)spec, ff_args(d),
                                                         (const float2*)tw.x, (const float2*)tw.y, (const float2*)tw.z);
  ++*nl;
  return cudaGetLastError();
}

cudaError_t launch_fft_fused_inverse(const void* spec, void* out, const Dims& d, int C, const FftTw& tw, cudaStream_t s,
                                     int* nl) {
  if (C <= 0) return cudaSuccess;
  const size_t smem = fused_smem(d);
  cudaError_t e = cudaFuncSetAttribute(fft3_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fft3_inv_kernel<<<(unsigned)C, FF_THREADS, smem, s>>>((const float2*)spec, (float*)out, ff_args(d),
                                                         (const float2*)tw.x, (const float2*)tw.y, (const float2*)tw.z);
  ++*nl;
  return cudaGetLastError();
}

}  // namespace pmmm
