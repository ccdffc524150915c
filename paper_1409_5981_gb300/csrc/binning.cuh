// Cell index along one axis, shared by the binning kernels (sort.cu, batch.cu).
//
// Cell index, in FP64 with every operation rounded (no contraction):
//   t = x - lo;  if t is outside [0, len):
//     periodic: t = t - len * floor(t / len), and t -= len if t >= len
//     open: flag OUT_OF_BOX
//   i = floor(t * (n / len)) clamped to [0, n-1]
#pragma once
#include <type_traits>

#include "internal.cuh"

namespace pmmm {

// Returns the cell index along one axis; error bits are OR-ed into *bits (a
// register of the caller), the binned coordinate t is stored in *tout.
__device__ __forceinline__ int bin_axis(double x, double lo, double len, double inv, int n, int periodic, int* bits,
                                        double* tout) {
  if (!isfinite(x)) {
    *bits |= ERRBIT_NONFINITE;
    *tout = 0.0;
    return 0;
  }
  double t = __dsub_rn(x, lo);
  if (!(t >= 0.0 && t < len)) {
    if (periodic) {
      const double qd = __ddiv_rn(t, len);
      const double fl = floor(qd);
      t = __dsub_rn(t, __dmul_rn(len, fl));
      if (t >= len) t = __dsub_rn(t, len);
    } else {
      *bits |= ERRBIT_OUT_OF_BOX;
    }
  }
  *tout = t;
  const double f = floor(__dmul_rn(t, inv));
  if (!(f >= 0.0)) return 0;
  if (f > (double)(n - 1)) return n - 1;
  return (int)f;
}

// FP32 inputs: the cell index of the FP64 formula without FP64 arithmetic.
// s = (x - lo) * inv is formed in double-float arithmetic (t = th + tl by an
// exact two-sum, s = sh + sl with an exact product error term), which is within
// 2^-44 |s| of the FP64 formula's rounded s.  When the fractional part of s is
// more than 1e-6 away from an integer and the cell lies inside the box, floor(s)
// therefore equals the FP64 result exactly; otherwise (a particle within 1e-6
// cell of a face, outside the box or not finite) the caller takes the FP64 path.
// u = frac(s) - 1/2 in cell units, times h / hs.
__device__ __forceinline__ bool bin_axis_fast(float x, const Geo& g, int a, int* ix, float* u) {
  const float th = x - g.loh[a];
  const float bv = th - x;
  float tl = (x - (th - bv)) + (-g.loh[a] - bv);
  tl -= g.lol[a];
  const float sh = th * g.invh[a];
  float sl = fmaf(th, g.invh[a], -sh);
  sl = fmaf(th, g.invl[a], sl);
  sl = fmaf(tl, g.invh[a], sl);
  float fl = floorf(sh);
  float fr = (sh - fl) + sl;
  if (fr < 0.f) {
    fl -= 1.f;
    fr += 1.f;
  } else if (fr >= 1.f) {
    fl += 1.f;
    fr -= 1.f;
  }
  if (!(fr > 1e-6f && fr < 1.f - 1e-6f)) return false;
  if (!(fl >= 0.f && fl <= (float)(g.n[a] - 1))) return false;
  *ix = (int)fl;
  *u = (fr - 0.5f) * g.csf[a];
  return true;
}

// Bins particle i: writes its key key0 + cell id and its record (u_x, u_y, u_z, q)
// in input order, u being the position relative to the cell centre in units of
// hs, rounded to T.  FP32 inputs take the fast path where it is exact.
template <typename T>
__device__ __forceinline__ void bin_record(const T* __restrict__ pos, const T* __restrict__ q, int64_t i,
                                           const Geo& g, uint32_t key0, uint32_t* __restrict__ keys,
                                           T* __restrict__ rec, int* __restrict__ err) {
  int ix[3];
  T u[3];
  bool fast = false;
  if (sizeof(T) == 4) {
    float uf[3];
    fast = bin_axis_fast((float)pos[3 * i + 0], g, 0, &ix[0], &uf[0]) &&
           bin_axis_fast((float)pos[3 * i + 1], g, 1, &ix[1], &uf[1]) &&
           bin_axis_fast((float)pos[3 * i + 2], g, 2, &ix[2], &uf[2]);
    if (fast)
      for (int a = 0; a < 3; ++a) u[a] = (T)uf[a];
  }
  if (!fast) {
    double t[3];
    int bits = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      ix[a] = bin_axis((double)pos[3 * i + a], g.lo[a], g.len[a], g.inv[a], g.n[a], g.periodic, &bits, &t[a]);
    if (bits) set_err(err, bits);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double rel = t[a] - (double)(2 * ix[a] + 1) * g.hh[a];  // relative to the cell centre
      u[a] = (T)(rel * g.ihs);
    }
  }
  keys[i] = key0 + (uint32_t)(ix[0] + g.n[0] * (ix[1] + g.n[1] * ix[2]));
  using V = typename std::conditional<sizeof(T) == 4, float4, double4>::type;
  V o;
  o.x = u[0];
  o.y = u[1];
  o.z = u[2];
  o.w = q[i];
  reinterpret_cast<V*>(rec)[i] = o;
}

}  // namespace pmmm
