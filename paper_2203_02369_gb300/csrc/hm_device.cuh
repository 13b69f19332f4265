// Device helpers shared by the point and HMC kernels.
#pragma once
#include "hm_internal.h"

namespace hm {

// Lower-corner cell and fractional offsets of x = o + d rhat, formed as
// t = (o + d*r)/Delta with one IEEE rounding per operation (no contraction),
// so that the cell indices are reproducible bit for bit on any IEEE host.
struct CellPos {
  int ix, iy, iz;
  double fx, fy, fz;
};

// The quotient is first formed as x * (1/Delta) (one multiply instead of a
// correctly rounded division, which costs many FP64 instructions on this
// part).  That product is within 3 ulp of x/Delta, so its floor equals the
// floor of the correctly rounded quotient unless x/Delta lies within a few
// ulp of an integer; there (rarely) the quotient is recomputed with the IEEE
// division, so the cell indices stay bit for bit those of floor(x/Delta).
// The fractional offset may differ from t - floor(t) of the IEEE quotient by
// a few ulp of t.
__device__ __forceinline__ void cell_axis(double o, double d, double r, double delta, double inv_delta, int N,
                                          int& i, double& f) {
  const double x = __dadd_rn(o, __dmul_rn(d, r));
  double t = __dmul_rn(x, inv_delta);
  if (fabs(t - rint(t)) <= 16.0 * 1.1102230246251565e-16 * fabs(t)) t = __ddiv_rn(x, delta);
  const double fl = floor(t);
  f = __dadd_rn(t, -fl);
  long long ii = (long long)fl;
  ii %= N;
  if (ii < 0) ii += N;
  i = (int)ii;
}

// ---------------------------------------------------------------------------
// The same cells from FP32 double-float arithmetic (the FP64 pipe of this part
// is narrow).  Every quantity is a float pair hi + lo carrying about 44
// significant bits: products by FMA (the exact error of hi*hi plus the cross
// terms), sums by Knuth's TwoSum.  For |t| < 2^11 the pair t_df is within
// 2^-33 of the exact (o + d r)/Delta, and the FP64 quotient of cell_axis
// within 2^-40 of it.  The fraction fr = t_df - floor is rounded to a float
// (to 2^-24 near 1), so the screen asks for 2^-20 < fr < 1 - 2^-20: then the
// floors of all three agree and the cell index is the bit-exact one.
// Otherwise (about one point in 10^6, or |t| >= 2^11) the caller falls back
// to cell_axis.  The fractional offset is FP32-accurate.
// ---------------------------------------------------------------------------

// v = hi + lo with hi its leading 24 significant bits (truncated) and lo the
// rest, from the bits alone (no FP64 instruction).  |v| < 2^-74 is taken as 0
// (an absolute error below 2^-74); false for |v| >= 2^100 or non-finite v.
__device__ __forceinline__ bool split_df(double v, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ue = (int)((b >> 52) & 0x7ff) - 1023;
  if (ue < -74) {
    hi = lo = 0.0f;
    return true;
  }
  if (ue >= 100) return false;
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;   // 52 fraction bits
  hi = __int_as_float((int)(sgn | ((unsigned)(ue + 127) << 23) | (unsigned)(m >> 29)));
  const float l = __fmul_rn(__uint2float_rn((unsigned)(m & 0x1FFFFFFFull)), __int_as_float((ue - 52 + 127) << 23));
  lo = sgn ? -l : l;
  return true;
}

__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Cell and fractional offset of t = (o + d r)/Delta on one axis from the
// float pairs o = (oh, ol), d = (dh, dl), 1/Delta = (ih, il); false when the
// screen above cannot decide.
__device__ __forceinline__ bool cell_axis_df(float oh, float ol, float dh, float dl, double r, float ih, float il,
                                             int N, int& i, float& f) {
  float rh, rl;
  if (!split_df(r, rh, rl)) return false;
  // p = d r
  const float p = __fmul_rn(dh, rh);
  float pe = __fmaf_rn(dh, rh, -p);
  pe = __fmaf_rn(dh, rl, pe);
  pe = __fmaf_rn(dl, rh, pe);
  // x = o + p
  float s, se;
  two_sum_f(oh, p, s, se);
  se = __fadd_rn(se, __fadd_rn(ol, pe));
  float xh, xl;
  two_sum_f(s, se, xh, xl);
  // t = x / Delta
  const float th = __fmul_rn(xh, ih);
  float te = __fmaf_rn(xh, ih, -th);
  te = __fmaf_rn(xh, il, te);
  te = __fmaf_rn(xl, ih, te);
  if (!(fabsf(th) < 2048.0f)) return false;
  float fl = floorf(th);
  float fr = __fadd_rn(__fsub_rn(th, fl), te);   // th - fl is exact
  if (fr < 0.0f) {
    fl = __fsub_rn(fl, 1.0f);
    fr = __fadd_rn(fr, 1.0f);
  } else if (fr >= 1.0f) {
    fl = __fadd_rn(fl, 1.0f);
    fr = __fsub_rn(fr, 1.0f);
  }
  constexpr float kEdge = 9.5367431640625e-07f;   // 2^-20; 1 - 2^-20 is a float
  if (fr < kEdge || fr > 1.0f - kEdge) return false;
  int ii = (int)fl % N;
  if (ii < 0) ii += N;
  i = ii;
  f = fr;
  return true;
}

// A distance that cannot be placed on the grid (non-finite or absurdly
// large) is bucketed as if it sat at the observer; its likelihood term is
// +inf and its residual 0, so the plane passes ignore it.
__device__ __forceinline__ double placeable(double d) {
  return (isfinite(d) && fabs(d) < 1e7) ? d : 0.0;
}

// Bucket key of a point: x-plane of its lower CIC corner, then the CTA of
// that plane's cluster that owns its row cy.
__device__ __forceinline__ int bucket_key(const PointParams& P, double d, double rx, double ry) {
  int cx, cy;
  float dh, dl, ff;
  // placeable() from the split: it fails for non-finite d and for |d| >=
  // 2^100, and 1e7 is a float, so |dh| < 1e7 exactly when |d| < 1e7
  double dd = d;
  if (!split_df(d, dh, dl) || !(fabsf(dh) < 1e7f)) {
    dd = 0.0;
    dh = dl = 0.0f;
  }
  const bool ok = cell_axis_df(P.obs_hi[0], P.obs_lo[0], dh, dl, rx, P.inv_delta_hi, P.inv_delta_lo, P.N, cx, ff) &&
                  cell_axis_df(P.obs_hi[1], P.obs_lo[1], dh, dl, ry, P.inv_delta_hi, P.inv_delta_lo, P.N, cy, ff);
  if (!ok) {
    double f;
    cell_axis(P.obs[0], dd, rx, P.delta, P.inv_delta, P.N, cx, f);
    cell_axis(P.obs[1], dd, ry, P.delta, P.inv_delta, P.N, cy, f);
  }
  return cx * P.ksplit + cy / P.rq;
}

}  // namespace hm
