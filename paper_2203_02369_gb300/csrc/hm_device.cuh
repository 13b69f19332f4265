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
  double f;
  const double dd = placeable(d);
  cell_axis(P.obs[0], dd, rx, P.delta, P.inv_delta, P.N, cx, f);
  cell_axis(P.obs[1], dd, ry, P.delta, P.inv_delta, P.N, cy, f);
  return cx * P.ksplit + cy / P.rq;
}

}  // namespace hm
