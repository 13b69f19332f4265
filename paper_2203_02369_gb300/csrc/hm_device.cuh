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

__device__ __forceinline__ void cell_axis(double o, double d, double r, double delta, int N, int& i,
                                          double& f) {
  const double t = __ddiv_rn(__dadd_rn(o, __dmul_rn(d, r)), delta);
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
  cell_axis(P.obs[0], dd, rx, P.delta, P.N, cx, f);
  cell_axis(P.obs[1], dd, ry, P.delta, P.N, cy, f);
  return cx * P.ksplit + cy / P.rq;
}

}  // namespace hm
