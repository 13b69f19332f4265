// Point-side kernels of the HAMLET posterior: positions and cells (bit-exact
// index work), the bucketing of the points by x-plane for the plane passes
// that run the CIC gather and scatter (hm_fft_kernels.cu), the likelihood
// terms with their gradients (eqs. lmu, vrobs, lvr, kappa, D; FP32 terms
// with FP64 sums on the FP32 path, FP64 throughout on the FP64 path), the
// leapfrog update of the distances (mass matrix eq. M_ab: (sigma_v/H0)^2 for
// d) and the stable cell sort.
#include "hm_fft.cuh"
#include "hm_internal.h"
#include "hm_device.cuh"

namespace hm {

constexpr int kPtsNT = 128;

__device__ __forceinline__ CellPos cell_of(const PointParams& P, double d, double rx, double ry, double rz) {
  CellPos c;
  cell_axis(P.obs[0], d, rx, P.delta, P.inv_delta, P.N, c.ix, c.fx);
  cell_axis(P.obs[1], d, ry, P.delta, P.inv_delta, P.N, c.iy, c.fy);
  cell_axis(P.obs[2], d, rz, P.delta, P.inv_delta, P.N, c.iz, c.fz);
  return c;
}

// The FP32 path's cells: the double-float screen (same indices, FP32
// offsets), FP64 for a point the screen cannot decide.
__device__ __forceinline__ CellPos cell_of_f32(const PointParams& P, double d, double rx, double ry, double rz) {
  CellPos c;
  float dh, dl, fx, fy, fz;
  const float ih = P.inv_delta_hi, il = P.inv_delta_lo;
  if (split_df(d, dh, dl) && cell_axis_df(P.obs_hi[0], P.obs_lo[0], dh, dl, rx, ih, il, P.N, c.ix, fx) &&
      cell_axis_df(P.obs_hi[1], P.obs_lo[1], dh, dl, ry, ih, il, P.N, c.iy, fy) &&
      cell_axis_df(P.obs_hi[2], P.obs_lo[2], dh, dl, rz, ih, il, P.N, c.iz, fz)) {
    c.fx = fx;
    c.fy = fy;
    c.fz = fz;
    return c;
  }
  return cell_of(P, d, rx, ry, rz);
}

// ln pi_D(d) and its derivative; returns false outside the support.  The
// table (eq. D's histogram) gives ln pi at the bin centres d0 + (b + 1/2) bin,
// interpolated linearly in between and flat in the outer half bins, so the
// potential stays continuous across bins.
__device__ __forceinline__ bool log_prior(const PointParams& P, double d, double& lp, double& dlp) {
  if (P.prior_kind == PRIOR_TABLE) {
    const int nb = P.prior_nbins;
    if (!(d >= P.prior_d0 && d < P.prior_d0 + nb * P.prior_bin)) return false;
    const double t = (d - P.prior_d0) / P.prior_bin - 0.5;
    const double b = floor(t);
    const double f = t - b;
    if (b < 0.0) {
      lp = P.prior_logdens[0];
      dlp = 0.0;
    } else if (b >= (double)(nb - 1)) {
      lp = P.prior_logdens[nb - 1];
      dlp = 0.0;
    } else {
      const int ib = (int)b;
      const double a0 = P.prior_logdens[ib], a1 = P.prior_logdens[ib + 1];
      lp = (1.0 - f) * a0 + f * a1;
      dlp = (a1 - a0) / P.prior_bin;
    }
    return true;
  }
  if (!(d >= P.prior_dmin && d <= P.prior_dmax)) return false;
  lp = P.prior_alpha * log(d);
  dlp = P.prior_alpha / d;
  return true;
}

// The prior table read in FP32 on the FP32 path: the support test stays in
// FP64 (it decides +inf exactly as the FP64 path does), the interpolation
// between bin centres runs in FP32 (ln pi and its slope to ~1e-7 relative).
__device__ __forceinline__ bool log_prior_f32(const PointParams& P, double d, float& lp, float& dlp) {
  if (P.prior_kind == PRIOR_TABLE) {
    const int nb = P.prior_nbins;
    if (!(d >= P.prior_d0 && d < P.prior_d0 + nb * P.prior_bin)) return false;
    const float t = (float)(d - P.prior_d0) / (float)P.prior_bin - 0.5f;
    const float b = floorf(t);
    const float f = t - b;
    if (b < 0.0f) {
      lp = (float)P.prior_logdens[0];
      dlp = 0.0f;
    } else if (b >= (float)(nb - 1)) {
      lp = (float)P.prior_logdens[nb - 1];
      dlp = 0.0f;
    } else {
      const int ib = (int)b;
      const float a0 = (float)P.prior_logdens[ib], a1 = (float)P.prior_logdens[ib + 1];
      lp = (1.0f - f) * a0 + f * a1;
      dlp = (a1 - a0) / (float)P.prior_bin;
    }
    return true;
  }
  if (!(d >= P.prior_dmin && d <= P.prior_dmax)) return false;
  const float df = (float)d;
  lp = (float)P.prior_alpha * logf(df);
  dlp = (float)P.prior_alpha / df;
  return true;
}

// ---------------------------------------------------------------------------
// Bucketing by the x index of the lower CIC corner: counts (and the rank of
// each point inside its bucket, in atomic order) ...
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPtsNT)
k_points_prep(const PointParams* __restrict__ pp, PointArrays pa) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.y;
  const PointParams& P = pp[c];
  const long long il = (long long)blockIdx.x * kPtsNT + threadIdx.x;
  if (il >= P.pt_n) return;
  const long long i = P.pt_off + il;
  const int key = bucket_key(P, pa.d[i], pa.rx[i], pa.ry[i]);
  pa.cx[i] = key;
  pa.slot[i] = atomicAdd(&pa.cnt[c * P.N * P.ksplit + key], 1);
}

// The terms of the point likelihood that depend on d alone (eqs. lmu, vrobs,
// kappa, D) with their derivatives, FP64 path: everything in FP64.
//   lk[0] = A   = (mu_i - mu(d))^2/(2 s_mu^2) + ln kappa - ln pi_D(d)  (+inf outside)
//   lk[1] = A'  = dA/dd
//   lk[2] = v_obs(d), lk[3] = v_obs'(d), lk[4] = 1/kappa^2, lk[5] = (kappa^2)'
__device__ __forceinline__ void place_terms_fp64(const PointParams& P, PointArrays& pa, ChainScal* cs, int c,
                                                 long long i, double d) {
  const double om = P.omega_m;
  const double x = 1.0 - 3.0 * om * kH0 * d / kC;
  double lp = 0.0, dlp = 0.0;
  const bool ok = d > 0.0 && x > 0.0 && log_prior(P, d, lp, dlp) && !(cs[c].sample_sig && !(cs[c].sig > 0.0));
  const long long nt = pa.ntot;
  if (!ok) {
    pa.lk[i] = __longlong_as_double(0x7ff0000000000000LL);  // +inf
    for (int k = 1; k < 6; ++k) pa.lk[k * nt + i] = 0.0;
    atomicOr(&cs[c].status, STATUS_DOMAIN);
    return;
  }
  const double sq = sqrt(x);
  const double zb = 2.0 / (3.0 * om) * (1.0 - sq);
  const double zbp = (kH0 / kC) / sq;
  const double opz = 1.0 + zb;
  const double iopz = 1.0 / opz;
  const double mu_d = 5.0 * log10(d * opz / P.h) + 25.0;
  const double mup = (5.0 / 2.302585092994045684) * (1.0 / d + zbp * iopz);
  const double z = pa.zobs[i];
  const double scz = pa.scz[i];
  // kappa^2 = sigma_NL^2 + sigma_cz^2 / (1 + zbar)^2 (eq. kappa); with
  // sigma_cz = 0 and a fixed sigma_NL it is a per-chain constant
  double ik2, lk2, k2p;
  if (scz == 0.0 && !cs[c].sample_sig) {
    ik2 = P.ik2_nl;
    lk2 = P.logk2_nl;
    k2p = 0.0;
  } else {
    const double scz2 = scz * scz;
    const double snl2 = cs[c].sample_sig ? cs[c].sig * cs[c].sig : P.sigma_nl2;
    const double k2 = snl2 + scz2 * iopz * iopz;
    ik2 = 1.0 / k2;
    lk2 = log(k2);
    k2p = -2.0 * scz2 * zbp * iopz * iopz * iopz;
  }
  const double ismu2 = pa.ismu2[i];
  const double res_mu = pa.mu[i] - mu_d;
  pa.lk[i] = 0.5 * res_mu * res_mu * ismu2 + 0.5 * lk2 - lp;
  const double t[5] = {-res_mu * mup * ismu2 + 0.5 * k2p * ik2 - dlp, kC * (z - zb) * iopz,
                       -kC * zbp * (1.0 + z) * iopz * iopz, ik2, k2p};
#pragma unroll
  for (int k = 0; k < 5; ++k) pa.lk[(k + 1) * nt + i] = t[k];
}

// The same terms on the FP32 path, where only the per-point sums and the
// energies need FP64.  Two differences cancel: z - zbar(d), a thousandth of
// z at these distances (the observed velocity is c (z - zbar)/(1 + zbar)),
// and mu_i - mu(d), a few tenths of ~35 mag.  With s = sqrt(1 - k3 d) and
// the per-point constants of XRef (d_z: zbar(d_z) = z; d_ref: x(d_ref) =
// x_ref, x(d) = d (1 + zbar)/h the luminosity distance in Mpc):
//   z - zbar(d)  = e_z - c23 k3 (d - d_z)/(s + s_z),
//   x(d) - x_ref = e_ref + (d - d_ref)/h [1 + zbar(d) + c23 k3 d_ref/(s + s_ref)],
// (zbar(a) - zbar(b) = c23 (s_b - s_a) = c23 k3 (a - b)/(s_a + s_b)), and
// mu_i - mu(d) = -(5/ln 10) ln(1 + (x - x_ref)/x_ref).  The two distance
// differences are formed from float pairs (TwoSum), so every term runs in
// FP32; the domain test and the sum A stay in FP64.  Layout: lk[0..nt)
// doubles A; then floats A', v_obs, v_obs', 1/kappa^2, (kappa^2)' at
// f[k nt + i], f = (float*)(lk + nt).
__device__ __forceinline__ float diff_df(float ah, float al, float bh, float bl) {
  float s, e;
  two_sum_f(ah, -bh, s, e);
  return __fadd_rn(s, __fadd_rn(e, __fsub_rn(al, bl)));
}

__device__ __forceinline__ void place_terms_fp32(const PointParams& P, PointArrays& pa, ChainScal* cs, int c,
                                                 long long i, double d) {
  const long long nt = pa.ntot;
  float* f = reinterpret_cast<float*>(pa.lk + nt);
  const double om1 = 1.0 - P.k3 * d;
  float lp = 0.0f, dlp = 0.0f;
  const bool ok = d > 0.0 && om1 > 0.0 && log_prior_f32(P, d, lp, dlp) && !(cs[c].sample_sig && !(cs[c].sig > 0.0));
  if (!ok) {
    pa.lk[i] = __longlong_as_double(0x7ff0000000000000LL);  // +inf
    for (int k = 0; k < 5; ++k) f[k * nt + i] = 0.0f;
    atomicOr(&cs[c].status, STATUS_DOMAIN);
    return;
  }
  const XRef xr = pa.xr[i];
  float dh, dl;
  split_df(d, dh, dl);            // 0 < d < 1/k3: always representable
  const float df = __fadd_rn(dh, dl);
  const float ck = P.c23k3_f;
  const float s = sqrtf(__fmaf_rn(-P.k3_f, df, 1.0f));
  const float zb = ck * df / (1.0f + s);          // c23 (1 - s) without cancellation
  const float opz = 1.0f + zb;
  const float iopz = 1.0f / opz;
  const float zmzb = xr.e_z - ck * diff_df(dh, dl, xr.dz_hi, xr.dz_lo) / (s + xr.s_z);
  const float dref = xr.dr_hi + xr.dr_lo;
  const float xmxr = xr.e_ref + diff_df(dh, dl, xr.dr_hi, xr.dr_lo) * P.inv_h_f * (opz + ck * dref / (xr.s_ref + s));
  const float xref = dref * (1.0f + ck * dref / (1.0f + xr.s_ref)) * P.inv_h_f - xr.e_ref;
  constexpr float k5ln10 = 2.1714724095162591f;                       // 5 / ln 10
  const float res_mu = -k5ln10 * log1pf(xmxr / xref);
  const float zbp = (float)(kH0 / kC) / s;                              // dzbar/dd
  const float mup = k5ln10 * (1.0f / df + zbp * iopz);
  const float vo = (float)kC * zmzb * iopz;
  const float vop = -(float)kC * zbp * (1.0f + (zb + zmzb)) * iopz * iopz;
  // kappa^2 = sigma_NL^2 + sigma_cz^2/(1 + zbar)^2 (eq. kappa); with
  // sigma_cz = 0 and a fixed sigma_NL it is a per-chain constant
  const double scz = pa.scz[i];
  float ik2, k2p;
  double lk2;
  if ((__double_as_longlong(scz) << 1) == 0 && !cs[c].sample_sig) {
    ik2 = (float)P.ik2_nl;
    lk2 = P.logk2_nl;
    k2p = 0.0f;
  } else {
    const float scz2 = (float)scz * (float)scz;
    const float snl2 = cs[c].sample_sig ? (float)cs[c].sig * (float)cs[c].sig : (float)P.sigma_nl2;
    const float k2 = snl2 + scz2 * iopz * iopz;
    ik2 = 1.0f / k2;
    lk2 = (double)logf(k2);
    k2p = -2.0f * scz2 * zbp * iopz * iopz * iopz;
  }
  const float ismu2 = (float)pa.ismu2[i];
  pa.lk[i] = (double)(0.5f * res_mu * res_mu * ismu2 - lp) + 0.5 * lk2;
  f[i] = -res_mu * mup * ismu2 + 0.5f * k2p * ik2 - dlp;
  f[nt + i] = vo;
  f[2 * nt + i] = vop;
  f[3 * nt + i] = ik2;
  f[4 * nt + i] = k2p;
}

// ... then the bucket offsets, the bucket-ordered point records, and the
// d-only likelihood terms (place_terms_fp64 / place_terms_fp32 above).
template <typename T>
__global__ void __launch_bounds__(kPtsNT)
k_points_place(const PointParams* __restrict__ pp, PointArrays pa, ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  constexpr int kMaxNB = kMaxBuckets;   // sub-buckets per chain (N * ksplit)
  constexpr int PERT = kMaxNB / kPtsNT;
  __shared__ int excl[kMaxNB + 1];   // written for b <= NB < kMaxNB
  __shared__ int wsum[kPtsNT / 32];
  const int c = blockIdx.y;
  const PointParams& P = pp[c];
  const int N = P.N;
  const int NB = N * P.ksplit;
  {
    // exclusive scan of the NB counts: PERT per thread, then warp and block
    const int* cnt = pa.cnt + (long long)c * NB;
    int v[PERT];
    int loc = 0;
#pragma unroll
    for (int k = 0; k < PERT; ++k) {
      const int b = threadIdx.x * PERT + k;
      v[k] = b < NB ? cnt[b] : 0;
      loc += v[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    int base = 0;
    for (int w2 = 0; w2 < wid; ++w2) base += wsum[w2];
    int run = base + x - loc;
#pragma unroll
    for (int k = 0; k < PERT; ++k) {
      const int b = threadIdx.x * PERT + k;
      if (b <= NB) excl[b] = run;
      run += v[k];
    }
    __syncthreads();
  }
  if (blockIdx.x == 0) {
    for (int b = threadIdx.x; b <= NB; b += kPtsNT) pa.off[(long long)c * (NB + 1) + b] = (int)P.pt_off + excl[b];
    // the other count half is free now: clear it for the likelihood kernel's counting
    for (int b = threadIdx.x; b < NB; b += kPtsNT) pa.cnt_next[(long long)c * NB + b] = 0;
  }
  const long long il = (long long)blockIdx.x * kPtsNT + threadIdx.x;
  if (il >= P.pt_n) return;
  const long long i = P.pt_off + il;
  const double rx = pa.rx[i], ry = pa.ry[i], rz = pa.rz[i];
  const double d = pa.d[i];
  const CellPos cp = (sizeof(T) == 4) ? cell_of_f32(P, placeable(d), rx, ry, rz) : cell_of(P, placeable(d), rx, ry, rz);
  // the bucket and rank come from the counting pass (same arithmetic, same d)
  const int pos = (int)P.pt_off + excl[pa.cx[i]] + pa.slot[i];
  pa.pos[i] = pos;
  PtRec<T> r;
  r.fx = (T)cp.fx;
  r.fy = (T)cp.fy;
  r.fz = (T)cp.fz;
  r.rx = (T)rx;
  r.ry = (T)ry;
  r.rz = (T)rz;
  r.yz = cp.iy * N + cp.iz;
  r.r = (T)0;
  static_cast<PtRec<T>*>(pa.rec)[pos] = r;
  if constexpr (sizeof(T) == 8) {
    place_terms_fp64(P, pa, cs, c, i, d);
  } else {
    place_terms_fp32(P, pa, cs, c, i, d);
  }
}

// ---------------------------------------------------------------------------
// Velocity term: u and du from the plane partials, then
//   Psi_i = A + (v_obs - u)^2/(2 kappa^2),  r_i = -(v_obs - u)/kappa^2,
//   dPsi_i/dd = A' + (v_obs - u)(v_obs' - u')/kappa^2 - (v_obs - u)^2 (kappa^2)'/(2 kappa^4).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kPtsNT)
k_points_lik(const PointParams* __restrict__ pp, PointArrays pa, double* __restrict__ pts_part,
             int part_stride, int mode, double* __restrict__ kin_part, ChainScal* __restrict__ cs,
             double* __restrict__ gsig_part) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[3][kPtsNT / 32];
  const int c = blockIdx.y;
  const PointParams& P = pp[c];
  const ChainScal& S = cs[c];
  const long long il = (long long)blockIdx.x * kPtsNT + threadIdx.x;
  double psi_i = 0.0, kin = 0.0, gsig = 0.0;
  const bool ssig = S.sample_sig != 0;
  // Psi and dPsi/dd at an intermediate leapfrog point (GM_KICK_DRIFT) are
  // used only for the kick done here: the energy sums and the stored
  // gradient are those of the trajectory's end point (and of GM_GRAD)
  const bool upd = mode != GM_GRAD, drift = mode == GM_KICK_DRIFT;
  if (il < P.pt_n) {
    const long long i = P.pt_off + il;
    const long long nt = pa.ntot;
    // every load that depends on i alone goes out before the first store
    // (the arrays are not restrict-qualified, so the compiler keeps loads
    // after stores in program order): one round of latency for all of them,
    // then the partials at the bucket position
    const int pos = pa.pos[i];
    const double A = pa.lk[i];
    const double d0 = upd ? pa.d[i] : 0.0;
    const double pd0 = (upd && S.sample_d) ? pa.pd[i] : 0.0;
    const double rx = drift ? pa.rx[i] : 0.0, ry = drift ? pa.ry[i] : 0.0;
    PtRec<T>* rec = static_cast<PtRec<T>*>(pa.rec);
    double gd;
    if constexpr (sizeof(T) == 4) {
      // FP32 path: the six FP32 partials summed with TwoSum, then the
      // velocity term in FP32 (v_obs - u is a few hundred km/s, kept to
      // ~1e-7 relative); Psi_i and the gradient go to FP64 for the sums and
      // the distance update
      const float* f = reinterpret_cast<const float*>(pa.lk + nt);
      const float Ap = f[i], vo = f[nt + i], vop = f[2 * nt + i], ik2 = f[3 * nt + i], k2p = f[4 * nt + i];
      const float* part = static_cast<const float*>(pa.part);
      float pu[6], pdu[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        pu[k] = part[(long long)k * nt + pos];
        pdu[k] = part[(long long)(6 + k) * nt + pos];
      }
      if (!isfinite(A)) {
        psi_i = A;
        rec[pos].r = 0.0f;
        gd = 0.0;
      } else {
        HalfSqAcc<float> su, sdu;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          su.add(pu[k]);
          sdu.add(pdu[k]);
        }
        const float u = su.hi + su.lo, du = sdu.hi + sdu.lo;
        const float res_v = vo - u;
        const float r2k = res_v * res_v * ik2;
        if (!drift) psi_i = A + (double)(0.5f * r2k);
        rec[pos].r = -res_v * ik2;
        if (ssig) gsig = (double)((float)S.sig * ik2 * (1.0f - r2k));
        gd = (double)(Ap + res_v * (vop - du) * ik2 - 0.5f * r2k * k2p * ik2);
      }
    } else {
      const double Ap = pa.lk[nt + i], vo = pa.lk[2 * nt + i], vop = pa.lk[3 * nt + i];
      const double ik2 = pa.lk[4 * nt + i], k2p = pa.lk[5 * nt + i];
      const T* part = static_cast<const T*>(pa.part);
      double pu[6], pdu[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        pu[k] = (double)part[(long long)k * nt + pos];
        pdu[k] = (double)part[(long long)(6 + k) * nt + pos];
      }
      if (!isfinite(A)) {
        psi_i = A;
        rec[pos].r = (T)0;
        gd = 0.0;
      } else {
        double u = 0.0, du = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          u += pu[k];
          du += pdu[k];
        }
        const double res_v = vo - u;
        if (!drift) psi_i = A + 0.5 * res_v * res_v * ik2;
        rec[pos].r = (T)(-res_v * ik2);
        if (ssig) gsig = S.sig * ik2 * (1.0 - res_v * res_v * ik2);
        gd = Ap + res_v * (vop - du) * ik2 - 0.5 * res_v * res_v * k2p * ik2 * ik2;
      }
    }
    if (!drift) pa.gd[i] = gd;
    if (upd) {
      // leapfrog update of the distance (the rest of this evaluation no
      // longer reads d: the plane records were formed from the old one)
      double d = d0;
      if (S.sample_d) {
        const double p = pd0 - (drift ? S.eps : 0.5 * S.eps) * gd;
        pa.pd[i] = p;
        if (drift) {
          d = d + S.eps * P.minv_d * p;
          pa.d[i] = d;
        } else {
          kin = 0.5 * P.minv_d * p * p;   // summed after the last half kick only
        }
      }
      if (drift) {
        // buckets of the new distance, for the next evaluation
        const int key = bucket_key(P, d, rx, ry);
        pa.cx[i] = key;
        pa.slot[i] = atomicAdd(&pa.cnt_next[c * P.N * P.ksplit + key], 1);
      }
    }
  }
  // the block's sums of Psi_i, of the kinetic term and of dPsi/dsigma_NL in
  // one pass (each a fixed shuffle tree per warp, then the warps in order)
  const bool last = mode == GM_KICK_LAST;
  if (drift && !ssig) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if (!drift) psi_i += __shfl_down_sync(0xffffffffu, psi_i, o);
    if (last) kin += __shfl_down_sync(0xffffffffu, kin, o);
    if (ssig) gsig += __shfl_down_sync(0xffffffffu, gsig, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = psi_i;
    red[1][wid] = kin;
    red[2][wid] = gsig;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sp = 0.0, sk = 0.0, sg = 0.0;
    for (int w = 0; w < kPtsNT / 32; ++w) {
      sp += red[0][w];
      sk += red[1][w];
      sg += red[2][w];
    }
    const long long k = (long long)c * part_stride + blockIdx.x;
    if (!drift) pts_part[k] = sp;
    if (last) kin_part[k] = sk;
    if (ssig) gsig_part[k] = sg;
  }
}

// Cells only (bit-exact index work), for the sort and for tests; formed by
// the double-float screen with its FP64 fallback, as the bucketing and the
// FP32 path's placement form them.
__global__ void k_cells(const PointParams* __restrict__ pp, PointArrays pa, const double* __restrict__ d,
                        int* __restrict__ cell_out) {
  const int c = blockIdx.y;
  const PointParams& P = pp[c];
  const long long il = (long long)blockIdx.x * kPtsNT + threadIdx.x;
  if (il >= P.pt_n) return;
  const long long i = P.pt_off + il;
  const CellPos cp = cell_of_f32(P, d[i], pa.rx[i], pa.ry[i], pa.rz[i]);
  cell_out[i] = (cp.ix * P.N + cp.iy) * P.N + cp.iz;
}

// ---------------------------------------------------------------------------
// Stable counting sort of n points by cell index (one CTA; keys < N3).
// Pass 1 histograms, pass 2 an exclusive scan over cells, pass 3 walks the
// points in index order in chunks of blockDim, ranking equal keys inside a
// chunk with warp match masks so that equal cells keep their index order.
// ---------------------------------------------------------------------------
constexpr int kSortNT = 1024;

__global__ void __launch_bounds__(kSortNT) k_cell_sort(int N3, long long n, const int* __restrict__ cell,
                                                       int* __restrict__ perm, int* __restrict__ hist) {
  __shared__ int wsum[kSortNT / 32];
  __shared__ int carry;
  for (int k = threadIdx.x; k < N3; k += kSortNT) hist[k] = 0;
  __syncthreads();
  for (long long i = threadIdx.x; i < n; i += kSortNT) atomicAdd(&hist[cell[i]], 1);
  __syncthreads();
  // exclusive scan of hist over N3 entries, chunks of kSortNT
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < N3; base += kSortNT) {
    const int k = base + threadIdx.x;
    int v = k < N3 ? hist[k] : 0;
    int x = v;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int s = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      wsum[lane] = s;
    }
    __syncthreads();
    const int excl = carry + (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    if (k < N3) hist[k] = excl;
    __syncthreads();
    if (threadIdx.x == kSortNT - 1) carry = excl + v;
    __syncthreads();
  }
  // stable placement
  for (long long base = 0; base < n; base += kSortNT) {
    const long long i = base + threadIdx.x;
    const bool valid = i < n;
    const int key = valid ? cell[i] : -1;
    const int lane = threadIdx.x & 31;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    const unsigned peers = __match_any_sync(0xffffffffu, key) & act;
    const int rank_in_warp = __popc(peers & ((1u << lane) - 1u));
    const int leader_last = 31 - __clz(peers);  // highest lane with this key
    // warps go one after another so that earlier indices are placed first
    for (int w = 0; w < kSortNT / 32; ++w) {
      if ((int)(threadIdx.x >> 5) == w && valid) {
        const int pos = hist[key] + rank_in_warp;
        perm[pos] = (int)i;
        __syncwarp(peers);
        if (lane == leader_last) hist[key] += __popc(peers);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
static inline dim3 pts_grid(int n_chains, int max_pts) {
  return dim3((unsigned)points_blocks(max_pts), n_chains);
}

int points_blocks(int max_pts) { return max_pts > 0 ? (max_pts + kPtsNT - 1) / kPtsNT : 1; }

cudaError_t launch_points_prep(int n_chains, int max_pts, const PointParams* pp, PointArrays pa,
                               cudaStream_t st) {
  if (max_pts <= 0) return cudaSuccess;
  return launch_k<PDL_POINTS>(k_points_prep, pts_grid(n_chains, max_pts), dim3(kPtsNT), 0, st, pp, pa);
}

cudaError_t launch_points_place(int prec, int n_chains, int max_pts, const PointParams* pp,
                                PointArrays pa, ChainScal* cs, cudaStream_t st) {
  // runs even without points: block 0 writes the (empty) bucket offsets
  if (prec == 0)
    return launch_k<PDL_POINTS>(k_points_place<float>, pts_grid(n_chains, max_pts), dim3(kPtsNT), 0, st, pp, pa, cs);
  return launch_k<PDL_POINTS>(k_points_place<double>, pts_grid(n_chains, max_pts), dim3(kPtsNT), 0, st, pp, pa, cs);
}

cudaError_t launch_points_lik(int prec, int n_chains, int max_pts, const PointParams* pp, PointArrays pa,
                              double* pts_part, int part_stride, int mode, double* kin_part, ChainScal* cs,
                              double* gsig_part, cudaStream_t st) {
  if (prec == 0)
    return launch_k<PDL_POINTS>(k_points_lik<float>, pts_grid(n_chains, max_pts), dim3(kPtsNT), 0, st, pp, pa, pts_part,
                    part_stride, mode, kin_part, cs, gsig_part);
  return launch_k<PDL_POINTS>(k_points_lik<double>, pts_grid(n_chains, max_pts), dim3(kPtsNT), 0, st, pp, pa, pts_part,
                  part_stride, mode, kin_part, cs, gsig_part);
}

cudaError_t launch_cells(int n_chains, int max_pts, const PointParams* pp, const double* d,
                         PointArrays pa, int* cell_out, cudaStream_t st) {
  if (max_pts <= 0) return cudaSuccess;
  dim3 g = pts_grid(n_chains, max_pts);
  k_cells<<<g, kPtsNT, 0, st>>>(pp, pa, d, cell_out);
  return cudaGetLastError();
}

cudaError_t launch_cell_sort(int N3, long long n, const int* cell, int* perm, int* hist_ws,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_cell_sort<<<1, kSortNT, 0, st>>>(N3, n, cell, perm, hist_ws);
  return cudaGetLastError();
}

}  // namespace hm
