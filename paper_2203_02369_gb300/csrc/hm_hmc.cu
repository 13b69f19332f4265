// HMC kernels: momentum refresh from the Philox-4x32-10 counter-based
// generator (Salmon et al., SC'11), the first half kick + drift of each
// trajectory, FP64 energy reductions, the Metropolis test and the predicated
// restore of a rejected proposal (sections "Construction of HMC chains",
// "Integrating the HMC trajectories", "The Mass matrix"; eqs. Hamiltonian,
// hamilton, M_ab).
#include "hm_fft.cuh"
#include "hm_internal.h"
#include "hm_device.cuh"
#include "hamlet.h"

namespace hm {

constexpr int kEwNT = 256;

// ---- Philox-4x32-10 ----
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const unsigned W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += W0;
      k.y += W1;
    }
    const unsigned lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const unsigned lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ double u53(unsigned a, unsigned b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ uint2 key_of(unsigned long long seed) {
  return make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32));
}

// k * 2^-53 rounded to the nearest float (ties to even) for 0 <= k <= 2^53,
// with integer operations only: the same value as (float)(k * 2^-53) formed
// in double, without using the FP64 units.
__device__ __forceinline__ float u53_float(unsigned long long k) {
  if (k == 0) return 0.f;
  const int nb = 64 - __clzll((long long)k);   // bit length, 1..54
  unsigned long long m = k;
  int sh = 0;
  if (nb > 24) {
    sh = nb - 24;
    m = k >> sh;
    const unsigned long long rem = k & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m == (1ull << 24)) {
        m >>= 1;
        ++sh;
      }
    }
  }
  // m < 2^24 converts exactly; 2^(sh - 53) is a normal float for sh <= 30
  return (float)(unsigned)m * __int_as_float((sh - 53 + 127) << 23);
}

// Two standard normals from counter (pair, traj, chain, tag): Box-Muller on
// u1 = words (0,1), u2 = words (2,3); radius sqrt(-2 ln(1-u1)), angle 2 pi u2.
__device__ __forceinline__ void normal_pair(unsigned long long seed, unsigned pair, unsigned traj,
                                            unsigned chain, unsigned tag, double& n0, double& n1) {
  const uint4 x = philox4x32_10(make_uint4(pair, traj, chain, tag), key_of(seed));
  const double u1 = u53(x.x, x.y), u2 = u53(x.z, x.w);
  const double r = sqrt(-2.0 * log(1.0 - u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  n0 = r * c;
  n1 = r * s;
}

// Normals in the field precision: FP64 Box-Muller for double fields; for
// float fields the same 53-bit uniforms go through FP32 log/sqrt/sincospi
// (the momenta are stored in FP32 anyway), which keeps the FP64 units free.
// ln(1 - u1) is taken as log1p(-u1) of the exactly rounded u1 where u1 <
// 1/2 and as log of the exactly rounded 1 - u1 elsewhere, so the radius
// keeps float precision at both ends (near u1 = 0 the rounding of 1 - u1
// alone would cost up to 2.4e-4 absolute in a small normal).
template <typename T>
__device__ __forceinline__ void normal_pair_t(unsigned long long seed, unsigned pair, unsigned traj,
                                              unsigned chain, unsigned tag, T& n0, T& n1) {
  if constexpr (sizeof(T) == 8) {
    double a, b;
    normal_pair(seed, pair, traj, chain, tag, a, b);
    n0 = a;
    n1 = b;
  } else {
    const uint4 x = philox4x32_10(make_uint4(pair, traj, chain, tag), key_of(seed));
    const unsigned long long k1 = ((unsigned long long)(x.x >> 5) << 26) + (x.y >> 6);
    const unsigned long long k2 = ((unsigned long long)(x.z >> 5) << 26) + (x.w >> 6);
    const float u2 = u53_float(k2);                  // (float)u53, exactly
    const float l = (k1 < (1ull << 52)) ? log1pf(-u53_float(k1))            // u1 < 1/2
                                        : logf(u53_float((1ull << 53) - k1));  // (float)(1 - u53), exactly
    const float r = sqrtf(-2.0f * l);
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    n0 = r * c;
    n1 = r * s;
  }
}

template <typename T>
__device__ __forceinline__ double block_sum2(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
  return s;
}

// ---------------------------------------------------------------------------
// Trajectory start, field part: draw p ~ N(0, I), kinetic partials, save
// (w, grad) for a possible restore, half kick and drift.
// Grid: (nparts, n_chains); element pairs strided across the chain's blocks.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kEwNT)
k_traj_begin_field(long long n3, T* __restrict__ w, T* __restrict__ pw, const T* __restrict__ gw,
                   T* __restrict__ w0, T* __restrict__ gw0, unsigned long long seed,
                   const int* __restrict__ chain_id, double* __restrict__ kin_part, int draw,
                   ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[kEwNT / 32];
  const int c = blockIdx.y;
  const long long off = (long long)c * n3;
  const T eps = (T)cs[c].eps;
  const unsigned traj = (unsigned)cs[c].traj;
  const unsigned cid = (unsigned)chain_id[c];
  HalfSqAcc<T> kin;
  const long long npair = n3 / 2;
  for (long long q = (long long)blockIdx.x * kEwNT + threadIdx.x; q < npair;
       q += (long long)gridDim.x * kEwNT) {
    const long long e = off + 2 * q;
    T p[2];
    if (draw) {
      normal_pair_t<T>(seed, (unsigned)q, traj, cid, 0u, p[0], p[1]);
    } else {
      p[0] = pw[e];
      p[1] = pw[e + 1];
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      kin.add_half_sq(p[h]);
      const T wi = w[e + h], gi = gw[e + h];
      w0[e + h] = wi;
      gw0[e + h] = gi;
      const T ph = p[h] - (T)0.5 * eps * gi;
      pw[e + h] = ph;
      w[e + h] = wi + eps * ph;
    }
  }
  kin.warp_reduce();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = kin.value();
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kEwNT / 32; ++i) s += red[i];
    kin_part[(long long)c * gridDim.x + blockIdx.x] = s;
  }
}

// Trajectory start, distance part: p_d ~ N(0, (H0/sigma_v)^2).  Small
// blocks (kBpNT threads, one point pair each), so that the FP64 Box-Muller
// of a catalogue spreads over every SM's FP64 unit.
constexpr int kBpNT = 64;
__global__ void __launch_bounds__(kBpNT)
k_traj_begin_points(const PointParams* __restrict__ pp, PointArrays pa, double* __restrict__ d0,
                    double* __restrict__ gd0, unsigned long long seed, const int* __restrict__ chain_id,
                    double* __restrict__ kin_part, int draw, ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[kBpNT / 32];
  const int c = blockIdx.y;
  const PointParams& P = pp[c];
  const double eps = cs[c].eps;
  const unsigned traj = (unsigned)cs[c].traj;
  const unsigned cid = (unsigned)chain_id[c];
  const int sd = cs[c].sample_d;
  double kin = 0.0;
  const long long npair = (P.pt_n + 1) / 2;
  for (long long q = (long long)blockIdx.x * kBpNT + threadIdx.x; q < npair;
       q += (long long)gridDim.x * kBpNT) {
    double nn[2] = {0.0, 0.0};
    if (draw) normal_pair(seed, (unsigned)q, traj, cid, 1u, nn[0], nn[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const long long il = 2 * q + h;
      if (il >= P.pt_n) break;
      const long long i = P.pt_off + il;
      const double di = pa.d[i], gi = pa.gd[i];
      d0[i] = di;
      gd0[i] = gi;
      double dn = di;
      if (sd) {
        const double p = draw ? nn[h] / sqrt(P.minv_d) : pa.pd[i];
        kin += 0.5 * P.minv_d * p * p;
        const double ph = p - 0.5 * eps * gi;
        pa.pd[i] = ph;
        dn = di + eps * P.minv_d * ph;
        pa.d[i] = dn;
      } else {
        pa.pd[i] = 0.0;
      }
      // buckets of the drifted distances for the first evaluation
      const int key = bucket_key(P, dn, pa.rx[i], pa.ry[i]);
      pa.cx[i] = key;
      pa.slot[i] = atomicAdd(&pa.cnt_next[c * P.N * P.ksplit + key], 1);
    }
  }
  const double s = block_sum2<double>(kin, red);
  if (threadIdx.x == 0) kin_part[(long long)c * gridDim.x + blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Per-chain scalar finalisation (one CTA per chain, fixed summation order).
// ---------------------------------------------------------------------------
// Fixed-order sum of n values by one warp: lane l adds l, l+32, ... in order,
// then a fixed shuffle tree; lane 0 gets the result.
__device__ __forceinline__ double warp_sum_fixed(const double* __restrict__ x, int n) {
  double s = 0.0;
  for (int i = threadIdx.x & 31; i < n; i += 32) s += x[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return s;
}

__global__ void k_finalize(const double* __restrict__ prior_part, int n_prior,
                           const double* __restrict__ pts_part, int n_pts,
                           const double* __restrict__ kin_part, int n_kin,
                           const double* __restrict__ kin_pts_part, int n_kin_pts, int what,
                           unsigned long long seed, const int* __restrict__ chain_id,
                           ChainScal* __restrict__ cs, hm_trace* __restrict__ trace) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.x;
  // the four sums, one warp each (the same fixed order as one warp doing
  // them one after another), met in shared memory
  __shared__ double sums[4];
  const int wid = threadIdx.x >> 5;
  const bool psi = (what & FIN_PSI) != 0, kin = (what & (FIN_HOLD | FIN_ACCEPT | FIN_KIN)) != 0;
  double v = 0.0;
  if (wid == 0 && psi) v = warp_sum_fixed(prior_part + (long long)c * n_prior, n_prior);
  if (wid == 1 && psi) v = warp_sum_fixed(pts_part + (long long)c * n_pts, n_pts);
  if (wid == 2 && kin) v = warp_sum_fixed(kin_part + (long long)c * n_kin, n_kin);
  if (wid == 3 && kin) v = warp_sum_fixed(kin_pts_part + (long long)c * n_kin_pts, n_kin_pts);
  if ((threadIdx.x & 31) == 0) sums[wid] = v;
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double a = sums[0], b = sums[1], k = sums[2], kp = sums[3];
  ChainScal& S = cs[c];
  if (what & FIN_PSI) {
    S.psi_prior = a;
    S.psi_pts = b;
    S.psi = a + b;
  }
  if (what & (FIN_HOLD | FIN_ACCEPT | FIN_KIN)) S.kin = (S.sample_d ? k + kp : k) + (S.sample_sig ? S.kin_sig : 0.0);
  if (what & FIN_HOLD) {
    S.psi0 = S.psi;
    S.H_old = S.psi + S.kin;
  }
  if (what & FIN_ACCEPT) {
    S.H_new = S.psi + S.kin;
    const uint4 x = philox4x32_10(make_uint4(0u, (unsigned)S.traj, (unsigned)chain_id[c], 2u), key_of(seed));
    const double u = u53(x.x, x.y);
    S.logu = log(1.0 - u);
    const double dH = S.H_old - S.H_new;
    const bool fin = isfinite(S.H_new);
    const int acc = (fin && S.logu < dH) ? 1 : 0;
    S.accept = acc;
    if (!fin) S.status |= STATUS_NONFINITE;
    if (trace) {
      hm_trace& t = trace[(S.traj - S.traj_run0) * gridDim.x + c];
      t.traj = S.traj;
      t.H_old = S.H_old;
      t.H_new = S.H_new;
      t.logu = S.logu;
      t.psi = acc ? S.psi : S.psi0;
      t.eps = S.eps;
      t.accept = acc;
      t.status = S.status;
    }
    if (!acc) {
      S.psi = S.psi0;
      if (S.sample_sig) {
        S.sig = S.sig0;
        S.g_sig = S.g_sig0;
      }
    }
    S.traj += 1;
    if (S.da_on) {
      // dual averaging (Hoffman & Gelman) toward acceptance probability da_delta
      const double alpha = fin ? fmin(1.0, exp(fmin(0.0, dH))) : 0.0;
      S.da_m += 1;
      const double m = (double)S.da_m;
      const double wgt = 1.0 / (m + 10.0);
      S.da_Hbar = (1.0 - wgt) * S.da_Hbar + wgt * (S.da_delta - alpha);
      const double leps = S.da_mu - sqrt(m) / 0.05 * S.da_Hbar;
      const double eta = pow(m, -0.75);
      S.da_lepsbar = eta * leps + (1.0 - eta) * S.da_lepsbar;
      S.eps = exp(leps);
    }
  }
}

// Restore (w, grad_w, d, grad_d) of chains whose proposal was rejected.
template <typename T>
__global__ void __launch_bounds__(kEwNT)
k_restore_field(long long n3, T* __restrict__ w, T* __restrict__ gw, const T* __restrict__ w0,
                const T* __restrict__ gw0, const ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.y;
  if (cs[c].accept) return;
  const long long off = (long long)c * n3;
  for (long long e = (long long)blockIdx.x * kEwNT + threadIdx.x; e < n3; e += (long long)gridDim.x * kEwNT) {
    w[off + e] = w0[off + e];
    gw[off + e] = gw0[off + e];
  }
}

__global__ void __launch_bounds__(kEwNT)
k_restore_points(const PointParams* __restrict__ pp, PointArrays pa, const double* __restrict__ d0,
                 const double* __restrict__ gd0, const ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.y;
  if (cs[c].accept) return;
  const PointParams& P = pp[c];
  for (long long il = (long long)blockIdx.x * kEwNT + threadIdx.x; il < P.pt_n;
       il += (long long)gridDim.x * kEwNT) {
    const long long i = P.pt_off + il;
    pa.d[i] = d0[i];
    pa.gd[i] = gd0[i];
  }
}

__global__ void k_set_run(int n_chains, const double* __restrict__ eps, int sample_d,
                          ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  if (eps) cs[c].eps = eps[c];   // nullptr: every chain keeps its own step
  cs[c].sample_d = sample_d;
  cs[c].traj_run0 = cs[c].traj;
  cs[c].status = 0;
}

// sigma_NL updates (one warp per chain; fixed-order reduction of the partials)
__global__ void k_sig_update(const double* __restrict__ gsig_part, int nparts, int mode, ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.x;
  ChainScal& S = cs[c];
  if (!S.sample_sig) return;
  double g = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) g += gsig_part[(long long)c * nparts + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) g += __shfl_down_sync(0xffffffffu, g, o);
  if (threadIdx.x != 0) return;
  S.g_sig = g;
  if (mode == GM_GRAD) return;
  const double ck = (mode == GM_KICK_DRIFT) ? S.eps : 0.5 * S.eps;
  S.p_sig -= ck * g;
  if (mode == GM_KICK_DRIFT) S.sig += S.eps * S.p_sig;
  if (mode == GM_KICK_LAST) S.kin_sig = 0.5 * S.p_sig * S.p_sig;
}

__global__ void k_sig_begin(unsigned long long seed, const int* __restrict__ chain_id, int draw,
                            ChainScal* __restrict__ cs) {
  pdl_wait();
  pdl_trigger();
  const int c = blockIdx.x;
  ChainScal& S = cs[c];
  if (threadIdx.x != 0 || !S.sample_sig) return;
  double p = S.p_sig;
  if (draw) {
    double n1;
    normal_pair(seed, 0u, (unsigned)S.traj, (unsigned)chain_id[c], 3u, p, n1);
  }
  S.kin_sig = 0.5 * p * p;
  S.sig0 = S.sig;
  S.g_sig0 = S.g_sig;
  S.p_sig = p - 0.5 * S.eps * S.g_sig;
  S.sig += S.eps * S.p_sig;
}

__global__ void k_sig_set(int n_chains, int enable, const double* __restrict__ sig, ChainScal* __restrict__ cs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  cs[c].sample_sig = enable;
  if (sig) cs[c].sig = sig[c];
  cs[c].p_sig = 0.0;
  cs[c].kin_sig = 0.0;
}

__global__ void k_da(int n_chains, int start, double delta, double* __restrict__ eps_out,
                     ChainScal* __restrict__ cs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  ChainScal& S = cs[c];
  if (start) {
    S.da_on = 1;
    S.da_m = 0;
    S.da_Hbar = 0.0;
    S.da_lepsbar = 0.0;
    S.da_mu = log(10.0 * S.eps);
    S.da_delta = delta;
  } else {
    S.da_on = 0;
    if (S.da_m > 0) S.eps = exp(S.da_lepsbar);
    if (eps_out) eps_out[c] = S.eps;
  }
}

__global__ void k_philox_raw(unsigned long long seed, long long n, unsigned c1, unsigned c2, unsigned c3,
                             unsigned* __restrict__ out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const uint4 x = philox4x32_10(make_uint4((unsigned)q, c1, c2, c3), key_of(seed));
  out[4 * q + 0] = x.x;
  out[4 * q + 1] = x.y;
  out[4 * q + 2] = x.z;
  out[4 * q + 3] = x.w;
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_traj_begin_field(int prec, int n_chains, long long n3, void* w, void* pw,
                                    const void* gw, void* w0, void* gw0, unsigned long long seed,
                                    const int* chain_id, double* kin_part, int nparts, int draw,
                                    ChainScal* cs, cudaStream_t st) {
  dim3 g(nparts, n_chains);
  if (prec == 0)
    return launch_k(k_traj_begin_field<float>, g, dim3(kEwNT), 0, st, n3, (float*)w, (float*)pw, (const float*)gw,
                    (float*)w0, (float*)gw0, seed, chain_id, kin_part, draw, cs);
  return launch_k(k_traj_begin_field<double>, g, dim3(kEwNT), 0, st, n3, (double*)w, (double*)pw,
                  (const double*)gw, (double*)w0, (double*)gw0, seed, chain_id, kin_part, draw, cs);
}

int traj_begin_points_blocks(int max_pts) { return std::max(1, std::min(512, (max_pts / 2 + kBpNT - 1) / kBpNT)); }

cudaError_t launch_traj_begin_points(int n_chains, int /*max_pts*/, const PointParams* pp,
                                     PointArrays pa, double* d0, double* gd0,
                                     unsigned long long seed, const int* chain_id,
                                     double* kin_part, int nparts, int draw, ChainScal* cs,
                                     cudaStream_t st) {
  dim3 g(nparts, n_chains);
  return launch_k(k_traj_begin_points, g, dim3(kBpNT), 0, st, pp, pa, d0, gd0, seed, chain_id, kin_part, draw, cs);
}

cudaError_t launch_set_run(int n_chains, const double* eps, int sample_d, ChainScal* cs,
                           cudaStream_t st) {
  return launch_k(k_set_run, dim3((n_chains + 127) / 128), dim3(128), 0, st, n_chains, eps, sample_d, cs);
}

cudaError_t launch_finalize(int n_chains, const double* prior_part, int n_prior, const double* pts_part,
                            int n_pts, const double* kin_part, int n_kin, const double* kin_pts_part,
                            int n_kin_pts, int what, unsigned long long seed, const int* chain_id,
                            ChainScal* cs, void* trace_dev, cudaStream_t st) {
  return launch_k(k_finalize, dim3(n_chains), dim3(128), 0, st, prior_part, n_prior, pts_part, n_pts, kin_part, n_kin,
                  kin_pts_part, n_kin_pts, what, seed, chain_id, cs, static_cast<hm_trace*>(trace_dev));
}

cudaError_t launch_restore(int prec, int n_chains, long long n3, void* w, void* gw, const void* w0,
                           const void* gw0, int max_pts, const PointParams* pp, PointArrays pa,
                           const double* d0, const double* gd0, const ChainScal* cs,
                           cudaStream_t st) {
  long long nb = (n3 + kEwNT - 1) / kEwNT;
  if (nb > 1024) nb = 1024;
  dim3 g((unsigned)nb, n_chains);
  cudaError_t e;
  if (prec == 0)
    e = launch_k(k_restore_field<float>, g, dim3(kEwNT), 0, st, n3, (float*)w, (float*)gw, (const float*)w0,
                 (const float*)gw0, cs);
  else
    e = launch_k(k_restore_field<double>, g, dim3(kEwNT), 0, st, n3, (double*)w, (double*)gw, (const double*)w0,
                 (const double*)gw0, cs);
  if (e != cudaSuccess) return e;
  if (max_pts > 0) {
    long long pb = (max_pts + kEwNT - 1) / kEwNT;
    if (pb > 256) pb = 256;
    return launch_k(k_restore_points, dim3((unsigned)pb, n_chains), dim3(kEwNT), 0, st, pp, pa, d0, gd0, cs);
  }
  return cudaSuccess;
}

cudaError_t launch_sig_update(int n_chains, const double* gsig_part, int nparts, int mode, ChainScal* cs,
                              cudaStream_t st) {
  return launch_k(k_sig_update, dim3(n_chains), dim3(32), 0, st, gsig_part, nparts, mode, cs);
}

cudaError_t launch_sig_begin(int n_chains, unsigned long long seed, const int* chain_id, int draw, ChainScal* cs,
                             cudaStream_t st) {
  return launch_k(k_sig_begin, dim3(n_chains), dim3(32), 0, st, seed, chain_id, draw, cs);
}

cudaError_t launch_sig_set(int n_chains, int enable, const double* sig, ChainScal* cs, cudaStream_t st) {
  k_sig_set<<<(n_chains + 127) / 128, 128, 0, st>>>(n_chains, enable, sig, cs);
  return cudaGetLastError();
}

cudaError_t launch_da(int n_chains, int start, double delta, double* eps_out, ChainScal* cs, cudaStream_t st) {
  k_da<<<(n_chains + 127) / 128, 128, 0, st>>>(n_chains, start, delta, eps_out, cs);
  return cudaGetLastError();
}

cudaError_t launch_philox_raw(unsigned long long seed, long long n, unsigned int c1, unsigned int c2,
                              unsigned int c3, unsigned int* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_philox_raw<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(seed, n, c1, c2, c3, out);
  return cudaGetLastError();
}

}  // namespace hm
