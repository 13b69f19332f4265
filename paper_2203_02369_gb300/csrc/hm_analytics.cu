// On-device chain analytics, one sample per HMC trajectory (the chain state
// after the Metropolis test):
//   * Monte-Carlo moments over chain states (eq. int_mc): running mean and
//     variance (Welford) of the density field delta and of the radial
//     velocity v_r = rhat . v at every grid node;
//   * the convergence monitor of section "Convergence": the root mean square
//     over the nodes of m_s/Sigma_s - m_{s-1}/Sigma_{s-1}, with m_s the running
//     mean of delta after s samples and Sigma_s^2 the variance over the grid of
//     the s-th sample's delta;
//   * the monopole (a f <delta>, the mean of -div v / H0 by linear continuity)
//     and the dipole (mean velocity) in spheres about the observer (section
//     "Monopole and dipole"), with their mean and variance over samples.
// The fields delta and v_j come from the usual plane and pencil passes; the
// kernels here read them once per sample.
#include <algorithm>

#include "hm_fft.cuh"
#include "hm_internal.h"

namespace hm {

constexpr int kAnNT = 256;

// Block partials of sum delta and sum delta^2 over a chain's nodes.
template <typename T>
__global__ void __launch_bounds__(kAnNT) k_an_sigma(AnArgs a) {
  __shared__ double red[2][kAnNT / 32];
  const int c = blockIdx.y, b = blockIdx.x;
  const T* x = static_cast<const T*>(a.delta_g) + (long long)c * a.n3;
  HalfSqAcc<T> s1, s2;
  for (long long e = (long long)b * kAnNT + threadIdx.x; e < a.n3; e += (long long)a.nblk * kAnNT) {
    const T v = x[e];
    s1.add(v);
    s2.add_half_sq(v);
  }
  s1.warp_reduce();
  s2.warp_reduce();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = s1.value();
    red[1][wid] = s2.value();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double p = 0.0, q = 0.0;
    for (int i = 0; i < kAnNT / 32; ++i) {
      p += red[0][i];
      q += red[1][i];
    }
    a.sig_part[((long long)c * a.nblk + b) * 2] = p;
    a.sig_part[((long long)c * a.nblk + b) * 2 + 1] = 2.0 * q;
  }
}

// Welford updates of the node moments, the convergence-metric partials and
// the per-shell sums of delta and v (shared-memory atomics per block).
template <typename T>
__global__ void __launch_bounds__(kAnNT) k_an_update(AnArgs a) {
  __shared__ double red[kAnNT / 32];
  __shared__ double sh_sig;
  __shared__ T ssum[kMaxShells * 4];
  const int c = blockIdx.y, b = blockIdx.x;
  if (threadIdx.x == 0) {
    // Sigma_s of this sample: every block sums the partials in the same order
    double s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < a.nblk; ++k) {
      s1 += a.sig_part[((long long)c * a.nblk + k) * 2];
      s2 += a.sig_part[((long long)c * a.nblk + k) * 2 + 1];
    }
    const double mean = s1 / (double)a.n3, var = s2 / (double)a.n3 - mean * mean;
    sh_sig = sqrt(var > 0.0 ? var : 0.0);
    if (b == 0) a.sig_cur[c] = sh_sig;
  }
  for (int k = threadIdx.x; k < a.nsh * 4; k += kAnNT) ssum[k] = (T)0;
  __syncthreads();
  const long long cnt = a.count[c] + 1;
  const T inv_n = (T)(1.0 / (double)cnt);
  const bool metric = cnt >= 2;
  const T isig = sh_sig > 0.0 ? (T)(1.0 / sh_sig) : (T)0;
  const T isigp = a.sig_prev[c] > 0.0 ? (T)(1.0 / a.sig_prev[c]) : (T)0;
  const T ox = (T)a.obs[3 * c], oy = (T)a.obs[3 * c + 1], oz = (T)a.obs[3 * c + 2];
  const T dl = (T)a.delta;
  const long long base = (long long)c * a.n3;
  const T* dg = static_cast<const T*>(a.delta_g) + base;
  const T* vx = static_cast<const T*>(a.vel_g) + 3 * base;
  const T* vy = vx + a.n3;
  const T* vz = vy + a.n3;
  T* md = static_cast<T*>(a.mean_d) + base;
  T* m2d = static_cast<T*>(a.m2_d) + base;
  T* mv = static_cast<T*>(a.mean_vr) + base;
  T* m2v = static_cast<T*>(a.m2_vr) + base;
  const unsigned char* shell = a.shell + base;
  const int N = a.N;
  HalfSqAcc<T> macc;
  for (long long e = (long long)b * kAnNT + threadIdx.x; e < a.n3; e += (long long)a.nblk * kAnNT) {
    const int ix = (int)(e / ((long long)N * N)), iy = (int)((e / N) % N), iz = (int)(e % N);
    const T d = dg[e], v0 = vx[e], v1 = vy[e], v2 = vz[e];
    const T dx = (T)ix * dl - ox, dy = (T)iy * dl - oy, dz = (T)iz * dl - oz;
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T vr = r2 > (T)0 ? (dx * v0 + dy * v1 + dz * v2) / sqrt(r2) : (T)0;
    // Welford: mean_n = mean_{n-1} + (x - mean_{n-1})/n, M2 += (x - mean_{n-1})(x - mean_n)
    const T mo = md[e], dm = d - mo, mn = mo + dm * inv_n;
    md[e] = mn;
    m2d[e] += dm * (d - mn);
    const T wo = mv[e], dw = vr - wo, wn = wo + dw * inv_n;
    mv[e] = wn;
    m2v[e] += dw * (vr - wn);
    if (metric) macc.add_half_sq(mn * isig - mo * isigp);
    const int k = shell[e];
    if (k < a.nsh) {
      atomicAdd(&ssum[4 * k], d);
      atomicAdd(&ssum[4 * k + 1], v0);
      atomicAdd(&ssum[4 * k + 2], v1);
      atomicAdd(&ssum[4 * k + 3], v2);
    }
  }
  macc.warp_reduce();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = macc.value();
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < kAnNT / 32; ++i) s += red[i];
    a.met_part[(long long)c * a.nblk + b] = 2.0 * s;
  }
  for (int k = threadIdx.x; k < a.nsh * 4; k += kAnNT)
    a.shell_part[((long long)c * a.nblk + b) * a.nsh * 4 + k] = (double)ssum[k];
}

// Per chain: the convergence metric of this sample, the sphere moments and
// their Welford moments over samples, then the sample count.
__global__ void __launch_bounds__(128) k_an_finalize(AnArgs a) {
  __shared__ double tot[kMaxShells * 4];
  const int c = blockIdx.x;
  const long long cnt = a.count[c] + 1;
  for (int t = threadIdx.x; t < a.nsh * 4; t += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < a.nblk; ++k) s += a.shell_part[((long long)c * a.nblk + k) * a.nsh * 4 + t];
    tot[t] = s;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  if (cnt >= 2) {
    double s = 0.0;
    for (int k = 0; k < a.nblk; ++k) s += a.met_part[(long long)c * a.nblk + k];
    if (cnt - 2 < a.max_samples) a.hist[(long long)c * a.max_samples + (cnt - 2)] = sqrt(s / (double)a.n3);
  }
  double run[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < a.nsh; ++k) {
    for (int q = 0; q < 4; ++q) run[q] += tot[4 * k + q];
    const double n = a.sph_cnt[(long long)c * a.nsh + k];
    double val[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (n > 0.0) {
      val[0] = a.f * run[0] / n;
      val[1] = run[1] / n;
      val[2] = run[2] / n;
      val[3] = run[3] / n;
      val[4] = sqrt(val[1] * val[1] + val[2] * val[2] + val[3] * val[3]);
    }
    for (int q = 0; q < 5; ++q) {
      double* acc = a.sph_acc + (((long long)c * a.nsh + k) * 5 + q) * 2;
      const double mo = acc[0], dm = val[q] - mo, mn = mo + dm / (double)cnt;
      acc[0] = mn;
      acc[1] += dm * (val[q] - mn);
    }
  }
  a.sig_prev[c] = a.sig_cur[c];
  a.count[c] = cnt;
}

// out[i] = in[i] * scale (variance = M2 / (n - 1) for the read-out).
template <typename T>
__global__ void __launch_bounds__(kAnNT) k_an_scale(long long n, const T* __restrict__ in, T* __restrict__ out,
                                                    double scale) {
  const T s = (T)scale;
  for (long long i = (long long)blockIdx.x * kAnNT + threadIdx.x; i < n; i += (long long)gridDim.x * kAnNT)
    out[i] = in[i] * s;
}

cudaError_t launch_analytics(int prec, const AnArgs& a, cudaStream_t st) {
  const dim3 grid(a.nblk, a.C);
  if (prec == 0) {
    k_an_sigma<float><<<grid, kAnNT, 0, st>>>(a);
    k_an_update<float><<<grid, kAnNT, 0, st>>>(a);
  } else {
    k_an_sigma<double><<<grid, kAnNT, 0, st>>>(a);
    k_an_update<double><<<grid, kAnNT, 0, st>>>(a);
  }
  k_an_finalize<<<a.C, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_an_scale(int prec, long long n, const void* in, void* out, double scale, cudaStream_t st) {
  const int blocks = (int)std::min<long long>((n + kAnNT - 1) / kAnNT, 4096);
  if (prec == 0)
    k_an_scale<float><<<blocks, kAnNT, 0, st>>>(n, static_cast<const float*>(in), static_cast<float*>(out), scale);
  else
    k_an_scale<double><<<blocks, kAnNT, 0, st>>>(n, static_cast<const double*>(in), static_cast<double*>(out),
                                                 scale);
  return cudaGetLastError();
}

}  // namespace hm
