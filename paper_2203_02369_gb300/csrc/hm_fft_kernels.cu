// 3D real-to-complex / complex-to-real FFT passes and the fused k-space
// weights of the linear velocity operator (eq. vel-field) and its adjoint.
//
// A 3D transform is two passes over HBM:
//   plane pass : one CTA per x-plane; z (real <-> half complex, two real rows
//                packed in one complex row) and y (complex) in shared memory;
//   pencil pass: one CTA per tile of TC contiguous (y, kz) columns; the x
//                transform runs in shared memory, with the k-space operator
//                applied between a forward and an inverse x transform so the
//                weighted spectra never take an extra trip through HBM.
// Spectrum layout: [kx][ky][kz], kz = 0..N/2, natural order on every axis.
#include <cuda.h>   // CUtensorMap; the encoder is fetched at run time from the driver

#include <algorithm>
#include <cstdint>

#include "hm_fft.cuh"
#include "hm_internal.h"

namespace hm {

template <int N> struct PlaneCfg {
  static constexpr int NH = N / 2 + 1;             // kz = 0..N/2 in the global half spectrum
  static constexpr int NC = N / 2;                 // spectrum columns per row in shared memory (see below)
  static constexpr int NR = N / 2;                 // packed z rows (two real rows each)
  static constexpr int ZP = N + 1;                 // odd pitch of a packed z row
  static constexpr int NT = N >= 128 ? 512 : (N >= 64 ? 256 : 128);
  static constexpr int SIZE = NR * ZP;             // complex elements of the plane buffer
  static constexpr int MINB = N >= 128 ? 2 : (N == 64 ? 4 : 1);   // CTAs per SM the register budget aims at
};

template <typename T, int N> constexpr size_t plane_smem_bytes() {
  return sizeof(cplx<T>) * PlaneCfg<N>::SIZE;
}

// The plane buffer B (N/2 rows of pitch ZP = N + 1) is read through two views
// that share memory:
//   packed view   Z[r][z] = B[r*ZP + z] (r < N/2, z < N): real and imaginary
//                 parts are the real rows y = 2r and 2r + 1;
//   spectrum view H[y][c] = B[hoff(y) + c] (y < N, c < N/2), hoff(y) =
//                 (y/2) ZP + (y odd) N/2: rows 2r and 2r + 1 fill Z row r.
// Column c = 0 of the spectrum view carries two real-symmetric lines at once:
// kz = 0 in its real part and kz = N/2 in its imaginary part (both are real
// after the z transform of real rows), so every y transform runs over N/2
// columns and all thread counts divide the work without a ragged tail.  The
// pitch ZP is odd, so a row-per-thread access (the z transform) hits
// distinct shared-memory banks.
template <int N> __device__ __forceinline__ int hoff(int y) {
  return (y >> 1) * PlaneCfg<N>::ZP + (y & 1) * (N / 2);
}

template <typename T, int N>
__device__ __forceinline__ T* zreal(cplx<T>* B, int y, int z) {
  return reinterpret_cast<T*>(&B[(y >> 1) * PlaneCfg<N>::ZP + z]) + (y & 1);
}

// z transform of the N/2 packed rows in place, one row per thread in both
// radix stages (conflict-free with the odd pitch).
template <typename T, int N, bool INV>
__device__ __forceinline__ void zfft(cplx<T>* B, const cplx<T>* __restrict__ tw) {
  using P = PlaneCfg<N>;
  fft_smem<T, N, INV, P::NR, P::NT, true>(B, P::ZP, 1, tw);
}

// Stage-1 radix-R1 group (offset m): DFT over j of a[j] = x[m + M j], then the
// twiddles W_N^{m k2}; the result a[k2] belongs at m + M k2.
template <typename T, int N, bool INV>
__device__ __forceinline__ void stage1_group(cplx<T>* a, int m, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  dft_reg<R1, INV>(a);
  if constexpr (M > 1) {
#pragma unroll
    for (int k2 = 1; k2 < R1; ++k2) {
      C wv = __ldg(&tw[m * k2]);
      if (INV) wv.y = -wv.y;
      a[k2] = cmul(a[k2], wv);
    }
  }
}

// Offset in the spectrum view of row y for a compile-time y relative to an
// even base row.
template <int N> __device__ __forceinline__ constexpr int yo(int y) {
  return (y >> 1) * PlaneCfg<N>::ZP + (y & 1) * (N / 2);
}

// Forward y transform of the plane held as Z rows (after the forward z
// transform); the result goes to the global half-spectrum plane dst[ky][kz]
// (pitch N/2 + 1).
//
// Stage 1 forms its operands from the Z rows as it loads them (the real ->
// half-spectrum unpacking): for a packed row pair Z = X_a + i X_b (X_a, X_b
// the spectra of the real rows 2r, 2r+1), X_a[k] = (Z[k] + conj Z[N-k]) / 2
// and X_b[k] = (Z[k] - conj Z[N-k]) / (2i); column 0 takes (X[0], X[N/2]),
// both real.  All loads finish before the in-place stores (they alias).
// Stage 2 stores columns c >= 1 straight to global memory; the packed column
// 0 is transformed in shared memory and split afterwards: with
// Y = DFT(a + i b) for real a, b, DFT(a)[k] = (Y[k] + conj Y[-k]) / 2 and
// DFT(b)[k] = (Y[k] - conj Y[-k]) / (2i).
template <typename T, int N>
__device__ __forceinline__ void yfft_fwd_store(cplx<T>* B, cplx<T>* __restrict__ dst,
                                               const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  constexpr int NT = P::NT, NC = P::NC, NH = P::NH, ZP = P::ZP;
  constexpr int G1 = NC * M;
  static_assert(G1 <= NT, "one stage-1 group per thread");
  // ---- stage 1: unpack on load, DFT, twiddles; barrier; store ----
  const int g = threadIdx.x;
  const bool act = g < G1;
  const int c = g % NC, m = (M == 1) ? 0 : g / NC;
  C a[R1];
  if (act) {
#pragma unroll
    for (int j = 0; j < R1; ++j) {
      const int y = m + M * j;
      const C* zr = B + (y >> 1) * ZP;
      C v;
      if (c == 0) {
        const C z0 = zr[0], zn = zr[N / 2];
        v = (y & 1) ? C{z0.y, zn.y} : C{z0.x, zn.x};
      } else {
        const C zk = zr[c], zm = cconj(zr[N - c]);
        const C sp = cadd(zk, zm), df = csub(zk, zm);
        v = (y & 1) ? C{(T)0.5 * df.y, (T)-0.5 * df.x} : C{(T)0.5 * sp.x, (T)0.5 * sp.y};
      }
      a[j] = v;
    }
    stage1_group<T, N, false>(a, m, tw);
  }
  __syncthreads();
  if (act) {
    C* p = B + c + hoff<N>(m);
    if constexpr (M == 1) {      // natural order already: this is the output
      if (c != 0) {
#pragma unroll
        for (int k = 0; k < R1; ++k) dst[k * NH + c] = a[k];
      } else {
#pragma unroll
        for (int k = 0; k < R1; ++k) p[yo<N>(k)] = a[k];
      }
    } else {
#pragma unroll
      for (int k2 = 0; k2 < R1; ++k2) p[k2 * (M / 2) * ZP] = a[k2];
    }
  }
  __syncthreads();
  if constexpr (M > 1) {
    // ---- stage 2 (load all groups, barrier, store in natural order) ----
    constexpr int G2 = NC * R1;
    constexpr int PER = (G2 + NT - 1) / NT;
    C b[PER][M];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int g2 = threadIdx.x + i * NT;
      if (G2 % NT == 0 || g2 < G2) {
        const int c2 = g2 % NC, k2 = g2 / NC;
        const C* q = B + c2 + (M * k2 / 2) * ZP;
#pragma unroll
        for (int mm = 0; mm < M; ++mm) b[i][mm] = q[yo<N>(mm)];
        dft_reg<M, false>(b[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int g2 = threadIdx.x + i * NT;
      if (G2 % NT == 0 || g2 < G2) {
        const int c2 = g2 % NC, k2 = g2 / NC;
        if (c2 != 0) {
#pragma unroll
          for (int k1 = 0; k1 < M; ++k1) dst[(k2 + R1 * k1) * NH + c2] = b[i][k1];
        } else {
          C* q = B + hoff<N>(k2);
#pragma unroll
          for (int k1 = 0; k1 < M; ++k1) q[k1 * (R1 / 2) * ZP] = b[i][k1];
        }
      }
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < N; k += NT) {
    const C y = B[hoff<N>(k)], ym = cconj(B[hoff<N>((N - k) & (N - 1))]);
    const C sp = cadd(y, ym), df = csub(y, ym);
    dst[k * NH] = C{(T)0.5 * sp.x, (T)0.5 * sp.y};
    dst[k * NH + N / 2] = C{(T)0.5 * df.y, (T)-0.5 * df.x};
  }
}

// Inverse z transform of the plane held in the spectrum view (after the
// inverse y transform), to Z rows of real values.  Stage 1 forms the packed
// rows as it loads them: Z[k] = X_a[k] + i X_b[k] with the Hermitian
// extension X[k] = conj X[N-k] for k > N/2 and the real kz = 0, N/2 values
// from column 0.  All loads finish before the in-place stores.
template <typename T, int N>
__device__ __forceinline__ void zfft_inv_packed(cplx<T>* B, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  constexpr int NT = P::NT, NC = P::NC, NR = P::NR, ZP = P::ZP;
  constexpr int G1 = NR * M;
  static_assert(G1 <= NT, "one stage-1 group per thread");
  const int g = threadIdx.x;
  const bool act = g < G1;
  const int r = g % NR, m = (M == 1) ? 0 : g / NR;
  C a[R1];
  if (act) {
    const C* zr = B + r * ZP;
#pragma unroll
    for (int j = 0; j < R1; ++j) {
      const int k = m + M * j;
      C v;
      if ((j == 0 || j == R1 / 2) && m == 0) {     // k = 0 or N/2: real parts from column 0
        const C x0 = zr[0], x1 = zr[NC];
        v = (j == 0) ? C{x0.x, x1.x} : C{x0.y, x1.y};
      } else if (j < R1 / 2) {                     // 0 < k < N/2
        const C x0 = zr[k], x1 = zr[NC + k];
        v = C{x0.x - x1.y, x0.y + x1.x};
      } else {                                     // k > N/2: conjugate of N - k
        const C x0 = cconj(zr[N - k]), x1 = cconj(zr[NC + N - k]);
        v = C{x0.x - x1.y, x0.y + x1.x};
      }
      a[j] = v;
    }
    stage1_group<T, N, true>(a, m, tw);
  }
  __syncthreads();
  if (act) {
    C* p = B + r * ZP + m;
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) p[M * k2] = a[k2];
  }
  __syncthreads();
  fft_smem_stage2<T, N, true, NR, NT>(B, ZP, 1);
}

// Inverse y transform of the global half-spectrum plane src[ky][kz] into the
// spectrum view.  Stage 1 reads global memory directly.  Column 0 packs the
// kz = 0 and kz = N/2 lines as P0 + i PN, where P0 and PN are their Hermitian
// parts along y: the inverse transform of P0 is the real part of the inverse
// transform of the kz = 0 line, which is what a c2r transform keeps.
template <typename T, int N>
__device__ __forceinline__ void yfft_inv_load(cplx<T>* B, const cplx<T>* __restrict__ src,
                                              const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  constexpr int NT = P::NT, NC = P::NC, NH = P::NH, ZP = P::ZP;
  constexpr int G1 = NC * M;
#pragma unroll 1
  for (int g = threadIdx.x; g < G1; g += NT) {
    const int c = g % NC, m = (M == 1) ? 0 : g / NC;
    C a[R1];
    if (c != 0) {
#pragma unroll
      for (int j = 0; j < R1; ++j) a[j] = __ldg(&src[(m + M * j) * NH + c]);
    } else {
#pragma unroll
      for (int j = 0; j < R1; ++j) {
        const int y = m + M * j, ym = (N - y) & (N - 1);
        const C h0 = __ldg(&src[y * NH]), h0m = __ldg(&src[ym * NH]);
        const C hn = __ldg(&src[y * NH + N / 2]), hnm = __ldg(&src[ym * NH + N / 2]);
        const C p0 = C{(T)0.5 * (h0.x + h0m.x), (T)0.5 * (h0.y - h0m.y)};
        const C pn = C{(T)0.5 * (hn.x + hnm.x), (T)0.5 * (hn.y - hnm.y)};
        a[j] = C{p0.x - pn.y, p0.y + pn.x};
      }
    }
    stage1_group<T, N, true>(a, m, tw);
    C* p = B + c + hoff<N>(m);
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) p[(M == 1) ? yo<N>(k2) : k2 * (M / 2) * ZP] = a[k2];
  }
  __syncthreads();
  if constexpr (M > 1) {
    constexpr int G2 = NC * R1;
    constexpr int PER = (G2 + NT - 1) / NT;
    C a[PER][M];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int g = threadIdx.x + i * NT;
      if (G2 % NT == 0 || g < G2) {
        const int c = g % NC, k2 = g / NC;
        const C* q = B + c + (M * k2 / 2) * ZP;
#pragma unroll
        for (int m = 0; m < M; ++m) a[i][m] = q[yo<N>(m)];
        dft_reg<M, true>(a[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int g = threadIdx.x + i * NT;
      if (G2 % NT == 0 || g < G2) {
        const int c = g % NC, k2 = g / NC;
        C* q = B + c + hoff<N>(k2);
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) q[k1 * (R1 / 2) * ZP] = a[i][k1];
      }
    }
    __syncthreads();
  }
}

// Bucket ranges of the plane's two point sets: side 0 has its lower CIC
// corner on this plane (bucket ix), side 1 its upper corner (bucket ix-1).
struct PlaneBuckets {
  int b0, n0, b1, n1;
};
template <int N>
__device__ __forceinline__ PlaneBuckets plane_buckets(const int* __restrict__ off, int c, int ix) {
  const int* o = off + (long long)c * (N + 1);
  const int ixm = (ix + N - 1) & (N - 1);
  PlaneBuckets pb;
  pb.b0 = o[ix];
  pb.n0 = o[ix + 1] - o[ix];
  pb.b1 = o[ixm];
  pb.n1 = o[ixm + 1] - o[ixm];
  return pb;
}

template <typename T> __device__ __forceinline__ T rcomp(const PtRec<T>& p, int j) {
  return j == 0 ? p.rx : (j == 1 ? p.ry : p.rz);
}

// ---------------------------------------------------------------------------
// Plane pass, forward: real plane x -> (z r2c, y c2c) -> spectrum plane.
// SCATTER builds the plane from the bucketed points instead of loading it:
// s_j(corner) += r rhat_j W(corner), with shared-memory atomics (the adjoint
// of the CIC gather, restricted to this plane).
// ---------------------------------------------------------------------------
template <typename T, int N, bool SCATTER>
__global__ void __launch_bounds__(PlaneCfg<N>::NT, (sizeof(T) == 4 ? PlaneCfg<N>::MINB : 1))
k_plane_r2c(const T* __restrict__ in, long long in_stride, cplx<T>* __restrict__ out,
            long long out_stride, const cplx<T>* __restrict__ tw, PlanePoints pts) {
  pdl_wait();
  pdl_trigger();
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int NT = P::NT, ZP = P::ZP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* B = reinterpret_cast<C*>(smem_raw);
  const int ix = blockIdx.x;
  const int s = blockIdx.y;
  if constexpr (!SCATTER) {
    const T* src = in + (long long)s * in_stride + (long long)ix * N * N;
    for (int e = threadIdx.x; e < P::NR * N; e += NT) {
      const int r = e / N, z = e % N;
      B[r * ZP + z] = C{__ldg(&src[(2 * r) * N + z]), __ldg(&src[(2 * r + 1) * N + z])};
    }
  } else {
    const int c = s / 3, j = s % 3;
    const PlaneBuckets pb = plane_buckets<N>(pts.off, c, ix);
    // no point has a CIC corner on this plane: its spectrum is zero, which
    // the adjoint pencil pass knows from the same bucket offsets, so nothing
    // is written
    if (pb.n0 + pb.n1 == 0) return;
    for (int e = threadIdx.x; e < P::SIZE; e += NT) B[e] = C{(T)0, (T)0};
    __syncthreads();
    const PtRec<T>* R = static_cast<const PtRec<T>*>(pts.rec);
    for (int t = threadIdx.x; t < pb.n0 + pb.n1; t += NT) {
      const bool lower = t < pb.n0;
      const PtRec<T> p = R[lower ? pb.b0 + t : pb.b1 + (t - pb.n0)];
      const T val = p.r * rcomp(p, j) * (lower ? (T)1 - p.fx : p.fx);
      if (val == (T)0) continue;
      const int iy = p.yz / N, iz = p.yz % N;
      const int iy1 = (iy + 1) & (N - 1), iz1 = (iz + 1) & (N - 1);
      const T wy1 = p.fy, wy0 = (T)1 - p.fy, wz1 = p.fz, wz0 = (T)1 - p.fz;
      atomicAdd(zreal<T, N>(B, iy, iz), val * wy0 * wz0);
      atomicAdd(zreal<T, N>(B, iy, iz1), val * wy0 * wz1);
      atomicAdd(zreal<T, N>(B, iy1, iz), val * wy1 * wz0);
      atomicAdd(zreal<T, N>(B, iy1, iz1), val * wy1 * wz1);
    }
  }
  __syncthreads();
  zfft<T, N, false>(B, tw);
  yfft_fwd_store<T, N>(B, out + (long long)s * out_stride + (long long)ix * N * P::NH, tw);
}

// ---------------------------------------------------------------------------
// Plane pass, inverse: spectrum plane -> (y c2c, z c2r) -> real plane, then
// MODE 0: plain store; 1: gradient / leapfrog epilogue; 2: CIC gather of the
// bucketed points (u and du partials of this plane and component).
// ---------------------------------------------------------------------------
enum C2RMode : int { C2R_STORE = 0, C2R_EPI = 1, C2R_GATHER = 2 };

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(PlaneCfg<N>::NT, (sizeof(T) == 4 ? PlaneCfg<N>::MINB : 1))
k_plane_c2r(const cplx<T>* __restrict__ in, long long in_stride, T* __restrict__ out,
            long long out_stride, const cplx<T>* __restrict__ tw, FieldEpi epi, PlanePoints pts,
            cplx<T>* __restrict__ next, long long next_stride) {
  pdl_wait();
  pdl_trigger();
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int NT = P::NT, ZP = P::ZP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* B = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[2][NT / 32];
  const int ix = blockIdx.x;
  const int s = blockIdx.y;
  if constexpr (MODE == C2R_GATHER) {
    // only the values at the points' corners are used: a plane that no
    // point touches needs no transform
    const PlaneBuckets pb = plane_buckets<N>(pts.off, s / 3, ix);
    if (pb.n0 + pb.n1 == 0) return;
  }
  yfft_inv_load<T, N>(B, in + (long long)s * in_stride + (long long)ix * N * P::NH, tw);
  zfft_inv_packed<T, N>(B, tw);
  constexpr int ITEMS = P::NR * N;   // item (r, z): real rows 2r, 2r+1 at column z
  if constexpr (MODE == C2R_STORE) {
    T* dst = out + (long long)s * out_stride + (long long)ix * N * N;
    for (int e = threadIdx.x; e < ITEMS; e += NT) {
      const int r = e / N, z = e % N;
      const C v = B[r * ZP + z];
      dst[(2 * r) * N + z] = v.x;
      dst[(2 * r + 1) * N + z] = v.y;
    }
  } else if constexpr (MODE == C2R_GATHER) {
    const int c = s / 3, j = s % 3;
    const PlaneBuckets pb = plane_buckets<N>(pts.off, c, ix);
    const PtRec<T>* R = static_cast<const PtRec<T>*>(pts.rec);
    T* part = static_cast<T*>(pts.part);
    const T idl = (T)pts.inv_delta;
    for (int t = threadIdx.x; t < pb.n0 + pb.n1; t += NT) {
      const bool lower = t < pb.n0;
      const int q = lower ? pb.b0 + t : pb.b1 + (t - pb.n0);
      const PtRec<T> p = R[q];
      const int iy = p.yz / N, iz = p.yz % N;
      const int iy1 = (iy + 1) & (N - 1), iz1 = (iz + 1) & (N - 1);
      const T v00 = *zreal<T, N>(B, iy, iz), v01 = *zreal<T, N>(B, iy, iz1);
      const T v10 = *zreal<T, N>(B, iy1, iz), v11 = *zreal<T, N>(B, iy1, iz1);
      const T wy1 = p.fy, wy0 = (T)1 - p.fy, wz1 = p.fz, wz0 = (T)1 - p.fz;
      const T a0 = wz0 * v00 + wz1 * v01, a1 = wz0 * v10 + wz1 * v11;
      const T S = wy0 * a0 + wy1 * a1;      // y-z interpolation on this plane
      const T Gy = a1 - a0;                 // d/dy (per cell) of it
      const T Gz = wy0 * (v01 - v00) + wy1 * (v11 - v10);
      const T wx = lower ? (T)1 - p.fx : p.fx;
      const T sx = lower ? (T)-1 : (T)1;
      const T rj = rcomp(p, j);
      const int side = lower ? 0 : 1;
      part[(long long)(side * 3 + j) * pts.ntot + q] = rj * wx * S;
      part[(long long)(6 + side * 3 + j) * pts.ntot + q] =
          rj * (p.rx * sx * S + p.ry * wx * Gy + p.rz * wx * Gz) * idl;
    }
  } else {
    // ---- gradient / leapfrog epilogue (one chain per blockIdx.y) ----
    const long long base = (long long)s * epi.grid_stride + (long long)ix * N * N;
    T* __restrict__ w = reinterpret_cast<T*>(epi.w) + base;
    T* __restrict__ pw = reinterpret_cast<T*>(epi.pw) + base;
    T* __restrict__ gw = reinterpret_cast<T*>(epi.gw) + base;
    const int mode = epi.mode;
    const T eps = (T)epi.cs[s].eps;
    const T ck = (mode == GM_KICK_DRIFT) ? eps : (T)0.5 * eps;
    const bool fuse_next = next != nullptr && mode == GM_KICK_DRIFT;
    const bool kick = mode != GM_GRAD;
    // the prior and kinetic sums are read only at the trajectory's end point
    // (and for GM_GRAD): an intermediate leapfrog evaluation skips them
    const bool sums = mode != GM_KICK_DRIFT, last = mode == GM_KICK_LAST;
    HalfSqAcc<T> aw, ap;
    // U items per thread per round: all their global loads are issued before
    // any store, so their latencies overlap
    constexpr int U = ITEMS >= 4 * NT ? 4 : 1;
    constexpr bool FULL = ITEMS % (U * NT) == 0;
#pragma unroll 1
    for (int e0 = threadIdx.x; e0 < ITEMS; e0 += U * NT) {
      T wv[U][2], pv[U][2];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NT, r = e / N, z = e % N;
        if (!FULL && e >= ITEMS) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int o = (2 * r + h) * N + z;
          wv[u][h] = w[o];
          pv[u][h] = kick ? pw[o] : (T)0;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NT, r = e / N, z = e % N;
        if (!FULL && e >= ITEMS) continue;
        const C g2 = B[r * ZP + z];
        T nv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // row 2r + h, column z
          const int o = (2 * r + h) * N + z;
          const T w0 = wv[u][h];
          const T g0 = w0 + (h == 0 ? g2.x : g2.y);
          if (sums) aw.add_half_sq(w0);
          nv[h] = w0;
          if (mode == GM_GRAD || mode == GM_KICK_LAST) gw[o] = g0;
          if (kick) {
            const T p0 = pv[u][h] - ck * g0;
            pw[o] = p0;
            if (last) ap.add_half_sq(p0);
            if (mode == GM_KICK_DRIFT) {
              nv[h] = w0 + eps * p0;
              w[o] = nv[h];
            }
          }
        }
        if (fuse_next) B[r * ZP + z] = C{nv[0], nv[1]};   // the drifted field replaces g in the buffer
      }
    }
    // deterministic block reduction: a fixed shuffle tree per warp, then
    // thread 0 over the warps in order (the barrier also completes the
    // drifted rows in B before the forward transform reads them)
    if (sums) {
      aw.warp_reduce();
      if (last) ap.warp_reduce();
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (sums && lane == 0) {
      red[0][wid] = aw.value();
      red[1][wid] = ap.value();
    }
    __syncthreads();
    if (sums && threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int i = 0; i < NT / 32; ++i) {
        a += red[0][i];
        b += red[1][i];
      }
      epi.prior_part[(long long)s * N + ix] = a;
      if (mode == GM_KICK_LAST) epi.kin_part[(long long)s * N + ix] = b;
    }
    if (fuse_next) {
      // forward plane transform of the drifted field for the next evaluation
      zfft<T, N, false>(B, tw);
      yfft_fwd_store<T, N>(B, next + (long long)s * next_stride + (long long)ix * N * P::NH, tw);
    }
  }
}

// ---------------------------------------------------------------------------
// Pencil pass along x with the fused k-space operator.
// amp[n2] = (2 pi/L) aHf sqrt(P(k)/Delta^3) / (k^2 N^3), amp[0] = 0, so that
// the velocity spectrum of axis j is i n_j^odd amp[n^2] w_k.
//
// A CTA owns a tile of kTC contiguous (ky, kz) columns over all N x rows and
// keeps one [N][kTC] buffer per component in shared memory.  The first radix
// stage of a transform reads global memory directly, the last radix stage
// of the final inverse writes global memory directly, and the k-space
// weights are applied while the inverse transform's first stage loads its
// operands, so only the middle of each transform passes through shared
// memory.
// ---------------------------------------------------------------------------
constexpr int kTC = 16;       // (ky, kz) columns per tile
// Threads of a pencil CTA: 128, or 256 at N = 256, where the three
// component tiles (96 KB) let only two CTAs share an SM and every thread
// then takes one stage-1 group instead of two.
template <int N> struct PencilNT { static constexpr int v = N >= 256 ? 256 : 128; };

template <typename T, int N> struct PencilMinB {
  static constexpr int v = N >= 256 ? 2 : (sizeof(T) == 4 ? 4 : 2);
};

// Stage 1 of the x transform for group (t, m), operands read from global
// memory (zero for a column past the end), result to the component buffer.
// rows: bit j set when row m + M j is to be read (else it is zero).
template <typename T, int N, bool INV, int W>
__device__ __forceinline__ void px_s1_global(cplx<T>* buf, const cplx<T>* __restrict__ src, long long col,
                                             bool ok, int t, int m, const cplx<T>* __restrict__ tw,
                                             unsigned rows) {
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M, NCOL = N * (N / 2 + 1);
  C a[R1];
#pragma unroll
  for (int j = 0; j < R1; ++j)
    a[j] = (ok && ((rows >> j) & 1u)) ? __ldg(&src[(long long)(m + M * j) * NCOL + col]) : C{(T)0, (T)0};
  stage1_group<T, N, INV>(a, m, tw);
#pragma unroll
  for (int k2 = 0; k2 < R1; ++k2) buf[(m + M * k2) * W + t] = a[k2];
}

// Stage 2 of the x transform of one component, in place in shared memory
// (natural order out).  Contains block barriers.
template <typename T, int N, bool INV, int W>
__device__ __forceinline__ void px_s2_smem(cplx<T>* buf) {
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  if constexpr (M > 1) {
    constexpr int G2 = kTC * R1;
    constexpr int PER = (G2 + PencilNT<N>::v - 1) / PencilNT<N>::v;
    C a[PER][M];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int g = threadIdx.x + i * PencilNT<N>::v;
      if (G2 % PencilNT<N>::v == 0 || g < G2) {
        const int t = g % kTC, k2 = g / kTC;
#pragma unroll
        for (int m = 0; m < M; ++m) a[i][m] = buf[(M * k2 + m) * W + t];
        dft_reg<M, INV>(a[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int g = threadIdx.x + i * PencilNT<N>::v;
      if (G2 % PencilNT<N>::v == 0 || g < G2) {
        const int t = g % kTC, k2 = g / kTC;
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) buf[(k2 + R1 * k1) * W + t] = a[i][k1];
      }
    }
    __syncthreads();
  }
}

// Stage 2 of the x transform of one component, results straight to global
// memory in natural order (a plain copy when N = R1).
template <typename T, int N, bool INV, int W>
__device__ __forceinline__ void px_s2_global(const cplx<T>* buf, cplx<T>* __restrict__ dst, int c0) {
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M, NCOL = N * (N / 2 + 1);
#pragma unroll 1
  for (int g = threadIdx.x; g < kTC * R1; g += PencilNT<N>::v) {
    const int t = g % kTC, k2 = g / kTC;
    C a[M];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = buf[(M * k2 + m) * W + t];
    dft_reg<M, INV>(a);
    const long long col = c0 + t;
    if (col < NCOL) {
#pragma unroll
      for (int k1 = 0; k1 < M; ++k1) dst[(long long)(k2 + R1 * k1) * NCOL + col] = a[k1];
    }
  }
}

// k-space geometry of column col of the tile: ny, nz (signed mode numbers)
// and the odd factors of the y and z axes (0 on their Nyquist planes).
template <int N> struct ColGeom {
  int ny2nz2;
  float oy, oz;
};
template <int N> __device__ __forceinline__ ColGeom<N> col_geom(long long col) {
  constexpr int NH = N / 2 + 1;
  const int ky = (int)(col / NH), kz = (int)(col % NH);
  const int ny = ky < N / 2 ? ky : ky - N;
  ColGeom<N> g;
  g.ny2nz2 = ny * ny + kz * kz;
  g.oy = (ky == N / 2) ? 0.f : (float)ny;
  g.oz = (kz == N / 2) ? 0.f : (float)kz;
  return g;
}

// Everything of the x pass after the first transform's stage 1 (whose result
// is in buf): its stage 2, the k-space operator and the inverse transform(s),
// the last stage written to global memory.  Shared by the pencil kernels.
template <typename T, int N, int MODE>
__device__ __forceinline__ void pencil_finish(cplx<T>* buf, cplx<T>* __restrict__ out, long long out_stride,
                                              int s, int c0, const cplx<T>* __restrict__ tw,
                                              const T* __restrict__ amp) {
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  constexpr int NCOL = N * (N / 2 + 1);
  constexpr int NCOMP = (MODE == PM_VEL || MODE == PM_ADJ) ? 3 : 1;
  constexpr int W = NCOMP * kTC;
  constexpr int NIN = (MODE == PM_ADJ) ? 3 : 1;
  constexpr bool INV1 = (MODE == PM_INV);
  if constexpr (MODE == PM_FWD || MODE == PM_INV) {
    px_s2_global<T, N, INV1, W>(buf, out + (long long)s * out_stride, c0);
  } else {
#pragma unroll 1
    for (int j = 0; j < NIN; ++j) px_s2_smem<T, N, false, W>(buf + j * kTC);
    // inverse transform(s): stage 1 loads the natural-order spectra and
    // applies the k-space operator on the way in
    if constexpr (MODE == PM_SCALE) {
      // real weight amp[n^2] applied as the inverse's first stage loads
#pragma unroll 1
      for (int g = threadIdx.x; g < kTC * M; g += PencilNT<N>::v) {
        const int t = g % kTC, m = g / kTC;
        const long long col = c0 + t;
        const ColGeom<N> cg = col_geom<N>(col < NCOL ? col : 0);
        C a[R1];
#pragma unroll
        for (int jj = 0; jj < R1; ++jj) {
          const int kx = m + M * jj;
          const int nx = kx < N / 2 ? kx : kx - N;
          const T am = __ldg(&amp[nx * nx + cg.ny2nz2]);
          const C wk = buf[kx * W + t];
          a[jj] = C{am * wk.x, am * wk.y};
        }
        stage1_group<T, N, true>(a, m, tw);
#pragma unroll
        for (int k2 = 0; k2 < R1; ++k2) buf[(m + M * k2) * W + t] = a[k2];
      }
      __syncthreads();
      px_s2_global<T, N, true, W>(buf, out + (long long)s * out_stride, c0);
    } else if constexpr (MODE == PM_VEL) {
      // component order y, z, x: x is written over the input spectrum, and
      // each group reads and writes only its own elements
#pragma unroll 1
      for (int q = 0; q < 3; ++q) {
        const int jo = q == 2 ? 0 : q + 1;
#pragma unroll 1
        for (int g = threadIdx.x; g < kTC * M; g += PencilNT<N>::v) {
          const int t = g % kTC, m = g / kTC;
          const long long col = c0 + t;
          const ColGeom<N> cg = col_geom<N>(col < NCOL ? col : 0);
          C a[R1];
#pragma unroll
          for (int jj = 0; jj < R1; ++jj) {
            const int kx = m + M * jj;
            const int nx = kx < N / 2 ? kx : kx - N;
            const T am = __ldg(&amp[nx * nx + cg.ny2nz2]);
            const T o = (T)(jo == 0 ? ((kx == N / 2) ? 0.f : (float)nx) : (jo == 1 ? cg.oy : cg.oz));
            const C wk = buf[kx * W + t];
            a[jj] = C{-am * o * wk.y, am * o * wk.x};   // i amp n_j w_k
          }
          stage1_group<T, N, true>(a, m, tw);
#pragma unroll
          for (int k2 = 0; k2 < R1; ++k2) buf[(m + M * k2) * W + jo * kTC + t] = a[k2];
        }
      }
      __syncthreads();
#pragma unroll 1
      for (int jo = 0; jo < 3; ++jo)
        px_s2_global<T, N, true, W>(buf + jo * kTC, out + (long long)(s * 3 + jo) * out_stride, c0);
    } else {
      // PM_ADJ: -i amp sum_j n_j s_j, written over component 0
#pragma unroll 1
      for (int g = threadIdx.x; g < kTC * M; g += PencilNT<N>::v) {
        const int t = g % kTC, m = g / kTC;
        const long long col = c0 + t;
        const ColGeom<N> cg = col_geom<N>(col < NCOL ? col : 0);
        C a[R1];
#pragma unroll
        for (int jj = 0; jj < R1; ++jj) {
          const int kx = m + M * jj;
          const int nx = kx < N / 2 ? kx : kx - N;
          const T am = __ldg(&amp[nx * nx + cg.ny2nz2]);
          const T ox = (kx == N / 2) ? (T)0 : (T)nx;
          const C sx = buf[kx * W + t], sy = buf[kx * W + kTC + t], sz = buf[kx * W + 2 * kTC + t];
          const C sum = C{ox * sx.x + (T)cg.oy * sy.x + (T)cg.oz * sz.x, ox * sx.y + (T)cg.oy * sy.y + (T)cg.oz * sz.y};
          a[jj] = C{am * sum.y, -am * sum.x};
        }
        stage1_group<T, N, true>(a, m, tw);
#pragma unroll
        for (int k2 = 0; k2 < R1; ++k2) buf[(m + M * k2) * W + t] = a[k2];
      }
      __syncthreads();
      px_s2_global<T, N, true, W>(buf, out + (long long)s * out_stride, c0);
    }
  }
}

// PM_ADJ reads the x-planes of the three scatter spectra whose planes carry
// points; plane_off (the per-chain bucket offsets of the points, ksplit
// sub-buckets per plane, as the scatter plane pass used them) says which:
// plane x is nonzero when bucket x or x-1 is non-empty.  plane_off ==
// nullptr reads every plane.
template <typename T, int N, int MODE>
__global__ void __launch_bounds__(PencilNT<N>::v, PencilMinB<T, N>::v)
k_pencil(const cplx<T>* __restrict__ in, long long in_stride, cplx<T>* __restrict__ out,
         long long out_stride, const cplx<T>* __restrict__ tw, const T* __restrict__ amp,
         const int* __restrict__ plane_off, int ksplit) {
  pdl_wait();
  pdl_trigger();
  // x-planes to read, one bit per plane, kept in registers (PM_ADJ only)
  constexpr int NW = N >= 32 ? N / 32 : 1;
  unsigned occw[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) occw[k] = 0xffffffffu;
  if constexpr (MODE == PM_ADJ) {
    __shared__ unsigned occ_s[NW];
    if (plane_off != nullptr) {
      const int* o = plane_off + (long long)blockIdx.y * (N * ksplit + 1);
      const int lane = threadIdx.x & 31;
      for (int x0 = (threadIdx.x >> 5) * 32; x0 < N; x0 += PencilNT<N>::v) {
        const int x = x0 + lane, xm = (x + N - 1) & (N - 1);
        const bool on = x < N && ((o[(x + 1) * ksplit] != o[x * ksplit]) || (o[(xm + 1) * ksplit] != o[xm * ksplit]));
        const unsigned word = __ballot_sync(0xffffffffu, on);
        if (lane == 0) occ_s[x0 >> 5] = word;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < NW; ++k) occw[k] = occ_s[k];
    }
  }
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  constexpr int NCOL = N * (N / 2 + 1);
  constexpr int NCOMP = (MODE == PM_VEL || MODE == PM_ADJ) ? 3 : 1;
  constexpr int W = NCOMP * kTC;   // smem row width: NCOMP tiles side by side
  constexpr int NIN = (MODE == PM_ADJ) ? 3 : 1;
  constexpr bool INV1 = (MODE == PM_INV);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [N][W]
  const int c0 = blockIdx.x * kTC;
  const int s = blockIdx.y;
  // first transform (forward; inverse for PM_INV), stage 1 from global memory
#pragma unroll 1
  for (int g = threadIdx.x; g < NIN * kTC * M; g += PencilNT<N>::v) {
    const int t = g % kTC, m = (g / kTC) % M, j = g / (kTC * M);
    const long long col = c0 + t;
    // rows m + M jj of this group: word (M jj) / 32, bit m + (M jj) % 32
    // (M divides 32 and m < M)
    unsigned rows = 0xffffffffu;
    if constexpr (MODE == PM_ADJ) {
      rows = 0;
#pragma unroll
      for (int jj = 0; jj < R1; ++jj) rows |= ((occw[(M * jj) >> 5] >> (m + ((M * jj) & 31))) & 1u) << jj;
    }
    px_s1_global<T, N, INV1, W>(buf + j * kTC, in + (long long)(s * NIN + j) * in_stride, col, col < NCOL, t, m,
                                tw, rows);
  }
  __syncthreads();
  pencil_finish<T, N, MODE>(buf, out, out_stride, s, c0, tw, amp);
}

// ---------------------------------------------------------------------------
// Pencil pass with TMA-staged input (FP32, N = 128 and 256; the single-input
// modes).  A persistent CTA walks the (grid, column tile) items with stride
// gridDim.x; while it transforms one tile, the tensor copy engine loads the
// next tile (N rows x kTC columns, N * 128 bytes, one cp.async.bulk.tensor)
// into the other of two shared-memory buffers, completing on an mbarrier.
// The global-load latency that bounds the plain pencil pass (its first radix
// stage reads global memory) is then hidden behind the previous tile's work.
// Every wait on a copy is bounded: after kTmaWaitPolls polls the CTA gives
// up, counts the event in g_tma_wait_timeouts, waits (bounded) for its other
// copy in flight and returns.
// ---------------------------------------------------------------------------
__device__ int g_tma_wait_timeouts;
constexpr int kTmaWaitPolls = 1 << 20;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (int it = 0; it < kTmaWaitPolls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// One tile of the grid `z`: columns [x, x + 2 kTC) floats (kTC complex) of all
// N rows; completes tx bytes on `bar`.
__device__ __forceinline__ void tma_tile_load(void* dst, const CUtensorMap* map, int x, int z,
                                              unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(0), "r"(z),
      "r"(smem_addr(bar))
      : "memory");
}

template <int N> constexpr unsigned tma_tile_bytes() { return (unsigned)(N * kTC * sizeof(float2)); }
template <int N, int MODE> constexpr size_t tma_pencil_smem() {
  constexpr int NCOMP = MODE == PM_VEL ? 3 : 1;
  return 128 + 2 * (size_t)tma_tile_bytes<N>() + sizeof(float2) * N * NCOMP * kTC;
}

template <int N, int MODE>
__global__ void __launch_bounds__(PencilNT<N>::v, 1)
k_pencil_tma(const __grid_constant__ CUtensorMap in_map, float2* __restrict__ out, long long out_stride,
             const float2* __restrict__ tw, const float* __restrict__ amp, int count) {
  static_assert(MODE != PM_ADJ, "single-input modes");
  using C = float2;
  constexpr int NT = PencilNT<N>::v;
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  constexpr int NCOL = N * (N / 2 + 1);
  static_assert(NCOL % kTC == 0, "whole tiles");
  constexpr int NTILE = NCOL / kTC;
  constexpr int NCOMP = MODE == PM_VEL ? 3 : 1;
  constexpr int W = NCOMP * kTC;
  constexpr bool INV1 = MODE == PM_INV;
  constexpr unsigned TB = tma_tile_bytes<N>();
  extern __shared__ unsigned char smem_raw[];
  // tensor copies land on 128-byte boundaries
  unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  auto stage = [&](int b) { return reinterpret_cast<C*>(base + (size_t)b * TB); };
  C* buf = reinterpret_cast<C*>(base + 2 * TB);   // [N][W]
  __shared__ __align__(8) unsigned long long bar[2];
  pdl_wait();
  pdl_trigger();
  const int items = NTILE * count;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int item = blockIdx.x;
  if (threadIdx.x == 0 && item < items)
    tma_tile_load(stage(0), &in_map, (item % NTILE) * kTC * 2, item / NTILE, &bar[0], TB);
  for (int k = 0; item < items; ++k, item += gridDim.x) {
    const int b = k & 1;
    const int next = item + gridDim.x;
    if (threadIdx.x == 0 && next < items) {
      // the other buffer was last read before the previous iteration's
      // final barrier; order those reads before the async-proxy write
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tma_tile_load(stage(b ^ 1), &in_map, (next % NTILE) * kTC * 2, next / NTILE, &bar[b ^ 1], TB);
    }
    const bool ok = mbar_wait_bounded(&bar[b], (unsigned)(k >> 1) & 1u);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicAdd(&g_tma_wait_timeouts, 1);
        if (next < items) mbar_wait_bounded(&bar[b ^ 1], (unsigned)((k + 1) >> 1) & 1u);
      }
      return;
    }
    const int s = item / NTILE, c0 = (item % NTILE) * kTC;
    const C* in = stage(b);
    // first transform (forward; inverse for PM_INV), stage 1 from the staged tile
#pragma unroll 1
    for (int g = threadIdx.x; g < kTC * M; g += NT) {
      const int t = g % kTC, m = g / kTC;
      C a[R1];
#pragma unroll
      for (int jj = 0; jj < R1; ++jj) a[jj] = in[(m + M * jj) * kTC + t];
      stage1_group<float, N, INV1>(a, m, tw);
#pragma unroll
      for (int k2 = 0; k2 < R1; ++k2) buf[(m + M * k2) * W + t] = a[k2];
    }
    __syncthreads();
    pencil_finish<float, N, MODE>(buf, out, out_stride, s, c0, tw, amp);
    __syncthreads();   // buf and this stage buffer are reused
  }
}

// cuTensorMapEncodeTiled from the driver (no link-time dependency on it).
typedef CUresult (*TensorMapEncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                           const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                           CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                           CUtensorMapFloatOOBfill);
static TensorMapEncodeTiledFn tensor_map_encoder() {
  static const TensorMapEncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<TensorMapEncodeTiledFn>(nullptr);
    return reinterpret_cast<TensorMapEncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor map of `count` spectra (N x N x (N/2+1) complex, `stride` complex
// apart) as floats [count][N][2 N (N/2+1)], tiles of 2 kTC floats x N rows.
template <int N>
static cudaError_t spectra_tensor_map(CUtensorMap* map, const void* in, long long stride, int count) {
  const TensorMapEncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  constexpr unsigned long long NCOL = (unsigned long long)N * (N / 2 + 1);
  const cuuint64_t dims[3] = {2 * NCOL, (cuuint64_t)N, (cuuint64_t)count};
  const cuuint64_t strides[2] = {NCOL * sizeof(float2), (cuuint64_t)stride * sizeof(float2)};
  const cuuint32_t box[3] = {2 * kTC, (cuuint32_t)N, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(in), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int N, int MODE>
static cudaError_t pencil_tma_t(const void* in, long long in_stride, void* out, long long out_stride, int count,
                                const void* tw, const void* amp, cudaStream_t st) {
  // the tensor map needs 16-byte aligned addresses and strides
  if ((reinterpret_cast<uintptr_t>(in) & 15u) != 0 || ((in_stride * (long long)sizeof(float2)) & 15) != 0)
    return cudaErrorMisalignedAddress;
  CUtensorMap map;
  cudaError_t e = spectra_tensor_map<N>(&map, in, in_stride, count);
  if (e != cudaSuccess) return e;
  constexpr size_t sm = tma_pencil_smem<N, MODE>();
  int dev = 0, nsm = 0, per = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pencil_tma<N, MODE>, PencilNT<N>::v, sm)) !=
      cudaSuccess)
    return e;
  const long long items = (long long)(N * (N / 2 + 1) / kTC) * count;
  const int grid = (int)std::min<long long>(items, (long long)nsm * std::max(per, 1));
  return launch_k<PDL_PENCIL>(k_pencil_tma<N, MODE>, dim3(grid), dim3(PencilNT<N>::v), sm, st, map,
                              static_cast<float2*>(out), out_stride, static_cast<const float2*>(tw),
                              static_cast<const float*>(amp), count);
}

template <int N>
static cudaError_t prepare_pencil_tma() {
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_pencil_tma<N, PM_FWD>, A, (int)tma_pencil_smem<N, PM_FWD>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_pencil_tma<N, PM_INV>, A, (int)tma_pencil_smem<N, PM_INV>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_pencil_tma<N, PM_SCALE>, A, (int)tma_pencil_smem<N, PM_SCALE>())) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(k_pencil_tma<N, PM_VEL>, A, (int)tma_pencil_smem<N, PM_VEL>());
}

int fft_tma_wait_timeouts(bool reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tma_wait_timeouts, sizeof(int)) != cudaSuccess) return -1;
  if (reset) {
    const int z = 0;
    if (cudaMemcpyToSymbol(g_tma_wait_timeouts, &z, sizeof(int)) != cudaSuccess) return -1;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <typename T, int N, bool SC>
static cudaError_t plane_r2c_t(const void* in, long long in_stride, void* out, long long out_stride,
                               int count, const void* tw, const PlanePoints& pts, cudaStream_t st) {
  constexpr size_t sm = plane_smem_bytes<T, N>();
  dim3 grid(N, count);
  return launch_k<PDL_PLANE>(k_plane_r2c<T, N, SC>, grid, dim3(PlaneCfg<N>::NT), sm, st, static_cast<const T*>(in), in_stride,
                  static_cast<cplx<T>*>(out), out_stride, static_cast<const cplx<T>*>(tw), pts);
}

template <typename T, int N, int MODE>
static cudaError_t plane_c2r_t(const void* in, long long in_stride, void* out, long long out_stride,
                               int count, const void* tw, const FieldEpi* epi, const PlanePoints& pts,
                               cudaStream_t st, void* next = nullptr) {
  constexpr size_t sm = plane_smem_bytes<T, N>();
  dim3 grid(N, count);
  FieldEpi e{};
  if (epi) e = *epi;
  return launch_k<PDL_PLANE>(k_plane_c2r<T, N, MODE>, grid, dim3(PlaneCfg<N>::NT), sm, st, static_cast<const cplx<T>*>(in),
                  in_stride, static_cast<T*>(out), out_stride, static_cast<const cplx<T>*>(tw), e, pts,
                  static_cast<cplx<T>*>(next), in_stride);
}

template <typename T, int N, int MODE>
static cudaError_t pencil_t(const void* in, long long in_stride, void* out, long long out_stride,
                            int count, const void* tw, const void* amp, cudaStream_t st,
                            const int* plane_off = nullptr, int ksplit = 1) {
  constexpr int NH = N / 2 + 1;
  constexpr int NCOMP = (MODE == PM_VEL || MODE == PM_ADJ) ? 3 : 1;
  constexpr size_t sm = sizeof(cplx<T>) * N * NCOMP * kTC;
  dim3 grid((N * NH + kTC - 1) / kTC, count);
  return launch_k<PDL_PENCIL>(k_pencil<T, N, MODE>, grid, dim3(PencilNT<N>::v), sm, st, static_cast<const cplx<T>*>(in), in_stride,
                  static_cast<cplx<T>*>(out), out_stride, static_cast<const cplx<T>*>(tw),
                  static_cast<const T*>(amp), plane_off, ksplit);
}

// Supported grids: N in {8, 16, 32, 64, 128} at both precisions (one x-plane
// of the half spectrum fits one CTA's shared memory), and N = 256 at FP32
// (plane passes as a z pass over row slabs and a y pass over column tiles,
// hm_fft_256.cu).
bool fft_supported(int prec, int N) {
  return N == 8 || N == 16 || N == 32 || N == 64 || N == 128 || (N == 256 && prec == 0);
}

int plane_split(int N) { return N == 256 ? 8 : 1; }

#define HM_DISPATCH_N(PREC, N, CALL_F, CALL_D)                          \
  do {                                                                  \
    if ((PREC) == 0) {                                                  \
      switch (N) {                                                      \
        case 8: { using T = float; constexpr int NN = 8; return CALL_F; }     \
        case 16: { using T = float; constexpr int NN = 16; return CALL_F; }   \
        case 32: { using T = float; constexpr int NN = 32; return CALL_F; }   \
        case 64: { using T = float; constexpr int NN = 64; return CALL_F; }   \
        case 128: { using T = float; constexpr int NN = 128; return CALL_F; } \
      }                                                                 \
    } else {                                                            \
      switch (N) {                                                      \
        case 8: { using T = double; constexpr int NN = 8; return CALL_D; }    \
        case 16: { using T = double; constexpr int NN = 16; return CALL_D; }  \
        case 32: { using T = double; constexpr int NN = 32; return CALL_D; }  \
        case 64: { using T = double; constexpr int NN = 64; return CALL_D; }  \
        case 128: { using T = double; constexpr int NN = 128; return CALL_D; } \
      }                                                                 \
    }                                                                   \
    return cudaErrorInvalidValue;                                       \
  } while (0)

#define HM_DISPATCH_PENCIL(PREC, N, CALL)                                       \
  do {                                                                          \
    if ((PREC) == 0 && (N) == 256) { using T = float; constexpr int NN = 256; return CALL; } \
    HM_DISPATCH_N(PREC, N, CALL, CALL);                                         \
  } while (0)

template <typename T, int N>
static cudaError_t prepare_pencil_t() {
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  constexpr int s1 = (int)(sizeof(cplx<T>) * N * kTC), s3 = (int)(sizeof(cplx<T>) * N * 3 * kTC);
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_FWD>, A, s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_INV>, A, s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_SCALE>, A, s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_VEL>, A, s3)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pencil<T, N, PM_ADJ>, A, s3);
}

template <typename T, int N>
static cudaError_t prepare_t() {
  cudaError_t e;
  constexpr int sp = (int)plane_smem_bytes<T, N>();
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_plane_r2c<T, N, false>, A, sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_r2c<T, N, true>, A, sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_c2r<T, N, C2R_STORE>, A, sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_c2r<T, N, C2R_EPI>, A, sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_c2r<T, N, C2R_GATHER>, A, sp)) != cudaSuccess) return e;
  constexpr int s1 = (int)(sizeof(cplx<T>) * N * kTC), s3 = (int)(sizeof(cplx<T>) * N * 3 * kTC);
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_FWD>, A, s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_INV>, A, s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_SCALE>, A, s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_VEL>, A, s3)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pencil<T, N, PM_ADJ>, A, s3);
}

cudaError_t fft_prepare(int prec, int N) {
  if (N == 256) {
    if (prec != 0) return cudaErrorInvalidValue;
    cudaError_t e = prepare_pencil_t<float, 256>();
    if (e == cudaSuccess) e = prepare_pencil_tma<256>();
    return e != cudaSuccess ? e : plane256_prepare();
  }
  HM_DISPATCH_N(prec, N, (prepare_t<T, NN>()), (prepare_t<T, NN>()));
}

cudaError_t launch_plane_r2c(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, cudaStream_t st) {
  if (N == 256) return prec == 0 ? launch_plane_r2c_256(in, in_stride, out, out_stride, count, tw, nullptr, st)
                                 : cudaErrorInvalidValue;
  PlanePoints none{};
  HM_DISPATCH_N(prec, N, (plane_r2c_t<T, NN, false>(in, in_stride, out, out_stride, count, tw, none, st)),
                (plane_r2c_t<T, NN, false>(in, in_stride, out, out_stride, count, tw, none, st)));
}

cudaError_t launch_plane_r2c_scatter(int prec, int N, const PlanePoints& pts, void* out, long long out_stride,
                                     int count, const void* tw, cudaStream_t st) {
  if (N == 256) return prec == 0 ? launch_plane_r2c_256(nullptr, 0, out, out_stride, count, tw, &pts, st)
                                 : cudaErrorInvalidValue;
  HM_DISPATCH_N(prec, N, (plane_r2c_t<T, NN, true>(nullptr, 0, out, out_stride, count, tw, pts, st)),
                (plane_r2c_t<T, NN, true>(nullptr, 0, out, out_stride, count, tw, pts, st)));
}

cudaError_t launch_plane_c2r(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, const FieldEpi* epi,
                             cudaStream_t st, void* next_spec) {
  if (N == 256)
    return prec == 0 ? launch_plane_c2r_256(epi ? C2R_EPI : C2R_STORE, in, in_stride, out, out_stride, count, tw, epi,
                                           nullptr, next_spec, st)
                     : cudaErrorInvalidValue;
  PlanePoints none{};
  if (epi) {
    HM_DISPATCH_N(prec, N, (plane_c2r_t<T, NN, C2R_EPI>(in, in_stride, out, out_stride, count, tw, epi, none, st, next_spec)),
                  (plane_c2r_t<T, NN, C2R_EPI>(in, in_stride, out, out_stride, count, tw, epi, none, st, next_spec)));
  }
  HM_DISPATCH_N(prec, N, (plane_c2r_t<T, NN, C2R_STORE>(in, in_stride, out, out_stride, count, tw, nullptr, none, st)),
                (plane_c2r_t<T, NN, C2R_STORE>(in, in_stride, out, out_stride, count, tw, nullptr, none, st)));
}

cudaError_t launch_plane_c2r_gather(int prec, int N, const void* in, long long in_stride,
                                    const PlanePoints& pts, int count, const void* tw, cudaStream_t st) {
  if (N == 256)
    return prec == 0 ? launch_plane_c2r_256(C2R_GATHER, in, in_stride, nullptr, 0, count, tw, nullptr, &pts, nullptr, st)
                     : cudaErrorInvalidValue;
  HM_DISPATCH_N(prec, N, (plane_c2r_t<T, NN, C2R_GATHER>(in, in_stride, nullptr, 0, count, tw, nullptr, pts, st)),
                (plane_c2r_t<T, NN, C2R_GATHER>(in, in_stride, nullptr, 0, count, tw, nullptr, pts, st)));
}

template <typename T, int N>
static cudaError_t pencil_mode(int mode, const void* in, long long in_stride, void* out,
                               long long out_stride, int count, const void* tw, const void* amp,
                               cudaStream_t st, const int* plane_off) {
  switch (mode) {
    case PM_FWD: return pencil_t<T, N, PM_FWD>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_INV: return pencil_t<T, N, PM_INV>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_VEL: return pencil_t<T, N, PM_VEL>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_ADJ:
      return pencil_t<T, N, PM_ADJ>(in, in_stride, out, out_stride, count, tw, amp, st, plane_off, plane_split(N));
    case PM_SCALE: return pencil_t<T, N, PM_SCALE>(in, in_stride, out, out_stride, count, tw, amp, st);
  }
  return cudaErrorInvalidValue;
}

template <int N>
static cudaError_t pencil_tma_mode(int mode, const void* in, long long in_stride, void* out, long long out_stride,
                                  int count, const void* tw, const void* amp, cudaStream_t st) {
  switch (mode) {
    case PM_FWD: return pencil_tma_t<N, PM_FWD>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_INV: return pencil_tma_t<N, PM_INV>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_VEL: return pencil_tma_t<N, PM_VEL>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_SCALE: return pencil_tma_t<N, PM_SCALE>(in, in_stride, out, out_stride, count, tw, amp, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_pencil(int prec, int N, int mode, const void* in, long long in_stride, void* out,
                          long long out_stride, int count, const void* tw, const void* amp,
                          cudaStream_t st, const int* plane_off) {
  // FP32 N = 256, single-input modes: the TMA-staged persistent form (a
  // caller's buffer that is not 16-byte aligned takes the plain form below).
  // Measured on GB300: the velocity pass at 256^3 111.7 -> 103.7 us; at
  // 128^3 the plain form, four 128-thread CTAs per SM, is faster (16.2 vs
  // 18.2 us for one chain, 150 vs 156 us for 16), so it stays there.
  const bool aligned = (reinterpret_cast<uintptr_t>(in) & 15u) == 0 && ((in_stride * 8) & 15) == 0;
  if (prec == 0 && N == 256 && mode != PM_ADJ && count > 0 && aligned)
    return pencil_tma_mode<256>(mode, in, in_stride, out, out_stride, count, tw, amp, st);
  HM_DISPATCH_PENCIL(prec, N, (pencil_mode<T, NN>(mode, in, in_stride, out, out_stride, count, tw, amp, st,
                                                  plane_off)));
}

}  // namespace hm
