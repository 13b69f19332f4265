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
#include "hm_fft.cuh"
#include "hm_internal.h"

namespace hm {

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

template <typename T> __device__ __forceinline__ T vget(const typename Vec16<T>::type& v, int q);
template <> __device__ __forceinline__ float vget<float>(const float4& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}
template <> __device__ __forceinline__ double vget<double>(const double2& v, int q) {
  return q == 0 ? v.x : v.y;
}

template <int N> struct PlaneCfg {
  static constexpr int NH = N / 2 + 1;
  static constexpr int ZP = 2 * NH;                // pitch of packed z rows (= 2 spectrum rows)
  static constexpr int NT = N >= 128 ? 512 : (N >= 64 ? 256 : 128);
  static constexpr int SIZE = N * NH;              // complex elements of the plane buffer
  static constexpr int MINB = N >= 128 ? 2 : 1;    // CTAs per SM the register budget aims at
};

template <typename T, int N> constexpr size_t plane_smem_bytes() {
  return sizeof(cplx<T>) * PlaneCfg<N>::SIZE;
}

// The plane buffer B holds N*(N/2+1) complex values and is read through two
// views that share memory:
//   spectrum view  H[y][k] = B[y*NH + k]            (y < N, k <= N/2)
//   packed view    Z[r][z] = B[r*ZP + z], ZP = 2 NH (r < N/2, z < N), whose
//                  real/imaginary parts are the real rows y = 2r and 2r+1.
// Z row r and H rows 2r, 2r+1 occupy the same addresses, so the real <->
// half-spectrum (un)packing runs in place, row pair by row pair.
template <typename T, int N>
__device__ __forceinline__ T* zreal(cplx<T>* B, int y, int z) {
  return reinterpret_cast<T*>(&B[(y >> 1) * PlaneCfg<N>::ZP + z]) + (y & 1);
}

// Z rows (after the forward z FFT) -> H rows (half spectra of the real rows).
template <typename T, int N>
__device__ __forceinline__ void unpack_rows(cplx<T>* B) {
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int NH = P::NH, ZP = P::ZP, NT = P::NT;
  constexpr int TOT = (N / 2) * NH;
  constexpr int PER = (TOT + NT - 1) / NT;
  C a[PER], b[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    if (e < TOT) {
      const int r = e / NH, k = e % NH;
      const C zk = B[r * ZP + k];
      const C zm = cconj(B[r * ZP + ((N - k) & (N - 1))]);
      const C sp = cadd(zk, zm), df = csub(zk, zm);
      a[i] = C{(T)0.5 * sp.x, (T)0.5 * sp.y};
      b[i] = C{(T)0.5 * df.y, (T)-0.5 * df.x};
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    if (e < TOT) {
      const int r = e / NH, k = e % NH;
      B[r * ZP + k] = a[i];
      B[r * ZP + NH + k] = b[i];
    }
  }
  __syncthreads();
}

// H rows (inverse-transformed along y) -> Z rows ready for the inverse z FFT.
// The imaginary parts at kz = 0 and N/2 are dropped (c2r semantics).
template <typename T, int N>
__device__ __forceinline__ void pack_rows(cplx<T>* B) {
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int NH = P::NH, ZP = P::ZP, NT = P::NT;
  constexpr int TOT = (N / 2) * N;
  constexpr int PER = (TOT + NT - 1) / NT;
  C o[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    if (e < TOT) {
      const int r = e / N, k = e % N;
      C a, b;
      if (k <= N / 2) {
        a = B[r * ZP + k];
        b = B[r * ZP + NH + k];
        if (k == 0 || k == N / 2) {
          a.y = 0;
          b.y = 0;
        }
      } else {
        a = cconj(B[r * ZP + (N - k)]);
        b = cconj(B[r * ZP + NH + (N - k)]);
      }
      o[i] = C{a.x - b.y, a.y + b.x};
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    if (e < TOT) B[(e / N) * ZP + (e % N)] = o[i];
  }
  __syncthreads();
}

// Real plane (rows y, contiguous z) <-> packed view.  Item (r, zp) covers
// rows 2r, 2r+1 and columns z = 2zp, 2zp+1: two 2-wide global accesses per
// row and one 16-byte (FP32) shared access, so consecutive threads touch
// consecutive shared words (no bank conflicts).
template <typename T, int N>
__device__ __forceinline__ void load_plane_packed(cplx<T>* B, const T* __restrict__ src) {
  using P = PlaneCfg<N>;
  constexpr int ITEMS = (N / 2) * (N / 2);
  for (int e = threadIdx.x; e < ITEMS; e += P::NT) {
    const int r = e / (N / 2), z = 2 * (e % (N / 2));
    if constexpr (sizeof(T) == 4) {
      const float2 a = __ldg(reinterpret_cast<const float2*>(src + (2 * r) * N + z));
      const float2 b = __ldg(reinterpret_cast<const float2*>(src + (2 * r + 1) * N + z));
      *reinterpret_cast<float4*>(&B[r * P::ZP + z]) = make_float4(a.x, b.x, a.y, b.y);
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(src + (2 * r) * N + z));
      const double2 b = __ldg(reinterpret_cast<const double2*>(src + (2 * r + 1) * N + z));
      B[r * P::ZP + z] = cplx<T>{a.x, b.x};
      B[r * P::ZP + z + 1] = cplx<T>{a.y, b.y};
    }
  }
}

// values of item (r, zp): v[0] = (2r, z), v[1] = (2r+1, z), v[2] = (2r, z+1), v[3] = (2r+1, z+1)
template <typename T, int N>
__device__ __forceinline__ void read_item(const cplx<T>* B, int r, int z, T* v) {
  using P = PlaneCfg<N>;
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(&B[r * P::ZP + z]);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    const cplx<T> a = B[r * P::ZP + z], b = B[r * P::ZP + z + 1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
}

template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

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
    load_plane_packed<T, N>(B, in + (long long)s * in_stride + (long long)ix * N * N);
  } else {
    for (int e = threadIdx.x; e < P::SIZE; e += NT) B[e] = C{(T)0, (T)0};
    __syncthreads();
    const int c = s / 3, j = s % 3;
    const PlaneBuckets pb = plane_buckets<N>(pts.off, c, ix);
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
  fft_smem<T, N, false, N / 2, NT, false>(B, ZP, 1, tw);
  unpack_rows<T, N>(B);
  fft_smem<T, N, false, P::NH, NT, true>(B, 1, P::NH, tw);
  C* dst = out + (long long)s * out_stride + (long long)ix * P::SIZE;
  if constexpr (sizeof(T) == 4) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4* s4 = reinterpret_cast<const float4*>(B);
    for (int e = threadIdx.x; e < P::SIZE / 2; e += NT) d4[e] = s4[e];
  } else {
    for (int e = threadIdx.x; e < P::SIZE; e += NT) dst[e] = B[e];
  }
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
  const C* src = in + (long long)s * in_stride + (long long)ix * P::SIZE;
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* b4 = reinterpret_cast<float4*>(B);
    for (int e = threadIdx.x; e < P::SIZE / 2; e += NT) b4[e] = __ldg(&s4[e]);
  } else {
    for (int e = threadIdx.x; e < P::SIZE; e += NT) B[e] = src[e];
  }
  __syncthreads();
  fft_smem<T, N, true, P::NH, NT, true>(B, 1, P::NH, tw);
  pack_rows<T, N>(B);
  fft_smem<T, N, true, N / 2, NT, false>(B, ZP, 1, tw);
  using V2 = typename Pair2<T>::type;
  constexpr int ITEMS = (N / 2) * (N / 2);
  if constexpr (MODE == C2R_STORE) {
    T* dst = out + (long long)s * out_stride + (long long)ix * N * N;
    for (int e = threadIdx.x; e < ITEMS; e += NT) {
      const int r = e / (N / 2), z = 2 * (e % (N / 2));
      T v[4];
      read_item<T, N>(B, r, z, v);
      *reinterpret_cast<V2*>(dst + (2 * r) * N + z) = V2{v[0], v[2]};
      *reinterpret_cast<V2*>(dst + (2 * r + 1) * N + z) = V2{v[1], v[3]};
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
    T* w = reinterpret_cast<T*>(epi.w) + base;
    T* pw = reinterpret_cast<T*>(epi.pw) + base;
    T* gw = reinterpret_cast<T*>(epi.gw) + base;
    const int mode = epi.mode;
    const T eps = (T)epi.cs[s].eps;
    const T ck = (mode == GM_KICK_DRIFT) ? eps : (T)0.5 * eps;
    HalfSqAcc<T> aw, ap;
    for (int e = threadIdx.x; e < ITEMS; e += NT) {
      const int r = e / (N / 2), z = 2 * (e % (N / 2));
      T g[4];
      read_item<T, N>(B, r, z, g);
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // row 2r + h, columns z, z + 1
        const long long o = (long long)(2 * r + h) * N + z;
        const V2 wq = *reinterpret_cast<const V2*>(w + o);
        const T w0 = wq.x, w1 = wq.y;
        const T g0 = w0 + g[h], g1 = w1 + g[2 + h];
        aw.add_half_sq(w0);
        aw.add_half_sq(w1);
        if (mode == GM_GRAD || mode == GM_KICK_LAST) *reinterpret_cast<V2*>(gw + o) = V2{g0, g1};
        if (mode != GM_GRAD) {
          const V2 pq = *reinterpret_cast<const V2*>(pw + o);
          const T p0 = pq.x - ck * g0, p1 = pq.y - ck * g1;
          *reinterpret_cast<V2*>(pw + o) = V2{p0, p1};
          ap.add_half_sq(p0);
          ap.add_half_sq(p1);
          if (mode == GM_KICK_DRIFT) {
            const T n0 = w0 + eps * p0, n1 = w1 + eps * p1;
            *reinterpret_cast<V2*>(w + o) = V2{n0, n1};
            g[h] = n0;        // the drifted field replaces g in the plane buffer
            g[2 + h] = n1;
          }
        }
      }
      if (next != nullptr && mode == GM_KICK_DRIFT) {
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4*>(&B[r * ZP + z]) = make_float4(g[0], g[1], g[2], g[3]);
        } else {
          B[r * ZP + z] = cplx<T>{g[0], g[1]};
          B[r * ZP + z + 1] = cplx<T>{g[2], g[3]};
        }
      }
    }
    double acc_w = aw.value(), acc_p = ap.value();
    // deterministic block reduction: warp shuffles, then thread 0 in order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc_w += __shfl_down_sync(0xffffffffu, acc_w, o);
      acc_p += __shfl_down_sync(0xffffffffu, acc_p, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][wid] = acc_w;
      red[1][wid] = acc_p;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int i = 0; i < NT / 32; ++i) {
        a += red[0][i];
        b += red[1][i];
      }
      epi.prior_part[(long long)s * N + ix] = a;
      if (mode == GM_KICK_LAST) epi.kin_part[(long long)s * N + ix] = b;
    }
    if (next != nullptr && mode == GM_KICK_DRIFT) {
      // forward plane transform of the drifted field for the next evaluation
      __syncthreads();
      fft_smem<T, N, false, N / 2, NT, false>(B, ZP, 1, tw);
      unpack_rows<T, N>(B);
      fft_smem<T, N, false, P::NH, NT, true>(B, 1, P::NH, tw);
      C* dst = next + (long long)s * next_stride + (long long)ix * P::SIZE;
      if constexpr (sizeof(T) == 4) {
        float4* d4 = reinterpret_cast<float4*>(dst);
        const float4* s4 = reinterpret_cast<const float4*>(B);
        for (int e = threadIdx.x; e < P::SIZE / 2; e += NT) d4[e] = s4[e];
      } else {
        for (int e = threadIdx.x; e < P::SIZE; e += NT) dst[e] = B[e];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Pencil pass along x with the fused k-space operator.
// amp[n2] = (2 pi/L) aHf sqrt(P(k)/Delta^3) / (k^2 N^3), amp[0] = 0, so that
// the velocity spectrum of axis j is i n_j^odd amp[n^2] w_k.
// ---------------------------------------------------------------------------
constexpr int kTC = 16;       // (ky, kz) columns per tile
constexpr int kPencilNT = 256;

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(kPencilNT)
k_pencil(const cplx<T>* __restrict__ in, long long in_stride, cplx<T>* __restrict__ out,
         long long out_stride, const cplx<T>* __restrict__ tw, const T* __restrict__ amp) {
  pdl_wait();
  pdl_trigger();
  using C = cplx<T>;
  constexpr int NH = N / 2 + 1;
  constexpr int NCOL = N * NH;
  constexpr int NCOMP = (MODE == PM_VEL || MODE == PM_ADJ) ? 3 : 1;
  constexpr int W = NCOMP * kTC;   // smem row width: NCOMP tiles side by side
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [N][W]
  const int c0 = blockIdx.x * kTC;
  const int s = blockIdx.y;
  const int tid = threadIdx.x;
  constexpr int NIN = (MODE == PM_ADJ) ? 3 : 1;
  // load input component(s)
  for (int e = tid; e < NIN * N * kTC; e += kPencilNT) {
    const int t = e % kTC;
    const int x = (e / kTC) % N;
    const int j = e / (kTC * N);
    const int col = c0 + t;
    C v = C{(T)0, (T)0};
    if (col < NCOL) v = in[(long long)(s * NIN + j) * in_stride + (long long)x * NCOL + col];
    buf[x * W + j * kTC + t] = v;
  }
  __syncthreads();
  if constexpr (MODE == PM_INV) {
    fft_smem<T, N, true, kTC, kPencilNT, true>(buf, 1, W, tw);
  } else {
    fft_smem<T, N, false, NIN * kTC, kPencilNT, true>(buf, 1, W, tw);
  }
  if constexpr (MODE == PM_VEL || MODE == PM_ADJ) {
    for (int e = tid; e < N * kTC; e += kPencilNT) {
      const int t = e % kTC, kx = e / kTC;
      const int col = c0 + t;
      if (col >= NCOL) continue;   // ragged last tile: nothing stored
      const int ky = col / NH, kz = col % NH;
      const int nx = kx < N / 2 ? kx : kx - N;
      const int ny = ky < N / 2 ? ky : ky - N;
      const int nz = kz;
      const T a = __ldg(&amp[nx * nx + ny * ny + nz * nz]);
      const T ox = (kx == N / 2) ? (T)0 : (T)nx;
      const T oy = (ky == N / 2) ? (T)0 : (T)ny;
      const T oz = (kz == N / 2) ? (T)0 : (T)nz;
      if constexpr (MODE == PM_VEL) {
        const C wk = buf[kx * W + t];
        const C iw = C{-a * wk.y, a * wk.x};   // i amp w_k
        buf[kx * W + t] = C{ox * iw.x, ox * iw.y};
        buf[kx * W + kTC + t] = C{oy * iw.x, oy * iw.y};
        buf[kx * W + 2 * kTC + t] = C{oz * iw.x, oz * iw.y};
      } else {
        const C sx = buf[kx * W + t], sy = buf[kx * W + kTC + t], sz = buf[kx * W + 2 * kTC + t];
        const C sum = C{ox * sx.x + oy * sy.x + oz * sz.x, ox * sx.y + oy * sy.y + oz * sz.y};
        buf[kx * W + t] = C{a * sum.y, -a * sum.x};   // -i amp sum_j n_j s_j
      }
    }
    __syncthreads();
    constexpr int NOUT = (MODE == PM_VEL) ? 3 : 1;
    fft_smem<T, N, true, NOUT * kTC, kPencilNT, true>(buf, 1, W, tw);
  }
  constexpr int NOUT = (MODE == PM_VEL) ? 3 : 1;
  for (int e = tid; e < NOUT * N * kTC; e += kPencilNT) {
    const int t = e % kTC;
    const int x = (e / kTC) % N;
    const int j = e / (kTC * N);
    const int col = c0 + t;
    if (col < NCOL) out[(long long)(s * NOUT + j) * out_stride + (long long)x * NCOL + col] = buf[x * W + j * kTC + t];
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
template <typename T, int N, bool SC>
static cudaError_t plane_r2c_t(const void* in, long long in_stride, void* out, long long out_stride,
                               int count, const void* tw, const PlanePoints& pts, cudaStream_t st) {
  constexpr size_t sm = plane_smem_bytes<T, N>();
  dim3 grid(N, count);
  return launch_k(k_plane_r2c<T, N, SC>, grid, dim3(PlaneCfg<N>::NT), sm, st, static_cast<const T*>(in), in_stride,
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
  return launch_k(k_plane_c2r<T, N, MODE>, grid, dim3(PlaneCfg<N>::NT), sm, st, static_cast<const cplx<T>*>(in),
                  in_stride, static_cast<T*>(out), out_stride, static_cast<const cplx<T>*>(tw), e, pts,
                  static_cast<cplx<T>*>(next), in_stride);
}

template <typename T, int N, int MODE>
static cudaError_t pencil_t(const void* in, long long in_stride, void* out, long long out_stride,
                            int count, const void* tw, const void* amp, cudaStream_t st) {
  constexpr int NH = N / 2 + 1;
  constexpr int NCOMP = (MODE == PM_VEL || MODE == PM_ADJ) ? 3 : 1;
  constexpr size_t sm = sizeof(cplx<T>) * N * NCOMP * kTC;
  dim3 grid((N * NH + kTC - 1) / kTC, count);
  return launch_k(k_pencil<T, N, MODE>, grid, dim3(kPencilNT), sm, st, static_cast<const cplx<T>*>(in), in_stride,
                  static_cast<cplx<T>*>(out), out_stride, static_cast<const cplx<T>*>(tw),
                  static_cast<const T*>(amp));
}

// Supported grids: N in {8, 16, 32, 64, 128} at both precisions (one x-plane
// of the half spectrum fits one CTA's shared memory), and N = 256 at FP32
// (plane passes as 4-CTA clusters, hm_fft_cluster.cu).
bool fft_supported(int prec, int N) {
  return N == 8 || N == 16 || N == 32 || N == 64 || N == 128 || (N == 256 && prec == 0);
}

int plane_split(int N) { return N == 256 ? 4 : 1; }

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
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_VEL>, A, s3)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pencil<T, N, PM_ADJ>, A, s3);
}

cudaError_t fft_prepare(int prec, int N) {
  if (N == 256) {
    if (prec != 0) return cudaErrorInvalidValue;
    cudaError_t e = prepare_pencil_t<float, 256>();
    return e != cudaSuccess ? e : plane_cl_prepare();
  }
  HM_DISPATCH_N(prec, N, (prepare_t<T, NN>()), (prepare_t<T, NN>()));
}

cudaError_t launch_plane_r2c(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, cudaStream_t st) {
  if (N == 256) return prec == 0 ? launch_plane_r2c_cl(in, in_stride, out, out_stride, count, tw, nullptr, st)
                                 : cudaErrorInvalidValue;
  PlanePoints none{};
  HM_DISPATCH_N(prec, N, (plane_r2c_t<T, NN, false>(in, in_stride, out, out_stride, count, tw, none, st)),
                (plane_r2c_t<T, NN, false>(in, in_stride, out, out_stride, count, tw, none, st)));
}

cudaError_t launch_plane_r2c_scatter(int prec, int N, const PlanePoints& pts, void* out, long long out_stride,
                                     int count, const void* tw, cudaStream_t st) {
  if (N == 256) return prec == 0 ? launch_plane_r2c_cl(nullptr, 0, out, out_stride, count, tw, &pts, st)
                                 : cudaErrorInvalidValue;
  HM_DISPATCH_N(prec, N, (plane_r2c_t<T, NN, true>(nullptr, 0, out, out_stride, count, tw, pts, st)),
                (plane_r2c_t<T, NN, true>(nullptr, 0, out, out_stride, count, tw, pts, st)));
}

cudaError_t launch_plane_c2r(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, const FieldEpi* epi,
                             cudaStream_t st, void* next_spec) {
  if (N == 256)
    return prec == 0 ? launch_plane_c2r_cl(epi ? C2R_EPI : C2R_STORE, in, in_stride, out, out_stride, count, tw, epi,
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
    return prec == 0 ? launch_plane_c2r_cl(C2R_GATHER, in, in_stride, nullptr, 0, count, tw, nullptr, &pts, nullptr, st)
                     : cudaErrorInvalidValue;
  HM_DISPATCH_N(prec, N, (plane_c2r_t<T, NN, C2R_GATHER>(in, in_stride, nullptr, 0, count, tw, nullptr, pts, st)),
                (plane_c2r_t<T, NN, C2R_GATHER>(in, in_stride, nullptr, 0, count, tw, nullptr, pts, st)));
}

template <typename T, int N>
static cudaError_t pencil_mode(int mode, const void* in, long long in_stride, void* out,
                               long long out_stride, int count, const void* tw, const void* amp,
                               cudaStream_t st) {
  switch (mode) {
    case PM_FWD: return pencil_t<T, N, PM_FWD>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_INV: return pencil_t<T, N, PM_INV>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_VEL: return pencil_t<T, N, PM_VEL>(in, in_stride, out, out_stride, count, tw, amp, st);
    case PM_ADJ: return pencil_t<T, N, PM_ADJ>(in, in_stride, out, out_stride, count, tw, amp, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_pencil(int prec, int N, int mode, const void* in, long long in_stride, void* out,
                          long long out_stride, int count, const void* tw, const void* amp,
                          cudaStream_t st) {
  HM_DISPATCH_PENCIL(prec, N, (pencil_mode<T, NN>(mode, in, in_stride, out, out_stride, count, tw, amp, st)));
}

}  // namespace hm
