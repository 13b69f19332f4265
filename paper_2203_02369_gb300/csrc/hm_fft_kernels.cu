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
  static constexpr int ZP = N + 1;                 // pitch of packed z rows
  static constexpr int NT = N >= 128 ? 512 : (N >= 64 ? 256 : 128);
  static constexpr int ZSIZE = (N / 2) * ZP;       // complex elements
  static constexpr int HSIZE = N * NH;
};

template <typename T, int N> constexpr size_t plane_smem_bytes() {
  return sizeof(cplx<T>) * (PlaneCfg<N>::ZSIZE + PlaneCfg<N>::HSIZE);
}

// ---------------------------------------------------------------------------
// Plane pass, forward: real plane x -> (z r2c, y c2c) -> spectrum plane.
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(PlaneCfg<N>::NT)
k_plane_r2c(const T* __restrict__ in, long long in_stride, cplx<T>* __restrict__ out,
            long long out_stride, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int NT = P::NT, NH = P::NH, ZP = P::ZP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Z = reinterpret_cast<C*>(smem_raw);
  C* H = Z + P::ZSIZE;
  const int ix = blockIdx.x;
  const int s = blockIdx.y;
  const T* src = in + (long long)s * in_stride + (long long)ix * N * N;
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::W;
  const V* srcv = reinterpret_cast<const V*>(src);
  for (int e = threadIdx.x; e < N * N / VW; e += NT) {
    V v = __ldg(&srcv[e]);
    const int y = (e * VW) / N, z0 = (e * VW) % N;
    T* zr = reinterpret_cast<T*>(&Z[(y >> 1) * ZP + z0]) + (y & 1);
#pragma unroll
    for (int q = 0; q < VW; ++q) zr[2 * q] = vget<T>(v, q);
  }
  __syncthreads();
  fft_smem<T, N, false, N / 2, NT, false>(Z, ZP, 1, tw);
  // unpack two real rows from each packed row
  for (int e = threadIdx.x; e < (N / 2) * NH; e += NT) {
    const int r = e / NH, k = e % NH;
    const C zk = Z[r * ZP + k];
    const C zm = cconj(Z[r * ZP + ((N - k) & (N - 1))]);
    const C sp = cadd(zk, zm), df = csub(zk, zm);
    H[(2 * r) * NH + k] = C{(T)0.5 * sp.x, (T)0.5 * sp.y};
    H[(2 * r + 1) * NH + k] = C{(T)0.5 * df.y, (T)-0.5 * df.x};
  }
  __syncthreads();
  fft_smem<T, N, false, NH, NT, true>(H, 1, NH, tw);
  C* dst = out + (long long)s * out_stride + (long long)ix * N * NH;
  // the plane is contiguous in both smem and global memory
  for (int e = threadIdx.x; e < N * NH; e += NT) dst[e] = H[e];
}

// ---------------------------------------------------------------------------
// Plane pass, inverse: spectrum plane -> (y c2c, z c2r) -> real plane, with
// either a plain store or the fused gradient / leapfrog epilogue.
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(PlaneCfg<N>::NT)
k_plane_c2r(const cplx<T>* __restrict__ in, long long in_stride, T* __restrict__ out,
            long long out_stride, const cplx<T>* __restrict__ tw, FieldEpi epi, int use_epi) {
  using C = cplx<T>;
  using P = PlaneCfg<N>;
  constexpr int NT = P::NT, NH = P::NH, ZP = P::ZP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Z = reinterpret_cast<C*>(smem_raw);
  C* H = Z + P::ZSIZE;
  __shared__ double red[2][NT / 32];
  const int ix = blockIdx.x;
  const int s = blockIdx.y;
  const C* src = in + (long long)s * in_stride + (long long)ix * N * NH;
  for (int e = threadIdx.x; e < N * NH; e += NT) H[e] = src[e];
  __syncthreads();
  fft_smem<T, N, true, NH, NT, true>(H, 1, NH, tw);
  // pack rows 2r (real part) and 2r+1 (imaginary part) into one complex row
  for (int e = threadIdx.x; e < (N / 2) * N; e += NT) {
    const int r = e / N, k = e % N;
    C a, b;
    if (k <= N / 2) {
      a = H[(2 * r) * NH + k];
      b = H[(2 * r + 1) * NH + k];
      if (k == 0 || k == N / 2) {
        a.y = 0;
        b.y = 0;
      }
    } else {
      a = cconj(H[(2 * r) * NH + (N - k)]);
      b = cconj(H[(2 * r + 1) * NH + (N - k)]);
    }
    Z[r * ZP + k] = C{a.x - b.y, a.y + b.x};
  }
  __syncthreads();
  fft_smem<T, N, true, N / 2, NT, false>(Z, ZP, 1, tw);
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::W;
  if (!use_epi) {
    T* dst = out + (long long)s * out_stride + (long long)ix * N * N;
    V* dstv = reinterpret_cast<V*>(dst);
    for (int e = threadIdx.x; e < N * N / VW; e += NT) {
      const int y = (e * VW) / N, z0 = (e * VW) % N;
      const T* zr = reinterpret_cast<const T*>(&Z[(y >> 1) * ZP + z0]) + (y & 1);
      T t[VW];
#pragma unroll
      for (int q = 0; q < VW; ++q) t[q] = zr[2 * q];
      V v;
      if constexpr (VW == 4) v = V{t[0], t[1], t[2], t[3]};
      else v = V{t[0], t[1]};
      dstv[e] = v;
    }
    return;
  }
  // ---- gradient / leapfrog epilogue (one chain per blockIdx.y) ----
  const long long base = (long long)s * epi.grid_stride + (long long)ix * N * N;
  T* w = reinterpret_cast<T*>(epi.w) + base;
  T* pw = reinterpret_cast<T*>(epi.pw) + base;
  T* gw = reinterpret_cast<T*>(epi.gw) + base;
  const int mode = epi.mode;
  const T eps = (T)epi.cs[s].eps;
  const T ck = (mode == GM_KICK_DRIFT) ? eps : (T)0.5 * eps;
  double acc_w = 0.0, acc_p = 0.0;
  V* wv = reinterpret_cast<V*>(w);
  V* pv = reinterpret_cast<V*>(pw);
  V* gv = reinterpret_cast<V*>(gw);
  for (int e = threadIdx.x; e < N * N / VW; e += NT) {
    const int y = (e * VW) / N, z0 = (e * VW) % N;
    const T* zr = reinterpret_cast<const T*>(&Z[(y >> 1) * ZP + z0]) + (y & 1);
    V wq = wv[e];
    T wt[VW], pt[VW], gt[VW];
    V pq;
    if (mode != GM_GRAD) pq = pv[e];
#pragma unroll
    for (int q = 0; q < VW; ++q) {
      const T wi = vget<T>(wq, q);
      const T g = wi + zr[2 * q];
      acc_w += 0.5 * (double)wi * (double)wi;
      gt[q] = g;
      if (mode != GM_GRAD) {
        T p = vget<T>(pq, q) - ck * g;
        pt[q] = p;
        wt[q] = (mode == GM_KICK_LAST) ? wi : wi + eps * p;
        acc_p += 0.5 * (double)p * (double)p;
      }
    }
    if (mode == GM_GRAD || mode == GM_KICK_LAST) {
      V g;
      if constexpr (VW == 4) g = V{gt[0], gt[1], gt[2], gt[3]};
      else g = V{gt[0], gt[1]};
      gv[e] = g;
    }
    if (mode != GM_GRAD) {
      V p, ww;
      if constexpr (VW == 4) {
        p = V{pt[0], pt[1], pt[2], pt[3]};
        ww = V{wt[0], wt[1], wt[2], wt[3]};
      } else {
        p = V{pt[0], pt[1]};
        ww = V{wt[0], wt[1]};
      }
      pv[e] = p;
      if (mode != GM_KICK_LAST) wv[e] = ww;
    }
  }
  // deterministic block reduction: warp shuffles, then warp 0
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
template <typename T, int N>
static cudaError_t plane_r2c_t(const void* in, long long in_stride, void* out, long long out_stride,
                               int count, const void* tw, cudaStream_t st) {
  constexpr size_t sm = plane_smem_bytes<T, N>();
  dim3 grid(N, count);
  k_plane_r2c<T, N><<<grid, PlaneCfg<N>::NT, sm, st>>>(
      static_cast<const T*>(in), in_stride, static_cast<cplx<T>*>(out), out_stride,
      static_cast<const cplx<T>*>(tw));
  return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t plane_c2r_t(const void* in, long long in_stride, void* out, long long out_stride,
                               int count, const void* tw, const FieldEpi* epi, cudaStream_t st) {
  constexpr size_t sm = plane_smem_bytes<T, N>();
  dim3 grid(N, count);
  FieldEpi e{};
  if (epi) e = *epi;
  k_plane_c2r<T, N><<<grid, PlaneCfg<N>::NT, sm, st>>>(
      static_cast<const cplx<T>*>(in), in_stride, static_cast<T*>(out), out_stride,
      static_cast<const cplx<T>*>(tw), e, epi ? 1 : 0);
  return cudaGetLastError();
}

template <typename T, int N, int MODE>
static cudaError_t pencil_t(const void* in, long long in_stride, void* out, long long out_stride,
                            int count, const void* tw, const void* amp, cudaStream_t st) {
  constexpr int NH = N / 2 + 1;
  constexpr int NCOMP = (MODE == PM_VEL || MODE == PM_ADJ) ? 3 : 1;
  constexpr size_t sm = sizeof(cplx<T>) * N * NCOMP * kTC;
  dim3 grid((N * NH + kTC - 1) / kTC, count);
  k_pencil<T, N, MODE><<<grid, kPencilNT, sm, st>>>(
      static_cast<const cplx<T>*>(in), in_stride, static_cast<cplx<T>*>(out), out_stride,
      static_cast<const cplx<T>*>(tw), static_cast<const T*>(amp));
  return cudaGetLastError();
}

// Supported grids: FP32 N in {8..128}; FP64 N in {8..64} (shared memory).
bool fft_supported(int prec, int N) {
  if (prec == 0) return N == 8 || N == 16 || N == 32 || N == 64 || N == 128;
  return N == 8 || N == 16 || N == 32 || N == 64;
}

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
      }                                                                 \
    }                                                                   \
    return cudaErrorInvalidValue;                                       \
  } while (0)

template <typename T, int N>
static cudaError_t prepare_t() {
  cudaError_t e;
  constexpr size_t sp = plane_smem_bytes<T, N>();
  if ((e = cudaFuncSetAttribute(k_plane_r2c<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_c2r<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp)) != cudaSuccess) return e;
  constexpr size_t s1 = sizeof(cplx<T>) * N * kTC, s3 = sizeof(cplx<T>) * N * 3 * kTC;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_pencil<T, N, PM_VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_pencil<T, N, PM_ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3);
}

cudaError_t fft_prepare(int prec, int N) {
  HM_DISPATCH_N(prec, N, (prepare_t<T, NN>()), (prepare_t<T, NN>()));
}

cudaError_t launch_plane_r2c(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, cudaStream_t st) {
  HM_DISPATCH_N(prec, N, (plane_r2c_t<T, NN>(in, in_stride, out, out_stride, count, tw, st)),
                (plane_r2c_t<T, NN>(in, in_stride, out, out_stride, count, tw, st)));
}

cudaError_t launch_plane_c2r(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, const FieldEpi* epi,
                             cudaStream_t st) {
  HM_DISPATCH_N(prec, N, (plane_c2r_t<T, NN>(in, in_stride, out, out_stride, count, tw, epi, st)),
                (plane_c2r_t<T, NN>(in, in_stride, out, out_stride, count, tw, epi, st)));
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
  HM_DISPATCH_N(prec, N, (pencil_mode<T, NN>(mode, in, in_stride, out, out_stride, count, tw, amp, st)),
                (pencil_mode<T, NN>(mode, in, in_stride, out, out_stride, count, tw, amp, st)));
}

}  // namespace hm
