// Shared-memory batched complex FFT building blocks for the 3D r2c/c2r
// passes of the HAMLET field operator (linear velocity, eq. vel-field, and
// its adjoint).  Data stay in shared memory; every length N <= 256 is done in
// at most two register-resident radix stages (N = R1 * M, R1, M <= 16):
//
//   stage 1: for each m < M, the R1-point DFT over j of x[m + M j], times the
//            twiddle W_N^{m k2}, written back in place at m + M k2;
//   stage 2: for each k2 < R1, the M-point DFT over the contiguous block
//            m + M k2 gives X[R1 k1 + k2], stored at its natural position
//            after a block barrier (all loads done first).
//
// Input and output are both in natural order, forward uses e^{-i}, inverse
// uses e^{+i} and no 1/N (the 1/N^3 of the inverse DFT is folded into the
// k-space weights).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace hm {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return C{a.x, -a.y}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C mul_mi(C a) {
  return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}

// Programmatic dependent launch: a kernel lets the next kernel in its
// stream start launching (pdl_trigger) and waits for the previous kernel's
// writes to be complete and visible (pdl_wait) before reading them.  Both
// are no-ops for a launch without the programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Small DFTs in registers, natural order in and out.
template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C* a) {
  C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  C t2 = cadd(a[1], a[3]), t3 = mul_mi<INV>(csub(a[1], a[3]));
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* a) {
  using R = decltype(a[0].x);
  const R s = (R)0.70710678118654752440;  // sqrt(1/2)
  C e[4] = {a[0], a[2], a[4], a[6]};
  C o[4] = {a[1], a[3], a[5], a[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  // W8^k = e^{-+ i pi k/4}
  C o1 = INV ? C{s * (o[1].x - o[1].y), s * (o[1].x + o[1].y)}
             : C{s * (o[1].x + o[1].y), s * (o[1].y - o[1].x)};
  C o2 = mul_mi<INV>(o[2]);
  C o3 = INV ? C{-s * (o[3].x + o[3].y), s * (o[3].x - o[3].y)}
             : C{s * (o[3].y - o[3].x), -s * (o[3].x + o[3].y)};
  a[0] = cadd(e[0], o[0]);
  a[4] = csub(e[0], o[0]);
  a[1] = cadd(e[1], o1);
  a[5] = csub(e[1], o1);
  a[2] = cadd(e[2], o2);
  a[6] = csub(e[2], o2);
  a[3] = cadd(e[3], o3);
  a[7] = csub(e[3], o3);
}

template <bool INV, typename C> __device__ __forceinline__ void dft16(C* a) {
  using R = decltype(a[0].x);
  // cos and sin of pi k / 8, k = 0..7
  const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173;
  const R c2 = (R)0.70710678118654752440;
  C e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = a[2 * i];
    o[i] = a[2 * i + 1];
  }
  dft8<INV>(e);
  dft8<INV>(o);
  const R cs[8] = {(R)1, c1, c2, s1, (R)0, -s1, -c2, -c1};
  const R sn[8] = {(R)0, s1, c2, c1, (R)1, c1, c2, s1};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    // W16^k = cos - (+) i sin for forward (inverse)
    const R wr = cs[k], wi = INV ? sn[k] : -sn[k];
    C t = C{o[k].x * wr - o[k].y * wi, o[k].x * wi + o[k].y * wr};
    a[k] = cadd(e[k], t);
    a[k + 8] = csub(e[k], t);
  }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft_reg(C* a) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<INV>(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4<INV>(a);
  } else if constexpr (R == 8) {
    dft8<INV>(a);
  } else {
    static_assert(R == 16, "radix must be 1, 2, 4, 8 or 16");
    dft16<INV>(a);
  }
}

template <int N> struct Radix {
  static_assert(N >= 2 && N <= 256 && (N & (N - 1)) == 0, "N must be a power of two in [2, 256]");
  static constexpr int R1 = N <= 16 ? N : (N == 32 ? 8 : (N == 64 ? 8 : 16));
  static constexpr int M = N / R1;
};

// Stage 2 of fft_smem on its own (after a stage 1 done elsewhere): for each
// k2 < R1 the M-point DFT of the contiguous block m + M k2, stored at its
// natural position after a block barrier.  Ends with a barrier.
template <typename T, int N, bool INV, int ROWS, int NT>
__device__ __forceinline__ void fft_smem_stage2(cplx<T>* buf, int rs, int es) {
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1;
  constexpr int M = Radix<N>::M;
  const int tid = threadIdx.x;
  if constexpr (M > 1) {
    constexpr int G2 = ROWS * R1;
    constexpr int PER = (G2 + NT - 1) / NT;
    C a[PER][M];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      int g = tid + i * NT;
      if (G2 % NT == 0 || g < G2) {
        int r = g % ROWS, k2 = g / ROWS;
        C* base = buf + r * rs + (M * k2) * es;
#pragma unroll
        for (int m = 0; m < M; ++m) a[i][m] = base[m * es];
        dft_reg<M, INV>(a[i]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      int g = tid + i * NT;
      if (G2 % NT == 0 || g < G2) {
        int r = g % ROWS, k2 = g / ROWS;
        C* base = buf + r * rs + k2 * es;
#pragma unroll
        for (int k1 = 0; k1 < M; ++k1) base[(R1 * k1) * es] = a[i][k1];
      }
    }
    __syncthreads();
  }
}

// Batched in-place FFT of ROWS rows of length N held in shared memory.
// Element k of row r lives at buf[r*rs + k*es].  NT threads take part; all of
// them must call this function (it contains block barriers).  tw[e] holds
// e^{-2 pi i e / N} for e < N (conjugated here for the inverse).
// S1_ROW_FAST selects which index varies fastest across threads in stage 1
// (row-fast suits column layouts, es > 1; m-fast suits row layouts, es = 1).
template <typename T, int N, bool INV, int ROWS, int NT, bool S1_ROW_FAST>
__device__ __forceinline__ void fft_smem(cplx<T>* buf, int rs, int es, const cplx<T>* __restrict__ tw) {
  using C = cplx<T>;
  constexpr int R1 = Radix<N>::R1;
  constexpr int M = Radix<N>::M;
  const int tid = threadIdx.x;
  // ---- stage 1 (in place per group) ----
  constexpr int G1 = ROWS * M;
#pragma unroll 1
  for (int g = tid; g < G1; g += NT) {
    int r, m;
    if (S1_ROW_FAST) {
      r = g % ROWS;
      m = g / ROWS;
    } else {
      m = g % M;
      r = g / M;
    }
    C a[R1];
    C* base = buf + r * rs + m * es;
#pragma unroll
    for (int j = 0; j < R1; ++j) a[j] = base[(M * j) * es];
    dft_reg<R1, INV>(a);
    if constexpr (M > 1) {
#pragma unroll
      for (int k2 = 1; k2 < R1; ++k2) {
        C wv = __ldg(&tw[m * k2]);
        if (INV) wv.y = -wv.y;
        a[k2] = cmul(a[k2], wv);
      }
    }
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) base[(M * k2) * es] = a[k2];
  }
  __syncthreads();
  fft_smem_stage2<T, N, INV, ROWS, NT>(buf, rs, es);
}

// Accumulator of 0.5 * sum x^2 for energy reductions.  For FP32 data it
// keeps an unevaluated pair (hi, lo) of floats: x*x is split exactly into
// p + e with an FMA, p/2 is added with Knuth's TwoSum and every rounding
// error goes to lo, so the sum carries about 48 significant bits without
// using the (slow on this part) FP64 pipe.  Partial sums of a warp are merged
// the same way (warp_reduce, a fixed shuffle tree), and the pair is converted
// to double once per warp for the FP64 block and grid reductions.  For FP64
// data it is a plain double sum.
template <typename T> struct HalfSqAcc;
template <> struct HalfSqAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_half_sq(double x) { s += 0.5 * x * x; }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct HalfSqAcc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fadd_rn(s, -hi);
    const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bp)), __fadd_rn(x, -bp));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ void add_half_sq(float x) {
    const float p = __fmul_rn(x, x);
    const float e = __fmaf_rn(x, x, -p);
    add(__fmul_rn(0.5f, p));
    lo = __fmaf_rn(0.5f, e, lo);
  }
  __device__ __forceinline__ void warp_reduce() {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h = __shfl_down_sync(0xffffffffu, hi, o);
      const float l = __shfl_down_sync(0xffffffffu, lo, o);
      add(h);
      lo = __fadd_rn(lo, l);
    }
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

}  // namespace hm
