// Plane passes for grids whose x-plane does not fit one CTA's shared memory
// (N = 256): a thread-block cluster of eight CTAs per plane.  CTA q owns N/8
// real rows (two packed per complex row) for the z transform; the CTAs then
// exchange their row slabs for column slabs through distributed shared
// memory and each runs the y transform of about (N/2+1)/8 columns.  At 66 KB
// of shared memory and ~75 registers a thread, three CTAs share an SM (at
// four CTAs a plane one 134 KB CTA filled an SM, which left it short of
// warps).  The point work of a plane (CIC gather after the inverse, CIC
// scatter before the forward) and the field's leapfrog epilogue are the same
// as in the single-CTA plane passes; a point's corner in the next CTA's row
// is read or atomically added through DSMEM.  The loops that read global or
// distributed shared memory are unrolled so that each thread keeps several
// loads in flight (the passes stalled on load latency).
#include <cooperative_groups.h>

#include "hm_fft.cuh"
#include "hm_internal.h"

namespace cg = cooperative_groups;

namespace hm {

template <typename T> struct Pair2Cl;
template <> struct Pair2Cl<float> { using type = float2; };
template <> struct Pair2Cl<double> { using type = double2; };

enum C2RModeCl : int { C2R_STORE = 0, C2R_EPI = 1, C2R_GATHER = 2 };

template <int N> struct ClCfg {
  static constexpr int NH = N / 2 + 1;
  static constexpr int ZP = 2 * NH;           // pitch of a packed row (= two half-spectrum rows)
  static constexpr int K = 8;                 // CTAs per plane (cluster size)
  static constexpr int RQ = N / K;            // real rows per CTA
  static constexpr int PR = RQ / 2;           // packed rows per CTA
  static constexpr int CW = (NH + K - 1) / K; // most half-spectrum columns of one CTA
  static constexpr int CWP = CW | 1;          // odd pitch of the column slab
  static constexpr int ROWSLAB = PR * ZP;     // complex elements
  static constexpr int COLSLAB = N * CWP;
  static constexpr int NT = N >= 128 ? 256 : 128;
};

template <typename T, int N> constexpr size_t plane_smem_bytes() {
  return sizeof(cplx<T>) * (ClCfg<N>::ROWSLAB + ClCfg<N>::COLSLAB);
}

// Row slab R of CTA q holds real rows y in [q*RQ, (q+1)*RQ) through two views
// sharing memory:
//   spectrum view  H[yl][k] = R[yl*NH + k]       (half spectrum of row q*RQ + yl)
//   packed view    Z[r][z]  = R[r*ZP + z]        (real rows 2r, 2r+1 in re, im)
// Z row r and H rows 2r, 2r+1 occupy the same addresses, so the real <->
// half-spectrum (un)packing runs in place.
template <typename T, int N>
__device__ __forceinline__ T* zreal_cl(cplx<T>* R, int yl, int z) {
  return reinterpret_cast<T*>(&R[(yl >> 1) * ClCfg<N>::ZP + z]) + (yl & 1);
}

// Z rows (after the forward z FFT) -> H rows (half spectra of the real rows).
template <typename T, int N>
__device__ __forceinline__ void unpack_rows_cl(cplx<T>* R) {
  using C = cplx<T>;
  using P = ClCfg<N>;
  constexpr int NH = P::NH, ZP = P::ZP, NT = P::NT;
  constexpr int TOT = P::PR * NH;
  constexpr int PER = (TOT + NT - 1) / NT;
  C a[PER], b[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    if (e < TOT) {
      const int r = e / NH, k = e % NH;
      const C zk = R[r * ZP + k];
      const C zm = cconj(R[r * ZP + ((N - k) & (N - 1))]);
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
      R[r * ZP + k] = a[i];
      R[r * ZP + NH + k] = b[i];
    }
  }
  __syncthreads();
}

// H rows (inverse-transformed along y) -> Z rows ready for the inverse z FFT.
// The imaginary parts at kz = 0 and N/2 are dropped (c2r semantics).
template <typename T, int N>
__device__ __forceinline__ void pack_rows_cl(cplx<T>* R) {
  using C = cplx<T>;
  using P = ClCfg<N>;
  constexpr int NH = P::NH, ZP = P::ZP, NT = P::NT;
  constexpr int TOT = P::PR * N;
  constexpr int PER = (TOT + NT - 1) / NT;
  C o[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    if (e < TOT) {
      const int r = e / N, k = e % N;
      C a, b;
      if (k <= N / 2) {
        a = R[r * ZP + k];
        b = R[r * ZP + NH + k];
        if (k == 0 || k == N / 2) {
          a.y = 0;
          b.y = 0;
        }
      } else {
        a = cconj(R[r * ZP + (N - k)]);
        b = cconj(R[r * ZP + NH + (N - k)]);
      }
      o[i] = C{a.x - b.y, a.y + b.x};
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int e = threadIdx.x + i * NT;
    if (e < TOT) R[(e / N) * ZP + (e % N)] = o[i];
  }
  __syncthreads();
}


// Own real rows (contiguous z) <-> packed view.  Item (r, zp) covers local
// rows 2r, 2r+1 and columns z = 2zp, 2zp+1: two 2-wide global accesses and
// one 16-byte (FP32) shared access, consecutive threads on consecutive
// shared words.
template <typename T, int N>
__device__ __forceinline__ void load_rows_packed_cl(cplx<T>* R, const T* __restrict__ src) {
  using P = ClCfg<N>;
  constexpr int ITEMS = P::PR * (N / 2);
  #pragma unroll 8
  for (int e = threadIdx.x; e < ITEMS; e += P::NT) {
    const int r = e / (N / 2), z = 2 * (e % (N / 2));
    if constexpr (sizeof(T) == 4) {
      const float2 a = __ldg(reinterpret_cast<const float2*>(src + (2 * r) * N + z));
      const float2 b = __ldg(reinterpret_cast<const float2*>(src + (2 * r + 1) * N + z));
      *reinterpret_cast<float4*>(&R[r * P::ZP + z]) = make_float4(a.x, b.x, a.y, b.y);
    } else {
      const double2 a = __ldg(reinterpret_cast<const double2*>(src + (2 * r) * N + z));
      const double2 b = __ldg(reinterpret_cast<const double2*>(src + (2 * r + 1) * N + z));
      R[r * P::ZP + z] = cplx<T>{a.x, b.x};
      R[r * P::ZP + z + 1] = cplx<T>{a.y, b.y};
    }
  }
}

// values of item (r, zp): v[0] = (2r, z), v[1] = (2r+1, z), v[2] = (2r, z+1), v[3] = (2r+1, z+1)
template <typename T, int N>
__device__ __forceinline__ void read_item_cl(const cplx<T>* R, int r, int z, T* v) {
  using P = ClCfg<N>;
  if constexpr (sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(&R[r * P::ZP + z]);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else {
    const cplx<T> a = R[r * P::ZP + z], b = R[r * P::ZP + z + 1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
}

// Sub-bucket ranges of this CTA's two point sets on plane ix: side 0 has its
// lower CIC corner on the plane (bucket ix), side 1 its upper corner (bucket
// ix-1); within a plane, points are split by the CTA owning their row cy.
struct PlaneBucketsCl {
  int b0, n0, b1, n1;
};
template <int N>
__device__ __forceinline__ PlaneBucketsCl plane_buckets_cl(const int* __restrict__ off, int c, int ix, int q) {
  constexpr int K = ClCfg<N>::K;
  const int* o = off + (long long)c * (N * K + 1);
  const int ixm = (ix + N - 1) & (N - 1);
  PlaneBucketsCl pb;
  pb.b0 = o[ix * K + q];
  pb.n0 = o[ix * K + q + 1] - pb.b0;
  pb.b1 = o[ixm * K + q];
  pb.n1 = o[ixm * K + q + 1] - pb.b1;
  return pb;
}

// True when no point of chain c has a CIC corner on plane ix (all K
// sub-buckets of buckets ix and ix-1 empty).
template <int N>
__device__ __forceinline__ bool plane_empty_cl(const int* __restrict__ off, int c, int ix) {
  constexpr int K = ClCfg<N>::K;
  const int* o = off + (long long)c * (N * K + 1);
  const int ixm = (ix + N - 1) & (N - 1);
  return o[(ix + 1) * K] == o[ix * K] && o[(ixm + 1) * K] == o[ixm * K];
}

template <typename T> __device__ __forceinline__ T rcomp_cl(const PtRec<T>& p, int j) {
  return j == 0 ? p.rx : (j == 1 ? p.ry : p.rz);
}

// Columns of CTA q: [c0, c1) of the NH half-spectrum columns.
template <int N> __device__ __forceinline__ void own_columns_cl(int q, int& c0, int& c1) {
  constexpr int NH = ClCfg<N>::NH, K = ClCfg<N>::K;
  c0 = (q * NH) / K;
  c1 = ((q + 1) * NH) / K;
}

// ---------------------------------------------------------------------------
// Plane pass, forward: real plane -> (z r2c, y c2c) -> spectrum plane.
// SCATTER builds the plane from the bucketed points instead of loading it:
// s_j(corner) += r rhat_j W(corner), with shared-memory atomics (the adjoint
// of the CIC gather, restricted to this plane); the corner row cy + 1 may
// belong to the next CTA of the cluster and is reached through DSMEM.
// ---------------------------------------------------------------------------
template <typename T, int N, bool SCATTER>
__global__ void __cluster_dims__(ClCfg<N>::K, 1, 1) __launch_bounds__(ClCfg<N>::NT)
k_plane_r2c_cl(const T* __restrict__ in, long long in_stride, cplx<T>* __restrict__ out,
            long long out_stride, const cplx<T>* __restrict__ tw, PlanePoints pts) {
  pdl_wait();
  pdl_trigger();
  using C = cplx<T>;
  using P = ClCfg<N>;
  constexpr int NT = P::NT, K = P::K, RQ = P::RQ, NH = P::NH, CWP = P::CWP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  C* Cs = R + P::ROWSLAB;
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int ix = blockIdx.x / K;
  const int s = blockIdx.y;
  const int row0 = q * RQ;
  auto rem = [&](int k) -> C* { return cl.map_shared_rank(R, k); };   // CTA k's row slab
  if constexpr (!SCATTER) {
    load_rows_packed_cl<T, N>(R, in + (long long)s * in_stride + ((long long)ix * N + row0) * N);
    __syncthreads();
  } else {
    const int c = s / 3, j = s % 3;
    // no point has a CIC corner on this plane (same answer in every CTA of
    // the cluster): its spectrum is zero, which the adjoint pencil pass
    // knows from the same bucket offsets, so nothing is written
    if (plane_empty_cl<N>(pts.off, c, ix)) return;
    for (int e = threadIdx.x; e < P::ROWSLAB; e += NT) R[e] = C{(T)0, (T)0};
    cl.sync();   // every slab of the cluster is zero before any remote add
    const PlaneBucketsCl pb = plane_buckets_cl<N>(pts.off, c, ix, q);
    const PtRec<T>* Rp = static_cast<const PtRec<T>*>(pts.rec);
    for (int t = threadIdx.x; t < pb.n0 + pb.n1; t += NT) {
      const bool lower = t < pb.n0;
      const PtRec<T> p = Rp[lower ? pb.b0 + t : pb.b1 + (t - pb.n0)];
      const T val = p.r * rcomp_cl(p, j) * (lower ? (T)1 - p.fx : p.fx);
      if (val == (T)0) continue;
      const int iy = p.yz / N, iz = p.yz % N;
      if (iy < row0 || iy >= row0 + RQ) continue;   // not this CTA's row (never for a consistent bucket)
      const int iy1 = (iy + 1) & (N - 1), iz1 = (iz + 1) & (N - 1);
      const T wy1 = p.fy, wy0 = (T)1 - p.fy, wz1 = p.fz, wz0 = (T)1 - p.fz;
      // row iy is ours; row iy + 1 belongs to CTA (iy + 1) / RQ
      const int o1 = iy1 / RQ;
      atomicAdd(zreal_cl<T, N>(R, iy - row0, iz), val * wy0 * wz0);
      atomicAdd(zreal_cl<T, N>(R, iy - row0, iz1), val * wy0 * wz1);
      atomicAdd(zreal_cl<T, N>(rem(o1), iy1 - o1 * RQ, iz), val * wy1 * wz0);
      atomicAdd(zreal_cl<T, N>(rem(o1), iy1 - o1 * RQ, iz1), val * wy1 * wz1);
    }
    cl.sync();
  }
  fft_smem<T, N, false, P::PR, NT, false>(R, P::ZP, 1, tw);
  unpack_rows_cl<T, N>(R);
  cl.sync();   // all row slabs hold half spectra
  int c0, c1;
  own_columns_cl<N>(q, c0, c1);
  const int nc = c1 - c0;
  #pragma unroll 17
  for (int e = threadIdx.x; e < N * P::CW; e += NT) {
    const int y = e / P::CW, cc = e % P::CW;
    C v = C{(T)0, (T)0};
    if (cc < nc) {
      const int o = y / RQ;
      v = rem(o)[(y - o * RQ) * NH + c0 + cc];
    }
    Cs[y * CWP + cc] = v;
  }
  cl.sync();   // remote reads done before any CTA moves on or exits
  fft_smem<T, N, false, P::CW, NT, true>(Cs, 1, CWP, tw);
  C* dst = out + (long long)s * out_stride + (long long)ix * N * NH;
  #pragma unroll 4
  for (int e = threadIdx.x; e < N * nc; e += NT) {
    const int y = e / nc, cc = e % nc;
    dst[y * NH + c0 + cc] = Cs[y * CWP + cc];
  }
}

// ---------------------------------------------------------------------------
// Plane pass, inverse: spectrum plane -> (y c2c, z c2r) -> real rows, then
// MODE 0: plain store; 1: gradient / leapfrog epilogue; 2: CIC gather of the
// bucketed points (u and du partials of this plane and component).
// ---------------------------------------------------------------------------


template <typename T, int N, int MODE>
__global__ void __cluster_dims__(ClCfg<N>::K, 1, 1) __launch_bounds__(ClCfg<N>::NT)
k_plane_c2r_cl(const cplx<T>* __restrict__ in, long long in_stride, T* __restrict__ out,
            long long out_stride, const cplx<T>* __restrict__ tw, FieldEpi epi, PlanePoints pts,
            cplx<T>* __restrict__ next, long long next_stride) {
  pdl_wait();
  pdl_trigger();
  using C = cplx<T>;
  using P = ClCfg<N>;
  constexpr int NT = P::NT, K = P::K, RQ = P::RQ, NH = P::NH, CWP = P::CWP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* R = reinterpret_cast<C*>(smem_raw);
  C* Cs = R + P::ROWSLAB;
  __shared__ double red[2][NT / 32];
  cg::cluster_group cl = cg::this_cluster();
  const int q = (int)cl.block_rank();
  const int ix = blockIdx.x / K;
  const int s = blockIdx.y;
  const int row0 = q * RQ;
  auto rem = [&](int k) -> C* { return cl.map_shared_rank(R, k); };   // CTA k's row slab
  // gather: only the values at the points' corners are used, so a plane
  // that no point touches needs no transform (same answer in every CTA of
  // the cluster, so the whole cluster leaves before any cluster barrier)
  if (MODE == C2R_GATHER && plane_empty_cl<N>(pts.off, s / 3, ix)) return;
  if constexpr (MODE == C2R_EPI) {
    // pull this CTA's rows of w and p_w toward L2 during the transforms
    const long long base = (long long)s * epi.grid_stride + ((long long)ix * N + row0) * N;
    const char* wb = reinterpret_cast<const char*>(reinterpret_cast<const T*>(epi.w) + base);
    const char* pb = reinterpret_cast<const char*>(reinterpret_cast<const T*>(epi.pw) + base);
    constexpr int LINES = (int)(sizeof(T) * RQ * N / 128);
    const bool kick = epi.mode != GM_GRAD;
    for (int l = threadIdx.x; l < LINES; l += NT) {
      asm volatile("prefetch.global.L2 [%0];" ::"l"(wb + 128 * (long long)l));
      if (kick) asm volatile("prefetch.global.L2 [%0];" ::"l"(pb + 128 * (long long)l));
    }
  }
  int c0, c1;
  own_columns_cl<N>(q, c0, c1);
  const int nc = c1 - c0;
  const C* src = in + (long long)s * in_stride + (long long)ix * N * NH;
  #pragma unroll 17
  for (int e = threadIdx.x; e < N * P::CW; e += NT) {
    const int y = e / P::CW, cc = e % P::CW;
    Cs[y * CWP + cc] = cc < nc ? src[y * NH + c0 + cc] : C{(T)0, (T)0};
  }
  __syncthreads();
  fft_smem<T, N, true, P::CW, NT, true>(Cs, 1, CWP, tw);
  cl.sync();   // every CTA of the cluster is running before remote stores
  #pragma unroll 4
  for (int e = threadIdx.x; e < N * nc; e += NT) {
    const int y = e / nc, cc = e % nc;
    const int o = y / RQ;
    rem(o)[(y - o * RQ) * NH + c0 + cc] = Cs[y * CWP + cc];
  }
  cl.sync();   // own row slab complete
  pack_rows_cl<T, N>(R);
  fft_smem<T, N, true, P::PR, NT, false>(R, P::ZP, 1, tw);
  using V2 = typename Pair2Cl<T>::type;
  constexpr int ITEMS = P::PR * (N / 2);
  if constexpr (MODE == C2R_STORE) {
    T* dst = out + (long long)s * out_stride + ((long long)ix * N + row0) * N;
    for (int e = threadIdx.x; e < ITEMS; e += NT) {
      const int r = e / (N / 2), z = 2 * (e % (N / 2));
      T v[4];
      read_item_cl<T, N>(R, r, z, v);
      *reinterpret_cast<V2*>(dst + (2 * r) * N + z) = V2{v[0], v[2]};
      *reinterpret_cast<V2*>(dst + (2 * r + 1) * N + z) = V2{v[1], v[3]};
    }
  } else if constexpr (MODE == C2R_GATHER) {
    cl.sync();   // every row slab holds its real rows before remote reads
    const int c = s / 3, j = s % 3;
    const PlaneBucketsCl pb = plane_buckets_cl<N>(pts.off, c, ix, q);
    const PtRec<T>* Rp = static_cast<const PtRec<T>*>(pts.rec);
    T* part = static_cast<T*>(pts.part);
    const T idl = (T)pts.inv_delta;
    for (int t = threadIdx.x; t < pb.n0 + pb.n1; t += NT) {
      const bool lower = t < pb.n0;
      const int qq = lower ? pb.b0 + t : pb.b1 + (t - pb.n0);
      const PtRec<T> p = Rp[qq];
      const int iy = p.yz / N, iz = p.yz % N;
      if (iy < row0 || iy >= row0 + RQ) continue;   // not this CTA's row (never for a consistent bucket)
      const int iy1 = (iy + 1) & (N - 1), iz1 = (iz + 1) & (N - 1);
      const int o1 = iy1 / RQ;
      const T v00 = *zreal_cl<T, N>(R, iy - row0, iz), v01 = *zreal_cl<T, N>(R, iy - row0, iz1);
      const T v10 = *zreal_cl<T, N>(rem(o1), iy1 - o1 * RQ, iz);
      const T v11 = *zreal_cl<T, N>(rem(o1), iy1 - o1 * RQ, iz1);
      const T wy1 = p.fy, wy0 = (T)1 - p.fy, wz1 = p.fz, wz0 = (T)1 - p.fz;
      const T a0 = wz0 * v00 + wz1 * v01, a1 = wz0 * v10 + wz1 * v11;
      const T S = wy0 * a0 + wy1 * a1;      // y-z interpolation on this plane
      const T Gy = a1 - a0;                 // d/dy (per cell) of it
      const T Gz = wy0 * (v01 - v00) + wy1 * (v11 - v10);
      const T wx = lower ? (T)1 - p.fx : p.fx;
      const T sx = lower ? (T)-1 : (T)1;
      const T rj = rcomp_cl(p, j);
      const int side = lower ? 0 : 1;
      part[(long long)(side * 3 + j) * pts.ntot + qq] = rj * wx * S;
      part[(long long)(6 + side * 3 + j) * pts.ntot + qq] =
          rj * (p.rx * sx * S + p.ry * wx * Gy + p.rz * wx * Gz) * idl;
    }
    cl.sync();   // remote reads done before any CTA exits
  } else {
    // ---- gradient / leapfrog epilogue (one chain per blockIdx.y) ----
    const long long base = (long long)s * epi.grid_stride + ((long long)ix * N + row0) * N;
    T* w = reinterpret_cast<T*>(epi.w) + base;
    T* pw = reinterpret_cast<T*>(epi.pw) + base;
    T* gw = reinterpret_cast<T*>(epi.gw) + base;
    const int mode = epi.mode;
    const T eps = (T)epi.cs[s].eps;
    const T ck = (mode == GM_KICK_DRIFT) ? eps : (T)0.5 * eps;
    HalfSqAcc<T> aw, ap;
    #pragma unroll 4
    for (int e = threadIdx.x; e < ITEMS; e += NT) {
      const int r = e / (N / 2), z = 2 * (e % (N / 2));
      T g[4];
      read_item_cl<T, N>(R, r, z, g);
#pragma unroll
      for (int h = 0; h < 2; ++h) {   // local row 2r + h, columns z, z + 1
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
            g[h] = n0;        // the drifted field replaces g in the row slab
            g[2 + h] = n1;
          }
        }
      }
      if (next != nullptr && mode == GM_KICK_DRIFT) {
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4*>(&R[r * P::ZP + z]) = make_float4(g[0], g[1], g[2], g[3]);
        } else {
          R[r * P::ZP + z] = cplx<T>{g[0], g[1]};
          R[r * P::ZP + z + 1] = cplx<T>{g[2], g[3]};
        }
      }
    }
    // deterministic block reduction: a fixed shuffle tree per warp, then
    // thread 0 over the warps in order
    aw.warp_reduce();
    ap.warp_reduce();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][wid] = aw.value();
      red[1][wid] = ap.value();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int i = 0; i < NT / 32; ++i) {
        a += red[0][i];
        b += red[1][i];
      }
      epi.prior_part[(long long)s * N * K + ix * K + q] = a;
      if (mode == GM_KICK_LAST) epi.kin_part[(long long)s * N * K + ix * K + q] = b;
    }
    if (next != nullptr && mode == GM_KICK_DRIFT) {
      // forward plane transform of the drifted field for the next evaluation
      __syncthreads();
      fft_smem<T, N, false, P::PR, NT, false>(R, P::ZP, 1, tw);
      unpack_rows_cl<T, N>(R);
      cl.sync();
      #pragma unroll 17
      for (int e = threadIdx.x; e < N * P::CW; e += NT) {
        const int y = e / P::CW, cc = e % P::CW;
        C v = C{(T)0, (T)0};
        if (cc < nc) {
          const int o = y / RQ;
          v = rem(o)[(y - o * RQ) * NH + c0 + cc];
        }
        Cs[y * CWP + cc] = v;
      }
      cl.sync();
      fft_smem<T, N, false, P::CW, NT, true>(Cs, 1, CWP, tw);
      C* dst = next + (long long)s * next_stride + (long long)ix * N * NH;
      #pragma unroll 4
      for (int e = threadIdx.x; e < N * nc; e += NT) {
        const int y = e / nc, cc = e % nc;
        dst[y * NH + c0 + cc] = Cs[y * CWP + cc];
      }
    }
  }
}


// ---------------------------------------------------------------------------
// Launchers (FP32, N = 256).
// ---------------------------------------------------------------------------
template <typename T, int N>
static cudaError_t prepare_cl_t() {
  cudaError_t e;
  constexpr int sp = (int)(sizeof(cplx<T>) * (ClCfg<N>::ROWSLAB + ClCfg<N>::COLSLAB));
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_plane_r2c_cl<T, N, false>, A, sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_r2c_cl<T, N, true>, A, sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_c2r_cl<T, N, C2R_STORE>, A, sp)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_plane_c2r_cl<T, N, C2R_EPI>, A, sp)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_plane_c2r_cl<T, N, C2R_GATHER>, A, sp);
}

cudaError_t plane_cl_prepare() {
  // the point sub-buckets of a plane are the cluster's row slabs
  if (plane_split(256) != ClCfg<256>::K) return cudaErrorInvalidConfiguration;
  return prepare_cl_t<float, 256>();
}

cudaError_t launch_plane_r2c_cl(const void* in, long long in_stride, void* out, long long out_stride, int count,
                                const void* tw, const PlanePoints* pts, cudaStream_t st) {
  using T = float;
  constexpr int N = 256;
  constexpr size_t sm = sizeof(cplx<T>) * (ClCfg<N>::ROWSLAB + ClCfg<N>::COLSLAB);
  const dim3 grid(N * ClCfg<N>::K, count);
  PlanePoints none{};
  if (pts)
    return launch_k<PDL_PLANE>(k_plane_r2c_cl<T, N, true>, grid, dim3(ClCfg<N>::NT), sm, st, static_cast<const T*>(nullptr),
                    0ll, static_cast<cplx<T>*>(out), out_stride, static_cast<const cplx<T>*>(tw), *pts);
  return launch_k<PDL_PLANE>(k_plane_r2c_cl<T, N, false>, grid, dim3(ClCfg<N>::NT), sm, st, static_cast<const T*>(in), in_stride,
                  static_cast<cplx<T>*>(out), out_stride, static_cast<const cplx<T>*>(tw), none);
}

cudaError_t launch_plane_c2r_cl(int mode, const void* in, long long in_stride, void* out, long long out_stride,
                                int count, const void* tw, const FieldEpi* epi, const PlanePoints* pts,
                                void* next, cudaStream_t st) {
  using T = float;
  constexpr int N = 256;
  constexpr size_t sm = sizeof(cplx<T>) * (ClCfg<N>::ROWSLAB + ClCfg<N>::COLSLAB);
  const dim3 grid(N * ClCfg<N>::K, count);
  FieldEpi e{};
  if (epi) e = *epi;
  PlanePoints p{};
  if (pts) p = *pts;
  auto args = [&](auto kern) {
    return launch_k<PDL_PLANE>(kern, grid, dim3(ClCfg<N>::NT), sm, st, static_cast<const cplx<T>*>(in), in_stride,
                    static_cast<T*>(out), out_stride, static_cast<const cplx<T>*>(tw), e, p,
                    static_cast<cplx<T>*>(next), in_stride);
  };
  if (mode == C2R_EPI) return args(k_plane_c2r_cl<T, N, C2R_EPI>);
  if (mode == C2R_GATHER) return args(k_plane_c2r_cl<T, N, C2R_GATHER>);
  return args(k_plane_c2r_cl<T, N, C2R_STORE>);
}

}  // namespace hm
