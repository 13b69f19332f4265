// Plane passes of the 3D transforms for N = 256 (FP32), where an x-plane of
// the half spectrum (256 x 129 complex, 264 KB) does not fit one CTA's shared
// memory.  Each plane pass is split into two passes over memory instead:
//
//   z pass : one CTA per (x-plane, slab of 32 rows); the rows are contiguous
//            in memory, two real rows are transformed as one complex row, and
//            the CIC gather/scatter and the field's leapfrog epilogue work on
//            the slab's rows (a point's corner rows iy, iy + 1 lie in its
//            slab and the next row, which the gather transforms as a halo row
//            and the scatter leaves to the next slab's CTA);
//   y pass : one CTA per (x-plane, tile of 16 kz columns); 256 rows of the
//            tile are loaded with row stride N/2 + 1 and transformed in place.
//
// The x transforms stay in the pencil kernels.  No CTA exchanges data with
// another, so there are no cluster barriers; the cost is one more read and
// write of the spectra, which at this size are HBM-resident anyway.  The
// points are bucketed by (x-plane, slab) -- the eight sub-buckets per plane
// of the point placement -- and slabs without points skip their transforms.
#include "hm_fft.cuh"
#include "hm_internal.h"

namespace hm {
namespace {

constexpr int N = 256;
constexpr int NH = N / 2 + 1;               // kz = 0..N/2
constexpr int K = 8;                        // row slabs per plane (= point sub-buckets per plane)
constexpr int RQ = N / K;                   // rows per slab
constexpr int PR = RQ / 2;                  // packed complex rows per slab
constexpr int ZP = N + 1;                   // odd pitch of a packed row in shared memory
constexpr int NT = 256;                     // threads per CTA
constexpr int TW = 16;                      // kz columns per y tile
constexpr int NTILE = (NH + TW - 1) / TW;   // y tiles per plane
using C = float2;

enum ZMode : int { Z_STORE = 0, Z_EPI = 1, Z_GATHER = 2 };

// Point bucket offsets of chain c: [N*K + 1] entries, sub-bucket (x, slab).
__device__ __forceinline__ const int* chain_off(const int* off, int c) { return off + (long long)c * (N * K + 1); }

// Plane x holds a CIC corner of some point of chain c: bucket x (lower
// corner on x) or bucket x - 1 (upper corner on x) is non-empty.
__device__ __forceinline__ bool plane_occupied(const int* __restrict__ off, int c, int ix) {
  const int* o = chain_off(off, c);
  const int ixm = (ix + N - 1) & (N - 1);
  return o[(ix + 1) * K] != o[ix * K] || o[(ixm + 1) * K] != o[ixm * K];
}

__device__ __forceinline__ float rcomp(const PtRec<float>& p, int j) { return j == 0 ? p.rx : (j == 1 ? p.ry : p.rz); }

// Real row yl (local to the slab) at z in the packed view (rows 2r, 2r + 1
// are the real and imaginary parts of packed row r).
__device__ __forceinline__ float* zreal(C* B, int yl, int z) {
  return reinterpret_cast<float*>(&B[(yl >> 1) * ZP + z]) + (yl & 1);
}

// After the forward z transform of the packed rows: split each packed row
// Z = X_a + i X_b into the half spectra of its two real rows,
// X_a[k] = (Z[k] + conj Z[N-k])/2, X_b[k] = (Z[k] - conj Z[N-k])/(2i), and
// store rows of NH entries to dst (rows of the slab, pitch NH).
__device__ __forceinline__ void store_half_spectra(const C* B, C* __restrict__ dst) {
#pragma unroll 4
  for (int e = threadIdx.x; e < PR * NH; e += NT) {
    const int r = e / NH, k = e - r * NH;
    const C zk = B[r * ZP + k], zm = cconj(B[r * ZP + ((N - k) & (N - 1))]);
    const C sp = cadd(zk, zm), df = csub(zk, zm);
    dst[(2 * r) * NH + k] = C{0.5f * sp.x, 0.5f * sp.y};
    dst[(2 * r + 1) * NH + k] = C{0.5f * df.y, -0.5f * df.x};
  }
}

// ---------------------------------------------------------------------------
// z pass, forward: real rows -> half spectra along z.  SCATTER builds the
// rows from the bucketed residuals (the adjoint of the CIC gather,
// s_j(corner) += r rhat_j W(corner), shared-memory atomics): the points whose
// lower y corner is in this slab, and those of the slab below whose upper
// y corner is this slab's first row, for both x sides of the plane.
// ---------------------------------------------------------------------------
template <bool SCATTER>
__global__ void __launch_bounds__(NT, 4)
k_z_r2c(const float* __restrict__ in, long long in_stride, C* __restrict__ out, long long out_stride,
        const C* __restrict__ tw, PlanePoints pts) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* B = reinterpret_cast<C*>(smem_raw);
  const int ix = blockIdx.x / K, q = blockIdx.x % K;
  const int s = blockIdx.y;
  const int row0 = q * RQ;
  C* dst = out + (long long)s * out_stride + ((long long)ix * N + row0) * NH;
  if constexpr (!SCATTER) {
    const float* src = in + (long long)s * in_stride + ((long long)ix * N + row0) * N;
#pragma unroll 8
    for (int e = threadIdx.x; e < PR * N; e += NT) {
      const int r = e / N, z = e - r * N;
      B[r * ZP + z] = C{__ldg(&src[(2 * r) * N + z]), __ldg(&src[(2 * r + 1) * N + z])};
    }
  } else {
    const int c = s / 3, j = s - 3 * c;
    // no point has a CIC corner on this plane: its spectrum is zero, which
    // the y pass and the adjoint pencils know from the same offsets
    if (!plane_occupied(pts.off, c, ix)) return;
    const int* o = chain_off(pts.off, c);
    const int ixm = (ix + N - 1) & (N - 1), qm = (q + K - 1) & (K - 1);
    // point sets: 0 own slab / 1 slab below, lower x corner on this plane;
    // 2 own slab / 3 slab below, upper x corner on this plane
    int b[4], n[4];
    b[0] = o[ix * K + q];
    n[0] = o[ix * K + q + 1] - b[0];
    b[1] = o[ix * K + qm];
    n[1] = o[ix * K + qm + 1] - b[1];
    b[2] = o[ixm * K + q];
    n[2] = o[ixm * K + q + 1] - b[2];
    b[3] = o[ixm * K + qm];
    n[3] = o[ixm * K + qm + 1] - b[3];
    const int tot = n[0] + n[1] + n[2] + n[3];
    if (tot == 0) {   // nothing lands in this slab: its rows are zero
      for (int e = threadIdx.x; e < RQ * NH; e += NT) dst[e] = C{0.f, 0.f};
      return;
    }
    for (int e = threadIdx.x; e < PR * ZP; e += NT) B[e] = C{0.f, 0.f};
    __syncthreads();
    const PtRec<float>* R = static_cast<const PtRec<float>*>(pts.rec);
    for (int t = threadIdx.x; t < tot; t += NT) {
      int set = 0, u = t;
      while (u >= n[set]) {
        u -= n[set];
        ++set;
      }
      const PtRec<float> p = R[b[set] + u];
      const bool lower = set < 2;
      const float val = p.r * rcomp(p, j) * (lower ? 1.0f - p.fx : p.fx);
      if (val == 0.0f) continue;
      const int iy = p.yz / N, iz = p.yz - (p.yz / N) * N;
      const int iz1 = (iz + 1) & (N - 1);
      const int yl0 = (iy - row0) & (N - 1), yl1 = (yl0 + 1) & (N - 1);   // local rows of the two y corners
      const float wy1 = p.fy, wy0 = 1.0f - p.fy, wz1 = p.fz, wz0 = 1.0f - p.fz;
      if (yl0 < RQ) {
        atomicAdd(zreal(B, yl0, iz), val * wy0 * wz0);
        atomicAdd(zreal(B, yl0, iz1), val * wy0 * wz1);
      }
      if (yl1 < RQ) {
        atomicAdd(zreal(B, yl1, iz), val * wy1 * wz0);
        atomicAdd(zreal(B, yl1, iz1), val * wy1 * wz1);
      }
    }
  }
  __syncthreads();
  fft_smem<float, N, false, PR, NT, false>(B, ZP, 1, tw);
  store_half_spectra(B, dst);
}

// ---------------------------------------------------------------------------
// y pass: the y transform of a tile of TW kz columns of one x-plane, in
// place (each CTA reads all of its columns before writing them).  The first
// radix stage reads global memory, the second writes it.  With plane_off,
// planes without a point corner are skipped (their spectra are not used, or
// are zero and known to be).
// ---------------------------------------------------------------------------
template <bool INV>
__global__ void __launch_bounds__(NT, 4)
k_y_pass(C* __restrict__ data, long long stride, const C* __restrict__ tw, const int* __restrict__ plane_off,
         int comps) {
  pdl_wait();
  pdl_trigger();
  constexpr int R1 = Radix<N>::R1, M = Radix<N>::M;
  static_assert(TW * M == NT && TW * R1 == NT, "one radix group per thread in both stages");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);   // [N][TW]
  const int ix = blockIdx.y, s = blockIdx.z;
  if (plane_off != nullptr && !plane_occupied(plane_off, s / comps, ix)) return;
  C* base = data + (long long)s * stride + (long long)ix * N * NH;
  const int t = threadIdx.x % TW, g = threadIdx.x / TW;
  const int col = blockIdx.x * TW + t;
  const bool ok = col < NH;
  {
    // stage 1: group m = g, rows m + M j
    C a[R1];
#pragma unroll
    for (int jj = 0; jj < R1; ++jj) a[jj] = ok ? base[(g + M * jj) * NH + col] : C{0.f, 0.f};
    dft_reg<R1, INV>(a);
#pragma unroll
    for (int k2 = 1; k2 < R1; ++k2) {
      C wv = __ldg(&tw[g * k2]);
      if (INV) wv.y = -wv.y;
      a[k2] = cmul(a[k2], wv);
    }
#pragma unroll
    for (int k2 = 0; k2 < R1; ++k2) buf[(g + M * k2) * TW + t] = a[k2];
  }
  __syncthreads();
  {
    // stage 2: group k2 = g, the M-point DFT of rows M k2 .. M k2 + M - 1
    C a[M];
#pragma unroll
    for (int mm = 0; mm < M; ++mm) a[mm] = buf[(M * g + mm) * TW + t];
    dft_reg<M, INV>(a);
    if (ok) {
#pragma unroll
      for (int k1 = 0; k1 < M; ++k1) base[(g + R1 * k1) * NH + col] = a[k1];
    }
  }
}

// ---------------------------------------------------------------------------
// z pass, inverse: half-spectrum rows -> real rows (c2r along z), then
// Z_STORE: plain store; Z_EPI: gradient / leapfrog epilogue (+ the forward z
// transform of the drifted field to `next`); Z_GATHER: CIC gather of the
// points whose lower y corner is in this slab (u and du partials of this
// plane and component), with the next slab's first row as a halo row.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(NT, MODE == Z_GATHER ? 3 : 4)   // the halo pair needs a second stage-2 group
k_z_c2r(const C* __restrict__ in, long long in_stride, float* __restrict__ out, long long out_stride,
        const C* __restrict__ tw, FieldEpi epi, PlanePoints pts, C* __restrict__ next, long long next_stride) {
  pdl_wait();
  pdl_trigger();
  constexpr int PRH = MODE == Z_GATHER ? PR + 1 : PR;   // packed rows incl. the halo pair
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* B = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[2][NT / 32];
  const int ix = blockIdx.x / K, q = blockIdx.x % K;
  const int s = blockIdx.y;
  const int row0 = q * RQ;
  int b0 = 0, n0 = 0, b1 = 0, n1 = 0;
  if constexpr (MODE == Z_GATHER) {
    // only the slab's points need the values: no points, no transform
    const int* o = chain_off(pts.off, s / 3);
    const int ixm = (ix + N - 1) & (N - 1);
    b0 = o[ix * K + q];
    n0 = o[ix * K + q + 1] - b0;
    b1 = o[ixm * K + q];
    n1 = o[ixm * K + q + 1] - b1;
    if (n0 + n1 == 0) return;
  }
  // packed row r = rows y = row0 + 2r, y + 1 (mod N): Z[k] = X_a[k] + i X_b[k]
  // with X[N-k] = conj X[k]; the imaginary parts at kz = 0 and N/2 are
  // dropped (what a c2r transform keeps)
  const C* src = in + (long long)s * in_stride + (long long)ix * N * NH;
#pragma unroll 4
  for (int e = threadIdx.x; e < PRH * NH; e += NT) {
    const int r = e / NH, k = e - r * NH;
    const int ya = (row0 + 2 * r) & (N - 1), yb = (ya + 1) & (N - 1);
    C xa = src[ya * NH + k], xb = src[yb * NH + k];
    if (k == 0 || k == N / 2) {
      xa.y = 0.f;
      xb.y = 0.f;
    }
    B[r * ZP + k] = C{xa.x - xb.y, xa.y + xb.x};
    if (k != 0 && k != N / 2) B[r * ZP + N - k] = C{xa.x + xb.y, xb.x - xa.y};
  }
  __syncthreads();
  fft_smem<float, N, true, PRH, NT, false>(B, ZP, 1, tw);
  constexpr int ITEMS = PR * N;   // item (r, z): real rows 2r, 2r + 1 at column z
  if constexpr (MODE == Z_STORE) {
    float* dst = out + (long long)s * out_stride + ((long long)ix * N + row0) * N;
#pragma unroll 4
    for (int e = threadIdx.x; e < ITEMS; e += NT) {
      const int r = e / N, z = e - r * N;
      const C v = B[r * ZP + z];
      dst[(2 * r) * N + z] = v.x;
      dst[(2 * r + 1) * N + z] = v.y;
    }
  } else if constexpr (MODE == Z_GATHER) {
    const int j = s % 3;
    const PtRec<float>* R = static_cast<const PtRec<float>*>(pts.rec);
    float* part = static_cast<float*>(pts.part);
    const float idl = (float)pts.inv_delta;
    for (int t = threadIdx.x; t < n0 + n1; t += NT) {
      const bool lower = t < n0;
      const int qq = lower ? b0 + t : b1 + (t - n0);
      const PtRec<float> p = R[qq];
      const int iy = p.yz / N, iz = p.yz - (p.yz / N) * N;
      const int iz1 = (iz + 1) & (N - 1);
      const int yl = iy - row0;   // in [0, RQ): the bucket is this slab
      const float v00 = *zreal(B, yl, iz), v01 = *zreal(B, yl, iz1);
      const float v10 = *zreal(B, yl + 1, iz), v11 = *zreal(B, yl + 1, iz1);
      const float wy1 = p.fy, wy0 = 1.0f - p.fy, wz1 = p.fz, wz0 = 1.0f - p.fz;
      const float a0 = wz0 * v00 + wz1 * v01, a1 = wz0 * v10 + wz1 * v11;
      const float S = wy0 * a0 + wy1 * a1;      // y-z interpolation on this plane
      const float Gy = a1 - a0;                 // d/dy (per cell) of it
      const float Gz = wy0 * (v01 - v00) + wy1 * (v11 - v10);
      const float wx = lower ? 1.0f - p.fx : p.fx;
      const float sx = lower ? -1.0f : 1.0f;
      const float rj = rcomp(p, j);
      const int side = lower ? 0 : 1;
      part[(long long)(side * 3 + j) * pts.ntot + qq] = rj * wx * S;
      part[(long long)(6 + side * 3 + j) * pts.ntot + qq] = rj * (p.rx * sx * S + p.ry * wx * Gy + p.rz * wx * Gz) * idl;
    }
  } else {
    // ---- gradient / leapfrog epilogue (one chain per blockIdx.y) ----
    const long long gbase = (long long)s * epi.grid_stride + ((long long)ix * N + row0) * N;
    float* __restrict__ w = reinterpret_cast<float*>(epi.w) + gbase;
    float* __restrict__ pw = reinterpret_cast<float*>(epi.pw) + gbase;
    float* __restrict__ gw = reinterpret_cast<float*>(epi.gw) + gbase;
    const int mode = epi.mode;
    const float eps = (float)epi.cs[s].eps;
    const float ck = (mode == GM_KICK_DRIFT) ? eps : 0.5f * eps;
    const bool fuse_next = next != nullptr && mode == GM_KICK_DRIFT;
    const bool kick = mode != GM_GRAD;
    // the prior and kinetic sums are read only at the trajectory's end point
    // (and for GM_GRAD): an intermediate leapfrog evaluation skips them
    const bool sums = mode != GM_KICK_DRIFT, last = mode == GM_KICK_LAST;
    HalfSqAcc<float> aw, ap;
    constexpr int U = 4;   // items per thread per round, loads issued before stores
    static_assert(ITEMS % (U * NT) == 0, "no ragged round");
#pragma unroll 1
    for (int e0 = threadIdx.x; e0 < ITEMS; e0 += U * NT) {
      float wv[U][2], pv[U][2];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NT, r = e / N, z = e - r * N;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int o = (2 * r + h) * N + z;
          wv[u][h] = w[o];
          pv[u][h] = kick ? pw[o] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NT, r = e / N, z = e - r * N;
        const C g2 = B[r * ZP + z];
        float nv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // row 2r + h, column z
          const int o = (2 * r + h) * N + z;
          const float w0 = wv[u][h];
          const float g0 = w0 + (h == 0 ? g2.x : g2.y);
          if (sums) aw.add_half_sq(w0);
          nv[h] = w0;
          if (mode == GM_GRAD || mode == GM_KICK_LAST) gw[o] = g0;
          if (kick) {
            const float p0 = pv[u][h] - ck * g0;
            pw[o] = p0;
            if (last) ap.add_half_sq(p0);
            if (mode == GM_KICK_DRIFT) {
              nv[h] = w0 + eps * p0;
              w[o] = nv[h];
            }
          }
        }
        if (fuse_next) B[r * ZP + z] = C{nv[0], nv[1]};   // the drifted field replaces g
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
      double a = 0.0, bsum = 0.0;
      for (int i = 0; i < NT / 32; ++i) {
        a += red[0][i];
        bsum += red[1][i];
      }
      epi.prior_part[(long long)s * N * K + ix * K + q] = a;
      if (mode == GM_KICK_LAST) epi.kin_part[(long long)s * N * K + ix * K + q] = bsum;
    }
    if (fuse_next) {
      // forward z transform of the drifted rows; the launcher follows with
      // the y pass of `next`
      fft_smem<float, N, false, PR, NT, false>(B, ZP, 1, tw);
      store_half_spectra(B, next + (long long)s * next_stride + ((long long)ix * N + row0) * NH);
    }
  }
}

constexpr size_t kZSmem = sizeof(C) * PR * ZP;
constexpr size_t kZSmemHalo = sizeof(C) * (PR + 1) * ZP;
constexpr size_t kYSmem = sizeof(C) * N * TW;

cudaError_t y_pass(bool inv, void* data, long long stride, int count, const void* tw, const int* plane_off,
                   int comps, cudaStream_t st) {
  const dim3 grid(NTILE, N, count);
  if (inv)
    return launch_k<PDL_PLANE>(k_y_pass<true>, grid, dim3(NT), kYSmem, st, static_cast<C*>(data), stride,
                               static_cast<const C*>(tw), plane_off, comps);
  return launch_k<PDL_PLANE>(k_y_pass<false>, grid, dim3(NT), kYSmem, st, static_cast<C*>(data), stride,
                             static_cast<const C*>(tw), plane_off, comps);
}

}  // namespace

cudaError_t plane256_prepare() {
  // the point sub-buckets of a plane are the z pass's row slabs
  if (plane_split(N) != K) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_z_r2c<false>, A, (int)kZSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_z_r2c<true>, A, (int)kZSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_z_c2r<Z_STORE>, A, (int)kZSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_z_c2r<Z_EPI>, A, (int)kZSmem)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_z_c2r<Z_GATHER>, A, (int)kZSmemHalo)) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_y_pass<false>, A, (int)kYSmem)) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_y_pass<true>, A, (int)kYSmem);
}

cudaError_t launch_plane_r2c_256(const void* in, long long in_stride, void* out, long long out_stride, int count,
                                 const void* tw, const PlanePoints* pts, cudaStream_t st) {
  const dim3 grid(N * K, count);
  cudaError_t e;
  if (pts) {
    e = launch_k<PDL_PLANE>(k_z_r2c<true>, grid, dim3(NT), kZSmem, st, static_cast<const float*>(nullptr), 0ll,
                            static_cast<C*>(out), out_stride, static_cast<const C*>(tw), *pts);
    if (e != cudaSuccess) return e;
    return y_pass(false, out, out_stride, count, tw, pts->off, 3, st);
  }
  PlanePoints none{};
  e = launch_k<PDL_PLANE>(k_z_r2c<false>, grid, dim3(NT), kZSmem, st, static_cast<const float*>(in), in_stride,
                          static_cast<C*>(out), out_stride, static_cast<const C*>(tw), none);
  if (e != cudaSuccess) return e;
  return y_pass(false, out, out_stride, count, tw, nullptr, 1, st);
}

cudaError_t launch_plane_c2r_256(int mode, const void* in, long long in_stride, void* out, long long out_stride,
                                 int count, const void* tw, const FieldEpi* epi, const PlanePoints* pts, void* next,
                                 cudaStream_t st) {
  // the y pass runs in place on `in`, a library workspace of every caller
  cudaError_t e = y_pass(true, const_cast<void*>(in), in_stride, count, tw,
                         mode == Z_GATHER && pts ? pts->off : nullptr, 3, st);
  if (e != cudaSuccess) return e;
  const dim3 grid(N * K, count);
  FieldEpi ep{};
  if (epi) ep = *epi;
  PlanePoints pp{};
  if (pts) pp = *pts;
  const C* src = static_cast<const C*>(in);
  const C* twc = static_cast<const C*>(tw);
  if (mode == Z_GATHER)
    return launch_k<PDL_PLANE>(k_z_c2r<Z_GATHER>, grid, dim3(NT), kZSmemHalo, st, src, in_stride,
                               static_cast<float*>(nullptr), 0ll, twc, ep, pp, static_cast<C*>(nullptr), 0ll);
  if (mode == Z_EPI) {
    e = launch_k<PDL_PLANE>(k_z_c2r<Z_EPI>, grid, dim3(NT), kZSmem, st, src, in_stride, static_cast<float*>(out),
                            out_stride, twc, ep, pp, static_cast<C*>(next), in_stride);
    if (e != cudaSuccess || next == nullptr || ep.mode != GM_KICK_DRIFT) return e;
    return y_pass(false, next, in_stride, count, tw, nullptr, 1, st);
  }
  return launch_k<PDL_PLANE>(k_z_c2r<Z_STORE>, grid, dim3(NT), kZSmem, st, src, in_stride, static_cast<float*>(out),
                             out_stride, twc, ep, pp, static_cast<C*>(nullptr), 0ll);
}

}  // namespace hm
