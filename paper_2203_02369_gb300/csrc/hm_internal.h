// Internal declarations shared by the HAMLET CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

namespace hm {

// Kernel launch, optionally with programmatic stream serialisation (the
// kernel may start while its predecessor in the stream finishes; it calls
// pdl_wait before reading the predecessor's output), for the categories
// that HM_PDL selects (default: the x pencils and the per-trajectory
// kernels: start, finalize, restore).  Launching the plane passes
// or the point kernels early made the 128^3 trajectory slower: the early
// CTAs wait on SMs that the predecessor's last CTAs or the side stream need.
// Launch categories for the programmatic-dependent-launch switch: the
// environment variable HM_PDL is a bit mask of the categories whose kernels
// may start early (the kernel launched with the attribute is the one that
// waits for its predecessor).
enum PdlCat : int { PDL_PLANE = 1, PDL_PENCIL = 2, PDL_POINTS = 4, PDL_OTHER = 8 };
bool pdl_enabled(int cat);
template <int CAT = PDL_OTHER, typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled(CAT) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

constexpr double kC = 299792.458;  // speed of light, km/s
constexpr double kH0 = 100.0;      // km/s/(Mpc/h)

enum PriorKind : int { PRIOR_TABLE = 0, PRIOR_POWER = 1 };

// Sub-buckets of the points per x-plane (the plane passes run one CTA per
// plane, so one bucket per plane: the points with lower CIC corner on it).
template <int N> struct PlaneSplit {
  static constexpr int K = 1;
};
int plane_split(int N);
// Most point sub-buckets per chain (N * plane_split(N) must stay below it):
// the placement kernel scans the bucket counts of a chain in shared memory.
constexpr int kMaxBuckets = 4096;

// Per-chain constants of the point likelihood (device resident).
struct PointParams {
  double obs[3];
  double delta;          // grid spacing L/N
  double inv_delta;      // 1/delta (rounded once, on the host)
  float obs_hi[3], obs_lo[3];          // obs and inv_delta as float pairs hi + lo
  float inv_delta_hi, inv_delta_lo;    // (hi = the value rounded to float)
  double omega_m, h;
  double sigma_nl2;      // sigma_NL^2
  double ik2_nl, logk2_nl;  // 1/sigma_NL^2 and ln sigma_NL^2 (kappa^2 of a point with sigma_cz = 0)
  double minv_d;         // (sigma_v/H0)^2, inverse mass of a distance
  double k3;             // 3 Omega_m H0 / c (zbar = c23 (1 - sqrt(1 - k3 d)))
  double c23;            // 2 / (3 Omega_m)
  double inv_h;          // 1 / h (luminosity distance in Mpc: d (1 + zbar) / h)
  float c23k3_f, inv_h_f, k3_f;   // c23 k3, 1/h and k3 rounded to float
  int N;
  int prior_kind;
  int prior_nbins;
  int ksplit;            // CTAs per plane (sub-buckets per x-plane)
  int rq;                // rows per CTA, N / ksplit
  double prior_d0, prior_bin;
  const double* prior_logdens;
  double prior_alpha, prior_dmin, prior_dmax;
  long long pt_off, pt_n;  // this chain's slice of the point arrays
};

// Per-chain scalars (device resident, FP64 energies).
struct ChainScal {
  double eps;            // leapfrog step
  double psi;            // Psi at the current position q
  double psi_prior;      // |w|^2/2 at q
  double psi_pts;        // sum of point terms at q
  double kin;            // kinetic energy of the current momenta
  double H_old, H_new, logu;
  double psi0;           // Psi at the trajectory start
  long long traj;        // trajectory counter (Philox counter word 1)
  long long traj_run0;   // counter at the start of the current run (trace row 0)
  int accept;            // last decision
  int status;            // bit flags, see STATUS_*
  int n_bad;             // unused (kept for layout)
  int sample_d;          // 1: distances move, 0: held fixed
  // dual-averaging step-size adaptation (active while da_on != 0)
  double da_Hbar, da_lepsbar, da_mu, da_delta;
  int da_on, da_m;
  // sigma_NL as a sampled coordinate (eq. q), unit mass (eq. M_ab)
  double sig, p_sig, g_sig, sig0, g_sig0, kin_sig;
  int sample_sig, pad1;
};

enum : int { STATUS_DOMAIN = 1, STATUS_NONFINITE = 2 };

// Epilogue modes of the last c2r pass of the gradient.  The energy partials
// (prior, kinetic, Psi_i) are formed only where they are read: a standalone
// gradient and the trajectory's end point; the intermediate leapfrog
// evaluations skip them.
enum GradMode : int {
  GM_GRAD = 0,        // grad_w = w + g, prior partials (no momentum update)
  GM_KICK_DRIFT = 1,  // p -= eps*grad; w += eps*p (no energy partials)
  GM_KICK_LAST = 2,   // p -= eps/2*grad; store grad; prior and kinetic partials
};

struct FieldEpi {
  void* w;          // T [C][N^3] position (read; written when drifting)
  void* pw;         // T [C][N^3] momenta
  void* gw;         // T [C][N^3] gradient out (GM_GRAD, GM_KICK_LAST)
  double* prior_part;  // [C][N] partial sums of w^2/2 (one per x-plane)
  double* kin_part;    // [C][N] partial sums of p^2/2
  ChainScal* cs;
  long long grid_stride;  // elements between chains
  int mode;
};

// One point as the plane passes see it, stored in x-plane bucket order:
// fractional offsets in its cell, direction, (iy*N + iz) of the lower
// corner, and the residual r = dPsi/du once the likelihood has run.
// Per-point constants of the FP32 path's distance-only terms, formed in FP64
// on the host when the catalogue is set.  With s(d) = sqrt(1 - k3 d) and
// zbar(d) = c23 (1 - s(d)):
//   d_z   solves zbar(d_z) = z (the observed redshift),
//   d_ref solves d_ref (1 + zbar(d_ref))/h = x_ref = 10^((mu - 25)/5),
// so that z - zbar(d) and x(d) - x_ref, the two differences that cancel,
// follow from d - d_z and d - d_ref (float pairs) times smooth factors.
struct XRef {
  float dz_hi, dz_lo;    // d_z as hi + lo
  float dr_hi, dr_lo;    // d_ref as hi + lo
  float s_z, s_ref;      // s(d_z), s(d_ref)
  float e_z, e_ref;      // residuals z - zbar(d_z) and x(d_ref) - x_ref
};

template <typename T> struct PtRec {
  T fx, fy, fz;
  T rx, ry, rz;
  int yz;
  T r;
};

// Point-side arrays of C chains (points of chain c at [pt_off, pt_off+pt_n)).
struct PointArrays {
  const double* rx;
  const double* ry;
  const double* rz;
  const double* mu;
  const struct XRef* xr; // per-point constants of the FP32 path's distance terms
  const double* ismu2;   // 1 / sigma_mu^2 per point
  const double* zobs;
  const double* scz;
  double* d;
  double* pd;
  double* gd;
  int* cx;        // bucket key cx*ksplit + cy/rq of the lower corner, per point
  int* slot;      // rank inside the bucket (atomic order), per point
  int* pos;       // position in bucket order, per point
  int* cnt;       // [C][NB] bucket sizes of the current distances (NB = N*ksplit)
  int* cnt_next;  // [C][NB] bucket sizes being counted for the next evaluation
  int* off;       // [C][NB+1] bucket starts in the global bucket order
  void* rec;      // PtRec<T> [ntot] in bucket order
  void* part;     // T [12][ntot]: per (side, component) u and du partials, bucket order
  double* lk;     // terms of the point likelihood that depend on d only: [6][ntot] doubles
                  // on the FP64 path; on the FP32 path [ntot] doubles then [5][ntot] floats
  long long ntot;
};

// ---- FFT passes (hm_fft_kernels.cu) ----
// Spectrum layout: [x][y][z], z in 0..N/2 (NH = N/2+1 entries), complex.
enum PencilMode : int { PM_FWD = 0, PM_INV = 1, PM_VEL = 2, PM_ADJ = 3, PM_SCALE = 4 };

// Plane-pass inputs/outputs beyond plain arrays.
struct PlanePoints {
  const int* off;       // [C][N*K+1]
  const void* rec;      // PtRec<T>, bucket order
  void* part;           // T [12][ntot]
  long long ntot;
  double inv_delta;     // 1/Delta for the spatial derivative
};

// count grids, real [count][N^3] -> plane-transformed spectra.
cudaError_t launch_plane_r2c(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, cudaStream_t st);
// 3C scatter planes built from the bucketed residuals, then transformed.
cudaError_t launch_plane_r2c_scatter(int prec, int N, const PlanePoints& pts, void* out, long long out_stride,
                                     int count, const void* tw, cudaStream_t st);
// count spectra -> real grids (plain store), or the gradient epilogue; with
// the epilogue and next_spec != nullptr (GM_KICK_DRIFT), the drifted field's
// forward plane transform is written to next_spec for the next evaluation.
cudaError_t launch_plane_c2r(int prec, int N, const void* in, long long in_stride, void* out,
                             long long out_stride, int count, const void* tw, const FieldEpi* epi,
                             cudaStream_t st, void* next_spec = nullptr);
// 3C velocity spectra -> CIC partials of u and du at the bucketed points.
cudaError_t launch_plane_c2r_gather(int prec, int N, const void* in, long long in_stride,
                                    const PlanePoints& pts, int count, const void* tw, cudaStream_t st);
// x-axis pass over count chains.  PM_VEL: 1 spectrum -> 3; PM_ADJ: 3 -> 1;
// PM_SCALE: 1 -> 1, the spectrum times the real table amp[n^2] (the
// colouring sqrt(P/Delta^3)/N^3 of the density field).
// For PM_ADJ, plane_off (the chains' point-bucket offsets, [count][N*K+1])
// marks the x-planes that the scatter plane pass left unwritten because no
// point touches them; they are read as zero.  nullptr reads every plane.
cudaError_t launch_pencil(int prec, int N, int mode, const void* in, long long in_stride, void* out,
                          long long out_stride, int count, const void* tw, const void* amp,
                          cudaStream_t st, const int* plane_off = nullptr);
bool fft_supported(int prec, int N);
// Bounded waits on tensor copies that gave up in the TMA-staged pencil pass
// (FP32, N = 256) on the current device since load (0 in correct
// operation); reset clears it.
int fft_tma_wait_timeouts(bool reset);
// N = 256 plane passes (FP32): a z pass over row slabs and a y pass over
// column tiles (hm_fft_256.cu).  pts == nullptr loads real grids, else
// scatters the bucketed residuals; mode is C2R_STORE (0), C2R_EPI (1) or
// C2R_GATHER (2).  The inverse runs its y pass in place on `in`.
cudaError_t plane256_prepare();
cudaError_t launch_plane_r2c_256(const void* in, long long in_stride, void* out, long long out_stride, int count,
                                 const void* tw, const PlanePoints* pts, cudaStream_t st);
cudaError_t launch_plane_c2r_256(int mode, const void* in, long long in_stride, void* out, long long out_stride,
                                 int count, const void* tw, const FieldEpi* epi, const PlanePoints* pts,
                                 void* next, cudaStream_t st);
// Raise the dynamic shared-memory limit of every FFT kernel for (prec, N) on
// the current device; call once per device before any launch or capture.
cudaError_t fft_prepare(int prec, int N);

// ---- points (hm_points.cu) ----
// bucket counts (x index of the lower corner) of the current distances into pa.cnt
cudaError_t launch_points_prep(int n_chains, int max_pts, const PointParams* pp, PointArrays pa,
                               cudaStream_t st);
// bucket offsets, full cells, bucket-ordered records, and the FP64 terms of
// the likelihood that depend on d alone (distance modulus, observed velocity,
// kappa, prior) with their derivatives; clears pa.cnt_next
cudaError_t launch_points_place(int prec, int n_chains, int max_pts, const PointParams* pp,
                                PointArrays pa, ChainScal* cs, cudaStream_t st);
// u, du from the plane partials, the velocity term, residuals and distance
// gradient, with the Psi partials and the stored gradient except in
// GM_KICK_DRIFT; then (mode != GM_GRAD) the leapfrog update of p_d and d,
// the kinetic partials (GM_KICK_LAST) and the bucket counts of the new
// distances into pa.cnt_next (GM_KICK_DRIFT).  dPsi/dsigma_NL partials in
// every mode when sigma_NL is sampled.
cudaError_t launch_points_lik(int prec, int n_chains, int max_pts, const PointParams* pp, PointArrays pa,
                              double* pts_part, int part_stride, int mode, double* kin_part, ChainScal* cs,
                              double* gsig_part, cudaStream_t st);
int points_blocks(int max_pts);
cudaError_t launch_cells(int n_chains, int max_pts, const PointParams* pp, const double* d,
                         PointArrays pa, int* cell_out, cudaStream_t st);
cudaError_t launch_cell_sort(int N3, long long n, const int* cell, int* perm, int* hist_ws,
                             cudaStream_t st);

// ---- HMC elementwise / scalar kernels (hm_hmc.cu) ----
// draw != 0: fresh momenta from Philox; draw == 0: keep the stored momenta.
cudaError_t launch_traj_begin_field(int prec, int n_chains, long long n3, void* w, void* pw,
                                    const void* gw, void* w0, void* gw0, unsigned long long seed,
                                    const int* chain_id, double* kin_part, int nparts, int draw,
                                    ChainScal* cs, cudaStream_t st);
// also counts the drifted distances into pa.cnt_next (zeroed beforehand)
// Blocks of the trajectory-start kernel of the distances (and slots of its
// kinetic partials) for a catalogue of max_pts points.
int traj_begin_points_blocks(int max_pts);
cudaError_t launch_traj_begin_points(int n_chains, int max_pts, const PointParams* pp,
                                     PointArrays pa, double* d0, double* gd0,
                                     unsigned long long seed, const int* chain_id,
                                     double* kin_part, int nparts, int draw, ChainScal* cs,
                                     cudaStream_t st);
// Set eps and sample_d of every chain from a device array of eps values.
cudaError_t launch_set_run(int n_chains, const double* eps, int sample_d, ChainScal* cs,
                           cudaStream_t st);
cudaError_t launch_finalize(int n_chains, const double* prior_part, int n_prior, const double* pts_part,
                            int n_pts, const double* kin_part, int n_kin, const double* kin_pts_part,
                            int n_kin_pts, int what, unsigned long long seed, const int* chain_id,
                            ChainScal* cs, void* trace_dev, cudaStream_t st);
cudaError_t launch_restore(int prec, int n_chains, long long n3, void* w, void* gw, const void* w0,
                           const void* gw0, int max_pts, const PointParams* pp, PointArrays pa,
                           const double* d0, const double* gd0, const ChainScal* cs,
                           cudaStream_t st);
// sigma_NL: reduce the per-block dPsi/dsigma partials, then (mode) kick and
// drift it; begin: momentum draw (Philox tag 3), save, half kick and drift.
cudaError_t launch_sig_update(int n_chains, const double* gsig_part, int nparts, int mode, ChainScal* cs,
                              cudaStream_t st);
cudaError_t launch_sig_begin(int n_chains, unsigned long long seed, const int* chain_id, int draw, ChainScal* cs,
                             cudaStream_t st);
cudaError_t launch_sig_set(int n_chains, int enable, const double* sig, ChainScal* cs, cudaStream_t st);
// Dual averaging: start (mu = log(10 eps), target delta) / finish (eps = epsbar,
// copied to eps_out[c]) on every chain.
cudaError_t launch_da(int n_chains, int start, double delta, double* eps_out, ChainScal* cs, cudaStream_t st);
cudaError_t launch_philox_raw(unsigned long long seed, long long n, unsigned int c1, unsigned int c2,
                              unsigned int c3, unsigned int* out, cudaStream_t st);

enum FinalizeWhat : int {
  FIN_PSI = 1,       // psi = prior + pts
  FIN_HOLD = 2,      // H_old = psi + kin(begin)
  FIN_ACCEPT = 4,    // H_new, Metropolis test, traj++
  FIN_KIN = 8,       // kin = sum of the kinetic partials given
};


// ---- chain analytics (hm_analytics.cu) ----
constexpr int kMaxShells = 32;   // sphere radii per state
struct AnArgs {
  int C, N, nsh, max_samples, nblk;
  long long n3;
  double delta;              // grid spacing
  double f;                  // growth rate: monopole = a f <delta>, a = 1
  const double* obs;         // [C][3] observer of each chain
  const void* delta_g;       // T [C][n3] density field of the current sample
  const void* vel_g;         // T [C][3][n3] velocity field of the current sample
  void *mean_d, *m2_d, *mean_vr, *m2_vr;   // T [C][n3] Welford mean and M2
  const unsigned char* shell;  // [C][n3] innermost sphere holding the node, 255 for none
  const double* sph_cnt;     // [C][nsh] nodes inside sphere k
  double* sig_part;          // [C][nblk][2] partial sums of delta and delta^2
  double* met_part;          // [C][nblk] partial sums of the metric's squares
  double* shell_part;        // [C][nblk][nsh][4] per-shell sums of delta, v_x, v_y, v_z
  double* sig_prev;          // [C] Sigma of the previous sample
  double* sig_cur;           // [C] Sigma of the current sample
  long long* count;          // [C] samples accumulated
  double* hist;              // [C][max_samples] metric of sample s >= 2 at index s - 2
  double* sph_acc;           // [C][nsh][5][2] Welford mean and M2 over samples of
                             // (monopole, V_x, V_y, V_z, |V|) in sphere k
};
// One sample: sigma partials, node moments and shell sums, per-chain finalize.
cudaError_t launch_analytics(int prec, const AnArgs& a, cudaStream_t st);
// out[i] = in[i] * scale for i < n (field precision prec).
cudaError_t launch_an_scale(int prec, long long n, const void* in, void* out, double scale, cudaStream_t st);

}  // namespace hm
