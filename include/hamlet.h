/* libhamlet -- C ABI of the GB300 HAMLET hot path.
 *
 * HAMLET (Valade, Hoffman & Libeskind) samples the posterior of the linear
 * density field and of the true distances of a peculiar-velocity catalogue
 * with Hamiltonian Monte Carlo.  This library evaluates the potential
 * Psi = -ln(posterior) (eq. Psi) and its gradient on one GPU and runs the
 * leapfrog / Metropolis chain, for one or many chains at once.
 *
 * Conventions (every entry point):
 *  - Units: lengths Mpc/h, velocities km/s, H0 = 100 km/s/(Mpc/h).
 *  - Grid: N^3 nodes at x = (i, j, l) * L/N, periodic, row-major [i][j][l]
 *    (l fastest).  The whitened field w has one real value per node; the
 *    density contrast is delta_k = sqrt(P(k)/Delta^3) DFT(w)_k (eq. prior-k
 *    in whitened form), so the Fourier-mode prior is |w|^2/2.
 *  - Spectra: [kx][ky][kz] complex, kz = 0..N/2, unnormalised forward DFT
 *    with e^{-i k.x}.
 *  - Field arrays are float (HM_FP32) or double (HM_FP64) as the problem's
 *    precision says; distances, momenta of distances and all energies are
 *    double.
 *  - Pointers named *_dev are device pointers on the problem's device
 *    (caller-owned, contiguous); *_host are host pointers (copied in or out
 *    before the call returns, caller keeps ownership).
 *  - Calls are ordered on the given CUDA stream (NULL = legacy default) and
 *    return without synchronising unless stated.
 *  - Return value: HM_OK or a negative HM_E* code; hm_last_error() gives a
 *    text for the calling thread.  No C++ exception crosses this boundary.
 */
#ifndef HAMLET_H
#define HAMLET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HM_OK = 0,
  HM_EINVAL = -1,   /* bad argument: size, NaN, sigma <= 0, unsupported N */
  HM_ENOMEM = -2,   /* device allocation failed */
  HM_ECUDA = -3,    /* a CUDA runtime call failed */
  HM_EDOMAIN = -4,  /* a distance left the prior support: Psi = +inf */
  HM_ESTATE = -5    /* call order: e.g. no catalogue set yet */
};

enum { HM_FP32 = 0, HM_FP64 = 1 };
enum { HM_PRIOR_TABLE = 0, HM_PRIOR_POWER = 1, HM_PRIOR_DZ = 2 };

typedef struct hm_problem hm_problem;
typedef struct hm_state hm_state;

/* Problem description (section "Bayesian posterior PDF and likelihood
 * function"; grid and mock geometry of section "Mock Catalogue
 * construction").  All fields are read once by hm_init_problem. */
typedef struct hm_problem_desc {
  int32_t N;             /* grid nodes per side, power of two (see hm_supported) */
  int32_t precision;     /* HM_FP32 (FP32 fields, FP64 energies) or HM_FP64 */
  double L;              /* box side, Mpc/h */
  double observer[3];    /* observer position; used when observer_set != 0 */
  int32_t observer_set;  /* 0: observer at the box centre (L/2, L/2, L/2) */
  int32_t prior_kind;    /* HM_PRIOR_DZ, HM_PRIOR_TABLE or HM_PRIOR_POWER (eq. D) */
  double omega_m, omega_b, h, n_s, sigma8, T_cmb; /* P(k): Eisenstein-Hu no-wiggle */
  double f_growth;       /* linear growth rate; <= 0 means omega_m^0.55 */
  double sigma_nl;       /* non-linear velocity dispersion sigma_NL, km/s (eq. kappa) */
  /* HM_PRIOR_DZ (section "Priors", eq. D from eq. e:dz), also taken for
   * HM_PRIOR_TABLE with prior_nbins = 0 and no table, so it is the default
   * of a zeroed description: every hm_set_catalog builds the histogram of
   * the redshift distances d_z of the catalogue's observed cz (as
   * hm_dz_prior_table) with bins of prior_bin (<= 0: 5 Mpc/h) on
   * [0, max d_z + prior_pad) (prior_pad <= 0: 3 sigma_v/H0), and the prior
   * is that table (d0 = 0), read as below.
   * HM_PRIOR_TABLE: eq. D's histogram as ln pi_D at the bin centres
   * d0 + (b + 1/2) bin, interpolated linearly between centres (flat in the
   * outer half bins); support [d0, d0 + nbins * bin), -inf outside */
  double prior_d0, prior_bin;
  int32_t prior_nbins;
  int32_t pad0;
  const double* prior_logdens_host;
  /* HM_PRIOR_POWER: ln pi_D(d) = alpha ln d on [dmin, dmax], -inf outside */
  double prior_alpha, prior_dmin, prior_dmax;
  int32_t device;        /* CUDA device ordinal */
  int32_t pad1;
  double prior_pad;      /* HM_PRIOR_DZ: support beyond the largest d_z, Mpc/h */
} hm_problem_desc;

/* Derived constants of a problem (host copy). */
typedef struct hm_problem_info {
  int32_t N, precision;
  int64_t n_points;
  double L, delta, f_growth, sigma_v, minv_d, pk_amplitude;
  int64_t grid_bytes;      /* bytes of one real N^3 field */
  int64_t spectrum_bytes;  /* bytes of one N*N*(N/2+1) complex spectrum */
} hm_problem_info;

/* One record per chain and trajectory written by hm_run_chain. */
typedef struct hm_trace {
  int64_t traj;      /* trajectory counter (Philox counter word 1) */
  double H_old;      /* Hamiltonian at the start (eq. Hamiltonian) */
  double H_new;      /* Hamiltonian at the end point */
  double logu;       /* ln U of the Metropolis test, U in (0, 1] */
  double psi;        /* Psi of the chain state after the decision */
  double eps;        /* leapfrog step used by this trajectory */
  int32_t accept;    /* 1 accepted, 0 rejected */
  int32_t status;    /* bit 1: a distance left the support; bit 2: H not finite */
} hm_trace;

/* 1 if grids of side N at this precision are built into the library. */
int hm_supported(int32_t N, int32_t precision);

/* Create a problem: tabulates P(k) on the grid's |k| values, sigma_v and the
 * velocity operator i aHf k_j/k^2 sqrt(P/Delta^3) (eq. vel-field with the
 * colouring of eq. prior-k).  *out is owned by the library; free with
 * hm_destroy_problem.  Errors: HM_EINVAL, HM_ENOMEM, HM_ECUDA. */
int hm_init_problem(const hm_problem_desc* desc, hm_problem** out);
void hm_destroy_problem(hm_problem* p);
int hm_problem_get_info(const hm_problem* p, hm_problem_info* out);

/* Upload the catalogue (section "Mock Catalogue construction": direction,
 * distance modulus mu with error sigma_mu, redshift cz with error sigma_cz).
 * rhat_host: n x 3 unit vectors (row-major), the direction r_i of eq. lvr;
 * cz_host in km/s (z = cz/c); sigma_cz_host may be NULL (zeros).  Replaces a
 * previous catalogue; with the HM_PRIOR_DZ prior it also rebuilds the
 * distance prior from these redshifts (states and slots made from an
 * earlier catalogue keep that catalogue and its table).  Errors: HM_EINVAL
 * (n < 0, non-finite value, sigma_mu <= 0, |rhat| != 1 beyond 1e-6),
 * HM_ENOMEM. */
int hm_set_catalog(hm_problem* p, int64_t n, const double* rhat_host, const double* mu_host,
                   const double* sigma_mu_host, const double* cz_host, const double* sigma_cz_host);

/* The catalogue in the coordinates the paper states its data in (section
 * "Mock Catalogue construction": supergalactic longitude SGL and latitude
 * SGB in degrees per point, with mu, sigma_mu, cz and sigma_cz as in
 * hm_set_catalog).  The direction of point i is
 * rhat = (cos SGB cos SGL, cos SGB sin SGL, sin SGB) in the grid frame, whose
 * axes are the supergalactic X, Y, Z; otherwise as hm_set_catalog.  Errors:
 * as hm_set_catalog, and HM_EINVAL for SGB outside [-90, 90] or a
 * non-finite angle. */
int hm_set_catalog_sg(hm_problem* p, int64_t n, const double* sgl_deg_host, const double* sgb_deg_host,
                      const double* mu_host, const double* sigma_mu_host, const double* cz_host,
                      const double* sigma_cz_host);

/* Psi(w, d) and its gradient (eqs. covfefe:bay, likelihood, lmu, vrobs,
 * vel-field, lvr, kappa, prior-k, D, Psi).  w_dev: N^3 field; d_dev: n
 * distances.  Outputs: psi_dev (1 double, device), grad_w_dev (N^3 field),
 * grad_d_dev (n doubles).  Psi omits additive constants independent of
 * (w, d).  A distance outside the support gives Psi = +inf, a zero gradient
 * for that point and return code HM_OK (read the status with
 * hm_problem_last_status).  Uses a workspace owned by the problem: calls on
 * one problem must not overlap. */
int hm_logpost_grad(hm_problem* p, const void* w_dev, const double* d_dev, double* psi_dev,
                    void* grad_w_dev, double* grad_d_dev, void* stream);

/* hm_logpost_grad for callers that cannot let the library allocate device
 * memory: code running inside another framework's memory pool, which has to
 * account for every device byte itself, and hosts that budget device memory
 * up front and allow no allocation (nor the device synchronisation that
 * cudaMalloc/cudaFree may cause) once they run.  The paper has no
 * counterpart; this is a deployment variant.  Same arguments, outputs and
 * error behaviour as hm_logpost_grad, and the same kernels, all launched on
 * `stream`; it never calls cudaMalloc, cudaFree or any other allocating
 * routine.  Scratch comes from one static 4 MiB device array that every GPU
 * loading this library keeps until the process exits; a problem needing
 * more (any N > 32; on a 32^3 grid more than about 19,000 points at FP32 or
 * 8,800 at FP64) is rejected with HM_EINVAL and a message naming the sizes.
 * The first call on a device looks up the array's device address with that
 * device current (once per device, also when host threads make their first
 * calls at the same time); make that first call before any stream capture.
 * Every call shares the one array and clears what must start at zero, so
 * calls whose work overlaps on the GPU race: serialise them on one stream or
 * with events. */
int hm_logpost_grad_noalloc(hm_problem* p, const void* w_dev, const double* d_dev, double* psi_dev,
                            void* grad_w_dev, double* grad_d_dev, void* stream);

/* Status bits of the last hm_logpost_grad (synchronises the stream). */
int hm_problem_last_status(hm_problem* p, void* stream, int32_t* status_out);

/* Linear velocity field v_j = IDFT(i aHf k_j/k^2 delta_k) of a whitened
 * field (eq. vel-field): v_dev receives 3 N^3 grids (x, y, z). */
int hm_velocity_field(hm_problem* p, const void* w_dev, void* v_dev, void* stream);

/* Unnormalised 3D real-to-complex DFT of `count` contiguous N^3 grids into
 * `count` spectra, and the inverse complex-to-real DFT (no 1/N^3).  The
 * inverse reads only the half spectrum and treats it as Hermitian. */
int hm_fft_r2c(hm_problem* p, const void* in_dev, void* out_dev, int32_t count, void* stream);
int hm_fft_c2r(hm_problem* p, const void* in_dev, void* out_dev, int32_t count, void* stream);

/* Cell index of each point at distances d_dev: (ix*N + iy)*N + iz of the
 * lower corner of x = o + d rhat (one IEEE rounding per operation), and the
 * stable order of the points by that index (perm_dev may be NULL). */
int hm_cells(hm_problem* p, const double* d_dev, int32_t* cell_dev, int32_t* perm_dev, void* stream);

/* Chains.  A state holds n_chains chains; chain c samples problem
 * problems[chain_problem[c]] (all problems of one state share N and
 * precision).  Chain c draws its random numbers with Philox key `seed` and
 * chain counter word chain_ids[c] (NULL: c).  Positions start at w = 0 and
 * d = d_init_host[c] (n doubles of that chain's problem, host; required when
 * n > 0).  Psi and the gradient are evaluated there before the call returns.
 * Owned by the library; free with hm_destroy_state. */
int hm_state_create(hm_problem* p, uint64_t seed, const double* d_init_host, hm_state** out);
/* (as above for one chain of one problem; chain counter word 0) */
int hm_state_create_batch(hm_problem* const* problems, int32_t n_problems, int32_t n_chains,
                          const int32_t* chain_problem, const int32_t* chain_ids, uint64_t seed,
                          const double* const* d_init_host, hm_state** out);
void hm_destroy_state(hm_state* s);

/* Copy a chain's position (w, d) and/or momenta (p_w, p_d) in or out, as
 * stream-ordered copies.  Each pointer may be device memory or host memory
 * (the copy direction follows from the address under unified addressing);
 * pinned host memory gives asynchronous copies, pageable host memory is
 * staged by the driver.  A host buffer must stay valid until the stream has
 * reached the copy.  NULL leaves that part alone.  After setting positions,
 * hm_state_refresh recomputes Psi and the gradient there. */
int hm_state_set(hm_state* s, int32_t chain, const void* w, const double* d, const void* pw, const double* pd,
                 void* stream);
int hm_state_get(hm_state* s, int32_t chain, void* w, double* d, void* pw, double* pd, void* stream);
/* (the same for the gradient (grad_w, grad_d) at the chain's position) */
int hm_state_get_grad(hm_state* s, int32_t chain, void* gw, double* gd, void* stream);
int hm_state_refresh(hm_state* s, void* stream);
/* Per-chain scalars: Psi at the current position, kinetic energy of the
 * current momenta, trajectory counter (synchronises the stream). */
int hm_state_scalars(hm_state* s, int32_t chain, double* psi, double* kinetic, int64_t* traj,
                     void* stream);
/* Trajectory counter of every chain (for resuming a chain bit-exactly). */
int hm_state_set_traj(hm_state* s, int32_t chain, int64_t traj);

/* n_steps kick-drift-kick leapfrog steps of every chain from its stored
 * momenta (no refresh, no Metropolis test): sections "Hamiltonian
 * trajectories in phase space" and "Integrating the HMC trajectories";
 * eq. hamilton with the mass matrix of eq. M_ab (identity on w,
 * (sigma_v/H0)^2 on d).  sample_distances = 0 holds d fixed. */
int hm_leapfrog(hm_state* s, int32_t n_steps, double eps, int32_t sample_distances, void* stream);

/* n_traj HMC transitions of every chain (section "Construction of HMC
 * chains"): fresh momenta from Philox, n_leapfrog leapfrog steps of size
 * eps_host[c] (one per chain), Metropolis test accept iff ln U < H_old -
 * H_new, restore on rejection.  trace_host receives n_traj * n_chains
 * records (trajectory-major) and the call synchronises the stream at the
 * end; trace_host may be NULL.  use_graph != 0 replays one captured CUDA
 * graph per trajectory. */
int hm_run_chain(hm_state* s, int32_t n_traj, int32_t n_leapfrog, const double* eps_host,
                 int32_t sample_distances, int32_t use_graph, hm_trace* trace_host, void* stream);

/* Slotted states: continuous batching of independent reconstruction jobs
 * of one grid (the HMC transitions of section "Construction of HMC chains",
 * run for many jobs at once; the batching is a serving pattern the paper
 * does not have).  A slotted state holds up to n_slots chains of the grid,
 * precision, box and power spectrum of `templ`, each with room for
 * max_points catalogue points.  Jobs are loaded and released while the
 * others keep running; every trajectory of hm_slots_run advances all loaded
 * chains in the same kernel launches (one captured graph per number of
 * loaded chains).  The loaded chains are packed at indices 0..n_active-1,
 * which hm_state_get/set/get_grad/scalars take as the chain index.  Each
 * chain keeps its own catalogue, step, trajectory counter and Philox chain
 * word, so its samples are those it would draw alone in a one-chain state
 * with the same seed and chain word (up to the order of the atomic scatter
 * additions).  Calls on one slotted state must be ordered on one stream.
 * Device memory is allocated once, at creation (HM_ENOMEM if it does not
 * fit): about 5 grids + 6 half spectra per slot and ~700 B per point of
 * room.  Not available on a slotted state: hm_adapt_step_size (use the
 * per-job adaptation below), the all-chain sigma_NL switch (each job chooses
 * at load) and chain analytics (HM_ESTATE).  hm_state_get_sigma_nl reports
 * each loaded chain's sigma_NL. */
int hm_slots_create(hm_problem* templ, int32_t n_slots, int64_t max_points, uint64_t seed, hm_state** out);
/* Number of loaded chains and of slots. */
int hm_slots_count(hm_state* s, int32_t* n_active_out, int32_t* n_slots_out);
/* Load job `job` (same N, precision, device, box and P(k) as the template;
 * its catalogue, set with hm_set_catalog, is copied; its distance-prior
 * table is read in place, so `job` must outlive the slot) as chain index
 * n_active: w = 0, d = d_init_host (job's n doubles, host), momenta 0,
 * trajectory counter 0, Philox chain word chain_id, step eps0.  With
 * adapt_target in (0, 1) the step adapts by dual averaging after every
 * trajectory (as hm_adapt_step_size) until hm_slots_adapt_end; 0 keeps it
 * fixed.  With sigma_nl0 > 0 the job samples sigma_NL as a chain coordinate
 * (as hm_state_sample_sigma_nl) starting there; 0 keeps the problem's
 * value.  Psi and the gradient of the new chain are evaluated on `stream`.
 * *index_out receives the chain index.  Errors: HM_EINVAL (mismatched job,
 * catalogue larger than a slot, bad eps0 or target, non-finite d),
 * negative sigma_nl0), HM_ESTATE (every slot in use). */
int hm_slots_load(hm_state* s, hm_problem* job, int32_t chain_id, const double* d_init_host, double eps0,
                  double adapt_target, double sigma_nl0, int32_t* index_out, void* stream);
/* End the step adaptation of chain `index`: its step becomes the averaged
 * iterate, copied to *eps_out_host (may be NULL).  Synchronises the stream. */
int hm_slots_adapt_end(hm_state* s, int32_t index, double* eps_out_host, void* stream);
/* Release chain `index` (read its state first with hm_state_get).  The last
 * loaded chain moves into `index`; *moved_from_out (may be NULL) receives
 * its old index, or -1 when none moved.  Stream-ordered. */
int hm_slots_release(hm_state* s, int32_t index, int32_t* moved_from_out, void* stream);
/* n_traj HMC transitions of every loaded chain at its own step (fresh
 * momenta, n_leapfrog leapfrog steps, Metropolis test, restore on
 * rejection).  trace_host (may be NULL) receives n_traj * n_active records,
 * trajectory-major; the call then synchronises the stream.  No loaded chain:
 * nothing runs. */
int hm_slots_run(hm_state* s, int32_t n_traj, int32_t n_leapfrog, int32_t use_graph, hm_trace* trace_host,
                 void* stream);

/* sigma_NL as a sampled parameter (eq. q; section "The Likelihood function:
 * velocities" makes it a model parameter, eq. M_ab gives it unit mass): with
 * enable != 0 every chain carries sigma_NL (starting at sigma0_host[c], or
 * the problem's value when NULL) and its momentum through the leapfrog, with
 * a flat prior on sigma_NL > 0 (the paper states none; sigma_NL <= 0 gives
 * Psi = +inf).  Psi and the gradient are re-evaluated before returning
 * (synchronises the stream).  enable = 0 returns to the problem's fixed
 * value.  hm_state_get_sigma_nl copies each chain's current sigma_NL and
 * dPsi/dsigma_NL (grad_out_host may be NULL; synchronises). */
int hm_state_sample_sigma_nl(hm_state* s, int32_t enable, const double* sigma0_host, void* stream);
int hm_state_get_sigma_nl(hm_state* s, double* sigma_out_host, double* grad_out_host, void* stream);

/* Step-size tuning (section "Integrating the HMC trajectories": the step
 * is tuned to a target acceptance, 0.65 in the paper, by dual averaging):
 * n_warmup HMC transitions of every chain starting from eps0_host[c], the
 * step adapted after each one from its acceptance probability
 * min(1, exp(H_old - H_new)) (Hoffman & Gelman's recursion, gamma = 0.05,
 * t0 = 10, kappa = 0.75, mu = log(10 eps0)); at the end each chain's step
 * is set to the averaged iterate and written to eps_out_host[c].
 * trace_host (may be NULL) receives the n_warmup * n_chains records,
 * including the step each trajectory used.  Synchronises the stream. */
int hm_adapt_step_size(hm_state* s, int32_t n_warmup, int32_t n_leapfrog, double target_accept,
                       const double* eps0_host, int32_t sample_distances, double* eps_out_host,
                       hm_trace* trace_host, void* stream);

/* Chain analytics on the device (eq. int_mc: Monte-Carlo means over chain
 * states; section "Convergence": the convergence monitor; section "Monopole
 * and dipole": velocity moments in spheres about the observer).  With
 * enable != 0, every trajectory of hm_run_chain (not of hm_adapt_step_size)
 * adds one sample per chain, the chain state after its Metropolis test:
 *   - running mean and variance (divisor n - 1) at every grid node of the
 *     density field delta = IDFT(sqrt(P/Delta^3) DFT(w)) and of the radial
 *     velocity v_r = rhat . v (rhat from the observer to the node; 0 on it);
 *   - for samples s >= 2, the root mean square over the nodes of
 *     m_s/Sigma_s - m_{s-1}/Sigma_{s-1} (m_s the running mean of delta after s
 *     samples, Sigma_s^2 the variance over the grid of sample s's delta), the
 *     first max_samples values kept;
 *   - in each sphere |x - o| <= radii_host[k] (n_radii <= 32, increasing,
 *     nodes at x = i*Delta, no periodic wrap): the monopole a f <delta>
 *     (= the mean of -div v/H0 by linear continuity, a = 1), the mean velocity
 *     V (dipole) and |V|, with their mean and variance over samples.
 * enable != 0 allocates and zeroes the accumulators (about 8 field-sized
 * arrays per chain; HM_ENOMEM when they do not fit), enable = 0 frees them.
 * Both synchronise the stream.  Errors: HM_EINVAL for bad radii or sizes. */
int hm_state_analytics(hm_state* s, int32_t enable, int32_t n_radii, const double* radii_host,
                       int32_t max_samples, void* stream);

/* Read the analytics of one chain.  Device outputs (field precision, layout
 * [x][y][z], may be NULL): mean and variance of delta and of v_r.  Host
 * outputs (may be NULL): metric_host[0 .. min(n-1, max_samples, max_metric))
 * the convergence values of samples 2, 3, ...; sphere_host[k][q][2] for the
 * n_radii spheres and q = monopole, V_x, V_y, V_z, |V|: mean and variance over
 * samples; *n_samples_out the sample count n.  Synchronises the stream.
 * Errors: HM_ESTATE when analytics are off, HM_EINVAL for a bad chain. */
int hm_state_analytics_read(hm_state* s, int32_t chain, void* mean_delta_dev, void* var_delta_dev,
                            void* mean_vr_dev, void* var_vr_dev, double* metric_host, int32_t max_metric,
                            double* sphere_host, int64_t* n_samples_out, void* stream);

/* Per-kernel timing of hm_run_chain: with profiling enabled, every kernel
 * launch of a trajectory is bracketed by a pair of CUDA events on the
 * launching stream (recorded as graph nodes when the trajectory is
 * replayed as a graph).  A run of several trajectories synchronises after
 * each one to accumulate the elapsed times per kernel kind; a run of one
 * trajectory returns without synchronising and leaves its events pending
 * until hm_state_profile_collect (which synchronises the stream the
 * trajectory ran on), the next run_chain or hm_state_profile_read.
 * enable != 0 on a profiled state resets the totals; enable = 0 frees the
 * events (and a trajectory graph captured with them).
 * hm_state_profile_read fills ms_out[k] (total milliseconds) and
 * launches_out[k] for k < min(max_kinds, *n_kinds); kind names come from
 * hm_kernel_kind_name (empty string for an unknown kind).  Errors:
 * HM_ESTATE when profiling is off. */
int hm_state_profile(hm_state* s, int32_t enable);
int hm_state_profile_collect(hm_state* s);
int hm_state_profile_read(hm_state* s, int32_t max_kinds, double* ms_out, int64_t* launches_out,
                          int32_t* n_kinds);
const char* hm_kernel_kind_name(int32_t kind);

/* The distance prior of eq. D from the observed redshifts (host only, no
 * device work): d_z of each cz_host[i]/c by eq. e:dz (flat LCDM, composite
 * Simpson with 64 intervals), histogram on [0, max d_z + pad) in bins of
 * bin_width, each count + 0.5, normalised to a density; logdens_out[b] =
 * ln density (the table of hm_problem_desc, d0 = 0).  *nbins_out receives
 * the bin count; with logdens_out NULL or max_bins too small only the count
 * is returned (HM_EINVAL in the latter case). */
int hm_dz_prior_table(double omega_m, int64_t n, const double* cz_host, double bin_width, double pad,
                      int32_t max_bins, double* logdens_out, int32_t* nbins_out);

/* The problem's distance-prior table (eq. D) as the device reads it: ln pi_D
 * at the bin centres d0 + (b + 1/2) bin for b < *nbins_out (host copies;
 * d0_out, bin_out and logdens_out may be NULL; with logdens_out NULL only
 * the sizes are returned).  For HM_PRIOR_DZ this is the histogram built by
 * the last hm_set_catalog (0 bins before any catalogue).  Errors: HM_ESTATE
 * for a power-law prior, HM_EINVAL when max_bins is too small. */
int hm_problem_prior_table(const hm_problem* p, int32_t max_bins, double* logdens_out, int32_t* nbins_out,
                           double* d0_out, double* bin_out);

/* Number of bounded device waits that gave up on `device` since the library
 * loaded (the x pass at FP32 N = 256 waits for tensor copies of its next
 * tile; a wait that never completes is abandoned after a fixed number
 * of polls, the CTA returns and the count grows).  0 in correct operation; a
 * positive count means the results since then are not to be trusted.
 * reset != 0 clears it.  Synchronises the device.  Not from the paper: a
 * fault check of this implementation. */
int hm_device_wait_timeouts(int32_t device, int32_t reset, int32_t* count_out);

/* Raw Philox-4x32-10 blocks for counters (q, c1, c2, c3), q = 0..n-1, key
 * seed: out_dev receives 4 n uint32 words. */
int hm_philox(uint64_t seed, int64_t n, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t* out_dev,
              void* stream);

/* Text of the last error on the calling thread ("" if none). */
const char* hm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HAMLET_H */
