// Host side of libhamlet: problem and chain-state objects, the tables of the
// linear velocity operator, the order of the kernel launches of one gradient
// evaluation and of one HMC trajectory, and the C ABI of include/hamlet.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "hamlet.h"
#include "hm_internal.h"

using namespace hm;

namespace hm {
bool pdl_enabled(int cat) {
  static const int mask = [] {
    // default: the x pencils and the per-trajectory kernels (measured on the
    // 128^3 trajectory: pencils 1.725 ms, none 1.750, plane passes 1.887,
    // point kernels 2.047, all 2.312; later, pencils 1.650 vs pencils and
    // per-trajectory kernels 1.648, and 19.92 vs 19.85 ms for 32 chains)
    const char* e = std::getenv("HM_PDL");
    return e ? std::atoi(e) : (int)(PDL_PENCIL | PDL_OTHER);
  }();
  return (mask & cat) != 0;
}
}  // namespace hm

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define HM_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

#define HM_TRY(call)            \
  do {                          \
    int r_ = (call);            \
    if (r_ != HM_OK) return r_; \
  } while (0)

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  int alloc(size_t n) {
    release();
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? HM_ENOMEM : HM_ECUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    bytes = n;
    return HM_OK;
  }
  template <typename X> X* as() const { return static_cast<X*>(p); }
};

// ---------------------------------------------------------------------------
// per-kernel event timing of the trajectory launches (stream or graph)
// ---------------------------------------------------------------------------
enum KernelKind : int {
  KK_R2C_FIELD = 0, KK_PENCIL_VEL, KK_C2R_GATHER, KK_MEMSET_CNT, KK_PREP, KK_PLACE, KK_LIK,
  KK_R2C_SCATTER, KK_PENCIL_ADJ, KK_C2R_GRAD, KK_BEGIN, KK_FINALIZE, KK_RESTORE, KK_COUNT
};
static const char* kKindNames[KK_COUNT] = {
    "plane_r2c_field", "pencil_velocity", "plane_c2r_velocity_gather", "memset_bucket_counts",
    "points_bucket_count_standalone",
    "points_bucket_place", "points_likelihood_kick", "plane_r2c_scatter_adjoint", "pencil_adjoint",
    "plane_c2r_gradient_kick", "trajectory_begin", "finalize_energy",
    "restore_rejected"};

struct Prof {
  std::vector<cudaEvent_t> ev;
  std::vector<int> kind;
  int idx = 0;
  bool overflow = false;
  double ms[KK_COUNT] = {0};
  long long launches[KK_COUNT] = {0};
  ~Prof() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  int reserve(int pairs) {
    while ((int)ev.size() < 2 * pairs) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return fail(HM_ECUDA, "cudaEventCreate failed");
      ev.push_back(e);
    }
    kind.resize(pairs);
    return HM_OK;
  }
  static cudaError_t rec(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, st, cudaEventRecordExternal)
                                                : cudaEventRecord(e, st);
  }
  cudaError_t begin(int k, cudaStream_t st) {
    if (2 * idx + 1 >= (int)ev.size()) {
      overflow = true;
      return cudaSuccess;
    }
    kind[idx] = k;
    return rec(ev[2 * idx], st);
  }
  cudaError_t end(cudaStream_t st) {
    if (2 * idx + 1 >= (int)ev.size()) return cudaSuccess;
    cudaError_t e = rec(ev[2 * idx + 1], st);
    ++idx;
    return e;
  }
  // after the recorded work has completed
  int collect(int n_pairs) {
    for (int i = 0; i < n_pairs; ++i) {
      float t = 0.f;
      cudaError_t e = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      if (e != cudaSuccess) return fail(HM_ECUDA, std::string("cudaEventElapsedTime: ") + cudaGetErrorString(e));
      ms[kind[i]] += t;
      launches[kind[i]] += 1;
    }
    return HM_OK;
  }
};

#define HM_PROF(prof, k, st, call)                \
  do {                                           \
    if (prof) HM_CUDA((prof)->begin((k), (st))); \
    HM_CUDA(call);                               \
    if (prof) HM_CUDA((prof)->end((st)));        \
  } while (0)

// ---------------------------------------------------------------------------
// linear power spectrum (Eisenstein & Hu 1998 no-wiggle), sigma8 and sigma_v
// ---------------------------------------------------------------------------
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kE = 2.71828182845904523536;

struct EH {
  double om, ob, h, ns, Tcmb;
  double A = 1.0;
  // EH98 eqs. 26 and 28-31 (k in h/Mpc)
  double transfer(double k) const {
    const double omh2 = om * h * h, obh2 = ob * h * h, fb = ob / om, th = Tcmb / 2.7;
    const double s = 44.5 * std::log(9.83 / omh2) / std::sqrt(1.0 + 10.0 * std::pow(obh2, 0.75));
    const double ag = 1.0 - 0.328 * std::log(431.0 * omh2) * fb + 0.38 * std::log(22.3 * omh2) * fb * fb;
    const double x = 0.43 * k * h * s;
    const double geff = om * h * (ag + (1.0 - ag) / (1.0 + x * x * x * x));
    const double q = k * th * th / geff;
    const double L0 = std::log(2.0 * kE + 1.8 * q);
    const double C0 = 14.2 + 731.0 / (1.0 + 62.5 * q);
    return L0 / (L0 + C0 * q * q);
  }
  double pk(double k) const {
    const double T = transfer(k);
    return A * std::pow(k, ns) * T * T;
  }
};

// composite Simpson rule in ln k on [1e-5, 1e2] h/Mpc with 16384 intervals
template <typename F> double simpson_lnk(F f) {
  const int n = 16384;
  const double a = std::log(1e-5), b = std::log(1e2);
  const double hstep = (b - a) / n;
  double s = 0.0;
  for (int i = 0; i <= n; ++i) {
    const double lk = a + (b - a) * i / n;
    const double wgt = (i == 0 || i == n) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
    s += wgt * f(std::exp(lk));
  }
  return s * hstep / 3.0;
}

double tophat(double x) { return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x); }

}  // namespace

// ---------------------------------------------------------------------------
// objects
// ---------------------------------------------------------------------------
// Per-evaluation point workspace (bucketing, records, partials) and the
// side stream on which the bucketing overlaps the first FFT passes.
struct PtWork {
  DevBuf cx, slot, pos, cnt, off, rec, part, lk;
  int CN = 0;          // C*NB: each count half holds CN ints (ping-pong)
  int OH = 0;          // C*(NB+1): ints in each offset half
  size_t recsz = 0;    // bytes of one point record
  long long nt = 1;    // records per half
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  ~PtWork() {
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
    if (aux) cudaStreamDestroy(aux);
  }
  int alloc(int prec, int C, int N, long long ntot) {
    N *= plane_split(N);   // sub-buckets per chain
    nt = std::max<long long>(ntot, 1);
    const size_t rsz = prec == HM_FP32 ? 4 : 8;
    recsz = prec == HM_FP32 ? sizeof(PtRec<float>) : sizeof(PtRec<double>);
    HM_TRY(cx.alloc(4 * nt));
    HM_TRY(slot.alloc(4 * nt));
    HM_TRY(pos.alloc(4 * nt));
    HM_TRY(cnt.alloc(4 * 2 * (size_t)C * N));
    HM_TRY(off.alloc(4 * 2 * (size_t)C * (N + 1)));
    HM_TRY(rec.alloc(2 * recsz * nt));
    HM_TRY(part.alloc(rsz * 12 * nt));
    HM_TRY(lk.alloc(8 * 6 * nt));
    CN = C * N;
    OH = C * (N + 1);
    if (cudaMemset(cnt.p, 0, 4 * 2 * (size_t)C * N) != cudaSuccess) return fail(HM_ECUDA, "cudaMemset failed");
    if (!aux) {
      if (cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess)
        return fail(HM_ECUDA, "stream/event creation failed");
    }
    return HM_OK;
  }
  int* half(int parity) const { return cnt.as<int>() + (size_t)(parity & 1) * CN; }
  // Buffers of evaluation parity `parity`: counts of its distances (cnt),
  // the other count half (cnt_next), and its records and offsets.
  void fill(PointArrays& pa, long long ntot, int parity = 0) const {
    pa.cx = cx.as<int>();
    pa.slot = slot.as<int>();
    pa.pos = pos.as<int>();
    pa.cnt = half(parity);
    pa.cnt_next = half(parity + 1);
    pa.off = off.as<int>() + (size_t)(parity & 1) * OH;
    pa.rec = static_cast<char*>(rec.p) + (size_t)(parity & 1) * recsz * nt;
    pa.part = part.p;
    pa.lk = lk.as<double>();
    pa.ntot = ntot;
  }
};

struct hm_problem {
  hm_problem_desc desc{};
  int N = 0, prec = 0, device = 0;
  double L = 0, delta = 0, obs[3] = {0, 0, 0};
  double f = 0, aHf = 0, sigma_v = 0, minv_d = 0, pkA = 0;
  size_t rsz = 4;            // bytes of one real
  long long n3 = 0, nspec = 0;
  DevBuf tw, amp, ampd, prior_logdens;   // ampd: colouring sqrt(P/Delta^3)/N^3 per n^2
  std::vector<double> prior_host;
  // eq. D from the observed redshifts: rebuilt by every hm_set_catalog; the
  // tables of earlier catalogues stay allocated (states and slots made from
  // them keep reading theirs) until the problem is destroyed
  bool prior_dz = false;
  double dz_bin = 0, dz_pad = 0;
  std::vector<std::unique_ptr<DevBuf>> prior_retired;
  // catalogue
  long long n = 0;
  DevBuf rx, ry, rz, mu, smu, zobs, scz;
  DevBuf xr;   // XRef per point: the FP32 path's constants of its distance terms
  // standalone workspace (one chain)
  DevBuf S1, S2, hist, prior_part, pts_part, kin_part, pp, cs, chain_id;
  PtWork pw;
  long long ws_points = -1;
};

struct hm_state {
  int C = 0, N = 0, prec = 0, device = 0;
  int NP = 0;    // plane-pass partial sums per chain: N planes * CTAs per plane
  long long n3 = 0, nspec = 0, ntot = 0;
  int max_pts = 0, pts_blocks = 1;
  int nparts_f = 1, nparts_p = 1;
  unsigned long long seed = 0;
  size_t rsz = 4;
  hm_problem* p0 = nullptr;       // problem providing the tables (same N, prec)
  std::vector<hm_problem*> chain_prob;
  DevBuf w, pw, gw, w0, gw0, S1, S2;
  DevBuf rx, ry, rz, mu, smu, zobs, scz, d, pd, gd, d0, gd0;
  DevBuf xr;
  PtWork work;
  DevBuf prior_part, pts_part, kinb_f, kinb_p, kinl_f, kinl_p;
  DevBuf pp, cs, chain_id, eps_dev, trace_dev, gsig_part, sig_dev;
  bool sample_sig = false;
  size_t trace_cap = 0;
  std::vector<PointParams> pp_host;
  std::vector<double> eps_host;
  std::unique_ptr<Prof> prof;
  int prof_pairs = 0;      // event pairs recorded by one trajectory
  int prof_pending = 0;    // pairs recorded by the last single-trajectory run, not yet read
  cudaStream_t prof_stream = nullptr;
  // chain analytics (one sample per trajectory when on)
  struct Analytics {
    bool on = false;
    int nsh = 0, max_samples = 0, nblk = 1;
    std::vector<double> radii;
    DevBuf delta_g, vel_g, mean_d, m2_d, mean_vr, m2_vr, shell, sph_cnt, sig_part, met_part, shell_part;
    DevBuf sig_prev, sig_cur, count, hist, sph_acc, obs;
  } an;
  // captured trajectory graphs, one per (active chains, leapfrog steps,
  // distances sampled, profiled); a slotted state changes its active count
  struct Graph {
    int C, L, sd, prof, pairs;
    cudaGraphExec_t exec;
  };
  std::vector<Graph> graphs;
  cudaStream_t gstream = nullptr;
  // slotted state (continuous batching): capacity, point room per slot,
  // point region of each active chain, free regions
  int C_cap = 0;
  bool slotted = false;
  long long slot_pts = 0;
  std::vector<int> region_of;
  std::vector<int> free_regions;
  void drop_graphs(bool profiled_only = false) {
    for (size_t k = 0; k < graphs.size();) {
      if (!profiled_only || graphs[k].prof) {
        cudaGraphExecDestroy(graphs[k].exec);
        graphs.erase(graphs.begin() + (long)k);
      } else {
        ++k;
      }
    }
  }
  ~hm_state() {
    drop_graphs();
    if (gstream) cudaStreamDestroy(gstream);
  }
};

static PointArrays point_arrays(hm_state* s) {
  PointArrays pa{};
  pa.rx = s->rx.as<double>();
  pa.ry = s->ry.as<double>();
  pa.rz = s->rz.as<double>();
  pa.mu = s->mu.as<double>();
  pa.xr = s->xr.as<XRef>();
  pa.ismu2 = s->smu.as<double>();
  pa.zobs = s->zobs.as<double>();
  pa.scz = s->scz.as<double>();
  pa.d = s->d.as<double>();
  pa.pd = s->pd.as<double>();
  pa.gd = s->gd.as<double>();
  s->work.fill(pa, s->ntot);
  return pa;
}

static PointParams point_params(const hm_problem* p, long long off) {
  PointParams P{};
  for (int j = 0; j < 3; ++j) P.obs[j] = p->obs[j];
  P.delta = p->delta;
  P.inv_delta = 1.0 / p->delta;
  for (int j = 0; j < 3; ++j) {
    P.obs_hi[j] = (float)P.obs[j];
    P.obs_lo[j] = (float)(P.obs[j] - (double)P.obs_hi[j]);
  }
  P.inv_delta_hi = (float)P.inv_delta;
  P.inv_delta_lo = (float)(P.inv_delta - (double)P.inv_delta_hi);
  P.omega_m = p->desc.omega_m;
  P.h = p->desc.h;
  P.sigma_nl2 = p->desc.sigma_nl * p->desc.sigma_nl;
  P.ik2_nl = 1.0 / P.sigma_nl2;
  P.logk2_nl = std::log(P.sigma_nl2);
  P.minv_d = p->minv_d;
  P.k3 = 3.0 * p->desc.omega_m * kH0 / kC;
  P.c23 = 2.0 / (3.0 * p->desc.omega_m);
  P.inv_h = 1.0 / p->desc.h;
  P.c23k3_f = (float)(P.c23 * P.k3);
  P.inv_h_f = (float)P.inv_h;
  P.k3_f = (float)P.k3;
  P.N = p->N;
  P.ksplit = plane_split(p->N);
  P.rq = p->N / P.ksplit;
  P.prior_kind = p->desc.prior_kind;
  P.prior_nbins = p->desc.prior_nbins;
  P.prior_d0 = p->desc.prior_d0;
  P.prior_bin = p->desc.prior_bin;
  P.prior_logdens = p->prior_logdens.as<double>();
  P.prior_alpha = p->desc.prior_alpha;
  P.prior_dmin = p->desc.prior_dmin;
  P.prior_dmax = p->desc.prior_dmax;
  P.pt_off = off;
  P.pt_n = p->n;
  return P;
}

// ---------------------------------------------------------------------------
// one gradient evaluation of C chains (forward operator, likelihood, adjoint)
// ---------------------------------------------------------------------------
struct GradArgs {
  int prec, N, C;
  long long n3, nspec;
  double delta;
  const void* tw;
  const void* amp;
  void *w, *pw, *gw;
  void *S1, *S2;
  PointArrays pa;
  const PointParams* pp;
  int max_pts, pts_blocks;
  double *prior_part, *pts_part, *kinl_f, *kinl_p;
  ChainScal* cs;
  const PtWork* work;
  Prof* prof;
  double* gsig_part;   // [C][pts_blocks] dPsi/dsigma_NL partials (sampled sigma_NL)
  bool sample_sig;
};

// The gradient evaluations of a leapfrog run (or one standalone evaluation)
// for C chains.  Streams: the side stream `aux` places the points of
// evaluation l+1 into x-plane buckets (and evaluates the likelihood terms
// that depend on d alone) while the main stream finishes evaluation l (its
// adjoint, or for one chain its gradient epilogue); the main stream of
// evaluation l is
//   [plane r2c of w] -> x pencils with the velocity weights -> plane c2r with
//   the CIC gather -> likelihood (+ distance kick/drift, next buckets) ->
//   plane CIC scatter + r2c -> x pencils with the adjoint weights -> plane
//   c2r with the field kick/drift (+ plane r2c of the drifted field).
// Precondition: the bucket counts of the current distances are in count
// half 0.  Evaluation l uses parity (l-1)&1 for counts, records, offsets.
static int place_points(const GradArgs& a, int parity, cudaStream_t st) {
  const PtWork& wk = *a.work;
  PointArrays pa = a.pa;
  wk.fill(pa, a.pa.ntot, parity);
  HM_CUDA(cudaEventRecord(wk.fork, st));
  HM_CUDA(cudaStreamWaitEvent(wk.aux, wk.fork, 0));
  HM_PROF(a.prof, KK_PLACE, wk.aux, launch_points_place(a.prec, a.C, a.max_pts, a.pp, pa, a.cs, wk.aux));
  HM_CUDA(cudaEventRecord(wk.join, wk.aux));
  return HM_OK;
}

static int eval_run(const GradArgs& a, int n, int last_mode, cudaStream_t st) {
  Prof* pf = a.prof;
  const PtWork& wk = *a.work;
  HM_TRY(place_points(a, 0, st));
  bool have_spec = false;
  for (int l = 1; l <= n; ++l) {
    const int par = (l - 1) & 1;
    const int mode = l < n ? GM_KICK_DRIFT : last_mode;
    PointArrays pa = a.pa;
    wk.fill(pa, a.pa.ntot, par);
    PlanePoints pts{};
    pts.off = pa.off;
    pts.rec = pa.rec;
    pts.part = pa.part;
    pts.ntot = pa.ntot;
    pts.inv_delta = 1.0 / a.delta;
    // forward field operator
    if (!have_spec)
      HM_PROF(pf, KK_R2C_FIELD, st, launch_plane_r2c(a.prec, a.N, a.w, a.n3, a.S1, a.nspec, a.C, a.tw, st));
    HM_PROF(pf, KK_PENCIL_VEL, st,
            launch_pencil(a.prec, a.N, PM_VEL, a.S1, a.nspec, a.S2, a.nspec, a.C, a.tw, a.amp, st));
    HM_CUDA(cudaStreamWaitEvent(st, wk.join, 0));   // buckets of this evaluation placed
    HM_PROF(pf, KK_C2R_GATHER, st, launch_plane_c2r_gather(a.prec, a.N, a.S2, a.nspec, pts, 3 * a.C, a.tw, st));
    HM_PROF(pf, KK_LIK, st,
            launch_points_lik(a.prec, a.C, a.max_pts, a.pp, pa, a.pts_part, a.pts_blocks, mode, a.kinl_p, a.cs,
                              a.gsig_part, st));
    if (a.sample_sig) HM_CUDA(launch_sig_update(a.C, a.gsig_part, a.pts_blocks, mode, a.cs, st));
    // next evaluation's buckets, off the critical path: forked right after
    // the likelihood for several chains; for one chain up to 128^3 after the
    // adjoint pencils, so that it runs beside the gradient epilogue and the
    // velocity pencils instead of taking SMs from the scatter pass (measured
    // on one box: plain 128^3 trajectory 1.690 -> 1.658 ms, 32-chain batch
    // 20.07 -> 20.18 ms, 256^3 unchanged)
    const bool late_fork = a.C == 1 && a.N <= 128;
    if (l < n && !late_fork) HM_TRY(place_points(a, par ^ 1, st));
    // adjoint: residuals scattered plane by plane, forward transform, weights
    HM_PROF(pf, KK_R2C_SCATTER, st, launch_plane_r2c_scatter(a.prec, a.N, pts, a.S1, a.nspec, 3 * a.C, a.tw, st));
    HM_PROF(pf, KK_PENCIL_ADJ, st,
            launch_pencil(a.prec, a.N, PM_ADJ, a.S1, a.nspec, a.S2, a.nspec, a.C, a.tw, a.amp, st, pts.off));
    if (l < n && late_fork) HM_TRY(place_points(a, par ^ 1, st));
    FieldEpi epi{};
    epi.w = a.w;
    epi.pw = a.pw;
    epi.gw = a.gw;
    epi.prior_part = a.prior_part;
    epi.kin_part = a.kinl_f;
    epi.cs = a.cs;
    epi.grid_stride = a.n3;
    epi.mode = mode;
    void* next = (mode == GM_KICK_DRIFT) ? a.S1 : nullptr;   // S1 is free after the adjoint pencils
    HM_PROF(pf, KK_C2R_GRAD, st,
            launch_plane_c2r(a.prec, a.N, a.S2, a.nspec, nullptr, 0, a.C, a.tw, &epi, st, next));
    have_spec = next != nullptr;
  }
  return HM_OK;
}

// One standalone evaluation (no leapfrog update): bucket counts first.
static int eval_single(const GradArgs& a, cudaStream_t st) {
  PointArrays pa = a.pa;
  a.work->fill(pa, a.pa.ntot, 0);
  HM_PROF(a.prof, KK_MEMSET_CNT, st, cudaMemsetAsync(pa.cnt, 0, sizeof(int) * (size_t)a.work->CN, st));
  HM_PROF(a.prof, KK_PREP, st, launch_points_prep(a.C, a.max_pts, a.pp, pa, st));
  return eval_run(a, 1, GM_GRAD, st);
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* hm_last_error(void) { return g_err.c_str(); }

int hm_supported(int32_t N, int32_t precision) { return fft_supported(precision, N) ? 1 : 0; }

static int check_finite(const double* x, long long n, const char* what) {
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return fail(HM_EINVAL, std::string(what) + " has a non-finite value");
  return HM_OK;
}

// eq. D's histogram from eq. e:dz: d_z of each cz/c (flat LCDM, composite
// Simpson with 64 intervals on [0, z]), bins of bin_width on [0, max d_z +
// pad), count + 0.5 per bin, normalised to a density; ln density per bin.
static std::vector<double> dz_histogram(double omega_m, long long n, const double* cz, double bin_width,
                                        double pad) {
  auto dz = [&](double z) {
    const int m = 64;
    double s = 0.0;
    for (int i = 0; i <= m; ++i) {
      const double x = z * i / m;
      const double f = 1.0 / std::sqrt(omega_m * (1.0 + x) * (1.0 + x) * (1.0 + x) + 1.0 - omega_m);
      s += ((i == 0 || i == m) ? 1.0 : ((i & 1) ? 4.0 : 2.0)) * f;
    }
    return kC / kH0 * (z / m) / 3.0 * s;
  };
  std::vector<double> d(n);
  double dmax = 0.0;
  for (long long i = 0; i < n; ++i) {
    d[i] = dz(std::max(cz[i], 0.0) / kC);
    dmax = std::max(dmax, d[i]);
  }
  const long long nb = (long long)std::ceil((dmax + pad) / bin_width);
  std::vector<double> cnt(nb, 0.0), out(nb);
  for (long long i = 0; i < n; ++i) cnt[std::min<long long>((long long)(d[i] / bin_width), nb - 1)] += 1.0;
  double tot = 0.0;
  for (long long b = 0; b < nb; ++b) tot += cnt[b] + 0.5;
  for (long long b = 0; b < nb; ++b) out[b] = std::log((cnt[b] + 0.5) / (tot * bin_width));
  return out;
}

int hm_init_problem(const hm_problem_desc* desc, hm_problem** out) {
  if (!desc || !out) return fail(HM_EINVAL, "null argument");
  *out = nullptr;
  const hm_problem_desc& d = *desc;
  if (d.precision != HM_FP32 && d.precision != HM_FP64) return fail(HM_EINVAL, "precision must be HM_FP32 or HM_FP64");
  if (!fft_supported(d.precision, d.N)) return fail(HM_EINVAL, "unsupported grid size N for this precision");
  if (d.N * plane_split(d.N) >= kMaxBuckets) return fail(HM_EINVAL, "too many point buckets per chain for this N");
  if (!(d.L > 0) || !(d.omega_m > 0) || !(d.omega_b > 0) || !(d.h > 0) || !(d.sigma8 > 0) ||
      !(d.T_cmb > 0) || !std::isfinite(d.n_s) || !(d.sigma_nl >= 0))
    return fail(HM_EINVAL, "bad cosmology or box parameters");
  // a table kind without a table is the default: eq. D from the redshifts
  const bool dz_prior = d.prior_kind == HM_PRIOR_DZ ||
                        (d.prior_kind == HM_PRIOR_TABLE && d.prior_nbins == 0 && !d.prior_logdens_host);
  if (dz_prior) {
    if (d.prior_bin < 0 || !std::isfinite(d.prior_bin) || d.prior_pad < 0 || !std::isfinite(d.prior_pad))
      return fail(HM_EINVAL, "redshift-distance prior needs prior_bin >= 0 and prior_pad >= 0");
  } else if (d.prior_kind == HM_PRIOR_TABLE) {
    if (d.prior_nbins <= 0 || !d.prior_logdens_host || !(d.prior_bin > 0))
      return fail(HM_EINVAL, "table prior needs prior_nbins > 0, prior_bin > 0 and prior_logdens_host");
  } else if (d.prior_kind == HM_PRIOR_POWER) {
    if (!(d.prior_dmax > d.prior_dmin)) return fail(HM_EINVAL, "power prior needs dmax > dmin");
  } else {
    return fail(HM_EINVAL, "unknown prior_kind");
  }
  HM_CUDA(cudaSetDevice(d.device));
  auto p = std::make_unique<hm_problem>();
  p->desc = d;
  p->N = d.N;
  p->prec = d.precision;
  p->device = d.device;
  p->L = d.L;
  p->delta = d.L / d.N;
  for (int j = 0; j < 3; ++j) p->obs[j] = d.observer_set ? d.observer[j] : 0.5 * d.L;
  p->rsz = d.precision == HM_FP32 ? 4 : 8;
  p->n3 = (long long)d.N * d.N * d.N;
  p->nspec = (long long)d.N * d.N * (d.N / 2 + 1);
  // power spectrum normalised to sigma8 (top-hat R = 8 Mpc/h), sigma_v
  EH eh{d.omega_m, d.omega_b, d.h, d.n_s, d.T_cmb};
  const double s2 = simpson_lnk([&](double k) {
                      const double W = tophat(8.0 * k);
                      return k * k * k * eh.pk(k) * W * W;
                    }) / (2.0 * kPi * kPi);
  eh.A = d.sigma8 * d.sigma8 / s2;
  p->pkA = eh.A;
  p->f = d.f_growth > 0 ? d.f_growth : std::pow(d.omega_m, 0.55);
  p->aHf = 1.0 * kH0 * p->f;
  const double Iv = simpson_lnk([&](double k) { return k * eh.pk(k); });
  p->sigma_v = std::sqrt((kH0 * p->f) * (kH0 * p->f) * Iv / (6.0 * kPi * kPi));
  p->minv_d = (p->sigma_v / kH0) * (p->sigma_v / kH0);
  // amp[n2] = (2 pi/L) aHf sqrt(P/Delta^3) / (k^2 N^3): velocity weights with
  // the 1/N^3 of the inverse DFT folded in
  const int N = d.N;
  const int nmax = 3 * (N / 2) * (N / 2);
  std::vector<double> ampd(nmax + 1, 0.0), colour(nmax + 1, 0.0);
  const double kf = 2.0 * kPi / d.L;
  const double d3 = p->delta * p->delta * p->delta;
  const double n3d = (double)N * N * N;
  for (int n2 = 1; n2 <= nmax; ++n2) {
    const double k = kf * std::sqrt((double)n2);
    ampd[n2] = kf * p->aHf * std::sqrt(eh.pk(k) / d3) / (k * k * n3d);
    colour[n2] = std::sqrt(eh.pk(k) / d3) / n3d;   // density field: delta = IDFT(sqrt(P/Delta^3) DFT(w))
  }
  std::vector<double> twd(2 * N);
  for (int e = 0; e < N; ++e) {
    twd[2 * e] = std::cos(2.0 * kPi * e / N);
    twd[2 * e + 1] = -std::sin(2.0 * kPi * e / N);
  }
  if (p->prec == HM_FP32) {
    std::vector<float> af(ampd.begin(), ampd.end()), tf(twd.begin(), twd.end());
    std::vector<float> cf(colour.begin(), colour.end());
    HM_TRY(p->amp.alloc(af.size() * 4));
    HM_CUDA(cudaMemcpy(p->amp.p, af.data(), af.size() * 4, cudaMemcpyHostToDevice));
    HM_TRY(p->ampd.alloc(cf.size() * 4));
    HM_CUDA(cudaMemcpy(p->ampd.p, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice));
    HM_TRY(p->tw.alloc(tf.size() * 4));
    HM_CUDA(cudaMemcpy(p->tw.p, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice));
  } else {
    HM_TRY(p->amp.alloc(ampd.size() * 8));
    HM_CUDA(cudaMemcpy(p->amp.p, ampd.data(), ampd.size() * 8, cudaMemcpyHostToDevice));
    HM_TRY(p->ampd.alloc(colour.size() * 8));
    HM_CUDA(cudaMemcpy(p->ampd.p, colour.data(), colour.size() * 8, cudaMemcpyHostToDevice));
    HM_TRY(p->tw.alloc(twd.size() * 8));
    HM_CUDA(cudaMemcpy(p->tw.p, twd.data(), twd.size() * 8, cudaMemcpyHostToDevice));
  }
  if (dz_prior) {
    // built by hm_set_catalog; the device sees a table (d0 = 0) once a catalogue is set
    p->prior_dz = true;
    p->dz_bin = d.prior_bin > 0 ? d.prior_bin : 5.0;
    p->dz_pad = d.prior_pad > 0 ? d.prior_pad : 3.0 * p->sigma_v / kH0;
    p->desc.prior_kind = HM_PRIOR_TABLE;
    p->desc.prior_d0 = 0.0;
    p->desc.prior_bin = p->dz_bin;
    p->desc.prior_nbins = 0;
  } else if (d.prior_kind == HM_PRIOR_TABLE) {
    p->prior_host.assign(d.prior_logdens_host, d.prior_logdens_host + d.prior_nbins);
    HM_TRY(p->prior_logdens.alloc(p->prior_host.size() * 8));
    HM_CUDA(cudaMemcpy(p->prior_logdens.p, p->prior_host.data(), p->prior_host.size() * 8, cudaMemcpyHostToDevice));
  }
  p->desc.prior_logdens_host = nullptr;
  HM_CUDA(fft_prepare(p->prec, N));
  *out = p.release();
  return HM_OK;
}

void hm_destroy_problem(hm_problem* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  delete p;
}

int hm_problem_get_info(const hm_problem* p, hm_problem_info* out) {
  if (!p || !out) return fail(HM_EINVAL, "null argument");
  out->N = p->N;
  out->precision = p->prec;
  out->n_points = p->n;
  out->L = p->L;
  out->delta = p->delta;
  out->f_growth = p->f;
  out->sigma_v = p->sigma_v;
  out->minv_d = p->minv_d;
  out->pk_amplitude = p->pkA;
  out->grid_bytes = (int64_t)(p->rsz * p->n3);
  out->spectrum_bytes = (int64_t)(2 * p->rsz * p->nspec);
  return HM_OK;
}

// The FP32 path's per-point constants (see XRef), in FP64 on the host.
static XRef xref_of(double omega_m, double h, double mu, double z) {
  const double k3 = 3.0 * omega_m * kH0 / kC, c23 = 2.0 / (3.0 * omega_m), dmax = 0.999 / k3;
  auto s_of = [&](double d) { return std::sqrt(1.0 - k3 * d); };
  auto zbar = [&](double d) { return c23 * k3 * d / (1.0 + s_of(d)); };   // c23 (1 - s) without cancellation
  auto x_of = [&](double d) { return d * (1.0 + zbar(d)) / h; };
  auto split = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  XRef r{};
  // d_z in closed form: s(d_z) = 1 - z/c23 (clamped where no distance has this zbar)
  double dz = (1.0 - (1.0 - z / c23) * (1.0 - z / c23)) / k3;
  if (!(dz < dmax)) dz = dmax;
  split(dz, r.dz_hi, r.dz_lo);
  r.s_z = (float)s_of(dz);
  r.e_z = (float)(z - zbar(dz));
  // d_ref by Newton on x(d) = x_ref (x increases with d), clamped to (0, dmax]
  const double xref = std::pow(10.0, (mu - 25.0) / 5.0);
  double dr = std::min(std::max(h * xref, 1e-6), dmax);
  for (int it = 0; it < 60; ++it) {
    const double sd = s_of(dr);
    const double g = x_of(dr) - xref;
    const double gp = (1.0 + zbar(dr) + dr * 0.5 * c23 * k3 / sd) / h;
    const double dn = std::min(std::max(dr - g / gp, 1e-6), dmax);
    if (dn == dr) break;
    dr = dn;
  }
  split(dr, r.dr_hi, r.dr_lo);
  r.s_ref = (float)s_of(dr);
  r.e_ref = (float)(x_of(dr) - xref);
  return r;
}

static int upload(DevBuf& b, const double* src, long long n) {
  HM_TRY(b.alloc(sizeof(double) * (size_t)std::max<long long>(n, 1)));
  if (n > 0) HM_CUDA(cudaMemcpy(b.p, src, sizeof(double) * n, cudaMemcpyHostToDevice));
  return HM_OK;
}

int hm_set_catalog(hm_problem* p, int64_t n, const double* rhat, const double* mu, const double* smu,
                   const double* cz, const double* scz) {
  if (!p) return fail(HM_EINVAL, "null problem");
  if (n < 0) return fail(HM_EINVAL, "n < 0");
  if (n > (1ll << 30)) return fail(HM_EINVAL, "catalogue larger than 2^30 points");
  if (n > 0 && (!rhat || !mu || !smu || !cz)) return fail(HM_EINVAL, "null catalogue array");
  HM_TRY(check_finite(rhat, 3 * n, "rhat"));
  HM_TRY(check_finite(mu, n, "mu"));
  HM_TRY(check_finite(smu, n, "sigma_mu"));
  HM_TRY(check_finite(cz, n, "cz"));
  if (scz) HM_TRY(check_finite(scz, n, "sigma_cz"));
  std::vector<double> rx(n), ry(n), rz(n), z(n), sc(n, 0.0);
  for (long long i = 0; i < n; ++i) {
    if (!(smu[i] > 0)) return fail(HM_EINVAL, "sigma_mu must be > 0");
    if (scz && !(scz[i] >= 0)) return fail(HM_EINVAL, "sigma_cz must be >= 0");
    rx[i] = rhat[3 * i];
    ry[i] = rhat[3 * i + 1];
    rz[i] = rhat[3 * i + 2];
    const double nn = rx[i] * rx[i] + ry[i] * ry[i] + rz[i] * rz[i];
    if (std::fabs(nn - 1.0) > 2e-6) return fail(HM_EINVAL, "rhat must be unit vectors");
    z[i] = cz[i] / kC;
    if (scz) sc[i] = scz[i];
  }
  HM_CUDA(cudaSetDevice(p->device));
  HM_TRY(upload(p->rx, rx.data(), n));
  HM_TRY(upload(p->ry, ry.data(), n));
  HM_TRY(upload(p->rz, rz.data(), n));
  HM_TRY(upload(p->mu, mu, n));
  std::vector<XRef> xr((size_t)std::max<long long>(n, 1));
  for (long long i = 0; i < n; ++i) xr[i] = xref_of(p->desc.omega_m, p->desc.h, mu[i], z[i]);
  static_assert(sizeof(XRef) == 4 * sizeof(double), "XRef is uploaded as four doubles");
  HM_TRY(upload(p->xr, reinterpret_cast<const double*>(xr.data()), 4 * n));
  std::vector<double> ismu2(n);
  for (long long i = 0; i < n; ++i) ismu2[i] = 1.0 / (smu[i] * smu[i]);
  HM_TRY(upload(p->smu, ismu2.data(), n));   // the device keeps 1/sigma_mu^2
  HM_TRY(upload(p->zobs, z.data(), n));
  HM_TRY(upload(p->scz, sc.data(), n));
  if (p->prior_dz) {
    if (p->prior_logdens.p) {   // states made from the previous catalogue keep reading its table
      p->prior_retired.push_back(std::make_unique<DevBuf>());
      std::swap(p->prior_retired.back()->p, p->prior_logdens.p);
      std::swap(p->prior_retired.back()->bytes, p->prior_logdens.bytes);
    }
    p->prior_host.clear();
    p->desc.prior_nbins = 0;
    if (n > 0) {
      p->prior_host = dz_histogram(p->desc.omega_m, n, cz, p->dz_bin, p->dz_pad);
      if (p->prior_host.size() > (size_t)(1 << 24)) return fail(HM_EINVAL, "redshift-distance histogram too long");
      HM_TRY(p->prior_logdens.alloc(p->prior_host.size() * 8));
      HM_CUDA(cudaMemcpy(p->prior_logdens.p, p->prior_host.data(), p->prior_host.size() * 8,
                         cudaMemcpyHostToDevice));
      p->desc.prior_nbins = (int32_t)p->prior_host.size();
    }
  }
  p->n = n;
  p->ws_points = -1;   // the standalone workspace takes the new catalogue's parameters
  return HM_OK;
}

int hm_problem_prior_table(const hm_problem* p, int32_t max_bins, double* logdens_out, int32_t* nbins_out,
                           double* d0_out, double* bin_out) {
  if (!p || !nbins_out) return fail(HM_EINVAL, "null argument");
  if (p->desc.prior_kind != HM_PRIOR_TABLE) return fail(HM_ESTATE, "the problem's distance prior is not a table");
  *nbins_out = (int32_t)p->prior_host.size();
  if (d0_out) *d0_out = p->desc.prior_d0;
  if (bin_out) *bin_out = p->desc.prior_bin;
  if (!logdens_out) return HM_OK;
  if ((size_t)max_bins < p->prior_host.size()) return fail(HM_EINVAL, "max_bins too small (see nbins_out)");
  std::copy(p->prior_host.begin(), p->prior_host.end(), logdens_out);
  return HM_OK;
}

int hm_set_catalog_sg(hm_problem* p, int64_t n, const double* sgl_deg, const double* sgb_deg, const double* mu,
                      const double* smu, const double* cz, const double* scz) {
  if (!p) return fail(HM_EINVAL, "null problem");
  if (n < 0) return fail(HM_EINVAL, "n < 0");
  if (n > (1ll << 30)) return fail(HM_EINVAL, "catalogue larger than 2^30 points");
  if (n > 0 && (!sgl_deg || !sgb_deg)) return fail(HM_EINVAL, "null catalogue array");
  HM_TRY(check_finite(sgl_deg, n, "SGL"));
  HM_TRY(check_finite(sgb_deg, n, "SGB"));
  // the direction on the sky in the grid frame, whose axes are the
  // supergalactic X, Y, Z
  const double rad = 3.14159265358979323846 / 180.0;
  std::vector<double> rhat(3 * (size_t)n);
  for (long long i = 0; i < n; ++i) {
    if (!(sgb_deg[i] >= -90.0 && sgb_deg[i] <= 90.0)) return fail(HM_EINVAL, "SGB must be in [-90, 90] degrees");
    const double l = sgl_deg[i] * rad, b = sgb_deg[i] * rad;
    const double cb = std::cos(b);
    rhat[3 * i] = cb * std::cos(l);
    rhat[3 * i + 1] = cb * std::sin(l);
    rhat[3 * i + 2] = std::sin(b);
  }
  return hm_set_catalog(p, n, rhat.data(), mu, smu, cz, scz);
}

// standalone workspace of a problem (one chain)
static int ensure_ws(hm_problem* p) {
  if (p->ws_points == p->n && p->S1.p) return HM_OK;
  const int N = p->N;
  HM_TRY(p->S1.alloc(2 * p->rsz * 3 * p->nspec));
  HM_TRY(p->S2.alloc(2 * p->rsz * 3 * p->nspec));
  HM_TRY(p->pw.alloc(p->prec, 1, N, p->n));
  HM_TRY(p->prior_part.alloc(8 * N * plane_split(N)));
  const int pb = points_blocks((int)p->n);
  HM_TRY(p->pts_part.alloc(8 * pb));
  HM_TRY(p->kin_part.alloc(8 * std::max(N * plane_split(N), pb)));
  HM_TRY(p->pp.alloc(sizeof(PointParams)));
  HM_TRY(p->cs.alloc(sizeof(ChainScal)));
  HM_TRY(p->chain_id.alloc(sizeof(int)));
  PointParams P = point_params(p, 0);
  HM_CUDA(cudaMemcpy(p->pp.p, &P, sizeof(P), cudaMemcpyHostToDevice));
  ChainScal S{};
  HM_CUDA(cudaMemcpy(p->cs.p, &S, sizeof(S), cudaMemcpyHostToDevice));
  int z = 0;
  HM_CUDA(cudaMemcpy(p->chain_id.p, &z, sizeof(z), cudaMemcpyHostToDevice));
  p->ws_points = p->n;
  return HM_OK;
}

int hm_logpost_grad(hm_problem* p, const void* w_dev, const double* d_dev, double* psi_dev,
                    void* grad_w_dev, double* grad_d_dev, void* stream) {
  if (!p || !w_dev || !psi_dev || !grad_w_dev) return fail(HM_EINVAL, "null argument");
  if (p->n > 0 && (!d_dev || !grad_d_dev)) return fail(HM_EINVAL, "null distance argument");
  if (p->ws_points < 0 && !p->rx.p) return fail(HM_ESTATE, "no catalogue set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(p->device));
  HM_TRY(ensure_ws(p));
  PointArrays pa{};
  pa.rx = p->rx.as<double>();
  pa.ry = p->ry.as<double>();
  pa.rz = p->rz.as<double>();
  pa.mu = p->mu.as<double>();
  pa.xr = p->xr.as<XRef>();
  pa.ismu2 = p->smu.as<double>();
  pa.zobs = p->zobs.as<double>();
  pa.scz = p->scz.as<double>();
  pa.d = const_cast<double*>(d_dev);
  pa.pd = nullptr;
  pa.gd = grad_d_dev;
  p->pw.fill(pa, p->n);
  ChainScal* cs = p->cs.as<ChainScal>();
  HM_CUDA(cudaMemsetAsync(&cs->status, 0, sizeof(int), st));
  GradArgs a{};
  a.prec = p->prec;
  a.N = p->N;
  a.C = 1;
  a.n3 = p->n3;
  a.nspec = p->nspec;
  a.delta = p->delta;
  a.tw = p->tw.p;
  a.amp = p->amp.p;
  a.w = const_cast<void*>(w_dev);
  a.pw = nullptr;
  a.gw = grad_w_dev;
  a.S1 = p->S1.p;
  a.S2 = p->S2.p;
  a.pa = pa;
  a.pp = p->pp.as<PointParams>();
  a.max_pts = (int)p->n;
  a.pts_blocks = points_blocks((int)p->n);
  a.prior_part = p->prior_part.as<double>();
  a.pts_part = p->pts_part.as<double>();
  a.kinl_f = p->kin_part.as<double>();
  a.kinl_p = p->kin_part.as<double>();
  a.cs = cs;
  a.work = &p->pw;
  HM_TRY(eval_single(a, st));
  HM_CUDA(launch_finalize(1, a.prior_part, p->N * plane_split(p->N), a.pts_part, a.pts_blocks, nullptr, 0, nullptr, 0, FIN_PSI,
                          0ull, p->chain_id.as<int>(), cs, nullptr, st));
  HM_CUDA(cudaMemcpyAsync(psi_dev, &cs->psi, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return HM_OK;
}

int hm_problem_last_status(hm_problem* p, void* stream, int32_t* status_out) {
  if (!p || !status_out) return fail(HM_EINVAL, "null argument");
  if (!p->cs.p) {
    *status_out = 0;
    return HM_OK;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(p->device));
  int v = 0;
  HM_CUDA(cudaMemcpyAsync(&v, &p->cs.as<ChainScal>()->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  *status_out = v;
  return HM_OK;
}

int hm_velocity_field(hm_problem* p, const void* w_dev, void* v_dev, void* stream) {
  if (!p || !w_dev || !v_dev) return fail(HM_EINVAL, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(p->device));
  HM_TRY(ensure_ws(p));
  HM_CUDA(launch_plane_r2c(p->prec, p->N, w_dev, p->n3, p->S1.p, p->nspec, 1, p->tw.p, st));
  HM_CUDA(launch_pencil(p->prec, p->N, PM_VEL, p->S1.p, p->nspec, p->S2.p, p->nspec, 1, p->tw.p, p->amp.p, st));
  HM_CUDA(launch_plane_c2r(p->prec, p->N, p->S2.p, p->nspec, v_dev, p->n3, 3, p->tw.p, nullptr, st));
  return HM_OK;
}

int hm_fft_r2c(hm_problem* p, const void* in_dev, void* out_dev, int32_t count, void* stream) {
  if (!p || !in_dev || !out_dev || count < 0) return fail(HM_EINVAL, "bad argument");
  if (count == 0) return HM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(p->device));
  HM_CUDA(launch_plane_r2c(p->prec, p->N, in_dev, p->n3, out_dev, p->nspec, count, p->tw.p, st));
  HM_CUDA(launch_pencil(p->prec, p->N, PM_FWD, out_dev, p->nspec, out_dev, p->nspec, count, p->tw.p, p->amp.p, st));
  return HM_OK;
}

int hm_fft_c2r(hm_problem* p, const void* in_dev, void* out_dev, int32_t count, void* stream) {
  if (!p || !in_dev || !out_dev || count < 0) return fail(HM_EINVAL, "bad argument");
  if (count == 0) return HM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(p->device));
  HM_TRY(ensure_ws(p));
  // x pass into the workspace (input untouched), then planes
  for (int c = 0; c < count; ++c) {
    const char* src = static_cast<const char*>(in_dev) + (size_t)c * 2 * p->rsz * p->nspec;
    char* dst = static_cast<char*>(out_dev) + (size_t)c * p->rsz * p->n3;
    HM_CUDA(launch_pencil(p->prec, p->N, PM_INV, src, p->nspec, p->S1.p, p->nspec, 1, p->tw.p, p->amp.p, st));
    HM_CUDA(launch_plane_c2r(p->prec, p->N, p->S1.p, p->nspec, dst, p->n3, 1, p->tw.p, nullptr, st));
  }
  return HM_OK;
}

int hm_cells(hm_problem* p, const double* d_dev, int32_t* cell_dev, int32_t* perm_dev, void* stream) {
  if (!p || !cell_dev || (p->n > 0 && !d_dev)) return fail(HM_EINVAL, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(p->device));
  HM_TRY(ensure_ws(p));
  PointArrays pa{};
  pa.rx = p->rx.as<double>();
  pa.ry = p->ry.as<double>();
  pa.rz = p->rz.as<double>();
  pa.ntot = p->n;
  HM_CUDA(launch_cells(1, (int)p->n, p->pp.as<PointParams>(), d_dev, pa, cell_dev, st));
  if (perm_dev) {
    if (!p->hist.p) HM_TRY(p->hist.alloc(4 * (size_t)p->n3));
    HM_CUDA(launch_cell_sort((int)p->n3, p->n, cell_dev, perm_dev, p->hist.as<int>(), st));
  }
  return HM_OK;
}

int hm_device_wait_timeouts(int32_t device, int32_t reset, int32_t* count_out) {
  if (!count_out) return fail(HM_EINVAL, "null argument");
  HM_CUDA(cudaSetDevice(device));
  const int v = fft_tma_wait_timeouts(reset != 0);
  if (v < 0) return fail(HM_ECUDA, "reading the wait counter failed");
  *count_out = v;
  return HM_OK;
}

int hm_dz_prior_table(double omega_m, int64_t n, const double* cz_host, double bin_width, double pad,
                      int32_t max_bins, double* logdens_out, int32_t* nbins_out) {
  if (n <= 0 || !cz_host || !nbins_out) return fail(HM_EINVAL, "need n > 0 redshifts and nbins_out");
  if (!(bin_width > 0) || !(pad >= 0) || !(omega_m > 0)) return fail(HM_EINVAL, "bad bin width, pad or omega_m");
  HM_TRY(check_finite(cz_host, n, "cz"));
  const std::vector<double> t = dz_histogram(omega_m, n, cz_host, bin_width, pad);
  *nbins_out = (int32_t)t.size();
  if ((long long)t.size() > max_bins || !logdens_out)
    return (long long)t.size() > max_bins ? fail(HM_EINVAL, "max_bins too small (see nbins_out)") : HM_OK;
  std::copy(t.begin(), t.end(), logdens_out);
  return HM_OK;
}

int hm_philox(uint64_t seed, int64_t n, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t* out_dev, void* stream) {
  if (n < 0 || (n > 0 && !out_dev)) return fail(HM_EINVAL, "bad argument");
  HM_CUDA(launch_philox_raw(seed, n, c1, c2, c3, out_dev, static_cast<cudaStream_t>(stream)));
  return HM_OK;
}

// ---------------------------------------------------------------------------
// chain states
// ---------------------------------------------------------------------------
// CTAs per chain of the trajectory-start field kernel (momentum draw, save,
// half kick and drift): enough that a single chain fills the GPU, no more
// threads than node pairs and at most 1024 blocks per chain.
static int field_parts(long long n3) {
  return (int)std::min<long long>(1024, std::max<long long>(1, (n3 / 2 + 255) / 256));
}

static GradArgs state_args(hm_state* s) {
  GradArgs a{};
  a.prec = s->prec;
  a.N = s->N;
  a.C = s->C;
  a.n3 = s->n3;
  a.nspec = s->nspec;
  a.delta = s->p0->delta;
  a.tw = s->p0->tw.p;
  a.amp = s->p0->amp.p;
  a.w = s->w.p;
  a.pw = s->pw.p;
  a.gw = s->gw.p;
  a.S1 = s->S1.p;
  a.S2 = s->S2.p;
  a.pa = point_arrays(s);
  a.pp = s->pp.as<PointParams>();
  a.max_pts = s->max_pts;
  a.pts_blocks = s->pts_blocks;
  a.prior_part = s->prior_part.as<double>();
  a.pts_part = s->pts_part.as<double>();
  a.kinl_f = s->kinl_f.as<double>();
  a.kinl_p = s->kinl_p.as<double>();
  a.cs = s->cs.as<ChainScal>();
  a.work = &s->work;
  a.gsig_part = s->gsig_part.as<double>();
  a.sample_sig = s->sample_sig;
  return a;
}

static int state_refresh(hm_state* s, cudaStream_t st) {
  GradArgs a = state_args(s);
  HM_TRY(eval_single(a, st));
  HM_CUDA(launch_finalize(s->C, a.prior_part, s->NP, a.pts_part, s->pts_blocks, nullptr, 0, nullptr, 0, FIN_PSI,
                          s->seed, s->chain_id.as<int>(), a.cs, nullptr, st));
  return HM_OK;
}

int hm_state_create_batch(hm_problem* const* problems, int32_t n_problems, int32_t n_chains,
                          const int32_t* chain_problem, const int32_t* chain_ids, uint64_t seed,
                          const double* const* d_init_host, hm_state** out) {
  if (!problems || n_problems <= 0 || n_chains <= 0 || !out) return fail(HM_EINVAL, "bad argument");
  *out = nullptr;
  hm_problem* p0 = problems[0];
  for (int i = 0; i < n_problems; ++i) {
    if (!problems[i]) return fail(HM_EINVAL, "null problem");
    if (problems[i]->N != p0->N || problems[i]->prec != p0->prec || problems[i]->device != p0->device)
      return fail(HM_EINVAL, "problems of one state must share N, precision and device");
    if (std::fabs(problems[i]->L - p0->L) > 0 || problems[i]->aHf != p0->aHf || problems[i]->pkA != p0->pkA)
      return fail(HM_EINVAL, "problems of one state must share the box and the power spectrum");
  }
  auto s = std::make_unique<hm_state>();
  s->C = n_chains;
  s->N = p0->N;
  s->NP = p0->N * plane_split(p0->N);
  s->prec = p0->prec;
  s->device = p0->device;
  s->n3 = p0->n3;
  s->nspec = p0->nspec;
  s->rsz = p0->rsz;
  s->seed = seed;
  s->p0 = p0;
  HM_CUDA(cudaSetDevice(s->device));
  std::vector<long long> off(n_chains);
  long long tot = 0;
  int maxp = 0;
  for (int c = 0; c < n_chains; ++c) {
    const int pi = chain_problem ? chain_problem[c] : 0;
    if (pi < 0 || pi >= n_problems) return fail(HM_EINVAL, "chain_problem out of range");
    hm_problem* p = problems[pi];
    if (p->n > 0 && (!d_init_host || !d_init_host[c])) return fail(HM_EINVAL, "d_init_host required");
    s->chain_prob.push_back(p);
    off[c] = tot;
    tot += p->n;
    maxp = (int)std::max<long long>(maxp, p->n);
  }
  s->ntot = tot;
  s->max_pts = maxp;
  s->pts_blocks = points_blocks(maxp);
  s->nparts_f = field_parts(s->n3);
  s->nparts_p = traj_begin_points_blocks(maxp);
  const size_t C = n_chains, rs = s->rsz;
  HM_TRY(s->w.alloc(rs * C * s->n3));
  HM_TRY(s->pw.alloc(rs * C * s->n3));
  HM_TRY(s->gw.alloc(rs * C * s->n3));
  HM_TRY(s->w0.alloc(rs * C * s->n3));
  HM_TRY(s->gw0.alloc(rs * C * s->n3));
  HM_TRY(s->S1.alloc(2 * rs * 3 * C * s->nspec));
  HM_TRY(s->S2.alloc(2 * rs * 3 * C * s->nspec));
  HM_CUDA(cudaMemset(s->w.p, 0, rs * C * s->n3));
  HM_CUDA(cudaMemset(s->pw.p, 0, rs * C * s->n3));
  const size_t nt = (size_t)std::max<long long>(tot, 1);
  DevBuf* dbl[] = {&s->rx, &s->ry, &s->rz, &s->mu, &s->smu, &s->zobs,
                   &s->scz, &s->d, &s->pd, &s->gd, &s->d0, &s->gd0};
  for (DevBuf* b : dbl) HM_TRY(b->alloc(8 * nt));
  HM_TRY(s->xr.alloc(sizeof(XRef) * nt));
  HM_CUDA(cudaMemset(s->pd.p, 0, 8 * nt));
  HM_TRY(s->work.alloc(s->prec, n_chains, s->N, tot));
  for (int c = 0; c < n_chains; ++c) {
    hm_problem* p = s->chain_prob[c];
    const long long n = p->n;
    if (n == 0) continue;
    const size_t b = 8 * (size_t)n, o = 8 * (size_t)off[c];
    HM_CUDA(cudaMemcpy((char*)s->rx.p + o, p->rx.p, b, cudaMemcpyDeviceToDevice));
    HM_CUDA(cudaMemcpy((char*)s->ry.p + o, p->ry.p, b, cudaMemcpyDeviceToDevice));
    HM_CUDA(cudaMemcpy((char*)s->rz.p + o, p->rz.p, b, cudaMemcpyDeviceToDevice));
    HM_CUDA(cudaMemcpy((char*)s->mu.p + o, p->mu.p, b, cudaMemcpyDeviceToDevice));
    HM_CUDA(cudaMemcpy((char*)s->xr.p + 4 * o, p->xr.p, 4 * b, cudaMemcpyDeviceToDevice));
    HM_CUDA(cudaMemcpy((char*)s->smu.p + o, p->smu.p, b, cudaMemcpyDeviceToDevice));
    HM_CUDA(cudaMemcpy((char*)s->zobs.p + o, p->zobs.p, b, cudaMemcpyDeviceToDevice));
    HM_CUDA(cudaMemcpy((char*)s->scz.p + o, p->scz.p, b, cudaMemcpyDeviceToDevice));
    HM_TRY(check_finite(d_init_host[c], n, "d_init"));
    HM_CUDA(cudaMemcpy((char*)s->d.p + o, d_init_host[c], b, cudaMemcpyHostToDevice));
    s->pp_host.push_back(point_params(p, off[c]));
  }
  // point params for chains without points too
  s->pp_host.clear();
  for (int c = 0; c < n_chains; ++c) s->pp_host.push_back(point_params(s->chain_prob[c], off[c]));
  HM_TRY(s->pp.alloc(sizeof(PointParams) * C));
  HM_CUDA(cudaMemcpy(s->pp.p, s->pp_host.data(), sizeof(PointParams) * C, cudaMemcpyHostToDevice));
  HM_TRY(s->cs.alloc(sizeof(ChainScal) * C));
  std::vector<ChainScal> csh(C);
  for (auto& x : csh) {
    x = ChainScal{};
    x.sample_d = 1;
  }
  HM_CUDA(cudaMemcpy(s->cs.p, csh.data(), sizeof(ChainScal) * C, cudaMemcpyHostToDevice));
  std::vector<int> ids(C);
  for (int c = 0; c < n_chains; ++c) ids[c] = chain_ids ? chain_ids[c] : c;
  HM_TRY(s->chain_id.alloc(sizeof(int) * C));
  HM_CUDA(cudaMemcpy(s->chain_id.p, ids.data(), sizeof(int) * C, cudaMemcpyHostToDevice));
  HM_TRY(s->prior_part.alloc(8 * C * s->NP));
  HM_TRY(s->pts_part.alloc(8 * C * s->pts_blocks));
  HM_TRY(s->kinb_f.alloc(8 * C * s->nparts_f));
  HM_TRY(s->kinb_p.alloc(8 * C * s->nparts_p));
  HM_TRY(s->kinl_f.alloc(8 * C * s->NP));
  HM_TRY(s->kinl_p.alloc(8 * C * s->pts_blocks));
  HM_CUDA(cudaMemset(s->kinl_p.p, 0, 8 * C * s->pts_blocks));
  HM_CUDA(cudaMemset(s->kinb_p.p, 0, 8 * C * s->nparts_p));
  HM_TRY(s->eps_dev.alloc(8 * C));
  HM_TRY(s->sig_dev.alloc(8 * C));
  HM_TRY(s->gsig_part.alloc(8 * C * s->pts_blocks));
  s->eps_host.assign(C, 0.0);
  // evaluate at the start on a private stream: a device-wide synchronisation
  // would be illegal while another thread captures a trajectory graph
  cudaStream_t init_st = nullptr;
  HM_CUDA(cudaStreamCreateWithFlags(&init_st, cudaStreamNonBlocking));
  int rc = state_refresh(s.get(), init_st);
  cudaError_t se = cudaStreamSynchronize(init_st);
  cudaStreamDestroy(init_st);
  if (rc != HM_OK) return rc;
  if (se != cudaSuccess) return fail(HM_ECUDA, std::string("state creation: ") + cudaGetErrorString(se));
  *out = s.release();
  return HM_OK;
}

int hm_state_create(hm_problem* p, uint64_t seed, const double* d_init_host, hm_state** out) {
  hm_problem* ps[1] = {p};
  const double* di[1] = {d_init_host};
  return hm_state_create_batch(ps, 1, 1, nullptr, nullptr, seed, di, out);
}

void hm_destroy_state(hm_state* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  delete s;
}

static int chain_ok(hm_state* s, int chain) {
  if (!s) return fail(HM_EINVAL, "null state");
  if (chain < 0 || chain >= s->C) return fail(HM_EINVAL, "chain out of range");
  return HM_OK;
}

int hm_state_set(hm_state* s, int32_t chain, const void* w, const double* d, const void* pw, const double* pd,
                 void* stream) {
  HM_TRY(chain_ok(s, chain));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const size_t gb = s->rsz * s->n3;
  const PointParams& P = s->pp_host[chain];
  if (w) HM_CUDA(cudaMemcpyAsync((char*)s->w.p + gb * chain, w, gb, cudaMemcpyDefault, st));
  if (pw) HM_CUDA(cudaMemcpyAsync((char*)s->pw.p + gb * chain, pw, gb, cudaMemcpyDefault, st));
  if (d && P.pt_n) HM_CUDA(cudaMemcpyAsync(s->d.as<double>() + P.pt_off, d, 8 * P.pt_n, cudaMemcpyDefault, st));
  if (pd && P.pt_n) HM_CUDA(cudaMemcpyAsync(s->pd.as<double>() + P.pt_off, pd, 8 * P.pt_n, cudaMemcpyDefault, st));
  return HM_OK;
}

int hm_state_get(hm_state* s, int32_t chain, void* w, double* d, void* pw, double* pd, void* stream) {
  HM_TRY(chain_ok(s, chain));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const size_t gb = s->rsz * s->n3;
  const PointParams& P = s->pp_host[chain];
  if (w) HM_CUDA(cudaMemcpyAsync(w, (char*)s->w.p + gb * chain, gb, cudaMemcpyDefault, st));
  if (pw) HM_CUDA(cudaMemcpyAsync(pw, (char*)s->pw.p + gb * chain, gb, cudaMemcpyDefault, st));
  if (d && P.pt_n) HM_CUDA(cudaMemcpyAsync(d, s->d.as<double>() + P.pt_off, 8 * P.pt_n, cudaMemcpyDefault, st));
  if (pd && P.pt_n) HM_CUDA(cudaMemcpyAsync(pd, s->pd.as<double>() + P.pt_off, 8 * P.pt_n, cudaMemcpyDefault, st));
  return HM_OK;
}

int hm_state_get_grad(hm_state* s, int32_t chain, void* gw, double* gd, void* stream) {
  HM_TRY(chain_ok(s, chain));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const size_t gb = s->rsz * s->n3;
  const PointParams& P = s->pp_host[chain];
  if (gw) HM_CUDA(cudaMemcpyAsync(gw, (char*)s->gw.p + gb * chain, gb, cudaMemcpyDefault, st));
  if (gd && P.pt_n) HM_CUDA(cudaMemcpyAsync(gd, s->gd.as<double>() + P.pt_off, 8 * P.pt_n, cudaMemcpyDefault, st));
  return HM_OK;
}

int hm_state_refresh(hm_state* s, void* stream) {
  if (!s) return fail(HM_EINVAL, "null state");
  HM_CUDA(cudaSetDevice(s->device));
  return state_refresh(s, static_cast<cudaStream_t>(stream));
}

int hm_state_scalars(hm_state* s, int32_t chain, double* psi, double* kinetic, int64_t* traj, void* stream) {
  HM_TRY(chain_ok(s, chain));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  ChainScal S{};
  HM_CUDA(cudaMemcpyAsync(&S, s->cs.as<ChainScal>() + chain, sizeof(S), cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  if (psi) *psi = S.psi;
  if (kinetic) *kinetic = S.kin;
  if (traj) *traj = S.traj;
  return HM_OK;
}

int hm_state_set_traj(hm_state* s, int32_t chain, int64_t traj) {
  HM_TRY(chain_ok(s, chain));
  HM_CUDA(cudaSetDevice(s->device));
  long long t = traj;
  HM_CUDA(cudaMemcpy(&(s->cs.as<ChainScal>() + chain)->traj, &t, sizeof(t), cudaMemcpyHostToDevice));
  return HM_OK;
}

static int set_run(hm_state* s, const double* eps, int sample_d, cudaStream_t st) {
  for (int c = 0; c < s->C; ++c) {
    if (!(eps[c] > 0) || !std::isfinite(eps[c])) return fail(HM_EINVAL, "eps must be finite and > 0");
    s->eps_host[c] = eps[c];
  }
  HM_CUDA(cudaMemcpyAsync(s->eps_dev.p, s->eps_host.data(), 8 * s->C, cudaMemcpyHostToDevice, st));
  HM_CUDA(launch_set_run(s->C, s->eps_dev.as<double>(), sample_d ? 1 : 0, s->cs.as<ChainScal>(), st));
  return HM_OK;
}

// leapfrog body: first half kick + drift from the stored gradient, then
// n_steps gradient evaluations with fused kick (+ drift)
static int leapfrog_body(hm_state* s, int n_steps, int draw, cudaStream_t st, Prof* pf) {
  GradArgs a = state_args(s);
  a.prof = pf;
  PointArrays pa = a.pa;
  s->work.fill(pa, s->ntot, 1);   // begin counts the drifted d into half 0 (pa.cnt_next)
  if (pf) HM_CUDA(pf->begin(KK_BEGIN, st));
  HM_CUDA(launch_traj_begin_field(s->prec, s->C, s->n3, s->w.p, s->pw.p, s->gw.p, s->w0.p, s->gw0.p, s->seed,
                                  s->chain_id.as<int>(), s->kinb_f.as<double>(), s->nparts_f, draw, a.cs, st));
  if (s->max_pts > 0) {
    HM_CUDA(cudaMemsetAsync(pa.cnt_next, 0, sizeof(int) * (size_t)s->work.CN, st));
    HM_CUDA(launch_traj_begin_points(s->C, s->max_pts, a.pp, pa, s->d0.as<double>(), s->gd0.as<double>(), s->seed,
                                     s->chain_id.as<int>(), s->kinb_p.as<double>(), s->nparts_p, draw, a.cs, st));
  }
  if (s->sample_sig) HM_CUDA(launch_sig_begin(s->C, s->seed, s->chain_id.as<int>(), draw, a.cs, st));
  HM_CUDA(launch_finalize(s->C, nullptr, 0, nullptr, 0, s->kinb_f.as<double>(), s->nparts_f,
                          s->kinb_p.as<double>(), s->max_pts > 0 ? s->nparts_p : 0, FIN_HOLD, s->seed,
                          s->chain_id.as<int>(), a.cs, nullptr, st));
  if (pf) HM_CUDA(pf->end(st));
  return eval_run(a, n_steps, GM_KICK_LAST, st);
}

int hm_leapfrog(hm_state* s, int32_t n_steps, double eps, int32_t sample_distances, void* stream) {
  if (!s) return fail(HM_EINVAL, "null state");
  if (n_steps <= 0) return fail(HM_EINVAL, "n_steps must be > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  std::vector<double> e(s->C, eps);
  HM_TRY(set_run(s, e.data(), sample_distances, st));
  HM_TRY(leapfrog_body(s, n_steps, 0, st, nullptr));
  GradArgs a = state_args(s);
  HM_CUDA(launch_finalize(s->C, a.prior_part, s->NP, a.pts_part, s->pts_blocks, a.kinl_f, s->NP, a.kinl_p,
                          s->max_pts > 0 ? s->pts_blocks : 0, FIN_PSI | FIN_KIN, s->seed, s->chain_id.as<int>(),
                          a.cs, nullptr, st));
  return HM_OK;
}

static int profile_collect(hm_state* s) {
  if (!s->prof || s->prof_pending == 0) return HM_OK;
  HM_CUDA(cudaStreamSynchronize(s->prof_stream));
  const int n = s->prof_pending;
  s->prof_pending = 0;
  return s->prof->collect(n);
}

static int trajectory(hm_state* s, int n_leapfrog, cudaStream_t st, Prof* pf) {
  HM_TRY(leapfrog_body(s, n_leapfrog, 1, st, pf));
  GradArgs a = state_args(s);
  HM_PROF(pf, KK_FINALIZE, st,
          launch_finalize(s->C, a.prior_part, s->NP, a.pts_part, s->pts_blocks, a.kinl_f, s->NP, a.kinl_p,
                          s->max_pts > 0 ? s->pts_blocks : 0, FIN_PSI | FIN_ACCEPT, s->seed,
                          s->chain_id.as<int>(), a.cs, s->trace_dev.p, st));
  HM_PROF(pf, KK_RESTORE, st,
          launch_restore(s->prec, s->C, s->n3, s->w.p, s->gw.p, s->w0.p, s->gw0.p, s->max_pts, a.pp, a.pa,
                         s->d0.as<double>(), s->gd0.as<double>(), a.cs, st));
  return HM_OK;
}

static int analytics_sample(hm_state* s, cudaStream_t st);

// sample != 0: one chain-analytics sample after every trajectory (when on).
static int run_traj_loop(hm_state* s, int32_t n_traj, int32_t n_leapfrog, int32_t sample_distances,
                         int32_t use_graph, cudaStream_t st, int sample = 0) {
  const bool an = sample && s->an.on;
  Prof* pf = s->prof.get();
  if (pf) {
    HM_TRY(profile_collect(s));
    HM_TRY(pf->reserve(14 * n_leapfrog + 8));
    pf->idx = 0;
  }
  // With profiling, a single-trajectory call leaves its events pending (read
  // by hm_state_profile_collect after the caller synchronises); longer runs
  // synchronise after every trajectory to read them before they are reused.
  if (!use_graph) {
    for (int t = 0; t < n_traj; ++t) {
      if (pf) pf->idx = 0;
      HM_TRY(trajectory(s, n_leapfrog, st, pf));
      if (an) HM_TRY(analytics_sample(s, st));
      if (pf) {
        if (n_traj == 1) {
          s->prof_pending = pf->idx;
          s->prof_stream = st;
        } else {
          HM_CUDA(cudaStreamSynchronize(st));
          HM_TRY(pf->collect(pf->idx));
        }
      }
    }
  } else if (n_traj > 0) {
    if (!s->gstream) HM_CUDA(cudaStreamCreateWithFlags(&s->gstream, cudaStreamNonBlocking));
    const int want_prof = pf ? 1 : 0;
    hm_state::Graph* gr = nullptr;
    for (auto& x : s->graphs)
      if (x.C == s->C && x.L == n_leapfrog && x.sd == sample_distances && x.prof == want_prof) gr = &x;
    if (!gr) {
      cudaGraph_t g = nullptr;
      if (pf) pf->idx = 0;
      HM_CUDA(cudaStreamBeginCapture(s->gstream, cudaStreamCaptureModeThreadLocal));
      int rc = trajectory(s, n_leapfrog, s->gstream, pf);
      cudaError_t ce = cudaStreamEndCapture(s->gstream, &g);
      if (rc != HM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ce != cudaSuccess) return fail(HM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
      cudaGraphExec_t ex = nullptr;
      ce = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return fail(HM_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
      s->graphs.push_back({s->C, n_leapfrog, sample_distances, want_prof, pf ? pf->idx : 0, ex});
      gr = &s->graphs.back();
    }
    if (pf) s->prof_pairs = gr->pairs;
    const cudaGraphExec_t gexec = gr->exec;
    cudaEvent_t ev;
    HM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    HM_CUDA(cudaEventRecord(ev, st));
    HM_CUDA(cudaStreamWaitEvent(s->gstream, ev, 0));
    for (int t = 0; t < n_traj; ++t) {
      HM_CUDA(cudaGraphLaunch(gexec, s->gstream));
      if (an) HM_TRY(analytics_sample(s, s->gstream));
      if (pf) {
        if (n_traj == 1) {
          s->prof_pending = s->prof_pairs;
          s->prof_stream = s->gstream;
        } else {
          HM_CUDA(cudaStreamSynchronize(s->gstream));
          HM_TRY(pf->collect(s->prof_pairs));
        }
      }
    }
    HM_CUDA(cudaEventRecord(ev, s->gstream));
    HM_CUDA(cudaStreamWaitEvent(st, ev, 0));
    HM_CUDA(cudaEventDestroy(ev));
  }
  return HM_OK;
}

int hm_run_chain(hm_state* s, int32_t n_traj, int32_t n_leapfrog, const double* eps_host, int32_t sample_distances,
                 int32_t use_graph, hm_trace* trace_host, void* stream) {
  if (!s || !eps_host) return fail(HM_EINVAL, "null argument");
  if (n_traj < 0 || n_leapfrog <= 0) return fail(HM_EINVAL, "n_traj >= 0 and n_leapfrog > 0 required");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const size_t need = sizeof(hm_trace) * (size_t)std::max(1, n_traj) * s->C;
  if (s->trace_cap < need) {
    HM_TRY(s->trace_dev.alloc(need));
    s->trace_cap = need;
    s->drop_graphs();
  }
  HM_TRY(set_run(s, eps_host, sample_distances, st));
  HM_TRY(run_traj_loop(s, n_traj, n_leapfrog, sample_distances, use_graph, st, 1));
  if (trace_host && n_traj > 0) {
    HM_CUDA(cudaMemcpyAsync(trace_host, s->trace_dev.p, sizeof(hm_trace) * (size_t)n_traj * s->C,
                            cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
  }
  return HM_OK;
}

int hm_adapt_step_size(hm_state* s, int32_t n_warmup, int32_t n_leapfrog, double target_accept,
                       const double* eps0_host, int32_t sample_distances, double* eps_out_host,
                       hm_trace* trace_host, void* stream) {
  if (!s || !eps0_host || !eps_out_host) return fail(HM_EINVAL, "null argument");
  if (s->slotted) return fail(HM_ESTATE, "a slotted state adapts per job (hm_slots_load, hm_slots_adapt_end)");
  if (n_warmup <= 0 || n_leapfrog <= 0) return fail(HM_EINVAL, "n_warmup and n_leapfrog must be > 0");
  if (!(target_accept > 0 && target_accept < 1)) return fail(HM_EINVAL, "target_accept must be in (0, 1)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const size_t need = sizeof(hm_trace) * (size_t)n_warmup * s->C;
  if (s->trace_cap < need) {
    HM_TRY(s->trace_dev.alloc(need));
    s->trace_cap = need;
    s->drop_graphs();
  }
  HM_TRY(set_run(s, eps0_host, sample_distances, st));
  HM_CUDA(launch_da(s->C, 1, target_accept, nullptr, s->cs.as<ChainScal>(), st));
  HM_TRY(run_traj_loop(s, n_warmup, n_leapfrog, sample_distances, 1, st));
  HM_CUDA(launch_da(s->C, 0, target_accept, s->eps_dev.as<double>(), s->cs.as<ChainScal>(), st));
  HM_CUDA(cudaMemcpyAsync(eps_out_host, s->eps_dev.p, 8 * s->C, cudaMemcpyDeviceToHost, st));
  if (trace_host)
    HM_CUDA(cudaMemcpyAsync(trace_host, s->trace_dev.p, need, cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  for (int c = 0; c < s->C; ++c) s->eps_host[c] = eps_out_host[c];
  return HM_OK;
}

int hm_state_sample_sigma_nl(hm_state* s, int32_t enable, const double* sigma0_host, void* stream) {
  if (!s) return fail(HM_EINVAL, "null state");
  if (s->slotted) return fail(HM_ESTATE, "sigma_NL sampling is not available on a slotted state");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  std::vector<double> sig(s->C);
  for (int c = 0; c < s->C; ++c) {
    sig[c] = sigma0_host ? sigma0_host[c] : s->chain_prob[c]->desc.sigma_nl;
    if (enable && !(sig[c] > 0) ) return fail(HM_EINVAL, "sigma_NL must start > 0");
  }
  HM_CUDA(cudaMemcpyAsync(s->sig_dev.p, sig.data(), 8 * s->C, cudaMemcpyHostToDevice, st));
  HM_CUDA(launch_sig_set(s->C, enable ? 1 : 0, s->sig_dev.as<double>(), s->cs.as<ChainScal>(), st));
  HM_CUDA(cudaStreamSynchronize(st));   // the host copy of sig must outlive the transfer
  s->sample_sig = enable != 0;
  s->drop_graphs();
  return state_refresh(s, st);
}

int hm_state_get_sigma_nl(hm_state* s, double* sigma_out_host, double* grad_out_host, void* stream) {
  if (!s || !sigma_out_host) return fail(HM_EINVAL, "null argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  std::vector<ChainScal> cs(s->C);
  HM_CUDA(cudaMemcpyAsync(cs.data(), s->cs.p, sizeof(ChainScal) * s->C, cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  for (int c = 0; c < s->C; ++c) {
    const bool smp = s->sample_sig && cs[c].sample_sig;
    sigma_out_host[c] = smp ? cs[c].sig : s->chain_prob[c]->desc.sigma_nl;
    if (grad_out_host) grad_out_host[c] = smp ? cs[c].g_sig : 0.0;
  }
  return HM_OK;
}

// ---------------------------------------------------------------------------
// Slotted states: continuous batching of independent jobs of one grid.  The
// active chains are packed at indices 0..C-1 so that every kernel launch of
// a trajectory covers exactly the loaded jobs; a released index is refilled
// by the last active chain.  Each chain keeps its catalogue in a point region
// of slot_pts entries (regions never move), its own step, trajectory counter
// and Philox chain word, so a job's chain does not depend on its neighbours.
// ---------------------------------------------------------------------------
static bool same_field_model(const hm_problem* a, const hm_problem* b) {
  return a->N == b->N && a->prec == b->prec && a->device == b->device && a->L == b->L && a->aHf == b->aHf &&
         a->pkA == b->pkA;
}

// Psi and the gradient of chain c alone (its position, its catalogue); the
// workspace of chain index 0 serves as scratch.
static int eval_chain(hm_state* s, int c, cudaStream_t st) {
  GradArgs a = state_args(s);
  const size_t gb = s->rsz * s->n3;
  a.C = 1;
  a.w = static_cast<char*>(s->w.p) + gb * c;
  a.pw = static_cast<char*>(s->pw.p) + gb * c;
  a.gw = static_cast<char*>(s->gw.p) + gb * c;
  a.pp = s->pp.as<PointParams>() + c;
  a.cs = s->cs.as<ChainScal>() + c;
  HM_TRY(eval_single(a, st));
  HM_CUDA(launch_finalize(1, a.prior_part, s->NP, a.pts_part, s->pts_blocks, nullptr, 0, nullptr, 0, FIN_PSI,
                          s->seed, s->chain_id.as<int>() + c, a.cs, nullptr, st));
  return HM_OK;
}

static int slotted_ok(hm_state* s) {
  if (!s) return fail(HM_EINVAL, "null state");
  if (!s->slotted) return fail(HM_ESTATE, "not a slotted state (hm_slots_create)");
  return HM_OK;
}

int hm_slots_create(hm_problem* templ, int32_t n_slots, int64_t max_points, uint64_t seed, hm_state** out) {
  if (!templ || !out || n_slots <= 0 || max_points < 0) return fail(HM_EINVAL, "bad argument");
  *out = nullptr;
  if (n_slots > 65535) return fail(HM_EINVAL, "n_slots must be <= 65535");
  const long long tot = (long long)n_slots * max_points;
  if (max_points > (1LL << 30) || tot > (1LL << 31) - 1) return fail(HM_EINVAL, "max_points too large");
  auto s = std::make_unique<hm_state>();
  s->slotted = true;
  s->C_cap = n_slots;
  s->C = 0;
  s->slot_pts = max_points;
  s->N = templ->N;
  s->NP = templ->N * plane_split(templ->N);
  s->prec = templ->prec;
  s->device = templ->device;
  s->n3 = templ->n3;
  s->nspec = templ->nspec;
  s->rsz = templ->rsz;
  s->seed = seed;
  s->p0 = templ;
  HM_CUDA(cudaSetDevice(s->device));
  s->ntot = tot;
  s->max_pts = (int)max_points;
  s->pts_blocks = points_blocks(s->max_pts);
  s->nparts_f = field_parts(s->n3);
  s->nparts_p = traj_begin_points_blocks(s->max_pts);
  const size_t C = n_slots, rs = s->rsz;
  DevBuf* grids[] = {&s->w, &s->pw, &s->gw, &s->w0, &s->gw0};
  for (DevBuf* b : grids) HM_TRY(b->alloc(rs * C * s->n3));
  HM_TRY(s->S1.alloc(2 * rs * 3 * C * s->nspec));
  HM_TRY(s->S2.alloc(2 * rs * 3 * C * s->nspec));
  const size_t nt = (size_t)std::max<long long>(tot, 1);
  DevBuf* dbl[] = {&s->rx, &s->ry, &s->rz, &s->mu, &s->smu, &s->zobs,
                   &s->scz, &s->d, &s->pd, &s->gd, &s->d0, &s->gd0};
  for (DevBuf* b : dbl) HM_TRY(b->alloc(8 * nt));
  HM_TRY(s->xr.alloc(sizeof(XRef) * nt));
  HM_TRY(s->work.alloc(s->prec, n_slots, s->N, tot));
  s->pp_host.assign(C, PointParams{});
  s->chain_prob.assign(C, nullptr);
  s->eps_host.assign(C, 0.0);
  HM_TRY(s->pp.alloc(sizeof(PointParams) * C));
  HM_TRY(s->cs.alloc(sizeof(ChainScal) * C));
  HM_TRY(s->chain_id.alloc(sizeof(int) * C));
  HM_TRY(s->prior_part.alloc(8 * C * s->NP));
  HM_TRY(s->pts_part.alloc(8 * C * s->pts_blocks));
  HM_TRY(s->kinb_f.alloc(8 * C * s->nparts_f));
  HM_TRY(s->kinb_p.alloc(8 * C * s->nparts_p));
  HM_TRY(s->kinl_f.alloc(8 * C * s->NP));
  HM_TRY(s->kinl_p.alloc(8 * C * s->pts_blocks));
  HM_TRY(s->eps_dev.alloc(8 * C));
  HM_TRY(s->sig_dev.alloc(8 * C));
  HM_TRY(s->gsig_part.alloc(8 * C * s->pts_blocks));
  HM_CUDA(cudaMemset(s->kinl_p.p, 0, 8 * C * s->pts_blocks));
  HM_CUDA(cudaMemset(s->kinb_p.p, 0, 8 * C * s->nparts_p));
  s->region_of.assign(C, -1);
  s->free_regions.clear();
  // sigma_NL sampling is chosen per job at load: the sigma_NL kernels run on
  // every trajectory and skip the chains that hold it fixed
  s->sample_sig = true;
  for (int r = n_slots - 1; r >= 0; --r) s->free_regions.push_back(r);
  *out = s.release();
  return HM_OK;
}

int hm_slots_count(hm_state* s, int32_t* n_active_out, int32_t* n_slots_out) {
  HM_TRY(slotted_ok(s));
  if (n_active_out) *n_active_out = s->C;
  if (n_slots_out) *n_slots_out = s->C_cap;
  return HM_OK;
}

int hm_slots_load(hm_state* s, hm_problem* job, int32_t chain_id, const double* d_init_host, double eps0,
                  double adapt_target, double sigma_nl0, int32_t* index_out, void* stream) {
  HM_TRY(slotted_ok(s));
  if (!job || !index_out) return fail(HM_EINVAL, "null argument");
  if (!same_field_model(job, s->p0))
    return fail(HM_EINVAL, "the job's grid, precision, device, box and power spectrum must be the state's");
  if (job->n > s->slot_pts) return fail(HM_EINVAL, "catalogue larger than the room of a slot");
  if (job->n > 0 && (!d_init_host || !job->rx.p)) return fail(HM_EINVAL, "catalogue and d_init_host required");
  if (!(eps0 > 0) || !std::isfinite(eps0)) return fail(HM_EINVAL, "eps0 must be finite and > 0");
  if (adapt_target != 0.0 && !(adapt_target > 0.0 && adapt_target < 1.0))
    return fail(HM_EINVAL, "adapt_target must be 0 (off) or in (0, 1)");
  if (!std::isfinite(sigma_nl0) || sigma_nl0 < 0.0) return fail(HM_EINVAL, "sigma_nl0 must be 0 (fixed) or > 0");
  if (s->C >= s->C_cap || s->free_regions.empty()) return fail(HM_ESTATE, "every slot is in use");
  if (job->n > 0) HM_TRY(check_finite(d_init_host, job->n, "d_init"));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const int c = s->C;
  const int r = s->free_regions.back();
  const long long off = (long long)r * s->slot_pts;
  const long long n = job->n;
  if (n > 0) {
    const size_t b = 8 * (size_t)n, o = 8 * (size_t)off;
    const DevBuf* src[] = {&job->rx, &job->ry, &job->rz, &job->mu, &job->xr, &job->smu, &job->zobs, &job->scz};
    DevBuf* dst[] = {&s->rx, &s->ry, &s->rz, &s->mu, &s->xr, &s->smu, &s->zobs, &s->scz};
    for (int k = 0; k < 8; ++k) {
      const size_t m = dst[k] == &s->xr ? sizeof(XRef) / 8 : 1;   // xr: 32 B per point
      HM_CUDA(cudaMemcpyAsync(static_cast<char*>(dst[k]->p) + m * o, src[k]->p, m * b, cudaMemcpyDeviceToDevice,
                              st));
    }
    // pageable host sources: each copy has consumed its source when it returns
    HM_CUDA(cudaMemcpyAsync(static_cast<char*>(s->d.p) + o, d_init_host, b, cudaMemcpyHostToDevice, st));
    HM_CUDA(cudaMemsetAsync(static_cast<char*>(s->pd.p) + o, 0, b, st));
  }
  s->pp_host[c] = point_params(job, off);
  HM_CUDA(cudaMemcpyAsync(s->pp.as<PointParams>() + c, &s->pp_host[c], sizeof(PointParams), cudaMemcpyHostToDevice,
                          st));
  ChainScal x{};
  x.sample_d = 1;
  x.eps = eps0;
  x.sample_sig = sigma_nl0 > 0.0 ? 1 : 0;
  x.sig = sigma_nl0;
  HM_CUDA(cudaMemcpyAsync(s->cs.as<ChainScal>() + c, &x, sizeof(x), cudaMemcpyHostToDevice, st));
  const int id = chain_id;
  HM_CUDA(cudaMemcpyAsync(s->chain_id.as<int>() + c, &id, sizeof(int), cudaMemcpyHostToDevice, st));
  const size_t gb = s->rsz * s->n3;
  HM_CUDA(cudaMemsetAsync(static_cast<char*>(s->w.p) + gb * c, 0, gb, st));
  HM_CUDA(cudaMemsetAsync(static_cast<char*>(s->pw.p) + gb * c, 0, gb, st));
  s->free_regions.pop_back();
  s->region_of[c] = r;
  s->chain_prob[c] = job;
  s->eps_host[c] = eps0;
  s->C = c + 1;
  if (adapt_target != 0.0) HM_CUDA(launch_da(1, 1, adapt_target, nullptr, s->cs.as<ChainScal>() + c, st));
  HM_TRY(eval_chain(s, c, st));
  *index_out = c;
  return HM_OK;
}

int hm_slots_adapt_end(hm_state* s, int32_t index, double* eps_out_host, void* stream) {
  HM_TRY(slotted_ok(s));
  HM_TRY(chain_ok(s, index));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  HM_CUDA(launch_da(1, 0, 0.0, s->eps_dev.as<double>() + index, s->cs.as<ChainScal>() + index, st));
  double e = 0.0;
  HM_CUDA(cudaMemcpyAsync(&e, s->eps_dev.as<double>() + index, 8, cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  s->eps_host[index] = e;
  if (eps_out_host) *eps_out_host = e;
  return HM_OK;
}

int hm_slots_release(hm_state* s, int32_t index, int32_t* moved_from_out, void* stream) {
  HM_TRY(slotted_ok(s));
  HM_TRY(chain_ok(s, index));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const int j = s->C - 1;
  s->free_regions.push_back(s->region_of[index]);
  if (index != j) {
    // the last active chain takes the released index: its grids, scalars
    // and chain word move; its point region stays where it is
    const size_t gb = s->rsz * s->n3;
    DevBuf* grids[] = {&s->w, &s->pw, &s->gw};
    for (DevBuf* b : grids)
      HM_CUDA(cudaMemcpyAsync(static_cast<char*>(b->p) + gb * index, static_cast<char*>(b->p) + gb * j, gb,
                              cudaMemcpyDeviceToDevice, st));
    HM_CUDA(cudaMemcpyAsync(s->cs.as<ChainScal>() + index, s->cs.as<ChainScal>() + j, sizeof(ChainScal),
                            cudaMemcpyDeviceToDevice, st));
    HM_CUDA(cudaMemcpyAsync(s->chain_id.as<int>() + index, s->chain_id.as<int>() + j, sizeof(int),
                            cudaMemcpyDeviceToDevice, st));
    HM_CUDA(cudaMemcpyAsync(s->pp.as<PointParams>() + index, s->pp.as<PointParams>() + j, sizeof(PointParams),
                            cudaMemcpyDeviceToDevice, st));
    s->pp_host[index] = s->pp_host[j];
    s->chain_prob[index] = s->chain_prob[j];
    s->region_of[index] = s->region_of[j];
    s->eps_host[index] = s->eps_host[j];
  }
  s->region_of[j] = -1;
  s->chain_prob[j] = nullptr;
  s->C = j;
  if (moved_from_out) *moved_from_out = index != j ? j : -1;
  return HM_OK;
}

int hm_slots_run(hm_state* s, int32_t n_traj, int32_t n_leapfrog, int32_t use_graph, hm_trace* trace_host,
                 void* stream) {
  HM_TRY(slotted_ok(s));
  if (n_traj < 0 || n_leapfrog <= 0) return fail(HM_EINVAL, "n_traj >= 0 and n_leapfrog > 0 required");
  if (s->C == 0 || n_traj == 0) return HM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  const size_t need = sizeof(hm_trace) * (size_t)n_traj * s->C_cap;
  if (s->trace_cap < need) {
    HM_TRY(s->trace_dev.alloc(need));
    s->trace_cap = need;
    s->drop_graphs();
  }
  HM_CUDA(launch_set_run(s->C, nullptr, 1, s->cs.as<ChainScal>(), st));
  HM_TRY(run_traj_loop(s, n_traj, n_leapfrog, 1, use_graph, st));
  if (trace_host) {
    HM_CUDA(cudaMemcpyAsync(trace_host, s->trace_dev.p, sizeof(hm_trace) * (size_t)n_traj * s->C,
                            cudaMemcpyDeviceToHost, st));
    HM_CUDA(cudaStreamSynchronize(st));
  }
  return HM_OK;
}

// ---------------------------------------------------------------------------
// Chain analytics (eq. int_mc; sections "Convergence", "Monopole and dipole")
// ---------------------------------------------------------------------------
static void analytics_release(hm_state::Analytics& A) {
  DevBuf* bufs[] = {&A.delta_g, &A.vel_g, &A.mean_d, &A.m2_d, &A.mean_vr, &A.m2_vr, &A.shell, &A.sph_cnt,
                    &A.sig_part, &A.met_part, &A.shell_part, &A.sig_prev, &A.sig_cur, &A.count, &A.hist,
                    &A.sph_acc, &A.obs};
  for (DevBuf* b : bufs) b->release();
  A.on = false;
  A.nsh = 0;
  A.max_samples = 0;
  A.radii.clear();
}

static AnArgs an_args(hm_state* s) {
  hm_state::Analytics& A = s->an;
  AnArgs a{};
  a.C = s->C;
  a.N = s->N;
  a.nsh = A.nsh;
  a.max_samples = A.max_samples;
  a.nblk = A.nblk;
  a.n3 = s->n3;
  a.delta = s->p0->delta;
  a.f = s->p0->f;
  a.obs = A.obs.as<double>();
  a.delta_g = A.delta_g.p;
  a.vel_g = A.vel_g.p;
  a.mean_d = A.mean_d.p;
  a.m2_d = A.m2_d.p;
  a.mean_vr = A.mean_vr.p;
  a.m2_vr = A.m2_vr.p;
  a.shell = A.shell.as<unsigned char>();
  a.sph_cnt = A.sph_cnt.as<double>();
  a.sig_part = A.sig_part.as<double>();
  a.met_part = A.met_part.as<double>();
  a.shell_part = A.shell_part.as<double>();
  a.sig_prev = A.sig_prev.as<double>();
  a.sig_cur = A.sig_cur.as<double>();
  a.count = A.count.as<long long>();
  a.hist = A.hist.as<double>();
  a.sph_acc = A.sph_acc.as<double>();
  return a;
}

// One sample of every chain from its current field w: forward plane pass,
// x pass with the velocity weights (3 spectra per chain in S2) and with the
// colouring (1 spectrum per chain after the first C spectra of S1), c2r to
// the real grids, then the analytics kernels.  S1 and S2 are free between
// trajectories (each trajectory starts from the plane pass of w).
static int analytics_sample(hm_state* s, cudaStream_t st) {
  hm_problem* p = s->p0;
  hm_state::Analytics& A = s->an;
  const size_t csz = 2 * s->rsz;
  void* dspec = static_cast<char*>(s->S1.p) + (size_t)s->C * s->nspec * csz;
  HM_CUDA(launch_plane_r2c(s->prec, s->N, s->w.p, s->n3, s->S1.p, s->nspec, s->C, p->tw.p, st));
  HM_CUDA(launch_pencil(s->prec, s->N, PM_VEL, s->S1.p, s->nspec, s->S2.p, s->nspec, s->C, p->tw.p, p->amp.p, st));
  HM_CUDA(launch_pencil(s->prec, s->N, PM_SCALE, s->S1.p, s->nspec, dspec, s->nspec, s->C, p->tw.p, p->ampd.p, st));
  HM_CUDA(launch_plane_c2r(s->prec, s->N, s->S2.p, s->nspec, A.vel_g.p, s->n3, 3 * s->C, p->tw.p, nullptr, st));
  HM_CUDA(launch_plane_c2r(s->prec, s->N, dspec, s->nspec, A.delta_g.p, s->n3, s->C, p->tw.p, nullptr, st));
  HM_CUDA(launch_analytics(s->prec, an_args(s), st));
  return HM_OK;
}

int hm_state_analytics(hm_state* s, int32_t enable, int32_t n_radii, const double* radii_host, int32_t max_samples,
                       void* stream) {
  if (!s) return fail(HM_EINVAL, "null state");
  if (s->slotted) return fail(HM_ESTATE, "chain analytics are not available on a slotted state");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  HM_CUDA(cudaStreamSynchronize(st));   // no sample in flight still uses the buffers
  if (s->gstream) HM_CUDA(cudaStreamSynchronize(s->gstream));
  hm_state::Analytics& A = s->an;
  analytics_release(A);
  if (!enable) return HM_OK;
  if (n_radii < 0 || n_radii > kMaxShells) return fail(HM_EINVAL, "n_radii must be in [0, 32]");
  if (n_radii > 0 && !radii_host) return fail(HM_EINVAL, "null radii");
  if (max_samples < 0) return fail(HM_EINVAL, "max_samples must be >= 0");
  for (int k = 0; k < n_radii; ++k) {
    if (!std::isfinite(radii_host[k]) || radii_host[k] < 0) return fail(HM_EINVAL, "radii must be finite and >= 0");
    if (k > 0 && !(radii_host[k] > radii_host[k - 1])) return fail(HM_EINVAL, "radii must increase");
  }
  const int C = s->C, N = s->N;
  const long long n3 = s->n3;
  A.nsh = n_radii;
  A.radii.assign(radii_host, radii_host + n_radii);
  A.max_samples = max_samples;
  A.nblk = (int)std::min<long long>(512, std::max<long long>(1, n3 / (256 * 8)));
  const size_t fb = (size_t)n3 * s->rsz;
  HM_TRY(A.delta_g.alloc(fb * C));
  HM_TRY(A.vel_g.alloc(fb * 3 * C));
  DevBuf* acc[] = {&A.mean_d, &A.m2_d, &A.mean_vr, &A.m2_vr};
  for (DevBuf* b : acc) {
    HM_TRY(b->alloc(fb * C));
    HM_CUDA(cudaMemsetAsync(b->p, 0, fb * C, st));
  }
  // sphere membership of every node (host, FP64): the innermost sphere
  // |x - o| <= R_k holding node x = i*Delta, 255 for none; chains with the
  // same observer share the computation
  std::vector<unsigned char> shell((size_t)n3 * C, 255);
  std::vector<double> cnt((size_t)C * std::max(1, n_radii), 0.0), obs(3 * C);
  const double dl = s->p0->delta;
  for (int c = 0; c < C; ++c) {
    const double* o = s->chain_prob[c]->obs;
    for (int j = 0; j < 3; ++j) obs[3 * c + j] = o[j];
    int same = -1;
    for (int c2 = 0; c2 < c && same < 0; ++c2)
      if (obs[3 * c2] == o[0] && obs[3 * c2 + 1] == o[1] && obs[3 * c2 + 2] == o[2]) same = c2;
    unsigned char* sc = shell.data() + (size_t)c * n3;
    if (same >= 0) {
      std::memcpy(sc, shell.data() + (size_t)same * n3, (size_t)n3);
      for (int k = 0; k < n_radii; ++k) cnt[(size_t)c * n_radii + k] = cnt[(size_t)same * n_radii + k];
      continue;
    }
    if (n_radii == 0) continue;
    for (int ix = 0; ix < N; ++ix)
      for (int iy = 0; iy < N; ++iy)
        for (int iz = 0; iz < N; ++iz) {
          const double dx = ix * dl - o[0], dy = iy * dl - o[1], dz = iz * dl - o[2];
          const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
          int k = 0;
          while (k < n_radii && r > radii_host[k]) ++k;
          if (k < n_radii) {
            sc[((size_t)ix * N + iy) * N + iz] = (unsigned char)k;
            for (int q = k; q < n_radii; ++q) cnt[(size_t)c * n_radii + q] += 1.0;
          }
        }
  }
  HM_TRY(A.shell.alloc((size_t)n3 * C));
  HM_CUDA(cudaMemcpyAsync(A.shell.p, shell.data(), (size_t)n3 * C, cudaMemcpyHostToDevice, st));
  HM_TRY(A.sph_cnt.alloc(8 * cnt.size()));
  HM_CUDA(cudaMemcpyAsync(A.sph_cnt.p, cnt.data(), 8 * cnt.size(), cudaMemcpyHostToDevice, st));
  HM_TRY(A.obs.alloc(8 * obs.size()));
  HM_CUDA(cudaMemcpyAsync(A.obs.p, obs.data(), 8 * obs.size(), cudaMemcpyHostToDevice, st));
  const size_t nsh1 = (size_t)std::max(1, n_radii);
  HM_TRY(A.sig_part.alloc(8 * 2 * (size_t)C * A.nblk));
  HM_TRY(A.met_part.alloc(8 * (size_t)C * A.nblk));
  HM_TRY(A.shell_part.alloc(8 * 4 * nsh1 * C * A.nblk));
  DevBuf* zero[] = {&A.sig_prev, &A.sig_cur, &A.count};
  for (DevBuf* b : zero) {
    HM_TRY(b->alloc(8 * (size_t)C));
    HM_CUDA(cudaMemsetAsync(b->p, 0, 8 * (size_t)C, st));
  }
  HM_TRY(A.hist.alloc(8 * (size_t)C * std::max(1, max_samples)));
  HM_CUDA(cudaMemsetAsync(A.hist.p, 0, 8 * (size_t)C * std::max(1, max_samples), st));
  HM_TRY(A.sph_acc.alloc(8 * 10 * nsh1 * C));
  HM_CUDA(cudaMemsetAsync(A.sph_acc.p, 0, 8 * 10 * nsh1 * C, st));
  HM_CUDA(cudaStreamSynchronize(st));   // the host staging vectors go out of scope
  A.on = true;
  return HM_OK;
}

int hm_state_analytics_read(hm_state* s, int32_t chain, void* mean_delta_dev, void* var_delta_dev,
                            void* mean_vr_dev, void* var_vr_dev, double* metric_host, int32_t max_metric,
                            double* sphere_host, int64_t* n_samples_out, void* stream) {
  if (!s) return fail(HM_EINVAL, "null state");
  hm_state::Analytics& A = s->an;
  if (!A.on) return fail(HM_ESTATE, "chain analytics are off (hm_state_analytics)");
  if (chain < 0 || chain >= s->C) return fail(HM_EINVAL, "chain out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(s->device));
  if (s->gstream) HM_CUDA(cudaStreamSynchronize(s->gstream));
  long long n = 0;
  HM_CUDA(cudaMemcpyAsync(&n, A.count.as<long long>() + chain, 8, cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  const double scale = n > 1 ? 1.0 / (double)(n - 1) : 0.0;
  const size_t fb = (size_t)s->n3 * s->rsz;
  const size_t off = fb * chain;
  if (mean_delta_dev)
    HM_CUDA(cudaMemcpyAsync(mean_delta_dev, A.mean_d.as<char>() + off, fb, cudaMemcpyDeviceToDevice, st));
  if (mean_vr_dev) HM_CUDA(cudaMemcpyAsync(mean_vr_dev, A.mean_vr.as<char>() + off, fb, cudaMemcpyDeviceToDevice, st));
  if (var_delta_dev) HM_CUDA(launch_an_scale(s->prec, s->n3, A.m2_d.as<char>() + off, var_delta_dev, scale, st));
  if (var_vr_dev) HM_CUDA(launch_an_scale(s->prec, s->n3, A.m2_vr.as<char>() + off, var_vr_dev, scale, st));
  if (metric_host && max_metric > 0 && n >= 2) {
    const long long m = std::min<long long>({n - 1, (long long)A.max_samples, (long long)max_metric});
    if (m > 0)
      HM_CUDA(cudaMemcpyAsync(metric_host, A.hist.as<double>() + (size_t)chain * std::max(1, A.max_samples),
                              8 * (size_t)m, cudaMemcpyDeviceToHost, st));
  }
  std::vector<double> sph((size_t)10 * std::max(1, A.nsh));
  if (sphere_host && A.nsh > 0)
    HM_CUDA(cudaMemcpyAsync(sph.data(), A.sph_acc.as<double>() + (size_t)chain * 10 * A.nsh, 8 * 10 * (size_t)A.nsh,
                            cudaMemcpyDeviceToHost, st));
  HM_CUDA(cudaStreamSynchronize(st));
  if (sphere_host)
    for (int k = 0; k < A.nsh; ++k)
      for (int q = 0; q < 5; ++q) {
        sphere_host[(k * 5 + q) * 2] = sph[(k * 5 + q) * 2];
        sphere_host[(k * 5 + q) * 2 + 1] = sph[(k * 5 + q) * 2 + 1] * scale;
      }
  if (n_samples_out) *n_samples_out = n;
  return HM_OK;
}

int hm_state_profile(hm_state* s, int32_t enable) {
  if (!s) return fail(HM_EINVAL, "null state");
  HM_CUDA(cudaSetDevice(s->device));
  if (enable) {
    if (!s->prof) s->prof = std::make_unique<Prof>();
    for (int k = 0; k < KK_COUNT; ++k) {
      s->prof->ms[k] = 0.0;
      s->prof->launches[k] = 0;
    }
  } else {
    HM_TRY(profile_collect(s));
    // a graph captured with profiling holds these events: drop it first
    s->drop_graphs(true);
    s->prof.reset();
  }
  return HM_OK;
}

int hm_state_profile_collect(hm_state* s) {
  if (!s) return fail(HM_EINVAL, "null state");
  HM_CUDA(cudaSetDevice(s->device));
  return profile_collect(s);
}

int hm_state_profile_read(hm_state* s, int32_t max_kinds, double* ms_out, int64_t* launches_out, int32_t* n_kinds) {
  if (!s) return fail(HM_EINVAL, "null state");
  if (n_kinds) *n_kinds = KK_COUNT;
  if (!s->prof) return fail(HM_ESTATE, "profiling is not enabled on this state");
  HM_CUDA(cudaSetDevice(s->device));
  HM_TRY(profile_collect(s));
  for (int k = 0; k < KK_COUNT && k < max_kinds; ++k) {
    if (ms_out) ms_out[k] = s->prof->ms[k];
    if (launches_out) launches_out[k] = s->prof->launches[k];
  }
  return HM_OK;
}

const char* hm_kernel_kind_name(int32_t kind) {
  if (kind < 0 || kind >= KK_COUNT) return "";
  return kKindNames[kind];
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Posterior gradient without any device allocation.
//
// Some callers cannot let a library allocate device memory: code that runs
// inside another framework's allocator or memory pool, which must account for
// every device byte itself, and hosts that budget device memory up front and
// allow no allocation once they run (cudaMalloc and cudaFree may also
// synchronise the device, which such hosts cannot afford mid-run).
// hm_logpost_grad_noalloc serves them by taking its scratch from one
// statically sized device array that every GPU loading this library holds
// until the process exits.  It launches the same kernels as hm_logpost_grad,
// all on the caller's stream, and never calls cudaMalloc, cudaFree or any
// other allocating routine.
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = 4u << 20;   // 4 MiB per device
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
// Device address of the array, looked up once per device with that device
// current (host code cannot use the symbol itself as a device pointer).
static std::once_flag g_noalloc_once[kNoAllocMaxDevices];
static void* g_noalloc_base[kNoAllocMaxDevices];

// The per-call constants, passed by value, and the state that must start at
// zero on every call (chain scalars, chain word, bucket counts).
__global__ void k_noalloc_init(PointParams P, PointParams* pp, ChainScal* cs, int* cid, int* cnt, int ncnt) {
  if (threadIdx.x == 0) {
    *pp = P;
    *cs = ChainScal{};
    *cid = 0;
  }
  for (int i = threadIdx.x; i < ncnt; i += blockDim.x) cnt[i] = 0;
}

namespace {
struct NoAllocLayout {
  size_t S1, S2, cx, slot, pos, cnt, off, rec, part, lk, prior, pts, kin, pp, cs, cid, total;
};

NoAllocLayout noalloc_layout(const hm_problem* p) {
  NoAllocLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) / 256 * 256;
    return at;
  };
  const size_t n = (size_t)std::max<long long>(p->n, 1);
  const size_t rsz = p->rsz;
  const size_t recsz = p->prec == HM_FP32 ? sizeof(PtRec<float>) : sizeof(PtRec<double>);
  const size_t NB = (size_t)p->N * plane_split(p->N);
  const size_t pb = (size_t)points_blocks((int)p->n);
  L.S1 = take(2 * rsz * 3 * p->nspec);
  L.S2 = take(2 * rsz * 3 * p->nspec);
  L.cx = take(4 * n);
  L.slot = take(4 * n);
  L.pos = take(4 * n);
  L.cnt = take(4 * 2 * NB);
  L.off = take(4 * 2 * (NB + 1));
  L.rec = take(2 * recsz * n);
  L.part = take(rsz * 12 * n);
  L.lk = take(8 * 6 * n);
  L.prior = take(8 * NB);
  L.pts = take(8 * pb);
  L.kin = take(8 * std::max(NB, pb));
  L.pp = take(sizeof(PointParams));
  L.cs = take(sizeof(ChainScal));
  L.cid = take(sizeof(int));
  L.total = o;
  return L;
}
}  // namespace

extern "C" int hm_logpost_grad_noalloc(hm_problem* p, const void* w_dev, const double* d_dev, double* psi_dev,
                                       void* grad_w_dev, double* grad_d_dev, void* stream) {
  if (!p || !w_dev || !psi_dev || !grad_w_dev) return fail(HM_EINVAL, "null argument");
  if (p->n > 0 && (!d_dev || !grad_d_dev)) return fail(HM_EINVAL, "null distance argument");
  if (!p->rx.p) return fail(HM_ESTATE, "no catalogue set");
  if (p->device < 0 || p->device >= kNoAllocMaxDevices)
    return fail(HM_EINVAL, "device ordinal out of range for the static scratch");
  const NoAllocLayout L = noalloc_layout(p);
  if (L.total > kNoAllocScratchBytes)
    return fail(HM_EINVAL, "problem too large for the no-allocation path: needs " + std::to_string(L.total) +
                               " bytes of scratch, the static array holds " +
                               std::to_string(kNoAllocScratchBytes) + " (use hm_logpost_grad)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  HM_CUDA(cudaSetDevice(p->device));
  // once per device, with that device current: the array's device address
  // (host threads making their first call at the same time wait for one
  // lookup; a failed lookup is retried by the next call)
  cudaError_t look = cudaSuccess;
  try {
    std::call_once(g_noalloc_once[p->device], [&] {
      void* base = nullptr;
      look = cudaGetSymbolAddress(&base, g_noalloc_scratch);
      if (look != cudaSuccess) throw look;
      g_noalloc_base[p->device] = base;
    });
  } catch (cudaError_t e) {
    return fail(HM_ECUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
  }
  char* b = static_cast<char*>(g_noalloc_base[p->device]);
  const int NB = p->N * plane_split(p->N);
  k_noalloc_init<<<1, 64, 0, st>>>(point_params(p, 0), reinterpret_cast<PointParams*>(b + L.pp),
                                   reinterpret_cast<ChainScal*>(b + L.cs), reinterpret_cast<int*>(b + L.cid),
                                   reinterpret_cast<int*>(b + L.cnt), 2 * NB);
  HM_CUDA(cudaGetLastError());
  PointArrays pa{};
  pa.rx = p->rx.as<double>();
  pa.ry = p->ry.as<double>();
  pa.rz = p->rz.as<double>();
  pa.mu = p->mu.as<double>();
  pa.xr = p->xr.as<XRef>();
  pa.ismu2 = p->smu.as<double>();
  pa.zobs = p->zobs.as<double>();
  pa.scz = p->scz.as<double>();
  pa.d = const_cast<double*>(d_dev);
  pa.pd = nullptr;
  pa.gd = grad_d_dev;
  pa.cx = reinterpret_cast<int*>(b + L.cx);
  pa.slot = reinterpret_cast<int*>(b + L.slot);
  pa.pos = reinterpret_cast<int*>(b + L.pos);
  pa.cnt = reinterpret_cast<int*>(b + L.cnt);
  pa.cnt_next = pa.cnt + NB;
  pa.off = reinterpret_cast<int*>(b + L.off);
  pa.rec = b + L.rec;
  pa.part = b + L.part;
  pa.lk = reinterpret_cast<double*>(b + L.lk);
  pa.ntot = p->n;
  const PointParams* pp = reinterpret_cast<const PointParams*>(b + L.pp);
  ChainScal* cs = reinterpret_cast<ChainScal*>(b + L.cs);
  double* prior_part = reinterpret_cast<double*>(b + L.prior);
  double* pts_part = reinterpret_cast<double*>(b + L.pts);
  double* kin_part = reinterpret_cast<double*>(b + L.kin);
  void* S1 = b + L.S1;
  void* S2 = b + L.S2;
  const int maxp = (int)p->n, pb = points_blocks((int)p->n);
  PlanePoints pts{};
  pts.off = pa.off;
  pts.rec = pa.rec;
  pts.part = pa.part;
  pts.ntot = pa.ntot;
  pts.inv_delta = 1.0 / p->delta;
  // the evaluation of hm_logpost_grad, every kernel on the caller's stream
  HM_CUDA(launch_points_prep(1, maxp, pp, pa, st));
  HM_CUDA(launch_points_place(p->prec, 1, maxp, pp, pa, cs, st));
  HM_CUDA(launch_plane_r2c(p->prec, p->N, w_dev, p->n3, S1, p->nspec, 1, p->tw.p, st));
  HM_CUDA(launch_pencil(p->prec, p->N, PM_VEL, S1, p->nspec, S2, p->nspec, 1, p->tw.p, p->amp.p, st));
  HM_CUDA(launch_plane_c2r_gather(p->prec, p->N, S2, p->nspec, pts, 3, p->tw.p, st));
  HM_CUDA(launch_points_lik(p->prec, 1, maxp, pp, pa, pts_part, pb, GM_GRAD, kin_part, cs, nullptr, st));
  HM_CUDA(launch_plane_r2c_scatter(p->prec, p->N, pts, S1, p->nspec, 3, p->tw.p, st));
  HM_CUDA(launch_pencil(p->prec, p->N, PM_ADJ, S1, p->nspec, S2, p->nspec, 1, p->tw.p, p->amp.p, st, pts.off));
  FieldEpi epi{};
  epi.w = const_cast<void*>(w_dev);
  epi.pw = nullptr;
  epi.gw = grad_w_dev;
  epi.prior_part = prior_part;
  epi.kin_part = kin_part;
  epi.cs = cs;
  epi.grid_stride = p->n3;
  epi.mode = GM_GRAD;
  HM_CUDA(launch_plane_c2r(p->prec, p->N, S2, p->nspec, nullptr, 0, 1, p->tw.p, &epi, st));
  HM_CUDA(launch_finalize(1, prior_part, NB, pts_part, pb, nullptr, 0, nullptr, 0, FIN_PSI, 0ull,
                          reinterpret_cast<const int*>(b + L.cid), cs, nullptr, st));
  HM_CUDA(cudaMemcpyAsync(psi_dev, &cs->psi, sizeof(double), cudaMemcpyDeviceToDevice, st));
  return HM_OK;
}
