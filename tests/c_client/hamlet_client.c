/* A plain C client of libhamlet: no Python, no torch.  It reads a problem
 * (grid, catalogue, distance-prior table, a field w and distances d) from a
 * binary file, evaluates Psi and its gradient through hm_logpost_grad on
 * device buffers it allocates itself, runs two HMC trajectories of a
 * one-chain state, and writes the results to a binary file.
 *
 * input  (little-endian): int32 N, int32 precision, int64 n, double L,
 *        double sigma_nl, double prior_d0, double prior_bin, int32 nbins,
 *        int32 pad, double logdens[nbins], double rhat[3n], double mu[n],
 *        double sigma_mu[n], double cz[n], double w[N^3], double d[n]
 *        (nbins = 0: the default distance prior, eq. D built by the library
 *        from the redshifts, bins of prior_bin or 5 Mpc/h when <= 0)
 * output: double psi, double grad_w[N^3], double grad_d[n],
 *         double H_new[2], int32 accept[2], int32 rc
 * usage:  hamlet_client in.bin out.bin
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "hamlet.h"

static int rd(FILE* f, void* p, size_t sz, size_t n) { return fread(p, sz, n, f) == n ? 0 : -1; }

#define CK(x)                                                                           \
  do {                                                                                  \
    int rc_ = (x);                                                                      \
    if (rc_ != 0) {                                                                     \
      fprintf(stderr, "%s failed: %d (%s)\n", #x, rc_, hm_last_error());                \
      return 2;                                                                         \
    }                                                                                   \
  } while (0)
#define CU(x)                                                                           \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess) {                                                            \
      fprintf(stderr, "%s failed: %s\n", #x, cudaGetErrorString(e_));                   \
      return 3;                                                                         \
    }                                                                                   \
  } while (0)

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s in.bin out.bin\n", argv[0]);
    return 1;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  int32_t N, prec, nbins, pad;
  int64_t n;
  double L, snl, d0, bin;
  if (rd(f, &N, 4, 1) || rd(f, &prec, 4, 1) || rd(f, &n, 8, 1) || rd(f, &L, 8, 1) || rd(f, &snl, 8, 1) ||
      rd(f, &d0, 8, 1) || rd(f, &bin, 8, 1) || rd(f, &nbins, 4, 1) || rd(f, &pad, 4, 1))
    return 1;
  const size_t n3 = (size_t)N * N * N;
  double* logd = malloc(8 * (size_t)(nbins > 0 ? nbins : 1));
  double* rhat = malloc(8 * 3 * (size_t)n);
  double* mu = malloc(8 * (size_t)n);
  double* smu = malloc(8 * (size_t)n);
  double* cz = malloc(8 * (size_t)n);
  double* w = malloc(8 * n3);
  double* d = malloc(8 * (size_t)n);
  if (rd(f, logd, 8, nbins) || rd(f, rhat, 8, 3 * n) || rd(f, mu, 8, n) || rd(f, smu, 8, n) || rd(f, cz, 8, n) ||
      rd(f, w, 8, n3) || rd(f, d, 8, n))
    return 1;
  fclose(f);

  hm_problem_desc desc;
  memset(&desc, 0, sizeof(desc));
  desc.N = N;
  desc.precision = prec;
  desc.L = L;
  desc.prior_kind = HM_PRIOR_TABLE;
  desc.omega_m = 0.3;
  desc.omega_b = 0.05;
  desc.h = 0.7;
  desc.n_s = 0.96;
  desc.sigma8 = 0.8;
  desc.T_cmb = 2.7255;
  desc.f_growth = -1.0;
  desc.sigma_nl = snl;
  desc.prior_d0 = d0;
  desc.prior_bin = bin;
  desc.prior_nbins = nbins;
  desc.prior_logdens_host = nbins > 0 ? logd : NULL;
  desc.device = 0;
  hm_problem* p = NULL;
  CK(hm_init_problem(&desc, &p));
  CK(hm_set_catalog(p, n, rhat, mu, smu, cz, NULL));

  /* caller-owned device buffers (FP64 field: precision HM_FP64) */
  double *w_dev, *d_dev, *psi_dev, *gw_dev, *gd_dev;
  CU(cudaMalloc((void**)&w_dev, 8 * n3));
  CU(cudaMalloc((void**)&d_dev, 8 * (size_t)n));
  CU(cudaMalloc((void**)&psi_dev, 8));
  CU(cudaMalloc((void**)&gw_dev, 8 * n3));
  CU(cudaMalloc((void**)&gd_dev, 8 * (size_t)n));
  CU(cudaMemcpy(w_dev, w, 8 * n3, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(d_dev, d, 8 * (size_t)n, cudaMemcpyHostToDevice));
  CK(hm_logpost_grad(p, w_dev, d_dev, psi_dev, gw_dev, gd_dev, NULL));
  double psi;
  double* gw = malloc(8 * n3);
  double* gd = malloc(8 * (size_t)n);
  CU(cudaMemcpy(&psi, psi_dev, 8, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(gw, gw_dev, 8 * n3, cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(gd, gd_dev, 8 * (size_t)n, cudaMemcpyDeviceToHost));

  /* a one-chain state from w = 0, d: two trajectories of 10 steps */
  hm_state* s = NULL;
  CK(hm_state_create(p, 3, d, &s));
  hm_trace tr[2];
  const double eps = 0.03;
  CK(hm_run_chain(s, 2, 10, &eps, 1, 1, tr, NULL));

  FILE* o = fopen(argv[2], "wb");
  if (!o) return 1;
  const double h[2] = {tr[0].H_new, tr[1].H_new};
  const int32_t acc[2] = {tr[0].accept, tr[1].accept};
  const int32_t rc = 0;
  fwrite(&psi, 8, 1, o);
  fwrite(gw, 8, n3, o);
  fwrite(gd, 8, (size_t)n, o);
  fwrite(h, 8, 2, o);
  fwrite(acc, 4, 2, o);
  fwrite(&rc, 4, 1, o);
  fclose(o);
  hm_destroy_state(s);
  hm_destroy_problem(p);
  cudaFree(w_dev);
  cudaFree(d_dev);
  cudaFree(psi_dev);
  cudaFree(gw_dev);
  cudaFree(gd_dev);
  free(logd), free(rhat), free(mu), free(smu), free(cz), free(w), free(d), free(gw), free(gd);
  return 0;
}
