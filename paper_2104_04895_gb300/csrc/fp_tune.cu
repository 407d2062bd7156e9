// Autotuner of the rate kernel's tiles: times each candidate (branch chunk J dividing nb, q'-tile,
// threads per block) on a sample of q-points with the real kernel and remembers the fastest per
// (precision, one or several temperatures) in the context.
#include <cstring>
#include <vector>

#include "fp_internal.cuh"

namespace {
int tfail(fp_ctx* c, int code, const std::string& m) {
  c->err = m;
  return code;
}
}  // namespace

extern "C" int fp_autotune(fp_ctx* c, int nT, const double* T, double scalebroad, fp_rates_opts* opts,
                           double* best_ms) {
  if (!c || !opts) return FP_EINVAL;
  if (!c->have_modes) return tfail(c, FP_ESTATE, "fp_autotune: call fp_modes or fp_set_modes first");
  if (nT < 1 || nT > fp::kMaxT || !T) return tfail(c, FP_EINVAL, "fp_autotune: nT must be in [1, 8]");
  if (opts->precision < FP_PREC_FP64 || opts->precision > FP_PREC_DOUBLE_FLOAT)
    return tfail(c, FP_EINVAL, "fp_autotune: unknown precision");
  const int N = c->N, nb = c->nb;
  const int maxth = nb == 3 ? 128 : nb == 6 ? 224 : 160;
  // q sample: about 64 x 512^2 (q, q', q'') triples per trial (a few percent of a 512-point grid), and at
  // least 4 q-points, so that every candidate is timed on the same, bounded work
  long long want = (64LL * 512 * 512) / ((long long)N * N);
  int nq = (int)(want < 4 ? 4 : want);
  if (nq > N) nq = N;
  double* d_out = nullptr;
  if (cudaSetDevice(c->device) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&d_out), (size_t)nT * N * nb * sizeof(double)) != cudaSuccess)
    return tfail(c, FP_ENOMEM, "fp_autotune: cannot allocate the trial output");
  double best = 1e300;
  int bj = 0, bt = 0, bth = 0;
  const int t1s[] = {1, 2, 4};
  for (int J = 1; J <= nb; ++J) {
    if (nb % J || J * nb * nb > maxth) continue;
    const int rows = J * nb * nb;
    const int th_min = ((rows + 31) / 32) * 32;
    for (int th = th_min; th <= maxth && th <= th_min; th += 32) {  // extra threads would idle
      for (int t1 : t1s) {
        fp_rates_opts o = *opts;
        o.block_j0 = J;
        o.k1_tile = t1;
        o.threads = th;
        o.q_begin = 0;
        o.q_end = nq;
        o.no_graph = 1;
        o.mode_mask = nullptr;
        fp_stats st;
        double ms = 0.0;
        int rc = FP_OK;
        for (int rep = 0; rep < 2 && rc == FP_OK; ++rep) {  // first run warms up
          rc = fp_rates4_device(c, nT, T, scalebroad, &o, d_out, &st);
          ms = st.ms;
        }
        if (rc != FP_OK) continue;  // a tile this device cannot hold
        if (ms < best) {
          best = ms;
          bj = J;
          bt = t1;
          bth = th;
        }
      }
    }
  }
  cudaFree(d_out);
  if (bj == 0) return tfail(c, FP_EINVAL, "fp_autotune: no tile could run");
  int* tt = c->tuned[opts->precision][nT == 1 ? 0 : 1];
  tt[0] = bj;
  tt[1] = bt;
  tt[2] = bth;
  opts->block_j0 = bj;
  opts->k1_tile = bt;
  opts->threads = bth;
  if (best_ms) *best_ms = best;
  c->err.clear();
  return FP_OK;
}
