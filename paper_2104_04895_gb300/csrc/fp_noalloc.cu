// fp_rates4_noalloc: the rate computation of fp_rates4_device without any device allocation.
//
// Who needs it: callers that must not call cudaMalloc / cudaFree while they run -- for example a host
// application whose device memory is owned by its own pool allocator with a fixed budget, or a
// latency-critical caller that cannot afford the device-wide synchronisation cudaFree implies.  The
// fp_rates4 paths grow per-context scratch (Bose weight table, per-work-item partial sums, queue
// counter) on demand with cudaMalloc; this variant takes all of that scratch from one statically
// sized device array instead, so a call allocates nothing.  The context itself (fp_init) and its
// mode tables (fp_modes / fp_set_modes) must have been created beforehand.
//
// The array below is a file-scope __device__ variable: every GPU that loads the library holds
// kScratchBytes of it until the process exits.  Host code must not use its name as a device address
// (in host code it is only a stand-in symbol); the device address is obtained once per device with
// cudaGetSymbolAddress, during the first call on that device, with that device current.  That first
// call should therefore happen before any stream capture is started.  All calls share the array and
// it keeps the contents of the last call, so the parts that must start at zero (queue counter,
// accepted-term counters) are cleared on every call; two calls whose work overlaps on the GPU (other
// streams, other contexts on the same device, other host threads) race on it and must be serialised
// by the caller.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fp_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_fp_scratch[kScratchBytes];

std::mutex g_scratch_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

int nfail(fp_ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

// Device address of the static scratch on the current device (set up once per device).
cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_fp_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace

#define NA_CUDA(ctx, call)                                                               \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return nfail((ctx), FP_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" int fp_rates4_noalloc(fp_ctx* c, int nT, const double* T, double sb, const fp_rates_opts* user,
                                 double* d_out, fp_stats* stats) {
  if (!c) return FP_EINVAL;
  if (!d_out) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: NULL output");
  fp_rates_opts o;
  fp_default_opts(&o);
  if (user) {
    o = *user;
    if (o.window == 0.0) o.window = 2.0;
    if (o.sigma_min == 0.0) o.sigma_min = 1e-10;
  }
  if (!c->have_modes) return nfail(c, FP_ESTATE, "fp_rates4_noalloc: call fp_modes or fp_set_modes first");
  if (nT < 1 || nT > fp::kMaxT || !T) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: nT must be in [1, 16]");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0) || !std::isfinite(T[i]))
      return nfail(c, FP_EINVAL, "fp_rates4_noalloc: temperatures must be > 0");
  if (!(sb > 0.0) || !std::isfinite(sb)) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: scalebroad must be > 0");
  if (!(o.window > 0.0) || !(o.sigma_min > 0.0))
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: window, sigma_min must be > 0");
  if (o.precision != FP_PREC_FP64 && o.precision != FP_PREC_MIXED)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: unknown precision");
  if (o.dq_mode != 0 && o.dq_mode != 1) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: dq_mode must be 0 or 1");
  if (c->device < 0 || c->device >= kMaxDevices) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: device ordinal too large");
  const int N = c->N, nb = c->nb;
  const int q_end = o.q_end <= 0 ? N : o.q_end;
  if (o.q_begin < 0 || o.q_begin > q_end || q_end > N) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: bad q range");
  const int nq_sel = q_end - o.q_begin;

  int J = o.block_j0;
  if (J <= 0) {
    J = nb;
    while (J > 1 && fp::rates_smem_bytes(o.precision, nb, J, c->G, c->nquart, nT, 384) > 112 * 1024) {
      int nj = J - 1;
      while (nj > 1 && nb % nj) --nj;
      J = nj;
    }
  }
  if (J < 1 || nb % J) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: block_j0 must divide nb");
  int threads = o.threads;
  if (threads <= 0) {
    threads = 32 * J;
    while (threads < 160) threads += 32 * J;
  }
  if (threads % (32 * J) || threads > 384)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: threads must be a multiple of 32*block_j0, <= 384");
  const size_t smem = fp::rates_smem_bytes(o.precision, nb, J, c->G, c->nquart, nT, threads);
  if (smem > 227 * 1024) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: tile does not fit in shared memory");

  // scratch layout: counters | temperatures | mode mask | Bose weights | per-item partials
  const size_t nm = (size_t)N * nb;
  const int nchunk = nb / J;
  const size_t off_cnt = 0;
  const size_t off_T = up256(4 * sizeof(unsigned long long));
  const size_t off_mask = off_T + up256(fp::kMaxT * sizeof(double));
  const size_t off_wt = off_mask + (o.mode_mask ? up256(nm) : 0);
  const size_t off_part = off_wt + up256(3 * nm * nT * sizeof(double));
  int t1 = o.k1_tile > 0 ? o.k1_tile : (N + 511) / 512;
  auto part_bytes = [&](int tile) {
    return (size_t)((N + tile - 1) / tile) * nq_sel * nchunk * J * nT * sizeof(double);
  };
  if (o.k1_tile <= 0)
    while (t1 < N && off_part + part_bytes(t1) > kScratchBytes) t1 = t1 < 8 ? t1 + 1 : t1 + t1 / 4;
  if (t1 > N) t1 = N;
  const size_t need = off_part + part_bytes(t1);
  if (need > kScratchBytes)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: this problem needs " + std::to_string(need) +
                                   " bytes of scratch; the static scratch holds " + std::to_string(kScratchBytes) +
                                   " bytes (use fp_rates4_device)");
  const int ntile = (N + t1 - 1) / t1;
  const long long n_items = (long long)ntile * nq_sel * nchunk;

  NA_CUDA(c, cudaSetDevice(c->device));
  unsigned char* base = nullptr;
  NA_CUDA(c, scratch_address(c->device, &base));
  unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(base + off_cnt);
  double* d_T = reinterpret_cast<double*>(base + off_T);
  unsigned char* d_mask = o.mode_mask ? base + off_mask : nullptr;
  double* d_wt = reinterpret_cast<double*>(base + off_wt);
  double* d_part = reinterpret_cast<double*>(base + off_part);
  cudaStream_t s = c->stream;

  NA_CUDA(c, cudaMemcpyAsync(d_T, T, nT * sizeof(double), cudaMemcpyHostToDevice, s));
  if (d_mask) NA_CUDA(c, cudaMemcpyAsync(d_mask, o.mode_mask, nm, cudaMemcpyHostToDevice, s));
  NA_CUDA(c, fp::launch_weights(c, nT, d_T, d_wt, s));

  fp::RatesArgs a;
  a.N = N;
  a.nb = nb;
  a.natoms = c->natoms;
  a.nT = nT;
  a.L = c->L;
  a.G = c->G;
  a.nquart = c->nquart;
  for (int d = 0; d < 3; ++d) {
    a.grid[d] = c->grid[d];
    a.Lfac[d] = c->L / c->grid[d];
  }
  a.J = J;
  a.t1 = t1;
  a.nchunk = nchunk;
  a.ntile = ntile;
  a.q_begin = o.q_begin;
  a.nq_sel = nq_sel;
  a.n_items = n_items;
  a.omega = c->d_omega;
  a.evec = c->d_evec;
  a.vel = c->d_vel;
  a.wt = d_wt;
  a.qmeta = c->d_qmeta;
  a.qfc = c->d_qfc;
  a.gmeta = c->d_gmeta;
  a.grp_qstart = c->d_grp_qstart;
  a.grp_q = c->d_grp_q;
  a.kl_start = c->d_kl_start;
  a.kl_grp = c->d_kl_grp;
  a.tw = c->d_tw;
  a.mask = d_mask;
  a.sb = sb;
  a.window = o.window;
  a.sigma_min = o.sigma_min;
  const double* B = c->rec;
  const double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6]);
  a.dq = std::cbrt(std::fabs(detB) / (double)N);
  a.dq_mode = o.dq_mode;
  for (int i = 0; i < 9; ++i) a.rec[i] = B[i];
  a.partial = d_part;
  a.counter = d_cnt;
  a.counts = d_cnt + 1;

  const int per_sm = fp::rates_max_ctas_per_sm(o.precision, threads, smem);
  if (per_sm < 1) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: kernel tile cannot be resident on an SM");
  int nsm = 0;
  NA_CUDA(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  long long ctas = (long long)nsm * per_sm;
  if (ctas > n_items) ctas = n_items > 0 ? n_items : 1;

  // the shared array keeps the previous call's contents: clear what must start at zero
  NA_CUDA(c, cudaMemsetAsync(d_cnt, 0, 4 * sizeof(unsigned long long), s));
  NA_CUDA(c, cudaMemsetAsync(d_out, 0, (size_t)nT * nm * sizeof(double), s));
  const double conv = fp::kConv;
  const double pref = fp::kPi * fp::kHbar * fp::kHbar * conv * conv * conv * conv / (8.0 * (double)N * (double)N);
  NA_CUDA(c, cudaEventRecord(c->ev0, s));
  if (n_items > 0) {
    NA_CUDA(c, fp::launch_rates(a, o.precision, threads, (int)ctas, smem, s));
    NA_CUDA(c, fp::launch_reduce(a, pref, d_out, q_end, s));
  }
  NA_CUDA(c, cudaEventRecord(c->ev1, s));
  unsigned long long counts[4] = {0, 0, 0, 0};
  NA_CUDA(c, cudaMemcpyAsync(counts, d_cnt, sizeof(counts), cudaMemcpyDeviceToHost, s));
  NA_CUDA(c, cudaStreamSynchronize(s));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    double nsel = 0;
    if (o.mode_mask) {
      for (int q = o.q_begin; q < q_end; ++q)
        for (int j = 0; j < nb; ++j) nsel += o.mode_mask[(size_t)q * nb + j] ? 1 : 0;
    } else {
      nsel = (double)nq_sel * nb;
    }
    stats->candidates = 3.0 * nsel * (double)N * (double)N * (double)nb * nb * nb;
    for (int p = 0; p < 3; ++p) stats->accepted[p] = (double)counts[1 + p];
    const double pairs = 0.5 * (double)N * (double)(N + 1);
    const double per_pair = 8.0 * (9.0 * J * nb * c->G + 2.0 * J * (double)nb * nb * nb * nb);
    const double prolog = 8.0 * 9.0 * J * nb * 9.0 * c->nquart;
    stats->flops = (double)nq_sel * nchunk * (pairs * per_pair + (double)N * prolog);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    stats->ms = ms;
    stats->tile[0] = J;
    stats->tile[1] = t1;
    stats->tile[2] = threads;
    stats->tile[3] = (int)ctas;
  }
  return FP_OK;
}
