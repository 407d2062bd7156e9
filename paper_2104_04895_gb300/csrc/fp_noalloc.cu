// fp_rates4_noalloc: the rate computation of fp_rates4_device without any device allocation.
//
// Who needs it: callers that must not call cudaMalloc / cudaFree while they run -- for example a host
// application whose device memory is owned by its own pool allocator with a fixed budget, or a
// latency-critical caller that cannot afford the device-wide synchronisation cudaFree implies.  The
// fp_rates4 paths grow per-context scratch (Bose weight tables, FP32 copies of the mode tables,
// per-work-item partial sums, counters) on demand with cudaMalloc; this variant takes all of that
// scratch from one statically sized device array instead, so a call allocates nothing.  The context itself (fp_init) and its
// mode tables (fp_modes / fp_set_modes) must have been created beforehand.
//
// The array below is a file-scope __device__ variable: every GPU that loads the library holds
// kScratchBytes of it until the process exits.  Host code must not use its name as a device address
// (in host code it is only a stand-in symbol); the device address is obtained once per device with
// cudaGetSymbolAddress, during the first call on that device, with that device current.  That first
// call should therefore happen before any stream capture is started.  Under lazy module loading (CUDA's
// default) the first call on a device may also load the module and reserve the array on that device, so a
// caller that must not see device memory taken makes one warm-up call first.  All calls share the array and
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
  if (nT < 1 || nT > fp::kMaxT || !T) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: nT must be in [1, 8]");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0) || !std::isfinite(T[i]))
      return nfail(c, FP_EINVAL, "fp_rates4_noalloc: temperatures must be > 0");
  if (!(sb > 0.0) || !std::isfinite(sb)) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: scalebroad must be > 0");
  if (!(o.window > 0.0) || !(o.sigma_min > 0.0))
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: window, sigma_min must be > 0");
  if (o.precision != FP_PREC_FP64 && o.precision != FP_PREC_MIXED && o.precision != FP_PREC_DOUBLE_FLOAT)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: unknown precision");
  if (o.dq_mode != 0 && o.dq_mode != 1) return nfail(c, FP_EINVAL, "fp_rates4_noalloc: dq_mode must be 0 or 1");
  if (o.process_mask < 0 || o.process_mask > 7)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: process_mask must be in [0, 7]");
  if (o.nu_select < 0 || o.nu_select > 2)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: nu_select must be 0, 1 or 2");
  if (o.no_time_reversal != 0 && o.no_time_reversal != 1)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: no_time_reversal must be 0 or 1");
  if (o.tensor_cores != 0 && o.tensor_cores != 1)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: tensor_cores must be 0 or 1");
  if (c->device < 0 || c->device >= kMaxDevices)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: device ordinal too large");
  NA_CUDA(c, cudaSetDevice(c->device));

  // everything except the per-item partial sums has a fixed size; the partials get the rest, and the
  // plan enlarges the q' tile until they fit
  std::string err;
  fp::Selection sel;
  int rc = fp::make_selection(c, o, true, &sel, &err);
  if (rc) return nfail(c, rc, "fp_rates4_noalloc: " + err);
  fp::Plan p0;
  fp_rates_opts o_probe = o;
  if (o_probe.k1_tile <= 0) o_probe.k1_tile = c->N;  // smallest partials, for the fixed-size part
  rc = fp::plan_rates(c, o_probe, nT, sel, 0, &p0, &err);
  if (rc) return nfail(c, rc, "fp_rates4_noalloc: " + err);
  size_t sz[fp::kScratchParts], fixed = 0;
  fp::scratch_sizes(c, p0, nT, sz);
  for (int i = 0; i < fp::kScratchParts; ++i)
    if (i != fp::kScratchPartial) fixed += sz[i];
  if (fixed + sz[fp::kScratchPartial] > kScratchBytes)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: this problem needs at least " +
                                   std::to_string(fixed + sz[fp::kScratchPartial]) +
                                   " bytes of scratch; the static scratch holds " + std::to_string(kScratchBytes) +
                                   " bytes (use fp_rates4_device)");
  fp::Plan p;
  rc = fp::plan_rates(c, o, nT, sel, kScratchBytes - fixed - 256, &p, &err);
  if (rc) return nfail(c, rc, "fp_rates4_noalloc: " + err);
  fp::scratch_sizes(c, p, nT, sz);
  size_t total = 0;
  for (size_t x : sz) total += x;
  if (total > kScratchBytes)
    return nfail(c, FP_EINVAL, "fp_rates4_noalloc: this problem needs " + std::to_string(total) +
                                   " bytes of scratch; the static scratch holds " + std::to_string(kScratchBytes) +
                                   " bytes (use fp_rates4_device)");

  unsigned char* b = nullptr;
  NA_CUDA(c, scratch_address(c->device, &b));
  const fp::Scratch sc = fp::carve_scratch(b, sz);
  // run_rates clears the counters and the output on every call (the array keeps the last call's contents)
  unsigned long long counts[fp::kCounters] = {0};
  rc = fp::run_rates(c, o, sel, p, sc, nT, T, sb, d_out, counts, false, &err);
  if (rc) return nfail(c, rc, "fp_rates4_noalloc: " + err);
  if (stats) fp::fill_stats(c, o, sel, p, counts, stats);
  return FP_OK;
}
