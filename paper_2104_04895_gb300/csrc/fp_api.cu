// C-ABI of libfourphonon: context, validation, device memory, launches (see include/fourphonon.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>

#include "fp_internal.cuh"

namespace {

std::string g_init_error;

int fail(fp_ctx* c, int code, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_init_error = msg;
  return code;
}

#define FP_CUDA(ctx, call)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

// Host-side fault injection for the allocation path: with FP_FAULT_ALLOC=k in the environment, the k-th
// device allocation of the context API after the variable was (re)set reports cudaErrorMemoryAllocation
// without allocating, so callers can test FP_ENOMEM handling without touching the GPU.
bool injected_alloc_failure() {
  static std::string last;
  static long count = 0;
  const char* env = std::getenv("FP_FAULT_ALLOC");
  const std::string cur = env ? env : "";
  if (cur != last) {
    last = cur;
    count = 0;
  }
  if (cur.empty()) return false;
  const long k = std::strtol(cur.c_str(), nullptr, 10);
  return k > 0 && ++count == k;
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T));
}

template <typename T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

int gcd(int a, int b) { return b == 0 ? a : gcd(b, a % b); }

void reciprocal(const double A[9], double B[9], double* det_out) {
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  // rows b_a = 2 pi (A^{-1})^T rows: b_a[c] = 2 pi inv[c][a]; inv = adj / det
  double adj[9] = {A[4] * A[8] - A[5] * A[7], A[2] * A[7] - A[1] * A[8], A[1] * A[5] - A[2] * A[4],
                   A[5] * A[6] - A[3] * A[8], A[0] * A[8] - A[2] * A[6], A[2] * A[3] - A[0] * A[5],
                   A[3] * A[7] - A[4] * A[6], A[1] * A[6] - A[0] * A[7], A[0] * A[4] - A[1] * A[3]};
  double inv[9];
  for (int k = 0; k < 9; ++k) inv[k] = adj[k] / det;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) B[3 * a + c] = 2.0 * fp::kPi * inv[3 * c + a];
  if (det_out) *det_out = det;
}

double det3(const double M[9]) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

int ensure_modes_buffers(fp_ctx* c) {
  if (!c->d_omega) {
    FP_CUDA(c, dalloc(&c->d_omega, (size_t)c->N * c->nb));
    FP_CUDA(c, dalloc(&c->d_evec, (size_t)c->N * c->nb * c->nb));
    FP_CUDA(c, dalloc(&c->d_vel, (size_t)c->N * c->nb * 3));
  }
  return FP_OK;
}

int grid_index(const fp_ctx* c, const int g[3]) { return (g[0] * c->grid[1] + g[1]) * c->grid[2] + g[2]; }

int neg_index(const fp_ctx* c, int q) {
  int g[3] = {q / (c->grid[1] * c->grid[2]), (q / c->grid[2]) % c->grid[1], q % c->grid[2]};
  int m[3];
  for (int d = 0; d < 3; ++d) m[d] = (c->grid[d] - g[d]) % c->grid[d];
  return grid_index(c, m);
}

}  // namespace

namespace fp {
int fail_global(int code, const std::string& msg) { return fail(nullptr, code, msg); }
}  // namespace fp

extern "C" {

int fp_version(void) { return 10000; }

void fp_default_opts(fp_rates_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = FP_PREC_FP64;
  o->window = 2.0;
  o->sigma_min = 1e-10;
  o->dq_mode = 0;
  o->mode_mask = nullptr;
  o->q_begin = 0;
  o->q_end = 0;
}

const char* fp_last_error(const fp_ctx* c) { return c ? c->err.c_str() : g_init_error.c_str(); }

void fp_free(fp_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->own_stream) cudaStreamSynchronize(c->own_stream);
  dfree(c->d_fc2_idx);
  dfree(c->d_fc2_val);
  dfree(c->d_mass);
  dfree(c->d_qmeta);
  dfree(c->d_qfc);
  dfree(c->d_gmeta);
  dfree(c->d_grp_qstart);
  dfree(c->d_grp_q);
  dfree(c->d_kl_start);
  dfree(c->d_kl_grp);
  dfree(c->d_tw);
  dfree(c->d_omega);
  dfree(c->d_evec);
  dfree(c->d_vel);
  dfree(c->d_flag);
  dfree(c->d_scratch);
  dfree(c->d_rates);
  dfree(c->d_star);
  dfree(c->d_bzm);
  dfree(c->d_t3_start);
  dfree(c->d_t3_cell);
  dfree(c->d_t3_fc);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
}

int fp_init(fp_ctx** out, const double lattice[9], int natoms, const double* frac_pos, const double* mass,
            int n_fc2, const fp_fc2* fc2, int n_fc4, const fp_fc4* fc4, const int grid[3], int device) {
  (void)frac_pos;
  if (!out) return fail(nullptr, FP_EINVAL, "fp_init: out is NULL");
  *out = nullptr;
  if (!lattice || !mass || !grid) return fail(nullptr, FP_EINVAL, "fp_init: NULL lattice, mass or grid");
  if (natoms < 1 || 3 * natoms > fp::kMaxNb)
    return fail(nullptr, FP_EINVAL, "fp_init: natoms must be in [1, 4]");
  for (int a = 0; a < 3; ++a)
    if (grid[a] < 1 || grid[a] > 64) return fail(nullptr, FP_EINVAL, "fp_init: grid dimensions must be in [1, 64]");
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(lattice[i])) return fail(nullptr, FP_EINVAL, "fp_init: non-finite lattice");
  if (std::fabs(det3(lattice)) < 1e-12) return fail(nullptr, FP_EINVAL, "fp_init: singular lattice");
  for (int i = 0; i < natoms; ++i)
    if (!(mass[i] > 0.0) || !std::isfinite(mass[i])) return fail(nullptr, FP_EINVAL, "fp_init: masses must be > 0");
  if (n_fc2 < 0 || (n_fc2 > 0 && !fc2)) return fail(nullptr, FP_EINVAL, "fp_init: bad Phi2 list");
  if (n_fc4 < 0 || (n_fc4 > 0 && !fc4)) return fail(nullptr, FP_EINVAL, "fp_init: bad Phi4 list");
  for (int b = 0; b < n_fc2; ++b) {
    if (fc2[b].i < 0 || fc2[b].i >= natoms || fc2[b].j < 0 || fc2[b].j >= natoms)
      return fail(nullptr, FP_EINVAL, "fp_init: Phi2 atom index out of range");
    for (int k = 0; k < 9; ++k)
      if (!std::isfinite(fc2[b].fc[k])) return fail(nullptr, FP_EINVAL, "fp_init: non-finite Phi2");
  }
  for (int b = 0; b < n_fc4; ++b) {
    const fp_fc4& f = fc4[b];
    int at[4] = {f.i, f.j, f.k, f.l};
    for (int k = 0; k < 4; ++k)
      if (at[k] < 0 || at[k] >= natoms) return fail(nullptr, FP_EINVAL, "fp_init: Phi4 atom index out of range");
    for (int k = 0; k < 81; ++k)
      if (!std::isfinite(f.fc[k])) return fail(nullptr, FP_EINVAL, "fp_init: non-finite Phi4");
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(nullptr, FP_ECUDA, "fp_init: no CUDA device");
  if (device < 0 || device >= ndev) return fail(nullptr, FP_EINVAL, "fp_init: bad device ordinal");

  fp_ctx* c = new fp_ctx();
  c->device = device;
  c->natoms = natoms;
  c->nb = 3 * natoms;
  for (int a = 0; a < 3; ++a) c->grid[a] = grid[a];
  c->N = grid[0] * grid[1] * grid[2];
  int L = 1;
  for (int a = 0; a < 3; ++a) L = L / gcd(L, grid[a]) * grid[a];
  c->L = L;
  std::memcpy(c->lattice, lattice, sizeof(c->lattice));
  reciprocal(lattice, c->rec, nullptr);
  c->mass.assign(mass, mass + natoms);

  int* d_atoms4 = nullptr;  // temporary (atoms of each quartet for the mass scaling)
  auto bail = [&](int rc) {
    g_init_error = c->err;
    if (d_atoms4) cudaFree(d_atoms4);
    fp_free(c);
    return rc;
  };
#define INIT_CUDA(call)                                                                               \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess)                                                                            \
      return bail(fail(c, e_ == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA,                     \
                       std::string(#call) + ": " + cudaGetErrorString(e_)));                          \
  } while (0)

  INIT_CUDA(cudaSetDevice(device));
  INIT_CUDA(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
  c->stream = c->own_stream;
  INIT_CUDA(cudaEventCreate(&c->ev0));
  INIT_CUDA(cudaEventCreate(&c->ev1));
  cudaStream_t s = c->stream;

  // harmonic pairs
  c->n_fc2 = n_fc2;
  std::vector<int> idx2(5 * (size_t)n_fc2);
  std::vector<double> val2(9 * (size_t)n_fc2);
  for (int b = 0; b < n_fc2; ++b) {
    idx2[5 * b] = fc2[b].i;
    idx2[5 * b + 1] = fc2[b].j;
    for (int d = 0; d < 3; ++d) idx2[5 * b + 2 + d] = fc2[b].Rj[d];
    for (int k = 0; k < 9; ++k) val2[9 * b + k] = fc2[b].fc[k];
  }
  INIT_CUDA(dalloc(&c->d_fc2_idx, idx2.size()));
  INIT_CUDA(dalloc(&c->d_fc2_val, val2.size()));
  INIT_CUDA(dalloc(&c->d_mass, (size_t)natoms));
  INIT_CUDA(cudaMemcpyAsync(c->d_fc2_idx, idx2.data(), idx2.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_fc2_val, val2.data(), val2.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_mass, mass, natoms * sizeof(double), cudaMemcpyHostToDevice, s));

  // quartets grouped by (atom k, atom l, D = R_k - R_l)
  c->nquart = n_fc4;
  std::map<std::tuple<int, int, int, int, int>, int> gid;
  std::vector<int> qgroup(n_fc4);
  for (int b = 0; b < n_fc4; ++b) {
    const fp_fc4& f = fc4[b];
    auto key = std::make_tuple(f.k, f.l, f.Rk[0] - f.Rl[0], f.Rk[1] - f.Rl[1], f.Rk[2] - f.Rl[2]);
    auto it = gid.find(key);
    if (it == gid.end()) it = gid.emplace(key, 0).first;
    (void)it;
  }
  {
    int n = 0;
    for (auto& kv : gid) kv.second = n++;  // sorted order: by (k, l, D)
  }
  c->G = (int)gid.size();
  std::vector<int> gmeta(5 * (size_t)c->G);
  for (auto& kv : gid) {
    int gi = kv.second;
    gmeta[5 * gi] = std::get<0>(kv.first);
    gmeta[5 * gi + 1] = std::get<1>(kv.first);
    gmeta[5 * gi + 2] = std::get<2>(kv.first);
    gmeta[5 * gi + 3] = std::get<3>(kv.first);
    gmeta[5 * gi + 4] = std::get<4>(kv.first);
  }
  std::vector<int> qmeta(9 * (size_t)n_fc4), atoms4(4 * (size_t)n_fc4);
  std::vector<double> qfc(81 * (size_t)n_fc4);
  for (int b = 0; b < n_fc4; ++b) {
    const fp_fc4& f = fc4[b];
    auto key = std::make_tuple(f.k, f.l, f.Rk[0] - f.Rl[0], f.Rk[1] - f.Rl[1], f.Rk[2] - f.Rl[2]);
    qgroup[b] = gid[key];
    qmeta[9 * b] = f.i;
    qmeta[9 * b + 1] = f.j;
    qmeta[9 * b + 2] = qgroup[b];
    for (int d = 0; d < 3; ++d) {
      qmeta[9 * b + 3 + d] = f.Rj[d];
      qmeta[9 * b + 6 + d] = f.Rl[d];
    }
    atoms4[4 * b] = f.i;
    atoms4[4 * b + 1] = f.j;
    atoms4[4 * b + 2] = f.k;
    atoms4[4 * b + 3] = f.l;
    std::memcpy(&qfc[81 * (size_t)b], f.fc, 81 * sizeof(double));
  }
  std::vector<int> grp_qstart(c->G + 1, 0), grp_q(n_fc4);
  for (int b = 0; b < n_fc4; ++b) grp_qstart[qgroup[b] + 1]++;
  for (int gi = 0; gi < c->G; ++gi) grp_qstart[gi + 1] += grp_qstart[gi];
  {
    std::vector<int> fill(grp_qstart.begin(), grp_qstart.end() - 1);
    for (int b = 0; b < n_fc4; ++b) grp_q[fill[qgroup[b]]++] = b;
  }
  const int na2 = natoms * natoms;
  std::vector<int> kl_start(na2 + 1, 0), kl_grp(c->G);
  for (int gi = 0; gi < c->G; ++gi) kl_start[gmeta[5 * gi] * natoms + gmeta[5 * gi + 1] + 1]++;
  for (int k = 0; k < na2; ++k) kl_start[k + 1] += kl_start[k];
  {
    std::vector<int> fill(kl_start.begin(), kl_start.end() - 1);
    for (int gi = 0; gi < c->G; ++gi) kl_grp[fill[gmeta[5 * gi] * natoms + gmeta[5 * gi + 1]]++] = gi;
  }
  INIT_CUDA(dalloc(&c->d_qmeta, qmeta.size()));
  INIT_CUDA(dalloc(&c->d_qfc, qfc.size()));
  INIT_CUDA(dalloc(&c->d_gmeta, gmeta.size()));
  INIT_CUDA(dalloc(&c->d_grp_qstart, grp_qstart.size()));
  INIT_CUDA(dalloc(&c->d_grp_q, grp_q.size()));
  INIT_CUDA(dalloc(&c->d_kl_start, kl_start.size()));
  INIT_CUDA(dalloc(&c->d_kl_grp, kl_grp.size()));
  INIT_CUDA(dalloc(&d_atoms4, atoms4.size()));
  INIT_CUDA(cudaMemcpyAsync(c->d_qmeta, qmeta.data(), qmeta.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_qfc, qfc.data(), qfc.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_gmeta, gmeta.data(), gmeta.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_grp_qstart, grp_qstart.data(), grp_qstart.size() * sizeof(int),
                            cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_grp_q, grp_q.data(), grp_q.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_kl_start, kl_start.data(), kl_start.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(c->d_kl_grp, kl_grp.data(), kl_grp.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  INIT_CUDA(cudaMemcpyAsync(d_atoms4, atoms4.data(), atoms4.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  INIT_CUDA(fp::launch_scale_fc4(c->d_qfc, d_atoms4, c->d_mass, n_fc4, s));
  INIT_CUDA(dalloc(&c->d_tw, (size_t)c->L));
  INIT_CUDA(fp::launch_twiddles(c, s));
  INIT_CUDA(dalloc(&c->d_flag, 1));
  {
    std::vector<int> bzm(3 * (size_t)c->N);
    fp::bz_shifts(c->grid, c->rec, bzm.data());
    INIT_CUDA(dalloc(&c->d_bzm, bzm.size()));
    INIT_CUDA(cudaMemcpyAsync(c->d_bzm, bzm.data(), bzm.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    INIT_CUDA(cudaStreamSynchronize(s));  // bzm is a local buffer
  }
  cudaFree(d_atoms4);
#undef INIT_CUDA
  *out = c;
  return FP_OK;
}

int fp_set_stream(fp_ctx* c, void* stream) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_set_stream: NULL context");
  c->stream = stream ? reinterpret_cast<cudaStream_t>(stream) : c->own_stream;
  return FP_OK;
}

int fp_modes(fp_ctx* c, double* omega, double* evec, double* vel) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_modes: NULL context");
  FP_CUDA(c, cudaSetDevice(c->device));
  int rc = ensure_modes_buffers(c);
  if (rc) return rc;
  cudaStream_t s = c->stream;
  FP_CUDA(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), s));
  FP_CUDA(c, fp::launch_modes(c, s));
  int flag = 0;
  FP_CUDA(c, cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  const size_t nm = (size_t)c->N * c->nb;
  if (omega) FP_CUDA(c, cudaMemcpyAsync(omega, c->d_omega, nm * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (evec) FP_CUDA(c, cudaMemcpyAsync(evec, c->d_evec, nm * c->nb * sizeof(double2), cudaMemcpyDeviceToHost, s));
  if (vel) FP_CUDA(c, cudaMemcpyAsync(vel, c->d_vel, nm * 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FP_CUDA(c, cudaStreamSynchronize(s));
  if (flag) {
    c->have_modes = false;
    return fail(c, FP_EUNSTABLE, "fp_modes: imaginary frequencies (omega^2 < -1e-8 max omega^2)");
  }
  c->have_modes = true;
  return FP_OK;
}

int fp_set_modes(fp_ctx* c, const double* omega, const double* evec, const double* vel) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_set_modes: NULL context");
  if (!omega || !evec || !vel) return fail(c, FP_EINVAL, "fp_set_modes: NULL table");
  const int nb = c->nb;
  for (int q = 0; q < c->N; ++q) {
    const int p = neg_index(c, q);
    for (int j = 0; j < nb; ++j) {
      double w = omega[q * nb + j];
      if (!(w >= 0.0) || !std::isfinite(w)) return fail(c, FP_EINVAL, "fp_set_modes: omega must be finite and >= 0");
      if (omega[p * nb + j] != w) return fail(c, FP_EINVAL, "fp_set_modes: omega(-q) != omega(q)");
      for (int d = 0; d < 3; ++d)
        if (vel[(q * nb + j) * 3 + d] != -vel[(p * nb + j) * 3 + d])
          return fail(c, FP_EINVAL, "fp_set_modes: v(-q) != -v(q)");
      for (int k = 0; k < nb; ++k) {
        const double* a = evec + 2 * (((size_t)q * nb + j) * nb + k);
        const double* b = evec + 2 * (((size_t)p * nb + j) * nb + k);
        if (a[0] != b[0] || a[1] != -b[1]) return fail(c, FP_EINVAL, "fp_set_modes: e(-q) != conj e(q)");
      }
    }
  }
  FP_CUDA(c, cudaSetDevice(c->device));
  int rc = ensure_modes_buffers(c);
  if (rc) return rc;
  const size_t nm = (size_t)c->N * nb;
  cudaStream_t s = c->stream;
  FP_CUDA(c, cudaMemcpyAsync(c->d_omega, omega, nm * sizeof(double), cudaMemcpyHostToDevice, s));
  FP_CUDA(c, cudaMemcpyAsync(c->d_evec, evec, nm * nb * sizeof(double2), cudaMemcpyHostToDevice, s));
  FP_CUDA(c, cudaMemcpyAsync(c->d_vel, vel, nm * 3 * sizeof(double), cudaMemcpyHostToDevice, s));
  FP_CUDA(c, cudaStreamSynchronize(s));
  c->have_modes = true;
  return FP_OK;
}

static int validate_opts(fp_ctx* c, int nT, const double* T, double sb, const fp_rates_opts* user,
                         fp_rates_opts* o) {
  fp_default_opts(o);
  if (user) {
    *o = *user;
    if (o->window == 0.0) o->window = 2.0;
    if (o->sigma_min == 0.0) o->sigma_min = 1e-10;
  }
  if (!c->have_modes) return fail(c, FP_ESTATE, "fp_rates4: call fp_modes or fp_set_modes first");
  if (nT < 1 || nT > fp::kMaxT || !T) return fail(c, FP_EINVAL, "fp_rates4: nT must be in [1, 8]");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0) || !std::isfinite(T[i])) return fail(c, FP_EINVAL, "fp_rates4: temperatures must be > 0");
  if (!(sb > 0.0) || !std::isfinite(sb)) return fail(c, FP_EINVAL, "fp_rates4: scalebroad must be > 0");
  if (!(o->window > 0.0) || !(o->sigma_min > 0.0)) return fail(c, FP_EINVAL, "fp_rates4: window, sigma_min > 0");
  if (o->precision != FP_PREC_FP64 && o->precision != FP_PREC_MIXED && o->precision != FP_PREC_DOUBLE_FLOAT)
    return fail(c, FP_EINVAL, "fp_rates4: unknown precision");
  if (o->dq_mode != 0 && o->dq_mode != 1) return fail(c, FP_EINVAL, "fp_rates4: dq_mode must be 0 or 1");
  if (o->process_mask < 0 || o->process_mask > 7)
    return fail(c, FP_EINVAL, "fp_rates4: process_mask must be in [0, 7]");
  if (o->nu_select < 0 || o->nu_select > 2) return fail(c, FP_EINVAL, "fp_rates4: nu_select must be 0, 1 or 2");
  if (o->no_time_reversal != 0 && o->no_time_reversal != 1)
    return fail(c, FP_EINVAL, "fp_rates4: no_time_reversal must be 0 or 1");
  if (o->tensor_cores != 0 && o->tensor_cores != 1) return fail(c, FP_EINVAL, "fp_rates4: tensor_cores must be 0 or 1");
  return FP_OK;
}

static int rates_impl(fp_ctx* c, int nT, const double* T, double sb, const fp_rates_opts* user, double* d_out,
                      fp_stats* stats) {
  fp_rates_opts o;
  int rc = validate_opts(c, nT, T, sb, user, &o);
  if (rc) return rc;
  FP_CUDA(c, cudaSetDevice(c->device));
  std::string err;
  fp::Selection sel;
  rc = fp::make_selection(c, o, true, &sel, &err);
  if (rc) return fail(c, rc, "fp_rates4: " + err);
  fp::Plan p;
  rc = fp::plan_rates(c, o, nT, sel, 0, &p, &err);
  if (rc) return fail(c, rc, "fp_rates4: " + err);
  size_t sz[fp::kScratchParts], total = 0;
  fp::scratch_sizes(c, p, nT, sz);
  for (size_t x : sz) total += x;
  if (c->scratch_cap < total) {
    dfree(c->d_scratch);
    c->scratch_cap = 0;
    FP_CUDA(c, dalloc(&c->d_scratch, total));
    c->scratch_cap = total;
  }
  const fp::Scratch sc = fp::carve_scratch(c->d_scratch, sz);
  unsigned long long counts[fp::kCounters] = {0};
  rc = fp::run_rates(c, o, sel, p, sc, nT, T, sb, d_out, counts, o.no_graph == 0, &err);
  if (rc) return fail(c, rc, "fp_rates4: " + err);
  if (stats) fp::fill_stats(c, o, sel, p, counts, stats);
  return FP_OK;
}

int fp_rates4_device(fp_ctx* c, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
                     double* d_rates, fp_stats* stats) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_rates4_device: NULL context");
  if (!d_rates) return fail(c, FP_EINVAL, "fp_rates4_device: NULL output");
  return rates_impl(c, nT, T, scalebroad, opts, d_rates, stats);
}

int fp_rates4(fp_ctx* c, int nT, const double* T, double scalebroad, const fp_rates_opts* opts, double* rates,
              fp_stats* stats) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_rates4: NULL context");
  if (!rates) return fail(c, FP_EINVAL, "fp_rates4: NULL output");
  if (nT < 1 || nT > fp::kMaxT) return fail(c, FP_EINVAL, "fp_rates4: nT must be in [1, 8]");
  FP_CUDA(c, cudaSetDevice(c->device));
  const size_t need = (size_t)nT * c->N * c->nb;
  if (c->rates_cap < need) {
    dfree(c->d_rates);
    c->rates_cap = 0;
    FP_CUDA(c, dalloc(&c->d_rates, need));
    c->rates_cap = need;
  }
  int rc = rates_impl(c, nT, T, scalebroad, opts, c->d_rates, stats);
  if (rc) return rc;
  FP_CUDA(c, cudaMemcpyAsync(rates, c->d_rates, need * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FP_CUDA(c, cudaStreamSynchronize(c->stream));
  return FP_OK;
}

}  // extern "C"

namespace {

// rate of (q, j) := the mean over the degenerate set of j at the representative of q's star
__global__ void star_gather_kernel(const double* __restrict__ in, const int* __restrict__ rep,
                                   const double* __restrict__ omega, int N, int nb, int nT, double tol,
                                   double* __restrict__ out) {
  const long long n = (long long)nT * N * nb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i % nb);
    const long long tq = i / nb;
    const int q = (int)(tq % N), t = (int)(tq / N);
    const int r = rep[q];
    const double* w = omega + (size_t)r * nb;
    int lo = j, hi = j;
    while (lo > 0 && w[lo] - w[lo - 1] <= tol) --lo;
    while (hi < nb - 1 && w[hi + 1] - w[hi] <= tol) ++hi;
    const double* src = in + ((size_t)t * N + r) * nb;
    double s = 0.0;
    for (int k = lo; k <= hi; ++k) s += src[k];
    out[i] = s / (double)(hi - lo + 1);
  }
}

}  // namespace

extern "C" {

int fp_rates4_irreducible(fp_ctx* c, int nrot, const int* rot, int nT, const double* T, double scalebroad,
                          const fp_rates_opts* opts, double* rates, fp_stats* stats, int* n_irr) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_rates4_irreducible: NULL context");
  if (!rates) return fail(c, FP_EINVAL, "fp_rates4_irreducible: NULL output");
  if (nT < 1 || nT > fp::kMaxT) return fail(c, FP_EINVAL, "fp_rates4_irreducible: nT must be in [1, 8]");
  if (!c->have_modes) return fail(c, FP_ESTATE, "fp_rates4_irreducible: call fp_modes or fp_set_modes first");
  if (opts && (opts->mode_mask || opts->q_begin != 0 || opts->q_end > 0))
    return fail(c, FP_EINVAL, "fp_rates4_irreducible: mode_mask and the q range are set by the star table");
  if (opts && opts->dq_mode != 0)
    return fail(c, FP_EINVAL, "fp_rates4_irreducible: dq_mode 1 is not point-group invariant");
  const int N = c->N, nb = c->nb;
  const size_t nm = (size_t)N * nb, need = (size_t)nT * nm;
  std::vector<int> rep(N);
  int nirr = 0;
  if (fp_star_table(c->grid, nrot, rot, rep.data(), &nirr) != FP_OK)
    return fail(c, FP_EINVAL, "fp_rates4_irreducible: an op is not unimodular or mixes grid axes of unequal size");
  std::vector<unsigned char> mask(nm, 0);
  for (int q = 0; q < N; ++q)
    if (rep[q] == q) std::memset(mask.data() + (size_t)q * nb, 1, nb);
  // degenerate sets as in the modes: |dw| <= 1e-8 max w
  std::vector<double> w(nm);
  FP_CUDA(c, cudaSetDevice(c->device));
  FP_CUDA(c, cudaMemcpyAsync(w.data(), c->d_omega, nm * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FP_CUDA(c, cudaStreamSynchronize(c->stream));
  double wmax = 0.0;
  for (double x : w) wmax = x > wmax ? x : wmax;
  if (c->rates_cap < 2 * need) {
    dfree(c->d_rates);
    c->rates_cap = 0;
    FP_CUDA(c, dalloc(&c->d_rates, 2 * need));
    c->rates_cap = 2 * need;
  }
  if (c->star_cap < (size_t)N) {
    dfree(c->d_star);
    c->star_cap = 0;
    FP_CUDA(c, dalloc(&c->d_star, (size_t)N));
    c->star_cap = (size_t)N;
  }
  fp_rates_opts o;
  fp_default_opts(&o);
  if (opts) o = *opts;
  o.mode_mask = mask.data();
  int rc = rates_impl(c, nT, T, scalebroad, &o, c->d_rates, stats);
  if (rc) return rc;
  FP_CUDA(c, cudaMemcpyAsync(c->d_star, rep.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  star_gather_kernel<<<(unsigned)std::min<size_t>((need + 255) / 256, 4096), 256, 0, c->stream>>>(
      c->d_rates, c->d_star, c->d_omega, N, nb, nT, 1e-8 * wmax, c->d_rates + need);
  FP_CUDA(c, cudaGetLastError());
  FP_CUDA(c, cudaMemcpyAsync(rates, c->d_rates + need, need * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  FP_CUDA(c, cudaStreamSynchronize(c->stream));
  if (n_irr) *n_irr = nirr;
  return FP_OK;
}

}  // extern "C"

namespace {

// npass rate passes, pass p with the options set(o, p), into rates[t][p][N][nb] (host); stats sums the
// passes' candidates, flops and time, and takes accepted[k] from every pass that counted process k
int rates_passes(fp_ctx* c, int nT, const double* T, double sb, const fp_rates_opts* opts, int npass,
                 void (*set)(fp_rates_opts&, int), double* rates, fp_stats* stats, const char* who) {
  const std::string name(who);
  if (!rates) return fail(c, FP_EINVAL, name + ": NULL output");
  if (nT < 1 || nT > fp::kMaxT) return fail(c, FP_EINVAL, name + ": nT must be in [1, 8]");
  FP_CUDA(c, cudaSetDevice(c->device));
  const size_t nm = (size_t)c->N * c->nb, need = (size_t)nT * nm;
  if (c->rates_cap < need) {
    dfree(c->d_rates);
    c->rates_cap = 0;
    FP_CUDA(c, dalloc(&c->d_rates, need));
    c->rates_cap = need;
  }
  fp_rates_opts o;
  fp_default_opts(&o);
  if (opts) o = *opts;
  o.no_graph = 1;  // several launch configurations in turn: plain launches rather than re-captured graphs
  fp_stats sum;
  std::memset(&sum, 0, sizeof(sum));
  std::vector<double> part(need);
  for (int p = 0; p < npass; ++p) {
    set(o, p);
    fp_stats st;
    int rc = rates_impl(c, nT, T, sb, &o, c->d_rates, &st);
    if (rc) return rc;
    FP_CUDA(c, cudaMemcpyAsync(part.data(), c->d_rates, need * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    FP_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int t = 0; t < nT; ++t)
      std::memcpy(rates + ((size_t)t * npass + p) * nm, part.data() + (size_t)t * nm, nm * sizeof(double));
    sum.candidates += st.candidates;
    for (int k = 0; k < 3; ++k) sum.accepted[k] += st.accepted[k];
    sum.flops += st.flops;
    sum.candidates_executed += st.candidates_executed;
    sum.vertex_entries += st.vertex_entries;
    sum.terms_executed += st.terms_executed;
    sum.ms += st.ms;
    std::memcpy(sum.tile, st.tile, sizeof(sum.tile));
  }
  if (stats) *stats = sum;
  return FP_OK;
}

}  // namespace

extern "C" {

int fp_rates4_channels(fp_ctx* c, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
                       double* rates, fp_stats* stats) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_rates4_channels: NULL context");
  if (opts && opts->process_mask != 0)
    return fail(c, FP_EINVAL, "fp_rates4_channels: process_mask must be 0 (all three channels are computed)");
  return rates_passes(c, nT, T, scalebroad, opts, 3, [](fp_rates_opts& o, int p) { o.process_mask = 1 << p; },
                      rates, stats, "fp_rates4_channels");
}

int fp_rates4_nu(fp_ctx* c, int nT, const double* T, double scalebroad, const fp_rates_opts* opts, double* rates,
                 fp_stats* stats) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_rates4_nu: NULL context");
  if (opts && opts->nu_select != 0)
    return fail(c, FP_EINVAL, "fp_rates4_nu: nu_select must be 0 (both parts are computed)");
  return rates_passes(c, nT, T, scalebroad, opts, 2, [](fp_rates_opts& o, int p) { o.nu_select = 1 + p; }, rates,
                      stats, "fp_rates4_nu");
}

}  // extern "C"


namespace {

// one unit-vertex pass (|W|^2 := 1) of the rate kernel over q' on a stride; d_out nT x N x nb, d_counts N x nb
int phase_pass(fp_ctx* c, const fp_rates_opts& o, int nT, const double* T, double sb, int stride, bool unit_weights,
               double* d_out, double* d_counts, std::string* err) {
  fp::Selection sel;
  int rc = fp::make_selection(c, o, stride == 1, &sel, err);  // a q' stride is not symmetric under q -> -q
  if (rc) return rc;
  fp::Plan p;
  rc = fp::plan_rates(c, o, nT, sel, 0, &p, err);
  if (rc) return rc;
  if (stride > 1) {  // a q' tile of one stride: every item owns exactly one sampled q'
    p.t1 = stride;
    p.ntile = (c->N + stride - 1) / stride;
    p.n_items = (long long)p.ntile * p.nq_sel * p.nchunk;
    if (p.ctas > p.n_items) p.ctas = (int)std::max<long long>(1, p.n_items);
  }
  size_t sz[fp::kScratchParts], total = 0;
  fp::scratch_sizes(c, p, nT, sz);
  for (size_t x : sz) total += x;
  const size_t cnt_bytes = (size_t)std::max<long long>(1, p.n_items) * p.J * sizeof(unsigned long long);
  unsigned char* b = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b), total + cnt_bytes);
  if (e != cudaSuccess) {
    *err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return FP_ENOMEM;
  }
  const fp::Scratch sc = fp::carve_scratch(b, sz);
  fp::RunExtra x;
  x.unit_stride = stride;
  x.unit_weights = unit_weights;
  x.d_item_counts = reinterpret_cast<unsigned long long*>(b + total);
  x.d_mode_counts = d_counts;
  unsigned long long counts[fp::kCounters];
  rc = fp::run_rates(c, o, sel, p, sc, nT, T, sb, d_out, counts, false, err, x);
  cudaFree(b);
  return rc;
}

}  // namespace

extern "C" int fp_phase_space4(fp_ctx* c, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
                               int stride, double* numprocess, double* p4, double* wp4) {
  if (!c) return fail(nullptr, FP_EINVAL, "fp_phase_space4: NULL context");
  fp_rates_opts o;
  int rc = validate_opts(c, nT, T, scalebroad, opts, &o);
  if (rc) return rc;
  if (stride < 1 || stride > c->N) return fail(c, FP_EINVAL, "fp_phase_space4: stride must be in [1, N]");
  o.no_graph = 1;
  FP_CUDA(c, cudaSetDevice(c->device));
  const size_t nm = (size_t)c->N * c->nb;
  double* d = nullptr;
  FP_CUDA(c, dalloc(&d, nm * (2 + (size_t)nT) + nm));
  double* d_p4 = d;
  double* d_cnt = d + nm;
  double* d_wp4 = d + 2 * nm;
  double* d_cnt2 = d + (2 + (size_t)nT) * nm;
  std::string err;
  // pass 1: unit weights (P4) and the accepted terms per mode; pass 2: Bose and frequency weights (WP4)
  rc = phase_pass(c, o, 1, T, scalebroad, stride, true, d_p4, d_cnt, &err);
  if (!rc && wp4) rc = phase_pass(c, o, nT, T, scalebroad, stride, false, d_wp4, d_cnt2, &err);
  cudaError_t e = cudaSuccess;
  if (!rc && numprocess) e = cudaMemcpyAsync(numprocess, d_cnt, nm * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!rc && e == cudaSuccess && p4) e = cudaMemcpyAsync(p4, d_p4, nm * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (!rc && e == cudaSuccess && wp4)
    e = cudaMemcpyAsync(wp4, d_wp4, nT * nm * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(d);
  if (rc) return fail(c, rc, "fp_phase_space4: " + err);
  if (e != cudaSuccess) return fail(c, FP_ECUDA, std::string("fp_phase_space4: ") + cudaGetErrorString(e));
  return FP_OK;
}
