// Three-phonon RTA rates (paper Sec. 2.2, Eqs. tao0, 3phgamma, V3): fp_set_fc3 and fp_rates3.
//
// With k2 = q + k1 (mod G) and e(-k) = conj e(k) one vertex
//   W3(q, j; k1, j1; k2, j2) = sum_triplets sum_{abg} Phi3 / sqrt(M^3) e_a(q, j) e_b(k1, j1) conj(e_g(k2, j2))
//                              exp(i (k1.R_j - k2.R_k))
// is V+ of the partner q' = k1 and V- of the partner q' = -k1 (both with q'' = k2), so every (q, k1) pair
// serves both processes.  One CTA per q walks k1 over the grid: it assembles the reciprocal force constants
// Phi~[(i a)(j b)(k g)] for (k1, k2), contracts them with e(q), e(k1) and conj e(k2) (three nb^4 steps
// through shared memory), and every thread then owns entries (j, j1, j2): the window test and Gaussian of
// both processes in FP64 with the oracle's operation order (decisions are identical), Bose factors,
// |W|^2, and a running sum in shared memory.  The rates of each j are summed over its entries in a fixed
// order at the end, so results do not depend on scheduling.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "fp_internal.cuh"

namespace {

struct Rates3Args {
  int N, nb, nT, L, n3, natoms;
  int grid[3], Lfac[3];
  const double* omega;
  const double2* evec;
  const double* vel;
  const double2* tw;
  const int* t3_start;  // [natoms^3 + 1] triplets grouped by atom triple (i, j, k)
  const int* t3_cell;   // [n3][6] Rj, Rk
  const double* t3_fc;  // [n3][27] Phi3 / sqrt(Mi Mj Mk)
  const double* bose;   // [nT][N nb] occupation numbers
  const unsigned char* mask;
  int q_begin, nq_sel;
  double sb, window, sigma_min, dq, pref;
  int dq_mode;
  double rec[9];
  double* rates;                 // [nT][N nb]
  unsigned long long* counts;    // [2]
};

__device__ __forceinline__ int wrap3(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

// sigma = sb |v' - v''| dq (dq_mode 0) or the per-axis form, in the oracle's operation order
__device__ double sigma3(const Rates3Args& a, const double* v1, const double* v2) {
  const double dx = __dsub_rn(v1[0], v2[0]), dy = __dsub_rn(v1[1], v2[1]), dz = __dsub_rn(v1[2], v2[2]);
  if (a.dq_mode == 0) {
    const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return __dmul_rn(__dmul_rn(a.sb, sqrt(s)), a.dq);
  }
  double pa[3];
  for (int d = 0; d < 3; ++d) {
    const double* b = a.rec + 3 * d;
    pa[d] = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, b[0]), __dmul_rn(dy, b[1])), __dmul_rn(dz, b[2])),
                      (double)a.grid[d]);
  }
  const double s = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(pa[0], pa[0]), __dmul_rn(pa[1], pa[1])), __dmul_rn(pa[2], pa[2])), 3.0);
  return __dmul_rn(a.sb, sqrt(s));
}

__global__ void bose3_kernel(const double* omega, const double* T, int nT, long long nm, double* out) {
  const long long n = (long long)nT * nm;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double w = omega[i % nm];
    const double t = T[i / nm];
    out[i] = w > 0.0 ? 1.0 / expm1(fp::kHbar * w / (fp::kBoltzmann * t)) : 0.0;
  }
}

template <int NB>
__global__ void __launch_bounds__(256) rates3_kernel(Rates3Args a) {
  constexpr int NB2 = NB * NB, NB3 = NB2 * NB, NA = NB / 3;
  extern __shared__ __align__(16) unsigned char smem[];
  double2* sPhi = reinterpret_cast<double2*>(smem);  // [a][b][c], then reused for Y[j][j1][c]
  double2* sX = sPhi + NB3;                            // [j][b][c]
  double2* sE0 = sX + NB3;                             // [j][a]
  double2* sE1 = sE0 + NB2;
  double2* sE2 = sE1 + NB2;
  double2* sTw = sE2 + NB2;                            // [n3]
  double* sAcc = reinterpret_cast<double*>(sTw + a.n3);  // [entry][t]
  double* sW1 = sAcc + (size_t)NB3 * a.nT;               // omega(k1), omega(-k1), omega(k2)
  double* sW1n = sW1 + NB;
  double* sW2 = sW1n + NB;
  double* sV1 = sW2 + NB;  // [3 NB] v(k1), v(-k1), v(k2)
  double* sV1n = sV1 + 3 * NB;
  double* sV2 = sV1n + 3 * NB;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int N = a.N, nT = a.nT;
  const long long NM = (long long)N * NB;
  const int q = a.q_begin + blockIdx.x;
  const int g[3] = {q / (a.grid[1] * a.grid[2]), (q / a.grid[2]) % a.grid[1], q % a.grid[2]};
  for (int o = tid; o < NB2; o += nthr) sE0[o] = a.evec[(size_t)q * NB2 + o];
  for (int o = tid; o < NB3 * nT; o += nthr) sAcc[o] = 0.0;
  unsigned long long cplus = 0, cminus = 0;
  __syncthreads();
  for (int k1 = 0; k1 < N; ++k1) {
    const int g1[3] = {k1 / (a.grid[1] * a.grid[2]), (k1 / a.grid[2]) % a.grid[1], k1 % a.grid[2]};
    int g2[3], gn[3];
    for (int d = 0; d < 3; ++d) {
      g2[d] = wrap3(g[d] + g1[d], a.grid[d]);
      gn[d] = wrap3(-g1[d], a.grid[d]);
    }
    const int k2 = (g2[0] * a.grid[1] + g2[1]) * a.grid[2] + g2[2];
    const int kn = (gn[0] * a.grid[1] + gn[1]) * a.grid[2] + gn[2];  // -k1, the partner of the - process
    for (int o = tid; o < NB2; o += nthr) {
      sE1[o] = a.evec[(size_t)k1 * NB2 + o];
      sE2[o] = a.evec[(size_t)k2 * NB2 + o];
    }
    for (int o = tid; o < NB; o += nthr) {
      sW1[o] = a.omega[(size_t)k1 * NB + o];
      sW1n[o] = a.omega[(size_t)kn * NB + o];
      sW2[o] = a.omega[(size_t)k2 * NB + o];
    }
    for (int o = tid; o < 3 * NB; o += nthr) {
      sV1[o] = a.vel[(size_t)k1 * NB * 3 + o];
      sV1n[o] = a.vel[(size_t)kn * NB * 3 + o];
      sV2[o] = a.vel[(size_t)k2 * NB * 3 + o];
    }
    for (int Q = tid; Q < a.n3; Q += nthr) {
      const int* R = a.t3_cell + 6 * Q;
      int e = 0;  // each term is below L, so e < 3 L
      for (int d = 0; d < 3; ++d) e += a.Lfac[d] * wrap3(g1[d] * R[d] - g2[d] * R[3 + d], a.grid[d]);
      while (e >= a.L) e -= a.L;
      sTw[Q] = a.tw[e];
    }
    __syncthreads();
    // Phi~[(i al)(j be)(k ga)] = sum over the triplets of atoms (i, j, k) of Phi3 / sqrt(M^3) exp(i(k1.Rj - k2.Rk))
    for (int o = tid; o < NB3; o += nthr) {
      const int ab = o / NB, c = o % NB, aa = ab / NB, b = ab % NB;
      const int t = (aa / 3 * NA + b / 3) * NA + c / 3;
      const int comp = ((aa % 3) * 3 + b % 3) * 3 + c % 3;
      double re = 0.0, im = 0.0;
      for (int Q = a.t3_start[t]; Q < a.t3_start[t + 1]; ++Q) {
        const double f = a.t3_fc[27 * (size_t)Q + comp];
        re = fma(f, sTw[Q].x, re);
        im = fma(f, sTw[Q].y, im);
      }
      sPhi[o] = make_double2(re, im);
    }
    __syncthreads();
    // X[j][b][c] = sum_a e_a(q, j) Phi~[a][b][c]
    for (int o = tid; o < NB3; o += nthr) {
      const int j = o / NB2, bc = o % NB2;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int aa = 0; aa < NB; ++aa) {
        const double2 e = sE0[j * NB + aa], p = sPhi[aa * NB2 + bc];
        re = fma(e.x, p.x, fma(-e.y, p.y, re));
        im = fma(e.x, p.y, fma(e.y, p.x, im));
      }
      sX[o] = make_double2(re, im);
    }
    __syncthreads();
    // Y[j][j1][c] = sum_b e_b(k1, j1) X[j][b][c]  (into sPhi)
    for (int o = tid; o < NB3; o += nthr) {
      const int j = o / NB2, j1 = (o / NB) % NB, c = o % NB;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const double2 e = sE1[j1 * NB + b], x = sX[(j * NB + b) * NB + c];
        re = fma(e.x, x.x, fma(-e.y, x.y, re));
        im = fma(e.x, x.y, fma(e.y, x.x, im));
      }
      sPhi[o] = make_double2(re, im);
    }
    __syncthreads();
    // W[j][j1][j2] = sum_c conj(e_c(k2, j2)) Y[j][j1][c]; then both processes of the entry
    for (int o = tid; o < NB3; o += nthr) {
      const int j = o / NB2, j1 = (o / NB) % NB, j2 = o % NB;
      const long long m0 = (long long)q * NB + j;
      const double w = a.omega[m0];
      if (w == 0.0 || (a.mask && !a.mask[m0])) continue;
      const double w2 = sW2[j2];
      if (w2 == 0.0) continue;
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        const double2 e = sE2[j2 * NB + c], y = sPhi[(j * NB + j1) * NB + c];
        re = fma(e.x, y.x, fma(e.y, y.y, re));
        im = fma(e.x, y.y, fma(-e.y, y.x, im));
      }
      const double W2 = re * re + im * im;
      for (int pr = 0; pr < 2; ++pr) {
        // + : partner k1; - : partner -k1 (same branch index; frequencies and velocities from its own entry)
        const double w1 = pr == 0 ? sW1[j1] : sW1n[j1];
        if (w1 == 0.0) continue;
        const double dw = __dsub_rn(pr == 0 ? __dadd_rn(w, w1) : __dsub_rn(w, w1), w2);
        const double sigma = sigma3(a, (pr == 0 ? sV1 : sV1n) + 3 * j1, sV2 + 3 * j2);
        const double sw = sigma < a.sigma_min ? a.sigma_min : sigma;
        if (!(fabs(dw) <= __dmul_rn(a.window, sw))) continue;
        const double delta = sigma < a.sigma_min ? 1.0 : exp(-(dw * dw) / (sigma * sigma)) / (sqrt(fp::kPi) * sigma);
        const double base = W2 * delta / (w * w1 * w2);
        const long long m1 = (long long)(pr == 0 ? k1 : kn) * NB + j1, m2 = (long long)k2 * NB + j2;
        for (int t = 0; t < nT; ++t) {
          const double n1 = a.bose[t * NM + m1], n2 = a.bose[t * NM + m2];
          sAcc[(size_t)o * nT + t] += pr == 0 ? (n1 - n2) * base : 0.5 * (n1 + n2 + 1.0) * base;
        }
        if (pr == 0)
          ++cplus;
        else
          ++cminus;
      }
    }
    __syncthreads();
  }
  // rate of (q, j): its entries (j, j1, j2) in order
  for (int o = tid; o < NB * nT; o += nthr) {
    const int j = o / nT, t = o % nT;
    double s = 0.0;
    for (int e = j * NB2; e < (j + 1) * NB2; ++e) s += sAcc[(size_t)e * nT + t];
    a.rates[t * NM + (long long)q * NB + j] = a.pref * s;
  }
  for (int off = 16; off > 0; off >>= 1) {
    cplus += __shfl_down_sync(0xffffffffu, cplus, off);
    cminus += __shfl_down_sync(0xffffffffu, cminus, off);
  }
  if ((tid & 31) == 0) {
    if (cplus) atomicAdd(a.counts, cplus);
    if (cminus) atomicAdd(a.counts + 1, cminus);
  }
}

size_t smem3_bytes(int nb, int n3, int nT) {
  const size_t nb3 = (size_t)nb * nb * nb, nb2 = (size_t)nb * nb;
  return (2 * nb3 + 3 * nb2 + n3) * sizeof(double2) + (nb3 * nT + 3 * nb + 9 * nb) * sizeof(double);
}

const void* rates3_ptr(int nb) {
  switch (nb) {
    case 3: return reinterpret_cast<const void*>(&rates3_kernel<3>);
    case 6: return reinterpret_cast<const void*>(&rates3_kernel<6>);
    case 12: return reinterpret_cast<const void*>(&rates3_kernel<12>);
    default: return nullptr;
  }
}

int fail3(fp_ctx* c, int code, const std::string& msg) {
  c->err = msg;
  return code;
}

}  // namespace

#define R3_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail3(c, e_ == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA,                      \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

extern "C" int fp_set_fc3(fp_ctx* c, int n_fc3, const fp_fc3* fc3) {
  if (!c) return FP_EINVAL;
  if (n_fc3 < 0 || (n_fc3 > 0 && !fc3)) return fail3(c, FP_EINVAL, "fp_set_fc3: bad triplet list");
  const int na = c->natoms;
  // group the triplets by atom triple; store Phi3 / sqrt(Mi Mj Mk) and the cells
  std::vector<std::vector<int>> by(na * na * na);
  for (int b = 0; b < n_fc3; ++b) {
    const fp_fc3& f = fc3[b];
    if (f.i < 0 || f.j < 0 || f.k < 0 || f.i >= na || f.j >= na || f.k >= na)
      return fail3(c, FP_EINVAL, "fp_set_fc3: atom index out of range");
    by[(f.i * na + f.j) * na + f.k].push_back(b);
  }
  std::vector<int> start(na * na * na + 1, 0), cell;
  std::vector<double> val;
  for (size_t t = 0; t < by.size(); ++t) {
    start[t + 1] = start[t] + (int)by[t].size();
    for (int b : by[t]) {
      const fp_fc3& f = fc3[b];
      for (int d = 0; d < 3; ++d) cell.push_back(f.Rj[d]);
      for (int d = 0; d < 3; ++d) cell.push_back(f.Rk[d]);
      const double m = std::sqrt(c->mass[f.i] * c->mass[f.j] * c->mass[f.k]);
      for (int x = 0; x < 27; ++x) val.push_back(f.fc[x] / m);
    }
  }
  R3_CUDA(cudaSetDevice(c->device));
  auto put = [&](auto*& dst, const auto& src) -> cudaError_t {
    using T = typename std::remove_reference<decltype(*dst)>::type;
    if (dst) cudaFree(dst);
    dst = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&dst), std::max<size_t>(1, src.size()) * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
  };
  R3_CUDA(put(c->d_t3_start, start));
  R3_CUDA(put(c->d_t3_cell, cell));
  R3_CUDA(put(c->d_t3_fc, val));
  c->n3 = n_fc3;
  c->have_fc3 = true;
  return FP_OK;
}

extern "C" int fp_rates3(fp_ctx* c, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
                         double* rates, fp_stats* stats) {
  if (!c) return FP_EINVAL;
  if (!rates) return fail3(c, FP_EINVAL, "fp_rates3: NULL output");
  if (!c->have_fc3) return fail3(c, FP_ESTATE, "fp_rates3: call fp_set_fc3 first");
  if (!c->have_modes) return fail3(c, FP_ESTATE, "fp_rates3: call fp_modes or fp_set_modes first");
  if (nT < 1 || nT > fp::kMaxT || !T) return fail3(c, FP_EINVAL, "fp_rates3: nT must be in [1, 8]");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0) || !std::isfinite(T[i])) return fail3(c, FP_EINVAL, "fp_rates3: temperatures must be > 0");
  if (!(scalebroad > 0.0) || !std::isfinite(scalebroad)) return fail3(c, FP_EINVAL, "fp_rates3: scalebroad must be > 0");
  fp_rates_opts o;
  fp_default_opts(&o);
  if (opts) o = *opts;
  if (o.window == 0.0) o.window = 2.0;
  if (o.sigma_min == 0.0) o.sigma_min = 1e-10;
  if (!(o.window > 0.0) || !(o.sigma_min > 0.0)) return fail3(c, FP_EINVAL, "fp_rates3: window, sigma_min > 0");
  if (o.dq_mode != 0 && o.dq_mode != 1) return fail3(c, FP_EINVAL, "fp_rates3: dq_mode must be 0 or 1");
  const int N = c->N, nb = c->nb;
  const int q_end = o.q_end > 0 ? o.q_end : N;
  if (o.q_begin < 0 || o.q_begin > q_end || q_end > N) return fail3(c, FP_EINVAL, "fp_rates3: bad q range");
  const void* k = rates3_ptr(nb);
  if (!k) return fail3(c, FP_EINVAL, "fp_rates3: nb must be 3, 6 or 12");
  const size_t nm = (size_t)N * nb;
  const size_t smem = smem3_bytes(nb, c->n3, nT);
  if (smem > 227 * 1024) return fail3(c, FP_EINVAL, "fp_rates3: tables do not fit in shared memory");
  R3_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  // working memory: T, occupation table, mask, counts, rates
  double *dT = nullptr, *dn = nullptr, *dr = nullptr;
  unsigned char* dm = nullptr;
  unsigned long long* dc = nullptr;
  auto cleanup = [&]() {
    cudaFree(dT);
    cudaFree(dn);
    cudaFree(dr);
    cudaFree(dm);
    cudaFree(dc);
  };
  cudaError_t e = cudaSuccess;
  if ((e = cudaMalloc(&dT, nT * sizeof(double))) != cudaSuccess || (e = cudaMalloc(&dn, nT * nm * sizeof(double))) ||
      (e = cudaMalloc(&dr, nT * nm * sizeof(double))) || (e = cudaMalloc(&dc, 2 * sizeof(unsigned long long))) ||
      (o.mode_mask && (e = cudaMalloc(&dm, nm)))) {
    cleanup();
    return fail3(c, e == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA, std::string("fp_rates3: ") + cudaGetErrorString(e));
  }
  Rates3Args a;
  std::memset(&a, 0, sizeof(a));
  a.N = N;
  a.nb = nb;
  a.nT = nT;
  a.L = c->L;
  a.n3 = c->n3;
  a.natoms = c->natoms;
  for (int d = 0; d < 3; ++d) {
    a.grid[d] = c->grid[d];
    a.Lfac[d] = c->L / c->grid[d];
  }
  a.omega = c->d_omega;
  a.evec = c->d_evec;
  a.vel = c->d_vel;
  a.tw = c->d_tw;
  a.t3_start = c->d_t3_start;
  a.t3_cell = c->d_t3_cell;
  a.t3_fc = c->d_t3_fc;
  a.bose = dn;
  a.mask = dm;
  a.q_begin = o.q_begin;
  a.nq_sel = q_end - o.q_begin;
  a.sb = scalebroad;
  a.window = o.window;
  a.sigma_min = o.sigma_min;
  const double* B = c->rec;
  const double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6]);
  a.dq = std::cbrt(std::fabs(detB) / (double)N);
  a.dq_mode = o.dq_mode;
  for (int i = 0; i < 9; ++i) a.rec[i] = B[i];
  a.pref = fp::kPi * fp::kHbar * fp::kConv * fp::kConv * fp::kConv / (4.0 * (double)N);
  a.rates = dr;
  a.counts = dc;
  bool ok = cudaMemcpyAsync(dT, T, nT * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            (!dm || cudaMemcpyAsync(dm, o.mode_mask, nm, cudaMemcpyHostToDevice, s) == cudaSuccess) &&
            cudaMemsetAsync(dr, 0, nT * nm * sizeof(double), s) == cudaSuccess &&
            cudaMemsetAsync(dc, 0, 2 * sizeof(unsigned long long), s) == cudaSuccess &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
            cudaEventRecord(c->ev0, s) == cudaSuccess;
  if (ok) {
    bose3_kernel<<<256, 256, 0, s>>>(c->d_omega, dT, nT, (long long)nm, dn);
    void* args[] = {&a};
    ok = cudaGetLastError() == cudaSuccess &&
         (a.nq_sel == 0 || cudaLaunchKernel(k, dim3(a.nq_sel), dim3(256), args, smem, s) == cudaSuccess) &&
         cudaEventRecord(c->ev1, s) == cudaSuccess;
  }
  unsigned long long cnt[2] = {0, 0};
  ok = ok && cudaMemcpyAsync(rates, dr, nT * nm * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
       cudaMemcpyAsync(cnt, dc, sizeof(cnt), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
       cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    const cudaError_t le = cudaGetLastError();
    cleanup();
    return fail3(c, FP_ECUDA, std::string("fp_rates3: ") + cudaGetErrorString(le));
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    double nsel = 0;
    for (int qq = o.q_begin; qq < q_end; ++qq)
      for (int j = 0; j < nb; ++j) nsel += (!o.mode_mask || o.mode_mask[(size_t)qq * nb + j]) ? 1 : 0;
    stats->candidates = 2.0 * nsel * (double)N * nb * nb;
    stats->accepted[0] = (double)cnt[0];
    stats->accepted[1] = (double)cnt[1];
    // per (q, k1): the reciprocal force constants (27 n3 real x complex) and three nb^4 contractions
    stats->flops = (double)a.nq_sel * N * (4.0 * 27.0 * c->n3 + 3.0 * 8.0 * nb * nb * nb * nb);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    stats->ms = ms;
    stats->tile[2] = 256;
    stats->tile[3] = a.nq_sel;
  }
  cleanup();
  return FP_OK;
}

namespace {

// RTA thermal conductivity (the tensor the paper's rates feed, Sec. 2.1): kappa_ab(T) = k_B / (N V)
// sum_l c(x_l) v_a v_b / rate_l, c(x) = x^2 e^x / (e^x - 1)^2 = (x/2 / sinh(x/2))^2, x = hbar w / (k_B T).
// One CTA per temperature; per-thread sums over a fixed mode stride, then a fixed-order tree in shared memory.
__global__ void kappa_kernel(const double* omega, const double* vel, const double* rates, const double* T, int nm,
                             double scale, double* kappa) {
  __shared__ double s[9][256];
  const int t = blockIdx.x, tid = threadIdx.x;
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int m = tid; m < nm; m += blockDim.x) {
    const double w = omega[m], r = rates[(size_t)t * nm + m];
    if (!(w > 0.0) || !(r > 0.0)) continue;
    const double h = 0.5 * fp::kHbar * w / (fp::kBoltzmann * T[t]);
    const double ch = h / sinh(h);
    const double f = ch * ch / r;
    const double* v = vel + 3 * (size_t)m;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) acc[3 * a + b] += f * v[a] * v[b];
  }
  for (int k = 0; k < 9; ++k) s[k][tid] = acc[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int k = 0; k < 9; ++k) s[k][tid] += s[k][tid + w];
    __syncthreads();
  }
  if (tid < 9) kappa[9 * t + tid] = scale * s[tid][0];
}

}  // namespace

extern "C" int fp_kappa_rta(fp_ctx* c, int nT, const double* T, const double* rates, double* kappa) {
  if (!c) return FP_EINVAL;
  if (!T || !rates || !kappa || nT < 1 || nT > fp::kMaxT) return fail3(c, FP_EINVAL, "fp_kappa_rta: bad arguments");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0) || !std::isfinite(T[i])) return fail3(c, FP_EINVAL, "fp_kappa_rta: temperatures must be > 0");
  if (!c->have_modes) return fail3(c, FP_ESTATE, "fp_kappa_rta: call fp_modes or fp_set_modes first");
  const int nm = c->N * c->nb;
  const double* A = c->lattice;
  const double vol = std::fabs(A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                               A[2] * (A[3] * A[7] - A[4] * A[6]));
  // k_B [J/K] (A/ps)^2 ps / A^3 = 1.380649e-23 * 1e4 * 1e-12 / 1e-30 W/(m K)
  const double scale = 1.380649e-23 * 1e4 * 1e-12 / 1e-30 / ((double)c->N * vol);
  R3_CUDA(cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  double *dT = nullptr, *dr = nullptr, *dk = nullptr;
  auto cleanup = [&]() {
    cudaFree(dT);
    cudaFree(dr);
    cudaFree(dk);
  };
  bool ok = cudaMalloc(&dT, nT * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&dr, (size_t)nT * nm * sizeof(double)) == cudaSuccess &&
            cudaMalloc(&dk, 9 * nT * sizeof(double)) == cudaSuccess &&
            cudaMemcpyAsync(dT, T, nT * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess &&
            cudaMemcpyAsync(dr, rates, (size_t)nT * nm * sizeof(double), cudaMemcpyHostToDevice, s) == cudaSuccess;
  if (ok) {
    kappa_kernel<<<nT, 256, 0, s>>>(c->d_omega, c->d_vel, dr, dT, nm, scale, dk);
    ok = cudaGetLastError() == cudaSuccess &&
         cudaMemcpyAsync(kappa, dk, 9 * nT * sizeof(double), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
         cudaStreamSynchronize(s) == cudaSuccess;
  }
  cleanup();
  if (!ok) return fail3(c, FP_ECUDA, "fp_kappa_rta: CUDA call failed");
  return FP_OK;
}
