// Internal definitions of libfourphonon (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fourphonon.h"

namespace fp {

// Physical constants (CODATA 2018 / SI exact).
constexpr double kHbar = 6.582119569e-4;     // eV ps
constexpr double kBoltzmann = 8.617333262e-5; // eV / K
constexpr double kECharge = 1.602176634e-19;  // C
constexpr double kAmu = 1.66053906660e-27;    // kg
// eV / (A^2 amu) in ps^-2: converts Phi2/M to omega^2 and, to the fourth power, hbar^2 |V4|^2 to ps^-6.
constexpr double kConv = kECharge / kAmu * 1e20 * 1e-24;
constexpr double kInvSqrtPi = 0.56418958354775628695;  // 1/sqrt(pi)
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxNb = 12;  // up to 4 atoms per cell (36 branches would not fit the on-chip tiles)
constexpr int kMaxT = 16;   // temperatures per call

// Work description of one rates launch (all device pointers).
struct RatesArgs {
  int N, nb, natoms, nT, L, G, nquart;
  int grid[3], Lfac[3];
  int J, t1, nchunk, ntile, q_begin, nq_sel;
  long long n_items;
  const double* omega;       // [N][nb]
  const double2* evec;       // [N][nb][nb]
  const double* vel;         // [N][nb][3]
  const double* wt;          // [nT][N*nb][3]: 1/(n w), (1+n)/w, n/w
  const int* qmeta;          // [nquart][9]: i, j, group, Rj[3], Rl[3]
  const double* qfc;         // [nquart][81], divided by sqrt(Mi Mj Mk Ml)
  const int* gmeta;          // [G][5]: k, l, D = Rk - Rl
  const int* grp_qstart;     // [G+1]
  const int* grp_q;          // [nquart]
  const int* kl_start;       // [natoms^2 + 1]
  const int* kl_grp;         // [G]
  const double2* tw;         // [L]: exp(2 pi i m / L)
  const unsigned char* mask; // [N*nb] or null
  double sb, window, sigma_min, dq;
  int dq_mode;
  double rec[9];
  double* partial;           // [n_items][J][nT]
  unsigned long long* counter;
  unsigned long long* counts; // [3]
};

}  // namespace fp

// The opaque context of the C-ABI.
struct fp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  int natoms = 0, nb = 0, N = 0, L = 1;
  int grid[3] = {1, 1, 1};
  double lattice[9] = {0}, rec[9] = {0};
  std::vector<double> mass;
  // harmonic force constants
  int n_fc2 = 0;
  int* d_fc2_idx = nullptr;     // [n_fc2][5]: i, j, R[3]
  double* d_fc2_val = nullptr;  // [n_fc2][9]
  double* d_mass = nullptr;
  // fourth-order force constants and their grouping
  int nquart = 0, G = 0;
  int* d_qmeta = nullptr;
  double* d_qfc = nullptr;
  int* d_gmeta = nullptr;
  int* d_grp_qstart = nullptr;
  int* d_grp_q = nullptr;
  int* d_kl_start = nullptr;
  int* d_kl_grp = nullptr;
  double2* d_tw = nullptr;
  // modes
  bool have_modes = false;
  double* d_omega = nullptr;
  double2* d_evec = nullptr;
  double* d_vel = nullptr;
  int* d_flag = nullptr;
  // per-call scratch (grown on demand)
  double* d_wt = nullptr;
  size_t wt_cap = 0;
  double* d_partial = nullptr;
  size_t partial_cap = 0;
  unsigned long long* d_counters = nullptr;  // [0]: queue, [1..3]: accepted counts
  double* d_T = nullptr;
  unsigned char* d_mask = nullptr;
  double* d_rates = nullptr;
  size_t rates_cap = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace fp {
// Kernels launchers (implemented in fp_modes.cu / fp_rates.cu); each returns a cudaError_t.
cudaError_t launch_scale_fc4(double* qfc, const int* d_atoms4, const double* d_mass, int nquart, cudaStream_t s);
cudaError_t launch_twiddles(fp_ctx* c, cudaStream_t s);
cudaError_t launch_modes(fp_ctx* c, cudaStream_t s);
cudaError_t launch_weights(fp_ctx* c, int nT, const double* d_T, double* d_wt, cudaStream_t s);
cudaError_t launch_rates(const RatesArgs& a, int precision, int threads, int ctas, size_t smem, cudaStream_t s);
cudaError_t launch_reduce(const RatesArgs& a, double pref, double* d_rates, int q_end, cudaStream_t s);
size_t rates_smem_bytes(int precision, int nb, int J, int G, int nquart, int nT, int threads);
int rates_max_ctas_per_sm(int precision, int threads, size_t smem);
}  // namespace fp
