// Internal definitions of libfourphonon (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>

#include <array>
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
constexpr int kMaxT = 8;    // temperatures per call

// Work description of one rates launch (all device pointers).
struct RatesArgs {
  int N, nb, natoms, nT, L, G, nquart;
  int grid[3], Lfac[3];
  int J, t1, nchunk, ntile, nq_sel;
  long long n_items;
  const int* qlist;          // [nq_sel] the q-points the kernel evaluates (work item -> q)
  const unsigned char* mult; // [N*nb] selected modes each evaluated row stands for: 0, 1, or 2 when the row's
                             // rate is also written at -q (time reversal); weights the accepted counts
  // reduction: outputs q in [q_out_begin, q_out_begin + q_out_n); a selected mode (sel) of q takes the partial
  // sums of the evaluated point qlist[qpos[q]] (q itself, or -q under time reversal)
  int q_out_begin, q_out_n;
  const int* qpos;           // [N]
  const unsigned char* sel;  // [N*nb]
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
  // FP32 copies prepared once per call (prep_kernel)
  const float* omh;          // [N*nb] two-float frequencies: omh + oml = omega
  const float* oml;
  const float* velh;         // [N*nb*3] two-float velocities
  const float* vell;
  const float2* evf;         // [N][nb][nb]
  const float* qfcf;         // [nquart][81]
  const float2* twf;         // [L]
  const float* wtf;          // [nT][N*nb][3]
  double sb, window, sigma_min, dq;
  int dq_mode;
  double rec[9];
  double* partial;           // [n_items][J][nT]
  unsigned long long* counter;
  unsigned long long* counts; // [6]: accepted ++, +-, -- (weighted by mult), vertex entries W formed, accepted
                              // terms evaluated, tensor-core completion waits that ran out of polls
  int unit_vertex;           // 1: |W|^2 = 1 (weighted phase space), q' on a stride, ordered (q', q'') pairs
  int k1_stride;             // q' stride of the unit-vertex mode
  unsigned cand_mask;        // candidates summed (bit c = ordering * 3 + process), from process_mask
  int nu_select;             // 0: all processes, 1: normal only, 2: Umklapp only
  const int* bzm;            // [N][3] Brillouin-zone shifts of the grid points (normal/Umklapp reading)
  unsigned long long* item_counts;  // [n_items][J] accepted terms per (item, j0), or null (not counted)
  double* mode_counts;       // [N*nb] reduction output: accepted terms per selected mode x count_scale, or null
  double count_scale;
};

// Which q-points a rates call evaluates, and for which modes.  Time reversal (e^{-lambda} = conj e^{lambda},
// Sec. 2.2) makes the rate of (-q, j) equal to that of (q, j) term by term: the terms at -q are those at q with
// every wavevector negated, with the same frequencies, |V|^2 and broadening.  With `fold` the kernel evaluates
// one point of each pair {q, -q} (the smaller index) and the reduction writes both.
struct Selection {
  bool fold = false;
  int q_out_begin = 0, q_out_end = 0;
  std::vector<int> qlist;           // evaluated q-points, ascending
  std::vector<int> qpos;            // [N] index in qlist of the point evaluated for q (-1: none)
  std::vector<unsigned char> mult;  // [N*nb] selected modes an evaluated row stands for (0, 1, 2)
  std::vector<unsigned char> sel;   // [N*nb] 1 = the rate of this mode is written
  double n_sel = 0;                 // selected modes
  double n_exec = 0;                // evaluated rows with mult > 0
  long long active_chunks = 0;      // (evaluated q, branch chunk) pairs with a row of mult > 0 (set by plan_rates)
};

// Tile plan of one rates call.
struct Plan {
  int J, threads, t1, nchunk, ntile, nq_sel, ctas;
  long long n_items;
  size_t smem;
};

// Device working memory of one rates call (owned by the caller of run_rates), in the order of scratch_sizes.
constexpr int kScratchParts = 16;
constexpr int kScratchPartial = 7;  // index of the per-item partial sums
constexpr int kCounters = 8;        // queue, accepted ++, +-, --, vertex entries, terms evaluated, wait timeouts, spare
struct Scratch {
  unsigned long long* counters;  // [kCounters]
  double* T;                     // [kMaxT]
  unsigned char* mult;           // [N*nb]
  unsigned char* sel;            // [N*nb]
  int* qlist;                    // [N]
  int* qpos;                     // [N]
  double* wt;                    // [nT][N*nb][3]
  double* partial;               // [n_items][J][nT]
  float* omh;                    // [N*nb]
  float* oml;
  float* velh;                   // [N*nb*3]
  float* vell;
  float2* evf;                   // [N*nb*nb]
  float* qfcf;                   // [nquart*81]
  float2* twf;                   // [L]
  float* wtf;                    // [nT][N*nb][3]
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
  int* d_bzm = nullptr;  // [N][3] Brillouin-zone shifts (bz_shifts)
  // third-order force constants (fp_set_fc3), grouped by atom triple
  bool have_fc3 = false;
  int n3 = 0;
  int* d_t3_start = nullptr;   // [natoms^3 + 1]
  int* d_t3_cell = nullptr;    // [n3][6] Rj, Rk
  double* d_t3_fc = nullptr;   // [n3][27] Phi3 / sqrt(Mi Mj Mk)
  // modes
  bool have_modes = false;
  double* d_omega = nullptr;
  double2* d_evec = nullptr;
  double* d_vel = nullptr;
  int* d_flag = nullptr;
  // per-call working memory (grown on demand) and the output staging buffer of fp_rates4
  unsigned char* d_scratch = nullptr;
  size_t scratch_cap = 0;
  double* d_rates = nullptr;
  size_t rates_cap = 0;
  int* d_star = nullptr;  // star representatives (fp_rates4_irreducible)
  size_t star_cap = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // tiles chosen by fp_autotune, per (precision FP_PREC_*, one or several temperatures): J, k1 tile, threads
  int tuned[3][2][3] = {};
  // the captured rate step and the launch parameters it was captured with
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<unsigned char> graph_key;
  // result of the last fp_surrogate_fit
  int sur_nT = 0;
  std::vector<double> sur_rates;
  std::vector<unsigned char> sur_used;
  std::string err;
};

namespace fp {
// Support kernels (fp_modes.cu).
cudaError_t launch_scale_fc4(double* qfc, const int* d_atoms4, const double* d_mass, int nquart, cudaStream_t s);
cudaError_t launch_twiddles(fp_ctx* c, cudaStream_t s);
cudaError_t launch_modes(fp_ctx* c, cudaStream_t s);
cudaError_t launch_weights(fp_ctx* c, int nT, const double* d_T, double* d_wt, cudaStream_t s);

// Rate path (fp_rates.cu).
// The evaluated q-points and mode weights of a call: the q range and mode mask of `o`, folded by time reversal
// unless o.no_time_reversal or o.nu_select is set or fold_allowed is false.  FP_EINVAL on a bad q range.
int make_selection(const fp_ctx* c, const fp_rates_opts& o, bool fold_allowed, Selection* s, std::string* err);
// Validate options and choose tiles; `partial_budget` (bytes, 0 = unlimited) enlarges the q'-tile until the
// per-item partial sums fit.  Returns FP_OK or an FP_E* code with a message in *err.
int plan_rates(fp_ctx* c, const fp_rates_opts& o, int nT, Selection& sel, size_t partial_budget, Plan* p,
               std::string* err);
// Byte sizes of the Scratch buffers of a plan, in the order of the Scratch fields (each rounded up to 256).
void scratch_sizes(const fp_ctx* c, const Plan& p, int nT, size_t sizes[kScratchParts]);
// Scratch pointers laid out from `base` with the sizes of scratch_sizes.
Scratch carve_scratch(unsigned char* base, const size_t sizes[kScratchParts]);
// Variants of a rates launch used by the phase-space entry points.
struct RunExtra {
  int unit_stride = 0;          // > 0: |W|^2 := 1, q' on this stride, ordered (q', q'') pairs, no prefactor
  bool unit_weights = false;    // Bose and frequency weights := 1 (the unweighted phase space)
  unsigned long long* d_item_counts = nullptr;  // [n_items][J]: with d_mode_counts, per-mode accepted terms
  double* d_mode_counts = nullptr;              // [N*nb] accepted terms of each selected mode x unit_stride
};
// Upload the selection, enqueue weights, FP32 prep, the persistent rate kernel and the reduction on c->stream,
// then wait and return the counters.  d_out: nT x N x nb doubles (zeroed here).
// use_graph: capture the device part once per set of launch parameters and replay it as a CUDA graph.
int run_rates(fp_ctx* c, const fp_rates_opts& o, const Selection& sel, const Plan& p, const Scratch& s, int nT,
              const double* T, double sb, double* d_out, unsigned long long counts[kCounters], bool use_graph,
              std::string* err, const RunExtra& x = RunExtra());
// Sampled four-phonon weighted phase space of every mode (surrogate feature): the rate sum with |W|^2 = 1
// over q' on a stride (ordered pairs), scaled to the full grid; d_out: nT x N x nb, mixed precision.
int phase4_sampled(fp_ctx* c, int nT, const double* T, double sb, int stride, double* d_out, std::string* err);
// Brillouin-zone shifts of the grid points (fp_sym.cu), N x 3
void bz_shifts(const int grid[3], const double rec[9], int* out);
// Record a message for fp_last_error(NULL) (calls without a context) and return code.
int fail_global(int code, const std::string& msg);
void fill_stats(const fp_ctx* c, const fp_rates_opts& o, const Selection& sel, const Plan& p,
                const unsigned long long counts[kCounters], fp_stats* st);
}  // namespace fp
