/*
 * fourphonon.h -- C-ABI of libfourphonon: four-phonon RTA scattering rates on one GB300 GPU.
 *
 * The library computes, for every phonon mode lambda = (q, j) of a regular q-grid, the
 * four-phonon part of the relaxation-time-approximation rate (paper: Sec. 2.2, Eq. tao0):
 *
 *   1/tau_lambda = (1/N) [ sum_{++} 1/2 Gamma++ + sum_{+-} 1/2 Gamma+- + sum_{--} 1/6 Gamma-- ]
 *
 * with Gamma from Eq. 4phgamma, the vertex V4 from Eq. V4 (r_j = cell vector of atom j),
 * momentum q''' = q +- q' +- q'' (mod G) (Sec. 2.2, text of Eq. tao0), and the adaptive
 * Gaussian delta of Sec. 2.4 / App. B, sigma = scalebroad |v'' - v'''| |dq|.
 *
 * Units: lengths in Angstrom, masses in amu, Phi2 in eV/A^2, Phi4 in eV/A^4, T in K,
 * frequencies in rad/ps, velocities in A/ps, rates in 1/ps.
 *
 * Conventions shared by every call:
 *   - grid index g = (g1 * N2 + g2) * N3 + g3, q_g = sum_a (g_a / N_a) b_a, b_a the reciprocal
 *     vectors including 2 pi; mode index lambda = g * nb + j, nb = 3 * natoms; branches ascend in omega;
 *   - eigenvector layout [g][j][3 * atom + alpha] as (re, im) double pairs;
 *   - all host pointers are owned by the caller and only read (inputs) or written (outputs)
 *     during the call; the library copies what it keeps;
 *   - device memory is owned by the context; one context = one device + one CUDA stream;
 *     a context is not thread-safe;
 *   - every entry point returns FP_OK (0) or a negative FP_E* code; fp_last_error() then
 *     holds a one-line message.  On FP_ECUDA the context should be freed.
 */
#ifndef FOURPHONON_H
#define FOURPHONON_H

#ifdef __cplusplus
extern "C" {
#endif

#define FP_OK 0
#define FP_EINVAL (-1)     /* invalid argument (sizes, indices, masses, temperatures ...) */
#define FP_ENOMEM (-2)     /* device or host allocation failed */
#define FP_ECUDA (-3)      /* a CUDA call failed */
#define FP_EUNSTABLE (-4)  /* omega^2 < -1e-8 max(omega^2) away from the three Gamma acoustic modes */
#define FP_ESTATE (-6)     /* call out of order (e.g. rates before modes) */

#define FP_PREC_FP64 0  /* vertex, Gaussian and sums in FP64 (parity path, 1e-10 vs the FP64 definition) */
#define FP_PREC_MIXED 1 /* vertex and Gaussian in FP32, window decisions exact, sums in FP64 */
#define FP_PREC_DOUBLE_FLOAT 2 /* FP64 path whose vertex contraction (Eq. V4 assembly and the two contractions)
                                  runs on the FP32 pipes in double-float: pairs of floats with exact high products
                                  (fma residual) and two-sum accumulation, about 2^-46 per operation; window
                                  decisions, Gaussian, Bose factors and sums as in FP_PREC_FP64 */

typedef struct fp_ctx fp_ctx;

/* Harmonic pair block Phi2(0 i; R j), 3x3 row-major (alpha, beta), eV/A^2 (Sec. 2.3, Eq. PE). */
typedef struct {
  int i, j;
  int Rj[3];  /* cell of atom j in lattice coordinates */
  double fc[9];
} fp_fc2;

/* Fourth-order block Phi4(0 i; Rj j; Rk k; Rl l), 81 values row-major (alpha, beta, gamma, theta),
 * eV/A^4 (Sec. 2.3, Eqs. PE and fourth-order IFCs); atom i lies in the home cell. */
typedef struct {
  int i, j, k, l;
  int Rj[3], Rk[3], Rl[3];
  double fc[81];
} fp_fc4;

/* Options of fp_rates4.  Zero-initialised fields take the defaults of fp_default_opts(). */
typedef struct {
  int precision;                   /* FP_PREC_FP64 (default), FP_PREC_DOUBLE_FLOAT or FP_PREC_MIXED */
  double window;                   /* a term enters when |dw| <= window * max(sigma, sigma_min); default 2 */
  double sigma_min;                /* delta := 1 below this sigma (Sec. 2.4), rad/ps; default 1e-10 */
  int dq_mode;                     /* 0: |dq| = (|det B|/N)^(1/3); 1: per-axis sqrt(sum_a ((dv.b_a)/N_a)^2/3) */
  const unsigned char* mode_mask;  /* host, N*nb bytes, nonzero = compute this mode; NULL = all */
  int q_begin, q_end;              /* q-points [q_begin, q_end) get rates (others 0); q_end <= 0 means N */
  int block_j0;                    /* kernel tile: branches j per work item (must divide nb); 0 = auto */
  int k1_tile;                     /* kernel tile: q' points per work item; 0 = auto */
  int threads;                     /* threads per block (>= block_j0 * nb^2, multiple of 32); 0 = auto */
  int no_graph;                    /* 0: run the device part as a CUDA graph, captured on first use and replayed
                                      while the launch parameters are unchanged; 1: plain stream launches */
  int process_mask;                /* processes summed (Eq. 4phgamma): bit 0 ++ (recombination), bit 1 +-
                                      (redistribution), bit 2 -- (splitting); 0 = all three */
  int nu_select;                   /* 0: all processes; 1: normal only; 2: Umklapp only (Sec. 2.2: Q = 0 or not;
                                      the representatives are described at fp_rates4_nu) */
  int no_time_reversal;            /* 0 (default): time reversal (e^{-lambda} = conj e^{lambda}, Sec. 2.2) makes
                                      the rate of (-q, j) equal to that of (q, j) term by term (the terms at -q are
                                      those at q with every wavevector negated: equal frequencies, |V4|^2 and
                                      broadening), so one point of each pair {q, -q} is evaluated and its rates are
                                      written at both (up to the order of the sum, the rates at -q are those an
                                      evaluation at -q gives; accepted counts are exact); 1: evaluate every
                                      selected q.  The normal/Umklapp split (nu_select != 0) evaluates every q,
                                      because a zone-boundary tie breaks the symmetry of the representatives. */
  int tensor_cores;                /* 1: in the mixed precision with nb = 6, the per-q'' contraction T = A conj(E3)
                                      of Eq. V4's vertex runs on the fifth-generation tensor cores (tcgen05 kind::tf32
                                      in split precision, A = A_hi + A_lo and E = E_hi + E_lo in tf32, three
                                      products, FP32 accumulation in tensor memory); 0 (default): CUDA cores.
                                      FP_EINVAL for other precisions or branch counts. */
} fp_rates_opts;

/* Counters of one fp_rates4 call. */
typedef struct {
  double candidates;   /* process terms of the selected modes: (processes) * (selected modes) * N^2 * nb^3 */
  double accepted[3];  /* terms of the selected modes inside the energy window for ++, +-, -- */
  double flops;        /* vertex assembly + contraction flops executed (8 per complex multiply-add): the
                          hoisted prologue and assembly per evaluated item and q'-pair, and one nb-term
                          contraction per vertex entry formed (vertex_entries) */
  double ms;           /* device time of the rate kernels (CUDA events on the context stream) */
  int tile[4];         /* block_j0, k1_tile, threads, CTAs launched */
  double candidates_executed;  /* candidates the kernel screened: those of the evaluated rows (time reversal
                                  evaluates one point of each pair {q, -q}) */
  double vertex_entries;       /* vertex entries W(j0, j1, j2, j3) formed: those with an accepted candidate */
  double terms_executed;       /* accepted terms the kernel evaluated (Gaussian, Bose factors, |W|^2), all
                                  processes; accepted[] counts each once per selected mode it stands for */
} fp_stats;

/* Library version (major * 10000 + minor * 100 + patch). */
int fp_version(void);

/* Fill *opts with the defaults described in fp_rates_opts. */
void fp_default_opts(fp_rates_opts* opts);

/*
 * Create a context on `device` and upload the crystal: lattice rows a1..a3 (A), natoms fractional
 * positions (natoms x 3, informational: phases use cell vectors, Eq. V4), masses (amu, > 0), the
 * Phi2 pair list and the Phi4 quartet list, and the q-grid (each N_a in [1, 64]).  natoms must lie in
 * [1, 4]; the four- and three-phonon rate kernels are built for 1, 2 and 4 atoms (nb = 3, 6, 12), and
 * the rate calls return FP_EINVAL for 3.  Indices must lie in [0, natoms).  On success *out owns all device
 * memory of the problem; free it with fp_free().
 */
int fp_init(fp_ctx** out, const double lattice[9], int natoms, const double* frac_pos, const double* mass,
            int n_fc2, const fp_fc2* fc2, int n_fc4, const fp_fc4* fc4, const int grid[3], int device);

/* Use an existing CUDA stream (a cudaStream_t passed as void*) for all later work; NULL = the
 * context's own stream.  The caller keeps the stream alive while the context uses it. */
int fp_set_stream(fp_ctx* ctx, void* stream);

/*
 * Harmonic modes on the grid on the GPU (paper Sec. 2.1 harmonic step; velocities for Sec. 2.4):
 * omega (N x nb), evec (N x nb x nb x 2), vel (N x nb x 3); each output may be NULL.
 * Time reversal is exact (omega(-q) = omega(q), e(-q) = conj e(q), v(-q) = -v(q)), e is real and v = 0
 * at self-conjugate q, the three Gamma acoustic modes have omega = 0, velocities are averaged over
 * degenerate sets.  Returns FP_EUNSTABLE for imaginary frequencies.
 */
int fp_modes(fp_ctx* ctx, double* omega, double* evec, double* vel);

/*
 * Replace the modes by caller-supplied tables (same layouts as fp_modes).  The tables must obey
 * exact time reversal as described for fp_modes (checked bitwise; FP_EINVAL otherwise); omega must
 * be >= 0 and finite.
 */
int fp_set_modes(fp_ctx* ctx, const double* omega, const double* evec, const double* vel);

/*
 * Four-phonon RTA rates (Eqs. tao0, 4phgamma, V4; Sec. 2.4) at nT <= 8 temperatures T (K, > 0) with
 * broadening scale `scalebroad` (> 0).  rates: host, nT x N x nb, ps^-1, written in full (modes not
 * selected by the mask / q-range, and zero-frequency modes, get 0).  opts and stats may be NULL.
 * Requires fp_modes or fp_set_modes first (FP_ESTATE otherwise).
 */
int fp_rates4(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
              double* rates, fp_stats* stats);

/* As fp_rates4, but `d_rates` is a device pointer (nT x N x nb doubles) on the context's device;
 * the call returns after the work is complete on the context stream. */
int fp_rates4_device(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
                     double* d_rates, fp_stats* stats);

/*
 * Tile autotuner (the paper has no counterpart: it chooses launch tiles of this library's rate kernel).
 * Times every admissible (block_j0, k1_tile, threads) on a sample of q-points with opts->precision and
 * the given temperatures, writes the fastest into opts and remembers it in the context for calls whose
 * tile fields are 0 at that precision and temperature count.  best_ms (nullable) receives its time.
 */
int fp_autotune(fp_ctx* ctx, int nT, const double* T, double scalebroad, fp_rates_opts* opts, double* best_ms);

/*
 * fp_rates4_noalloc -- fp_rates4_device without any device allocation.  The paper has no counterpart;
 * this is a service of the library for callers that must not call cudaMalloc/cudaFree during the call,
 * e.g. an application whose device memory belongs to its own pool allocator with a fixed budget, or a
 * latency-critical caller that cannot accept the device synchronisation cudaFree implies.
 *
 * Same arguments and results as fp_rates4_device (d_rates: device pointer, nT x N x nb doubles,
 * caller-owned).  The context and its modes (fp_init, fp_modes or fp_set_modes) must already exist;
 * this call only uses them.  All working memory (Bose weights, per-work-item partial sums, queue and
 * accepted-term counters, temperatures, mode mask) comes from one static device array of 16 MiB that
 * every GPU loading the library holds until the process exits.  The q'-tile is enlarged automatically
 * to fit; a problem that still needs more than 16 MiB returns FP_EINVAL with the required size in
 * fp_last_error() (use fp_rates4_device for it).  The first call on a device looks up the array's
 * device address on that device; make that first call before starting any stream capture.  With CUDA's
 * lazy module loading (the default) that first call may also load the library's device code on the device
 * and reserve the array there, which is device memory taken then; make a warm-up call before the phase in
 * which nothing may be allocated.  Every call
 * shares the array (counters are cleared on each call), so calls whose GPU work overlaps -- other
 * streams, other contexts on the same device, other host threads -- race and must be serialised.
 */
int fp_rates4_noalloc(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
                      double* d_rates, fp_stats* stats);

/* ---------------------------------------------------------------------------------------------------
 * Phase space and the learned (surrogate) rates.
 */

/*
 * Three-phonon-like phase space of every mode, used as features of the surrogate (the paper's P3 and
 * WP3 outputs, Sec. 2.1, weighted as in Eq. 3phgamma without |V3|^2 and without hbar pi / 4):
 * processes q'' = q + q' (dw = (w + w') - w'') and q'' = q - q' (dw = (w - w') - w''), with the window,
 * Gaussian and small-sigma rule of fp_rates4 and sigma = scalebroad |v(q',j') - v(q'',j'')| |dq|.
 *   p3[m]        = (1/N) sum [ delta+ + 1/2 delta- ]                                 (host, N x nb; ps)
 *   wp3[t][m]    = (1/N) sum [ (n' - n'') delta+ + 1/2 (n' + n'' + 1) delta- ] / (w w' w'')   (host, nT x N x nb)
 * Either output may be NULL.  Requires modes (FP_ESTATE otherwise).
 */
int fp_phase3(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts, double* p3,
              double* wp3);

/*
 * Four-phonon weighted phase space of every mode: the sum of fp_rates4 with |V|^2 replaced by 1 and without
 * hbar^2 pi / 8, i.e. (1/N^2) sum over (q', q'') and branch triples of c_p B_p/n delta_p / (w w1 w2 w3)
 * (Eqs. tao0 and 4phgamma without V4; the paper's WP4 output, Sec. 2.1), estimated from q' on a stride
 * (stride 1 = the full sum; stride s uses every s-th q' with all q'', scaled by s).  FP32 Gaussian, exact
 * window decisions.  wp4: host, nT x N x nb.
 */
int fp_phase4(fp_ctx* ctx, int nT, const double* T, double scalebroad, int stride, double* wp4);

/*
 * Four-phonon phase space of every mode: the paper's onlyharmonic task with four_phonon on (Sec. 2.1), whose
 * outputs are BTE.Numprocess_4ph, BTE.P4 and BTE.WP4 (Appendix A).  The sums are those of fp_rates4 with |V4|^2
 * replaced by 1 and without hbar^2 pi / 8 (Eqs. tao0 and 4phgamma without V4), over q' on a stride (stride 1 =
 * the full sums; stride s uses every s-th q' with all q'' and scales by s):
 *   numprocess[m] = number of accepted process terms (q', q'', branch triple, process) of mode m (host, N x nb);
 *   p4[m]         = (1/N^2) sum c_p delta_p                                                (host, N x nb; ps);
 *   wp4[t][m]     = (1/N^2) sum c_p B_p/n delta_p / (w w' w'' w''')                        (host, nT x N x nb).
 * The paper prints no formula for P4 and WP4 (it cites them); these are the rate's sum with the vertex, and for
 * P4 also the Bose and frequency factors, set to 1.  Window, Gaussian, small-sigma rule, multiplicities c_p and
 * time reversal (stride 1) as in fp_rates4; opts: precision (FP64 default), window, sigma_min, dq_mode,
 * mode_mask, q range, process_mask and nu_select apply.  Any output may be NULL.  Two kernel passes (unit weights,
 * then Bose weights).  Requires modes (FP_ESTATE otherwise); FP_EINVAL for stride outside [1, N].
 */
int fp_phase_space4(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts, int stride,
                    double* numprocess, double* p4, double* wp4);

/*
 * Channel-resolved rates: the ++ (recombination), +- (redistribution) and -- (splitting) parts of Eq.
 * 4phgamma, whose sum is fp_rates4's rate.  rates: host, nT x 3 x N x nb, channel index in the order ++, +-,
 * --.  opts->process_mask must be 0.  Each channel is one rate-kernel pass (the vertex is recomputed), so
 * the call costs about three fp_rates4 calls.  stats (nullable) sums the candidates, flops and time of the
 * three passes; accepted[p] is channel p's count.  Errors as fp_rates4.
 */
int fp_rates4_channels(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts,
                       double* rates, fp_stats* stats);

/*
 * Third-order force constants for the three-phonon rates (Eq. V3): triplet (i, j, k) with atom i in the home
 * cell and atoms j, k in cells Rj, Rk (lattice units); fc[(a*3 + b)*3 + g] in eV/A^3.
 */
typedef struct {
  int i, j, k;
  int Rj[3], Rk[3];
  double fc[27];
} fp_fc3;

/*
 * Force-constant files (host only; no GPU is touched).  The paper's program reads the fourth-order force
 * constants from FORCE_CONSTANTS_4TH beside the third-order FORCE_CONSTANTS_3RD (Appendix A) and does not print
 * the layout.  These calls use the block layout of ShengBTE's third-order file, extended by one atom:
 *   <number of blocks> <blank> then per block: <block number, 1-based>; one line "x y z" per partner atom with
 *   the Cartesian position (A) of that atom's cell (n . A, A the lattice rows); the 1-based atom indices;
 *   3^order lines "alpha beta gamma [theta] value" (1-based Cartesian indices, eV/A^3 or eV/A^4); <blank>.
 * The first atom lies in the home cell.  Values are written with 17 significant digits, so writing and reading
 * back returns every value bit for bit.  Positions are read back as the nearest lattice vector, which must
 * reproduce them within 1e-6 A (FP_EINVAL otherwise).
 *   fp_write_fc4 / fp_write_fc3: write n blocks (fp_fc4 / fp_fc3, atom indices 0-based) to `path`.
 *   fp_read_fc4 / fp_read_fc3: *n receives the number of blocks in `path`; with out != NULL and cap >= *n the
 *   blocks are stored in out (0-based atom indices, cells in lattice coordinates).  out = NULL only counts.
 * Errors: FP_EINVAL (unreadable or malformed file, a position that is not a lattice vector, cap too small);
 * the message is in fp_last_error(NULL).
 */
int fp_write_fc4(const char* path, const double lattice[9], int n, const fp_fc4* fc4);
int fp_read_fc4(const char* path, const double lattice[9], fp_fc4* out, int cap, int* n);
int fp_write_fc3(const char* path, const double lattice[9], int n, const fp_fc3* fc3);
int fp_read_fc3(const char* path, const double lattice[9], fp_fc3* out, int cap, int* n);

/* Store (replace) the third-order force constants of the context.  The library copies them. */
int fp_set_fc3(fp_ctx* ctx, int n_fc3, const fp_fc3* fc3);

/*
 * Three-phonon RTA rates (Eqs. tao0, 3phgamma, V3): 1/tau3 = (1/N) [sum^(+) G+ + 1/2 sum^(-) G-] with
 * G+- = (hbar pi / 4) B+- |V+-|^2 delta(w +- w' - w'') / (w w' w''), B+ = n' - n'', B- = n' + n'' + 1,
 * q'' = q +- q'.  The broadening is sb |v' - v''| dq at the two partner modes (Sec. 2.4), with the window and
 * sigma_min rules of fp_rates4.  FP64.  opts: window, sigma_min, dq_mode, mode_mask and the q range apply;
 * the other fields are ignored.  rates: host, nT x N x nb, ps^-1 (add fp_rates4's rates for the total).
 * stats: candidates 2 N nb^2 per selected mode, accepted[0] (+) and accepted[1] (-).  FP_ESTATE before
 * fp_set_fc3 or the modes.
 */
int fp_rates3(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts, double* rates,
              fp_stats* stats);

/*
 * RTA lattice thermal conductivity from total rates (e.g. fp_rates3 + fp_rates4): kappa_ab(T) = k_B / (N V)
 * sum_l c(x_l) v_a(l) v_b(l) / rate_l with c(x) = x^2 e^x / (e^x - 1)^2, x = hbar w / (k_B T), V the cell
 * volume; modes with w = 0 or rate <= 0 are left out.  The paper's rates are the RTA input of this tensor
 * (Sec. 2.1, Eq. tao0); the paper has no kappa formula of its own, so this is the standard kinetic form.
 * rates: host, nT x N x nb (ps^-1); kappa: host, nT x 9 (row-major 3 x 3), W/(m K).  Uses the context's
 * modes.  FP_ESTATE before the modes.
 */
int fp_kappa_rta(fp_ctx* ctx, int nT, const double* T, const double* rates, double* kappa);

/*
 * Normal and Umklapp rates (the paper's separate normal and Umklapp RTA rate outputs, Appendix A): a process
 * q''' = q + s1 q' + s2 q'' + Q is normal when Q = 0 (Sec. 2.2).  Q depends on how each grid wavevector is
 * represented, which the paper does not state; here each is its shortest translate sum_a (g_a / N_a - m_a) b_a
 * over integers m_a in [-2, 2], with squared lengths within 1e-9 relative counted as equal and such ties won by
 * the lexicographically smallest (m_0, m_1, m_2).  rates: host, nT x 2 x N x nb (normal, then Umklapp); their
 * sum is fp_rates4's rate.  opts->nu_select must be 0; process_mask and the other options apply to both parts.
 * Two rate-kernel passes.  stats (nullable) sums the passes.  Errors as fp_rates4.
 */
int fp_rates4_nu(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_rates_opts* opts, double* rates,
                 fp_stats* stats);

/*
 * Stars of the q-grid (host only, no GPU).  Force constants that obey the crystal's space-group symmetry
 * (imposed on the IFCs in Sec. 2.3) give equal rates at q-points related by a point-group operation, so one
 * q-point per star suffices; the paper states no q-point reduction of its own.  rot: nrot integer 3x3
 * matrices, row-major, acting on the reciprocal-lattice fractional coordinates of q (q = sum_a f_a b_a,
 * f -> R f); generators suffice, the orbit is closed under them, and time reversal (q -> -q) is always
 * added.  An op may mix two grid axes only if they have the same number of points.  rep: N ints, out: the
 * smallest grid index of each point's star; *n_irr: the number of stars.  FP_EINVAL for a non-unimodular op
 * or one that mixes axes of unequal size.
 */
int fp_star_table(const int grid[3], int nrot, const int* rot, int* rep, int* n_irr);

/*
 * fp_rates4 evaluated on one q-point per star (fp_star_table) and mapped to the whole grid.  The caller
 * states that the force constants and masses are invariant under the ops; the rates of equivalent q are
 * then equal.  The rates of a degenerate set of branches (|dw| <= 1e-8 max w) depend on the basis chosen
 * inside the set, so every rate is returned as the mean over its degenerate set at the star's
 * representative.  opts: mode_mask and the q range must be unset and dq_mode 0 (dq_mode 1 is not
 * point-group invariant).  rates: host, nT x N x nb.  *n_irr (nullable): the number of stars evaluated;
 * stats: those of the rate pass.  Errors as fp_rates4, and FP_EINVAL as fp_star_table.
 */
int fp_rates4_irreducible(fp_ctx* ctx, int nrot, const int* rot, int nT, const double* T, double scalebroad,
                          const fp_rates_opts* opts, double* rates, fp_stats* stats, int* n_irr);

/* Number of parameters of the surrogate network for n_in input features (3 tanh layers of 128). */
int fp_mlp_params_size(int n_in);

/*
 * Loss and gradient of the surrogate network on one batch, on `device`, with the library's FP32 kernels:
 * y_hat = w4 . tanh(W3 tanh(W2 tanh(W1 x + b1) + b2) + b3) + b4, loss = mean (y_hat - y)^2.
 * X: batch x n_in (row-major), y: batch, params/grad: fp_mlp_params_size(n_in) floats packed as
 * W1 (128 x n_in), b1, W2 (128 x 128), b2, W3, b3, w4 (128), b4 (1).  Host pointers.
 */
int fp_mlp_loss_grad(int device, int n_in, int batch, const float* X, const float* y, const float* params,
                     float* grad, float* loss);

/* Options of fp_surrogate_fit; zero fields are not defaults: start from fp_surrogate_default_opts. */
typedef struct {
  double train_frac;       /* share of the pairs {q, -q} whose positive-frequency modes get exact training
                              rates (0.10); whole pairs, because the rate path evaluates a pair at once */
  double holdout_frac;     /* share of the pairs whose exact rates only judge the network (0.05) */
  double tol;              /* held-out relative error bound above which a bin falls back to exact rates (0.05) */
  unsigned long long seed; /* seeds the mode subsets, the initial weights and the minibatch order */
  int epochs;              /* Adam epochs (400) */
  int batch;               /* minibatch rows (1024) */
  double lr;               /* Adam learning rate (2e-3) */
  int precision;           /* precision of the exact evaluations, FP_PREC_* (mixed) */
} fp_surrogate_opts;

/* What fp_surrogate_fit did. */
typedef struct {
  int n_modes, n_train, n_holdout, n_fallback_modes, n_bins, n_bins_fallback;
  double final_loss;
  double holdout_median_rel_err, holdout_p90_rel_err, holdout_max_rel_err;
  double ms_exact, ms_features, ms_train, ms_predict, ms_fallback, ms_total;
} fp_surrogate_report;

void fp_surrogate_default_opts(fp_surrogate_opts* opts);

/*
 * Learned four-phonon rates (the paper has no learned component).  Exact rates (fp_rates4) of a seeded
 * train_frac share of the modes train a 3 x 128 tanh network on the GPU (hand-written forward, backward
 * and Adam kernels) that maps per-mode features (w, |v|, branch, T, n0, P3, WP3, WP4 sampled on every
 * (N/32)-th q', and the q-point as cos/sin(2 pi g_a / N_a)) to log(rate).  Exact
 * rates of a further holdout_frac share judge it per bin (branch x frequency quartile); a bin keeps the
 * network's rates only when it has at least 16 held-out (mode, T) rows and the upper confidence bound of
 * their mean relative error (mean + 2 standard errors) is within tol; every other bin is evaluated exactly.  Every
 * trained, held-out or fallback mode keeps its exact rate.  Results are read with fp_surrogate_rates.
 */
int fp_surrogate_fit(fp_ctx* ctx, int nT, const double* T, double scalebroad, const fp_surrogate_opts* opts,
                     fp_surrogate_report* report);

/*
 * Learned rates at new temperatures (the paper has no learned component): a temperature sweep with more
 * temperatures than one batched evaluation takes (8).  Exact rates (fp_rates4) of every mode at nA anchor
 * temperatures (one batched evaluation, 1 <= nA <= 8) and exact rates of a seeded train_frac share of the pairs
 * {q, -q} at the nT output temperatures (1 <= nT <= 64, evaluated 8 at a time) train the 3 x 128 tanh network on
 * the GPU (the same hand-written kernels as fp_surrogate_fit) to map, per (mode, T), the mode's anchor log rates,
 * log(T/300), log n0(T), w/w_max and a branch one-hot to log(rate(T)).  Exact rates of a further holdout_frac share
 * of the pairs judge it per bin (branch x frequency quartile) with the rule of fp_surrogate_fit; every other bin is
 * evaluated exactly at the output temperatures.  Every trained, held-out or fallback entry keeps its exact rate.
 *   rates: host nT x N x nb (ps^-1); used_exact: host nT x N x nb, 1 = exact, 0 = predicted; either may be NULL.
 * opts as for fp_surrogate_fit (NULL = defaults).  report (nullable): ms_exact covers the anchor and subset
 * evaluations.  FP_EINVAL for nA or nT out of range or temperatures <= 0; FP_ESTATE before the modes.
 */
int fp_surrogate_sweep(fp_ctx* ctx, int nA, const double* T_anchor, int nT, const double* T, double scalebroad,
                       const fp_surrogate_opts* opts, double* rates, unsigned char* used_exact,
                       fp_surrogate_report* report);

/* Rates of the last fp_surrogate_fit (host, nT x N x nb) and per-entry flags: 1 = exact, 0 = predicted. */
int fp_surrogate_rates(fp_ctx* ctx, double* rates, unsigned char* used_exact);

/* Release the context and all its device memory.  NULL is ignored. */
void fp_free(fp_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed fp_init when ctx is NULL). */
const char* fp_last_error(const fp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* FOURPHONON_H */
