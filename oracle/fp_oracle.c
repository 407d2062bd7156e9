/*
 * Plain FP64 CPU oracle for the four-phonon RTA scattering rates.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It shares no code, header,
 * table or constant generator with the CUDA path; it is written to be read
 * against the paper, not to be fast.
 *
 * What it computes (paper, Sec. 2.2 and 2.4):
 *   1/tau_4ph(lambda) = (1/N) [ sum_{++} 1/2 Gamma++ + sum_{+-} 1/2 Gamma+- + sum_{--} 1/6 Gamma-- ]  (Eq. tao0)
 *   Gamma_p = hbar^2 pi / (8N) * B_p / n_lambda * |V_p|^2 * delta(dw_p) / (w w' w'' w''')           (Eq. 4phgamma)
 *     B++ = (1+n')(1+n'')n''',  B+- = (1+n')n''n''',  B-- = n'n''n'''
 *   V_p from Eq. V4: sum over quartets (i in the home cell; j,k,l in cells R_j,R_k,R_l) and
 *     Cartesian indices of Phi4 e^{lambda}(i) e^{s1 lambda'}(j) e^{s2 lambda''}(k) e^{-lambda'''}(l)
 *     / sqrt(M_i M_j M_k M_l) * exp(i (s1 q'.R_j + s2 q''.R_k - q'''.R_l)),  e^{-lambda} = conj(e^{lambda}).
 *   Momentum: q''' = q + s1 q' + s2 q'' (mod the reciprocal lattice), all q on the regular grid.
 *   delta(dw) = exp(-dw^2/sigma^2)/(sqrt(pi) sigma), sigma = scalebroad |v'' - v'''| |dq| (Sec. 2.4,
 *     App. B), with delta := 1 when sigma < sigma_min (the small-sigma rule of Sec. 2.4).
 *
 * Readings where the paper is silent (stated in the design notes): units A, amu, eV, K, rad/ps;
 * a term enters only when |dw| <= window * max(sigma, sigma_min) (window = 2 by default), so that
 * the small-sigma rule applies on a window of width window * sigma_min; dw is evaluated as
 * ((w + s1 w') + s2 w'') - w''' in FP64 without contraction; sigma as (sb * sqrt((dx^2 + dy^2) + dz^2)) * dq;
 * terms with a zero-frequency mode are skipped and a zero-frequency lambda has rate 0;
 * |dq| = (|det B| / N)^(1/3) (isotropic) or the per-axis form sqrt(sum_a ((dv.b_a)/N_a)^2 / 3).
 *
 * Build with -ffp-contract=off so that the screening arithmetic is evaluated exactly as written.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* CODATA 2018 / SI exact values */
#define ORC_HBAR 6.582119569e-4      /* eV ps */
#define ORC_KB 8.617333262e-5        /* eV / K */
#define ORC_ECHARGE 1.602176634e-19  /* C */
#define ORC_AMU 1.66053906660e-27    /* kg */

/* eV / (A^2 amu) expressed in ps^-2 */
static double orc_conv(void) { return ORC_ECHARGE / ORC_AMU * 1e20 * 1e-24; }

typedef struct {
  int grid[3];
  int nq, natoms, nb;
  double lat[9];  /* rows a1, a2, a3 (A) */
  double rec[9];  /* rows b1, b2, b3 (1/A), a_i . b_j = 2 pi delta_ij */
  const double* mass;
  int nquart;
  const int* qidx;   /* nquart x 13: i j k l Rj[3] Rk[3] Rl[3] */
  const double* qfc; /* nquart x 81 */
  const double* omega; /* nq x nb */
  const double* evec;  /* nq x nb(branch) x nb(component) x 2 */
  const double* vel;   /* nq x nb x 3 */
} orc_problem;

static void orc_setup(orc_problem* p, const int grid[3], const double lattice[9], int natoms,
                      const double* mass, int nquart, const int* qidx, const double* qfc,
                      const double* omega, const double* evec, const double* vel) {
  for (int a = 0; a < 3; ++a) p->grid[a] = grid[a];
  p->nq = grid[0] * grid[1] * grid[2];
  p->natoms = natoms;
  p->nb = 3 * natoms;
  memcpy(p->lat, lattice, 9 * sizeof(double));
  /* B = 2 pi (A^{-1})^T, rows b_a */
  const double* A = lattice;
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
               A[2] * (A[3] * A[7] - A[4] * A[6]);
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) p->rec[3 * a + c] = 2.0 * M_PI * inv[3 * c + a];
  p->mass = mass;
  p->nquart = nquart;
  p->qidx = qidx;
  p->qfc = qfc;
  p->omega = omega;
  p->evec = evec;
  p->vel = vel;
}

static int orc_idx(const orc_problem* p, const int g[3]) {
  return (g[0] * p->grid[1] + g[1]) * p->grid[2] + g[2];
}

static void orc_unidx(const orc_problem* p, int q, int g[3]) {
  g[2] = q % p->grid[2];
  g[1] = (q / p->grid[2]) % p->grid[1];
  g[0] = q / (p->grid[1] * p->grid[2]);
}

static int orc_wrap(int x, int n) { return ((x % n) + n) % n; }

/* Cartesian wavevector of grid point g: q = sum_a (g_a / N_a) b_a */
static void orc_qcart(const orc_problem* p, int q, double out[3]) {
  int g[3];
  orc_unidx(p, q, g);
  for (int c = 0; c < 3; ++c) {
    out[c] = 0.0;
    for (int a = 0; a < 3; ++a) out[c] += ((double)g[a] / (double)p->grid[a]) * p->rec[3 * a + c];
  }
}

static void orc_rcart(const orc_problem* p, const int n[3], double out[3]) {
  for (int c = 0; c < 3; ++c) {
    out[c] = 0.0;
    for (int a = 0; a < 3; ++a) out[c] += (double)n[a] * p->lat[3 * a + c];
  }
}

static cplx orc_e(const orc_problem* p, int q, int branch, int comp) {
  const double* e = p->evec + (((size_t)q * p->nb + branch) * p->nb + comp) * 2;
  return e[0] + I * e[1];
}

static double orc_bose(double w, double T) { return 1.0 / expm1(ORC_HBAR * w / (ORC_KB * T)); }

/*
 * Normal / Umklapp (Sec. 2.2: q''' = q + s1 q' + s2 q'' + Q, with Q = 0 for a normal process).  Reading:
 * each grid wavevector is taken as its shortest translate k = sum_a (g_a / N_a - m_a) b_a over integers m_a in
 * [-2, 2]; squared lengths within 1e-9 relative of each other are a tie, won by the lexicographically
 * smallest m.  The process is normal when these representatives satisfy q + s1 q' + s2 q'' - q''' = 0.
 */
static void orc_bz_shift(const orc_problem* p, int q, int m[3]) {
  int g[3];
  orc_unidx(p, q, g);
  double best = -1.0;
  for (int m0 = -2; m0 <= 2; ++m0)
    for (int m1 = -2; m1 <= 2; ++m1)
      for (int m2 = -2; m2 <= 2; ++m2) {
        const int mm[3] = {m0, m1, m2};
        double k2 = 0.0;
        for (int c = 0; c < 3; ++c) {
          double kc = 0.0;
          for (int a = 0; a < 3; ++a) kc += ((double)g[a] / (double)p->grid[a] - (double)mm[a]) * p->rec[3 * a + c];
          k2 += kc * kc;
        }
        /* the loops run in lexicographic order of m, so a tie keeps the earlier (smaller) m */
        if (best < 0.0 || k2 < best * (1.0 - 1e-9)) {
          best = k2;
          m[0] = m0;
          m[1] = m1;
          m[2] = m2;
        }
      }
}

/* 1 if process (s1, s2) with partners q1, q2 (q3 = q + s1 q1 + s2 q2 on the grid) is Umklapp, else 0;
   shift: nq x 3, orc_bz_shift of every grid point */
static int orc_is_umklapp(const orc_problem* p, const int* shift, int q, int q1, int q2, int s1, int s2) {
  int g[3], g1[3], g2[3], g3[3];
  orc_unidx(p, q, g);
  orc_unidx(p, q1, g1);
  orc_unidx(p, q2, g2);
  for (int a = 0; a < 3; ++a) g3[a] = orc_wrap(g[a] + s1 * g1[a] + s2 * g2[a], p->grid[a]);
  const int* m = shift + 3 * q;
  const int* m1 = shift + 3 * q1;
  const int* m2 = shift + 3 * q2;
  const int* m3 = shift + 3 * orc_idx(p, g3);
  for (int a = 0; a < 3; ++a) {
    /* N_a times the a-th reduced coordinate of q + s1 q1 + s2 q2 - q3, taken in the representatives */
    const int n = p->grid[a];
    const int num = (g[a] - n * m[a]) + s1 * (g1[a] - n * m1[a]) + s2 * (g2[a] - n * m2[a]) - (g3[a] - n * m3[a]);
    if (num != 0) return 1;
  }
  return 0;
}

/* Third wavevector of process (s1, s2): q''' = q + s1 q' + s2 q'' on the grid. */
static int orc_third(const orc_problem* p, int q, int q1, int q2, int s1, int s2) {
  int g[3], g1[3], g2[3], g3[3];
  orc_unidx(p, q, g);
  orc_unidx(p, q1, g1);
  orc_unidx(p, q2, g2);
  for (int a = 0; a < 3; ++a) g3[a] = orc_wrap(g[a] + s1 * g1[a] + s2 * g2[a], p->grid[a]);
  return orc_idx(p, g3);
}

/*
 * Reciprocal-space force constants of process (s1, s2) for the wavevector triple (q', q'', q''') (Eq. V4):
 *   phi[(i a)(j b)(k c)(l d)] = sum_{quartets with these atoms} Phi4 / sqrt(M_i M_j M_k M_l)
 *                                 * exp(i (s1 q'.R_j + s2 q''.R_k - q'''.R_l))
 */
static void orc_phi(const orc_problem* p, int q1, int q2, int q3, int s1, int s2, cplx* phi) {
  const int nb = p->nb;
  double k1[3], k2[3], k3[3];
  orc_qcart(p, q1, k1);
  orc_qcart(p, q2, k2);
  orc_qcart(p, q3, k3);
  memset(phi, 0, sizeof(cplx) * (size_t)nb * nb * nb * nb);
  for (int Q = 0; Q < p->nquart; ++Q) {
    const int* ix = p->qidx + 13 * Q;
    double rj[3], rk[3], rl[3];
    orc_rcart(p, ix + 4, rj);
    orc_rcart(p, ix + 7, rk);
    orc_rcart(p, ix + 10, rl);
    double ang = 0.0;
    for (int c = 0; c < 3; ++c) ang += s1 * k1[c] * rj[c] + s2 * k2[c] * rk[c] - k3[c] * rl[c];
    cplx ph = cos(ang) + I * sin(ang);
    double msq = sqrt(p->mass[ix[0]] * p->mass[ix[1]] * p->mass[ix[2]] * p->mass[ix[3]]);
    const double* fc = p->qfc + 81 * Q;
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be)
        for (int ga = 0; ga < 3; ++ga)
          for (int th = 0; th < 3; ++th) {
            int a = 3 * ix[0] + al, b = 3 * ix[1] + be, c = 3 * ix[2] + ga, d = 3 * ix[3] + th;
            phi[((a * nb + b) * nb + c) * nb + d] += fc[((al * 3 + be) * 3 + ga) * 3 + th] / msq * ph;
          }
  }
}

/* V_p(lambda, lambda', lambda'', lambda''') = sum_abcd phi[abcd] e^{l}_a e^{s1 l'}_b e^{s2 l''}_c conj(e^{l'''}_d) */
static cplx orc_vertex(const orc_problem* p, const cplx* phi, int q, int j, int q1, int j1, int q2, int j2,
                       int q3, int j3, int s1, int s2) {
  const int nb = p->nb;
  cplx acc = 0.0;
  for (int a = 0; a < nb; ++a) {
    cplx ea = orc_e(p, q, j, a);
    for (int b = 0; b < nb; ++b) {
      cplx eb = orc_e(p, q1, j1, b);
      if (s1 < 0) eb = conj(eb);
      for (int c = 0; c < nb; ++c) {
        cplx ec = orc_e(p, q2, j2, c);
        if (s2 < 0) ec = conj(ec);
        for (int d = 0; d < nb; ++d) {
          cplx ed = conj(orc_e(p, q3, j3, d));
          acc += phi[((a * nb + b) * nb + c) * nb + d] * ea * eb * ec * ed;
        }
      }
    }
  }
  return acc;
}

static double orc_dq_iso(const orc_problem* p) {
  const double* B = p->rec;
  double det = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
               B[2] * (B[3] * B[7] - B[4] * B[6]);
  return cbrt(fabs(det) / (double)p->nq);
}

/* sigma = scalebroad |v'' - v'''| |dq| (Sec. 2.4); evaluated in a fixed order. */
static double orc_sigma(const orc_problem* p, const double* v2, const double* v3, double sb, double dq,
                        int dq_mode) {
  double dx = v2[0] - v3[0];
  double dy = v2[1] - v3[1];
  double dz = v2[2] - v3[2];
  if (dq_mode == 0) {
    double s = (dx * dx + dy * dy) + dz * dz;
    return (sb * sqrt(s)) * dq;
  }
  double pa[3];
  for (int a = 0; a < 3; ++a) {
    const double* b = p->rec + 3 * a;
    pa[a] = ((dx * b[0] + dy * b[1]) + dz * b[2]) / (double)p->grid[a];
  }
  double s = ((pa[0] * pa[0] + pa[1] * pa[1]) + pa[2] * pa[2]) / 3.0;
  return sb * sqrt(s);
}

static const int ORC_S1[3] = {+1, +1, -1};
static const int ORC_S2[3] = {+1, -1, -1};
static const double ORC_MULT[3] = {0.5, 0.5, 1.0 / 6.0};

/*
 * Four-phonon RTA rates of selected modes.
 *   sel[s] = q * nb + j (mode id); rates[t * nsel + s] in ps^-1.
 *   accepted[3]: number of terms that passed the energy window, per process, over the selected modes.
 *   unit_vertex: 0 the rates; 1 replaces |V|^2 by 1 (the weighted phase space WP4 of the same processes); 2 also
 *   replaces B_p / n_lambda / (w w' w'' w''') by 1 (the phase space P4: sum of c_p delta_p).  With 1 or 2 the sum
 *   is returned without the prefactor hbar^2 pi / (8 N^2) and without the 1/N^2.
 *   proc_mask selects the process classes summed in Eq. 4phgamma: bit 0 ++ (recombination), bit 1 +-
 *   (redistribution), bit 2 -- (splitting); 7 gives the full rate.
 *   nu_select: 0 all processes, 1 normal ones only, 2 Umklapp ones only (orc_is_umklapp).
 * Returns 0, or -1 on bad arguments.
 */
int oracle_rates4(const int grid[3], const double lattice[9], int natoms, const double* mass, int nquart,
                  const int* qidx, const double* qfc, const double* omega, const double* evec,
                  const double* vel, int nT, const double* T, double scalebroad, double window,
                  double sigma_min, int dq_mode, int nsel, const int* sel, int unit_vertex, int proc_mask,
                  int nu_select, int nthreads, double* rates, double* accepted) {
  if (!grid || !lattice || natoms <= 0 || nT <= 0 || nsel < 0 || proc_mask < 0 || proc_mask > 7) return -1;
  if (nu_select < 0 || nu_select > 2) return -1;
  orc_problem P;
  orc_setup(&P, grid, lattice, natoms, mass, nquart, qidx, qfc, omega, evec, vel);
  const int nb = P.nb, nq = P.nq;
  const double dq = orc_dq_iso(&P);
  const double conv = orc_conv();
  /* hbar^2 pi / (8 N) from Gamma, 1/N from Eq. tao0; the units bring (conv)^4 (see header) */
  const double pref = M_PI * ORC_HBAR * ORC_HBAR * conv * conv * conv * conv / (8.0 * (double)nq * (double)nq);
  for (int k = 0; k < 3; ++k) accepted[k] = 0.0;
  memset(rates, 0, sizeof(double) * (size_t)nT * nsel);
  int* shift = (int*)malloc(sizeof(int) * 3 * (size_t)nq);
  for (int k = 0; k < nq; ++k) orc_bz_shift(&P, k, shift + 3 * k);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (int s = 0; s < nsel; ++s) {
    const int q = sel[s] / nb, j = sel[s] % nb;
    const double w = omega[sel[s]];
    if (w == 0.0) continue;
    double* part = (double*)calloc((size_t)nq * nT, sizeof(double));
    double* cnt = (double*)calloc((size_t)nq * 3, sizeof(double));
#pragma omp parallel
    {
      cplx* phi = (cplx*)malloc(sizeof(cplx) * (size_t)nb * nb * nb * nb);
      double* nbose = (double*)malloc(sizeof(double) * 4 * nT);
#pragma omp for schedule(dynamic, 1)
      for (int q1 = 0; q1 < nq; ++q1) {
        for (int q2 = 0; q2 < nq; ++q2) {
          for (int pr = 0; pr < 3; ++pr) {
            if (!((proc_mask >> pr) & 1)) continue;
            const int s1 = ORC_S1[pr], s2 = ORC_S2[pr];
            const int q3 = orc_third(&P, q, q1, q2, s1, s2);
            if (nu_select != 0) {
              const int u = orc_is_umklapp(&P, shift, q, q1, q2, s1, s2);
              if ((nu_select == 1) == (u != 0)) continue;
            }
            int have_phi = 0;
            for (int j1 = 0; j1 < nb; ++j1) {
              const double w1 = omega[q1 * nb + j1];
              if (w1 == 0.0) continue;
              for (int j2 = 0; j2 < nb; ++j2) {
                const double w2 = omega[q2 * nb + j2];
                if (w2 == 0.0) continue;
                for (int j3 = 0; j3 < nb; ++j3) {
                  const double w3 = omega[q3 * nb + j3];
                  if (w3 == 0.0) continue;
                  double t = (s1 > 0) ? (w + w1) : (w - w1);
                  t = (s2 > 0) ? (t + w2) : (t - w2);
                  const double dw = t - w3;
                  const double sigma = orc_sigma(&P, vel + 3 * (q2 * nb + j2), vel + 3 * (q3 * nb + j3),
                                                 scalebroad, dq, dq_mode);
                  /* the window uses the broadening actually applied: sigma, or sigma_min where delta := 1 */
                  const double sw = (sigma < sigma_min) ? sigma_min : sigma;
                  if (!(fabs(dw) <= window * sw)) continue;
                  const double delta =
                      (sigma < sigma_min) ? 1.0 : exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma);
                  double v2 = 1.0;
                  if (!unit_vertex) {
                    if (!have_phi) {
                      orc_phi(&P, q1, q2, q3, s1, s2, phi);
                      have_phi = 1;
                    }
                    cplx V = orc_vertex(&P, phi, q, j, q1, j1, q2, j2, q3, j3, s1, s2);
                    v2 = creal(V) * creal(V) + cimag(V) * cimag(V);
                  }
                  cnt[3 * q1 + pr] += 1.0;
                  for (int it = 0; it < nT; ++it) {
                    const double n0 = orc_bose(w, T[it]);
                    const double n1 = orc_bose(w1, T[it]);
                    const double n2 = orc_bose(w2, T[it]);
                    const double n3 = orc_bose(w3, T[it]);
                    double B;
                    if (pr == 0)
                      B = (1.0 + n1) * (1.0 + n2) * n3;
                    else if (pr == 1)
                      B = (1.0 + n1) * n2 * n3;
                    else
                      B = n1 * n2 * n3;
                    if (unit_vertex == 2)
                      part[(size_t)q1 * nT + it] += ORC_MULT[pr] * delta;
                    else
                      part[(size_t)q1 * nT + it] += ORC_MULT[pr] * B / n0 * v2 * delta / (w * w1 * w2 * w3);
                  }
                }
              }
            }
          }
        }
      }
      free(phi);
      free(nbose);
    }
    /* fixed-order reduction over q' */
    for (int q1 = 0; q1 < nq; ++q1) {
      for (int it = 0; it < nT; ++it) rates[(size_t)it * nsel + s] += part[(size_t)q1 * nT + it];
      for (int k = 0; k < 3; ++k) accepted[k] += cnt[3 * q1 + k];
    }
    for (int it = 0; it < nT; ++it) rates[(size_t)it * nsel + s] *= unit_vertex ? 1.0 : pref;
    free(part);
    free(cnt);
  }
  free(shift);
  return 0;
}

/*
 * Normal (0) or Umklapp (1) classification of process pr (0 ++, 1 +-, 2 --) with explicit partners q1, q2
 * (orc_is_umklapp); -1 on bad arguments.  Exposed so that tests can check hand-worked cases.
 */
int oracle_umklapp(const int grid[3], const double lattice[9], int q, int q1, int q2, int pr) {
  if (!grid || !lattice || pr < 0 || pr > 2) return -1;
  orc_problem P;
  orc_setup(&P, grid, lattice, 1, NULL, 0, NULL, NULL, NULL, NULL, NULL);
  if (q < 0 || q1 < 0 || q2 < 0 || q >= P.nq || q1 >= P.nq || q2 >= P.nq) return -1;
  int* shift = (int*)malloc(sizeof(int) * 3 * (size_t)P.nq);
  for (int k = 0; k < P.nq; ++k) orc_bz_shift(&P, k, shift + 3 * k);
  const int u = orc_is_umklapp(&P, shift, q, q1, q2, ORC_S1[pr], ORC_S2[pr]);
  free(shift);
  return u;
}

/*
 * The full branch tensor of one vertex, out[((j*nb + j1)*nb + j2)*nb + j3] = V_p (re, im), for the
 * wavevectors (q, q', q'') of process pr (0: ++, 1: +-, 2: --).  *q3_out receives q'''.
 */
int oracle_v4(const int grid[3], const double lattice[9], int natoms, const double* mass, int nquart,
              const int* qidx, const double* qfc, const double* evec, int q, int q1, int q2, int pr,
              double* out, int* q3_out) {
  if (pr < 0 || pr > 2) return -1;
  orc_problem P;
  orc_setup(&P, grid, lattice, natoms, mass, nquart, qidx, qfc, NULL, evec, NULL);
  const int nb = P.nb;
  const int s1 = ORC_S1[pr], s2 = ORC_S2[pr];
  const int q3 = orc_third(&P, q, q1, q2, s1, s2);
  cplx* phi = (cplx*)malloc(sizeof(cplx) * (size_t)nb * nb * nb * nb);
  orc_phi(&P, q1, q2, q3, s1, s2, phi);
  for (int j = 0; j < nb; ++j)
    for (int j1 = 0; j1 < nb; ++j1)
      for (int j2 = 0; j2 < nb; ++j2)
        for (int j3 = 0; j3 < nb; ++j3) {
          cplx V = orc_vertex(&P, phi, q, j, q1, j1, q2, j2, q3, j3, s1, s2);
          size_t o = (((size_t)j * nb + j1) * nb + j2) * nb + j3;
          out[2 * o] = creal(V);
          out[2 * o + 1] = cimag(V);
        }
  free(phi);
  if (q3_out) *q3_out = q3;
  return 0;
}

/* Bose-Einstein occupation n0 = 1/(exp(hbar w / kB T) - 1), exported for the detailed-balance pins. */
double oracle_bose(double w, double T) { return orc_bose(w, T); }

/* Rate prefactor pi hbar^2 conv^4 / (8 N^2), exported for the closed-form pins. */
double oracle_prefactor(int nq) {
  const double c = orc_conv();
  return M_PI * ORC_HBAR * ORC_HBAR * c * c * c * c / (8.0 * (double)nq * (double)nq);
}

/*
 * Three-phonon-like phase space of selected modes (features of the surrogate; the paper's P3 / WP3
 * outputs, Sec. 2.1, with the weighting of Eq. 3phgamma without |V3|^2 and without hbar pi / 4):
 *   (+): q'' = q + q', dw = (w + w') - w'';  (-): q'' = q - q', dw = (w - w') - w''
 *   sigma = sb |v(q',j') - v(q'',j'')| |dq|, the same window and Gaussian as the four-phonon rates.
 *   p3[s]        = (1/N) sum [ delta+ + 1/2 delta- ]
 *   wp3[t*nsel+s] = (1/N) sum [ (n' - n'') delta+ + 1/2 (n' + n'' + 1) delta- ] / (w w' w'')
 */
int oracle_phase3(const int grid[3], const double lattice[9], int natoms, const double* omega, const double* vel,
                  int nT, const double* T, double scalebroad, double window, double sigma_min, int dq_mode,
                  int nsel, const int* sel, double* p3, double* wp3) {
  if (!grid || !lattice || natoms <= 0 || nT <= 0 || nsel < 0) return -1;
  orc_problem P;
  orc_setup(&P, grid, lattice, natoms, NULL, 0, NULL, NULL, omega, NULL, vel);
  const int nb = P.nb, nq = P.nq;
  const double dq = orc_dq_iso(&P);
  memset(p3, 0, sizeof(double) * (size_t)nsel);
  memset(wp3, 0, sizeof(double) * (size_t)nsel * nT);
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < nsel; ++s) {
    const int q = sel[s] / nb;
    const double w = omega[sel[s]];
    if (w == 0.0) continue;
    double acc_p = 0.0;
    double acc_w[64];
    for (int it = 0; it < nT && it < 64; ++it) acc_w[it] = 0.0;
    for (int q1 = 0; q1 < nq; ++q1) {
      for (int pm = 0; pm < 2; ++pm) {
        const int sgn = pm == 0 ? +1 : -1;
        int g[3], g1[3], g2[3];
        orc_unidx(&P, q, g);
        orc_unidx(&P, q1, g1);
        for (int a = 0; a < 3; ++a) g2[a] = orc_wrap(g[a] + sgn * g1[a], P.grid[a]);
        const int q2 = orc_idx(&P, g2);
        for (int j1 = 0; j1 < nb; ++j1) {
          const double w1 = omega[q1 * nb + j1];
          if (w1 == 0.0) continue;
          for (int j2 = 0; j2 < nb; ++j2) {
            const double w2 = omega[q2 * nb + j2];
            if (w2 == 0.0) continue;
            const double t = (sgn > 0) ? (w + w1) : (w - w1);
            const double dw = t - w2;
            const double sigma = orc_sigma(&P, vel + 3 * (q1 * nb + j1), vel + 3 * (q2 * nb + j2), scalebroad, dq,
                                           dq_mode);
            const double sw = (sigma < sigma_min) ? sigma_min : sigma;
            if (!(fabs(dw) <= window * sw)) continue;
            const double delta =
                (sigma < sigma_min) ? 1.0 : exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma);
            acc_p += (sgn > 0 ? 1.0 : 0.5) * delta;
            for (int it = 0; it < nT && it < 64; ++it) {
              const double n1 = orc_bose(w1, T[it]), n2 = orc_bose(w2, T[it]);
              const double B = (sgn > 0) ? (n1 - n2) : 0.5 * (n1 + n2 + 1.0);
              acc_w[it] += B * delta / (w * w1 * w2);
            }
          }
        }
      }
    }
    p3[s] = acc_p / (double)nq;
    for (int it = 0; it < nT && it < 64; ++it) wp3[(size_t)it * nsel + s] = acc_w[it] / (double)nq;
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------------------
 * Three-phonon rates (Eqs. tao0, 3phgamma, V3), the same conventions as the four-phonon part:
 *   1/tau3_l = (1/N) [ sum_{l' l''}^{(+)} G+ + 1/2 sum_{l' l''}^{(-)} G- ],
 *   G+- = (hbar pi / 4) B+- / (w w' w'') |V+-|^2 delta(w +- w' - w''),  B+ = n' - n'',  B- = n' + n'' + 1,
 *   q'' = q +- q' on the grid,
 *   V+- = sum_{ijk} sum_{abg} Phi3 e_a(l)(i) e_b(+-l')(j) e_g(-l'')(k) / sqrt(Mi Mj Mk) exp(+-i q'.r_j) exp(-i q''.r_k),
 * with e(-l) = conj e(l).  sigma = sb |v' - v''| dq at the actual q', q'' (the adaptive broadening of
 * Sec. 2.4 applied to the two partner modes); the window and delta follow the four-phonon rules.
 * |V|^2 in eV^2/(A^6 amu^3) = conv^3 ps^-6 / eV, so the prefactor is (pi/4) hbar conv^3 / N.
 * ------------------------------------------------------------------------------------------------------ */
static void orc_phi3(const orc_problem* p, int n3, const int* idx3, const double* fc3, int q1, int q2, int s1,
                     cplx* phi) {
  const int nb = p->nb;
  double k1[3], k2[3];
  orc_qcart(p, q1, k1);
  orc_qcart(p, q2, k2);
  memset(phi, 0, sizeof(cplx) * (size_t)nb * nb * nb);
  for (int Q = 0; Q < n3; ++Q) {
    const int* ix = idx3 + 9 * Q;
    double rj[3], rk[3];
    orc_rcart(p, ix + 3, rj);
    orc_rcart(p, ix + 6, rk);
    double ang = 0.0;
    for (int c = 0; c < 3; ++c) ang += s1 * k1[c] * rj[c] - k2[c] * rk[c];
    cplx ph = cos(ang) + I * sin(ang);
    double msq = sqrt(p->mass[ix[0]] * p->mass[ix[1]] * p->mass[ix[2]]);
    const double* fc = fc3 + 27 * Q;
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be)
        for (int ga = 0; ga < 3; ++ga) {
          int a = 3 * ix[0] + al, b = 3 * ix[1] + be, c = 3 * ix[2] + ga;
          phi[(a * nb + b) * nb + c] += fc[(al * 3 + be) * 3 + ga] / msq * ph;
        }
  }
}

static cplx orc_vertex3(const orc_problem* p, const cplx* phi, int q, int j, int q1, int j1, int q2, int j2,
                        int s1) {
  const int nb = p->nb;
  cplx acc = 0.0;
  for (int a = 0; a < nb; ++a) {
    cplx ea = orc_e(p, q, j, a);
    for (int b = 0; b < nb; ++b) {
      cplx eb = orc_e(p, q1, j1, b);
      if (s1 < 0) eb = conj(eb);
      for (int c = 0; c < nb; ++c) acc += phi[(a * nb + b) * nb + c] * ea * eb * conj(orc_e(p, q2, j2, c));
    }
  }
  return acc;
}

/* V+- tensor out[((j nb + j1) nb + j2)] (re, im) of process 0 (+) or 1 (-) with partner q1; *q2_out = q'' */
int oracle_v3(const int grid[3], const double lattice[9], int natoms, const double* mass, int n3, const int* idx3,
              const double* fc3, const double* evec, int q, int q1, int process, double* out, int* q2_out) {
  if (!grid || !lattice || natoms <= 0 || process < 0 || process > 1) return -1;
  orc_problem P;
  orc_setup(&P, grid, lattice, natoms, mass, 0, NULL, NULL, NULL, evec, NULL);
  const int nb = P.nb, s1 = process == 0 ? 1 : -1;
  if (q < 0 || q1 < 0 || q >= P.nq || q1 >= P.nq) return -1;
  int g[3], g1[3], g2[3];
  orc_unidx(&P, q, g);
  orc_unidx(&P, q1, g1);
  for (int a = 0; a < 3; ++a) g2[a] = orc_wrap(g[a] + s1 * g1[a], grid[a]);
  const int q2 = orc_idx(&P, g2);
  cplx* phi = (cplx*)malloc(sizeof(cplx) * (size_t)nb * nb * nb);
  orc_phi3(&P, n3, idx3, fc3, q1, q2, s1, phi);
  for (int j = 0; j < nb; ++j)
    for (int j1 = 0; j1 < nb; ++j1)
      for (int j2 = 0; j2 < nb; ++j2) {
        cplx V = orc_vertex3(&P, phi, q, j, q1, j1, q2, j2, s1);
        out[2 * ((j * nb + j1) * nb + j2)] = creal(V);
        out[2 * ((j * nb + j1) * nb + j2) + 1] = cimag(V);
      }
  free(phi);
  *q2_out = q2;
  return 0;
}

/*
 * Three-phonon RTA rates of selected modes: rates[t * nsel + s] in ps^-1; accepted[2]: terms inside the
 * window, + and - processes.  unit_vertex != 0 replaces |V|^2 by 1 (then the sum, without the prefactor, is
 * the weighted phase space WP3 of oracle_phase3).
 */
int oracle_rates3(const int grid[3], const double lattice[9], int natoms, const double* mass, int n3,
                  const int* idx3, const double* fc3, const double* omega, const double* evec, const double* vel,
                  int nT, const double* T, double scalebroad, double window, double sigma_min, int dq_mode, int nsel,
                  const int* sel, int unit_vertex, int nthreads, double* rates, double* accepted) {
  if (!grid || !lattice || natoms <= 0 || nT <= 0 || nsel < 0) return -1;
  orc_problem P;
  orc_setup(&P, grid, lattice, natoms, mass, 0, NULL, NULL, omega, evec, vel);
  const int nb = P.nb, nq = P.nq;
  const double dq = orc_dq_iso(&P);
  const double conv = orc_conv();
  const double pref = M_PI * ORC_HBAR * conv * conv * conv / (4.0 * (double)nq);
  accepted[0] = accepted[1] = 0.0;
  memset(rates, 0, sizeof(double) * (size_t)nT * nsel);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (int s = 0; s < nsel; ++s) {
    const int q = sel[s] / nb, j = sel[s] % nb;
    const double w = omega[sel[s]];
    if (w == 0.0) continue;
    double* part = (double*)calloc((size_t)nq * nT, sizeof(double));
    double* cnt = (double*)calloc((size_t)nq * 2, sizeof(double));
#pragma omp parallel
    {
      cplx* phi = (cplx*)malloc(sizeof(cplx) * (size_t)nb * nb * nb);
#pragma omp for schedule(dynamic, 1)
      for (int q1 = 0; q1 < nq; ++q1) {
        for (int pr = 0; pr < 2; ++pr) {
          const int s1 = pr == 0 ? 1 : -1;
          int g[3], g1[3], g2[3];
          orc_unidx(&P, q, g);
          orc_unidx(&P, q1, g1);
          for (int a = 0; a < 3; ++a) g2[a] = orc_wrap(g[a] + s1 * g1[a], grid[a]);
          const int q2 = orc_idx(&P, g2);
          int have_phi = 0;
          for (int j1 = 0; j1 < nb; ++j1) {
            const double w1 = omega[q1 * nb + j1];
            if (w1 == 0.0) continue;
            for (int j2 = 0; j2 < nb; ++j2) {
              const double w2 = omega[q2 * nb + j2];
              if (w2 == 0.0) continue;
              const double dw = ((s1 > 0) ? (w + w1) : (w - w1)) - w2;
              const double sigma =
                  orc_sigma(&P, vel + 3 * (q1 * nb + j1), vel + 3 * (q2 * nb + j2), scalebroad, dq, dq_mode);
              const double sw = (sigma < sigma_min) ? sigma_min : sigma;
              if (!(fabs(dw) <= window * sw)) continue;
              const double delta =
                  (sigma < sigma_min) ? 1.0 : exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma);
              double v2 = 1.0;
              if (!unit_vertex) {
                if (!have_phi) {
                  orc_phi3(&P, n3, idx3, fc3, q1, q2, s1, phi);
                  have_phi = 1;
                }
                cplx V = orc_vertex3(&P, phi, q, j, q1, j1, q2, j2, s1);
                v2 = creal(V) * creal(V) + cimag(V) * cimag(V);
              }
              cnt[2 * q1 + pr] += 1.0;
              for (int it = 0; it < nT; ++it) {
                const double n1 = orc_bose(w1, T[it]);
                const double n2 = orc_bose(w2, T[it]);
                const double B = (pr == 0) ? (n1 - n2) : (n1 + n2 + 1.0);
                const double mult = (pr == 0) ? 1.0 : 0.5;
                part[(size_t)q1 * nT + it] += mult * B * v2 * delta / (w * w1 * w2);
              }
            }
          }
        }
      }
      free(phi);
    }
    for (int q1 = 0; q1 < nq; ++q1) {
      for (int it = 0; it < nT; ++it) rates[(size_t)it * nsel + s] += part[(size_t)q1 * nT + it];
      accepted[0] += cnt[2 * q1];
      accepted[1] += cnt[2 * q1 + 1];
    }
    for (int it = 0; it < nT; ++it) rates[(size_t)it * nsel + s] *= unit_vertex ? 1.0 / (double)nq : pref;
    free(part);
    free(cnt);
  }
  return 0;
}
