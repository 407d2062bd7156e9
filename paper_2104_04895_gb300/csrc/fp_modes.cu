// Support kernels of the rate path: twiddle table, mass scaling of Phi4, harmonic modes
// (dynamical matrix + complex Jacobi eigensolver + Hellmann-Feynman velocities) and the
// per-temperature Bose weight tables.
#include "fp_internal.cuh"

namespace fp {
namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int wrap(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

// tw[m] = exp(2 pi i m / L): phases exp(i q.R) of grid wavevectors and lattice vectors are
// exactly tw[sum_a (L/N_a) (g_a R_a mod N_a) mod L].
__global__ void twiddle_kernel(double2* tw, int L) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)L, &s, &c);
  tw[m] = make_double2(c, s);
}

// Phi4 / sqrt(Mi Mj Mk Ml) (the mass denominator of Eq. V4), in place.
__global__ void scale_fc4_kernel(double* qfc, const int* atoms4, const double* mass, int nquart) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nquart * 81) return;
  int Q = t / 81;
  const int* a = atoms4 + 4 * Q;
  double m = mass[a[0]] * mass[a[1]] * mass[a[2]] * mass[a[3]];
  qfc[t] = qfc[t] / sqrt(m);
}

struct ModesArgs {
  int N, nb, natoms, L, n_fc2;
  int grid[3], Lfac[3];
  double lattice[9];
  const int* fc2_idx;
  const double* fc2_val;
  const double* mass;
  const double2* tw;
  double* omega;
  double2* evec;
  double* vel;
  int* flag;
};

__device__ int phase_index(const ModesArgs& a, const int g[3], const int R[3]) {
  long long m = 0;
  for (int d = 0; d < 3; ++d) m += (long long)a.Lfac[d] * wrap(g[d] * R[d], a.grid[d]);
  return (int)(m % a.L);
}

// One thread per time-reversal pair {q, -q}: D(q) = sum_R Phi2(0i; Rj) e^{iq.R} / sqrt(Mi Mj)
// (cell-phase convention of Eq. V4), eigenpairs by cyclic complex Jacobi rotations,
// v = conv Re(e^H dD/dq e) / (2 omega) averaged over degenerate sets.
__global__ void modes_kernel(ModesArgs a) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= a.N) return;
  const int nb = a.nb;
  int g[3] = {q / (a.grid[1] * a.grid[2]), (q / a.grid[2]) % a.grid[1], q % a.grid[2]};
  int gm[3] = {wrap(-g[0], a.grid[0]), wrap(-g[1], a.grid[1]), wrap(-g[2], a.grid[2])};
  int partner = (gm[0] * a.grid[1] + gm[1]) * a.grid[2] + gm[2];
  if (partner < q) return;
  const bool selfconj = partner == q;

  double2 A[kMaxNb * kMaxNb];
  double2 V[kMaxNb * kMaxNb];
  for (int i = 0; i < nb * nb; ++i) {
    A[i] = make_double2(0.0, 0.0);
    V[i] = make_double2(0.0, 0.0);
  }
  for (int i = 0; i < nb; ++i) V[i * nb + i].x = 1.0;
  for (int b = 0; b < a.n_fc2; ++b) {
    const int* ix = a.fc2_idx + 5 * b;
    double2 ph = a.tw[phase_index(a, g, ix + 2)];
    double s = 1.0 / sqrt(a.mass[ix[0]] * a.mass[ix[1]]);
    for (int al = 0; al < 3; ++al)
      for (int be = 0; be < 3; ++be) {
        double f = a.fc2_val[9 * b + 3 * al + be] * s;
        double2& x = A[(3 * ix[0] + al) * nb + 3 * ix[1] + be];
        x.x += f * ph.x;
        x.y += f * ph.y;
      }
  }
  // exact Hermiticity (and exact realness at self-conjugate q, where D(q) = D(-q) = conj D(q))
  for (int i = 0; i < nb; ++i)
    for (int j = i; j < nb; ++j) {
      double2 u = A[i * nb + j], w = A[j * nb + i];
      double re = 0.5 * (u.x + w.x), im = 0.5 * (u.y - w.y);
      if (selfconj || i == j) im = 0.0;
      A[i * nb + j] = make_double2(re, im);
      A[j * nb + i] = make_double2(re, -im);
    }
  // cyclic Jacobi: per pair (p, r) a phase on column r makes A_pr real, then a real rotation
  double fro = 0.0;
  for (int i = 0; i < nb * nb; ++i) fro += A[i].x * A[i].x + A[i].y * A[i].y;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < nb; ++p)
      for (int r = p + 1; r < nb; ++r) off += A[p * nb + r].x * A[p * nb + r].x + A[p * nb + r].y * A[p * nb + r].y;
    if (off <= 1e-32 * fro) break;
    for (int p = 0; p < nb; ++p)
      for (int r = p + 1; r < nb; ++r) {
        double2 apr = A[p * nb + r];
        double mag = sqrt(apr.x * apr.x + apr.y * apr.y);
        if (mag <= 1e-300) continue;
        // phase u = conj(a_pr)/|a_pr| applied to column r (and conj to row r)
        double2 u = make_double2(apr.x / mag, -apr.y / mag);
        for (int k = 0; k < nb; ++k) {
          A[k * nb + r] = cmul(A[k * nb + r], u);
          V[k * nb + r] = cmul(V[k * nb + r], u);
        }
        for (int k = 0; k < nb; ++k) A[r * nb + k] = cmul(make_double2(u.x, -u.y), A[r * nb + k]);
        // now A_pr = mag (real); symmetric Schur rotation on (p, r)
        double app = A[p * nb + p].x, arr = A[r * nb + r].x;
        double tau = (arr - app) / (2.0 * mag);
        double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < nb; ++k) {
          double2 x = A[k * nb + p], y = A[k * nb + r];
          A[k * nb + p] = make_double2(cs * x.x - sn * y.x, cs * x.y - sn * y.y);
          A[k * nb + r] = make_double2(sn * x.x + cs * y.x, sn * x.y + cs * y.y);
          double2 vx = V[k * nb + p], vy = V[k * nb + r];
          V[k * nb + p] = make_double2(cs * vx.x - sn * vy.x, cs * vx.y - sn * vy.y);
          V[k * nb + r] = make_double2(sn * vx.x + cs * vy.x, sn * vx.y + cs * vy.y);
        }
        for (int k = 0; k < nb; ++k) {
          double2 x = A[p * nb + k], y = A[r * nb + k];
          A[p * nb + k] = make_double2(cs * x.x - sn * y.x, cs * x.y - sn * y.y);
          A[r * nb + k] = make_double2(sn * x.x + cs * y.x, sn * x.y + cs * y.y);
        }
        A[p * nb + r] = make_double2(0.0, 0.0);
        A[r * nb + p] = make_double2(0.0, 0.0);
      }
  }
  // sort eigenpairs ascending
  double lam[kMaxNb];
  int ord[kMaxNb];
  for (int i = 0; i < nb; ++i) {
    lam[i] = A[i * nb + i].x;
    ord[i] = i;
  }
  for (int i = 1; i < nb; ++i)
    for (int j = i; j > 0 && lam[ord[j]] < lam[ord[j - 1]]; --j) {
      int tmp = ord[j];
      ord[j] = ord[j - 1];
      ord[j - 1] = tmp;
    }
  double lmax = 0.0;
  for (int i = 0; i < nb; ++i) lmax = fmax(lmax, fabs(lam[i]));
  double w[kMaxNb];
  for (int b = 0; b < nb; ++b) {
    double l = lam[ord[b]];
    if (q == 0 && b < 3) {
      w[b] = 0.0;
    } else if (l < -1e-8 * lmax) {
      atomicExch(a.flag, 1);
      w[b] = 0.0;
    } else {
      w[b] = sqrt(fmax(l, 0.0) * kConv);
    }
  }
  // eigenvectors as rows e[b][comp], normalised
  double2 E[kMaxNb * kMaxNb];
  for (int b = 0; b < nb; ++b) {
    double nrm = 0.0;
    for (int k = 0; k < nb; ++k) {
      double2 x = V[k * nb + ord[b]];
      nrm += x.x * x.x + x.y * x.y;
    }
    nrm = 1.0 / sqrt(nrm);
    for (int k = 0; k < nb; ++k) {
      double2 x = V[k * nb + ord[b]];
      E[b * nb + k] = make_double2(x.x * nrm, selfconj ? 0.0 : x.y * nrm);
    }
  }
  // Hellmann-Feynman: raw[b][c] = Re(e_b^H dD/dq_c e_b), dD/dq_c = sum_R i R_c Phi2 e^{iq.R}/sqrt(M M)
  double raw[kMaxNb * 3];
  for (int i = 0; i < nb * 3; ++i) raw[i] = 0.0;
  for (int bk = 0; bk < a.n_fc2; ++bk) {
    const int* ix = a.fc2_idx + 5 * bk;
    double2 ph = a.tw[phase_index(a, g, ix + 2)];
    double s = 1.0 / sqrt(a.mass[ix[0]] * a.mass[ix[1]]);
    double Rc[3];
    for (int c = 0; c < 3; ++c)
      Rc[c] = ix[2] * a.lattice[c] + ix[3] * a.lattice[3 + c] + ix[4] * a.lattice[6 + c];
    for (int b = 0; b < nb; ++b) {
      double2 acc = make_double2(0.0, 0.0);
      for (int al = 0; al < 3; ++al) {
        double2 ei = E[b * nb + 3 * ix[0] + al];
        for (int be = 0; be < 3; ++be) {
          double2 ej = E[b * nb + 3 * ix[1] + be];
          double f = a.fc2_val[9 * bk + 3 * al + be];
          // conj(ei) * ej
          acc.x += f * (ei.x * ej.x + ei.y * ej.y);
          acc.y += f * (ei.x * ej.y - ei.y * ej.x);
        }
      }
      acc = cmul(acc, ph);
      // Re(i R_c s acc) = -R_c s Im(acc)
      for (int c = 0; c < 3; ++c) raw[b * 3 + c] += -Rc[c] * s * acc.y;
    }
  }
  double v[kMaxNb * 3];
  double wmax = 0.0;
  for (int b = 0; b < nb; ++b) wmax = fmax(wmax, w[b]);
  for (int b = 0; b < nb;) {
    int e = b + 1;
    while (e < nb && fabs(w[e] - w[e - 1]) <= 1e-8 * wmax) ++e;
    for (int c = 0; c < 3; ++c) {
      double avg = 0.0;
      for (int k = b; k < e; ++k) avg += raw[k * 3 + c];
      avg /= (double)(e - b);
      for (int k = b; k < e; ++k) v[k * 3 + c] = (w[k] == 0.0 || selfconj) ? 0.0 : kConv * avg / (2.0 * w[k]);
    }
    b = e;
  }
  for (int b = 0; b < nb; ++b) {
    a.omega[q * nb + b] = w[b];
    a.omega[partner * nb + b] = w[b];
    for (int k = 0; k < nb; ++k) {
      double2 x = E[b * nb + k];
      a.evec[((size_t)q * nb + b) * nb + k] = x;
      a.evec[((size_t)partner * nb + b) * nb + k] = make_double2(x.x, -x.y);
    }
    for (int c = 0; c < 3; ++c) {
      a.vel[((size_t)q * nb + b) * 3 + c] = v[b * 3 + c];
      a.vel[((size_t)partner * nb + b) * 3 + c] = -v[b * 3 + c];
    }
  }
}

// Bose weights per temperature and mode: wt = (1/(n w), (1+n)/w, n/w), n = 1/expm1(hbar w / kB T)
// (the Bose-Einstein occupation of Eq. 4phgamma); zero for zero-frequency modes.
__global__ void weights_kernel(const double* omega, int nmodes, int nT, const double* T, double* wt) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nmodes * nT) return;
  int it = t / nmodes, m = t % nmodes;
  double w = omega[m];
  double* o = wt + 3 * (size_t)t;
  if (w <= 0.0) {
    o[0] = o[1] = o[2] = 0.0;
    return;
  }
  double n = 1.0 / expm1(kHbar * w / (kBoltzmann * T[it]));
  o[0] = 1.0 / (n * w);
  o[1] = (1.0 + n) / w;
  o[2] = n / w;
}

}  // namespace

cudaError_t launch_twiddles(fp_ctx* c, cudaStream_t s) {
  twiddle_kernel<<<(c->L + 127) / 128, 128, 0, s>>>(c->d_tw, c->L);
  return cudaGetLastError();
}

cudaError_t launch_scale_fc4(double* qfc, const int* d_atoms4, const double* d_mass, int nquart, cudaStream_t s) {
  int n = nquart * 81;
  if (n == 0) return cudaSuccess;
  scale_fc4_kernel<<<(n + 255) / 256, 256, 0, s>>>(qfc, d_atoms4, d_mass, nquart);
  return cudaGetLastError();
}

cudaError_t launch_modes(fp_ctx* c, cudaStream_t s) {
  ModesArgs a;
  a.N = c->N;
  a.nb = c->nb;
  a.natoms = c->natoms;
  a.L = c->L;
  a.n_fc2 = c->n_fc2;
  for (int d = 0; d < 3; ++d) {
    a.grid[d] = c->grid[d];
    a.Lfac[d] = c->L / c->grid[d];
  }
  for (int i = 0; i < 9; ++i) a.lattice[i] = c->lattice[i];
  a.fc2_idx = c->d_fc2_idx;
  a.fc2_val = c->d_fc2_val;
  a.mass = c->d_mass;
  a.tw = c->d_tw;
  a.omega = c->d_omega;
  a.evec = c->d_evec;
  a.vel = c->d_vel;
  a.flag = c->d_flag;
  modes_kernel<<<(c->N + 63) / 64, 64, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_weights(fp_ctx* c, int nT, const double* d_T, double* d_wt, cudaStream_t s) {
  int n = c->N * c->nb * nT;
  weights_kernel<<<(n + 255) / 256, 256, 0, s>>>(c->d_omega, c->N * c->nb, nT, d_T, d_wt);
  return cudaGetLastError();
}

}  // namespace fp
