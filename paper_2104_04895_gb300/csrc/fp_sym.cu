// Host-only grid geometry: the stars of the q-grid under a point group and time reversal (fp_star_table, used by
// fp_rates4_irreducible) and the Brillouin-zone representatives behind the normal/Umklapp split (bz_shifts).
#include <cstdlib>
#include <vector>

#include "fp_internal.cuh"

namespace {

// q -> sign * R q on the grid, R acting on reciprocal-lattice fractional coordinates f_a = g_a / N_a. An op
// only mixes axes of equal N (checked by fp_star_table), so g'_a = sign * sum_b R_ab g_b mod N_a.
void apply(const int* R, const int grid[3], const int g[3], int sign, int out[3]) {
  for (int a = 0; a < 3; ++a) {
    long long s = 0;
    for (int b = 0; b < 3; ++b) s += (long long)R[3 * a + b] * g[b];
    s *= sign;
    long long m = s % grid[a];
    out[a] = (int)(m < 0 ? m + grid[a] : m);
  }
}

}  // namespace

extern "C" int fp_star_table(const int grid[3], int nrot, const int* rot, int* rep, int* n_irr) {
  if (!grid || nrot < 0 || (nrot > 0 && !rot) || !rep || !n_irr) return FP_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (grid[a] < 1) return FP_EINVAL;
  for (int r = 0; r < nrot; ++r) {
    const int* R = rot + 9 * r;
    const long long det = (long long)R[0] * (R[4] * R[8] - R[5] * R[7]) - (long long)R[1] * (R[3] * R[8] - R[5] * R[6]) +
                          (long long)R[2] * (R[3] * R[7] - R[4] * R[6]);
    if (det != 1 && det != -1) return FP_EINVAL;
    // an op that mixes two axes maps the grid to itself only if they have the same number of points
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        if (R[3 * a + b] != 0 && grid[a] != grid[b]) return FP_EINVAL;
  }
  const int N = grid[0] * grid[1] * grid[2];
  for (int q = 0; q < N; ++q) rep[q] = -1;
  std::vector<int> orbit;
  int count = 0;
  for (int q = 0; q < N; ++q) {
    if (rep[q] >= 0) continue;
    // closure of the orbit of q under the ops and q -> -q; q is its smallest member
    orbit.assign(1, q);
    rep[q] = q;
    for (size_t i = 0; i < orbit.size(); ++i) {
      const int p = orbit[i];
      const int g[3] = {p / (grid[1] * grid[2]), (p / grid[2]) % grid[1], p % grid[2]};
      for (int r = -1; r < nrot; ++r) {
        for (int sign = 1; sign >= -1; sign -= 2) {
          int h[3];
          if (r < 0) {
            for (int a = 0; a < 3; ++a) h[a] = ((sign * g[a]) % grid[a] + grid[a]) % grid[a];
          } else {
            apply(rot + 9 * r, grid, g, sign, h);
          }
          const int k = (h[0] * grid[1] + h[1]) * grid[2] + h[2];
          if (rep[k] < 0) {
            rep[k] = q;
            orbit.push_back(k);
          }
        }
      }
    }
    ++count;
  }
  *n_irr = count;
  return FP_OK;
}

namespace fp {

// Brillouin-zone representative of every grid point, for the normal/Umklapp split: the translate
// sum_a (g_a / N_a - m_a) b_a of smallest length over integer m_a in [-2, 2] (b_a: rows of rec); squared lengths
// within 1e-9 relative are equal, and then the lexicographically smallest (m_0, m_1, m_2) is taken.
// out: N x 3 shifts m.
void bz_shifts(const int grid[3], const double rec[9], int* out) {
  const int N = grid[0] * grid[1] * grid[2];
  for (int q = 0; q < N; ++q) {
    const int g[3] = {q / (grid[1] * grid[2]), (q / grid[2]) % grid[1], q % grid[2]};
    double best = -1.0;
    int bm[3] = {0, 0, 0};
    for (int m0 = -2; m0 <= 2; ++m0)
      for (int m1 = -2; m1 <= 2; ++m1)
        for (int m2 = -2; m2 <= 2; ++m2) {
          const double f[3] = {(double)g[0] / grid[0] - m0, (double)g[1] / grid[1] - m1, (double)g[2] / grid[2] - m2};
          double len2 = 0.0;
          for (int c = 0; c < 3; ++c) {
            const double k = f[0] * rec[c] + f[1] * rec[3 + c] + f[2] * rec[6 + c];
            len2 += k * k;
          }
          if (best < 0.0 || len2 < best * (1.0 - 1e-9)) {  // visited in lexicographic order of m
            best = len2;
            bm[0] = m0;
            bm[1] = m1;
            bm[2] = m2;
          }
        }
    for (int a = 0; a < 3; ++a) out[3 * q + a] = bm[a];
  }
}

}  // namespace fp
