// Four-phonon RTA rate kernels (paper Sec. 2.2 Eqs. tao0, 4phgamma, V4; Sec. 2.4).
//
// One function W serves all three processes.  With k3 = q + k1 + k2 (mod G) and e(-k) = conj e(k),
//   W(q,j0; k1,j1; k2,j2; k3,j3) = sum_quartets sum_{abgt} Phi4/sqrt(M^4) e_a(q,j0) e_b(k1,j1) e_g(k2,j2)
//                                  conj(e_t(k3,j3)) exp(i (k1.R_j + k2.R_k - k3.R_l))
// gives V++(q,k1,k2) = W(q;k1,k2), V+-(q,k1,-k2) = W(q;k1,k2), V--(q,-k1,-k2) = W(q;k1,k2), and
// W(q;k2,k1)[j0 j2 j1 j3] = W(q;k1,k2)[j0 j1 j2 j3] (transposition symmetry, Sec. 2.3 Eq. TS), so one W
// per unordered pair {k1, k2} serves six (ordering, process) terms.
//
// The phase factorises as exp(i(k1.R_j - (q+k1).R_l)) * exp(i k2.(R_k - R_l)); the first factor and the
// contractions with e(q) and e(k1) are hoisted out of the k2 loop:
//   Psi[j0][g][j1][gt] = sum_{Q in group g} tw1_Q sum_{ab} phi_Q[a b g t] e_{ia}(q,j0) e_{jb}(k1,j1)
//   A[j0][j1][(k g)][(l t)] = sum_{groups g of atoms (k,l)} exp(i k2.D_g) Psi[j0][g][j1][g t]
//   T[j0][j1][(k g)][j3]    = sum_{(l t)} A[..][(l t)] conj(e_{lt}(k3,j3))
//   W[j0][j1][j2][j3]       = sum_{(k g)} T[..][(k g)][j3] e_{kg}(k2,j2)
// Groups collect quartets with equal (atom k, atom l, D = R_k - R_l).
//
// Window and Gaussian (Sec. 2.4): the decision |dw| <= window * max(sigma, sigma_min) is the FP64 one,
// with dw = ((w0 +- w') +- w'') - w''' and sigma = (sb * sqrt((dx^2 + dy^2) + dz^2)) * dq evaluated in that
// order without contraction.  An FP32 prefilter with a proven error margin settles almost every
// candidate; only candidates inside the rounding band are re-evaluated in FP64, so decisions are
// identical to the FP64 evaluation.  delta = exp(-(dw/sigma)^2)/(sqrt(pi) sigma), or 1 when
// sigma < sigma_min.
//
// Precision of the two instantiations:
//   double: vertex, sigma, dw, Gaussian, Bose weights and sums in FP64.
//   float:  vertex assembly and contraction in FP32; dw from two-float frequencies (error-free sums,
//           |error| <= 2^-44 sum(w)); sigma from two-float velocities; Gaussian and Bose weights in FP32;
//           compensated (two-float) per-thread sums, FP64 across threads and work items.
#include "fp_internal.cuh"

namespace fp {
namespace {

template <typename R>
struct __align__(2 * sizeof(R)) Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cmk(R a, R b) {
  Cx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return cmk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc += a * b
template <typename R>
__device__ __forceinline__ void cfma(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, fma(-a.im, b.im, acc.re));
  acc.im = fma(a.re, b.im, fma(a.im, b.re, acc.im));
}
// acc += a * conj(b)
template <typename R>
__device__ __forceinline__ void cfma_conj(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, fma(a.im, b.im, acc.re));
  acc.im = fma(a.im, b.re, fma(-a.re, b.im, acc.im));
}
template <typename R>
__device__ __forceinline__ Cx<R> cload(const double2& d) {
  return cmk<R>((R)d.x, (R)d.y);
}

__device__ __forceinline__ int wrapi(int x, int n) {
  int r = x % n;
  return r < 0 ? r + n : r;
}

// s + e = a + b exactly (Knuth's two-sum); the compiler does not reassociate FP additions.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// two-float split of a double: h + l = x to about 2^-48 |x|
__device__ __forceinline__ void split2(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

constexpr float kRelS = 1.0f / 524288.0f;   // 2^-19: prefilter margin per unit of sum(w) and of sigma
constexpr float kRelP = 1.0f / 4194304.0f;  // 2^-22: prefilter margin per unit of window*sigma
constexpr float kAbsV = 1.0f / 1099511627776.0f;  // 2^-40: two-float velocity difference error per |v|_1

// Shared-memory carve shared by the kernel and the host-side size query.
struct Carve {
  size_t E0, E1, E2, E3, Psi, A, T, Tw2, TwQ, ncx;                       // complex elements
  size_t Om0, Om1, Om2, Om3, V1, V2, V3, Sig, W0, W1, W2, W3, Red, ndbl;   // doubles
  size_t Hq, Lq, H1, L1, H2, L2, H3, L3, VH1, VL1, VH2, VL2, VH3, VL3, Sigf, F0, F1, F2, F3, nflt;  // floats
  size_t Mask;  // bytes
  size_t bytes(size_t cx_size) const {
    return ncx * cx_size + ndbl * sizeof(double) + nflt * sizeof(float) + Mask + 16;
  }
};

__host__ __device__ inline Carve make_carve(int nb, int J, int G, int nquart, int nT, int threads) {
  Carve c;
  size_t nb2 = (size_t)nb * nb, nb3 = nb2 * nb;
  size_t o = 0;
  c.E0 = o; o += (size_t)J * nb;
  c.E1 = o; o += nb2;
  c.E2 = o; o += nb2;
  c.E3 = o; o += nb2;
  c.Psi = o; o += (size_t)J * G * nb * 9;
  c.A = o; o += (size_t)J * nb3;
  c.T = o; o += (size_t)J * nb3;
  c.Tw2 = o; o += G;
  c.TwQ = o; o += nquart;
  c.ncx = o;
  size_t d = 0;
  c.Om0 = d; d += J;
  c.Om1 = d; d += nb;
  c.Om2 = d; d += nb;
  c.Om3 = d; d += nb;
  c.V1 = d; d += 3 * nb;
  c.V2 = d; d += 3 * nb;
  c.V3 = d; d += 3 * nb;
  c.Sig = d; d += 8 * nb2;
  c.W0 = d; d += (size_t)nT * J;
  c.W1 = d; d += 2 * (size_t)nT * nb;
  c.W2 = d; d += 2 * (size_t)nT * nb;
  c.W3 = d; d += (size_t)nT * nb;
  c.Red = d; d += (size_t)(threads / 32) * nT;
  c.ndbl = d;
  size_t f = 0;
  c.Hq = f; f += J;
  c.Lq = f; f += J;
  c.H1 = f; f += nb;
  c.L1 = f; f += nb;
  c.H2 = f; f += nb;
  c.L2 = f; f += nb;
  c.H3 = f; f += nb;
  c.L3 = f; f += nb;
  c.VH1 = f; f += 3 * nb;
  c.VL1 = f; f += 3 * nb;
  c.VH2 = f; f += 3 * nb;
  c.VL2 = f; f += 3 * nb;
  c.VH3 = f; f += 3 * nb;
  c.VL3 = f; f += 3 * nb;
  c.Sigf = f; f += 12 * nb2;
  c.F0 = f; f += (size_t)nT * J;
  c.F1 = f; f += 2 * (size_t)nT * nb;
  c.F2 = f; f += 2 * (size_t)nT * nb;
  c.F3 = f; f += (size_t)nT * nb;
  c.nflt = f;
  c.Mask = (size_t)J;
  return c;
}

// FP64 sigma entry for the leg velocity vl (sign s = +1 or -1) and the outgoing mode velocity v3:
// out = (window * max(sigma, sigma_min), 1/sigma or -1 when delta := 1).
__device__ __noinline__ void sigma_entry(const RatesArgs& a, const double* vl, double s, const double* v3,
                                         double* out) {
  double dx = __dsub_rn(s * vl[0], v3[0]);
  double dy = __dsub_rn(s * vl[1], v3[1]);
  double dz = __dsub_rn(s * vl[2], v3[2]);
  double sigma;
  if (a.dq_mode == 0) {
    double s2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    sigma = __dmul_rn(__dmul_rn(a.sb, __dsqrt_rn(s2)), a.dq);
  } else {
    double p[3];
    for (int ax = 0; ax < 3; ++ax) {
      const double* b = a.rec + 3 * ax;
      double t = __dadd_rn(__dadd_rn(__dmul_rn(dx, b[0]), __dmul_rn(dy, b[1])), __dmul_rn(dz, b[2]));
      p[ax] = __ddiv_rn(t, (double)a.grid[ax]);
    }
    double s2 = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(p[0], p[0]), __dmul_rn(p[1], p[1])), __dmul_rn(p[2], p[2])), 3.0);
    sigma = __dmul_rn(a.sb, __dsqrt_rn(s2));
  }
  const bool small = sigma < a.sigma_min;
  out[0] = __dmul_rn(a.window, small ? a.sigma_min : sigma);
  out[1] = small ? -1.0 : __drcp_rn(sigma);
}

// Prefilter entry from an exact FP64 entry: (P~, margin, 1/sigma~).
__device__ __forceinline__ void sigma_f_from_exact(const double* ex, float* out) {
  float P = __double2float_rn(ex[0]);
  out[0] = P;
  out[1] = kRelP * P;
  out[2] = ex[1] < 0.0 ? -1.0f : __double2float_rn(ex[1]);
}

// FP32 sigma entry from two-float velocities (isotropic |dq| only), with a rigorous bound; entries whose
// relation to sigma_min is not settled in FP32 fall back to the exact FP64 entry.
__device__ __forceinline__ void sigma_entry_f32(const RatesArgs& a, const float* vlh, const float* vll, float s,
                                                const float* v3h, const float* v3l, const double* vl64,
                                                const double* v364, float* out) {
  float d[3];
  float v1n = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float h, e;
    two_sum(s * vlh[c], -v3h[c], h, e);
    d[c] = h + (e + (s * vll[c] - v3l[c]));
    v1n += fabsf(vlh[c]) + fabsf(v3h[c]);
  }
  const float sbdq = (float)(a.sb * a.dq);
  const float sig = sbdq * sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
  const float E = kRelS * sig + kAbsV * sbdq * v1n;
  const float smin = (float)a.sigma_min;
  const float window = (float)a.window;
  if (sig - E > 2.0f * smin) {
    const float P = window * sig;
    out[0] = P;
    out[1] = window * E + kRelP * P;
    out[2] = 1.0f / sig;
  } else if (sig + E < 0.5f * smin) {
    const float P = __double2float_rn(a.window * a.sigma_min);
    out[0] = P;
    out[1] = kRelP * P;
    out[2] = -1.0f;
  } else {
    double ex[2];
    sigma_entry(a, vl64, (double)s, v364, ex);
    sigma_f_from_exact(ex, out);
  }
}

// exact FP64 energy mismatch of candidate c (order of the FP64 definition)
__device__ __forceinline__ double dw_fp64(int c, double w0, double wx, double wy, double w3) {
  const double first = c < 3 ? wx : wy, second = c < 3 ? wy : wx;
  const double t1 = (c == 2 || c == 5) ? __dsub_rn(w0, first) : __dadd_rn(w0, first);
  const double t2 = (c == 0 || c == 3) ? __dadd_rn(t1, second) : __dsub_rn(t1, second);
  return __dsub_rn(t2, w3);
}

// candidate c: 0..2 = ordering A (partners (k1,x), (k2,y)) ++, +-, --; 3..5 = ordering B ((k2,y), (k1,x))
__device__ __forceinline__ float mult_of(int c) { return (c % 3 == 2) ? (1.0f / 6.0f) : 0.5f; }

template <typename R>
__global__ void __launch_bounds__(384) rates_kernel(RatesArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  constexpr bool kF64 = sizeof(R) == 8;
  const int nb = a.nb, J = a.J, G = a.G, nT = a.nT, N = a.N;
  const int nb2 = nb * nb, nb3 = nb2 * nb;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const Carve cv = make_carve(nb, J, G, a.nquart, nT, nthr);
  Cx<R>* cx = reinterpret_cast<Cx<R>*>(smem);
  Cx<R>* sE0 = cx + cv.E0;
  Cx<R>* sE1 = cx + cv.E1;
  Cx<R>* sE2 = cx + cv.E2;
  Cx<R>* sE3 = cx + cv.E3;
  Cx<R>* sPsi = cx + cv.Psi;
  Cx<R>* sA = cx + cv.A;
  Cx<R>* sT = cx + cv.T;
  Cx<R>* sTw2 = cx + cv.Tw2;
  Cx<R>* sTwQ = cx + cv.TwQ;
  double* db = reinterpret_cast<double*>(cx + cv.ncx);
  double* sOm0 = db + cv.Om0;
  double* sOm1 = db + cv.Om1;
  double* sOm2 = db + cv.Om2;
  double* sOm3 = db + cv.Om3;
  double* sV1 = db + cv.V1;
  double* sV2 = db + cv.V2;
  double* sV3 = db + cv.V3;
  double* sSig = db + cv.Sig;
  double* sW0 = db + cv.W0;
  double* sW1 = db + cv.W1;
  double* sW2 = db + cv.W2;
  double* sW3 = db + cv.W3;
  double* sRed = db + cv.Red;
  float* fb = reinterpret_cast<float*>(db + cv.ndbl);
  float* sHq = fb + cv.Hq;
  float* sLq = fb + cv.Lq;
  float* sH1 = fb + cv.H1;
  float* sL1 = fb + cv.L1;
  float* sH2 = fb + cv.H2;
  float* sL2 = fb + cv.L2;
  float* sH3 = fb + cv.H3;
  float* sL3 = fb + cv.L3;
  float* sVH1 = fb + cv.VH1;
  float* sVL1 = fb + cv.VL1;
  float* sVH2 = fb + cv.VH2;
  float* sVL2 = fb + cv.VL2;
  float* sVH3 = fb + cv.VH3;
  float* sVL3 = fb + cv.VL3;
  float* sSigf = fb + cv.Sigf;
  float* sF0 = fb + cv.F0;
  float* sF1 = fb + cv.F1;
  float* sF2 = fb + cv.F2;
  float* sF3 = fb + cv.F3;
  unsigned char* sMask = reinterpret_cast<unsigned char*>(fb + cv.nflt);

  const int TPJ = nthr / J;  // threads per j0 in the accumulation phase (multiple of 32)
  const int my_jj = tid / TPJ;
  const int my_lane = tid % TPJ;
  unsigned long long cnt0 = 0, cnt1 = 0, cnt2 = 0;
  const size_t NM = (size_t)N * nb;
  const bool f32_sigma = !kF64 && a.dq_mode == 0;

  for (;;) {
    if (tid == 0) s_item = (long long)atomicAdd(a.counter, 1ULL);
    __syncthreads();
    const long long item = s_item;
    if (item >= a.n_items) break;
    const int chunk = (int)(item % a.nchunk);
    const long long rest = item / a.nchunk;
    const int qi = (int)(rest % a.nq_sel);
    const int tile = (int)(rest / a.nq_sel);
    const int q = a.q_begin + qi;
    const int j0b = chunk * J;
    const int g[3] = {q / (a.grid[1] * a.grid[2]), (q / a.grid[2]) % a.grid[1], q % a.grid[2]};

    for (int o = tid; o < J * nb; o += nthr) {
      int jj = o / nb, comp = o % nb;
      sE0[o] = cload<R>(a.evec[((size_t)q * nb + j0b + jj) * nb + comp]);
    }
    for (int jj = tid; jj < J; jj += nthr) {
      int m = q * nb + j0b + jj;
      double w = a.omega[m];
      sOm0[jj] = w;
      split2(w, sHq[jj], sLq[jj]);
      sMask[jj] = (w > 0.0 && (a.mask == nullptr || a.mask[m])) ? 1 : 0;
    }
    for (int o = tid; o < nT * J; o += nthr) {
      int it = o / J, jj = o % J;
      double w = a.wt[3 * ((size_t)it * NM + (size_t)q * nb + j0b + jj) + 0];
      sW0[o] = w;
      sF0[o] = (float)w;
    }
    __syncthreads();
    int any = 0;
    for (int jj = 0; jj < J; ++jj) any |= sMask[jj];

    double acc[kMaxT];
    float acch[kMaxT], accl[kMaxT];
#pragma unroll
    for (int t = 0; t < kMaxT; ++t) {
      acc[t] = 0.0;
      acch[t] = 0.f;
      accl[t] = 0.f;
    }

    const int k1_begin = tile * a.t1;
    const int k1_end = min(N, k1_begin + a.t1);
    for (int k1 = any ? k1_begin : k1_end; k1 < k1_end; ++k1) {
      const int g1[3] = {k1 / (a.grid[1] * a.grid[2]), (k1 / a.grid[2]) % a.grid[1], k1 % a.grid[2]};
      for (int o = tid; o < nb2; o += nthr) sE1[o] = cload<R>(a.evec[(size_t)k1 * nb2 + o]);
      for (int o = tid; o < nb; o += nthr) {
        double w = a.omega[k1 * nb + o];
        sOm1[o] = w;
        split2(w, sH1[o], sL1[o]);
      }
      for (int o = tid; o < 3 * nb; o += nthr) {
        double v = a.vel[(size_t)k1 * nb * 3 + o];
        sV1[o] = v;
        split2(v, sVH1[o], sVL1[o]);
      }
      for (int o = tid; o < nT * nb; o += nthr) {
        int it = o / nb, j = o % nb;
        const double* w = a.wt + 3 * ((size_t)it * NM + (size_t)k1 * nb + j);
        sW1[2 * o] = w[1];
        sW1[2 * o + 1] = w[2];
        sF1[2 * o] = (float)w[1];
        sF1[2 * o + 1] = (float)w[2];
      }
      for (int Q = tid; Q < a.nquart; Q += nthr) {
        const int* m = a.qmeta + 9 * Q;
        long long e = 0;
        for (int d = 0; d < 3; ++d)
          e += (long long)a.Lfac[d] * wrapi(g1[d] * m[3 + d] - (g[d] + g1[d]) * m[6 + d], a.grid[d]);
        sTwQ[Q] = cload<R>(a.tw[(int)(e % a.L)]);
      }
      __syncthreads();
      // Psi[jj][grp][j1][gt]
      const int npsi = J * G * nb * 9;
      for (int o = tid; o < npsi; o += nthr) {
        const int gt = o % 9;
        const int j1 = (o / 9) % nb;
        const int grp = (o / (9 * nb)) % G;
        const int jj = o / (9 * nb * G);
        Cx<R> sum = cmk<R>(0, 0);
        for (int qq = a.grp_qstart[grp]; qq < a.grp_qstart[grp + 1]; ++qq) {
          const int Q = a.grp_q[qq];
          const int ia = a.qmeta[9 * Q], ja = a.qmeta[9 * Q + 1];
          const double* f = a.qfc + 81 * Q + gt;
          Cx<R> s = cmk<R>(0, 0);
#pragma unroll
          for (int al = 0; al < 3; ++al) {
            Cx<R> e0 = sE0[jj * nb + 3 * ia + al];
#pragma unroll
            for (int be = 0; be < 3; ++be) {
              Cx<R> p = cmul(e0, sE1[j1 * nb + 3 * ja + be]);
              R fv = (R)f[(al * 3 + be) * 9];
              s.re = fma(fv, p.re, s.re);
              s.im = fma(fv, p.im, s.im);
            }
          }
          cfma(sum, sTwQ[Q], s);
        }
        sPsi[o] = sum;
      }
      __syncthreads();

      for (int k2 = k1; k2 < N; ++k2) {
        const int g2[3] = {k2 / (a.grid[1] * a.grid[2]), (k2 / a.grid[2]) % a.grid[1], k2 % a.grid[2]};
        const int g3[3] = {(g[0] + g1[0] + g2[0]) % a.grid[0], (g[1] + g1[1] + g2[1]) % a.grid[1],
                           (g[2] + g1[2] + g2[2]) % a.grid[2]};
        const int k3 = (g3[0] * a.grid[1] + g3[1]) * a.grid[2] + g3[2];
        for (int o = tid; o < nb2; o += nthr) {
          sE2[o] = cload<R>(a.evec[(size_t)k2 * nb2 + o]);
          sE3[o] = cload<R>(a.evec[(size_t)k3 * nb2 + o]);
        }
        for (int o = tid; o < nb; o += nthr) {
          double w2 = a.omega[k2 * nb + o], w3 = a.omega[k3 * nb + o];
          sOm2[o] = w2;
          sOm3[o] = w3;
          split2(w2, sH2[o], sL2[o]);
          split2(w3, sH3[o], sL3[o]);
        }
        for (int o = tid; o < 3 * nb; o += nthr) {
          double v2 = a.vel[(size_t)k2 * nb * 3 + o], v3 = a.vel[(size_t)k3 * nb * 3 + o];
          sV2[o] = v2;
          sV3[o] = v3;
          split2(v2, sVH2[o], sVL2[o]);
          split2(v3, sVH3[o], sVL3[o]);
        }
        for (int o = tid; o < nT * nb; o += nthr) {
          int it = o / nb, j = o % nb;
          const double* w2 = a.wt + 3 * ((size_t)it * NM + (size_t)k2 * nb + j);
          const double w3b = a.wt[3 * ((size_t)it * NM + (size_t)k3 * nb + j) + 2];
          sW2[2 * o] = w2[1];
          sW2[2 * o + 1] = w2[2];
          sW3[o] = w3b;
          sF2[2 * o] = (float)w2[1];
          sF2[2 * o + 1] = (float)w2[2];
          sF3[o] = (float)w3b;
        }
        for (int gi = tid; gi < G; gi += nthr) {
          const int* gm = a.gmeta + 5 * gi;
          long long e = 0;
          for (int d = 0; d < 3; ++d) e += (long long)a.Lfac[d] * wrapi(g2[d] * gm[2 + d], a.grid[d]);
          sTw2[gi] = cload<R>(a.tw[(int)(e % a.L)]);
        }
        __syncthreads();
        // sigma tables [tab][u][j3]: tab 0: v(k2,u)-v3, 1: -v(k2,u)-v3, 2: v(k1,u)-v3, 3: -v(k1,u)-v3
        for (int o = tid; o < 4 * nb2; o += nthr) {
          const int tab = o / nb2, u = (o / nb) % nb, j3 = o % nb;
          const double* vl = (tab < 2 ? sV2 : sV1) + 3 * u;
          const float sgn = (tab & 1) ? -1.0f : 1.0f;
          if (f32_sigma) {
            const float* vlh = (tab < 2 ? sVH2 : sVH1) + 3 * u;
            const float* vll = (tab < 2 ? sVL2 : sVL1) + 3 * u;
            sigma_entry_f32(a, vlh, vll, sgn, sVH3 + 3 * j3, sVL3 + 3 * j3, vl, sV3 + 3 * j3, sSigf + 3 * o);
          } else {
            sigma_entry(a, vl, (double)sgn, sV3 + 3 * j3, sSig + 2 * o);
            sigma_f_from_exact(sSig + 2 * o, sSigf + 3 * o);
          }
        }
        // assembly of A[jj][j1][c][d]
        for (int o = tid; o < J * nb3; o += nthr) {
          const int dd = o % nb, c = (o / nb) % nb;
          const int j1 = (o / nb2) % nb, jj = o / nb3;
          const int ka = c / 3, ga = c % 3, la = dd / 3, th = dd % 3;
          Cx<R> sum = cmk<R>(0, 0);
          const int kl = ka * a.natoms + la;
          for (int gi = a.kl_start[kl]; gi < a.kl_start[kl + 1]; ++gi) {
            const int grp = a.kl_grp[gi];
            cfma(sum, sTw2[grp], sPsi[((jj * G + grp) * nb + j1) * 9 + ga * 3 + th]);
          }
          sA[o] = sum;
        }
        __syncthreads();
        // T[jj][j1][c][j3] = sum_d A[jj][j1][c][d] conj(e_d(k3, j3))
        for (int o = tid; o < J * nb3; o += nthr) {
          const int j3 = o % nb;
          const Cx<R>* arow = sA + (o - j3);
          const Cx<R>* erow = sE3 + j3 * nb;
          Cx<R> sum = cmk<R>(0, 0);
          for (int d = 0; d < nb; ++d) cfma_conj(sum, arow[d], erow[d]);
          sT[o] = sum;
        }
        __syncthreads();
        // W[jj][j1][j2][j3] = sum_c T[jj][j1][c][j3] e_c(k2, j2)  (into sA)
        for (int o = tid; o < J * nb3; o += nthr) {
          const int j3 = o % nb, j2 = (o / nb) % nb;
          const int base = o - j3 - j2 * nb;  // (jj, j1) row start
          const Cx<R>* erow = sE2 + j2 * nb;
          Cx<R> sum = cmk<R>(0, 0);
          for (int c = 0; c < nb; ++c) cfma(sum, sT[base + c * nb + j3], erow[c]);
          sA[o] = sum;
        }
        __syncthreads();
        // window, Gaussian, Bose weights
        if (my_jj < J && sMask[my_jj]) {
          const float h0 = sHq[my_jj], l0 = sLq[my_jj];
          const double w0 = sOm0[my_jj];
          const int ncand = (k1 != k2) ? 6 : 3;
          for (int r = my_lane; r < nb3; r += TPJ) {
            const int x = r / nb2, y = (r / nb) % nb, j3 = r % nb;
            const float hx = sH1[x], hy = sH2[y], h3 = sH3[j3];
            if (hx == 0.f || hy == 0.f || h3 == 0.f) continue;
            const float S = (h0 + hx) + (hy + h3);
            const float ap = h0 + hx, am = h0 - hx, bp = h0 + hy, bm = h0 - hy;
            const float dt[6] = {(ap + hy) - h3, (ap - hy) - h3, (am - hy) - h3,
                                 (bp + hx) - h3, (bp - hx) - h3, (bm - hx) - h3};
            unsigned accm = 0;
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              if (c >= ncand) break;
              const int tab = (c < 3) ? (c == 0 ? 0 : 1) : (c == 3 ? 2 : 3);
              const int ent = tab * nb2 + ((c < 3) ? y : x) * nb + j3;
              const float P = sSigf[3 * ent], M = fmaf(kRelS, S, sSigf[3 * ent + 1]);
              const float ad = fabsf(dt[c]);
              if (ad > P + M) continue;
              if (ad < P - M) {
                accm |= 1u << c;
                continue;
              }
              // rounding band: the FP64 decision
              const double d64 = dw_fp64(c, w0, sOm1[x], sOm2[y], sOm3[j3]);
              double P64;
              if (kF64 || !f32_sigma) {
                P64 = sSig[2 * ent];
              } else {
                double ex[2];
                const double* vl = ((tab < 2) ? sV2 + 3 * y : sV1 + 3 * x);
                sigma_entry(a, vl, (tab & 1) ? -1.0 : 1.0, sV3 + 3 * j3, ex);
                P64 = ex[0];
              }
              if (fabs(d64) <= P64) accm |= 1u << c;
            }
            if (!accm) continue;
            const Cx<R> Wv = sA[my_jj * nb3 + r];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
              if (!(accm & (1u << c))) continue;
              const int p = c % 3;
              cnt0 += (p == 0);
              cnt1 += (p == 1);
              cnt2 += (p == 2);
              const bool ordA = c < 3;
              const int tab = (c < 3) ? (c == 0 ? 0 : 1) : (c == 3 ? 2 : 3);
              const int ent = tab * nb2 + (ordA ? y : x) * nb + j3;
              // Bose factor selectors: leg q' gets (1+n)/w unless --, leg q'' gets (1+n)/w only for ++
              const int s1 = (p == 2) ? 1 : 0, s2 = (p == 0) ? 0 : 1;
              const int i1 = ordA ? x : y, i2 = ordA ? y : x;
              if constexpr (kF64) {
                const double W2 = Wv.re * Wv.re + Wv.im * Wv.im;
                const double d64 = dw_fp64(c, w0, sOm1[x], sOm2[y], sOm3[j3]);
                const double inv = sSig[2 * ent + 1];
                double delta = 1.0;
                if (inv >= 0.0) {
                  const double xx = d64 * inv;
                  delta = exp(-xx * xx) * inv * kInvSqrtPi;
                }
                const double base = (p == 2 ? (1.0 / 6.0) : 0.5) * W2 * delta;
                const double* wq1 = ordA ? sW1 : sW2;  // table of leg q'
                const double* wq2 = ordA ? sW2 : sW1;  // table of leg q''
#pragma unroll
                for (int t = 0; t < kMaxT; ++t) {
                  if (t >= nT) break;
                  acc[t] += base * sW0[t * J + my_jj] * wq1[2 * (t * nb + i1) + s1] * wq2[2 * (t * nb + i2) + s2] *
                            sW3[t * nb + j3];
                }
              } else {
                const float W2 = Wv.re * Wv.re + Wv.im * Wv.im;
                // dw from two-float frequencies with error-free sums
                const float fh = ordA ? hx : hy, fl = ordA ? sL1[x] : sL2[y];
                const float sh = ordA ? hy : hx, sl = ordA ? sL2[y] : sL1[x];
                const float sg1 = (p == 2) ? -1.f : 1.f, sg2 = (p == 0) ? 1.f : -1.f;
                float t0, e1, e2, e3;
                two_sum(h0, sg1 * fh, t0, e1);
                two_sum(t0, sg2 * sh, t0, e2);
                two_sum(t0, -h3, t0, e3);
                const float lo = (((l0 + sg1 * fl) + sg2 * sl) - sL3[j3]) + ((e1 + e2) + e3);
                const float dwf = t0 + lo;
                const float inv = sSigf[3 * ent + 2];
                float delta = 1.0f;
                if (inv >= 0.f) {
                  const float xx = dwf * inv;
                  delta = __expf(-xx * xx) * inv * (float)kInvSqrtPi;
                }
                const float base = mult_of(c) * W2 * delta;
                const float* fq1 = ordA ? sF1 : sF2;
                const float* fq2 = ordA ? sF2 : sF1;
#pragma unroll
                for (int t = 0; t < kMaxT; ++t) {
                  if (t >= nT) break;
                  const float term = base * sF0[t * J + my_jj] * fq1[2 * (t * nb + i1) + s1] *
                                     fq2[2 * (t * nb + i2) + s2] * sF3[t * nb + j3];
                  float s, e;
                  two_sum(acch[t], term, s, e);
                  acch[t] = s;
                  accl[t] += e;
                }
              }
            }
          }
        }
        __syncthreads();
      }
    }
    // reduce per j0 group (TPJ is a multiple of 32: a warp never mixes two j0)
    const int warp = tid / 32, lane = tid % 32;
#pragma unroll
    for (int t = 0; t < kMaxT; ++t) {
      if (t >= nT) break;
      double v = kF64 ? acc[t] : (double)acch[t] + (double)accl[t];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) sRed[warp * nT + t] = v;
    }
    __syncthreads();
    const int wpj = TPJ / 32;
    for (int o = tid; o < J * nT; o += nthr) {
      const int jj = o / nT, t = o % nT;
      double s = 0.0;
      for (int w = 0; w < wpj; ++w) s += sRed[(jj * wpj + w) * nT + t];
      a.partial[(size_t)item * J * nT + o] = s;
    }
    __syncthreads();
  }
  // accepted counts
  for (int off = 16; off > 0; off >>= 1) {
    cnt0 += __shfl_down_sync(0xffffffffu, cnt0, off);
    cnt1 += __shfl_down_sync(0xffffffffu, cnt1, off);
    cnt2 += __shfl_down_sync(0xffffffffu, cnt2, off);
  }
  if ((tid & 31) == 0) {
    if (cnt0) atomicAdd(a.counts + 0, cnt0);
    if (cnt1) atomicAdd(a.counts + 1, cnt1);
    if (cnt2) atomicAdd(a.counts + 2, cnt2);
  }
}

// rates[t][q][j] = pref * sum_tiles partial[(tile, q, chunk)][jj][t], in a fixed order.
__global__ void reduce_kernel(RatesArgs a, double pref, double* rates) {
  const long long n = (long long)a.nT * a.nq_sel * a.nb;
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int j = (int)(o % a.nb);
  const int qi = (int)((o / a.nb) % a.nq_sel);
  const int t = (int)(o / ((long long)a.nb * a.nq_sel));
  const int chunk = j / a.J, jj = j % a.J;
  double s = 0.0;
  for (int tile = 0; tile < a.ntile; ++tile) {
    const long long item = ((long long)tile * a.nq_sel + qi) * a.nchunk + chunk;
    s += a.partial[((size_t)item * a.J + jj) * a.nT + t];
  }
  const int q = a.q_begin + qi;
  rates[((size_t)t * a.N + q) * a.nb + j] = s * pref;
}

}  // namespace

size_t rates_smem_bytes(int precision, int nb, int J, int G, int nquart, int nT, int threads) {
  Carve c = make_carve(nb, J, G, nquart, nT, threads);
  return c.bytes(precision == FP_PREC_FP64 ? sizeof(Cx<double>) : sizeof(Cx<float>));
}

int rates_max_ctas_per_sm(int precision, int threads, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (precision == FP_PREC_FP64) {
    cudaFuncSetAttribute(rates_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rates_kernel<double>, threads, smem);
  } else {
    cudaFuncSetAttribute(rates_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rates_kernel<float>, threads, smem);
  }
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_rates(const RatesArgs& a, int precision, int threads, int ctas, size_t smem, cudaStream_t s) {
  if (precision == FP_PREC_FP64)
    rates_kernel<double><<<ctas, threads, smem, s>>>(a);
  else
    rates_kernel<float><<<ctas, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const RatesArgs& a, double pref, double* d_rates, int q_end, cudaStream_t s) {
  (void)q_end;
  long long n = (long long)a.nT * a.nq_sel * a.nb;
  if (n == 0) return cudaSuccess;
  reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, pref, d_rates);
  return cudaGetLastError();
}

}  // namespace fp
