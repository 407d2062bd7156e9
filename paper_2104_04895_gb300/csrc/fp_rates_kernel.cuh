// Four-phonon RTA rate kernel template (paper Sec. 2.2 Eqs. tao0, 4phgamma, V4; Sec. 2.4).
// Instantiated per precision in fp_rates_f64.cu, fp_rates_df.cu and fp_rates_f32.cu; host logic is in fp_rates.cu.
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
//   Psi[j0][j1][g][gt] = sum_{Q in group g} tw1_Q sum_{ab} phi_Q[a b g t] e_{ia}(q,j0) e_{jb}(k1,j1)
//   A[j0][j1][(k g)][(l t)] = sum_{groups g of atoms (k,l)} exp(i k2.D_g) Psi[j0][j1][g][g t]
//   T[j0][j1][(k g)][j3]    = sum_{(l t)} A[..][(l t)] conj(e_{lt}(k3,j3))
//   W[j0][j1][j2][j3]       = sum_{(k g)} e_{kg}(k2,j2) T[..][(k g)][j3]
// Groups collect quartets with equal (atom k, atom l, D = R_k - R_l).  Thread r < J*nb^2 owns the row
// (j0, j1, c) when it builds A and T (registers -> shared T) and the row (j0, j1 = x, j2 = y) when it
// screens the nb entries (x, y, j3) of that row.  The FP64 path queues the entries with an accepted
// candidate per warp; the warp forms their W 32 at a time and queues their accepted terms, which it
// evaluates 32 at a time.  The FP32 path builds W in the lane's registers and evaluates the lane's
// accepted terms in that lane.
//
// Window and Gaussian (Sec. 2.4): the decision |dw| <= window * max(sigma, sigma_min) is the FP64 one,
// with dw = ((w0 +- w') +- w'') - w''' and sigma = (sb * sqrt((dx^2 + dy^2) + dz^2)) * dq evaluated in that
// order without contraction.  An FP32 prefilter with a proven error margin settles almost every
// candidate; only candidates inside the rounding band are re-evaluated in FP64, so decisions are
// identical to the FP64 evaluation.  delta = exp(-(dw/sigma)^2)/(sqrt(pi) sigma), or 1 when
// sigma < sigma_min.
//
// Precision of the instantiations:
//   double: vertex, sigma, dw, Gaussian (table-driven exp), Bose weights and sums in FP64.
//   double with DF = true: as double, but the vertex assembly and both contractions run in double-float
//           (pairs of floats, about 2^-46 per operation) on the FP32 pipes, and with one temperature so do the
//           accepted terms (dw from two-float frequencies, Gaussian, Bose and row weights, running sums that
//           move into FP64 sums at fixed points); window decisions and sums across lanes and items stay FP64.
//   float:  vertex assembly and contraction in FP32; dw from two-float frequencies (error-free sums,
//           |error| <= 2^-24 |dw| + 2^-44 sum(w)); sigma from two-float velocities; Gaussian and Bose weights in FP32;
//           compensated (two-float) per-thread sums, FP64 across threads and work items.  With TC = true the
//           per-q'' contraction T runs on the tensor cores (fp_tc.cuh).
#pragma once
#include <cmath>
#include <cstring>
#include <type_traits>

#include "fp_internal.cuh"
#include "fp_tc.cuh"

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
__device__ __forceinline__ Cx<R> ld_e(const RatesArgs& a, size_t i);
template <>
__device__ __forceinline__ Cx<double> ld_e<double>(const RatesArgs& a, size_t i) {
  double2 d = a.evec[i];
  return cmk<double>(d.x, d.y);
}
template <>
__device__ __forceinline__ Cx<float> ld_e<float>(const RatesArgs& a, size_t i) {
  float2 d = a.evf[i];
  return cmk<float>(d.x, d.y);
}
template <typename R>
__device__ __forceinline__ Cx<R> ld_tw(const RatesArgs& a, int m);
template <>
__device__ __forceinline__ Cx<double> ld_tw<double>(const RatesArgs& a, int m) {
  double2 d = a.tw[m];
  return cmk<double>(d.x, d.y);
}
template <>
__device__ __forceinline__ Cx<float> ld_tw<float>(const RatesArgs& a, int m) {
  float2 d = a.twf[m];
  return cmk<float>(d.x, d.y);
}
template <typename R>
__device__ __forceinline__ R ld_fc(const RatesArgs& a, size_t i);
template <>
__device__ __forceinline__ double ld_fc<double>(const RatesArgs& a, size_t i) {
  return a.qfc[i];
}
template <>
__device__ __forceinline__ float ld_fc<float>(const RatesArgs& a, size_t i) {
  return a.qfcf[i];
}

// Double-float arithmetic for the FP64-accurate vertex contraction of FP_PREC_DOUBLE_FLOAT: a real is a pair of
// floats (h, l) with value h + l; a complex is a float4 (re.h, re.l, im.h, im.l).  A product keeps the high parts'
// product exactly (fma residual) and the cross terms in FP32; a sum adds the high parts by Knuth's two-sum and the
// low parts in FP32, so each operation keeps about 46 bits (Dekker 1971; the pair is renormalised when stored).
__device__ __forceinline__ float4 cdf_from(double re, double im) {
  const float rh = __double2float_rn(re), ih = __double2float_rn(im);
  return make_float4(rh, __double2float_rn(re - (double)rh), ih, __double2float_rn(im - (double)ih));
}
// (h, l) += (ah + al) (bh + bl), dropping al bl
__device__ __forceinline__ void df_mac(float& h, float& l, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -p)));
  const float s = __fadd_rn(h, p);
  const float bb = __fsub_rn(s, h);
  const float t = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  l = __fadd_rn(l, __fadd_rn(t, e));
  h = s;
}
// acc += a * b
__device__ __forceinline__ void cdf_mac(float4& acc, float4 a, float4 b) {
  df_mac(acc.x, acc.y, a.x, a.y, b.x, b.y);
  df_mac(acc.x, acc.y, -a.z, -a.w, b.z, b.w);
  df_mac(acc.z, acc.w, a.x, a.y, b.z, b.w);
  df_mac(acc.z, acc.w, a.z, a.w, b.x, b.y);
}
// acc += a * conj(b)
__device__ __forceinline__ void cdf_mac_conj(float4& acc, float4 a, float4 b) {
  df_mac(acc.x, acc.y, a.x, a.y, b.x, b.y);
  df_mac(acc.x, acc.y, a.z, a.w, b.z, b.w);
  df_mac(acc.z, acc.w, a.z, a.w, b.x, b.y);
  df_mac(acc.z, acc.w, -a.x, -a.y, b.z, b.w);
}
// (h, l) with |l| <= ulp(h) / 2 (fast two-sum; |h| >= |l| after the accumulation above)
__device__ __forceinline__ float4 cdf_norm(float4 a) {
  const float rs = __fadd_rn(a.x, a.y), is = __fadd_rn(a.z, a.w);
  return make_float4(rs, __fsub_rn(a.y, __fsub_rn(rs, a.x)), is, __fsub_rn(a.w, __fsub_rn(is, a.z)));
}
// |w|^2 in double from a double-float complex: squares with exact high products, two-sum of the two squares
__device__ __forceinline__ double cdf_abs2(float4 w) {
  const float ph = __fmul_rn(w.x, w.x), qh = __fmul_rn(w.z, w.z);
  const float pe = __fmaf_rn(2.0f * w.x, w.y, __fmaf_rn(w.x, w.x, -ph));
  const float qe = __fmaf_rn(2.0f * w.z, w.w, __fmaf_rn(w.z, w.z, -qh));
  const float s = __fadd_rn(ph, qh);
  const float bb = __fsub_rn(s, ph);
  const float t = __fadd_rn(__fsub_rn(ph, __fsub_rn(s, bb)), __fsub_rn(qh, bb));
  return (double)s + (double)__fadd_rn(t, __fadd_rn(pe, qe));
}

// Double-float reals (float2: x high, y low) for the accepted-term evaluation of FP_PREC_DOUBLE_FLOAT with one
// temperature: the frequency difference, the Gaussian and the products run on the FP32 pipes at about 2^-46
// relative error per operation.
__device__ __forceinline__ float2 df_make(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
// (h, l) renormalised, |h| >= |l| (fast two-sum)
__device__ __forceinline__ float2 df_fast(float h, float l) {
  const float s = __fadd_rn(h, l);
  return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}
// a b: the high product exact through its fma residual, the cross terms in FP32, al bl dropped
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p)));
  return df_fast(p, e);
}
// a + b: two-sum of the high parts, low parts in FP32, renormalised
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float bb = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, bb)), __fsub_rn(b.x, bb));
  return df_fast(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
// |w|^2 of a double-float complex (re.h, re.l, im.h, im.l), as a double-float
__device__ __forceinline__ float2 cdf_abs2_df(float4 w) {
  const float ph = __fmul_rn(w.x, w.x), qh = __fmul_rn(w.z, w.z);
  const float pe = __fmaf_rn(2.0f * w.x, w.y, __fmaf_rn(w.x, w.x, -ph));
  const float qe = __fmaf_rn(2.0f * w.z, w.w, __fmaf_rn(w.z, w.z, -qh));
  const float s = __fadd_rn(ph, qh);
  const float bb = __fsub_rn(s, ph);
  const float t = __fadd_rn(__fsub_rn(ph, __fsub_rn(s, bb)), __fsub_rn(qh, bb));
  return df_fast(s, __fadd_rn(t, __fadd_rn(pe, qe)));
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

constexpr float kRelS = 1.0f / 524288.0f;         // 2^-19: prefilter margin per unit of sum(w) and of sigma
constexpr float kRelP = 1.0f / 4194304.0f;        // 2^-22: prefilter margin per unit of window*sigma
constexpr float kAbsV = 1.0f / 1099511627776.0f;  // 2^-40: two-float velocity difference error per |v|_1

// exp(-u) for the FP64 Gaussian, table-driven (P. T. P. Tang, ACM TOMS 15 (1989) 144-157), taking v = 64 u:
// u = k h + r with h = 1/64, k = rint(v) and |r| <= h/2, exp(-u) = exp(-k h) exp(-r); exp(-k h) comes from a table
// of kExpTab entries (0 <= u <= 4), exp(-r) from its Taylor polynomial of degree 5, whose truncation error
// (h/2)^6/6! = 3.2e-16 is about three units of 2^-53. The polynomial runs in t = k - v = -64 r (exact: |t| <= 1/2
// and k lies within a factor 2 of v), with the coefficients 1/n! scaled by 64^-n, exact powers of two. Larger u (only when
// the window exceeds 2) takes exp().
constexpr double kSqrtPi = 1.7724538509055160273;  // sqrt(pi)
constexpr int kExpTab = 264;
constexpr double kExpH = 1.0 / 64.0;
__device__ __forceinline__ double exp_neg64(double v, const double* tab) {
  if (!(v <= 256.0)) return exp(-v * kExpH);
  const int k = __double2int_rn(v);
  const double t = (double)k - v;
  double p = (1.0 / 120.0) / 1073741824.0;  // 64^-5 = 2^-30
  p = fma(p, t, (1.0 / 24.0) / 16777216.0);  // 2^-24
  p = fma(p, t, (1.0 / 6.0) / 262144.0);     // 2^-18
  p = fma(p, t, 0.5 / 4096.0);               // 2^-12
  p = fma(p, t, kExpH);
  p = fma(p, t, 1.0);
  return tab[k] * p;
}

// exp(-v / 64) in double-float for the double-float path, by the method of exp_neg64: k = rint(v), t = k - v
// (|t| <= 1/2, a double-float), exp(-v / 64) = tab[k] exp(t / 64) with the degree-5 Taylor polynomial in t. Its
// two smallest coefficients run in FP32 (their contribution is below 1e-10 and known to 2^-24 of it), the rest
// in double-float; tab holds exp(-k / 64) as double-floats. v beyond the table (a window above 2) takes exp().
constexpr double kE3 = 1.0 / 1572864.0;  // 1 / (3! 64^3)
constexpr float kE3h = (float)kE3;
constexpr float kE3l = (float)(kE3 - (double)kE3h);
__device__ __forceinline__ float2 df_exp_neg64(float2 v, const float2* tab) {
  if (!(v.x <= 256.0f)) return df_make(exp(-((double)v.x + (double)v.y) * kExpH));
  const float kf = rintf(v.x);
  const int k = (int)kf;
  const float2 t = df_add(make_float2(__fsub_rn(kf, v.x), 0.f), make_float2(-v.y, 0.f));  // k - v.x is exact
  const float c45 = __fmaf_rn((float)(1.0 / 128849018880.0), t.x, (float)(1.0 / 402653184.0));  // 1/(5! 64^5), 1/(4! 64^4)
  float2 p = df_add(df_mul(make_float2(c45, 0.f), t), make_float2(kE3h, kE3l));
  p = df_add(df_mul(p, t), make_float2(1.0f / 8192.0f, 0.f));  // 1 / (2! 64^2)
  p = df_add(df_mul(p, t), make_float2(1.0f / 64.0f, 0.f));
  p = df_add(df_mul(p, t), make_float2(1.0f, 0.f));
  return df_mul(tab[k], p);
}

// Shared-memory carve shared by the kernel and the host-side size query.
struct Carve {
  size_t E0, E1, E2, E3, Psi, T, Tw2, TwQ, ncx;                           // complex elements
  size_t Om0, Om1, Om2, Om3, V1, V2, V3, Sig, SigW, W0, W1, W2, W3, Red, Wp, Wq, WA, WB, QD, ndbl, ExpT;  // doubles
  size_t Hq, Lq, H1, L1, H2, L2, H3, L3, VH1, VL1, VH2, VL2, VH3, VL3, Sigf, F0, F1, F2, F3, nflt;  // floats
  size_t KL, QI, EQ, nint;                                                        // ints
  size_t Mask;                                                                // bytes
  __host__ __device__ size_t bytes(size_t cx_size) const {
    return ncx * cx_size + ndbl * sizeof(double) + nflt * sizeof(float) + nint * sizeof(int) + Mask + 16;
  }
};

// terms queued per warp in the screening phase (a power of two)
constexpr int kQCap = 128;
// entries queued per warp (a power of two, at least 64: the queue holds fewer than 32 before a j3 step adds
// at most 32)
constexpr int kEQCap = 64;
// accumulator slots per lane: the j0 values that the 32 rows of one warp can span
__host__ __device__ constexpr int acc_slots(int nb) { return nb == 3 ? 3 : 2; }

// f32: the FP32 path, which has no term queue, weight-product rows or exp table
__host__ __device__ inline Carve make_carve(int nb, int J, int G, int nquart, int nT, int threads, bool f32) {
  Carve c;
  const size_t nb2 = (size_t)nb * nb, na = nb / 3;
  size_t o = 0;
  c.E0 = o; o += (size_t)J * nb;
  c.E1 = o; o += nb2;
  c.E2 = o; o += nb2;
  c.E3 = o; o += nb2;
  c.Psi = o; o += (size_t)J * nb * G * 9;
  c.T = o; o += (size_t)J * nb * (nb2 + 1);  // (j0, j1) blocks padded by one entry (bank spread)
  c.Tw2 = o; o += G;
  c.TwQ = o; o += nquart;
  const size_t nwarps = ((size_t)threads + 31) / 32;
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
  c.SigW = d; d += f32 ? 0 : 4 * nb2;  // FP64: (1/sigma) W3(j3) per sigma entry (one temperature)
  c.W0 = d; d += (size_t)nT * J;
  c.W1 = d; d += 2 * (size_t)nT * nb;
  c.W2 = d; d += 2 * (size_t)nT * nb;
  c.W3 = d; d += (size_t)nT * nb;
  c.Red = d; d += (size_t)threads * acc_slots(nb) * nT;
  c.Wp = d; d += f32 ? 0 : (size_t)threads * 4;  // FP64, one temperature: per-row weight products
  c.Wq = d; d += f32 ? 0 : (size_t)J * nb * 3;    // FP64, one temperature: their (j0, q' branch) factors
  // FP64, several temperatures: Bose-weight products of the q leg with the k1 leg [T][j0][k1 branch][2] and of the
  // k2 leg with the k3 leg [T][k2 branch][k3 branch][2]
  c.WA = d; d += (f32 || nT == 1) ? 0 : (size_t)nT * J * nb * 2;
  c.WB = d; d += (f32 || nT == 1) ? 0 : (size_t)nT * nb * nb * 2;
  c.QD = d; d += f32 ? 0 : nwarps * kQCap;         // FP64: |W|^2 of queued terms
  c.ExpT = d; d += f32 ? 0 : kExpTab;
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
  size_t k = 0;
  c.KL = k; k += na * na + 1 + G;
  c.QI = k; k += f32 ? 0 : nwarps * kQCap;  // FP64: queued term indices
  c.EQ = k; k += f32 ? 0 : nwarps * kEQCap;  // FP64: queued entries
  c.nint = k;
  c.Mask = (size_t)J;
  return c;
}

// FP64 sigma entry for the leg velocity vl (sign s = +1 or -1) and the outgoing mode velocity v3:
// out = (window * max(sigma, sigma_min), 1/sigma or -1 when delta := 1).
__device__ __noinline__ void sigma_entry(const RatesArgs& a, const double* vl, double s, const double* v3,
                                         double* out) {
  // s * vl with s = +1 or -1 is a sign flip: an integer operation rather than an FP64 multiply, same value
  const unsigned long long flip = s < 0.0 ? 0x8000000000000000ULL : 0ULL;
  double dx = __dsub_rn(__longlong_as_double(__double_as_longlong(vl[0]) ^ flip), v3[0]);
  double dy = __dsub_rn(__longlong_as_double(__double_as_longlong(vl[1]) ^ flip), v3[1]);
  double dz = __dsub_rn(__longlong_as_double(__double_as_longlong(vl[2]) ^ flip), v3[2]);
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

// Prefilter entry from an exact FP64 entry: (P~, margin) and 1/sigma~.
__device__ __forceinline__ void sigma_f_from_exact(const double* ex, float2* pm, float* inv) {
  float P = __double2float_rn(ex[0]);
  *pm = make_float2(P, kRelP * P);
  *inv = ex[1] < 0.0 ? -1.0f : __double2float_rn(ex[1]);
}

// FP32 sigma entry from two-float velocities (isotropic |dq| only), with a rigorous bound; entries whose
// relation to sigma_min is not settled in FP32 fall back to the exact FP64 entry.
__device__ __forceinline__ void sigma_entry_f32(const RatesArgs& a, const float* vlh, const float* vll, float s,
                                                const float* v3h, const float* v3l, const double* vl64,
                                                const double* v364, float2* pm, float* inv) {
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
    *pm = make_float2(P, window * E + kRelP * P);
    *inv = 1.0f / sig;
  } else if (sig + E < 0.5f * smin) {
    const float P = __double2float_rn(a.window * a.sigma_min);
    *pm = make_float2(P, kRelP * P);
    *inv = -1.0f;
  } else {
    double ex[2];
    sigma_entry(a, vl64, (double)s, v364, ex);
    sigma_f_from_exact(ex, pm, inv);
  }
}

// exact FP64 energy mismatch of candidate c (order of the FP64 definition)
__device__ __forceinline__ double dw_fp64(int c, double w0, double wx, double wy, double w3) {
  const double first = c < 3 ? wx : wy, second = c < 3 ? wy : wx;
  const double t1 = (c == 2 || c == 5) ? __dsub_rn(w0, first) : __dadd_rn(w0, first);
  const double t2 = (c == 0 || c == 3) ? __dadd_rn(t1, second) : __dsub_rn(t1, second);
  return __dsub_rn(t2, w3);
}

// Tensor-core variant of the mixed path (nb = 6): shared-memory region after the carve, 128-byte aligned.
// A operand of the T contraction: two M = 128 row tiles x (hi, lo) tf32 parts x 128 rows x 16 K; B operand: (hi,
// lo) x 16 N x 16 K; then the mbarrier of the MMA completion and the TMEM base address.
constexpr size_t kTcTile = 128 * 64;
constexpr size_t kTcA = 4 * kTcTile;
constexpr size_t kTcB = 2 * 16 * 64;
constexpr size_t kTcBytes = kTcA + kTcB + 16;
constexpr uint32_t kTcCols = 32;               // TMEM columns: two 128 x 16 FP32 accumulators
constexpr uint32_t kTcMaxPolls = 1u << 22;     // bound of the MMA-completion wait (one timeout ends all MMAs)
__host__ __device__ constexpr size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// largest block of each branch count (J * nb^2 rows, rounded up to warps); two blocks per SM
// Umklapp candidates of one (q, k1, k2) triple (k3 = q + k1 + k2): bit c set when candidate c is an Umklapp
// process (Sec. 2.2: q''' = q + s1 q' + s2 q'' + Q with Q != 0), every wavevector taken as its
// Brillouin-zone representative g / N - m (a.bzm). The candidates' partners (q', q'') with signs (s1, s2):
// ++ (k1, k2) or (k2, k1), +- A (k1, -k2), +- B (k2, -k1), -- (-k1, -k2) or (-k2, -k1); the third is always k3.
__device__ unsigned umklapp_bits(const RatesArgs& a, const int g[3], const int g1[3], const int g2[3],
                                 const int g3[3]) {
  int n1[3], n2[3];
  for (int d = 0; d < 3; ++d) {
    n1[d] = g1[d] ? a.grid[d] - g1[d] : 0;
    n2[d] = g2[d] ? a.grid[d] - g2[d] : 0;
  }
  auto idx = [&](const int* x) { return (x[0] * a.grid[1] + x[1]) * a.grid[2] + x[2]; };
  const int* m0 = a.bzm + 3 * idx(g);
  const int* m3 = a.bzm + 3 * idx(g3);
  // 1 if q + sa qa + sb qb - k3 in representatives is nonzero
  auto umk = [&](const int* ga, int sa, const int* gb, int sb) -> unsigned {
    const int* ma = a.bzm + 3 * idx(ga);
    const int* mb = a.bzm + 3 * idx(gb);
    unsigned u = 0;
    for (int d = 0; d < 3; ++d) {
      const int n = a.grid[d];
      const int num = (g[d] - n * m0[d]) + sa * (ga[d] - n * ma[d]) + sb * (gb[d] - n * mb[d]) - (g3[d] - n * m3[d]);
      u |= num != 0 ? 1u : 0u;
    }
    return u;
  };
  const unsigned upp = umk(g1, 1, g2, 1), upa = umk(g1, 1, n2, -1), upb = umk(g2, 1, n1, -1);
  const unsigned umm = umk(n1, -1, n2, -1);
  return upp | (upa << 1) | (umm << 2) | (upp << 3) | (upb << 4) | (umm << 5);
}

__host__ __device__ constexpr int max_threads_for(int nb) { return nb == 3 ? 128 : nb == 6 ? 224 : 160; }

// blocks per SM the register budget is sized for (three FP32 blocks measured 11% faster than two on the
// diamond 8x8x8 workload despite a few spilled registers)
#ifndef FP_F32_MIN_BLOCKS
#define FP_F32_MIN_BLOCKS 3
#endif
template <typename R>
__host__ __device__ constexpr int min_blocks_for() { return sizeof(R) == 4 ? FP_F32_MIN_BLOCKS : 2; }

// Window test of the six candidates of entry (x, y, j3), written as a macro over the names of the
// screening scope (row sums apy .. bmm, h3, sS, the sigma pairs a0 a1 b0 b1, cand, w0): sets accm to the
// accepted candidates. The FP32 prefilter accepts when |dw~| < P - M and rejects when |dw~| > P + M;
// candidates in between (band) are decided in FP64 exactly as the FP64 definition decides them.
#define FP_SCREEN(c, dv, pm)                                               \
  {                                                                        \
    const float M_ = sS + (pm).y, ad_ = fabsf(dv);                         \
    accm |= (ad_ < (pm).x - M_ ? 1u : 0u) << (c);                          \
    band |= (ad_ <= (pm).x + M_ && !(ad_ < (pm).x - M_) ? 1u : 0u) << (c); \
  }
// ++ in both orderings (and -- likewise) have nearly equal dw~ and are rarely accepted: one combined
// rejection (the same float comparisons as the individual tests) covers the pair
#define FP_WINDOW_TEST()                                                                               \
  {                                                                                                    \
    const float d0 = apy - h3, d3 = bpx - h3;                                                          \
    if (fminf(fabsf(d0), fabsf(d3)) <= fmaxf(a0.x + (sS + a0.y), b0.x + (sS + b0.y))) {                \
      FP_SCREEN(0, d0, a0)                                                                             \
      FP_SCREEN(3, d3, b0)                                                                             \
    }                                                                                                  \
    const float d2 = amm - h3, d5 = bmm - h3;                                                          \
    if (fminf(fabsf(d2), fabsf(d5)) <= fmaxf(a1.x + (sS + a1.y), b1.x + (sS + b1.y))) {                \
      FP_SCREEN(2, d2, a1)                                                                             \
      FP_SCREEN(5, d5, b1)                                                                             \
    }                                                                                                  \
    FP_SCREEN(1, apm - h3, a1)                                                                         \
    FP_SCREEN(4, bpm - h3, b1)                                                                         \
    accm &= cand;                                                                                      \
    band &= cand;                                                                                      \
    while (band) {                                                                                     \
      const int c_ = __ffs(band) - 1;                                                                  \
      band &= band - 1;                                                                                \
      const int tab_ = (c_ < 3) ? (c_ == 0 ? 0 : 1) : (c_ == 3 ? 2 : 3);                              \
      const int ent_ = tab_ * NB2 + ((c_ < 3) ? y : x) * NB + j3;                                      \
      const double d64_ = dw_fp64(c_, w0, sOm1[x], sOm2[y], sOm3[j3]);                                 \
      double P64_;                                                                                     \
      if (!f32_sigma) {                                                                                \
        P64_ = sSig[2 * ent_];                                                                         \
      } else {                                                                                         \
        double ex_[2];                                                                                 \
        const double* vl_ = ((tab_ < 2) ? sV2 + 3 * y : sV1 + 3 * x);                                  \
        sigma_entry(a, vl_, (tab_ & 1) ? -1.0 : 1.0, sV3 + 3 * j3, ex_);                               \
        P64_ = ex_[0];                                                                                 \
      }                                                                                                \
      if (fabs(d64_) <= P64_) accm |= 1u << c_;                                                        \
    }                                                                                                  \
  }

// TC: the T contraction of the mixed path on the tensor cores (tcgen05 kind::tf32 in split precision, 3xTF32),
// for nb = 6 only; the rest of the kernel is unchanged.
// DF: the FP64 path with its vertex contraction (A, T, W) in double-float on the FP32 pipes (Psi, twiddles and
// eigenvectors stored as float pairs in the same shared-memory slots); everything else as in the FP64 path.
template <typename R, int NB, int MAXT, bool TC = false, bool DF = false>
__global__ void __launch_bounds__(max_threads_for(NB), TC ? 2 : min_blocks_for<R>()) rates_kernel(RatesArgs a) {
  constexpr int NB2 = NB * NB, NA = NB / 3;
  constexpr bool kF64 = sizeof(R) == 8;
  constexpr bool kDF = DF;
  // double-float path with one temperature: the accepted terms are evaluated in double-float on the FP32 pipes
  constexpr bool kDFC = DF && MAXT == 1;
  using QT = typename std::conditional<kDFC, float2, double>::type;  // |W|^2 of a queued term
  static_assert(!TC || (!kF64 && NB == 6), "the tensor-core T contraction is built for the mixed path, nb = 6");
  static_assert(!DF || kF64, "the double-float contraction belongs to the FP64 path");
  using C = Cx<R>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ unsigned s_umask;  // Umklapp candidates of the current (k1, k2)
  __shared__ int s_tc_fail;     // a tensor-core completion wait ran out of polls: no further MMAs or waits
  const int J = a.J, G = a.G, nT = a.nT, N = a.N;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rows = J * NB2;
  const Carve cv = make_carve(NB, J, G, a.nquart, nT, nthr, !kF64);
  C* cx = reinterpret_cast<C*>(smem);
  C* sE0 = cx + cv.E0;
  C* sE1 = cx + cv.E1;
  C* sE2 = cx + cv.E2;
  C* sE3 = cx + cv.E3;
  C* sPsi = cx + cv.Psi;
  C* sT = cx + cv.T;
  C* sTw2 = cx + cv.Tw2;
  C* sTwQ = cx + cv.TwQ;
  double* db = reinterpret_cast<double*>(cx + cv.ncx);
  double* sOm0 = db + cv.Om0;
  double* sOm1 = db + cv.Om1;
  double* sOm2 = db + cv.Om2;
  double* sOm3 = db + cv.Om3;
  double* sV1 = db + cv.V1;
  double* sV2 = db + cv.V2;
  double* sV3 = db + cv.V3;
  double* sSig = db + cv.Sig;  // [4][NB][NB] (window * max(sigma, sigma_min), 8/sigma or -1 when delta := 1)
  double* sSigW = db + cv.SigW;  // [4][NB][NB] (1/sigma) W3(j3), or sqrt(pi) W3(j3) when delta := 1
  double* sW0 = db + cv.W0;
  double* sW1 = db + cv.W1;
  double* sW2 = db + cv.W2;
  double* sW3 = db + cv.W3;
  double* sRed = db + cv.Red;
  double* sExpT = db + cv.ExpT;
  double* sWp = db + cv.Wp;  // [thread][4] (FP64, one temperature)
  double* sWq = db + cv.Wq;  // [j0][q' branch][3] (FP64, one temperature)
  double* sWA = db + cv.WA;  // [T][j0][k1 branch][2] (FP64, several temperatures)
  double* sWB = db + cv.WB;  // [T][k2 branch][k3 branch][2] (FP64, several temperatures)
  QT* sQD = reinterpret_cast<QT*>(db + cv.QD);  // [warp][kQCap]
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
  float2* sSigPM = reinterpret_cast<float2*>(fb + cv.Sigf);  // [4][NB][NB] (P~, margin)
  float* sSigI = fb + cv.Sigf + 8 * NB2;                      // [4][NB][NB] 1/sigma~ (-1: delta := 1)
  float* sF0 = fb + cv.F0;
  float* sF1 = fb + cv.F1;
  float* sF2 = fb + cv.F2;
  float* sF3 = fb + cv.F3;
  int* ib = reinterpret_cast<int*>(fb + cv.nflt);
  int* sKLs = ib + cv.KL;            // [NA*NA + 1]
  int* sKLg = sKLs + NA * NA + 1;    // [G]
  int* sQI = ib + cv.QI;             // [warp][kQCap]
  int* sEQ = ib + cv.EQ;             // [warp][kEQCap]
  // per j0 of the item: the selected modes the row stands for (0: inactive; 2: also written at -q)
  unsigned char* sMult = reinterpret_cast<unsigned char*>(ib + cv.nint);

  // the row this thread owns in the contraction and screening phases
  const bool has_row = tid < rows;
  const int rjj = tid / NB2, rj1 = (tid / NB) % NB, rc = tid % NB;
  const size_t NM = (size_t)N * NB;
  // isotropic |dq|: the window's sigma tables come from two-float velocities with a rigorous bound (exact
  // decisions; FP64 entries only where the bound does not settle them), in both precisions
  const bool f32_sigma = a.dq_mode == 0;
  const double inv_sbdq = kF64 ? 1.0 / (a.sb * a.dq) : 0.0;  // FP64 path: 1/sigma = inv_sbdq / |dv|
  constexpr int S = acc_slots(NB);
  const int lane = tid & 31;
  const int qbase = (tid >> 5) * kQCap;
  const int ebase = (tid >> 5) * kEQCap;
  const int jj_lo = (tid & ~31) / NB2;  // the j0 of this warp's first row; its rows span jj_lo .. jj_lo + S - 1

  // tensor-core state: operand buffers (zeroed once: padding rows and columns stay zero), TMEM accumulators
  unsigned char* tcbuf = TC ? smem + align128(cv.bytes(sizeof(C))) : smem;
  uint64_t* s_mbar = reinterpret_cast<uint64_t*>(tcbuf + kTcA + kTcB);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(tcbuf + kTcA + kTcB + 8);
  uint32_t tmem_base = 0, tc_phase = 0;
  if constexpr (TC) {
    for (int o = tid; o < (int)((kTcA + kTcB) / 16); o += nthr) reinterpret_cast<uint4*>(tcbuf)[o] = make_uint4(0, 0, 0, 0);
    if ((tid >> 5) == 0) tc::tmem_alloc(s_tmem, kTcCols);
    if (tid == 0) {
      s_tc_fail = 0;
      tc::mbar_init(s_mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tmem_base = *s_tmem;
  }
  if constexpr (kDFC)
    for (int o = tid; o < kExpTab; o += nthr) reinterpret_cast<float2*>(sExpT)[o] = df_make(exp(-(double)o * kExpH));
  else if constexpr (kF64)
    for (int o = tid; o < kExpTab; o += nthr) sExpT[o] = exp(-(double)o * kExpH);
  for (int o = tid; o < NA * NA + 1; o += nthr) sKLs[o] = a.kl_start[o];
  for (int o = tid; o < G; o += nthr) sKLg[o] = a.kl_grp[o];

  for (;;) {
    if (tid == 0) s_item = (long long)atomicAdd(a.counter, 1ULL);
    __syncthreads();
    const long long item = s_item;
    if (item >= a.n_items) break;
    const int chunk = (int)(item % a.nchunk);
    const long long rest = item / a.nchunk;
    const int qi = (int)(rest % a.nq_sel);
    const int tile = (int)(rest / a.nq_sel);
    const int q = a.qlist[qi];
    const int j0b = chunk * J;
    const int g[3] = {q / (a.grid[1] * a.grid[2]), (q / a.grid[2]) % a.grid[1], q % a.grid[2]};

    for (int o = tid; o < J * NB; o += nthr) sE0[o] = ld_e<R>(a, ((size_t)q * NB + j0b) * NB + o);
    for (int jj = tid; jj < J; jj += nthr) {
      const int m = q * NB + j0b + jj;
      const double w = a.omega[m];
      sOm0[jj] = w;
      sHq[jj] = a.omh[m];
      sLq[jj] = a.oml[m];
      sMult[jj] = w > 0.0 ? a.mult[m] : 0;
    }
    for (int o = tid; o < nT * J; o += nthr) {
      const int it = o / J, jj = o % J;
      const size_t idx = 3 * ((size_t)it * NM + (size_t)q * NB + j0b + jj);
      if (kF64)
        sW0[o] = a.wt[idx];
      else
        sF0[o] = a.wtf[idx];
    }
    __syncthreads();
    int any = 0;
    for (int jj = 0; jj < J; ++jj) any |= sMult[jj];
    const bool active = has_row && sMult[rjj] != 0;
    const unsigned row_mult = active ? sMult[rjj] : 0u;

    double acc[S][MAXT];
    float acch[S][MAXT], accl[S][MAXT];
#pragma unroll
    for (int sl = 0; sl < S; ++sl)
#pragma unroll
      for (int t = 0; t < MAXT; ++t) {
        acc[sl][t] = 0.0;
        acch[sl][t] = 0.f;
        accl[sl][t] = 0.f;
      }
    // FP64 path: one queued term (|W|^2 and info = c | j3 << 3 | y << 7 | x << 11 | jj << 15): Gaussian and
    // Bose weights into the accumulator slot of its j0
    auto consume = [&](const QT W2, const int info) {
      const int c = info & 7, j3 = (info >> 3) & 15, iy = (info >> 7) & 15, ix = (info >> 11) & 15;
      const int jq = info >> 15;
      const int slot = jq - jj_lo;
      const int p = c % 3;
      const bool ordA = c < 3;
      const int tab = ordA ? (c == 0 ? 0 : 1) : (c == 3 ? 2 : 3);
      const int ent = tab * NB2 + (ordA ? iy : ix) * NB + j3;
      // Bose selectors: leg q' takes (1+n)/w unless --, leg q'' takes (1+n)/w only for ++
      const int s1 = (p == 2) ? 1 : 0, s2 = (p == 0) ? 0 : 1;
      const int cls = (p == 0) ? 0 : (p == 2) ? 3 : ordA ? 1 : 2;
      if constexpr (kDFC) {
        // double-float: dw from the two-float frequencies by error-free sums, 64 x^2 = (dw 8/sigma)^2, the
        // Gaussian, and the products, on the FP32 pipes
        const float fh = ordA ? sH1[ix] : sH2[iy], fl = ordA ? sL1[ix] : sL2[iy];
        const float sh = ordA ? sH2[iy] : sH1[ix], sl2 = ordA ? sL2[iy] : sL1[ix];
        const float sg1 = (p == 2) ? -1.f : 1.f, sg2 = (p == 0) ? 1.f : -1.f;
        float t0, e1, e2, e3;
        two_sum(sHq[jq], sg1 * fh, t0, e1);
        two_sum(t0, sg2 * sh, t0, e2);
        two_sum(t0, -sH3[j3], t0, e3);
        const float lo = (((sLq[jq] + sg1 * fl) + sg2 * sl2) - sL3[j3]) + ((e1 + e2) + e3);
        const float2 dw = df_add(make_float2(t0, 0.f), make_float2(lo, 0.f));
        const float2 iv8 = reinterpret_cast<const float2*>(sSig)[2 * ent + 1];  // 8 / sigma, or (-1, 0)
        float2 g = reinterpret_cast<const float2*>(sSigW)[ent];                  // (1/sigma) W3, or sqrt(pi) W3
        if (iv8.x >= 0.f) {
          const float2 x8 = df_mul(dw, iv8);
          g = df_mul(g, df_exp_neg64(df_mul(x8, x8), reinterpret_cast<const float2*>(sExpT)));
        }
        const float2 term =
            df_mul(df_mul(W2, g), reinterpret_cast<const float2*>(sWp)[4 * (jq * NB2 + ix * NB + iy) + cls]);
        // two-float running sum of the slot (all terms are positive), moved to the FP64 sum every few q''
#pragma unroll
        for (int sl = 0; sl < S; ++sl)
          if (sl == slot) {
            float sm, er;
            two_sum(acch[sl][0], term.x, sm, er);
            const float2 n = df_fast(sm, __fadd_rn(er, __fadd_rn(accl[sl][0], term.y)));
            acch[sl][0] = n.x;
            accl[sl][0] = n.y;
          }
      } else {
        const double d64 = dw_fp64(c, sOm0[jq], sOm1[ix], sOm2[iy], sOm3[j3]);
        const double iv8 = sSig[2 * ent + 1];  // 8 / sigma, or -1 when delta := 1
        // sqrt(pi) delta; the 1/sqrt(pi) is folded into the row weights (one temperature) or the multiplicity
        if constexpr (MAXT == 1) {
          double g = sSigW[ent];  // sqrt(pi) delta W3 = exp(-x^2) (1/sigma) W3
          if (iv8 >= 0.0) {
            const double x8 = d64 * iv8;
            g *= exp_neg64(x8 * x8, sExpT);
          }
          const double term = (W2 * g) * sWp[4 * (jq * NB2 + ix * NB + iy) + cls];
#pragma unroll
          for (int sl = 0; sl < S; ++sl)
            if (sl == slot) acc[sl][0] += term;
        } else {
          double delta = kSqrtPi;
          if (iv8 >= 0.0) {
            const double x8 = d64 * iv8;
            delta = exp_neg64(x8 * x8, sExpT) * (0.125 * iv8);
          }
          const double base = (p == 2 ? kInvSqrtPi / 6.0 : 0.5 * kInvSqrtPi) * W2 * delta;
          // the k1 leg is q' in ordering A (selector s1) and q'' in ordering B (s2); the k2 leg the other one
          const int sx = ordA ? s1 : s2, sy = ordA ? s2 : s1;
          const double* wa = sWA + 2 * (jq * NB + ix) + sx;
          const double* wb = sWB + 2 * (iy * NB + j3) + sy;
#pragma unroll
          for (int t = 0; t < MAXT; ++t) {
            if (t >= nT) break;
            const double term = (base * wa[2 * t * J * NB]) * wb[2 * t * NB2];
#pragma unroll
            for (int sl = 0; sl < S; ++sl)
              if (sl == slot) acc[sl][t] += term;
          }
        }
      }
    };

    // double-float path, one temperature: the slots' two-float running sums into the FP64 sums (every 64 q'' and
    // at the end of each q', so that a running sum holds a bounded number of terms)
    auto flush_df = [&]() {
      if constexpr (kDFC) {
#pragma unroll
        for (int sl = 0; sl < S; ++sl) {
          acc[sl][0] += (double)acch[sl][0] + (double)accl[sl][0];
          acch[sl][0] = 0.f;
          accl[sl][0] = 0.f;
        }
      }
    };

    // counters of this item, flushed to the launch totals at its end: accepted terms per process, weighted by the
    // row's multiplicity (the evaluated terms are these over the multiplicity), and vertex entries formed
    unsigned cnt0 = 0, cnt1 = 0, cnt2 = 0, nwf = 0;
    const int k1_begin = tile * a.t1;
    const int k1_end = min(N, k1_begin + a.t1);
    // unit-vertex (phase-space) mode: q' on a stride, every q'' in one ordering, |W|^2 = 1
    const bool unit = a.unit_vertex != 0;
    const int k1_first = unit ? ((k1_begin + a.k1_stride - 1) / a.k1_stride) * a.k1_stride : k1_begin;
    const int k1_step = unit ? a.k1_stride : 1;
    for (int k1 = any ? k1_first : k1_end; k1 < k1_end; k1 += k1_step) {
      const int g1[3] = {k1 / (a.grid[1] * a.grid[2]), (k1 / a.grid[2]) % a.grid[1], k1 % a.grid[2]};
      for (int o = tid; o < NB2; o += nthr) sE1[o] = ld_e<R>(a, (size_t)k1 * NB2 + o);
      for (int o = tid; o < NB; o += nthr) {
        sOm1[o] = a.omega[k1 * NB + o];
        sH1[o] = a.omh[k1 * NB + o];
        sL1[o] = a.oml[k1 * NB + o];
      }
      for (int o = tid; o < 3 * NB; o += nthr) {
        sV1[o] = a.vel[(size_t)k1 * NB * 3 + o];
        sVH1[o] = a.velh[(size_t)k1 * NB * 3 + o];
        sVL1[o] = a.vell[(size_t)k1 * NB * 3 + o];
      }
      for (int o = tid; o < nT * NB; o += nthr) {
        const int it = o / NB, j = o % NB;
        const size_t idx = 3 * ((size_t)it * NM + (size_t)k1 * NB + j);
        if (kF64) {
          sW1[2 * o] = a.wt[idx + 1];
          sW1[2 * o + 1] = a.wt[idx + 2];
        } else {
          sF1[2 * o] = a.wtf[idx + 1];
          sF1[2 * o + 1] = a.wtf[idx + 2];
        }
      }
      for (int Q = tid; Q < a.nquart; Q += nthr) {
        const int* m = a.qmeta + 9 * Q;
        int e = 0;  // each term is below L, so e < 3 L
        for (int d = 0; d < 3; ++d) e += a.Lfac[d] * wrapi(g1[d] * m[3 + d] - (g[d] + g1[d]) * m[6 + d], a.grid[d]);
        while (e >= a.L) e -= a.L;
        sTwQ[Q] = ld_tw<R>(a, e);
      }
      __syncthreads();
      if constexpr (kF64 && MAXT == 1) {
        // the (j0, q' branch) factors of the row weight products below: c_p (1/(n0 w0)) times the q' leg's
        // (1+n)/w or n/w, with the 1/sqrt(pi) of the Gaussian; read after the barrier that ends the Psi prologue
        for (int o = tid; o < J * NB; o += nthr) {
          const double f0 = sW0[o / NB], a1 = sW1[2 * (o % NB)], b1 = sW1[2 * (o % NB) + 1];
          const double w0 = (0.5 * kInvSqrtPi) * f0 * a1, w1 = (0.5 * kInvSqrtPi) * f0 * b1;
          const double w2 = (kInvSqrtPi / 6.0) * f0 * b1;
          if constexpr (kDFC) {  // as double-floats in the same slots
            float2* wf = reinterpret_cast<float2*>(sWq + 3 * o);
            wf[0] = df_make(w0);
            wf[1] = df_make(w1);
            wf[2] = df_make(w2);
          } else {
            sWq[3 * o] = w0;
            sWq[3 * o + 1] = w1;
            sWq[3 * o + 2] = w2;
          }
        }
      }
      if constexpr (kF64 && MAXT > 1) {
        // W0(T, j0) times the k1 leg's (1+n)/w and n/w, per temperature; read after the Psi prologue's barrier
        for (int o = tid; o < nT * J * NB; o += nthr) {
          const int t = o / (J * NB), jq = (o / NB) % J, xb = o % NB;
          const double w0 = sW0[t * J + jq];
          sWA[2 * o] = w0 * sW1[2 * (t * NB + xb)];
          sWA[2 * o + 1] = w0 * sW1[2 * (t * NB + xb) + 1];
        }
      }
      // Psi[jj][j1][grp][gt]: one thread per (jj, j1, grp) and block of kGtb of the nine (gamma, theta); the
      // nine products e0(alpha) e1(beta) of each quartet are formed once per block. Tasks are numbered group-major,
      // so the lanes of a warp mostly share one group: the same quartets, and the same trip count
      constexpr int kGtb = 3;
      const int npsi = unit ? 0 : J * NB * G * (9 / kGtb);
      for (int o = tid; o < npsi; o += nthr) {
        const int gb = o % (9 / kGtb);
        const int jr = (o / (9 / kGtb)) % (J * NB);  // jj * NB + j1
        const int grp = o / ((9 / kGtb) * J * NB);
        const int t9 = jr * G + grp;
        const int j1 = jr % NB, jj = jr / NB;
        C sum[kGtb];
#pragma unroll
        for (int u = 0; u < kGtb; ++u) sum[u] = cmk<R>(0, 0);
        for (int qq = a.grp_qstart[grp]; qq < a.grp_qstart[grp + 1]; ++qq) {
          const int Q = a.grp_q[qq];
          const int ia = a.qmeta[9 * Q], ja = a.qmeta[9 * Q + 1];
          C p[9];
#pragma unroll
          for (int al = 0; al < 3; ++al) {
            const C e0 = sE0[jj * NB + 3 * ia + al];
#pragma unroll
            for (int be = 0; be < 3; ++be) p[al * 3 + be] = cmul(e0, sE1[j1 * NB + 3 * ja + be]);
          }
          const C tq = sTwQ[Q];
          const size_t fo = 81 * (size_t)Q + gb * kGtb;
#pragma unroll
          for (int u = 0; u < kGtb; ++u) {
            C s = cmk<R>(0, 0);
#pragma unroll
            for (int ab = 0; ab < 9; ++ab) {
              const R fv = ld_fc<R>(a, fo + ab * 9 + u);
              s.re = fma(fv, p[ab].re, s.re);
              s.im = fma(fv, p[ab].im, s.im);
            }
            cfma(sum[u], tq, s);
          }
        }
        if constexpr (kDF) {
#pragma unroll
          for (int u = 0; u < kGtb; ++u)
            reinterpret_cast<float4*>(sPsi)[(size_t)t9 * 9 + gb * kGtb + u] = cdf_from(sum[u].re, sum[u].im);
        } else {
#pragma unroll
          for (int u = 0; u < kGtb; ++u) sPsi[(size_t)t9 * 9 + gb * kGtb + u] = sum[u];
        }
      }
      __syncthreads();

      const int k2_first = unit ? 0 : k1;
      // grid coordinates of q'' (advanced in row-major order) and of q + q'; the third partner is q + q' + q''
      int g2[3] = {k2_first / (a.grid[1] * a.grid[2]), (k2_first / a.grid[2]) % a.grid[1], k2_first % a.grid[2]};
      const int gs[3] = {(g[0] + g1[0]) % a.grid[0], (g[1] + g1[1]) % a.grid[1], (g[2] + g1[2]) % a.grid[2]};
      for (int k2 = k2_first; k2 < N; ++k2) {
        // ---- phase 1: per-k2 tables
        if (k2 != k2_first && ++g2[2] == a.grid[2]) {
          g2[2] = 0;
          if (++g2[1] == a.grid[1]) {
            g2[1] = 0;
            ++g2[0];
          }
        }
        int g3[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          g3[d] = gs[d] + g2[d];
          if (g3[d] >= a.grid[d]) g3[d] -= a.grid[d];
        }
        const int k3 = (g3[0] * a.grid[1] + g3[1]) * a.grid[2] + g3[2];
        if (a.nu_select != 0 && tid == 0) s_umask = umklapp_bits(a, g, g1, g2, g3);  // read after the barrier
        for (int o = tid; o < NB2; o += nthr) {
          if constexpr (kDF) {
            const double2 e2v = a.evec[(size_t)k2 * NB2 + o], e3v = a.evec[(size_t)k3 * NB2 + o];
            reinterpret_cast<float4*>(sE2)[o] = cdf_from(e2v.x, e2v.y);
            reinterpret_cast<float4*>(sE3)[o] = cdf_from(e3v.x, e3v.y);
          } else {
            sE2[o] = ld_e<R>(a, (size_t)k2 * NB2 + o);
            sE3[o] = ld_e<R>(a, (size_t)k3 * NB2 + o);
          }
        }
        for (int o = tid; o < NB; o += nthr) {
          sOm2[o] = a.omega[k2 * NB + o];
          sOm3[o] = a.omega[k3 * NB + o];
          sH2[o] = a.omh[k2 * NB + o];
          sL2[o] = a.oml[k2 * NB + o];
          sH3[o] = a.omh[k3 * NB + o];
          sL3[o] = a.oml[k3 * NB + o];
        }
        for (int o = tid; o < 3 * NB; o += nthr) {
          sV2[o] = a.vel[(size_t)k2 * NB * 3 + o];
          sV3[o] = a.vel[(size_t)k3 * NB * 3 + o];
          if (f32_sigma) {
            sVH2[o] = a.velh[(size_t)k2 * NB * 3 + o];
            sVL2[o] = a.vell[(size_t)k2 * NB * 3 + o];
            sVH3[o] = a.velh[(size_t)k3 * NB * 3 + o];
            sVL3[o] = a.vell[(size_t)k3 * NB * 3 + o];
          }
        }
        for (int o = tid; o < nT * NB; o += nthr) {
          const int it = o / NB, j = o % NB;
          const size_t i2 = 3 * ((size_t)it * NM + (size_t)k2 * NB + j);
          const size_t i3 = 3 * ((size_t)it * NM + (size_t)k3 * NB + j);
          if constexpr (kDFC) {  // the q'' leg weights as double-floats in the same slots
            reinterpret_cast<float2*>(sW2)[2 * o] = df_make(a.wt[i2 + 1]);
            reinterpret_cast<float2*>(sW2)[2 * o + 1] = df_make(a.wt[i2 + 2]);
            sW3[o] = a.wt[i3 + 2];
          } else if (kF64) {
            sW2[2 * o] = a.wt[i2 + 1];
            sW2[2 * o + 1] = a.wt[i2 + 2];
            sW3[o] = a.wt[i3 + 2];
          } else {
            sF2[2 * o] = a.wtf[i2 + 1];
            sF2[2 * o + 1] = a.wtf[i2 + 2];
            sF3[o] = a.wtf[i3 + 2];
          }
        }
        for (int gi = tid; gi < G; gi += nthr) {
          const int* gm = a.gmeta + 5 * gi;
          int e = 0;  // each term is below L, so e < 3 L
          for (int d = 0; d < 3; ++d) e += a.Lfac[d] * wrapi(g2[d] * gm[2 + d], a.grid[d]);
          while (e >= a.L) e -= a.L;
          if constexpr (kDF) {
            const double2 t = a.tw[e];
            reinterpret_cast<float4*>(sTw2)[gi] = cdf_from(t.x, t.y);
          } else {
            sTw2[gi] = ld_tw<R>(a, e);
          }
        }
        __syncthreads();
        // ---- phase 2: sigma tables; A row and T row
        if constexpr (kF64 && MAXT > 1) {
          // the k2 leg's (1+n)/w and n/w times W3(T, k3 branch), per temperature (read in phase 3)
          for (int o = tid; o < nT * NB2; o += nthr) {
            const int t = o / NB2, yb = (o / NB) % NB, j3b = o % NB;
            const double w3 = sW3[t * NB + j3b];
            sWB[2 * o] = sW2[2 * (t * NB + yb)] * w3;
            sWB[2 * o + 1] = sW2[2 * (t * NB + yb) + 1] * w3;
          }
        }
        // sigma tables [tab][u][j3]: tab 0: v(k2,u)-v3, 1: -v(k2,u)-v3, 2: v(k1,u)-v3, 3: -v(k1,u)-v3
        for (int o = tid; o < 4 * NB2; o += nthr) {
          const int tab = o / NB2, u = (o / NB) % NB, j3 = o % NB;
          const double* vl = (tab < 2 ? sV2 : sV1) + 3 * u;
          const float sgn = (tab & 1) ? -1.0f : 1.0f;
          if (f32_sigma) {
            const float* vlh = (tab < 2 ? sVH2 : sVH1) + 3 * u;
            const float* vll = (tab < 2 ? sVL2 : sVL1) + 3 * u;
            sigma_entry_f32(a, vlh, vll, sgn, sVH3 + 3 * j3, sVL3 + 3 * j3, vl, sV3 + 3 * j3, sSigPM + o, sSigI + o);
            if constexpr (kF64) {
              // the FP64 Gaussian's 8/sigma and, with one temperature, (1/sigma) W3(j3), from 1/sqrt(|dv|^2) (CUDA's
              // rsqrt): the Gaussian's value needs 1/sigma to a few ulp, not the correctly rounded sigma that the
              // window's exact decisions use; delta := 1 is the prefilter's exact decision (inverse -1)
              double iv = -1.0;
              if (sSigI[o] >= 0.f) {
                const unsigned long long flip = sgn < 0.f ? 0x8000000000000000ULL : 0ULL;
                const double dx = __dsub_rn(__longlong_as_double(__double_as_longlong(vl[0]) ^ flip), sV3[3 * j3]);
                const double dy = __dsub_rn(__longlong_as_double(__double_as_longlong(vl[1]) ^ flip), sV3[3 * j3 + 1]);
                const double dz = __dsub_rn(__longlong_as_double(__double_as_longlong(vl[2]) ^ flip), sV3[3 * j3 + 2]);
                iv = rsqrt(fma(dx, dx, fma(dy, dy, dz * dz))) * inv_sbdq;
              }
              if constexpr (kDFC) {  // as double-floats in the same slots
                reinterpret_cast<float2*>(sSigW)[o] = df_make((iv >= 0.0 ? iv : kSqrtPi) * sW3[j3]);
                reinterpret_cast<float2*>(sSig)[2 * o + 1] = iv >= 0.0 ? df_make(8.0 * iv) : make_float2(-1.f, 0.f);
              } else {
                if (MAXT == 1) sSigW[o] = (iv >= 0.0 ? iv : kSqrtPi) * sW3[j3];
                sSig[2 * o + 1] = iv >= 0.0 ? 8.0 * iv : -1.0;
              }
            }
          } else {
            sigma_entry(a, vl, (double)sgn, sV3 + 3 * j3, sSig + 2 * o);
            sigma_f_from_exact(sSig + 2 * o, sSigPM + o, sSigI + o);
            if constexpr (kF64) {
              // the FP64 Gaussian takes (8 / sigma)^2 dw^2 = 64 x^2 and, with one temperature, the product
              // (1/sigma) W3(j3) of two of its factors
              const double inv = sSig[2 * o + 1];
              if constexpr (kDFC) {  // as double-floats in the same slots
                reinterpret_cast<float2*>(sSigW)[o] = df_make((inv >= 0.0 ? inv : kSqrtPi) * sW3[j3]);
                reinterpret_cast<float2*>(sSig)[2 * o + 1] = inv >= 0.0 ? df_make(8.0 * inv) : make_float2(-1.f, 0.f);
              } else {
                if (MAXT == 1) sSigW[o] = (inv >= 0.0 ? inv : kSqrtPi) * sW3[j3];
                sSig[2 * o + 1] = inv >= 0.0 ? 8.0 * inv : -1.0;
              }
            }
          }
        }
        if constexpr (kDF) {
          if (has_row && !unit) {
            // A row and T row in double-float
            float4 Ad[NB];
#pragma unroll
            for (int d = 0; d < NB; ++d) Ad[d] = make_float4(0.f, 0.f, 0.f, 0.f);
            const int ka = rc / 3, ga = rc % 3;
            const float4* psi_row = reinterpret_cast<const float4*>(sPsi) + (size_t)(rjj * NB + rj1) * G * 9 + ga * 3;
            const float4* twd = reinterpret_cast<const float4*>(sTw2);
            // one pass over the groups of atom ka with every l (see the FP64 form below)
            float4 cur[3] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                             make_float4(0.f, 0.f, 0.f, 0.f)};
            int la = 0, seg_end = sKLs[ka * NA + 1];
            auto put = [&]() {
#pragma unroll
              for (int l = 0; l < NA; ++l)
                if (l == la)
#pragma unroll
                  for (int th = 0; th < 3; ++th) Ad[3 * l + th] = cur[th];
#pragma unroll
              for (int th = 0; th < 3; ++th) cur[th] = make_float4(0.f, 0.f, 0.f, 0.f);
            };
            const int g_end = sKLs[ka * NA + NA];
            for (int gi = sKLs[ka * NA]; gi < g_end; ++gi) {
              while (gi >= seg_end) {
                put();
                seg_end = sKLs[ka * NA + (++la) + 1];
              }
              const int grp = sKLg[gi];
              const float4 tw = twd[grp];
              const float4* ps = psi_row + grp * 9;
#pragma unroll
              for (int th = 0; th < 3; ++th) cdf_mac(cur[th], tw, ps[th]);
            }
            put();
            const float4* e3d = reinterpret_cast<const float4*>(sE3);
            float4* trow = reinterpret_cast<float4*>(sT + (size_t)(rjj * NB + rj1) * (NB2 + 1) + rc * NB);
#pragma unroll
            for (int j3 = 0; j3 < NB; ++j3) {
              float4 sd = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
              for (int d = 0; d < NB; ++d) cdf_mac_conj(sd, Ad[d], e3d[j3 * NB + d]);
              trow[j3] = cdf_norm(sd);
            }
          }
        } else if (has_row && !unit) {
          // A row (jj, j1 = rj1, c = rc): d = (l, theta)
          C Arow[NB];
#pragma unroll
          for (int d = 0; d < NB; ++d) Arow[d] = cmk<R>(0, 0);
          const int ka = rc / 3, ga = rc % 3;
          const C* psi_row = sPsi + (size_t)(rjj * NB + rj1) * G * 9 + ga * 3;
          // one pass over the groups of atom ka with every l, which sit contiguously in l order: a lane's trip
          // count is the number of groups of its atom, so lanes of different ka (in the same warp) run about the
          // same count, where separate passes per l would each run the longest list of the warp. The running sum
          // of the current l moves into Arow when l changes (register moves only)
          C cur[3] = {cmk<R>(0, 0), cmk<R>(0, 0), cmk<R>(0, 0)};
          int la = 0, seg_end = sKLs[ka * NA + 1];
          auto put = [&]() {
#pragma unroll
            for (int l = 0; l < NA; ++l)
              if (l == la)
#pragma unroll
                for (int th = 0; th < 3; ++th) Arow[3 * l + th] = cur[th];
#pragma unroll
            for (int th = 0; th < 3; ++th) cur[th] = cmk<R>(0, 0);
          };
          const int g_end = sKLs[ka * NA + NA];
          for (int gi = sKLs[ka * NA]; gi < g_end; ++gi) {
            while (gi >= seg_end) {
              put();
              seg_end = sKLs[ka * NA + (++la) + 1];
            }
            const int grp = sKLg[gi];
            const C tw = sTw2[grp];
            const C* ps = psi_row + grp * 9;
#pragma unroll
            for (int th = 0; th < 3; ++th) cfma(cur[th], tw, ps[th]);
          }
          put();
          if constexpr (TC) {
            // A operand row tid (real part in K 0..5, imaginary in K 6..11), split into tf32 hi + lo
            unsigned char* Ah = tcbuf + (size_t)(tid >> 7) * 2 * kTcTile;
            const int r = tid & 127;
#pragma unroll
            for (int k = 0; k < 2 * NB; ++k) {
              const float x = k < NB ? (float)Arow[k].re : (float)Arow[k - NB].im;
              const float hi = tc::to_tf32(x);
              const uint32_t off = tc::kmajor_offset(r, k);
              *reinterpret_cast<float*>(Ah + off) = hi;
              *reinterpret_cast<float*>(Ah + kTcTile + off) = tc::to_tf32(x - hi);
            }
          } else {
            C* trow = sT + (size_t)(rjj * NB + rj1) * (NB2 + 1) + rc * NB;
#pragma unroll
            for (int j3 = 0; j3 < NB; ++j3) {
              C s = cmk<R>(0, 0);
#pragma unroll
              for (int d = 0; d < NB; ++d) cfma_conj(s, Arow[d], sE3[j3 * NB + d]);
              trow[j3] = s;
            }
          }
        }
        if constexpr (TC) {
          if (!unit) {
            // B operand: T = A conj(E3)^T as a real product; column n = 2 j3 (+1) gives Re (Im) of T[.][j3]
            unsigned char* Bh = tcbuf + kTcA;
            for (int o = tid; o < 2 * NB * 2 * NB; o += nthr) {
              const int n = o / (2 * NB), k = o % (2 * NB);
              const int j3 = n >> 1, d = k % NB;
              const C ev = sE3[j3 * NB + d];
              const bool im_col = n & 1, im_row = k >= NB;
              const float x = !im_col ? (!im_row ? (float)ev.re : (float)ev.im) : (!im_row ? -(float)ev.im : (float)ev.re);
              const float hi = tc::to_tf32(x);
              const uint32_t off = tc::kmajor_offset(n, k);
              *reinterpret_cast<float*>(Bh + off) = hi;
              *reinterpret_cast<float*>(Bh + 1024 + off) = tc::to_tf32(x - hi);
            }
            tc::fence_async_smem();
            __syncthreads();
            const bool live = s_tc_fail == 0;  // uniform: read after the barrier above
            if (tid == 0 && live) {
              tc::fence_after_sync();
              constexpr uint32_t idesc = tc::idesc_tf32(128, 16);
              const uint32_t b0 = tc::smem_u32(Bh);
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const uint32_t a0 = tc::smem_u32(tcbuf + (size_t)t * 2 * kTcTile);
                const uint32_t d = tmem_base + (uint32_t)(t * 16);
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {  // K = 16 in two steps of 8 (two core matrices, 256 bytes)
                  const uint32_t ko = (uint32_t)ks * 2u * tc::kLbo;
                  tc::mma_tf32(d, tc::make_desc(a0 + ko), tc::make_desc(b0 + ko), idesc, ks);
                  tc::mma_tf32(d, tc::make_desc(a0 + ko), tc::make_desc(b0 + 1024 + ko), idesc, 1);
                  tc::mma_tf32(d, tc::make_desc(a0 + (uint32_t)kTcTile + ko), tc::make_desc(b0 + ko), idesc, 1);
                }
              }
              tc::mma_commit(s_mbar);
            }
            const bool done = live && tc::mbar_wait(s_mbar, tc_phase, kTcMaxPolls);
            tc_phase ^= 1u;
            if (live && !done) {
              s_tc_fail = 1;
              if (lane == 0) atomicAdd(a.counts + 5, 1ULL);
            }
            tc::fence_after_sync();
            const int warp = tid >> 5;
            float v[16];
            tc::tmem_ld16(tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 16), v);
            if (has_row) {
              C* trow = sT + (size_t)(rjj * NB + rj1) * (NB2 + 1) + rc * NB;
#pragma unroll
              for (int j3 = 0; j3 < NB; ++j3) trow[j3] = cmk<R>(v[2 * j3], v[2 * j3 + 1]);
            }
            tc::fence_before_sync();
          }
        }
        __syncthreads();
        if constexpr (kF64) {
          // ---- phase 3 (FP64 path): every lane screens the window of its row (jj, x, y) for all j3; entries with
          // an accepted candidate enter a per-warp entry queue, whose entries the warp takes 32 at a time to form
          // W and to append their accepted terms to a per-warp term queue, evaluated 32 at a time: W, the
          // Gaussian and the Bose arithmetic run on full warps however unevenly the accepted terms fall on lanes
          const int x = rj1, y = rc;
          const int jq0 = active ? rjj : 0;
          const bool row_ok = active && sH1[x] != 0.f && sH2[y] != 0.f;
          // candidates 0..2: ordering A (q' = (k1,x), q'' = (k2,y)) ++, +-, --; 3..5: ordering B, swapped
          const unsigned cand = ((k1 != k2 && !unit) ? 0x3Fu : 0x07u) & a.cand_mask &
                                (a.nu_select == 0 ? 0x3Fu : a.nu_select == 1 ? ~s_umask : s_umask);
          const double w0 = sOm0[jq0];
          const float h0 = sHq[jq0];
          const float hx = sH1[x], hy = sH2[y];
          const float ap = h0 + hx, am = h0 - hx, bp = h0 + hy, bm = h0 - hy;
          const float apy = ap + hy, apm = ap - hy, amm = am - hy;
          const float bpx = bp + hx, bpm = bp - hx, bmm = bm - hx;
          const float s0 = (h0 + hx) + hy;
          if constexpr (MAXT == 1) {
            // the four distinct products c_p (1/(n0 w0)) x leg weights of this row, per candidate class
            // (++ both orderings, +- ordering A, +- ordering B, -- both orderings), read by any lane
            if (row_ok) {
              if constexpr (kDFC) {
                const float2* fq = reinterpret_cast<const float2*>(sWq + 3 * (jq0 * NB + x));
                const float2 a2 = reinterpret_cast<const float2*>(sW2)[2 * y];
                const float2 b2 = reinterpret_cast<const float2*>(sW2)[2 * y + 1];
                float2* wp = reinterpret_cast<float2*>(sWp + 4 * tid);
                wp[0] = df_mul(fq[0], a2);
                wp[1] = df_mul(fq[0], b2);
                wp[2] = df_mul(fq[1], a2);
                wp[3] = df_mul(fq[2], b2);
              } else {
                const double* fq = sWq + 3 * (jq0 * NB + x);
                const double a2 = sW2[2 * y], b2 = sW2[2 * y + 1];
                double* wp = sWp + 4 * tid;
                wp[0] = fq[0] * a2;
                wp[1] = fq[0] * b2;
                wp[2] = fq[1] * a2;
                wp[3] = fq[2] * b2;
              }
            }
          }
          const float2* PA0 = sSigPM + 0 * NB2 + y * NB;
          const float2* PA1 = sSigPM + 1 * NB2 + y * NB;
          const float2* PB0 = sSigPM + 2 * NB2 + x * NB;
          const float2* PB1 = sSigPM + 3 * NB2 + x * NB;
          int qh = 0, qn = 0;  // warp-uniform term-queue head and length
          int eh = 0, en = 0;  // warp-uniform entry-queue head and length
          // lanes take up to 32 queued entries: W of each, then its accepted candidates into the term queue,
          // which the warp evaluates 32 at a time
          auto run_entries = [&](int count) {
            unsigned ent = 0;
            if (lane < count) ent = (unsigned)sEQ[ebase + ((eh + lane) & (kEQCap - 1))];
            eh = (eh + count) & (kEQCap - 1);
            en -= count;
            QT W2;
            if constexpr (kDFC)
              W2 = make_float2(1.f, 0.f);
            else
              W2 = 1.0;
            if (ent && !unit) {
              ++nwf;
              const int ej3 = (ent >> 6) & 15, ey = (ent >> 10) & 15, ex = (ent >> 14) & 15, ejq = ent >> 18;
              if constexpr (kDF) {
                const float4* tbe = reinterpret_cast<const float4*>(sT + (size_t)(ejq * NB + ex) * (NB2 + 1) + ej3);
                const float4* e2 = reinterpret_cast<const float4*>(sE2 + ey * NB);
                float4 Wd = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int c = 0; c < NB; ++c) cdf_mac(Wd, e2[c], tbe[c * NB]);
                if constexpr (kDFC)
                  W2 = cdf_abs2_df(Wd);
                else
                  W2 = cdf_abs2(Wd);
              } else {
                const C* tbe = sT + (size_t)(ejq * NB + ex) * (NB2 + 1) + ej3;
                const C* e2 = sE2 + ey * NB;
                C Wv = cmk<R>(0, 0);
#pragma unroll
                for (int c = 0; c < NB; ++c) cfma(Wv, e2[c], tbe[c * NB]);
                W2 = Wv.re * Wv.re + Wv.im * Wv.im;
              }
            }
            unsigned m = ent & 63u;
            const int nmy = __popc(m);
            int incl = nmy;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int v = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= o) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            int pos = qn + incl - nmy;
            const int info0 = (int)(((ent >> 6) & 15) << 3 | ((ent >> 10) & 15) << 7 | ((ent >> 14) & 15) << 11 |
                                    (ent >> 18) << 15);
            while (m) {
              const int c = __ffs(m) - 1;
              m &= m - 1;
              if (pos < kQCap) {
                const int sl = (qh + pos) & (kQCap - 1);
                sQD[qbase + sl] = W2;
                sQI[qbase + sl] = info0 | c;
              } else {
                consume(W2, info0 | c);  // term queue full (rare): the producing lane evaluates the term
              }
              ++pos;
            }
            qn = min(qn + total, kQCap);
            __syncwarp();
            while (qn >= 32) {
              const int sl = (qh + lane) & (kQCap - 1);
              consume(sQD[qbase + sl], sQI[qbase + sl]);
              qh = (qh + 32) & (kQCap - 1);
              qn -= 32;
            }
            __syncwarp();
          };
#pragma unroll 1
          for (int j3 = 0; j3 < NB; ++j3) {
            const float h3 = sH3[j3];
            if (h3 == 0.f) continue;  // uniform: j3 and k2 are the same on all lanes
            unsigned accm = 0;
            if (row_ok) {
              const float sS = kRelS * (s0 + h3);
              const float2 a0 = PA0[j3], a1 = PA1[j3], b0 = PB0[j3], b1 = PB1[j3];
              unsigned band = 0;
              FP_WINDOW_TEST()
              cnt0 += row_mult * __popc(accm & 0x09u);
              cnt1 += row_mult * __popc(accm & 0x12u);
              cnt2 += row_mult * __popc(accm & 0x24u);
            }
            // entries with an accepted candidate, one per lane at most, in lane order
            const unsigned bal = __ballot_sync(0xffffffffu, accm != 0);
            if (accm) {
              const int pos = en + __popc(bal & ((1u << lane) - 1u));
              sEQ[ebase + ((eh + pos) & (kEQCap - 1))] = (int)(accm | (j3 << 6) | (y << 10) | (x << 14) | (jq0 << 18));
            }
            en += __popc(bal);
            __syncwarp();
            while (en >= 32) run_entries(32);
          }
          if (en > 0) run_entries(en);
          if (lane < qn) {
            const int sl = (qh + lane) & (kQCap - 1);
            consume(sQD[qbase + sl], sQI[qbase + sl]);
          }
          __syncwarp();
          if (((k2 - k2_first) & 63) == 63) flush_df();
        } else {
          // ---- phase 3 (FP32 path): window of the row (jj, x, y), W in registers where a candidate is accepted,
          // then Gaussian and Bose weights
          if (active) {
            const int x = rj1, y = rc;
            const double w0 = sOm0[rjj];
            const float h0 = sHq[rjj], l0 = sLq[rjj];
            const float hx = sH1[x], hy = sH2[y];
            // candidates 0..2: ordering A (q' = (k1,x), q'' = (k2,y)) ++, +-, --; 3..5: ordering B, swapped
            const unsigned cand = ((k1 != k2 && !unit) ? 0x3Fu : 0x07u) & a.cand_mask &
                                  (a.nu_select == 0 ? 0x3Fu : a.nu_select == 1 ? ~s_umask : s_umask);
            if (hx != 0.f && hy != 0.f) {
              const C* e2row = sE2 + y * NB;  // read from shared memory where W is formed
              const C* tb = sT + (size_t)(rjj * NB + x) * (NB2 + 1);
              const float ap = h0 + hx, am = h0 - hx, bp = h0 + hy, bm = h0 - hy;
              const float apy = ap + hy, apm = ap - hy, amm = am - hy;
              const float bpx = bp + hx, bpm = bp - hx, bmm = bm - hx;
              const float s0 = (h0 + hx) + hy;
              // one temperature: the four distinct products c_p (1/(n0 w0)) x leg weights of this row, per
              // candidate class (++ both orderings, +- ordering A, +- ordering B, -- both orderings)
              float wpp = 0.f, wpa = 0.f, wpb = 0.f, wmm = 0.f;
              if constexpr (MAXT == 1) {
                const float f0 = sF0[rjj], a1 = sF1[2 * x], b1 = sF1[2 * x + 1], a2 = sF2[2 * y], b2 = sF2[2 * y + 1];
                wpp = 0.5f * f0 * (a1 * a2);
                wpa = 0.5f * f0 * (a1 * b2);
                wpb = 0.5f * f0 * (a2 * b1);
                wmm = (1.0f / 6.0f) * f0 * (b1 * b2);
              }
              const float2* PA0 = sSigPM + 0 * NB2 + y * NB;
              const float2* PA1 = sSigPM + 1 * NB2 + y * NB;
              const float2* PB0 = sSigPM + 2 * NB2 + x * NB;
              const float2* PB1 = sSigPM + 3 * NB2 + x * NB;
#pragma unroll 1
              for (int j3 = 0; j3 < NB; ++j3) {
                const float h3 = sH3[j3];
                if (h3 == 0.f) continue;
                const float sS = kRelS * (s0 + h3);
                const float2 a0 = PA0[j3], a1 = PA1[j3], b0 = PB0[j3], b1 = PB1[j3];
                unsigned accm = 0, band = 0;
                FP_WINDOW_TEST()
                if (!accm) continue;
                cnt0 += row_mult * __popc(accm & 0x09u);
                cnt1 += row_mult * __popc(accm & 0x12u);
                cnt2 += row_mult * __popc(accm & 0x24u);
                C Wv = cmk<R>(unit ? 1 : 0, 0);
                if (!unit) {
                  ++nwf;
#pragma unroll
                  for (int c = 0; c < NB; ++c) cfma(Wv, e2row[c], tb[c * NB + j3]);
                }
                const float W2 = Wv.re * Wv.re + Wv.im * Wv.im;
                while (accm) {
                  const int c = __ffs(accm) - 1;
                  accm &= accm - 1;
                  const int p = c % 3;
                  const bool ordA = c < 3;
                  const int tab = (c < 3) ? (c == 0 ? 0 : 1) : (c == 3 ? 2 : 3);
                  const int ent = tab * NB2 + (ordA ? y : x) * NB + j3;
                  // Bose selectors: leg q' takes (1+n)/w unless --, leg q'' takes (1+n)/w only for ++
                  const int s1 = (p == 2) ? 1 : 0, s2 = (p == 0) ? 0 : 1;
                  const int i1 = ordA ? x : y, i2 = ordA ? y : x;
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
                  const float inv = sSigI[ent];
                  float delta = 1.0f;
                  if (inv >= 0.f) {
                    const float xx = dwf * inv;
                    delta = __expf(-xx * xx) * inv * (float)kInvSqrtPi;
                  }
                  if constexpr (MAXT == 1) {
                    const float wsel = (p == 0) ? wpp : (p == 2) ? wmm : ordA ? wpa : wpb;
                    const float term = (W2 * delta) * wsel * sF3[j3];
                    float s, e;
                    two_sum(acch[0][0], term, s, e);
                    acch[0][0] = s;
                    accl[0][0] += e;
                  } else {
                    const float base = ((p == 2) ? (1.0f / 6.0f) : 0.5f) * W2 * delta;
                    const float* fq1 = ordA ? sF1 : sF2;
                    const float* fq2 = ordA ? sF2 : sF1;
#pragma unroll
                    for (int t = 0; t < MAXT; ++t) {
                      if (t >= nT) break;
                      const float term = base * sF0[t * J + rjj] * fq1[2 * (t * NB + i1) + s1] *
                                         fq2[2 * (t * NB + i2) + s2] * sF3[t * NB + j3];
                      float s, e;
                      two_sum(acch[0][t], term, s, e);
                      acch[0][t] = s;
                      accl[0][t] += e;
                    }
                  }
                }
              }
            }
          }
        }
        __syncthreads();
      }
      flush_df();
    }
    // deterministic reduction. FP64: per-lane slot sums in shared memory, then for each j0 the lanes of the
    // warps that hold its rows, in lane order. FP32: per-row sums, then the rows of each j0 in order.
    if constexpr (kF64) {
#pragma unroll
      for (int sl = 0; sl < S; ++sl)
#pragma unroll
        for (int t = 0; t < MAXT; ++t) {
          if (t >= nT) break;
          sRed[((size_t)tid * S + sl) * nT + t] = acc[sl][t];
        }
    } else if (has_row) {
#pragma unroll
      for (int t = 0; t < MAXT; ++t) {
        if (t >= nT) break;
        sRed[(size_t)tid * nT + t] = (double)acch[0][t] + (double)accl[0][t];
      }
    }
    __syncthreads();
    for (int o = tid; o < J * nT; o += nthr) {
      const int jj = o / nT, t = o % nT;
      double sum = 0.0;
      if constexpr (kF64) {
        for (int w = (jj * NB2) >> 5; w <= ((jj + 1) * NB2 - 1) >> 5; ++w) {
          const int sl = jj - (w * 32) / NB2;
          for (int l = 0; l < 32 && w * 32 + l < nthr; ++l) sum += sRed[((size_t)(w * 32 + l) * S + sl) * nT + t];
        }
      } else {
        for (int r = 0; r < NB2; ++r) sum += sRed[(size_t)(jj * NB2 + r) * nT + t];
      }
      a.partial[(size_t)item * J * nT + o] = sum;
    }
    __syncthreads();
    // accepted terms this row evaluated (the weighted counts over the row's multiplicity)
    const unsigned nte = row_mult ? (unsigned)(((unsigned long long)cnt0 + cnt1 + cnt2) / row_mult) : 0u;
    if (a.item_counts) {
      // accepted terms per j0 of the item: the rows jj * nb^2 .. (jj + 1) * nb^2 - 1, in row order
      unsigned long long* sCnt = reinterpret_cast<unsigned long long*>(sRed);  // reuses the reduction buffer
      sCnt[tid] = nte;
      __syncthreads();
      for (int jj = tid; jj < J; jj += nthr) {
        unsigned long long sum = 0;
        for (int r = jj * NB2; r < (jj + 1) * NB2; ++r) sum += sCnt[r];
        a.item_counts[(size_t)item * J + jj] = sum;
      }
      __syncthreads();
    }
    // the item's counters into the launch totals: warp sums, one atomic per counter and warp
    unsigned long long c0 = cnt0, c1 = cnt1, c2 = cnt2, cw = nwf, ct = nte;
    for (int off = 16; off > 0; off >>= 1) {
      c0 += __shfl_down_sync(0xffffffffu, c0, off);
      c1 += __shfl_down_sync(0xffffffffu, c1, off);
      c2 += __shfl_down_sync(0xffffffffu, c2, off);
      cw += __shfl_down_sync(0xffffffffu, cw, off);
      ct += __shfl_down_sync(0xffffffffu, ct, off);
    }
    if (lane == 0) {
      if (c0) atomicAdd(a.counts + 0, c0);
      if (c1) atomicAdd(a.counts + 1, c1);
      if (c2) atomicAdd(a.counts + 2, c2);
      if (cw) atomicAdd(a.counts + 3, cw);
      if (ct) atomicAdd(a.counts + 4, ct);
    }
  }
  if constexpr (TC) {
    tc::fence_before_sync();
    __syncthreads();
    if ((tid >> 5) == 0) {
      tc::fence_after_sync();
      tc::tmem_dealloc(tmem_base, kTcCols);
    }
  }
}

}  // namespace
}  // namespace fp
