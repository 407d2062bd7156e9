// Learned four-phonon rates: phase-space features, a 3 x 128 tanh network trained on exact rates of a
// seeded subset of modes with hand-written FP32 kernels, held-out error per bin, and exact fallback.
//
// The paper has no learned component.  The network replaces exact evaluation only where its held-out
// error is below the tolerance; every mode it is trained or judged on keeps its exact rate.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fp_internal.cuh"

namespace fp {
namespace {

constexpr int kH = 128;  // hidden width

// ------------------------------------------------------------------------------------------------
// Three-phonon-like phase space (features): one warp per mode, FP64 window decisions in the order of
// the four-phonon path: q'' = q +- q', dw = (w +- w') - w'', sigma = sb |v(q',j') - v(q'',j'')| |dq|.
struct Phase3Args {
  int N, nb, nT, grid[3];
  const double* omega;
  const double* vel;
  const double* nbose;  // [nT][N*nb]
  double sb, window, sigma_min, dq;
  int dq_mode;
  double rec[9];
  double* p3;   // [N*nb]
  double* wp3;  // [nT][N*nb]
};

__device__ double sigma3(const Phase3Args& a, const double* v1, const double* v2, double* inv) {
  double dx = __dsub_rn(v1[0], v2[0]);
  double dy = __dsub_rn(v1[1], v2[1]);
  double dz = __dsub_rn(v1[2], v2[2]);
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
  *inv = small ? -1.0 : 1.0 / sigma;
  return __dmul_rn(a.window, small ? a.sigma_min : sigma);
}

__global__ void phase3_kernel(Phase3Args a) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nb = a.nb, N = a.N;
  if (warp >= N * nb) return;
  const int q = warp / nb;
  const double w = a.omega[warp];
  double p = 0.0, wp[kMaxT];
  for (int t = 0; t < kMaxT; ++t) wp[t] = 0.0;
  if (w > 0.0) {
    const int g[3] = {q / (a.grid[1] * a.grid[2]), (q / a.grid[2]) % a.grid[1], q % a.grid[2]};
    const long long per = (long long)N * nb * nb;
    for (long long idx = lane; idx < 2 * per; idx += 32) {
      const int pm = (int)(idx / per);
      const long long rem = idx % per;
      const int q1 = (int)(rem / (nb * nb));
      const int j1 = (int)((rem / nb) % nb), j2 = (int)(rem % nb);
      const int g1[3] = {q1 / (a.grid[1] * a.grid[2]), (q1 / a.grid[2]) % a.grid[1], q1 % a.grid[2]};
      int g2[3];
      for (int d = 0; d < 3; ++d) {
        int x = pm == 0 ? g[d] + g1[d] : g[d] - g1[d];
        x %= a.grid[d];
        g2[d] = x < 0 ? x + a.grid[d] : x;
      }
      const int q2 = (g2[0] * a.grid[1] + g2[1]) * a.grid[2] + g2[2];
      const double w1 = a.omega[q1 * nb + j1], w2 = a.omega[q2 * nb + j2];
      if (w1 == 0.0 || w2 == 0.0) continue;
      const double t1 = pm == 0 ? __dadd_rn(w, w1) : __dsub_rn(w, w1);
      const double dw = __dsub_rn(t1, w2);
      double inv;
      const double P = sigma3(a, a.vel + 3 * (q1 * nb + j1), a.vel + 3 * (q2 * nb + j2), &inv);
      if (!(fabs(dw) <= P)) continue;
      double delta = 1.0;
      if (inv >= 0.0) {
        const double x = dw * inv;
        delta = exp(-x * x) * inv * kInvSqrtPi;
      }
      p += (pm == 0 ? 1.0 : 0.5) * delta;
      for (int t = 0; t < a.nT; ++t) {
        const double n1 = a.nbose[(size_t)t * N * nb + q1 * nb + j1];
        const double n2 = a.nbose[(size_t)t * N * nb + q2 * nb + j2];
        const double B = pm == 0 ? (n1 - n2) : 0.5 * (n1 + n2 + 1.0);
        wp[t] += B * delta / (w * w1 * w2);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) p += __shfl_down_sync(0xffffffffu, p, off);
  for (int t = 0; t < kMaxT; ++t)
    for (int off = 16; off > 0; off >>= 1) wp[t] += __shfl_down_sync(0xffffffffu, wp[t], off);
  if (lane == 0) {
    a.p3[warp] = p / (double)N;
    for (int t = 0; t < a.nT; ++t) a.wp3[(size_t)t * N * nb + warp] = wp[t] / (double)N;
  }
}

// Bose occupations n[t][m] = 1/expm1(hbar w / kB T) (0 for zero frequency)
__global__ void bose_kernel(const double* omega, int nm, int nT, const double* T, double* n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nm * nT) return;
  const int t = i / nm, m = i % nm;
  const double w = omega[m];
  n[i] = w > 0.0 ? 1.0 / expm1(kHbar * w / (kBoltzmann * T[t])) : 0.0;
}

// ------------------------------------------------------------------------------------------------
// Features per (temperature, mode): [w/wmax, |v|/vmax, branch one-hot (nb), log(T/300), log n0,
// log P3, log WP3, cos and sin of 2 pi g_a / N_a (a = 1..3), log WP4 (sampled)] -> F = nb + 13 columns;
// rows r = t * N*nb + m.
__global__ void features_kernel(const double* omega, const double* vel, const double* nbose, const double* p3,
                                const double* wp3, const double* wp4, const double* T, int nm, int nb, int nT,
                                int g0, int g1n, int g2n, double wmax, double vmax, float* X) {
  const int F = nb + 13;
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nm * nT) return;
  const int t = r / nm, m = r % nm;
  const double w = omega[m];
  const double* v = vel + 3 * m;
  float* x = X + (size_t)r * F;
  x[0] = (float)(w / wmax);
  x[1] = (float)(sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / vmax);
  for (int j = 0; j < nb; ++j) x[2 + j] = (j == m % nb) ? 1.0f : 0.0f;
  x[2 + nb] = (float)log(T[t] / 300.0);
  x[3 + nb] = (float)log(nbose[r] + 1e-30);
  x[4 + nb] = (float)log(p3[m] + 1e-30);
  x[5 + nb] = (float)log(fabs(wp3[r]) + 1e-30);
  const int q = m / nb;
  const int g[3] = {q / (g1n * g2n), (q / g2n) % g1n, q % g2n};
  const int n[3] = {g0, g1n, g2n};
  for (int a = 0; a < 3; ++a) {
    double sv, cv;
    sincospi(2.0 * g[a] / n[a], &sv, &cv);
    x[6 + nb + 2 * a] = (float)cv;
    x[7 + nb + 2 * a] = (float)sv;
  }
  x[12 + nb] = (float)log(fabs(wp4[r]) + 1e-30);
}

// Features of the temperature sweep per (output temperature, mode): [log anchor rate (nA), log(T/300), log n0(T),
// w/wmax, branch one-hot (nb)] -> F = nA + 3 + nb columns; rows r = t * N*nb + m.
__global__ void sweep_features_kernel(const double* anchor, const double* omega, const double* T, int nm, int nb,
                                      int nT, int nA, double wmax, float* X) {
  const int F = nA + 3 + nb;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nm * nT) return;
  const int t = r / nm, m = r % nm;
  float* x = X + (size_t)r * F;
  for (int k = 0; k < nA; ++k) x[k] = (float)log(fmax(anchor[(size_t)k * nm + m], 1e-300));
  const double w = omega[m];
  x[nA] = (float)log(T[t] / 300.0);
  x[nA + 1] = (float)log((w > 0.0 ? 1.0 / expm1(kHbar * w / (kBoltzmann * T[t])) : 0.0) + 1e-30);
  x[nA + 2] = (float)(w / wmax);
  for (int j = 0; j < nb; ++j) x[nA + 3 + j] = (j == m % nb) ? 1.0f : 0.0f;
}

// column mean and standard deviation over the listed rows (one thread per column, fixed order)
__global__ void col_stats_kernel(const float* X, int F, const int* rows, int n, float* mean, float* stdv) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  double s = 0.0, s2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = X[(size_t)rows[i] * F + f];
    s += x;
    s2 += x * x;
  }
  const double mu = n > 0 ? s / n : 0.0;
  const double var = n > 0 ? s2 / n - mu * mu : 0.0;
  mean[f] = (float)mu;
  stdv[f] = (float)(var > 1e-12 ? sqrt(var) : 1.0);
}

__global__ void normalize_kernel(float* X, int F, long long n, const float* mean, const float* stdv) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * F) return;
  const int f = (int)(i % F);
  X[i] = (X[i] - mean[f]) / stdv[f];
}

// gather rows of X (and targets) for a minibatch
__global__ void gather_kernel(const float* X, int F, const int* rows, int n, float* out, const float* y,
                              float* yout) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * F) return;
  const int b = i / F, f = i % F;
  out[i] = X[(size_t)rows[b] * F + f];
  if (f == 0 && y) yout[b] = y[rows[b]];
}

// ------------------------------------------------------------------------------------------------
// FP32 network kernels.  C[M][N] = act(sum_k A(m,k) B(k,n) + bias[n]); A(m,k) = A[m*lda+k] or A[k*lda+m]
// (transA), B(k,n) = B[k*ldb+n] or B[n*ldb+k] (transB).  32x32 tiles, one output per thread, k in order
// (deterministic).
constexpr int kTile = 32;

__global__ void gemm_kernel(int M, int Nn, int K, const float* A, int lda, int transA, const float* B, int ldb,
                            int transB, float* C, int ldc, const float* bias, int act_tanh) {
  __shared__ float As[kTile][kTile + 1];
  __shared__ float Bs[kTile][kTile + 1];
  const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;  // 32 x 8 threads
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += kTile) {
    for (int r = ty; r < kTile; r += 8) {
      const int m = m0 + r, k = k0 + tx;
      As[r][tx] = (m < M && k < K) ? (transA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
      const int kk = k0 + r, n = n0 + tx;
      Bs[r][tx] = (kk < K && n < Nn) ? (transB ? B[(size_t)n * ldb + kk] : B[(size_t)kk * ldb + n]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTile; ++kk) {
      const float b = Bs[kk][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fmaf(As[ty + 8 * i][kk], b, acc[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 8 * i, n = n0 + tx;
    if (m < M && n < Nn) {
      float v = acc[i] + (bias ? bias[n] : 0.f);
      C[(size_t)m * ldc + n] = act_tanh ? tanhf(v) : v;
    }
  }
}

// dZ = dH * (1 - H^2) (in place on dH)
__global__ void tanh_back_kernel(float* dH, const float* H, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dH[i] *= (1.f - H[i] * H[i]);
}

// column sums (bias gradients), fixed order
__global__ void colsum_kernel(const float* Z, int rows, int cols, float* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += Z[(size_t)r * cols + c];
  out[c] = s;
}

// residual r = y - t, dy = 2 r / B, loss = mean r^2 (single block, fixed order)
__global__ void loss_kernel(const float* y, const float* t, int B, float* dy, float* loss) {
  __shared__ double part[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const float r = y[i] - t[i];
    dy[i] = 2.f * r / (float)B;
    s += (double)r * r;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < blockDim.x; ++i) tot += part[i];
    *loss = (float)(tot / B);
  }
}

// Adam (Kingma & Ba 2015) with bias correction
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void exp_kernel(const float* y, int n, const int* rows, int nm, double* rates_out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rates_out[rows[i]] = exp((double)y[i]);
}

size_t nparams(int F) { return (size_t)kH * F + kH + 2 * ((size_t)kH * kH + kH) + kH + 1; }

// Network workspace on the device (layout of the packed parameters: W1 b1 W2 b2 W3 b3 w4 b4).
struct Net {
  int F = 0, Bmax = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  float *X = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *y = nullptr, *t = nullptr, *dy = nullptr;
  float *D1 = nullptr, *D2 = nullptr, *D3 = nullptr, *loss = nullptr;
  float* W1() const { return p; }
  float* b1() const { return p + kH * F; }
  float* W2() const { return b1() + kH; }
  float* b2() const { return W2() + kH * kH; }
  float* W3() const { return b2() + kH; }
  float* b3() const { return W3() + kH * kH; }
  float* w4() const { return b3() + kH; }
  float* b4() const { return w4() + kH; }
};

cudaError_t gemm(cudaStream_t s, int M, int Nn, int K, const float* A, int lda, int tA, const float* B, int ldb,
                 int tB, float* C, int ldc, const float* bias, int act) {
  dim3 grid((Nn + kTile - 1) / kTile, (M + kTile - 1) / kTile);
  gemm_kernel<<<grid, 256, 0, s>>>(M, Nn, K, A, lda, tA, B, ldb, tB, C, ldc, bias, act);
  return cudaGetLastError();
}

// forward pass of B rows already in net.X; output in net.y
cudaError_t net_forward(const Net& n, int B, cudaStream_t s) {
  cudaError_t e;
  if ((e = gemm(s, B, kH, n.F, n.X, n.F, 0, n.W1(), n.F, 1, n.H1, kH, n.b1(), 1))) return e;
  if ((e = gemm(s, B, kH, kH, n.H1, kH, 0, n.W2(), kH, 1, n.H2, kH, n.b2(), 1))) return e;
  if ((e = gemm(s, B, kH, kH, n.H2, kH, 0, n.W3(), kH, 1, n.H3, kH, n.b3(), 1))) return e;
  return gemm(s, B, 1, kH, n.H3, kH, 0, n.w4(), 1, 0, n.y, 1, n.b4(), 0);
}

// loss and gradient of B rows (targets in net.t); gradient in net.g
cudaError_t net_backward(const Net& n, int B, cudaStream_t s) {
  cudaError_t e;
  const int F = n.F;
  float* g = n.g;
  float *gW1 = g, *gb1 = g + kH * F, *gW2 = gb1 + kH, *gb2 = gW2 + kH * kH, *gW3 = gb2 + kH,
        *gb3 = gW3 + kH * kH, *gw4 = gb3 + kH, *gb4 = gw4 + kH;
  loss_kernel<<<1, 256, 0, s>>>(n.y, n.t, B, n.dy, n.loss);
  // output layer: gw4 = H3^T dy, gb4 = sum dy, D3 = dy w4^T
  if ((e = gemm(s, kH, 1, B, n.H3, kH, 1, n.dy, 1, 0, gw4, 1, nullptr, 0))) return e;
  colsum_kernel<<<1, 32, 0, s>>>(n.dy, B, 1, gb4);
  if ((e = gemm(s, B, kH, 1, n.dy, 1, 0, n.w4(), kH, 0, n.D3, kH, nullptr, 0))) return e;
  const long long bh = (long long)B * kH;
  tanh_back_kernel<<<(unsigned)((bh + 255) / 256), 256, 0, s>>>(n.D3, n.H3, bh);
  if ((e = gemm(s, kH, kH, B, n.D3, kH, 1, n.H2, kH, 0, gW3, kH, nullptr, 0))) return e;
  colsum_kernel<<<(kH + 127) / 128, 128, 0, s>>>(n.D3, B, kH, gb3);
  if ((e = gemm(s, B, kH, kH, n.D3, kH, 0, n.W3(), kH, 0, n.D2, kH, nullptr, 0))) return e;
  tanh_back_kernel<<<(unsigned)((bh + 255) / 256), 256, 0, s>>>(n.D2, n.H2, bh);
  if ((e = gemm(s, kH, kH, B, n.D2, kH, 1, n.H1, kH, 0, gW2, kH, nullptr, 0))) return e;
  colsum_kernel<<<(kH + 127) / 128, 128, 0, s>>>(n.D2, B, kH, gb2);
  if ((e = gemm(s, B, kH, kH, n.D2, kH, 0, n.W2(), kH, 0, n.D1, kH, nullptr, 0))) return e;
  tanh_back_kernel<<<(unsigned)((bh + 255) / 256), 256, 0, s>>>(n.D1, n.H1, bh);
  if ((e = gemm(s, kH, F, B, n.D1, kH, 1, n.X, F, 0, gW1, F, nullptr, 0))) return e;
  colsum_kernel<<<(kH + 127) / 128, 128, 0, s>>>(n.D1, B, kH, gb1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  return cudaMalloc(reinterpret_cast<void**>(p), (n ? n : 1) * sizeof(T));
}

cudaError_t net_alloc(Net& n, int F, int Bmax) {
  n.F = F;
  n.Bmax = Bmax;
  const size_t P = nparams(F);
  cudaError_t e;
  if ((e = dalloc(&n.p, P)) || (e = dalloc(&n.g, P)) || (e = dalloc(&n.m, P)) || (e = dalloc(&n.v, P))) return e;
  if ((e = dalloc(&n.X, (size_t)Bmax * F)) || (e = dalloc(&n.H1, (size_t)Bmax * kH)) ||
      (e = dalloc(&n.H2, (size_t)Bmax * kH)) || (e = dalloc(&n.H3, (size_t)Bmax * kH)))
    return e;
  if ((e = dalloc(&n.y, Bmax)) || (e = dalloc(&n.t, Bmax)) || (e = dalloc(&n.dy, Bmax))) return e;
  if ((e = dalloc(&n.D1, (size_t)Bmax * kH)) || (e = dalloc(&n.D2, (size_t)Bmax * kH)) ||
      (e = dalloc(&n.D3, (size_t)Bmax * kH)) || (e = dalloc(&n.loss, 1)))
    return e;
  return cudaSuccess;
}

void net_free(Net& n) {
  float* ptrs[] = {n.p, n.g, n.m, n.v, n.X, n.H1, n.H2, n.H3, n.y, n.t, n.dy, n.D1, n.D2, n.D3, n.loss};
  for (float* q : ptrs)
    if (q) cudaFree(q);
  n = Net();
}

// SplitMix64 (Steele, Lea and Flood 2014): seeded, counter-based draws for subsets and initial weights
struct SplitMix64 {
  unsigned long long s;
  unsigned long long next() {
    unsigned long long z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
  double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Glorot-uniform weights, zero biases
std::vector<float> init_params(int F, unsigned long long seed) {
  std::vector<float> p(nparams(F), 0.f);
  SplitMix64 r{seed ^ 0x5DEECE66DULL};
  size_t o = 0;
  auto fill = [&](int fan_in, int fan_out) {
    const double lim = std::sqrt(6.0 / (fan_in + fan_out));
    for (int i = 0; i < fan_in * fan_out; ++i) p[o++] = (float)((2.0 * r.uniform() - 1.0) * lim);
    o += (fan_out > 1 ? fan_out : 0);
  };
  fill(F, kH);
  fill(kH, kH);
  fill(kH, kH);
  const double lim = std::sqrt(6.0 / (kH + 1));
  for (int i = 0; i < kH; ++i) p[o++] = (float)((2.0 * r.uniform() - 1.0) * lim);
  return p;
}

// The pairs {q, -q} of the grid with all their positive-frequency branches (mode indices q * nb + j), one entry per
// pair, by smallest q.  Subsets are drawn in these units because the rate path evaluates a pair at once (time
// reversal), so the exact share of the cost is the share of pairs drawn.
std::vector<std::vector<int>> pair_units(const int grid[3], int nb, const std::vector<double>& om) {
  const int N = grid[0] * grid[1] * grid[2];
  std::vector<std::vector<int>> units;
  std::vector<char> seen(N, 0);
  for (int q = 0; q < N; ++q) {
    if (seen[q]) continue;
    const int g0 = q / (grid[1] * grid[2]), g1 = (q / grid[2]) % grid[1], g2 = q % grid[2];
    const int p = (((grid[0] - g0) % grid[0]) * grid[1] + (grid[1] - g1) % grid[1]) * grid[2] +
                  (grid[2] - g2) % grid[2];
    seen[q] = seen[p] = 1;
    std::vector<int> u;
    const int members[2] = {q, p};
    for (int k = 0; k < (p == q ? 1 : 2); ++k)
      for (int j = 0; j < nb; ++j)
        if (om[(size_t)members[k] * nb + j] > 0.0) u.push_back(members[k] * nb + j);
    if (!u.empty()) units.push_back(u);
  }
  return units;
}

}  // namespace
}  // namespace fp

// ------------------------------------------------------------------------------------------------
// C-ABI
namespace {
int sfail(fp_ctx* c, int code, const std::string& m) {
  if (c) c->err = m;
  return code;
}
}  // namespace

#define SG_CUDA(ctx, call)                                                                                     \
  do {                                                                                                         \
    cudaError_t e_ = (call);                                                                                   \
    if (e_ != cudaSuccess)                                                                                     \
      return sfail((ctx), e_ == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA,                              \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                                        \
  } while (0)

extern "C" int fp_phase3(fp_ctx* c, int nT, const double* T, double sb, const fp_rates_opts* user, double* p3,
                         double* wp3) {
  using namespace fp;
  if (!c) return FP_EINVAL;
  if (!c->have_modes) return sfail(c, FP_ESTATE, "fp_phase3: call fp_modes or fp_set_modes first");
  if (nT < 1 || nT > kMaxT || !T) return sfail(c, FP_EINVAL, "fp_phase3: nT must be in [1, 8]");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0)) return sfail(c, FP_EINVAL, "fp_phase3: temperatures must be > 0");
  if (!(sb > 0.0)) return sfail(c, FP_EINVAL, "fp_phase3: scalebroad must be > 0");
  fp_rates_opts o;
  fp_default_opts(&o);
  if (user) {
    o = *user;
    if (o.window == 0.0) o.window = 2.0;
    if (o.sigma_min == 0.0) o.sigma_min = 1e-10;
  }
  SG_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int nm = c->N * c->nb;
  double *dT = nullptr, *dn = nullptr, *dp = nullptr, *dw = nullptr;
  SG_CUDA(c, dalloc(&dT, kMaxT));
  SG_CUDA(c, dalloc(&dn, (size_t)nm * nT));
  SG_CUDA(c, dalloc(&dp, nm));
  SG_CUDA(c, dalloc(&dw, (size_t)nm * nT));
  SG_CUDA(c, cudaMemcpyAsync(dT, T, nT * sizeof(double), cudaMemcpyHostToDevice, s));
  bose_kernel<<<(nm * nT + 255) / 256, 256, 0, s>>>(c->d_omega, nm, nT, dT, dn);
  Phase3Args a;
  a.N = c->N;
  a.nb = c->nb;
  a.nT = nT;
  for (int d = 0; d < 3; ++d) a.grid[d] = c->grid[d];
  a.omega = c->d_omega;
  a.vel = c->d_vel;
  a.nbose = dn;
  a.sb = sb;
  a.window = o.window;
  a.sigma_min = o.sigma_min;
  const double* B = c->rec;
  const double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6]);
  a.dq = std::cbrt(std::fabs(detB) / (double)c->N);
  a.dq_mode = o.dq_mode;
  for (int i = 0; i < 9; ++i) a.rec[i] = B[i];
  a.p3 = dp;
  a.wp3 = dw;
  phase3_kernel<<<(nm * 32 + 255) / 256, 256, 0, s>>>(a);
  SG_CUDA(c, cudaGetLastError());
  if (p3) SG_CUDA(c, cudaMemcpyAsync(p3, dp, nm * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (wp3) SG_CUDA(c, cudaMemcpyAsync(wp3, dw, (size_t)nm * nT * sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_CUDA(c, cudaStreamSynchronize(s));
  cudaFree(dT);
  cudaFree(dn);
  cudaFree(dp);
  cudaFree(dw);
  return FP_OK;
}

extern "C" int fp_phase4(fp_ctx* c, int nT, const double* T, double sb, int stride, double* wp4) {
  using namespace fp;
  if (!c) return FP_EINVAL;
  if (!c->have_modes) return sfail(c, FP_ESTATE, "fp_phase4: call fp_modes or fp_set_modes first");
  if (nT < 1 || nT > kMaxT || !T) return sfail(c, FP_EINVAL, "fp_phase4: nT must be in [1, 8]");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0)) return sfail(c, FP_EINVAL, "fp_phase4: temperatures must be > 0");
  if (!(sb > 0.0) || stride < 1 || stride > c->N) return sfail(c, FP_EINVAL, "fp_phase4: bad scalebroad or stride");
  if (!wp4) return sfail(c, FP_EINVAL, "fp_phase4: NULL output");
  SG_CUDA(c, cudaSetDevice(c->device));
  const size_t n = (size_t)nT * c->N * c->nb;
  double* d = nullptr;
  SG_CUDA(c, dalloc(&d, n));
  std::string err;
  int rc = phase4_sampled(c, nT, T, sb, stride, d, &err);
  if (rc) {
    cudaFree(d);
    return sfail(c, rc, "fp_phase4: " + err);
  }
  cudaError_t e = cudaMemcpy(wp4, d, n * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return sfail(c, FP_ECUDA, std::string("fp_phase4: ") + cudaGetErrorString(e));
  return FP_OK;
}

extern "C" int fp_mlp_loss_grad(int device, int n_in, int batch, const float* X, const float* y,
                                const float* params, float* grad, float* loss) {
  using namespace fp;
  if (n_in < 1 || batch < 1 || !X || !y || !params || !grad || !loss) return FP_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return FP_ECUDA;
  Net n;
  if (net_alloc(n, n_in, batch) != cudaSuccess) {
    net_free(n);
    return FP_ENOMEM;
  }
  const size_t P = nparams(n_in);
  cudaStream_t s = nullptr;
  int rc = FP_OK;
  if (cudaMemcpy(n.p, params, P * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(n.X, X, (size_t)batch * n_in * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(n.t, y, batch * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      net_forward(n, batch, s) != cudaSuccess || net_backward(n, batch, s) != cudaSuccess ||
      cudaMemcpy(grad, n.g, P * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(loss, n.loss, sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = FP_ECUDA;
  net_free(n);
  return rc;
}

extern "C" int fp_mlp_params_size(int n_in) { return (int)fp::nparams(n_in); }

#include <chrono>

namespace {
double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}
}  // namespace

extern "C" void fp_surrogate_default_opts(fp_surrogate_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->train_frac = 0.10;
  o->holdout_frac = 0.05;
  o->tol = 0.05;
  o->seed = 2104;
  o->epochs = 400;
  o->batch = 1024;
  o->lr = 2e-3;
  o->precision = FP_PREC_MIXED;
}

extern "C" int fp_surrogate_fit(fp_ctx* c, int nT, const double* T, double sb, const fp_surrogate_opts* user,
                                fp_surrogate_report* rep) {
  using namespace fp;
  if (!c) return FP_EINVAL;
  fp_surrogate_opts so;
  fp_surrogate_default_opts(&so);
  if (user) so = *user;
  if (!c->have_modes) return sfail(c, FP_ESTATE, "fp_surrogate_fit: call fp_modes or fp_set_modes first");
  if (nT < 1 || nT > kMaxT || !T) return sfail(c, FP_EINVAL, "fp_surrogate_fit: nT must be in [1, 8]");
  if (!(so.train_frac > 0.0) || !(so.holdout_frac > 0.0) || so.train_frac + so.holdout_frac > 1.0 ||
      !(so.tol > 0.0) || so.epochs < 1 || so.batch < 1 || !(so.lr > 0.0))
    return sfail(c, FP_EINVAL, "fp_surrogate_fit: bad options");
  const double t_start = now_ms();
  SG_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int nb = c->nb, nm = c->N * nb, F = nb + 13;
  const size_t rows_all = (size_t)nm * nT;

  // modes with positive frequency
  std::vector<double> om(nm);
  SG_CUDA(c, cudaMemcpyAsync(om.data(), c->d_omega, nm * sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_CUDA(c, cudaStreamSynchronize(s));
  std::vector<int> pos;
  for (int m = 0; m < nm; ++m)
    if (om[m] > 0.0) pos.push_back(m);
  // training and held-out modes: whole pairs {q, -q} with all their branches
  std::vector<std::vector<int>> units = fp::pair_units(c->grid, nb, om);
  SplitMix64 rng{so.seed};
  for (size_t i = units.size(); i > 1; --i) std::swap(units[i - 1], units[rng.next() % i]);
  const int u_train = std::max(1, (int)std::ceil(so.train_frac * units.size()));
  const int u_hold = std::max(1, (int)std::ceil(so.holdout_frac * units.size()));
  if (u_train + u_hold > (int)units.size()) return sfail(c, FP_EINVAL, "fp_surrogate_fit: too few modes");
  std::vector<unsigned char> role(nm, 0);  // 1 train, 2 holdout, 3 fallback
  int n_train = 0, n_hold = 0;
  for (int i = 0; i < u_train + u_hold; ++i)
    for (int m : units[i]) {
      role[m] = i < u_train ? 1 : 2;
      (i < u_train ? n_train : n_hold) += 1;
    }

  // exact rates of the training and held-out modes (one batched evaluation for all temperatures)
  double t0 = now_ms();
  std::vector<unsigned char> mask(nm, 0);
  for (int m = 0; m < nm; ++m) mask[m] = role[m] ? 1 : 0;
  fp_rates_opts ro;
  fp_default_opts(&ro);
  ro.precision = so.precision;
  ro.mode_mask = mask.data();
  std::vector<double> exact(rows_all, 0.0);
  int rc = fp_rates4(c, nT, T, sb, &ro, exact.data(), nullptr);
  if (rc) return rc;
  const double ms_exact = now_ms() - t0;

  // features for every (temperature, mode)
  t0 = now_ms();
  double *dT = nullptr, *dn = nullptr, *dp3 = nullptr, *dwp3 = nullptr, *dwp4 = nullptr;
  float *dX = nullptr, *dY = nullptr, *dmean = nullptr, *dstd = nullptr;
  int* drows = nullptr;
  std::vector<int> train_rows;
  for (int m = 0; m < nm; ++m)
    if (role[m] == 1)
      for (int t = 0; t < nT; ++t)
        if (exact[(size_t)t * nm + m] > 0.0) train_rows.push_back(t * nm + m);
  if (train_rows.empty()) return sfail(c, FP_EINVAL, "fp_surrogate_fit: no training rates > 0");
  Net net;
  auto cleanup = [&]() {
    cudaFree(dT);
    cudaFree(dn);
    cudaFree(dp3);
    cudaFree(dwp3);
    cudaFree(dwp4);
    cudaFree(dX);
    cudaFree(dY);
    cudaFree(dmean);
    cudaFree(dstd);
    cudaFree(drows);
    net_free(net);
  };
#define SG_TRY(call)                                                                                          \
  do {                                                                                                        \
    cudaError_t e_ = (call);                                                                                  \
    if (e_ != cudaSuccess) {                                                                                  \
      cleanup();                                                                                              \
      return sfail(c, e_ == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA,                                 \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                                       \
    }                                                                                                         \
  } while (0)
  const int Bmax = std::max(so.batch, 4096);
  SG_TRY(dalloc(&dT, kMaxT));
  SG_TRY(dalloc(&dn, rows_all));
  SG_TRY(dalloc(&dp3, (size_t)nm));
  SG_TRY(dalloc(&dwp3, rows_all));
  SG_TRY(dalloc(&dwp4, rows_all));
  SG_TRY(dalloc(&dX, rows_all * F));
  SG_TRY(dalloc(&dY, rows_all));
  SG_TRY(dalloc(&dmean, F));
  SG_TRY(dalloc(&dstd, F));
  SG_TRY(dalloc(&drows, std::max(rows_all, (size_t)Bmax)));
  SG_TRY(net_alloc(net, F, Bmax));
  SG_TRY(cudaMemcpyAsync(dT, T, nT * sizeof(double), cudaMemcpyHostToDevice, s));
  bose_kernel<<<(unsigned)((rows_all + 255) / 256), 256, 0, s>>>(c->d_omega, nm, nT, dT, dn);
  {
    Phase3Args a;
    a.N = c->N;
    a.nb = nb;
    a.nT = nT;
    for (int d = 0; d < 3; ++d) a.grid[d] = c->grid[d];
    a.omega = c->d_omega;
    a.vel = c->d_vel;
    a.nbose = dn;
    a.sb = sb;
    a.window = 2.0;
    a.sigma_min = 1e-10;
    const double* B = c->rec;
    const double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                        B[2] * (B[3] * B[7] - B[4] * B[6]);
    a.dq = std::cbrt(std::fabs(detB) / (double)c->N);
    a.dq_mode = 0;
    for (int i = 0; i < 9; ++i) a.rec[i] = B[i];
    a.p3 = dp3;
    a.wp3 = dwp3;
    phase3_kernel<<<(unsigned)(((size_t)nm * 32 + 255) / 256), 256, 0, s>>>(a);
    SG_TRY(cudaGetLastError());
  }
  {
    // sampled four-phonon weighted phase space: q' on a stride giving about 1/16 of the ordered pairs
    const int stride = std::max(1, c->N / 32);
    std::string perr;
    const int prc = phase4_sampled(c, nT, T, sb, stride, dwp4, &perr);
    if (prc) {
      cleanup();
      return sfail(c, prc, "fp_surrogate_fit: " + perr);
    }
  }
  double wmax = 0.0;
  for (double w : om) wmax = std::max(wmax, w);
  std::vector<double> vel((size_t)nm * 3);
  SG_TRY(cudaMemcpyAsync(vel.data(), c->d_vel, vel.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_TRY(cudaStreamSynchronize(s));
  double vmax = 1e-30;
  for (int m = 0; m < nm; ++m)
    vmax = std::max(vmax, std::sqrt(vel[3 * m] * vel[3 * m] + vel[3 * m + 1] * vel[3 * m + 1] +
                                    vel[3 * m + 2] * vel[3 * m + 2]));
  features_kernel<<<(unsigned)((rows_all + 255) / 256), 256, 0, s>>>(c->d_omega, c->d_vel, dn, dp3, dwp3, dwp4, dT,
                                                                     nm, nb, nT, c->grid[0], c->grid[1], c->grid[2],
                                                                     wmax, vmax, dX);
  SG_TRY(cudaMemcpyAsync(drows, train_rows.data(), train_rows.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  col_stats_kernel<<<1, 64, 0, s>>>(dX, F, drows, (int)train_rows.size(), dmean, dstd);
  normalize_kernel<<<(unsigned)((rows_all * F + 255) / 256), 256, 0, s>>>(dX, F, (long long)rows_all, dmean, dstd);
  std::vector<float> y(rows_all, 0.f);
  for (size_t r = 0; r < rows_all; ++r)
    if (exact[r] > 0.0) y[r] = (float)std::log(exact[r]);
  SG_TRY(cudaMemcpyAsync(dY, y.data(), rows_all * sizeof(float), cudaMemcpyHostToDevice, s));
  SG_TRY(cudaStreamSynchronize(s));
  const double ms_features = now_ms() - t0;

  // training: Adam on minibatches, rows reshuffled every epoch
  t0 = now_ms();
  {
    std::vector<float> p0 = init_params(F, so.seed);
    SG_TRY(cudaMemcpyAsync(net.p, p0.data(), p0.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    SG_TRY(cudaMemsetAsync(net.m, 0, p0.size() * sizeof(float), s));
    SG_TRY(cudaMemsetAsync(net.v, 0, p0.size() * sizeof(float), s));
  }
  const int P = (int)nparams(F);
  const int nrows = (int)train_rows.size();
  // at least 8 minibatches per epoch, so that small training sets still get enough Adam steps
  const int B = std::max(1, std::min(so.batch, std::max(32, nrows / 8)));
  std::vector<int> order(train_rows);
  int step = 0;
  const float b1 = 0.9f, b2 = 0.999f;
  for (int ep = 0; ep < so.epochs; ++ep) {
    for (size_t i = order.size(); i > 1; --i) std::swap(order[i - 1], order[rng.next() % i]);
    SG_TRY(cudaMemcpyAsync(drows, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int b0 = 0; b0 + B <= nrows; b0 += B) {
      gather_kernel<<<(B * F + 255) / 256, 256, 0, s>>>(dX, F, drows + b0, B, net.X, dY, net.t);
      SG_TRY(net_forward(net, B, s));
      SG_TRY(net_backward(net, B, s));
      ++step;
      const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
      adam_kernel<<<(P + 255) / 256, 256, 0, s>>>(net.p, net.g, net.m, net.v, P, (float)so.lr, b1, b2, 1e-8f, c1, c2);
    }
  }
  float final_loss = 0.f;
  SG_TRY(cudaMemcpyAsync(&final_loss, net.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  SG_TRY(cudaStreamSynchronize(s));
  const double ms_train = now_ms() - t0;

  // prediction for every (temperature, mode) row
  t0 = now_ms();
  double* dpred = nullptr;
  SG_TRY(dalloc(&dpred, rows_all));
  std::vector<int> all(rows_all);
  std::iota(all.begin(), all.end(), 0);
  SG_TRY(cudaMemcpyAsync(drows, all.data(), rows_all * sizeof(int), cudaMemcpyHostToDevice, s));
  for (size_t r0 = 0; r0 < rows_all; r0 += Bmax) {
    const int nb_rows = (int)std::min((size_t)Bmax, rows_all - r0);
    gather_kernel<<<(nb_rows * F + 255) / 256, 256, 0, s>>>(dX, F, drows + r0, nb_rows, net.X, nullptr, nullptr);
    SG_TRY(net_forward(net, nb_rows, s));
    exp_kernel<<<(nb_rows + 255) / 256, 256, 0, s>>>(net.y, nb_rows, drows + r0, (int)rows_all, dpred);
  }
  std::vector<double> pred(rows_all);
  SG_TRY(cudaMemcpyAsync(pred.data(), dpred, rows_all * sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_TRY(cudaStreamSynchronize(s));
  cudaFree(dpred);
  const double ms_predict = now_ms() - t0;

  // held-out error per bin (branch x frequency quartile); bins above tol fall back to exact rates
  std::vector<double> wsorted;
  for (int m : pos) wsorted.push_back(om[m]);
  std::sort(wsorted.begin(), wsorted.end());
  double qcut[3];
  for (int k = 0; k < 3; ++k) qcut[k] = wsorted[(size_t)((k + 1) * wsorted.size() / 4)];
  auto bin_of = [&](int m) {
    int qb = 0;
    while (qb < 3 && om[m] >= qcut[qb]) ++qb;
    return (m % nb) * 4 + qb;
  };
  const int nbins = nb * 4;
  std::vector<double> bin_err(nbins, 0.0), bin_err2(nbins, 0.0);
  std::vector<int> bin_cnt(nbins, 0);
  std::vector<double> errs;
  for (int m = 0; m < nm; ++m) {
    if (role[m] != 2) continue;
    for (int t = 0; t < nT; ++t) {
      const size_t r = (size_t)t * nm + m;
      if (!(exact[r] > 0.0)) continue;
      const double e = std::fabs(pred[r] - exact[r]) / exact[r];
      errs.push_back(e);
      bin_err[bin_of(m)] += e;
      bin_err2[bin_of(m)] += e * e;
      bin_cnt[bin_of(m)] += 1;
    }
  }
  int n_bins_fb = 0;
  std::vector<unsigned char> bin_fb(nbins, 0);
  // a bin stays on the network only when it has at least 16 held-out rows and the upper confidence bound
  // (mean + 2 standard errors) of their relative error is within the tolerance
  for (int b = 0; b < nbins; ++b) {
    double e = 1e30;
    if (bin_cnt[b] >= 16) {
      const double n = bin_cnt[b], mu = bin_err[b] / n;
      const double var = std::max(0.0, bin_err2[b] / n - mu * mu);
      e = mu + 2.0 * std::sqrt(var / n);
    }
    if (e > so.tol) {
      bin_fb[b] = 1;
      ++n_bins_fb;
    }
  }
  t0 = now_ms();
  std::fill(mask.begin(), mask.end(), 0);
  int n_fb = 0;
  for (int m : pos)
    if (!role[m] && bin_fb[bin_of(m)]) {
      mask[m] = 1;
      role[m] = 3;
      ++n_fb;
    }
  std::vector<double> fb(rows_all, 0.0);
  if (n_fb) {
    ro.mode_mask = mask.data();
    rc = fp_rates4(c, nT, T, sb, &ro, fb.data(), nullptr);
    if (rc) {
      cleanup();
      return rc;
    }
  }
  const double ms_fallback = now_ms() - t0;

  c->sur_nT = nT;
  c->sur_rates.assign(rows_all, 0.0);
  c->sur_used.assign(rows_all, 1);
  for (int m = 0; m < nm; ++m) {
    for (int t = 0; t < nT; ++t) {
      const size_t r = (size_t)t * nm + m;
      if (!(om[m] > 0.0)) {
        c->sur_rates[r] = 0.0;
      } else if (role[m] == 1 || role[m] == 2) {
        c->sur_rates[r] = exact[r];
      } else if (role[m] == 3) {
        c->sur_rates[r] = fb[r];
      } else {
        c->sur_rates[r] = pred[r];
        c->sur_used[r] = 0;
      }
    }
  }
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->n_modes = (int)pos.size();
    rep->n_train = n_train;
    rep->n_holdout = n_hold;
    rep->n_fallback_modes = n_fb;
    rep->n_bins = nbins;
    rep->n_bins_fallback = n_bins_fb;
    rep->final_loss = final_loss;
    std::sort(errs.begin(), errs.end());
    if (!errs.empty()) {
      rep->holdout_median_rel_err = errs[errs.size() / 2];
      rep->holdout_p90_rel_err = errs[(size_t)(0.9 * (errs.size() - 1))];
      rep->holdout_max_rel_err = errs.back();
    }
    rep->ms_exact = ms_exact;
    rep->ms_features = ms_features;
    rep->ms_train = ms_train;
    rep->ms_predict = ms_predict;
    rep->ms_fallback = ms_fallback;
    rep->ms_total = now_ms() - t_start;
  }
  cleanup();
#undef SG_TRY
  return FP_OK;
}

extern "C" int fp_surrogate_rates(fp_ctx* c, double* rates, unsigned char* used_exact) {
  if (!c) return FP_EINVAL;
  if (c->sur_nT == 0) return sfail(c, FP_ESTATE, "fp_surrogate_rates: call fp_surrogate_fit first");
  if (rates) std::memcpy(rates, c->sur_rates.data(), c->sur_rates.size() * sizeof(double));
  if (used_exact) std::memcpy(used_exact, c->sur_used.data(), c->sur_used.size());
  return FP_OK;
}

// ------------------------------------------------------------------------------------------------
// Learned rates at new temperatures (fp_surrogate_sweep)
extern "C" int fp_surrogate_sweep(fp_ctx* c, int nA, const double* TA, int nT, const double* T, double sb,
                                  const fp_surrogate_opts* user, double* rates, unsigned char* used_exact,
                                  fp_surrogate_report* rep) {
  using namespace fp;
  if (!c) return FP_EINVAL;
  fp_surrogate_opts so;
  fp_surrogate_default_opts(&so);
  if (user) so = *user;
  if (!c->have_modes) return sfail(c, FP_ESTATE, "fp_surrogate_sweep: call fp_modes or fp_set_modes first");
  if (nA < 1 || nA > kMaxT || !TA) return sfail(c, FP_EINVAL, "fp_surrogate_sweep: nA must be in [1, 8]");
  if (nT < 1 || nT > 64 || !T) return sfail(c, FP_EINVAL, "fp_surrogate_sweep: nT must be in [1, 64]");
  for (int i = 0; i < nA; ++i)
    if (!(TA[i] > 0.0) || !std::isfinite(TA[i])) return sfail(c, FP_EINVAL, "fp_surrogate_sweep: temperatures > 0");
  for (int i = 0; i < nT; ++i)
    if (!(T[i] > 0.0) || !std::isfinite(T[i])) return sfail(c, FP_EINVAL, "fp_surrogate_sweep: temperatures > 0");
  if (!(so.train_frac > 0.0) || !(so.holdout_frac > 0.0) || so.train_frac + so.holdout_frac > 1.0 ||
      !(so.tol > 0.0) || so.epochs < 1 || so.batch < 1 || !(so.lr > 0.0))
    return sfail(c, FP_EINVAL, "fp_surrogate_sweep: bad options");
  const double t_start = now_ms();
  SG_CUDA(c, cudaSetDevice(c->device));
  cudaStream_t s = c->stream;
  const int nb = c->nb, nm = c->N * nb, F = nA + 3 + nb;
  const size_t rows_all = (size_t)nm * nT;

  std::vector<double> om(nm);
  SG_CUDA(c, cudaMemcpyAsync(om.data(), c->d_omega, nm * sizeof(double), cudaMemcpyDeviceToHost, s));
  SG_CUDA(c, cudaStreamSynchronize(s));
  std::vector<int> pos;
  for (int m = 0; m < nm; ++m)
    if (om[m] > 0.0) pos.push_back(m);
  // training and held-out modes: whole pairs {q, -q} with all their branches
  std::vector<std::vector<int>> units = fp::pair_units(c->grid, nb, om);
  SplitMix64 rng{so.seed};
  for (size_t i = units.size(); i > 1; --i) std::swap(units[i - 1], units[rng.next() % i]);
  const int u_train = std::max(1, (int)std::ceil(so.train_frac * units.size()));
  const int u_hold = std::max(1, (int)std::ceil(so.holdout_frac * units.size()));
  if (u_train + u_hold > (int)units.size()) return sfail(c, FP_EINVAL, "fp_surrogate_sweep: too few modes");
  std::vector<unsigned char> role(nm, 0);  // 1 train, 2 holdout, 3 fallback
  int n_train = 0, n_hold = 0;
  for (int i = 0; i < u_train + u_hold; ++i)
    for (int m : units[i]) {
      role[m] = i < u_train ? 1 : 2;
      (i < u_train ? n_train : n_hold) += 1;
    }

  // exact rates: every mode at the anchors; the training and held-out modes at the output temperatures
  double t0 = now_ms();
  fp_rates_opts ro;
  fp_default_opts(&ro);
  ro.precision = so.precision;
  std::vector<double> anchor((size_t)nA * nm);
  int rc = fp_rates4(c, nA, TA, sb, &ro, anchor.data(), nullptr);
  if (rc) return rc;
  auto exact_at = [&](const std::vector<unsigned char>& mk, std::vector<double>& dst) -> int {
    std::vector<double> tmp((size_t)kMaxT * nm);
    fp_rates_opts o = ro;
    o.mode_mask = mk.data();
    for (int t0b = 0; t0b < nT; t0b += kMaxT) {
      const int nc = std::min(kMaxT, nT - t0b);
      const int r = fp_rates4(c, nc, T + t0b, sb, &o, tmp.data(), nullptr);
      if (r) return r;
      std::memcpy(dst.data() + (size_t)t0b * nm, tmp.data(), (size_t)nc * nm * sizeof(double));
    }
    return FP_OK;
  };
  std::vector<unsigned char> mask(nm, 0);
  for (int m = 0; m < nm; ++m) mask[m] = role[m] ? 1 : 0;
  std::vector<double> exact(rows_all, 0.0);
  if ((rc = exact_at(mask, exact))) return rc;
  const double ms_exact = now_ms() - t0;

  // features on the device
  t0 = now_ms();
  double *dA = nullptr, *dT = nullptr;
  float *dX = nullptr, *dY = nullptr, *dmean = nullptr, *dstd = nullptr;
  int* drows = nullptr;
  Net net;
  auto cleanup = [&]() {
    cudaFree(dA);
    cudaFree(dT);
    cudaFree(dX);
    cudaFree(dY);
    cudaFree(dmean);
    cudaFree(dstd);
    cudaFree(drows);
    net_free(net);
  };
#define SW_TRY(call)                                                                                          \
  do {                                                                                                        \
    cudaError_t e_ = (call);                                                                                  \
    if (e_ != cudaSuccess) {                                                                                  \
      cleanup();                                                                                              \
      return sfail(c, e_ == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_ECUDA,                                 \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                                       \
    }                                                                                                         \
  } while (0)
  std::vector<int> train_rows;
  for (int m = 0; m < nm; ++m) {
    if (role[m] != 1) continue;
    bool anchors_ok = true;
    for (int k = 0; k < nA; ++k) anchors_ok = anchors_ok && anchor[(size_t)k * nm + m] > 0.0;
    for (int t = 0; t < nT && anchors_ok; ++t)
      if (exact[(size_t)t * nm + m] > 0.0) train_rows.push_back(t * nm + m);
  }
  if (train_rows.empty()) return sfail(c, FP_EINVAL, "fp_surrogate_sweep: no training rates > 0");
  const int Bmax = std::max(so.batch, 4096);
  SW_TRY(dalloc(&dA, (size_t)nA * nm));
  SW_TRY(dalloc(&dT, (size_t)nT));
  SW_TRY(dalloc(&dX, rows_all * F));
  SW_TRY(dalloc(&dY, rows_all));
  SW_TRY(dalloc(&dmean, F));
  SW_TRY(dalloc(&dstd, F));
  SW_TRY(dalloc(&drows, std::max(rows_all, (size_t)Bmax)));
  SW_TRY(net_alloc(net, F, Bmax));
  SW_TRY(cudaMemcpyAsync(dA, anchor.data(), anchor.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  SW_TRY(cudaMemcpyAsync(dT, T, nT * sizeof(double), cudaMemcpyHostToDevice, s));
  double wmax = 0.0;
  for (double w : om) wmax = std::max(wmax, w);
  sweep_features_kernel<<<(unsigned)((rows_all + 255) / 256), 256, 0, s>>>(dA, c->d_omega, dT, nm, nb, nT, nA, wmax,
                                                                          dX);
  SW_TRY(cudaGetLastError());
  SW_TRY(cudaMemcpyAsync(drows, train_rows.data(), train_rows.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  col_stats_kernel<<<1, 64, 0, s>>>(dX, F, drows, (int)train_rows.size(), dmean, dstd);
  normalize_kernel<<<(unsigned)((rows_all * F + 255) / 256), 256, 0, s>>>(dX, F, (long long)rows_all, dmean, dstd);
  std::vector<float> y(rows_all, 0.f);
  for (size_t r = 0; r < rows_all; ++r)
    if (exact[r] > 0.0) y[r] = (float)std::log(exact[r]);
  SW_TRY(cudaMemcpyAsync(dY, y.data(), rows_all * sizeof(float), cudaMemcpyHostToDevice, s));
  SW_TRY(cudaStreamSynchronize(s));
  const double ms_features = now_ms() - t0;

  // training: Adam on minibatches, rows reshuffled every epoch
  t0 = now_ms();
  {
    std::vector<float> p0 = init_params(F, so.seed);
    SW_TRY(cudaMemcpyAsync(net.p, p0.data(), p0.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    SW_TRY(cudaMemsetAsync(net.m, 0, p0.size() * sizeof(float), s));
    SW_TRY(cudaMemsetAsync(net.v, 0, p0.size() * sizeof(float), s));
  }
  const int P = (int)nparams(F);
  const int nrows = (int)train_rows.size();
  const int B = std::max(1, std::min(so.batch, std::max(32, nrows / 8)));
  std::vector<int> order(train_rows);
  int step = 0;
  const float b1 = 0.9f, b2 = 0.999f;
  for (int ep = 0; ep < so.epochs; ++ep) {
    for (size_t i = order.size(); i > 1; --i) std::swap(order[i - 1], order[rng.next() % i]);
    SW_TRY(cudaMemcpyAsync(drows, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    for (int b0 = 0; b0 + B <= nrows; b0 += B) {
      gather_kernel<<<(B * F + 255) / 256, 256, 0, s>>>(dX, F, drows + b0, B, net.X, dY, net.t);
      SW_TRY(net_forward(net, B, s));
      SW_TRY(net_backward(net, B, s));
      ++step;
      const float c1 = 1.f - std::pow(b1, (float)step), c2 = 1.f - std::pow(b2, (float)step);
      adam_kernel<<<(P + 255) / 256, 256, 0, s>>>(net.p, net.g, net.m, net.v, P, (float)so.lr, b1, b2, 1e-8f, c1, c2);
    }
  }
  float final_loss = 0.f;
  SW_TRY(cudaMemcpyAsync(&final_loss, net.loss, sizeof(float), cudaMemcpyDeviceToHost, s));
  SW_TRY(cudaStreamSynchronize(s));
  const double ms_train = now_ms() - t0;

  // prediction for every (temperature, mode) row
  t0 = now_ms();
  double* dpred = nullptr;
  SW_TRY(dalloc(&dpred, rows_all));
  std::vector<int> all(rows_all);
  std::iota(all.begin(), all.end(), 0);
  SW_TRY(cudaMemcpyAsync(drows, all.data(), rows_all * sizeof(int), cudaMemcpyHostToDevice, s));
  for (size_t r0 = 0; r0 < rows_all; r0 += Bmax) {
    const int nr = (int)std::min((size_t)Bmax, rows_all - r0);
    gather_kernel<<<(nr * F + 255) / 256, 256, 0, s>>>(dX, F, drows + r0, nr, net.X, nullptr, nullptr);
    SW_TRY(net_forward(net, nr, s));
    exp_kernel<<<(nr + 255) / 256, 256, 0, s>>>(net.y, nr, drows + r0, (int)rows_all, dpred);
  }
  std::vector<double> pred(rows_all);
  SW_TRY(cudaMemcpyAsync(pred.data(), dpred, rows_all * sizeof(double), cudaMemcpyDeviceToHost, s));
  SW_TRY(cudaStreamSynchronize(s));
  cudaFree(dpred);
  const double ms_predict = now_ms() - t0;

  // held-out error per bin (branch x frequency quartile): the rule of fp_surrogate_fit
  std::vector<double> wsorted;
  for (int m : pos) wsorted.push_back(om[m]);
  std::sort(wsorted.begin(), wsorted.end());
  double qcut[3];
  for (int k = 0; k < 3; ++k) qcut[k] = wsorted[(size_t)((k + 1) * wsorted.size() / 4)];
  auto bin_of = [&](int m) {
    int qb = 0;
    while (qb < 3 && om[m] >= qcut[qb]) ++qb;
    return (m % nb) * 4 + qb;
  };
  const int nbins = nb * 4;
  std::vector<double> bin_err(nbins, 0.0), bin_err2(nbins, 0.0), errs;
  std::vector<int> bin_cnt(nbins, 0);
  for (int m = 0; m < nm; ++m) {
    if (role[m] != 2) continue;
    for (int t = 0; t < nT; ++t) {
      const size_t r = (size_t)t * nm + m;
      if (!(exact[r] > 0.0)) continue;
      const double e = std::fabs(pred[r] - exact[r]) / exact[r];
      errs.push_back(e);
      bin_err[bin_of(m)] += e;
      bin_err2[bin_of(m)] += e * e;
      bin_cnt[bin_of(m)] += 1;
    }
  }
  int n_bins_fb = 0;
  std::vector<unsigned char> bin_fb(nbins, 0);
  for (int b = 0; b < nbins; ++b) {
    double e = 1e30;
    if (bin_cnt[b] >= 16) {
      const double n = bin_cnt[b], mu = bin_err[b] / n;
      const double var = std::max(0.0, bin_err2[b] / n - mu * mu);
      e = mu + 2.0 * std::sqrt(var / n);
    }
    if (e > so.tol) {
      bin_fb[b] = 1;
      ++n_bins_fb;
    }
  }
  t0 = now_ms();
  std::fill(mask.begin(), mask.end(), 0);
  int n_fb = 0;
  for (int m : pos)
    if (!role[m] && bin_fb[bin_of(m)]) {
      mask[m] = 1;
      role[m] = 3;
      ++n_fb;
    }
  std::vector<double> fb(rows_all, 0.0);
  if (n_fb && (rc = exact_at(mask, fb))) {
    cleanup();
    return rc;
  }
  const double ms_fallback = now_ms() - t0;
  for (int m = 0; m < nm; ++m)
    for (int t = 0; t < nT; ++t) {
      const size_t r = (size_t)t * nm + m;
      double v;
      unsigned char ex = 1;
      if (!(om[m] > 0.0)) {
        v = 0.0;
      } else if (role[m] == 1 || role[m] == 2) {
        v = exact[r];
      } else if (role[m] == 3) {
        v = fb[r];
      } else {
        v = pred[r];
        ex = 0;
      }
      if (rates) rates[r] = v;
      if (used_exact) used_exact[r] = ex;
    }
  if (rep) {
    std::memset(rep, 0, sizeof(*rep));
    rep->n_modes = (int)pos.size();
    rep->n_train = n_train;
    rep->n_holdout = n_hold;
    rep->n_fallback_modes = n_fb;
    rep->n_bins = nbins;
    rep->n_bins_fallback = n_bins_fb;
    rep->final_loss = final_loss;
    std::sort(errs.begin(), errs.end());
    if (!errs.empty()) {
      rep->holdout_median_rel_err = errs[errs.size() / 2];
      rep->holdout_p90_rel_err = errs[(size_t)(0.9 * (errs.size() - 1))];
      rep->holdout_max_rel_err = errs.back();
    }
    rep->ms_exact = ms_exact;
    rep->ms_features = ms_features;
    rep->ms_train = ms_train;
    rep->ms_predict = ms_predict;
    rep->ms_fallback = ms_fallback;
    rep->ms_total = now_ms() - t_start;
  }
  cleanup();
#undef SW_TRY
  return FP_OK;
}
