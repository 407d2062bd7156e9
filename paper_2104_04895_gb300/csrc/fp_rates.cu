// Host side of the rate path: FP32 prep kernel, fixed-order reduction, tile plan and the launch routine
// shared by fp_rates4, fp_rates4_device and fp_rates4_noalloc.  The rate kernel itself is in
// fp_rates_kernel.cuh.
#include "fp_rates_kernel.cuh"

namespace fp {
// kernel pointers of the two precision instantiations (fp_rates_f64.cu, fp_rates_f32.cu)
const void* rates_kernel_f64(int nb, int maxt);
const void* rates_kernel_f32(int nb, int maxt);
const void* rates_kernel_f32_tc(int nb, int maxt);
const void* rates_kernel_df(int nb, int maxt);

namespace {

// two-float split of a double: h + l = x to about 2^-48 |x|
__device__ __forceinline__ void split2(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

// FP32 copies of the tables for one call
__global__ void prep_kernel(RatesArgs a, float* omh, float* oml, float* velh, float* vell, float2* evf,
                            float* qfcf, float2* twf, float* wtf, int want_f32) {
  const long long NM = (long long)a.N * a.nb;
  const long long n_e = NM * a.nb, n_w = 3 * NM * a.nT, n_q = 81LL * a.nquart;
  const long long total = NM + 3 * NM + (want_f32 ? n_e + n_q + a.L + n_w : 0);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    long long k = i;
    if (k < NM) {
      split2(a.omega[k], omh[k], oml[k]);
      continue;
    }
    k -= NM;
    if (k < 3 * NM) {
      split2(a.vel[k], velh[k], vell[k]);
      continue;
    }
    k -= 3 * NM;
    if (k < n_e) {
      double2 e = a.evec[k];
      evf[k] = make_float2((float)e.x, (float)e.y);
      continue;
    }
    k -= n_e;
    if (k < n_q) {
      qfcf[k] = (float)a.qfc[k];
      continue;
    }
    k -= n_q;
    if (k < a.L) {
      double2 t = a.tw[k];
      twf[k] = make_float2((float)t.x, (float)t.y);
      continue;
    }
    k -= a.L;
    wtf[k] = (float)a.wt[k];
  }
}

// rates[t][q][j] = pref * sum_tiles partial[(tile, qpos[q], chunk)][jj][t], in a fixed order, for every selected
// mode of the output range (the others stay zero); under time reversal q and -q read the same partial sums.
__global__ void reduce_kernel(RatesArgs a, double pref, double* rates) {
  const long long n = (long long)a.nT * a.q_out_n * a.nb;
  long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int j = (int)(o % a.nb);
  const int q = a.q_out_begin + (int)((o / a.nb) % a.q_out_n);
  const int t = (int)(o / ((long long)a.nb * a.q_out_n));
  if (!a.sel[(size_t)q * a.nb + j]) return;
  const int qi = a.qpos[q];
  const int chunk = j / a.J, jj = j % a.J;
  double s = 0.0;
  for (int tile = 0; tile < a.ntile; ++tile) {
    const long long item = ((long long)tile * a.nq_sel + qi) * a.nchunk + chunk;
    s += a.partial[((size_t)item * a.J + jj) * a.nT + t];
  }
  rates[((size_t)t * a.N + q) * a.nb + j] = s * pref;
  if (a.mode_counts && t == 0) {
    unsigned long long cnt = 0;
    for (int tile = 0; tile < a.ntile; ++tile) {
      const long long item = ((long long)tile * a.nq_sel + qi) * a.nchunk + chunk;
      cnt += a.item_counts[(size_t)item * a.J + jj];
    }
    a.mode_counts[(size_t)q * a.nb + j] = (double)cnt * a.count_scale;
  }
}

// p[i] = v (the unit weight table of the unweighted phase space)
__global__ void fill_kernel(double* p, long long n, double v) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

// kernel for (precision, nb, number of temperatures, tensor cores): one accumulator per temperature, 1 or up to 8
const void* rates_kernel_ptr(int precision, int nb, int nT, bool tc) {
  const int maxt = nT == 1 ? 1 : kMaxT;
  if (tc) return precision == FP_PREC_MIXED ? rates_kernel_f32_tc(nb, maxt) : nullptr;
  if (precision == FP_PREC_DOUBLE_FLOAT) return rates_kernel_df(nb, maxt);
  return precision == FP_PREC_FP64 ? rates_kernel_f64(nb, maxt) : rates_kernel_f32(nb, maxt);
}

size_t smem_bytes(int precision, int nb, int J, int G, int nquart, int nT, int threads, bool tc) {
  const bool f32 = precision == FP_PREC_MIXED;  // the double-float path has the FP64 path's shared memory
  Carve c = make_carve(nb, J, G, nquart, nT, threads, f32);
  const size_t b = c.bytes(f32 ? sizeof(Cx<float>) : sizeof(Cx<double>));
  return tc ? align128(b) + kTcBytes : b;
}

int max_ctas_per_sm(int precision, int nb, int nT, int threads, size_t smem, bool tc) {
  const void* k = rates_kernel_ptr(precision, nb, nT, tc);
  if (!k) return 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  if (tc) {
    // For the tensor-core kernel the occupancy query reports one CTA per SM although its registers and shared
    // memory fit two (ncu's launch limits agree: two by registers, two by shared memory), and two use 64 of the
    // 512 TMEM columns.  Size the persistent grid from the registers and shared memory; a CTA that cannot be
    // resident yet starts later and finds fewer work items.
    cudaFuncAttributes fa;
    int dev = 0, regs_sm = 0, smem_sm = 0;
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess) {
      const long long warp_regs = ((long long)fa.numRegs * 32 + 255) / 256 * 256;
      const long long by_regs = regs_sm / (warp_regs * ((threads + 31) / 32));
      const long long by_smem = smem_sm / ((long long)smem + fa.sharedSizeBytes + 1024);
      const int est = (int)std::min(by_regs, by_smem);
      if (est > n) n = std::min(est, 2);
    }
  }
  return n;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int make_selection(const fp_ctx* c, const fp_rates_opts& o, bool fold_allowed, Selection* s, std::string* err) {
  const int N = c->N, nb = c->nb;
  const int q_end = o.q_end <= 0 ? N : o.q_end;
  if (o.q_begin < 0 || o.q_begin > q_end || q_end > N) {
    *err = "bad q range";
    return FP_EINVAL;
  }
  s->fold = fold_allowed && o.no_time_reversal == 0 && o.nu_select == 0;
  s->q_out_begin = o.q_begin;
  s->q_out_end = q_end;
  const size_t nm = (size_t)N * nb;
  s->sel.assign(nm, 0);
  s->mult.assign(nm, 0);
  s->qpos.assign(N, -1);
  s->qlist.clear();
  s->n_sel = 0;
  s->n_exec = 0;
  for (int q = o.q_begin; q < q_end; ++q)
    for (int j = 0; j < nb; ++j) {
      const size_t m = (size_t)q * nb + j;
      s->sel[m] = (o.mode_mask == nullptr || o.mode_mask[m]) ? 1 : 0;
      s->n_sel += s->sel[m];
    }
  // -q on the grid, componentwise (N_a - g_a) mod N_a
  auto neg = [&](int q) {
    const int g0 = q / (c->grid[1] * c->grid[2]), g1 = (q / c->grid[2]) % c->grid[1], g2 = q % c->grid[2];
    const int m0 = (c->grid[0] - g0) % c->grid[0], m1 = (c->grid[1] - g1) % c->grid[1],
              m2 = (c->grid[2] - g2) % c->grid[2];
    return (m0 * c->grid[1] + m1) * c->grid[2] + m2;
  };
  for (int q = 0; q < N; ++q) {
    const int p = s->fold ? neg(q) : q;
    if (s->fold && p < q) continue;  // the pair {p, q} is evaluated at its smaller index p
    int any = 0;
    for (int j = 0; j < nb; ++j) {
      int m = s->sel[(size_t)q * nb + j];
      if (p != q) m += s->sel[(size_t)p * nb + j];
      s->mult[(size_t)q * nb + j] = (unsigned char)m;
      any |= m;
      s->n_exec += m > 0 ? 1 : 0;
    }
    if (!any) continue;
    s->qpos[q] = (int)s->qlist.size();
    if (p != q) s->qpos[p] = (int)s->qlist.size();
    s->qlist.push_back(q);
  }
  return FP_OK;
}

int plan_rates(fp_ctx* c, const fp_rates_opts& o, int nT, Selection& sel, size_t partial_budget, Plan* p,
               std::string* err) {
  const int N = c->N, nb = c->nb;
  const bool tc = o.tensor_cores != 0;
  if (tc && (o.precision != FP_PREC_MIXED || nb != 6)) {
    *err = "tensor_cores needs the mixed precision and 6 branches";
    return FP_EINVAL;
  }
  if (!rates_kernel_ptr(o.precision, nb, nT, tc)) {
    *err = "unsupported number of branches";
    return FP_EINVAL;
  }
  int J = o.block_j0;
  int t1_tuned = 0, th_tuned = 0;
  if (J <= 0 && o.k1_tile <= 0 && o.threads <= 0) {
    const int* tt = c->tuned[o.precision][nT == 1 ? 0 : 1];
    if (tt[0] > 0) {
      J = tt[0];
      t1_tuned = tt[1];
      th_tuned = tt[2];
    }
  }
  if (J <= 0) {
    // largest divisor of nb whose rows fit a block and whose tile leaves room for two blocks per SM
    J = nb;
    while (J > 1 && (J * nb * nb > max_threads_for(nb) ||
                     smem_bytes(o.precision, nb, J, c->G, c->nquart, nT, max_threads_for(nb), tc) > 110 * 1024)) {
      int nj = J - 1;
      while (nj > 1 && nb % nj) --nj;
      J = nj;
    }
  }
  if (J < 1 || nb % J) {
    *err = "block_j0 must divide nb";
    return FP_EINVAL;
  }
  const int rows = J * nb * nb;
  int threads = o.threads > 0 ? o.threads : th_tuned > 0 ? th_tuned : ((rows + 31) / 32) * 32;
  if (threads < 32) threads = 32;
  if (threads % 32 || threads < rows || threads > max_threads_for(nb)) {
    *err = "threads must be a multiple of 32, >= block_j0*nb^2 and <= " + std::to_string(max_threads_for(nb));
    return FP_EINVAL;
  }
  const int nq_sel = (int)sel.qlist.size();
  const int nchunk = nb / J;
  int t1 = o.k1_tile > 0 ? o.k1_tile : t1_tuned > 0 ? t1_tuned : (N + 511) / 512;
  auto part_bytes = [&](int tile) {
    return (size_t)((N + tile - 1) / tile) * nq_sel * nchunk * J * nT * sizeof(double);
  };
  if (o.k1_tile <= 0 && partial_budget)
    while (t1 < N && part_bytes(t1) > partial_budget) t1 = t1 < 8 ? t1 + 1 : t1 + t1 / 4;
  if (t1 > N) t1 = N;
  // the kernel counts an item's accepted terms in 32 bits: at most 6 per (q', q'', j''') of a row, times the
  // row's multiplicity 2, over the tile's t1 q' values
  const double max_t1 = 4294967295.0 / (12.0 * (double)N * nb);
  if (max_t1 < 1.0) {
    *err = "grid too large for the per-item counters";
    return FP_EINVAL;
  }
  if ((double)t1 > max_t1) {
    if (o.k1_tile > 0) {
      *err = "k1_tile too large for the per-item counters of this grid";
      return FP_EINVAL;
    }
    t1 = (int)max_t1;
  }
  if (partial_budget && part_bytes(t1) > partial_budget) {
    *err = "per-item partial sums do not fit the scratch";
    return FP_EINVAL;
  }
  const size_t smem = smem_bytes(o.precision, nb, J, c->G, c->nquart, nT, threads, tc);
  if (smem > 227 * 1024) {
    *err = "tile does not fit in shared memory";
    return FP_EINVAL;
  }
  const int per_sm = max_ctas_per_sm(o.precision, nb, nT, threads, smem, tc);
  if (per_sm < 1) {
    *err = "kernel tile cannot be resident on an SM";
    return FP_EINVAL;
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    *err = "cudaDeviceGetAttribute failed";
    return FP_ECUDA;
  }
  p->J = J;
  p->threads = threads;
  p->t1 = t1;
  p->nchunk = nchunk;
  p->ntile = (N + t1 - 1) / t1;
  p->nq_sel = nq_sel;
  p->n_items = (long long)p->ntile * nq_sel * nchunk;
  p->smem = smem;
  long long ctas = (long long)nsm * per_sm;
  if (ctas > p->n_items) ctas = p->n_items > 0 ? p->n_items : 1;
  p->ctas = (int)ctas;
  sel.active_chunks = 0;
  for (int q : sel.qlist)
    for (int ch = 0; ch < nchunk; ++ch) {
      int any = 0;
      for (int jj = 0; jj < J; ++jj) any |= sel.mult[(size_t)q * nb + ch * J + jj];
      sel.active_chunks += any ? 1 : 0;
    }
  return FP_OK;
}

void scratch_sizes(const fp_ctx* c, const Plan& p, int nT, size_t s[kScratchParts]) {
  const size_t nm = (size_t)c->N * c->nb;
  s[0] = up256(kCounters * sizeof(unsigned long long));
  s[1] = up256(kMaxT * sizeof(double));
  s[2] = up256(nm);                                       // mult
  s[3] = up256(nm);                                       // sel
  s[4] = up256((size_t)c->N * sizeof(int));               // qlist
  s[5] = up256((size_t)c->N * sizeof(int));               // qpos
  s[6] = up256(3 * nm * nT * sizeof(double));             // wt
  s[kScratchPartial] = up256((size_t)p.n_items * p.J * nT * sizeof(double));
  s[8] = up256(nm * sizeof(float));
  s[9] = up256(nm * sizeof(float));
  s[10] = up256(3 * nm * sizeof(float));
  s[11] = up256(3 * nm * sizeof(float));
  s[12] = up256(nm * c->nb * sizeof(float2));
  s[13] = up256((size_t)81 * c->nquart * sizeof(float));
  s[14] = up256((size_t)c->L * sizeof(float2));
  s[15] = up256(3 * nm * nT * sizeof(float));
}

Scratch carve_scratch(unsigned char* b, const size_t sz[kScratchParts]) {
  size_t off[kScratchParts], acc = 0;
  for (int i = 0; i < kScratchParts; ++i) {
    off[i] = acc;
    acc += sz[i];
  }
  Scratch sc;
  sc.counters = reinterpret_cast<unsigned long long*>(b + off[0]);
  sc.T = reinterpret_cast<double*>(b + off[1]);
  sc.mult = b + off[2];
  sc.sel = b + off[3];
  sc.qlist = reinterpret_cast<int*>(b + off[4]);
  sc.qpos = reinterpret_cast<int*>(b + off[5]);
  sc.wt = reinterpret_cast<double*>(b + off[6]);
  sc.partial = reinterpret_cast<double*>(b + off[kScratchPartial]);
  sc.omh = reinterpret_cast<float*>(b + off[8]);
  sc.oml = reinterpret_cast<float*>(b + off[9]);
  sc.velh = reinterpret_cast<float*>(b + off[10]);
  sc.vell = reinterpret_cast<float*>(b + off[11]);
  sc.evf = reinterpret_cast<float2*>(b + off[12]);
  sc.qfcf = reinterpret_cast<float*>(b + off[13]);
  sc.twf = reinterpret_cast<float2*>(b + off[14]);
  sc.wtf = reinterpret_cast<float*>(b + off[15]);
  return sc;
}

int run_rates(fp_ctx* c, const fp_rates_opts& o, const Selection& sel, const Plan& p, const Scratch& sc, int nT,
              const double* T, double sb, double* d_out, unsigned long long counts[kCounters], bool use_graph,
              std::string* err, const RunExtra& x) {
  const int unit_stride = x.unit_stride;
  cudaStream_t s = c->stream;
  const int N = c->N, nb = c->nb;
  const size_t nm = (size_t)N * nb;
#define RR_CUDA(call)                                                 \
  do {                                                                \
    cudaError_t e_ = (call);                                          \
    if (e_ != cudaSuccess) {                                          \
      *err = std::string(#call) + ": " + cudaGetErrorString(e_);      \
      return FP_ECUDA;                                                \
    }                                                                 \
  } while (0)
  RR_CUDA(cudaMemcpyAsync(sc.T, T, nT * sizeof(double), cudaMemcpyHostToDevice, s));
  RR_CUDA(cudaMemcpyAsync(sc.mult, sel.mult.data(), nm, cudaMemcpyHostToDevice, s));
  RR_CUDA(cudaMemcpyAsync(sc.sel, sel.sel.data(), nm, cudaMemcpyHostToDevice, s));
  RR_CUDA(cudaMemcpyAsync(sc.qpos, sel.qpos.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice, s));
  if (!sel.qlist.empty())
    RR_CUDA(cudaMemcpyAsync(sc.qlist, sel.qlist.data(), sel.qlist.size() * sizeof(int), cudaMemcpyHostToDevice, s));

  RatesArgs a;
  std::memset(&a, 0, sizeof(a));  // padding included: the graph cache compares launch parameters bytewise
  a.N = N;
  a.nb = nb;
  a.natoms = c->natoms;
  a.nT = nT;
  a.L = c->L;
  a.G = c->G;
  a.nquart = c->nquart;
  for (int d = 0; d < 3; ++d) {
    a.grid[d] = c->grid[d];
    a.Lfac[d] = c->L / c->grid[d];
  }
  a.J = p.J;
  a.t1 = p.t1;
  a.nchunk = p.nchunk;
  a.ntile = p.ntile;
  a.nq_sel = p.nq_sel;
  a.n_items = p.n_items;
  a.qlist = sc.qlist;
  a.mult = sc.mult;
  a.q_out_begin = sel.q_out_begin;
  a.q_out_n = sel.q_out_end - sel.q_out_begin;
  a.qpos = sc.qpos;
  a.sel = sc.sel;
  a.omega = c->d_omega;
  a.evec = c->d_evec;
  a.vel = c->d_vel;
  a.wt = sc.wt;
  a.qmeta = c->d_qmeta;
  a.qfc = c->d_qfc;
  a.gmeta = c->d_gmeta;
  a.grp_qstart = c->d_grp_qstart;
  a.grp_q = c->d_grp_q;
  a.kl_start = c->d_kl_start;
  a.kl_grp = c->d_kl_grp;
  a.tw = c->d_tw;
  a.omh = sc.omh;
  a.oml = sc.oml;
  a.velh = sc.velh;
  a.vell = sc.vell;
  a.evf = sc.evf;
  a.qfcf = sc.qfcf;
  a.twf = sc.twf;
  a.wtf = sc.wtf;
  a.sb = sb;
  a.window = o.window;
  a.sigma_min = o.sigma_min;
  const double* B = c->rec;
  const double detB = B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6]) +
                      B[2] * (B[3] * B[7] - B[4] * B[6]);
  a.dq = std::cbrt(std::fabs(detB) / (double)N);
  a.dq_mode = o.dq_mode;
  for (int i = 0; i < 9; ++i) a.rec[i] = B[i];
  a.partial = sc.partial;
  a.counter = sc.counters;
  a.counts = sc.counters + 1;
  a.unit_vertex = unit_stride > 0 ? 1 : 0;
  a.k1_stride = unit_stride > 0 ? unit_stride : 1;
  {
    const int pm = o.process_mask == 0 ? 7 : o.process_mask;
    a.cand_mask = (unsigned)(pm | (pm << 3));  // both orderings of each selected process
  }
  a.nu_select = o.nu_select;
  a.bzm = c->d_bzm;
  a.item_counts = x.d_mode_counts ? x.d_item_counts : nullptr;
  a.mode_counts = x.d_mode_counts;
  a.count_scale = unit_stride > 0 ? (double)unit_stride : 1.0;

  const int want_f32 = o.precision == FP_PREC_MIXED;
  const double conv = kConv;
  // unit-vertex mode: no physical prefactor; scale the strided ordered-pair sum to the full grid
  const double pref = unit_stride > 0
                          ? (double)unit_stride / ((double)N * (double)N)
                          : kPi * kHbar * kHbar * conv * conv * conv * conv / (8.0 * (double)N * (double)N);
  const void* k = rates_kernel_ptr(o.precision, nb, nT, o.tensor_cores != 0);
  // the device part of a rate set: Bose weights, FP32 tables, cleared counters and output, the persistent
  // rate kernel and the reduction
  auto enqueue = [&]() -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (x.unit_weights) {
      fill_kernel<<<152, 256, 0, s>>>(sc.wt, 3LL * (long long)nm * nT, 1.0);
      e = cudaGetLastError();
    } else {
      e = launch_weights(c, nT, sc.T, sc.wt, s);
    }
    if (e != cudaSuccess) return e;
    if (x.d_mode_counts &&
        (e = cudaMemsetAsync(x.d_mode_counts, 0, nm * sizeof(double), s)) != cudaSuccess)
      return e;
    prep_kernel<<<4 * 152, 256, 0, s>>>(a, sc.omh, sc.oml, sc.velh, sc.vell, sc.evf, sc.qfcf, sc.twf, sc.wtf,
                                        want_f32);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(sc.counters, 0, kCounters * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d_out, 0, (size_t)nT * nm * sizeof(double), s)) != cudaSuccess) return e;
    if (p.n_items > 0) {
      RatesArgs aa = a;
      void* args[] = {&aa};
      if ((e = cudaLaunchKernel(k, dim3(p.ctas), dim3(p.threads), args, p.smem, s)) != cudaSuccess) return e;
      const long long n = (long long)nT * (sel.q_out_end - sel.q_out_begin) * nb;
      reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, pref, d_out);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  RR_CUDA(cudaEventRecord(c->ev0, s));
  if (use_graph) {
    // replay the captured graph when every launch parameter is unchanged, else capture a new one
    struct Key {
      RatesArgs a;
      const void* k;
      double* out;
      int ctas, threads, want_f32, nT;
      size_t smem;
      double pref;
    } key;
    std::memset(&key, 0, sizeof(key));
    key.a = a;
    key.k = k;
    key.out = d_out;
    key.ctas = p.ctas;
    key.threads = p.threads;
    key.want_f32 = want_f32;
    key.nT = nT;
    key.smem = p.smem;
    key.pref = pref;
    const unsigned char* kb = reinterpret_cast<const unsigned char*>(&key);
    if (!c->graph_exec || c->graph_key.size() != sizeof(key) ||
        std::memcmp(c->graph_key.data(), kb, sizeof(key)) != 0) {
      if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
      }
      cudaGraph_t g = nullptr;
      RR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      cudaError_t ce = enqueue();
      cudaError_t ee = cudaStreamEndCapture(s, &g);
      if (ce != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        *err = std::string("graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee);
        return FP_ECUDA;
      }
      cudaError_t ie = cudaGraphInstantiate(&c->graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        c->graph_exec = nullptr;
        *err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie);
        return FP_ECUDA;
      }
      c->graph_key.assign(kb, kb + sizeof(key));
    }
    RR_CUDA(cudaGraphLaunch(c->graph_exec, s));
  } else {
    RR_CUDA(enqueue());
  }
  RR_CUDA(cudaEventRecord(c->ev1, s));
  RR_CUDA(cudaMemcpyAsync(counts, sc.counters, kCounters * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  RR_CUDA(cudaStreamSynchronize(s));
#undef RR_CUDA
  if (counts[6] != 0) {
    *err = "a tensor-core completion wait ran out of polls (" + std::to_string(counts[6]) + " warps); results invalid";
    return FP_ECUDA;
  }
  return FP_OK;
}

void fill_stats(const fp_ctx* c, const fp_rates_opts& o, const Selection& sel, const Plan& p,
                const unsigned long long counts[kCounters], fp_stats* st) {
  const int N = c->N, nb = c->nb;
  std::memset(st, 0, sizeof(*st));
  const int pm = o.process_mask == 0 ? 7 : o.process_mask;
  const double nproc = (double)((pm & 1) + ((pm >> 1) & 1) + ((pm >> 2) & 1));
  const double per_mode = nproc * (double)N * (double)N * (double)nb * nb * nb;
  st->candidates = per_mode * sel.n_sel;
  st->candidates_executed = per_mode * sel.n_exec;
  for (int k = 0; k < 3; ++k) st->accepted[k] = (double)counts[1 + k];
  st->vertex_entries = (double)counts[4];
  st->terms_executed = (double)counts[5];
  // complex multiply-adds (8 flops each) of the evaluated items: per item and q' the Psi prologue, per unordered
  // (q', q'') pair the grouped assembly (9 J nb G) and T (J nb^3 nb), and nb per vertex entry W formed
  const double J = p.J;
  const double pairs = 0.5 * (double)N * (double)(N + 1);
  const double per_pair = 8.0 * (9.0 * J * nb * c->G + J * (double)nb * nb * nb * nb);
  const double prolog = 8.0 * 9.0 * J * nb * 9.0 * c->nquart;
  st->flops = (double)sel.active_chunks * (pairs * per_pair + (double)N * prolog) + 8.0 * nb * st->vertex_entries;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  st->ms = ms;
  st->tile[0] = p.J;
  st->tile[1] = p.t1;
  st->tile[2] = p.threads;
  st->tile[3] = p.ctas;
}

}  // namespace fp

namespace fp {
int phase4_sampled(fp_ctx* c, int nT, const double* T, double sb, int stride, double* d_out, std::string* err) {
  fp_rates_opts o;
  fp_default_opts(&o);
  o.precision = FP_PREC_MIXED;
  o.no_graph = 1;
  Selection sel;
  int rc = make_selection(c, o, false, &sel, err);  // q' on a stride is not symmetric under q -> -q
  if (rc) return rc;
  Plan p;
  rc = plan_rates(c, o, nT, sel, 0, &p, err);
  if (rc) return rc;
  // a q' tile of one stride: every item owns exactly one sampled q'
  p.t1 = stride;
  p.ntile = (c->N + stride - 1) / stride;
  p.n_items = (long long)p.ntile * p.nq_sel * p.nchunk;
  if (p.ctas > p.n_items) p.ctas = (int)p.n_items;
  size_t sz[kScratchParts], total = 0;
  scratch_sizes(c, p, nT, sz);
  for (size_t x : sz) total += x;
  unsigned char* b = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b), total);
  if (e != cudaSuccess) {
    *err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return FP_ENOMEM;
  }
  Scratch sc = carve_scratch(b, sz);
  unsigned long long counts[kCounters];
  RunExtra x;
  x.unit_stride = stride;
  rc = run_rates(c, o, sel, p, sc, nT, T, sb, d_out, counts, false, err, x);
  cudaFree(b);
  return rc;
}
}  // namespace fp
