// Batched form: many registration pairs of uneven sizes evaluated, and
// registered, together.  One launch per phase covers every (pair, tile) work
// item (kernels_batch.cuh); the phases of one evaluation, or of one L-BFGS
// round, can be captured once in a CUDA graph and replayed.
//
// The batched L-BFGS keeps the whole optimiser state on the device: after
// each batched evaluation one CTA per pair takes the line-search decision
// (Armijo and weak-Wolfe tests, halve or double the step), accepts the step
// and updates the (s, y) history, runs the two-loop recursion for the next
// direction and writes the next trial point, all with FP64 inner products in
// a fixed order.  A round is therefore the same fixed sequence of launches
// for every pair and every iteration; pairs that stop drop out through their
// active flag.  The host only checks, every few rounds, whether any pair is
// still active.  The method per pair is the one of lbfgs.cuh (Sec. II-F).
// Included once, at the end of srwcr.cu.
#pragma once

#include "kernels_batch.cuh"

namespace {

constexpr int kLbHist = 64;  // ring of accepted values for the stability test

struct LbOpts {
  int m, max_iter, window, max_ls;
  double rtol, c1, c2;
};

struct LbState {
  double f;            // value at x
  double gd;           // g . d at x
  double alpha;        // current trial step
  double rho[16];      // 1 / (s . y) per history slot
  double fh[kLbHist];  // accepted values (including the start), ring
  int nfh;
  int head, hist_len;  // history ring: next slot, entries in use
  int iter, evals, trials, restart, phase, status;
  int max_iter;        // this pair's iteration limit (its level's entry of the options)
};

// FP64 inner product over one pair's vectors by one CTA, in a fixed order;
// every thread receives the same value.  All threads must call it.
__device__ double block_dot(const float* __restrict__ a, const float* __restrict__ b,
                            long long n, double* sh) {
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) s += (double)a[i] * (double)b[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();  // earlier readers of sh are done
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  const int nw = blockDim.x >> 5;
  for (int w = 0; w < nw; ++w) t += sh[w];
  return t;
}

// Start: trial point = start point, first evaluation pending.
__global__ void k_lbfgs_init(LbState* __restrict__ st, int* __restrict__ active,
                             const long long* __restrict__ off, const float* __restrict__ x,
                             float* __restrict__ xn, const int* __restrict__ max_iter) {
  const int p = blockIdx.x;
  for (long long i = off[p] + threadIdx.x; i < off[p + 1]; i += blockDim.x) xn[i] = x[i];
  if (threadIdx.x == 0) {
    LbState s;
    memset(&s, 0, sizeof s);
    s.restart = 1;
    s.max_iter = max_iter[p];
    st[p] = s;
    active[p] = 1;
  }
}

struct LbVectors {
  float *x, *g, *xn, *gn, *d, *S, *Y;
  const long long* off;  // [n+1] offsets of each pair's vectors
  double* D;             // [n] values at xn; a finished pair's final value
};

// One CTA per pair: consume the evaluation at xn, decide, and prepare the
// next trial point.  Control flow is uniform across the CTA: it depends only
// on the shared state and on values every thread computes identically.
__global__ void __launch_bounds__(1024)
k_lbfgs_step(LbState* __restrict__ st_all, int* __restrict__ active, LbVectors v, LbOpts o) {
  const int p = blockIdx.x;
  if (!active[p]) return;
  __shared__ LbState s;
  __shared__ double sh[32];
  __shared__ double ak[16];
  if (threadIdx.x == 0) s = st_all[p];
  __syncthreads();
  const long long n = v.off[p + 1] - v.off[p];
  float* __restrict__ x = v.x + v.off[p];
  float* __restrict__ g = v.g + v.off[p];
  float* __restrict__ xn = v.xn + v.off[p];
  float* __restrict__ gn = v.gn + v.off[p];
  float* __restrict__ d = v.d + v.off[p];
  float* __restrict__ S = v.S + (long long)o.m * v.off[p];
  float* __restrict__ Y = v.Y + (long long)o.m * v.off[p];
  const double fn = v.D[p];
  const int tid = threadIdx.x, nt = blockDim.x;
  int done = 0, status = SRWCR_OK;

  if (s.phase == 0) {
    // First evaluation: x = xn already.
    for (long long i = tid; i < n; i += nt) g[i] = gn[i];
    __syncthreads();
    if (tid == 0) {
      s.f = fn;
      s.evals = 1;
      s.fh[0] = fn;
      s.nfh = 1;
    }
    if (!isfinite(fn)) { done = 1; status = SRWCR_ENUMERIC; }
    else if (s.max_iter <= 0) { done = 1; status = SRWCR_ENOTCONVERGED; }
  } else {
    if (tid == 0) s.evals += 1;
    int act = 0;  // 0 accept, 1 shrink, 2 grow
    if (!isfinite(fn) || fn > s.f + o.c1 * s.alpha * s.gd) {
      act = 1;
    } else {
      const double gnd = block_dot(gn, d, n, sh);
      if (gnd < o.c2 * s.gd) act = 2;
    }
    if (act != 0) {
      __syncthreads();
      const double alpha = act == 1 ? 0.5 * s.alpha : 2.0 * s.alpha;
      const int trials = s.trials + 1;
      if (trials >= o.max_ls) {
        done = 1;
        status = SRWCR_ELINESEARCH;
      } else {
        for (long long i = tid; i < n; i += nt) xn[i] = x[i] + (float)alpha * d[i];
      }
      __syncthreads();
      if (tid == 0) { s.alpha = alpha; s.trials = trials; }
      __syncthreads();
      if (!done) {
        if (tid == 0) st_all[p] = s;
        return;
      }
    } else {
      // Accept: s = xn - x, y = gn - g into the head slot; x = xn, g = gn.
      float* sv = S + (long long)s.head * n;
      float* yv = Y + (long long)s.head * n;
      for (long long i = tid; i < n; i += nt) {
        sv[i] = xn[i] - x[i];
        yv[i] = gn[i] - g[i];
        x[i] = xn[i];
        g[i] = gn[i];
      }
      __syncthreads();
      const double sy = block_dot(sv, yv, n, sh);
      __syncthreads();
      if (tid == 0) {
        if (sy > 0.0) {
          s.rho[s.head] = 1.0 / sy;
          s.head = (s.head + 1) % o.m;
          s.hist_len = min(s.hist_len + 1, o.m);
        }
        s.f = fn;
        s.restart = 0;
        s.iter += 1;
        s.fh[s.nfh % kLbHist] = fn;
        s.nfh += 1;
      }
      __syncthreads();
      const int w = o.window;
      if (w > 0 && s.nfh > w &&
          fabs(s.fh[(s.nfh - 1) % kLbHist] - s.fh[(s.nfh - 1 - w) % kLbHist]) <=
              o.rtol * fabs(s.fh[(s.nfh - 1) % kLbHist])) {
        done = 1;
        status = SRWCR_OK;
      } else if (s.iter >= s.max_iter) {
        done = 1;
        status = SRWCR_ENOTCONVERGED;
      }
    }
  }

  if (!done) {
    // Next direction d = -H g by the two-loop recursion.
    const double gg = block_dot(g, g, n, sh);
    if (!(gg > 0.0)) {
      done = 1;
      status = SRWCR_OK;
    } else {
      for (long long i = tid; i < n; i += nt) d[i] = g[i];
      __syncthreads();
      const int m = o.m, head = s.head, hl = s.hist_len;
      for (int t = 0; t < hl; ++t) {
        const int slot = (head - 1 - t + m) % m;
        const double a = s.rho[slot] * block_dot(S + (long long)slot * n, d, n, sh);
        if (tid == 0) ak[slot] = a;
        const float* yv = Y + (long long)slot * n;
        for (long long i = tid; i < n; i += nt) d[i] = (float)-a * yv[i] + d[i];
        __syncthreads();
      }
      if (hl > 0) {
        const int nw = (head - 1 + m) % m;
        const double sy = block_dot(S + (long long)nw * n, Y + (long long)nw * n, n, sh);
        const double yy = block_dot(Y + (long long)nw * n, Y + (long long)nw * n, n, sh);
        const float sc = (float)(sy / yy);
        for (long long i = tid; i < n; i += nt) d[i] = sc * d[i];
        __syncthreads();
      }
      for (int t = hl - 1; t >= 0; --t) {
        const int slot = (head - 1 - t + m) % m;
        const double beta = s.rho[slot] * block_dot(Y + (long long)slot * n, d, n, sh);
        const float coef = (float)(ak[slot] - beta);
        const float* sv = S + (long long)slot * n;
        for (long long i = tid; i < n; i += nt) d[i] = coef * sv[i] + d[i];
        __syncthreads();
      }
      for (long long i = tid; i < n; i += nt) d[i] = -d[i];
      __syncthreads();
      double gd = block_dot(g, d, n, sh);
      int restart = s.restart, clear = 0;
      if (!(gd < 0.0)) {
        // Not a descent direction: drop the history, steepest descent.
        for (long long i = tid; i < n; i += nt) d[i] = -g[i];
        __syncthreads();
        gd = -gg;
        restart = 1;
        clear = 1;
      }
      const double dd = block_dot(d, d, n, sh);
      const double alpha = restart ? 1.0 / sqrt(dd) : 1.0;
      for (long long i = tid; i < n; i += nt) xn[i] = x[i] + (float)alpha * d[i];
      __syncthreads();
      if (tid == 0) {
        if (clear) { s.hist_len = 0; s.head = 0; }
        s.restart = restart;
        s.gd = gd;
        s.alpha = alpha;
        s.trials = 0;
        s.phase = 1;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (done) {
      s.status = status;
      active[p] = 0;
      v.D[p] = s.f;
    }
    st_all[p] = s;
  }
}

}  // namespace

struct srwcr_batch {
  int n = 0;
  std::vector<int> level;      // caller order: each pair's pyramid level
  int ndim = 0;
  bool bf16 = false;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<srwcr_ctx*> ctx;
  std::vector<long long> off;  // caller order, n+1 float offsets into c and g
  // Row-kernel launches.  Pairs are grouped by x-bins per row (4, 8 or 12, a
  // template parameter) and by how many CTAs of their shared-memory size fit
  // on an SM (a launch's dynamic shared memory is the largest of its pairs',
  // so mixing sizes would lower the occupancy of the smaller ones); at most
  // kBatchChunk pairs per launch.  Each launch keeps its parameter table for
  // the plain evaluation and for the optimiser's (reads xn, writes gn).
  struct AccLaunch {
    int nxb, nblk;
    size_t smem;
    AccTable t, t_lb;
  };
  struct AdjLaunch {
    int nxb, nblk;
    size_t smem;
    AdjTable t, t_lb;
  };
  std::vector<AccLaunch> acc_launches;
  std::vector<AdjLaunch> adj_launches;
  std::vector<BatchPair> host_tab;  // table order (by group, then size)
  long long total_regions = 0;
  int fin_lanes = 32;               // lanes per region of the finalisation
  long long total_vox = 0;
  long long work_items = 0;
  float* c = nullptr;
  float* g = nullptr;
  double* D = nullptr;  // [n] caller order
  int* ndeg = nullptr;
  long long* off_dev = nullptr;
  BatchPair* tab_eval = nullptr;
  BatchPair* tab_lb = nullptr;
  // L-BFGS work (allocated on first registration).
  float *xn = nullptr, *gn = nullptr, *d = nullptr, *S = nullptr, *Y = nullptr;
  int lb_m = 0;
  LbState* lbs = nullptr;
  int* lb_max_iter = nullptr;       // [n] each pair's iteration limit
  int* active = nullptr;
  int* active_host = nullptr;
  cudaGraphExec_t graph_eval = nullptr;
  cudaGraphExec_t graph_round = nullptr;
  LbOpts graph_round_opts{};
  long long launches = 0;
};

namespace {

template <int DIM, typename T>
void launch_batch_rows(srwcr_batch* b, bool lb, const int* active, bool adj) {
  if (adj) {
    for (const auto& L : b->adj_launches) {
      const AdjTable& t = lb ? L.t_lb : L.t;
      if (L.nxb == 4)
        k_adjoint_rows_batch<DIM, T, 4><<<L.nblk, kAdjWarps * 32, L.smem, b->stream>>>(t, active);
      else if (L.nxb == 8)
        k_adjoint_rows_batch<DIM, T, 8><<<L.nblk, kAdjWarps * 32, L.smem, b->stream>>>(t, active);
      else
        k_adjoint_rows_batch<DIM, T, 12><<<L.nblk, kAdjWarps * 32, L.smem, b->stream>>>(t, active);
    }
  } else {
    for (const auto& L : b->acc_launches) {
      const AccTable& t = lb ? L.t_lb : L.t;
      if (L.nxb == 4)
        k_accumulate_rows_batch<DIM, T, 4><<<L.nblk, kAccWarps * 32, L.smem, b->stream>>>(t, active);
      else if (L.nxb == 8)
        k_accumulate_rows_batch<DIM, T, 8><<<L.nblk, kAccWarps * 32, L.smem, b->stream>>>(t, active);
      else
        k_accumulate_rows_batch<DIM, T, 12><<<L.nblk, kAccWarps * 32, L.smem, b->stream>>>(t, active);
    }
  }
}

void launch_rows_any(srwcr_batch* b, bool lb, const int* active, bool adj) {
  if (b->ndim == 3) {
    if (b->bf16) launch_batch_rows<3, __nv_bfloat16>(b, lb, active, adj);
    else launch_batch_rows<3, float>(b, lb, active, adj);
  } else {
    if (b->bf16) launch_batch_rows<2, __nv_bfloat16>(b, lb, active, adj);
    else launch_batch_rows<2, float>(b, lb, active, adj);
  }
}

template <typename T>
srwcr_status set_smem_limits_batch_t() {
  // The row path keeps dynamic shared memory at or below 220 KB; the batched
  // kernels also hold a few hundred bytes of static descriptors.
  const int mx = 221 * 1024;
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  CK(cudaFuncSetAttribute(k_accumulate_rows_batch<3, T, 12>, a, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_batch<2, T, 12>, a, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_batch<3, T, 12>, a, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_batch<2, T, 12>, a, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_batch<3, T, 4>, a, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_batch<3, T, 8>, a, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_batch<2, T, 4>, a, mx));
  CK(cudaFuncSetAttribute(k_accumulate_rows_batch<2, T, 8>, a, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_batch<3, T, 4>, a, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_batch<3, T, 8>, a, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_batch<2, T, 4>, a, mx));
  CK(cudaFuncSetAttribute(k_adjoint_rows_batch<2, T, 8>, a, mx));
  return SRWCR_OK;
}

srwcr_status set_smem_limits_batch() {
  RET_IF(set_smem_limits_batch_t<float>());
  return set_smem_limits_batch_t<__nv_bfloat16>();
}

// The phases of one batched value+gradient, queued on the batch stream.
// lb selects the optimiser's tables (xn -> gn) instead of (c -> g).
srwcr_status queue_batch_eval(srwcr_batch* b, bool lb, const int* active) {
  const BatchPair* tab = lb ? b->tab_lb : b->tab_eval;
  k_zero_batch<<<dim3(64, b->n), 256, 0, b->stream>>>(tab, active);
  CKL();
  launch_rows_any(b, lb, active, false);
  CKL();
  const long long threads = ((b->total_regions * b->fin_lanes + 31) / 32) * 32;
  const unsigned fblocks = (unsigned)((threads + 255) / 256);
#define SRWCR_FIN_CALL(G) \
  k_finalize_batch<G><<<fblocks, 256, 0, b->stream>>>(tab, b->n, b->total_regions, active)
  SRWCR_FIN_LANES_SWITCH(b->fin_lanes, SRWCR_FIN_CALL)
#undef SRWCR_FIN_CALL
  CKL();
  k_reduce_D_batch<<<b->n, 1024, 0, b->stream>>>(tab, active);
  CKL();
  if (b->ndim == 3) k_zcontract_batch<3><<<dim3(64, b->n), 256, 0, b->stream>>>(tab, active);
  else k_zcontract_batch<2><<<dim3(64, b->n), 256, 0, b->stream>>>(tab, active);
  CKL();
  launch_rows_any(b, lb, active, true);
  CKL();
  return SRWCR_OK;
}

int launches_per_eval(const srwcr_batch* b) {
  return 4 + (int)b->acc_launches.size() + (int)b->adj_launches.size();
}

// CTAs of a given dynamic shared-memory size that fit on one SM (228 KB of
// shared memory, 1 KB reserved per CTA).
int ctas_per_sm(size_t smem) { return (int)std::min<size_t>(4, (228 * 1024) / (smem + 1024)); }

srwcr_status queue_lbfgs_round(srwcr_batch* b, const LbOpts& o) {
  RET_IF(queue_batch_eval(b, true, b->active));
  LbVectors v{b->c, b->g, b->xn, b->gn, b->d, b->S, b->Y, b->off_dev, b->D};
  k_lbfgs_step<<<b->n, 1024, 0, b->stream>>>(b->lbs, b->active, v, o);
  CKL();
  return SRWCR_OK;
}

// Capture `fn` on the batch stream into an executable graph.
template <typename Fn>
srwcr_status capture(srwcr_batch* b, cudaGraphExec_t* out, Fn fn) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  srwcr_status st = fn();
  cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
  if (st != SRWCR_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(SRWCR_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(SRWCR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  return SRWCR_OK;
}

void invalidate_member_tables(srwcr_batch* b) {
  for (int i = 0; i < b->n; ++i) b->ctx[i]->lev[b->level[i]].tables = false;
}

srwcr_status batch_alloc_lbfgs(srwcr_batch* b, int m) {
  if (b->lb_m == m) return SRWCR_OK;
  if (b->graph_round) { cudaGraphExecDestroy(b->graph_round); b->graph_round = nullptr; }
  void* ptrs[] = {b->xn, b->gn, b->d, b->S, b->Y};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  b->xn = b->gn = b->d = b->S = b->Y = nullptr;
  b->lb_m = 0;
  const long long tot = b->off[b->n];
  CK(cudaMalloc((void**)&b->xn, sizeof(float) * tot));
  CK(cudaMalloc((void**)&b->gn, sizeof(float) * tot));
  CK(cudaMalloc((void**)&b->d, sizeof(float) * tot));
  CK(cudaMalloc((void**)&b->S, sizeof(float) * tot * m));
  CK(cudaMalloc((void**)&b->Y, sizeof(float) * tot * m));
  // Padding between pairs must read as zero in every inner product.
  CK(cudaMemsetAsync(b->xn, 0, sizeof(float) * tot, b->stream));
  CK(cudaMemsetAsync(b->gn, 0, sizeof(float) * tot, b->stream));
  CK(cudaMemsetAsync(b->d, 0, sizeof(float) * tot, b->stream));
  CK(cudaMemsetAsync(b->S, 0, sizeof(float) * tot * m, b->stream));
  CK(cudaMemsetAsync(b->Y, 0, sizeof(float) * tot * m, b->stream));
  if (!b->lbs) CK(cudaMalloc((void**)&b->lbs, sizeof(LbState) * b->n));
  if (!b->lb_max_iter) CK(cudaMalloc((void**)&b->lb_max_iter, sizeof(int) * b->n));
  // Evaluation table of the optimiser: reads xn, writes gn.
  std::vector<BatchPair> tab = b->host_tab;
  for (auto& bp : tab) {
    const long long o = (const float*)bp.acc.c - b->c;
    bp.acc.c = bp.adj.c = b->xn + o;
    bp.adj.grad = b->gn + o;
  }
  if (!b->tab_lb) CK(cudaMalloc((void**)&b->tab_lb, sizeof(BatchPair) * b->n));
  CK(cudaMemcpy(b->tab_lb, tab.data(), sizeof(BatchPair) * b->n, cudaMemcpyHostToDevice));
  for (auto& L : b->acc_launches)
    for (int k = 0; k < L.t.n; ++k) L.t_lb.it[k].a.c = b->xn + (L.t.it[k].a.c - b->c);
  for (auto& L : b->adj_launches)
    for (int k = 0; k < L.t.n; ++k) {
      const long long o = L.t.it[k].a.c - b->c;
      L.t_lb.it[k].a.c = b->xn + o;
      L.t_lb.it[k].a.grad = b->gn + o;
    }
  b->lb_m = m;
  return SRWCR_OK;
}

}  // namespace

extern "C" {

void srwcr_batch_destroy(srwcr_batch* b) {
  if (!b) return;
  if (b->graph_eval) cudaGraphExecDestroy(b->graph_eval);
  if (b->graph_round) cudaGraphExecDestroy(b->graph_round);
  void* ptrs[] = {b->c, b->g, b->D, b->ndeg, b->off_dev, b->tab_eval, b->tab_lb, b->xn, b->gn,
                  b->d, b->S, b->Y, b->lbs, b->lb_max_iter, b->active};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (b->active_host) cudaFreeHost(b->active_host);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

static srwcr_status batch_create_impl(srwcr_batch* b, srwcr_ctx* const* ctxs, const int* levels,
                                      int n, void* stream) {
  b->n = n;
  b->level.assign(levels, levels + n);
  b->ctx.assign(ctxs, ctxs + n);
  CK(cudaGetDevice(&b->device));
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  b->ndim = ctxs[0]->cfg.ndim;
  b->bf16 = is_bf16(ctxs[0]);
  for (int i = 0; i < n; ++i) {
    const srwcr_ctx* c = ctxs[i];
    if (!c) return fail(SRWCR_EINVAL, "pair %d: null context", i);
    if (c->device != b->device) return fail(SRWCR_EINVAL, "pair %d: context on another device", i);
    if (c->cfg.ndim != b->ndim || is_bf16(c) != b->bf16)
      return fail(SRWCR_EINVAL, "pair %d: dimension or storage differs from pair 0", i);
    const int level = levels[i];
    if (level < 0 || level >= c->nlev) return fail(SRWCR_EINVAL, "pair %d has no level %d", i, level);
    if (!c->lev[level].rows)
      return fail(SRWCR_EINVAL, "pair %d: level %d is not on the row-parallel kernels", i, level);
    if (c->cfg.role != SRWCR_ROLE_M_AS_B)
      return fail(SRWCR_EINVAL, "pair %d: the batched form takes the moving image as B", i);
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(SRWCR_EINVAL, "pair %d repeats pair %d", i, j);
  }
  // Packed coefficient layout (caller order), 64-float aligned per pair.
  b->off.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    const Geo& g = ctxs[i]->lev[levels[i]].g;
    const long long np = g.ncoef * b->ndim;
    b->off[i + 1] = b->off[i] + (np + 63) / 64 * 64;
  }
  const long long tot = b->off[n];
  CK(cudaMalloc((void**)&b->c, sizeof(float) * tot));
  CK(cudaMalloc((void**)&b->g, sizeof(float) * tot));
  CK(cudaMemsetAsync(b->c, 0, sizeof(float) * tot, b->stream));
  CK(cudaMemsetAsync(b->g, 0, sizeof(float) * tot, b->stream));
  CK(cudaMalloc((void**)&b->D, sizeof(double) * n));
  CK(cudaMalloc((void**)&b->ndeg, sizeof(int) * n));
  CK(cudaMalloc((void**)&b->active, sizeof(int) * n));
  CK(cudaMallocHost((void**)&b->active_host, sizeof(int) * n));
  CK(cudaMalloc((void**)&b->off_dev, sizeof(long long) * (n + 1)));
  CK(cudaMemcpy(b->off_dev, b->off.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice));

  // Table order: by launch group (x-bins per row), then by decreasing voxel
  // count, so the largest pairs' tiles are issued first.
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    const Level& la = ctxs[a]->lev[levels[a]];
    const Level& lc = ctxs[c]->lev[levels[c]];
    if (la.nxb_rows != lc.nxb_rows) return la.nxb_rows < lc.nxb_rows;
    return la.g.nvox > lc.g.nvox;
  });
  b->host_tab.resize(n);
  long long region = 0;
  for (int t = 0; t < n; ++t) {
    const int i = order[t];
    Level& lv = ctxs[i]->lev[levels[i]];
    BatchPair& bp = b->host_tab[t];
    memset(&bp, 0, sizeof bp);
    bp.g = lv.g;
    bp.id = i;
    float* ci = b->c + b->off[i];
    float* gi = b->g + b->off[i];
    bp.acc = acc_args(lv, ci, true);
    bp.adj = adj_args(lv, ci, nullptr, gi, true);
    bp.group = lv.nxb_rows;
    bp.region_begin = region;
    region += lv.g.R;
    bp.rs = region_static(lv);
    bp.inv_s1 = 1.0 / lv.s1;
    bp.inv_s2 = 1.0 / lv.s2;
    bp.invZ = 1.0 / lv.Z;
    bp.U = lv.U;
    bp.V = lv.V;
    bp.X = lv.X;
    bp.uvxz = lv.uvxz;
    bp.ubins = lv.ubins;
    bp.nu = lv.nu;
    bp.Dr = lv.Dr;
    bp.stats = lv.stats;
    bp.D = b->D + i;
    bp.ndeg = b->ndeg + i;
    bp.acc_len = lv.g.R * lv.g.nbins * 2;
    bp.grad_len = lv.g.ncoef * b->ndim;
    b->total_vox += lv.g.nvox;
  }
  b->total_regions = region;
  {
    // One launch finalises every pair: the first pair's explicit setting,
    // else the cost model over all pairs' region lists.
    const int req = ctxs[0]->cfg.finalize_lanes;
    std::vector<const std::vector<int>*> lists;
    for (int i = 0; i < n; ++i) lists.push_back(&ctxs[i]->lev[levels[i]].nz_ptr_host);
    b->fin_lanes = req > 0 ? req : finalize_lanes_auto(lists, ctxs[0]->device);
  }
  // Row-kernel launches: pairs bucketed by (x-bins per row, CTAs per SM),
  // in table order (largest first), at most kBatchChunk per launch.
  {
    std::vector<std::pair<std::pair<int, int>, std::vector<int>>> acc_b, adj_b;
    auto bucket = [](std::vector<std::pair<std::pair<int, int>, std::vector<int>>>& bs,
                     std::pair<int, int> key, int t) {
      for (auto& e : bs)
        if (e.first == key) { e.second.push_back(t); return; }
      bs.push_back({key, {t}});
    };
    for (int t = 0; t < n; ++t) {
      const Level& lv = ctxs[order[t]]->lev[levels[order[t]]];
      bucket(acc_b, {lv.nxb_rows, ctas_per_sm(lv.smem_acc_rows)}, t);
      bucket(adj_b, {lv.nxb_rows, ctas_per_sm(lv.smem_adj_rows)}, t);
    }
    for (const auto& e : acc_b) {
      for (size_t s0 = 0; s0 < e.second.size(); s0 += kBatchChunk) {
        srwcr_batch::AccLaunch L;
        memset(&L, 0, sizeof L);
        L.nxb = e.first.first;
        int tile = 0;
        for (size_t k = s0; k < std::min(e.second.size(), s0 + kBatchChunk); ++k) {
          const int t = e.second[k];
          const BatchPair& bp = b->host_tab[t];
          AccItem& it = L.t.it[L.t.n++];
          it.g = bp.g;
          it.a = bp.acc;
          it.id = bp.id;
          it.tile_begin = tile;
          tile += bp.g.ntile[0] * bp.g.ntile[1] * bp.g.ntile[2];
          L.smem = std::max(L.smem, ctxs[order[t]]->lev[levels[order[t]]].smem_acc_rows);
        }
        L.nblk = tile;
        L.t_lb = L.t;
        b->work_items += tile;
        b->acc_launches.push_back(L);
      }
    }
    for (const auto& e : adj_b) {
      for (size_t s0 = 0; s0 < e.second.size(); s0 += kBatchChunk) {
        srwcr_batch::AdjLaunch L;
        memset(&L, 0, sizeof L);
        L.nxb = e.first.first;
        int tile = 0;
        for (size_t k = s0; k < std::min(e.second.size(), s0 + kBatchChunk); ++k) {
          const int t = e.second[k];
          const BatchPair& bp = b->host_tab[t];
          AdjItem& it = L.t.it[L.t.n++];
          it.g = bp.g;
          it.a = bp.adj;
          it.id = bp.id;
          it.tile_begin = tile;
          tile += bp.g.ntile[0] * bp.g.ntile[1] * bp.g.ntile[2];
          L.smem = std::max(L.smem, ctxs[order[t]]->lev[levels[order[t]]].smem_adj_rows);
        }
        L.nblk = tile;
        L.t_lb = L.t;
        b->adj_launches.push_back(L);
      }
    }
  }
  CK(cudaMalloc((void**)&b->tab_eval, sizeof(BatchPair) * n));
  CK(cudaMemcpy(b->tab_eval, b->host_tab.data(), sizeof(BatchPair) * n, cudaMemcpyHostToDevice));
  RET_IF(set_smem_limits_batch());
  CK(cudaStreamSynchronize(b->stream));
  return SRWCR_OK;
}

srwcr_status srwcr_batch_create_levels(srwcr_ctx* const* ctxs, const int* levels, int n_pairs,
                                       void* stream, srwcr_batch** out) {
  if (!out) return fail(SRWCR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!ctxs || !levels || n_pairs < 1 || n_pairs > 65535)
    return fail(SRWCR_EINVAL, "need 1..65535 contexts and their levels");
  srwcr_batch* b = new (std::nothrow) srwcr_batch();
  if (!b) return fail(SRWCR_ENOMEM, "host allocation failed");
  srwcr_status st = batch_create_impl(b, ctxs, levels, n_pairs, stream);
  if (st != SRWCR_OK) {
    std::string keep = g_err;
    srwcr_batch_destroy(b);
    g_err = keep;
    return st;
  }
  *out = b;
  return SRWCR_OK;
}

srwcr_status srwcr_batch_create(srwcr_ctx* const* ctxs, int n_pairs, int level, void* stream,
                                srwcr_batch** out) {
  if (n_pairs < 1 || n_pairs > 65535) {
    if (out) *out = nullptr;
    return fail(SRWCR_EINVAL, "need 1..65535 contexts");
  }
  std::vector<int> levels(n_pairs, level);
  return srwcr_batch_create_levels(ctxs, levels.data(), n_pairs, stream, out);
}

srwcr_status srwcr_batch_info(const srwcr_batch* b, srwcr_batch_desc* out) {
  if (!b || !out) return fail(SRWCR_EINVAL, "null argument");
  out->n_pairs = b->n;
  out->launches_per_eval = launches_per_eval(b);
  out->n_params_total = b->off[b->n];
  out->n_voxels_total = b->total_vox;
  out->work_items = b->work_items;
  out->launches = b->launches;
  out->finalize_lanes = b->fin_lanes;
  return SRWCR_OK;
}

srwcr_status srwcr_batch_layout(const srwcr_batch* b, int64_t* offsets, int64_t* n_params) {
  if (!b) return fail(SRWCR_EINVAL, "null batch");
  for (int i = 0; i <= b->n && offsets; ++i) offsets[i] = b->off[i];
  for (int i = 0; i < b->n && n_params; ++i)
    n_params[i] = b->ctx[i]->lev[b->level[i]].g.ncoef * b->ndim;
  return SRWCR_OK;
}

srwcr_status srwcr_batch_buffers(srwcr_batch* b, float** c_dev, float** g_dev, double** D_dev) {
  if (!b) return fail(SRWCR_EINVAL, "null batch");
  if (c_dev) *c_dev = b->c;
  if (g_dev) *g_dev = b->g;
  if (D_dev) *D_dev = b->D;
  return SRWCR_OK;
}

srwcr_status srwcr_batch_value_and_grad(srwcr_batch* b, int use_graph) {
  if (!b) return fail(SRWCR_EINVAL, "null batch");
  if (use_graph) {
    if (!b->graph_eval)
      RET_IF(capture(b, &b->graph_eval, [&] { return queue_batch_eval(b, false, nullptr); }));
    CK(cudaGraphLaunch(b->graph_eval, b->stream));
  } else {
    RET_IF(queue_batch_eval(b, false, nullptr));
  }
  b->launches += launches_per_eval(b);
  invalidate_member_tables(b);
  return SRWCR_OK;
}

srwcr_status srwcr_batch_sync(srwcr_batch* b, double* D_host) {
  if (!b) return fail(SRWCR_EINVAL, "null batch");
  if (D_host) CK(cudaMemcpyAsync(D_host, b->D, sizeof(double) * b->n, cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return SRWCR_OK;
}

srwcr_status srwcr_batch_register(srwcr_batch* b, const srwcr_lbfgs_opts* opts, int use_graph,
                                  int* iterations, int* evaluations, double* final_value,
                                  int* status) {
  if (!b) return fail(SRWCR_EINVAL, "null batch");
  srwcr_lbfgs_opts oo;
  srwcr_lbfgs_default_opts(&oo);
  if (opts) oo = *opts;
  // Each pair runs at most opts->max_iter[its level] iterations.
  std::vector<int> mi(b->n);
  int mi_max = 0;
  for (int i = 0; i < b->n; ++i) {
    mi[i] = oo.max_iter[b->level[i]];
    mi_max = std::max(mi_max, mi[i]);
    if (mi[i] < 0) return fail(SRWCR_EINVAL, "negative max_iter for level %d", b->level[i]);
  }
  if (oo.m < 1 || oo.m > 16 || oo.max_ls < 1 || oo.stable_window >= kLbHist)
    return fail(SRWCR_EINVAL, "bad L-BFGS options (m in 1..16, max_ls >= 1, window < %d)", kLbHist);
  if (oo.penalty_weight != 0.0)
    return fail(SRWCR_EINVAL, "the batched driver minimises D alone (penalty_weight must be 0)");
  LbOpts o{oo.m, mi_max, oo.stable_window, oo.max_ls, oo.stable_rtol, oo.c1, oo.c2};
  RET_IF(batch_alloc_lbfgs(b, o.m));
  CK(cudaMemcpyAsync(b->lb_max_iter, mi.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice,
                     b->stream));
  k_lbfgs_init<<<b->n, 256, 0, b->stream>>>(b->lbs, b->active, b->off_dev, b->c, b->xn,
                                             b->lb_max_iter);
  CKL();
  b->launches += 1;
  if (use_graph && b->graph_round &&
      memcmp(&b->graph_round_opts, &o, sizeof o) != 0) {
    cudaGraphExecDestroy(b->graph_round);
    b->graph_round = nullptr;
  }
  if (use_graph && !b->graph_round) {
    RET_IF(capture(b, &b->graph_round, [&] { return queue_lbfgs_round(b, o); }));
    b->graph_round_opts = o;
  }
  // Every round spends one evaluation per active pair; a pair needs at most
  // 1 + max_iter * max_ls of them.
  const long long max_rounds = 1 + (long long)o.max_iter * o.max_ls;
  const int chunk = 4;
  long long rounds = 0;
  while (rounds < max_rounds) {
    for (int k = 0; k < chunk && rounds < max_rounds; ++k, ++rounds) {
      if (use_graph) CK(cudaGraphLaunch(b->graph_round, b->stream));
      else RET_IF(queue_lbfgs_round(b, o));
      b->launches += launches_per_eval(b) + 1;
    }
    CK(cudaMemcpyAsync(b->active_host, b->active, sizeof(int) * b->n, cudaMemcpyDeviceToHost,
                       b->stream));
    CK(cudaStreamSynchronize(b->stream));
    bool any = false;
    for (int i = 0; i < b->n; ++i) any = any || b->active_host[i] != 0;
    if (!any) break;
  }
  invalidate_member_tables(b);
  std::vector<LbState> hs(b->n);
  CK(cudaMemcpyAsync(hs.data(), b->lbs, sizeof(LbState) * b->n, cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  bool bad = false;
  for (int i = 0; i < b->n; ++i) {
    // Pairs still active ran out of rounds, which the bound above excludes;
    // report them as not converged.
    const int stt = b->active_host[i] ? SRWCR_ENOTCONVERGED : hs[i].status;
    if (iterations) iterations[i] = hs[i].iter;
    if (evaluations) evaluations[i] = hs[i].evals;
    if (final_value) final_value[i] = hs[i].f;
    if (status) status[i] = stt;
    bad = bad || stt == SRWCR_ENUMERIC;
  }
  // The batch's coefficient buffer holds each pair's accepted point and the
  // gradient buffer the gradient there.
  if (bad) return fail(SRWCR_ENUMERIC, "non-finite SRWCR value in the batch");
  return SRWCR_OK;
}

}  // extern "C"
