// Serving runtime: continuous batching of factor and append requests over
// many device-resident bases.
//
// Requests arrive (cqr_server_submit_*) in any order from any host thread.
// A request is admitted, in arrival order, once
//   * its target basis is idle (requests on one basis run in order),
//   * its transient device memory fits the HBM budget, and
//   * an executor is free: one of `slots` worker threads (each with its own
//     CUDA stream) for factors and large appends, or the batcher for small
//     appends.
// Admitted work overlaps on the device: workers run concurrently on their
// streams while the batcher runs all pending small appends together.
//
// Batched appends (Alg. 2 for several bases at once) run as persistent
// kernels over descriptor arrays held in device memory: one launch per step
// covers every problem in the batch.  The step sequence (init, Gramian
// sweep, reduction, control, then fused solve+Gramian passes) is captured
// once into CUDA graphs and replayed for every batch; only the descriptor
// contents change.  Each problem in a batch uses the CTA split, tile size and
// reduction order it would use alone, so its result is bitwise the same alone
// and in the mix.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_set>
#include <vector>

#include "cqr_internal.cuh"

using namespace cqr;

namespace {

constexpr int kSmallMaxP = 32;
constexpr int kGraphPasses = 3;  // fused passes in the first graph
constexpr int kMorePasses = 2;   // fused passes per follow-up graph

struct Request {
  uint64_t id = 0;
  int kind = 0;  // 0 factor, 1 append
  cqr_basis *b = nullptr;
  int64_t w = 0;  // n (factor) or p (append)
  const double *A = nullptr;
  int64_t lda = 0;
  cqr_opts opts{};
  size_t mem = 0;
  bool small = false;
  bool done = false;
  int status = 0;
  int batched = 0, batch_size = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  cqr_info info{};
};

// Fixed device workspace of the batcher (pointers stay valid for the graphs).
struct BatchWS {
  int cap = 0, max_items = 0, max_red = 0;
  size_t part_doubles = 0, c_doubles = 0, bt_doubles = 0;
  char *dev = nullptr;   // descriptors + items + counts (copied from host each batch)
  char *host = nullptr;  // pinned mirror
  size_t desc_bytes = 0;
  // device views
  RowSweep *d_gram = nullptr, *d_first = nullptr, *d_next = nullptr;
  Reduce *d_red = nullptr;
  Ctrl *d_ctrl = nullptr;
  int *d_item_req = nullptr, *d_item_cta = nullptr, *d_red_req = nullptr, *d_red_chunk = nullptr;
  int *d_counts = nullptr;  // [0] nitems, [1] nred, [2] nreq
  // per-problem scratch
  DevState *d_st = nullptr;
  double *d_C = nullptr, *d_Rt = nullptr, *d_Rd = nullptr, *d_Bt = nullptr, *d_part = nullptr;
  DevState *h_st = nullptr;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t g_start = nullptr, g_more = nullptr;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct cqr_server {
  cqr_server_opts o{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_batch, cv_done;
  std::deque<Request *> pending, work_q, batch_q;
  std::vector<Request *> all;
  std::unordered_set<cqr_basis *> busy;
  size_t mem_in_use = 0;
  int idle_workers = 0;
  int running = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::thread batcher;
  BatchWS ws;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

// Transient device memory of one request (what admission budgets for).
size_t request_mem(const Request &r) {
  const int64_t m = r.b->m;
  const int q = (r.kind == 0) ? 0 : (int)r.b->q;
  const int p = (int)r.w;
  int tr, lds;
  size_t smem;
  rowsweep_geometry(q, p, &tr, &lds, &smem);
  const int G = rowsweep_grid(m, tr);
  const size_t E = (size_t)q * p + (size_t)p * (p + 1) / 2;
  size_t bytes = 8 * ((size_t)G * E + (size_t)(q + p) * p + (size_t)p * p + (size_t)std::max(q, 1) * p) + 4096;
  if (r.kind == 0) bytes += 8 * ((size_t)m * p + (size_t)p * p);  // staging Q and R
  return bytes;
}

bool is_small_append(const cqr_server *s, const Request &r) {
  if (r.kind != 1) return false;
  const int64_t q = r.b->q, p = r.w;
  const int64_t E = q * p + p * (p + 1) / 2;
  // a basis with a digit cache takes basis_append, which keeps the cache;
  // so does an append past the capacity, which basis_append rejects (the
  // batched launch writes the new columns without that check)
  return p <= kSmallMaxP && E <= (int64_t)kThreads * kBatchEPT && r.b->m <= s->o.small_rows &&
         s->ws.cap > 0 && r.b->Qd == nullptr && q + p <= r.b->n_max;
}

void finish_locked(cqr_server *s, Request *r) {
  r->done = true;
  r->t_done = s->now();
  s->mem_in_use -= r->mem;
  s->busy.erase(r->b);
  --s->running;
}

// Admit pending requests in arrival order.  A request whose basis is busy
// waits (its basis's order is kept); the first request that does not fit the
// budget stops admission so that large requests are not starved.
void dispatch_locked(cqr_server *s) {
  std::unordered_set<cqr_basis *> seen;  // keep per-basis order among pending
  for (auto it = s->pending.begin(); it != s->pending.end();) {
    Request *r = *it;
    if (s->busy.count(r->b) || seen.count(r->b)) {
      seen.insert(r->b);
      ++it;
      continue;
    }
    if (s->mem_in_use + r->mem > (size_t)s->o.hbm_budget_bytes && s->running > 0) break;
    r->small = is_small_append(s, *r);
    if (!r->small && s->idle_workers == 0) {
      seen.insert(r->b);
      ++it;
      continue;
    }
    s->mem_in_use += r->mem;
    s->busy.insert(r->b);
    ++s->running;
    it = s->pending.erase(it);
    if (r->small) {
      s->batch_q.push_back(r);
      s->cv_batch.notify_one();
    } else {
      --s->idle_workers;
      s->work_q.push_back(r);
      s->cv_work.notify_one();
    }
  }
}

// ---- worker: one request at a time on its own stream
void execute_single(cqr_server *s, Request *r, cudaStream_t str) {
  cqr_basis *b = r->b;
  if (r->kind == 1) {
    r->status = basis_append(b, r->w, r->A, r->lda, &r->info, str);
    return;
  }
  const int64_t m = b->m, n = r->w;
  if (n > b->n_max) {
    r->status = CQR_ERR_CAPACITY;
    return;
  }
  double *Qs = nullptr, *Rs = nullptr;
  cudaError_t e = cudaMallocAsync((void **)&Qs, sizeof(double) * (size_t)m * n, str);
  if (e == cudaSuccess) e = cudaMallocAsync((void **)&Rs, sizeof(double) * (size_t)n * n, str);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    if (Qs) cudaFreeAsync(Qs, str);
    r->status = CQR_ERR_OOM;
    return;
  }
  cqr_status st = cholqr_factor(&r->opts, m, n, r->A, r->lda, Qs, m, Rs, n, &r->info, str);
  if (st >= 0) {
    // the factor replaces the basis: Q -> columns 0..n-1, R -> leading block
    e = cudaMemcpy2DAsync(b->Q, sizeof(double) * b->ldq, Qs, sizeof(double) * m,
                          sizeof(double) * m, n, cudaMemcpyDeviceToDevice, str);
    if (e == cudaSuccess)
      e = cudaMemset2DAsync(b->R, sizeof(double) * b->ldr, 0, sizeof(double) * b->n_max, b->n_max, str);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(b->R, sizeof(double) * b->ldr, Rs, sizeof(double) * n, sizeof(double) * n,
                            n, cudaMemcpyDeviceToDevice, str);
    // the basis's digit cache (if it keeps one) follows its new columns
    if (e == cudaSuccess && b->Qd != nullptr)
      e = launch_cache_fill(b->Q, b->ldq, m, 0, (int)n, b->Qe, b->Qd, b->ldc, b->ldc * b->n_max, str);
    if (e == cudaSuccess) e = cudaStreamSynchronize(str);
    if (e == cudaSuccess) b->q = n;
    else st = CQR_ERR_CUDA;
  }
  cudaFreeAsync(Qs, str);
  cudaFreeAsync(Rs, str);
  cudaStreamSynchronize(str);
  (void)cudaGetLastError();
  r->status = st;
}

void worker_loop(cqr_server *s) {
  cudaSetDevice(s->device);
  cudaStream_t str;
  cudaStreamCreateWithFlags(&str, cudaStreamNonBlocking);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_work.wait(lk, [&] { return s->stop || !s->work_q.empty(); });
    if (s->work_q.empty() && s->stop) break;
    Request *r = s->work_q.front();
    s->work_q.pop_front();
    r->t_start = s->now();
    lk.unlock();
    execute_single(s, r, str);
    lk.lock();
    finish_locked(s, r);
    ++s->idle_workers;
    dispatch_locked(s);
    s->cv_done.notify_all();
  }
  lk.unlock();
  cudaStreamDestroy(str);
}

// ---- batcher
cudaError_t batch_ws_create(BatchWS &w, int cap, int device) {
  cudaSetDevice(device);
  w.cap = cap;
  const int G = 2 * num_sms();
  w.max_items = cap * G;
  const int E = kThreads * kBatchEPT;
  w.max_red = cap * ((E + 63) / 64);
  w.part_doubles = (size_t)G * E;
  w.c_doubles = (size_t)E + kSmallMaxP * kSmallMaxP;  // (q+p) p = qp + p^2 <= E + p^2
  w.bt_doubles = (size_t)E;
  w.desc_bytes = al(3 * cap * sizeof(RowSweep)) + al(cap * sizeof(Reduce)) + al(cap * sizeof(Ctrl)) +
                 al(2 * w.max_items * sizeof(int)) + al(2 * w.max_red * sizeof(int)) + al(4 * sizeof(int));
  const size_t scratch = al(cap * sizeof(DevState)) +
                         8 * (size_t)cap * (w.c_doubles + kSmallMaxP * kSmallMaxP + kSmallMaxP + w.bt_doubles +
                                            w.part_doubles) + 4096 * 8;
  cudaError_t e = cudaMalloc((void **)&w.dev, w.desc_bytes + scratch);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&w.host, w.desc_bytes);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&w.h_st, cap * sizeof(DevState));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return e;
  char *p = w.dev;
  w.d_gram = (RowSweep *)p;
  w.d_first = w.d_gram + cap;
  w.d_next = w.d_first + cap;
  p += al(3 * cap * sizeof(RowSweep));
  w.d_red = (Reduce *)p;
  p += al(cap * sizeof(Reduce));
  w.d_ctrl = (Ctrl *)p;
  p += al(cap * sizeof(Ctrl));
  w.d_item_req = (int *)p;
  w.d_item_cta = w.d_item_req + w.max_items;
  p += al(2 * w.max_items * sizeof(int));
  w.d_red_req = (int *)p;
  w.d_red_chunk = w.d_red_req + w.max_red;
  p += al(2 * w.max_red * sizeof(int));
  w.d_counts = (int *)p;
  p += al(4 * sizeof(int));
  // scratch
  w.d_st = (DevState *)p;
  p += al(cap * sizeof(DevState));
  double *d = (double *)p;
  w.d_C = d;
  d += (size_t)cap * w.c_doubles;
  w.d_Rt = d;
  d += (size_t)cap * kSmallMaxP * kSmallMaxP;
  w.d_Rd = d;
  d += (size_t)cap * kSmallMaxP;
  w.d_Bt = d;
  d += (size_t)cap * w.bt_doubles;
  w.d_part = d;
  return cudaSuccess;
}

// The launches of one graph, on the capturing stream.
cudaError_t batch_launches(BatchWS &w, bool start, int passes) {
  const int grid = 2 * num_sms();
  const size_t smem_tile = 196608;
  const size_t smem_ctrl = ctrl_smem_bytes(kSmallMaxP);
  cudaError_t e = cudaSuccess;
  auto red = [&]() {
    return launch_reduce_batched(w.d_red, w.d_red_req, w.d_red_chunk, w.d_counts + 1, grid, w.stream);
  };
  auto ctl = [&]() { return launch_ctrl_batched(w.d_ctrl, w.d_counts + 2, w.cap, smem_ctrl, w.stream); };
  if (start) {
    e = launch_init_batched(w.d_ctrl, w.d_counts + 2, w.cap, w.stream);
    if (e == cudaSuccess)
      e = launch_rowsweep_batched(w.d_gram, w.d_item_req, w.d_item_cta, w.d_counts, grid, smem_tile, w.stream);
    if (e == cudaSuccess) e = red();
    if (e == cudaSuccess) e = ctl();
    if (e == cudaSuccess)
      e = launch_rowsweep_batched(w.d_first, w.d_item_req, w.d_item_cta, w.d_counts, grid, smem_tile, w.stream);
    if (e == cudaSuccess) e = red();
    if (e == cudaSuccess) e = ctl();
    passes -= 1;
  }
  for (int k = 0; e == cudaSuccess && k < passes; ++k) {
    e = launch_rowsweep_batched(w.d_next, w.d_item_req, w.d_item_cta, w.d_counts, grid, smem_tile, w.stream);
    if (e == cudaSuccess) e = red();
    if (e == cudaSuccess) e = ctl();
  }
  return e;
}

cudaError_t capture(BatchWS &w, bool start, int passes, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(w.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t el = batch_launches(w, start, passes);
  e = cudaStreamEndCapture(w.stream, &g);
  if (el != cudaSuccess) e = el;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

// Runs Alg. 2 for every request of the batch (distinct bases, all small).
void run_batch(cqr_server *s, std::vector<Request *> &rs) {
  BatchWS &w = s->ws;
  const int nreq = (int)rs.size();
  char *h = w.host;
  RowSweep *hg = (RowSweep *)h, *hf = hg + w.cap, *hn = hf + w.cap;
  char *p = h + al(3 * w.cap * sizeof(RowSweep));
  Reduce *hr = (Reduce *)p;
  p += al(w.cap * sizeof(Reduce));
  Ctrl *hc = (Ctrl *)p;
  p += al(w.cap * sizeof(Ctrl));
  int *item_req = (int *)p, *item_cta = item_req + w.max_items;
  p += al(2 * w.max_items * sizeof(int));
  int *red_req = (int *)p, *red_chunk = red_req + w.max_red;
  p += al(2 * w.max_red * sizeof(int));
  int *counts = (int *)p;
  int nitems = 0, nred = 0;
  for (int r = 0; r < nreq; ++r) {
    Request *rq = rs[r];
    cqr_basis *b = rq->b;
    const int q = (int)b->q, pw = (int)rq->w;
    int tr, lds;
    size_t smem;
    rowsweep_geometry(q, pw, &tr, &lds, &smem);
    const int G = rowsweep_grid(b->m, tr);
    const int64_t tiles = (b->m + tr - 1) / tr;
    const int64_t E = (int64_t)q * pw + (int64_t)pw * (pw + 1) / 2;
    RowSweep a{};
    a.m = b->m;
    a.q = q;
    a.p = pw;
    a.Qin = b->Q;
    a.ldqin = b->ldq;
    a.Yin = rq->A;
    a.ldyin = rq->lda;
    a.Yout = b->Q + (int64_t)q * b->ldq;
    a.ldyout = b->ldq;
    a.Rt = w.d_Rt + (size_t)r * kSmallMaxP * kSmallMaxP;
    a.Rdinv = w.d_Rd + (size_t)r * kSmallMaxP;
    a.Bt = w.d_Bt + (size_t)r * w.bt_doubles;
    a.partials = w.d_part + (size_t)r * w.part_doubles;
    a.E = E;
    a.rows_per_cta = ((tiles + G - 1) / G) * tr;
    a.tile_rows = tr;
    a.lds = lds;
    a.st = w.d_st + r;
    a.do_trsm = 0;
    hg[r] = a;
    a.do_trsm = 1;
    hf[r] = a;
    a.Yin = a.Yout;
    a.ldyin = a.ldyout;
    hn[r] = a;
    Reduce rd{a.partials, G, E, q, pw, w.d_C + (size_t)r * w.c_doubles, a.st};
    hr[r] = rd;
    Ctrl c{};
    c.m = b->m;
    c.q = q;
    c.p = pw;
    c.mode = MODE_UPDATE;
    c.shift_policy = b->opts.shift_policy;
    c.max_iter = b->opts.max_iter;
    c.min_iter = b->opts.update_min_iter;
    c.max_escalations = b->opts.max_escalations;
    c.stop_rule = b->opts.stop_rule;
    c.tol = b->opts.tol;
    c.first_shift_coeff = 0.0;
    c.C = rd.C;
    c.Rt = (double *)a.Rt;
    c.Rdinv = (double *)a.Rdinv;
    c.Bt = (double *)a.Bt;
    c.R = b->R + q + (int64_t)q * b->ldr;
    c.ldr = b->ldr;
    c.B = (q > 0) ? b->R + (int64_t)q * b->ldr : nullptr;
    c.ldb = b->ldr;
    c.st = w.d_st + r;
    hc[r] = c;
    for (int g = 0; g < G; ++g) {
      item_req[nitems] = r;
      item_cta[nitems] = g;
      ++nitems;
    }
    for (int ch = 0; ch < (int)((E + 63) / 64); ++ch) {
      red_req[nred] = r;
      red_chunk[nred] = ch;
      ++nred;
    }
  }
  counts[0] = nitems;
  counts[1] = nred;
  counts[2] = nreq;
  counts[3] = 0;
  cudaError_t e = cudaMemcpyAsync(w.dev, w.host, w.desc_bytes, cudaMemcpyHostToDevice, w.stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(w.g_start, w.stream);
  int launched = kGraphPasses;
  int max_iter = 0;
  for (Request *rq : rs) max_iter = std::max(max_iter, rq->b->opts.max_iter);
  while (e == cudaSuccess) {
    e = cudaMemcpyAsync(w.h_st, w.d_st, nreq * sizeof(DevState), cudaMemcpyDeviceToHost, w.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w.stream);
    if (e != cudaSuccess) break;
    bool all = true;
    for (int r = 0; r < nreq; ++r) all = all && w.h_st[r].done;
    if (all || launched >= max_iter) break;
    e = cudaGraphLaunch(w.g_more, w.stream);
    launched += kMorePasses;
  }
  for (int r = 0; r < nreq; ++r) {
    Request *rq = rs[r];
    rq->batched = 1;
    rq->batch_size = nreq;
    if (e != cudaSuccess) {
      rq->status = CQR_ERR_CUDA;
      continue;
    }
    const DevState &st = w.h_st[r];
    if (!st.done) {
      rq->status = CQR_ERR_CUDA;
      continue;
    }
    rq->status = st.status;
    rq->info.iters = st.iters;
    rq->info.chol_attempts = st.chol_attempts;
    rq->info.shifts = st.shifts;
    rq->info.escalations = st.escalations;
    rq->info.sigma_first = st.sigma_first;
    rq->info.sigma_last = st.sigma_last;
    rq->info.orth_frob = st.orth_frob;
    rq->info.proj_frob = st.proj_frob;
    cqr_basis *b = rq->b;
    if (st.status >= 0) {
      if (st.iters == 0)
        cudaMemcpy2DAsync(b->Q + b->q * b->ldq, sizeof(double) * b->ldq, rq->A, sizeof(double) * rq->lda,
                          sizeof(double) * b->m, rq->w, cudaMemcpyDeviceToDevice, w.stream);
      b->q += rq->w;
    }
  }
  cudaStreamSynchronize(w.stream);
  (void)cudaGetLastError();
}

void batcher_loop(cqr_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    s->cv_batch.wait(lk, [&] { return s->stop || !s->batch_q.empty(); });
    if (s->batch_q.empty() && s->stop) break;
    std::vector<Request *> rs;
    while (!s->batch_q.empty() && (int)rs.size() < s->ws.cap) {
      rs.push_back(s->batch_q.front());
      s->batch_q.pop_front();
    }
    const double ts = s->now();
    for (Request *r : rs) r->t_start = ts;
    lk.unlock();
    run_batch(s, rs);
    lk.lock();
    for (Request *r : rs) finish_locked(s, r);
    dispatch_locked(s);
    s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

void cqr_server_default_opts(cqr_server_opts *o) {
  if (o == nullptr) return;
  o->slots = 4;
  o->batch_max = 16;
  o->hbm_budget_bytes = (int64_t)8 << 30;
  o->small_rows = 262144;
}

cqr_status cqr_server_create(const cqr_server_opts *opts, cqr_server **out) {
  if (out == nullptr) return CQR_ERR_INVALID;
  *out = nullptr;
  cqr_server_opts o;
  cqr_server_default_opts(&o);
  if (opts != nullptr) o = *opts;
  if (o.slots < 1 || o.slots > 64 || o.batch_max < 0 || o.batch_max > 256 || o.hbm_budget_bytes <= 0 ||
      o.small_rows < 0)
    return CQR_ERR_INVALID;
  cqr_server *s = new (std::nothrow) cqr_server();
  if (s == nullptr) return CQR_ERR_OOM;
  s->o = o;
  cudaGetDevice(&s->device);
  s->t0 = std::chrono::steady_clock::now();
  if (o.batch_max > 0) {
    cudaError_t e = batch_ws_create(s->ws, o.batch_max, s->device);
    // graphs: a no-op launch first (sets kernel attributes outside capture)
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ws.dev, 0, s->ws.desc_bytes, s->ws.stream);
    if (e == cudaSuccess) e = batch_launches(s->ws, true, kGraphPasses);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->ws.stream);
    if (e == cudaSuccess) e = capture(s->ws, true, kGraphPasses, &s->ws.g_start);
    if (e == cudaSuccess) e = capture(s->ws, false, kMorePasses, &s->ws.g_more);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      if (s->ws.dev) cudaFree(s->ws.dev);
      if (s->ws.host) cudaFreeHost(s->ws.host);
      if (s->ws.h_st) cudaFreeHost(s->ws.h_st);
      delete s;
      return e == cudaErrorMemoryAllocation ? CQR_ERR_OOM : CQR_ERR_CUDA;
    }
  }
  s->idle_workers = o.slots;
  for (int i = 0; i < o.slots; ++i) s->workers.emplace_back(worker_loop, s);
  if (o.batch_max > 0) s->batcher = std::thread(batcher_loop, s);
  *out = s;
  return CQR_OK;
}

static cqr_status submit(cqr_server *s, Request *r, uint64_t *ticket) {
  r->mem = request_mem(*r);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return CQR_ERR_INVALID;
  }
  r->id = s->all.size();
  r->t_submit = s->now();
  s->all.push_back(r);
  s->pending.push_back(r);
  if (ticket) *ticket = r->id;
  dispatch_locked(s);
  return CQR_OK;
}

cqr_status cqr_server_submit_factor(cqr_server *s, cqr_basis *b, int64_t n, const double *A, int64_t lda,
                                    const cqr_opts *opts, uint64_t *ticket) {
  if (s == nullptr || b == nullptr || A == nullptr) return CQR_ERR_INVALID;
  if (n < 1 || n > CQR_MAX_N || n > b->n_max || b->m < n || lda < b->m) return CQR_ERR_INVALID;
  Request *r = new (std::nothrow) Request();
  if (r == nullptr) return CQR_ERR_OOM;
  r->kind = 0;
  r->b = b;
  r->w = n;
  r->A = A;
  r->lda = lda;
  cqr_default_opts(&r->opts);
  if (opts != nullptr) r->opts = *opts;
  return submit(s, r, ticket);
}

cqr_status cqr_server_submit_append(cqr_server *s, cqr_basis *b, int64_t p, const double *A_in,
                                    int64_t lda, uint64_t *ticket) {
  if (s == nullptr || b == nullptr || A_in == nullptr) return CQR_ERR_INVALID;
  if (p < 1 || p > CQR_MAX_N || lda < b->m) return CQR_ERR_INVALID;
  {
    // as basis_append: the block must not overlap the basis storage
    const char *a0 = (const char *)A_in, *a1 = (const char *)(A_in + lda * (p - 1) + b->m);
    const char *q0 = (const char *)b->Q, *q1 = (const char *)(b->Q + b->ldq * b->n_max);
    if (a0 < q1 && q0 < a1) return CQR_ERR_INVALID;
  }
  Request *r = new (std::nothrow) Request();
  if (r == nullptr) return CQR_ERR_OOM;
  r->kind = 1;
  r->b = b;
  r->w = p;
  r->A = A_in;
  r->lda = lda;
  r->opts = b->opts;
  return submit(s, r, ticket);
}

cqr_status cqr_server_wait(cqr_server *s, uint64_t ticket, cqr_request_result *out) {
  if (s == nullptr) return CQR_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket >= s->all.size()) return CQR_ERR_INVALID;
  Request *r = s->all[ticket];
  s->cv_done.wait(lk, [&] { return r->done; });
  if (out != nullptr) {
    out->status = r->status;
    out->kind = r->kind;
    out->batched = r->batched;
    out->batch_size = r->batch_size;
    out->t_submit = r->t_submit;
    out->t_start = r->t_start;
    out->t_done = r->t_done;
    out->info = r->info;
  }
  return CQR_OK;
}

cqr_status cqr_server_drain(cqr_server *s) {
  if (s == nullptr) return CQR_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait(lk, [&] { return s->pending.empty() && s->running == 0; });
  return CQR_OK;
}

double cqr_server_now(const cqr_server *s) { return s ? s->now() : -1.0; }

cqr_status cqr_server_destroy(cqr_server *s) {
  if (s == nullptr) return CQR_OK;
  cqr_server_drain(s);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_batch.notify_all();
  for (auto &t : s->workers) t.join();
  if (s->batcher.joinable()) s->batcher.join();
  if (s->ws.g_start) cudaGraphExecDestroy(s->ws.g_start);
  if (s->ws.g_more) cudaGraphExecDestroy(s->ws.g_more);
  if (s->ws.stream) cudaStreamDestroy(s->ws.stream);
  if (s->ws.dev) cudaFree(s->ws.dev);
  if (s->ws.host) cudaFreeHost(s->ws.host);
  if (s->ws.h_st) cudaFreeHost(s->ws.h_st);
  for (Request *r : s->all) delete r;
  delete s;
  return CQR_OK;
}

}  // extern "C"
