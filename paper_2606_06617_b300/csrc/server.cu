// Request server: continuous batching of independent structures over batch
// plans (include/pswf_lr.h, "request server").
//
// Structures are routed to the smallest grid bucket that holds their box at
// the server's largest grid spacing h_max.  Each bucket owns a fixed number
// of batch contexts (a batch plan on its own stream, device buffers for one
// batch, pinned staging); device memory is therefore bounded at creation and
// a request waits in its bucket's queue until a context is free (admission
// by memory).  A scheduler thread takes, for every free context, the
// bucket's oldest pending requests up to the context's structure and atom
// capacity, stages them, and launches: table and input copies, the batch
// kernels (a captured CUDA graph per context and launch size -- a power of
// two >= the batch's structures -- replayed for every batch of that size:
// the plan's launch shapes depend only on that size), output copies, and
// a host callback that marks the context finished.  Requests that arrive
// while batches run are admitted as soon as a context frees up; batches of
// different contexts overlap on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "deadline.hpp"
#include "internal.hpp"
#include "pswf_lr.h"

namespace {

using Clock = std::chrono::steady_clock;

// A structure in flight.  Charges and results are held in the server's
// precision (rs bytes a value): the submitting thread converts the charges,
// the waiting thread converts the results it asks for, so the scheduler
// thread only copies.  Finished requests return to a pool and keep their
// buffers' capacity, so a stream of requests does not allocate.
struct Request {
  int64_t id = 0;
  int64_t n = 0;
  double box[3] = {0, 0, 0};
  std::vector<int> ps;          // [K]
  std::vector<double> pos;      // [n][3]
  std::vector<char> q;          // real [K][n]
  // borrowed inputs (pswf_server_submit_many with PSWF_SUBMIT_BORROW): the
  // caller's arrays, read when the batch is staged; null when copied
  const double* pos_ref = nullptr;   // [n][3]
  const double* q_ref = nullptr;     // [K][n]
  int bucket = 0;
  int status = 1;               // 1 pending, 0 done, < 0 failed
  Clock::time_point t_submit, t_done;
  std::vector<double> energy;   // [K + 1]
  std::vector<char> phi;        // real [K][n]
  std::vector<char> forces;     // real [n][3]
};

constexpr size_t kRequestPool = 8192;   // finished requests kept for reuse

struct Context {
  pswf_plan plan = nullptr;
  cudaStream_t stream = nullptr;
  void* ws = nullptr;
  double* d_pos = nullptr;   // [n_max][3]
  void* d_q = nullptr;       // real [K][n_max]
  double* d_e = nullptr;     // [b_max][K + 1]
  void* d_phi = nullptr;     // real [K][n_max]
  void* d_f = nullptr;       // real [n_max][3]
  double* h_pos = nullptr;   // pinned mirrors
  void* h_q = nullptr;
  double* h_e = nullptr;
  void* h_phi = nullptr;
  void* h_f = nullptr;
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;   // per launch size
  bool busy = false;
  bool finished = false;     // set by the host callback
  std::vector<Request*> reqs;
  std::vector<int64_t> offsets;
  struct pswf_server_s* srv = nullptr;
};

struct Bucket {
  int grid = 0;
  int b_max = 0;
  int64_t n_max = 0;
  double box_max[3] = {0, 0, 0};
  std::deque<Request*> pending;
  std::vector<std::unique_ptr<Context>> ctx;
};

}  // namespace

struct pswf_server_s {
  pswf_server_opts opt{};
  int K = 0;
  size_t rs = 4;
  int device = 0;
  std::vector<std::unique_ptr<Bucket>> buckets;
  std::unordered_map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<std::unique_ptr<Request>> pool;   // finished requests (pool_mu)
  std::mutex pool_mu;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::thread th;
  bool stop = false;
  bool paused = false;       // pswf_server_pause: no new batches are started
  int64_t next_id = 1;
  int64_t n_batches = 0, n_requests = 0, n_atoms = 0;
  int fatal = 0;
  std::string error;
};

namespace {

int cuda_ok(pswf_server srv, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return PSWF_OK;
  srv->error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? PSWF_ENOMEM : PSWF_ECUDA;
}

void CUDART_CB on_batch_done(void* arg) {
  Context* c = static_cast<Context*>(arg);
  pswf_server srv = c->srv;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    c->finished = true;
  }
  srv->cv_sched.notify_one();
}

int make_context(pswf_server srv, Bucket& b, Context& c) {
  const pswf_server_opts& o = srv->opt;
  const int K = srv->K;
  const size_t rs = srv->rs;
  int rc;
  c.srv = srv;
  if ((rc = cuda_ok(srv, cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "stream"))) return rc;
  pswf_opts po;
  pswf_opts_default(&po);
  po.tol = o.tol;
  po.r_c = o.r_c;
  po.c = o.c;
  po.P = o.P;
  po.precision = o.precision;
  for (int d = 0; d < 3; ++d) po.grid[d] = b.grid;
  if ((rc = pswf_batch_plan_create(b.box_max, b.b_max, b.n_max, K, o.pset, o.npset, &po, c.stream, &c.plan))) {
    srv->error = "batch plan for grid " + std::to_string(b.grid) + ": " + pswf_strerror(rc);
    return rc;
  }
  pswf_info info;
  pswf_plan_info(c.plan, &info);
  if ((rc = cuda_ok(srv, cudaMalloc(&c.ws, size_t(info.workspace_bytes)), "workspace"))) return rc;
  if ((rc = pswf_plan_set_workspace(c.plan, c.ws, info.workspace_bytes))) {
    srv->error = "workspace";
    return rc;
  }
  const size_t n = size_t(std::max<int64_t>(b.n_max, 1));
  if ((rc = cuda_ok(srv, cudaMalloc(&c.d_pos, n * 3 * 8), "buffers"))) return rc;
  if ((rc = cuda_ok(srv, cudaMalloc(&c.d_q, n * K * rs), "buffers"))) return rc;
  if ((rc = cuda_ok(srv, cudaMalloc(&c.d_e, size_t(b.b_max) * (K + 1) * 8), "buffers"))) return rc;
  if ((rc = cuda_ok(srv, cudaMalloc(&c.d_phi, n * K * rs), "buffers"))) return rc;
  if ((rc = cuda_ok(srv, cudaMalloc(&c.d_f, n * 3 * rs), "buffers"))) return rc;
  if ((rc = cuda_ok(srv, cudaMallocHost(&c.h_pos, n * 3 * 8), "pinned"))) return rc;
  if ((rc = cuda_ok(srv, cudaMallocHost(&c.h_q, n * K * rs), "pinned"))) return rc;
  if ((rc = cuda_ok(srv, cudaMallocHost(&c.h_e, size_t(b.b_max) * (K + 1) * 8), "pinned"))) return rc;
  if ((rc = cuda_ok(srv, cudaMallocHost(&c.h_phi, n * K * rs), "pinned"))) return rc;
  if ((rc = cuda_ok(srv, cudaMallocHost(&c.h_f, n * 3 * rs), "pinned"))) return rc;
  return PSWF_OK;
}

void free_context(Context& c) {
  if (c.stream) cudaStreamSynchronize(c.stream);
  for (auto& g : c.graphs) cudaGraphExecDestroy(g.second);
  if (c.plan) pswf_plan_destroy(c.plan);
  for (void* p : {static_cast<void*>(c.d_pos), c.d_q, static_cast<void*>(c.d_e), c.d_phi, c.d_f, c.ws})
    if (p) cudaFree(p);
  for (void* p : {static_cast<void*>(c.h_pos), c.h_q, static_cast<void*>(c.h_e), c.h_phi, c.h_f})
    if (p) cudaFreeHost(p);
  if (c.stream) cudaStreamDestroy(c.stream);
}

// The context's graph of set_points + execute for the plan's current run
// size (captured on first use).
int graph_for_run(pswf_server srv, Bucket& b, Context& c, cudaGraphExec_t* out) {
  const int nrun = pswf::plan_run_size(c.plan);
  for (auto& g : c.graphs)
    if (g.first == nrun) {
      *out = g.second;
      return PSWF_OK;
    }
  int rc;
  cudaGraph_t g = nullptr;
  if ((rc = cuda_ok(srv, cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeRelaxed), "begin capture"))) return rc;
  int rc1 = pswf::plan_run_set_points(c.plan, b.n_max, c.d_pos, 1, c.d_q);
  int rc2 = rc1 ? rc1 : pswf::plan_run_execute(c.plan, c.d_e, c.d_phi, c.d_f);
  const cudaError_t ec = cudaStreamEndCapture(c.stream, &g);
  if (rc2) {
    if (g) cudaGraphDestroy(g);
    srv->error = pswf::plan_error(c.plan);
    return rc2;
  }
  if ((rc = cuda_ok(srv, ec, "end capture"))) return rc;
  cudaGraphExec_t gexec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&gexec, g, 0);
  cudaGraphDestroy(g);
  if ((rc = cuda_ok(srv, ei, "graph instantiate"))) return rc;
  c.graphs.emplace_back(nrun, gexec);
  *out = gexec;
  return PSWF_OK;
}

// Captures the context's graphs for every run size ahead of serving, so no
// capture (milliseconds each) delays a request: tables of `size` empty
// structures set the run size; nothing is launched.
int precapture(pswf_server srv, Bucket& b, Context& c) {
  int count = 0;
  const int* sizes = pswf::plan_run_sizes(c.plan, &count);
  const std::vector<int> runs(sizes, sizes + count);
  const int K = srv->K;
  for (int sz : runs) {
    std::vector<double> boxes(size_t(sz) * 3, 0.5 * b.box_max[0]);
    std::vector<int> ps(size_t(sz) * K, srv->opt.pset[0]);
    std::vector<int64_t> offsets(size_t(sz) + 1, 0);
    int rc;
    if ((rc = pswf::plan_fill_tables(c.plan, sz, boxes.data(), ps.data(), offsets.data()))) {
      srv->error = pswf::plan_error(c.plan);
      return rc;
    }
    cudaGraphExec_t gexec = nullptr;
    if ((rc = graph_for_run(srv, b, c, &gexec))) return rc;
  }
  return PSWF_OK;
}

// Stages the batch in c.reqs and enqueues it on the context's stream.
int launch_batch(pswf_server srv, Bucket& b, Context& c) {
  const int K = srv->K;
  const size_t rs = srv->rs;
  const int nb = int(c.reqs.size());
  c.offsets.assign(nb + 1, 0);
  std::vector<double> boxes(size_t(nb) * 3);
  std::vector<int> ps(size_t(nb) * K);
  for (int i = 0; i < nb; ++i) {
    const Request* r = c.reqs[i];
    c.offsets[i + 1] = c.offsets[i] + r->n;
    for (int d = 0; d < 3; ++d) boxes[3 * i + d] = r->box[d];
    for (int k = 0; k < K; ++k) ps[size_t(i) * K + k] = r->ps[k];
  }
  const int64_t n = c.offsets[nb];
  for (int i = 0; i < nb; ++i) {
    const Request* r = c.reqs[i];
    if (!r->n) continue;
    std::memcpy(c.h_pos + 3 * c.offsets[i], r->pos_ref ? r->pos_ref : r->pos.data(), size_t(r->n) * 24);
    for (int k = 0; k < K; ++k) {
      char* dst = static_cast<char*>(c.h_q) + (size_t(k) * n + c.offsets[i]) * rs;
      if (r->q_ref) {   // borrowed: rounded to the server's precision on the way
        const double* src = r->q_ref + size_t(k) * r->n;
        if (rs == 4) {
          float* d = reinterpret_cast<float*>(dst);
          for (int64_t a = 0; a < r->n; ++a) d[a] = float(src[a]);
        } else {
          std::memcpy(dst, src, size_t(r->n) * 8);
        }
      } else {
        std::memcpy(dst, r->q.data() + size_t(k) * r->n * rs, size_t(r->n) * rs);
      }
    }
  }
  int rc;
  if ((rc = pswf::plan_fill_tables(c.plan, nb, boxes.data(), ps.data(), c.offsets.data()))) {
    srv->error = pswf::plan_error(c.plan);
    return rc;
  }
  if ((rc = pswf::plan_upload_tables(c.plan))) return rc;
  if ((rc = cuda_ok(srv, cudaMemcpyAsync(c.d_pos, c.h_pos, size_t(n) * 24, cudaMemcpyHostToDevice, c.stream), "h2d")))
    return rc;
  if ((rc = cuda_ok(srv, cudaMemcpyAsync(c.d_q, c.h_q, size_t(n) * K * rs, cudaMemcpyHostToDevice, c.stream), "h2d")))
    return rc;
  if (srv->opt.use_graphs) {
    cudaGraphExec_t gexec = nullptr;
    if ((rc = graph_for_run(srv, b, c, &gexec))) return rc;
    if ((rc = cuda_ok(srv, cudaGraphLaunch(gexec, c.stream), "graph launch"))) return rc;
  } else {
    if ((rc = pswf::plan_run_set_points(c.plan, n, c.d_pos, 1, c.d_q))) return rc;
    if ((rc = pswf::plan_run_execute(c.plan, c.d_e, c.d_phi, c.d_f))) return rc;
  }
  if ((rc = cuda_ok(srv, cudaMemcpyAsync(c.h_e, c.d_e, size_t(nb) * (K + 1) * 8, cudaMemcpyDeviceToHost, c.stream),
                    "d2h")))
    return rc;
  if ((rc = cuda_ok(srv, cudaMemcpyAsync(c.h_phi, c.d_phi, size_t(n) * K * rs, cudaMemcpyDeviceToHost, c.stream),
                    "d2h")))
    return rc;
  if ((rc = cuda_ok(srv, cudaMemcpyAsync(c.h_f, c.d_f, size_t(n) * 3 * rs, cudaMemcpyDeviceToHost, c.stream), "d2h")))
    return rc;
  return cuda_ok(srv, cudaLaunchHostFunc(c.stream, on_batch_done, &c), "host callback");
}

// Copies a finished batch's results into its requests (outside the lock),
// in the server's precision.
void collect_batch(pswf_server srv, Context& c) {
  const int K = srv->K;
  const size_t rs = srv->rs;
  const int nb = int(c.reqs.size());
  const int64_t n = c.offsets[nb];
  for (int i = 0; i < nb; ++i) {
    Request* r = c.reqs[i];
    r->energy.assign(c.h_e + size_t(i) * (K + 1), c.h_e + size_t(i + 1) * (K + 1));
    r->phi.resize(size_t(K) * r->n * rs);
    r->forces.resize(size_t(r->n) * 3 * rs);
    if (!r->n) continue;
    for (int k = 0; k < K; ++k)
      std::memcpy(r->phi.data() + size_t(k) * r->n * rs,
                  static_cast<const char*>(c.h_phi) + (size_t(k) * n + c.offsets[i]) * rs, size_t(r->n) * rs);
    std::memcpy(r->forces.data(), static_cast<const char*>(c.h_f) + size_t(3 * c.offsets[i]) * rs,
                size_t(r->n) * 3 * rs);
  }
}

// Values of the server's precision to double.
void widen(const char* src, size_t rs, size_t count, double* dst) {
  if (rs == 8) {
    std::memcpy(dst, src, count * 8);
  } else {
    const float* f = reinterpret_cast<const float*>(src);
    for (size_t i = 0; i < count; ++i) dst[i] = double(f[i]);
  }
}

void fail_requests(std::vector<Request*>& rs, int status) {
  for (Request* r : rs) {
    r->status = status;
    r->t_done = Clock::now();
  }
}

void scheduler(pswf_server srv) {
  cudaSetDevice(srv->device);
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop) {
    bool progress = false;
    for (auto& bp : srv->buckets) {
      Bucket& b = *bp;
      for (auto& cp : b.ctx) {
        Context& c = *cp;
        if (c.busy && c.finished) {
          lk.unlock();
          collect_batch(srv, c);
          lk.lock();
          const auto now = Clock::now();
          for (Request* r : c.reqs) {
            r->status = 0;
            r->t_done = now;
          }
          c.reqs.clear();
          c.busy = false;
          c.finished = false;
          progress = true;
          srv->cv_done.notify_all();
        }
        if (!c.busy && !b.pending.empty() && !srv->fatal && !srv->paused) {
          int64_t atoms = 0;
          while (!b.pending.empty() && int(c.reqs.size()) < b.b_max && atoms + b.pending.front()->n <= b.n_max) {
            atoms += b.pending.front()->n;
            c.reqs.push_back(b.pending.front());
            b.pending.pop_front();
          }
          if (c.reqs.empty()) continue;
          c.busy = true;
          lk.unlock();
          const int rc = launch_batch(srv, b, c);
          lk.lock();
          if (rc) {
            srv->fatal = rc;
            fail_requests(c.reqs, rc);
            c.reqs.clear();
            c.busy = false;
            srv->cv_done.notify_all();
          } else {
            ++srv->n_batches;
            srv->n_requests += int64_t(c.reqs.size());
            srv->n_atoms += atoms;
          }
          progress = true;
        }
      }
    }
    if (srv->fatal) {
      for (auto& bp : srv->buckets) {
        Bucket& b = *bp;
        std::vector<Request*> rs(b.pending.begin(), b.pending.end());
        b.pending.clear();
        fail_requests(rs, srv->fatal);
      }
      srv->cv_done.notify_all();
    }
    if (!progress) srv->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
  }
}

int route(pswf_server srv, int64_t n, const double box[3]) {
  const double lmax = std::max(box[0], std::max(box[1], box[2]));
  for (size_t i = 0; i < srv->buckets.size(); ++i) {
    const Bucket& b = *srv->buckets[i];
    if (lmax <= b.box_max[0] * (1.0 + 1e-12) && n <= b.n_max) return int(i);
  }
  return -1;
}

}  // namespace

extern "C" {

void pswf_server_opts_default(pswf_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-5;
  o->inflight = 2;
  o->use_graphs = 1;
}

int pswf_server_create(const pswf_server_opts* opts, pswf_server* out) {
  if (!opts || !out) return PSWF_EINVAL;
  *out = nullptr;
  const pswf_server_opts& o = *opts;
  if (o.K < 1 || o.K > 64 || o.npset < 1 || o.npset > 6 || o.nbucket < 1 || o.nbucket > PSWF_MAX_BUCKETS ||
      !(o.r_c > 0) || o.inflight < 1 || o.inflight > 16 || (o.precision != 0 && o.precision != 1))
    return PSWF_EINVAL;
  pswf_server srv = new (std::nothrow) pswf_server_s();
  if (!srv) return PSWF_ENOMEM;
  srv->opt = o;
  srv->K = o.K;
  srv->rs = o.precision == 1 ? 8 : 4;
  cudaGetDevice(&srv->device);
  const double tol = o.tol > 0 ? o.tol : 1e-5;
  srv->opt.tol = tol;
  const double c = o.c > 0 ? o.c : std::log(3.0 / tol);
  const double h_max = o.h_max > 0 ? o.h_max : 0.5 * 3.14159265358979323846 * o.r_c / c;
  int rc = PSWF_OK;
  for (int i = 0; i < o.nbucket && !rc; ++i) {
    if (o.grid[i] < 4 || o.b_max[i] < 1 || o.n_max[i] < 1 || (i > 0 && o.grid[i] <= o.grid[i - 1])) {
      rc = PSWF_EINVAL;
      srv->error = "buckets need ascending grids >= 4 and positive capacities";
      break;
    }
    auto b = std::make_unique<Bucket>();
    b->grid = o.grid[i];
    b->b_max = o.b_max[i];
    b->n_max = o.n_max[i];
    for (int d = 0; d < 3; ++d) b->box_max[d] = o.grid[i] * h_max;
    srv->buckets.push_back(std::move(b));
  }
  for (size_t i = 0; i < srv->buckets.size() && !rc; ++i) {
    Bucket& b = *srv->buckets[i];
    for (int j = 0; j < o.inflight && !rc; ++j) {
      b.ctx.push_back(std::make_unique<Context>());
      rc = make_context(srv, b, *b.ctx.back());
      if (!rc && o.use_graphs) rc = precapture(srv, b, *b.ctx.back());
    }
  }
  if (rc) {
    for (auto& b : srv->buckets)
      for (auto& c : b->ctx) free_context(*c);
    delete srv;
    return rc;
  }
  srv->th = std::thread(scheduler, srv);
  *out = srv;
  return PSWF_OK;
}

int pswf_server_route(pswf_server srv, int64_t n, const double box[3], pswf_info* info) {
  if (!srv || !box || n < 0) return PSWF_EINVAL;
  const int bi = route(srv, n, box);
  if (bi < 0) return PSWF_EINVAL;
  if (info) pswf_plan_info(srv->buckets[bi]->ctx[0]->plan, info);
  return bi;
}

int pswf_server_submit(pswf_server srv, int64_t n, const double box[3], const int* ps, const double* pos,
                       const double* q, int64_t* ticket) {
  return pswf_server_submit_many(srv, 1, &n, box, ps, &pos, &q, ticket, 0);
}

int pswf_server_wait(pswf_server srv, int64_t ticket, double* energy, double* phi, double* forces,
                     double* latency_ms) {
  return pswf_server_wait_for(srv, ticket, -1.0, energy, phi, forces, latency_ms);
}

int pswf_server_pause(pswf_server srv, int pause) {
  if (!srv) return PSWF_EINVAL;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->paused = pause != 0;
  }
  srv->cv_sched.notify_one();
  return PSWF_OK;
}

int pswf_server_wait_for(pswf_server srv, int64_t ticket, double timeout_ms, double* energy, double* phi,
                         double* forces, double* latency_ms) {
  if (!srv) return PSWF_EINVAL;
  std::unique_ptr<Request> r;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(ticket);
    if (it == srv->reqs.end()) return PSWF_EINVAL;
    Request* rp = it->second.get();
    if (!pswf::wait_until_done(lk, srv->cv_done, timeout_ms, [&] { return rp->status != 1; }))
      return PSWF_ETIMEOUT;   // still pending: the ticket stays valid
    r = std::move(it->second);
    srv->reqs.erase(it);
  }
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const int status = r->status;
  if (!status) {
    const int K = srv->K;
    if (energy) std::memcpy(energy, r->energy.data(), size_t(K + 1) * 8);
    if (phi && r->n) widen(r->phi.data(), srv->rs, size_t(K) * r->n, phi);
    if (forces && r->n) widen(r->forces.data(), srv->rs, size_t(r->n) * 3, forces);
  }
  {
    std::lock_guard<std::mutex> lk(srv->pool_mu);
    if (srv->pool.size() < kRequestPool) srv->pool.push_back(std::move(r));
  }
  return status;
}

int pswf_server_submit_many(pswf_server srv, int64_t count, const int64_t* n, const double* boxes, const int* ps,
                            const double* const* pos, const double* const* q, int64_t* tickets, int flags) {
  if (!srv || count < 0 || (count > 0 && (!n || !boxes || !ps || !pos || !q || !tickets))) return PSWF_EINVAL;
  if (flags & ~PSWF_SUBMIT_BORROW) return PSWF_EINVAL;
  const bool borrow = (flags & PSWF_SUBMIT_BORROW) != 0;
  const int K = srv->K;
  // routes first: the structures before the first invalid one are submitted
  std::vector<int> bucket(static_cast<size_t>(count));
  int64_t nok = 0;
  int status = PSWF_OK;
  for (; nok < count; ++nok) {
    const int64_t i = nok, ni = n[i];
    const double* box = boxes + 3 * i;
    bool ok = ni >= 0 && (ni == 0 || (pos[i] && q[i]));
    for (int d = 0; d < 3 && ok; ++d) ok = box[d] > 0.0;
    for (int k = 0; k < K && ok; ++k) {
      bool in = false;
      for (int j = 0; j < srv->opt.npset; ++j) in = in || srv->opt.pset[j] == ps[size_t(K) * i + k];
      ok = in;
    }
    const int bi = ok ? route(srv, ni, box) : -1;
    if (bi < 0) {
      status = PSWF_EINVAL;
      break;
    }
    bucket[size_t(i)] = bi;
  }
  // requests from the pool, filled (copies, charges to the server's
  // precision) and queued in chunks of about kSubmitChunk atoms, so the
  // scheduler starts on the first chunk while the next is filled
  constexpr int64_t kSubmitChunk = 32768;
  const size_t rs = srv->rs;
  int64_t i0 = 0;
  while (i0 < nok) {
    int64_t i1 = i0, chunk_atoms = 0;
    while (i1 < nok && (i1 == i0 || chunk_atoms + n[i1] <= kSubmitChunk)) chunk_atoms += n[i1++];
    std::vector<std::unique_ptr<Request>> rq(static_cast<size_t>(i1 - i0));
    {
      std::lock_guard<std::mutex> lk(srv->pool_mu);
      for (size_t j = 0; j < rq.size() && !srv->pool.empty(); ++j) {
        rq[j] = std::move(srv->pool.back());
        srv->pool.pop_back();
      }
    }
    for (int64_t i = i0; i < i1; ++i) {
      auto& r = rq[size_t(i - i0)];
      if (!r) r = std::make_unique<Request>();
      const int64_t ni = n[i];
      r->n = ni;
      r->status = 1;
      for (int d = 0; d < 3; ++d) r->box[d] = boxes[3 * i + d];
      r->ps.assign(ps + size_t(K) * i, ps + size_t(K) * (i + 1));
      r->bucket = bucket[size_t(i)];
      if (borrow) {
        r->pos_ref = pos[i];
        r->q_ref = q[i];
        continue;
      }
      r->pos_ref = nullptr;
      r->q_ref = nullptr;
      r->pos.assign(pos[i], pos[i] + 3 * ni);
      r->q.resize(size_t(K) * ni * rs);
      if (rs == 4) {
        float* dst = reinterpret_cast<float*>(r->q.data());
        for (size_t j = 0; j < size_t(K) * ni; ++j) dst[j] = float(q[i][j]);
      } else if (ni) {
        std::memcpy(r->q.data(), q[i], size_t(K) * ni * 8);
      }
    }
    const auto now = Clock::now();
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      if (srv->fatal) return srv->fatal;
      for (int64_t i = i0; i < i1; ++i) {
        auto& r = rq[size_t(i - i0)];
        r->t_submit = now;
        r->id = srv->next_id++;
        tickets[i] = r->id;
        srv->buckets[size_t(r->bucket)]->pending.push_back(r.get());
        srv->reqs.emplace(r->id, std::move(r));
      }
    }
    srv->cv_sched.notify_one();
    i0 = i1;
  }
  return status;
}

int pswf_server_wait_many(pswf_server srv, int64_t count, const int64_t* tickets, const int64_t* offsets,
                          double* energies, double* phi, double* forces, double* latency_ms) {
  if (!srv || count < 0 || (count > 0 && (!tickets || !offsets))) return PSWF_EINVAL;
  const int K = srv->K;
  int first = PSWF_OK;
  for (int64_t i = 0; i < count; ++i) {
    const int64_t a = offsets[i];
    const int rc = pswf_server_wait(srv, tickets[i], energies ? energies + size_t(K + 1) * i : nullptr,
                                    phi ? phi + size_t(K) * a : nullptr, forces ? forces + 3 * a : nullptr,
                                    latency_ms ? latency_ms + i : nullptr);
    if (rc && first == PSWF_OK) first = rc;   // every ticket is still waited for and released
  }
  return first;
}

int pswf_server_stats(pswf_server srv, int64_t* batches, int64_t* requests, int64_t* atoms) {
  if (!srv) return PSWF_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (batches) *batches = srv->n_batches;
  if (requests) *requests = srv->n_requests;
  if (atoms) *atoms = srv->n_atoms;
  return srv->fatal;
}

int pswf_server_last_error(pswf_server srv, char* buf, int len) {
  if (!srv || !buf || len <= 0) return PSWF_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  std::snprintf(buf, size_t(len), "%s", srv->error.c_str());
  return PSWF_OK;
}

void pswf_server_destroy(pswf_server srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_sched.notify_all();
  if (srv->th.joinable()) srv->th.join();
  for (auto& b : srv->buckets)
    for (auto& c : b->ctx) free_context(*c);
  delete srv;
}

}  // extern "C"
