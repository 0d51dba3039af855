// Request server: many independent coupled solves in flight on one GPU.
//
// Each worker thread owns one CUDA stream and runs whole requests on it
// (setup phase, one FGMRES solve per right-hand side, free), so requests that
// arrive while others run are admitted as soon as a worker is idle and the
// device-memory budget allows, and their kernels overlap on the device.
// Admission is first come, first served: the queue head waits until the bytes
// its handle is estimated to hold fit under the budget next to the requests
// already in flight.  A request whose estimate alone exceeds the budget is
// refused at submission.  The kernels are the ones of ps_setup / ps_solve, so a
// request gives the same result alone and in the mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "flow.cuh"
#include "internal.cuh"

namespace {

struct Request {
  uint64_t ticket = 0;
  ps_jacobian jac;
  ps_grid grid;
  std::vector<const double*> rhs;
  std::vector<double*> x;
  double tol = 1e-8;
  int64_t est = 0;
  ps_request_info info;
  bool done = false;
};

}  // namespace

struct ps_server {
  ps_server_params prm;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  std::vector<std::thread> workers;
  uint64_t next_ticket = 1;
  int64_t inflight_bytes = 0, inflight = 0;
  ps_server_info stats;
  bool stop = false;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // the queue head may start when a worker is free and its estimate fits next to the requests in flight
  bool admissible() const {
    if (queue.empty()) return false;
    if (prm.hbm_budget <= 0 || inflight == 0) return true;
    return inflight_bytes + queue.front()->est <= prm.hbm_budget;
  }

  void run(Request* r, cudaStream_t st) {
    ps_params p = prm.params;
    p.stream = st;
    ps_handle* h = nullptr;
    ps_status s = ps_setup(&r->jac, &r->grid, &p, &h);
    int iters = 0;
    double worst = 0.0;
    int64_t bytes = 0;
    if (s == PS_OK) {
      for (size_t k = 0; k < r->rhs.size(); ++k) {
        ps_stats so;
        ps_status sk = ps_solve(h, r->rhs[k], r->x[k], r->tol, &so);
        iters += so.iters;
        if (so.true_relres > worst || so.true_relres != so.true_relres) worst = so.true_relres;
        bytes = so.handle_bytes;
        if (sk != PS_OK && s == PS_OK) s = sk;
      }
      ps_free(h);
    }
    r->info.status = s;
    r->info.iters = iters;
    r->info.worst_relres = worst;
    r->info.bytes = bytes;
  }

  void worker() {
    cudaSetDevice(device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      Request* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return admissible() || (stop && queue.empty()); });
        if (!admissible()) break;  // stopping and nothing left to run
        r = queue.front();
        queue.pop_front();
        inflight_bytes += r->est;
        ++inflight;
        if (inflight_bytes > stats.max_inflight_bytes) stats.max_inflight_bytes = inflight_bytes;
        if (inflight > stats.max_inflight_requests) stats.max_inflight_requests = inflight;
        r->info.t_start = now();
      }
      run(r, st);
      {
        std::lock_guard<std::mutex> lk(mu);
        r->info.t_end = now();
        inflight_bytes -= r->est;
        --inflight;
        ++stats.completed;
        r->done = true;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (st) cudaStreamDestroy(st);
  }
};

namespace {

int64_t bsr_bytes(const ps_bsr& b) {
  return b.nnzb * (int64_t(b.br) * b.bc * 8 + 4) + (b.n_brow + 1) * 4;
}

}  // namespace

extern "C" {

int64_t ps_setup_bytes_estimate(const ps_jacobian* jac, const ps_grid* g, const ps_params* p) {
  if (!jac || !g || !p) return 0;
  int64_t nn = int64_t(g->nx + 1) * (g->ny + 1) * (g->nz + 1);
  int64_t nc = int64_t(g->nx) * g->ny * g->nz;
  int64_t n = 3 * nn + 2 * nc;
  int64_t m = p->restart > 0 ? p->restart : 100;
  bool mixed = p->precision == PS_MIXED_FP32 || p->precision == PS_MIXED_BF16P;
  int64_t b = 0;
  b += bsr_bytes(jac->A_uu) + bsr_bytes(jac->A_uf) + bsr_bytes(jac->A_fu) + bsr_bytes(jac->A_ff);
  b += nn * (27 * 9 + 8 * 6) * 8 + nc * (8 * 6 + 7 * 4) * 8;               // stencil copy of the Jacobian
  b += n * (2 * m + 4) * 8;                                                 // V, Z, r, b, x
  int64_t lev0 = jac->A_uu.nnzb * 3 * 8 + jac->A_ff.nnzb * 8;               // SDC and S_pp values
  b += lev0 * 3 / 2 * (mixed ? 2 : 1) + (mixed ? nn * 27 * 3 * 4 + nc * 7 * 4 : nn * 27 * 3 * 8 + nc * 7 * 8);
  b += jac->A_ff.nnzb * 48 + nc * 28 * 8;                                   // flow stage
  const int w = mixed ? ps_internal::win_cells<float>() : ps_internal::win_cells<double>();
  b += 2 * ps_internal::sweep_tiles(g->ny, g->nz) * ps_internal::sweep_steps(g->nx, w) *
       (ps_internal::kTY * ps_internal::kTZ) * ps_internal::kRec * (mixed ? 4 : 8);  // ILU sweep records
  b += n * 8 * 24;                                                          // work vectors
  return b + b / 5;                                                         // 20 % margin
}

ps_status ps_server_create(const ps_server_params* p, ps_server** out) {
  if (!p || !out || p->slots < 1 || p->slots > 256) return PS_ERR_INVALID;
  ps_server* s = new ps_server();
  s->prm = *p;
  std::memset(&s->stats, 0, sizeof(s->stats));
  cudaGetDevice(&s->device);
  s->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < p->slots; ++i) s->workers.emplace_back([s] { s->worker(); });
  *out = s;
  return PS_OK;
}

double ps_server_clock(const ps_server* s) { return s ? s->now() : 0.0; }

ps_status ps_server_submit(ps_server* s, const ps_jacobian* jac, const ps_grid* grid, int32_t nrhs,
                           const double* const* rhs, double* const* x, double tol, double t_arrival,
                           uint64_t* ticket) {
  if (!s || !jac || !grid || !rhs || !x || !ticket || nrhs < 1 || nrhs > 64 || !(tol > 0.0)) return PS_ERR_INVALID;
  Request* r = new Request();
  r->jac = *jac;
  r->grid = *grid;
  r->rhs.assign(rhs, rhs + nrhs);
  r->x.assign(x, x + nrhs);
  r->tol = tol;
  r->est = ps_setup_bytes_estimate(jac, grid, &s->prm.params);
  std::memset(&r->info, 0, sizeof(r->info));
  r->info.nrhs = nrhs;
  if (s->prm.hbm_budget > 0 && r->est > s->prm.hbm_budget) {
    ps_internal::set_reason("request needs an estimated %lld bytes, above the server budget of %lld",
                            (long long)r->est, (long long)s->prm.hbm_budget);
    delete r;
    return PS_ERR_BUDGET;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->info.ticket = r->ticket;
    r->info.t_arrival = t_arrival >= 0.0 ? t_arrival : s->now();
    s->queue.push_back(r);
    s->all[r->ticket] = r;
    ++s->stats.submitted;
    *ticket = r->ticket;
  }
  s->cv_work.notify_one();
  return PS_OK;
}

ps_status ps_server_wait(ps_server* s, uint64_t ticket, ps_request_info* info) {
  if (!s) return PS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return PS_ERR_INVALID;
  Request* r = it->second;
  s->cv_done.wait(lk, [&] { return r->done; });
  if (info) *info = r->info;
  s->all.erase(it);
  ps_status st = r->info.status;
  delete r;
  return st;
}

ps_status ps_server_info_get(ps_server* s, ps_server_info* info) {
  if (!s || !info) return PS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  *info = s->stats;
  return PS_OK;
}

void ps_server_destroy(ps_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->all) delete kv.second;
  delete s;
}

}  // extern "C"
