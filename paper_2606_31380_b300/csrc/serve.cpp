// Serving loop: admission by device footprint, one stream and one library
// context per admitted request, requests overlapping on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "qams_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  std::vector<qams_body_desc> bodies;
  std::vector<BodyCopy> copies;  // owns the arrays `bodies` points into
  std::vector<double> dirs, far_dirs;
  qams_request r{};
  size_t footprint = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  int cancel = 0;
  qams_result res{};
  Clock::time_point t_submit, t_start, t_end;
};

double ms(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct qams_server {
  int device = 0;
  size_t budget = 0, in_use = 0;
  int slots = 1, running = 0;
  bool stop = false;
  uint64_t next = 1;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Req>> queue;
  std::map<uint64_t, std::shared_ptr<Req>> all;
  std::vector<std::thread> workers;

  void worker();
  void run(Req& q);
};

void qams_server::run(Req& q) {
  qams_result& res = q.res;
  qams_ctx* c = nullptr;
  cudaStream_t st = nullptr;
  void *rhs = nullptr, *mu = nullptr, *uinf = nullptr;
  int rc = QAMS_OK;
  const int R = q.r.R, M = q.r.M;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = QAMS_ECUDA; break; }
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { rc = QAMS_ECUDA; break; }
    if ((rc = qams_create(&c, device, 0))) break;
    c->cancel = &q.cancel;
    if ((rc = qams_set_bodies(c, (int)q.bodies.size(), q.bodies.data(), 0.0))) break;
    res.n_nodes = c->N;
    if ((rc = qams_set_wavenumber(c, q.r.k, q.r.eta))) break;
    if ((rc = qams_assemble(c, st))) break;
    const size_t vb = sizeof(double) * 2 * (size_t)c->N * R;
    if (cudaMalloc(&rhs, vb) != cudaSuccess || cudaMalloc(&mu, vb) != cudaSuccess) { rc = QAMS_ECUDA; break; }
    if ((rc = qams_incident_plane(c, R, q.dirs.data(), rhs, st))) break;
    qams_solve_opts o;
    qams_solve_opts_default(&o);
    o.precision = q.r.precision;
    if (q.r.tol > 0) o.tol = q.r.tol;
    qams_solve_stats ss{};
    rc = qams_solve(c, R, rhs, mu, &o, &ss, st);
    res.iterations = ss.iterations;
    res.refinements = ss.refinements;
    res.rel_residual = ss.rel_residual;
    if (rc) break;
    if (M > 0) {
      if (cudaMalloc(&uinf, sizeof(double) * 2 * (size_t)M * R) != cudaSuccess) { rc = QAMS_ECUDA; break; }
      if ((rc = qams_farfield(c, R, mu, M, q.far_dirs.data(), uinf, st))) break;
      if (q.r.uinf_host &&
          cudaMemcpyAsync(q.r.uinf_host, uinf, sizeof(double) * 2 * (size_t)M * R, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess) { rc = QAMS_ECUDA; break; }
    }
    if (q.r.mu_host && cudaMemcpyAsync(q.r.mu_host, mu, vb, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
      rc = QAMS_ECUDA;
      break;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = QAMS_ECUDA;
  } while (false);
  if (st) cudaStreamSynchronize(st);
  if (rhs) cudaFree(rhs);
  if (mu) cudaFree(mu);
  if (uinf) cudaFree(uinf);
  if (c) qams_destroy(c);
  if (st) cudaStreamDestroy(st);
  res.status = rc;
}

void qams_server::worker() {
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    std::shared_ptr<Req> pick;
    cv.wait(lk, [&] {
      if (stop) return true;
      if (running >= slots) return false;
      for (auto& q : queue)
        if (q->footprint + in_use <= budget) return true;
      return false;
    });
    if (stop) return;
    // first queued request that fits (later small requests may pass a large one)
    for (auto it = queue.begin(); it != queue.end(); ++it)
      if ((*it)->footprint + in_use <= budget) {
        pick = *it;
        queue.erase(it);
        break;
      }
    if (!pick) continue;
    in_use += pick->footprint;
    ++running;
    pick->state = 1;
    pick->t_start = Clock::now();
    lk.unlock();
    run(*pick);
    lk.lock();
    pick->t_end = Clock::now();
    pick->res.queue_ms = ms(pick->t_submit, pick->t_start);
    pick->res.run_ms = ms(pick->t_start, pick->t_end);
    pick->res.latency_ms = ms(pick->t_submit, pick->t_end);
    pick->res.footprint = pick->footprint;
    pick->state = 2;
    in_use -= pick->footprint;
    --running;
    cv.notify_all();
  }
}

extern "C" {

int qams_footprint(const qams_body_desc* bodies, int n_bodies, int R, int restart, size_t* bytes) {
  if (!bodies || n_bodies < 1 || R < 1 || restart < 1 || !bytes) return QAMS_EINVAL;
  size_t N = 0, blk = 0;
  for (int b = 0; b < n_bodies; ++b) {
    BodyCopy bc;
    int rc = qams_copy_body(bodies[b], &bc);
    if (rc) return rc;
    const size_t n = (size_t)bodies[b].n_panels * bodies[b].order * bodies[b].n_theta;
    N += n;
    blk += n * n;
  }
  size_t f = N * (32 + 32 + 16 + 16 + 8);            // node tables
  f += blk * (16 + 8 + 8 + 16);                       // self blocks and preconditioner
  f += (size_t)(restart + 1) * N * R * 16;            // Krylov basis
  f += N * R * (16 * 8 + 8 * 3);                      // solver and apply workspaces
  f += 16 * N * (size_t)std::min(n_bodies, 64) * 16;  // pair-sum split partial sums
  f += 64u << 20;                                     // tables, cuBLAS and rounding slack
  *bytes = f;
  return QAMS_OK;
}

int qams_server_create(qams_server** out, int cuda_device, size_t hbm_budget, int max_slots) {
  if (!out || max_slots < 1) return QAMS_EINVAL;
  *out = nullptr;
  int count = 0;
  QAMS_CUDA(cudaGetDeviceCount(&count));
  if (cuda_device < 0 || cuda_device >= count) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(cuda_device));
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    QAMS_CUDA(cudaMemGetInfo(&fr, &tot));
    hbm_budget = fr - fr / 10;
  }
  qams_server* s = new qams_server();
  s->device = cuda_device;
  s->budget = hbm_budget;
  s->slots = max_slots;
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back([s] { s->worker(); });
  *out = s;
  return QAMS_OK;
}

void qams_server_destroy(qams_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->queue.clear();
    // let running requests finish, then stop the workers
    s->cv.wait(lk, [&] { return s->running == 0; });
    s->stop = true;
    s->cv.notify_all();
  }
  for (auto& t : s->workers) t.join();
  delete s;
}

int qams_submit(qams_server* s, const qams_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket || r->n_bodies < 1 || !r->bodies || r->R < 1 || r->R > 16 || !r->dirs || r->M < 0 ||
      (r->M > 0 && !r->far_dirs) || !(r->k > 0) ||
      (r->precision != QAMS_PREC_FP64 && r->precision != QAMS_PREC_FP32))
    return QAMS_EINVAL;
  auto q = std::make_shared<Req>();
  q->r = *r;
  q->copies.resize(r->n_bodies);
  for (int b = 0; b < r->n_bodies; ++b) {
    int rc = qams_copy_body(r->bodies[b], &q->copies[b]);
    if (rc) return rc;
  }
  q->bodies.resize(r->n_bodies);
  for (int b = 0; b < r->n_bodies; ++b) q->bodies[b] = qams_desc_view(q->copies[b]);
  q->dirs.assign(r->dirs, r->dirs + 3 * r->R);
  if (r->M > 0) q->far_dirs.assign(r->far_dirs, r->far_dirs + 3 * (size_t)r->M);
  int rc = qams_footprint(q->bodies.data(), r->n_bodies, r->R, 50, &q->footprint);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(s->mu);
  if (q->footprint > s->budget) return QAMS_EBUDGET;
  q->ticket = s->next++;
  q->t_submit = Clock::now();
  s->queue.push_back(q);
  s->all[q->ticket] = q;
  *ticket = q->ticket;
  s->cv.notify_all();
  return QAMS_OK;
}

int qams_poll(qams_server* s, uint64_t ticket, qams_result* result) {
  if (!s || !result) return QAMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return QAMS_EINVAL;
  if (it->second->state != 2) return QAMS_EAGAIN;
  *result = it->second->res;
  s->all.erase(it);
  return QAMS_OK;
}

int qams_cancel(qams_server* s, uint64_t ticket) {
  if (!s) return QAMS_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return QAMS_EINVAL;
  auto q = it->second;
  if (q->state == 0) {
    s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), q), s->queue.end());
    q->state = 2;
    q->res.status = QAMS_ECANCELLED;
    q->t_end = Clock::now();
    q->res.latency_ms = ms(q->t_submit, q->t_end);
  } else if (q->state == 1) {
    __atomic_store_n(&q->cancel, 1, __ATOMIC_RELAXED);
  }
  return QAMS_OK;
}

}  // extern "C"
