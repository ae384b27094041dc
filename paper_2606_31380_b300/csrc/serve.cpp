// Serving loop: admission by device footprint, one stream and one library
// context per admitted request, requests overlapping on the device.
//
// Device memory: one pool of the server's budget is allocated when the
// server starts.  Admitting a request reserves a contiguous region of its
// footprint in the pool (first fit); the request's context draws every
// buffer from that region (qams_dev_alloc), so serving makes no cudaMalloc
// or cudaFree -- neither of which could overlap with other requests' work,
// since both synchronise the device -- and an admitted request cannot run
// out of memory through fragmentation.  A request whose footprint fits the
// budget but finds no free region of that size waits in the queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qams_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  long long region = -1;  // offset of its reservation in the pool
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
  char* pool = nullptr;  // the whole budget, allocated at start
  FitAlloc regions;      // reservations of running requests
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
  DeviceBuf b_rhs, b_mu, b_uinf;
  DevArena arena;  // outlives the context: its buffers go back here on destroy
  int rc = QAMS_OK;
  const int R = q.r.R, M = q.r.M;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = QAMS_ECUDA; break; }
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { rc = QAMS_ECUDA; break; }
    if ((rc = qams_create(&c, device, 0))) break;
    c->cancel = &q.cancel;
    arena.base = pool + q.region;
    arena.fa.init(q.footprint);
    c->arena = &arena;
    if ((rc = qams_set_bodies(c, (int)q.bodies.size(), q.bodies.data(), 0.0))) break;
    res.n_nodes = c->N;
    if ((rc = qams_set_wavenumber(c, q.r.k, q.r.eta))) break;
    if ((rc = qams_assemble(c, st))) break;
    const size_t vb = sizeof(double) * 2 * (size_t)c->N * R;
    if ((rc = qams_dev_alloc(c, &b_rhs, vb)) || (rc = qams_dev_alloc(c, &b_mu, vb))) break;
    rhs = b_rhs.p;
    mu = b_mu.p;
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
      if ((rc = qams_dev_alloc(c, &b_uinf, sizeof(double) * 2 * (size_t)M * R))) break;
      uinf = b_uinf.p;
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
  if (c) {
    qams_dev_free(c, &b_rhs);
    qams_dev_free(c, &b_mu);
    qams_dev_free(c, &b_uinf);
    qams_destroy(c);  // returns every buffer to the reservation
  }
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
        if (q->footprint + in_use <= budget && q->footprint <= regions.largest_free()) return true;
      return false;
    });
    if (stop) return;
    // first queued request that fits and finds a free region (later small
    // requests may pass a large one)
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      if ((*it)->footprint + in_use > budget) continue;
      const long long off = regions.alloc((*it)->footprint);
      if (off < 0) continue;
      pick = *it;
      pick->region = off;
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
    regions.release((size_t)pick->region, pick->footprint);
    in_use -= pick->footprint;
    --running;
    cv.notify_all();
  }
}

extern "C" {

int qams_footprint(const qams_body_desc* bodies, int n_bodies, int R, int restart, size_t* bytes) {
  if (!bodies || n_bodies < 1 || R < 1 || restart < 1 || !bytes) return QAMS_EINVAL;
  size_t N = 0, blk = 0;
  std::map<std::string, int> classes;  // congruent bodies share one block
  for (int b = 0; b < n_bodies; ++b) {
    BodyCopy bc;
    int rc = qams_copy_body(bodies[b], &bc);
    if (rc) return rc;
    const size_t n = (size_t)bodies[b].n_panels * bodies[b].order * bodies[b].n_theta;
    N += n;
    if (classes.emplace(qams_shape_key(bc), b).second) blk += n * n;
  }
  // an upper bound of the peak device use of one request
  int sms = 148;
  const long long tiles = (long long)((N + 127) / 128) + n_bodies;
  const size_t S = (size_t)std::max(1LL, std::min<long long>(n_bodies, (8LL * sms + tiles - 1) / tiles));
  size_t f = N * (32 + 32 + 16 + 16 + 16 + 16 + 8);   // node tables (FP64, FP32 and float-float tails, |J|)
  f += blk * (16 + 8 + 8 + 8 + 16 + 8);               // blocks c128, c64, split copies; inverse c64, c128, split
  f += (size_t)(restart + 1) * N * R * 16;            // Krylov basis
  f += N * R * (16 * 9 + 8 * 3);                      // solver, refinement and apply workspaces; rhs and mu
  f += N * 4 * 64 * 2;                                // tensor-core sigma tiles (split, padded)
  f += N * 3 * 64 * 8;                                // preconditioner panels (R, C, T of width 64)
  f += (S > 1 ? S : 0) * N * 16 * 16;                 // pair-sum split partial sums
  f += 64u << 20;                                     // tables, far field, alignment slack
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
  hbm_budget &= ~(size_t)255;
  char* pool = nullptr;
  QAMS_CUDA(cudaMalloc(&pool, hbm_budget));
  qams_server* s = new qams_server();
  s->device = cuda_device;
  s->budget = hbm_budget;
  s->slots = max_slots;
  s->pool = pool;
  s->regions.init(hbm_budget);
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
  cudaSetDevice(s->device);
  cudaFree(s->pool);
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
