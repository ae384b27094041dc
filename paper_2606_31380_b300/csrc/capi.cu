// C ABI entry points (declared in include/qams.h).
#include <cmath>
#include <cstdio>
#include <cstring>

#include "qams_internal.h"

#include <algorithm>
#include <atomic>
#include <map>
#include <string>
#include <iterator>

static thread_local char g_last_cuda[256];
static std::atomic<long long> g_launches{0};

void qams_count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void qams_internal_last_cuda_error(cudaError_t e, const char* what) {
  snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", what, cudaGetErrorString(e));
}

void FitAlloc::init(size_t size) {
  std::lock_guard<std::mutex> lk(mu_);
  size_ = size & ~(size_t)255;
  free_.clear();
  if (size_) free_[0] = size_;
}

long long FitAlloc::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  std::lock_guard<std::mutex> lk(mu_);
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second < bytes) continue;
    const size_t off = it->first, len = it->second;
    free_.erase(it);
    if (len > bytes) free_[off + bytes] = len - bytes;
    return (long long)off;
  }
  return -1;
}

void FitAlloc::release(size_t off, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  std::lock_guard<std::mutex> lk(mu_);
  auto it = free_.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != free_.end() && it->first + it->second == nx->first) {  // merge with the next range
    it->second += nx->second;
    free_.erase(nx);
  }
  if (it != free_.begin()) {  // and with the previous one
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      free_.erase(it);
    }
  }
}

size_t FitAlloc::largest_free() {
  std::lock_guard<std::mutex> lk(mu_);
  size_t m = 0;
  for (auto& f : free_) m = std::max(m, f.second);
  return m;
}

int qams_dev_alloc(qams_ctx* c, DeviceBuf* b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (c->budget && c->allocated + bytes > c->budget) return QAMS_EBUDGET;
  if (c->arena) {
    // a serving reservation: no cudaMalloc (and no device synchronisation)
    const long long off = c->arena->fa.alloc(bytes);
    if (off < 0) return QAMS_EBUDGET;
    b->p = c->arena->base + off;
  } else {
    QAMS_CUDA(cudaMalloc(&b->p, bytes));
  }
  b->bytes = bytes;
  c->allocated += bytes;
  return QAMS_OK;
}

void qams_dev_free(qams_ctx* c, DeviceBuf* b) {
  if (b->p) {
    // in a reservation the range is reused by later work of the same request,
    // which runs on the same stream after every kernel that read it
    if (c->arena)
      c->arena->fa.release((size_t)((char*)b->p - c->arena->base), b->bytes);
    else
      cudaFree(b->p);
    c->allocated -= b->bytes;
  }
  b->p = nullptr;
  b->bytes = 0;
}

cudaEvent_t qams_prof_begin(qams_ctx* c, int slot, cudaStream_t st) {
  if (!c->prof || slot < 0 || slot >= QAMS_PROF_COUNT) return nullptr;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  cudaEventRecord(e, st);
  return e;
}

void qams_prof_end(qams_ctx* c, int slot, cudaStream_t st, cudaEvent_t start) {
  if (!start) return;
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaEventDestroy(start);
    return;
  }
  cudaEventRecord(e, st);
  c->prof_slots[slot].pending.push_back(start);
  c->prof_slots[slot].pending.push_back(e);
}

static void prof_drain(qams_ctx* c) {
  for (ProfSlot& ps : c->prof_slots) {
    for (size_t i = 0; i + 1 < ps.pending.size(); i += 2) {
      float ms = 0.f;
      if (cudaEventSynchronize(ps.pending[i + 1]) == cudaSuccess &&
          cudaEventElapsedTime(&ms, ps.pending[i], ps.pending[i + 1]) == cudaSuccess) {
        ps.ms += ms;
        ps.launches += 1;
      }
      cudaEventDestroy(ps.pending[i]);
      cudaEventDestroy(ps.pending[i + 1]);
    }
    ps.pending.clear();
  }
}

qams_ctx::~qams_ctx() {
  cudaSetDevice(device);
  prof_drain(this);
  for (DeviceBuf* b : {&x64, &n64, &x32, &n32, &x32lo, &n32lo, &centers, &boff, &jac64, &d_tiles, &d_splits, &partial,
                        &blocks64, &blocks32, &blk_off, &ws_sigma, &ws_y, &pinv32, &pinv64, &tc_blk_hi, &tc_blk_lo,
                        &tc_pinv_hi, &tc_pinv_lo, &tc_bt, &tc_amax, &tc_err, &d_tiles2})
    qams_dev_free(this, b);
  qams_lattice_reset(this);
}

extern "C" {

long long qams_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int qams_set_option(qams_ctx* c, int key, long long value) {
  if (!c) return QAMS_EINVAL;
  switch (key) {
    case QAMS_OPT_TC_MIN_RHS:
      if (value < 1 || value > 17) return QAMS_EINVAL;
      c->tc_min_r = (int)value;
      return QAMS_OK;
    case QAMS_OPT_TC_PAIR_MIN_RHS:
      if (value < 1 || value > 17) return QAMS_EINVAL;
      c->tc_pair_min_r = (int)value;
      return QAMS_OK;
    case QAMS_OPT_PAIR_TARGETS:
      if (value != 1 && value != 2) return QAMS_EINVAL;
      c->ps_tt = (int)value;
      return QAMS_OK;
    case QAMS_OPT_LATTICE:
      if (value != 0 && value != 1) return QAMS_EINVAL;
      c->lat.use = value != 0;
      return QAMS_OK;
    case QAMS_OPT_NEAR_FIELD:
      if (value < 0 || value > 64) return QAMS_EINVAL;
      c->near_factor = (int)value;
      return QAMS_OK;
    default: return QAMS_EINVAL;
  }
}

int qams_get_option(const qams_ctx* c, int key, long long* value) {
  if (!c || !value) return QAMS_EINVAL;
  switch (key) {
    case QAMS_OPT_TC_MIN_RHS: *value = c->tc_min_r; return QAMS_OK;
    case QAMS_OPT_TC_PAIR_MIN_RHS: *value = c->tc_pair_min_r; return QAMS_OK;
    case QAMS_OPT_PAIR_TARGETS: *value = c->ps_tt; return QAMS_OK;
    case QAMS_OPT_LATTICE: *value = c->lat.use ? 1 : 0; return QAMS_OK;
    case QAMS_OPT_NEAR_FIELD: *value = c->near_factor; return QAMS_OK;
    default: return QAMS_EINVAL;
  }
}

int qams_profile_enable(qams_ctx* c, int on) {
  if (!c) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  prof_drain(c);
  if (on)
    for (ProfSlot& ps : c->prof_slots) ps = ProfSlot{};
  c->prof = on != 0;
  return QAMS_OK;
}

int qams_profile_read(qams_ctx* c, int slot, long long* launches, double* total_ms) {
  if (!c || slot < 0 || slot >= QAMS_PROF_COUNT || !launches || !total_ms) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  prof_drain(c);
  *launches = c->prof_slots[slot].launches;
  *total_ms = c->prof_slots[slot].ms;
  return QAMS_OK;
}

const char* qams_strerror(int code) {
  switch (code) {
    case QAMS_OK: return "ok";
    case QAMS_EINVAL: return "invalid argument or call order";
    case QAMS_EBUDGET: return "footprint exceeds the context's HBM budget";
    case QAMS_EGEOM: return "bodies overlap or violate the minimum gap";
    case QAMS_ENOCONV: return "iteration limit reached";
    case QAMS_ENUMERIC: return "non-finite residual";
    case QAMS_ETIMEOUT: return "bounded device wait timed out";
    case QAMS_ECANCELLED: return "cancelled";
    case QAMS_ECUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case QAMS_ESCRATCH: return "problem exceeds the static scratch of the no-allocation entry point";
    case QAMS_EAGAIN: return "request not finished yet";
    default: return "unknown error";
  }
}

int qams_create(qams_ctx** out, int cuda_device, size_t hbm_budget_bytes) {
  if (!out) return QAMS_EINVAL;
  *out = nullptr;
  int count = 0;
  QAMS_CUDA(cudaGetDeviceCount(&count));
  if (cuda_device < 0 || cuda_device >= count) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(cuda_device));
  qams_ctx* c = new qams_ctx();
  c->device = cuda_device;
  c->budget = hbm_budget_bytes;
  *out = c;
  return QAMS_OK;
}

void qams_destroy(qams_ctx* ctx) { delete ctx; }

int qams_set_bodies(qams_ctx* c, int n_bodies, const qams_body_desc* bodies, double min_gap) {
  if (!c || n_bodies < 1 || !bodies) return QAMS_EINVAL;
  std::vector<BodyHost> bh(n_bodies);
  std::vector<double> rad(n_bodies);
  for (int i = 0; i < n_bodies; ++i) {
    int rc = qams_copy_body(bodies[i], &bh[i]);
    if (rc) return rc;
    rad[i] = bh[i].radius;
  }
  for (int i = 0; i < n_bodies; ++i)
    for (int j = i + 1; j < n_bodies; ++j) {
      double dx = bodies[i].center[0] - bodies[j].center[0];
      double dy = bodies[i].center[1] - bodies[j].center[1];
      double dz = bodies[i].center[2] - bodies[j].center[2];
      if (std::sqrt(dx * dx + dy * dy + dz * dz) < rad[i] + rad[j] + min_gap) return QAMS_EGEOM;
    }
  QAMS_CUDA(cudaSetDevice(c->device));
  qams_lattice_reset(c);
  for (DeviceBuf* b : {&c->x64, &c->n64, &c->x32, &c->n32, &c->x32lo, &c->n32lo, &c->centers, &c->boff, &c->jac64, &c->blocks64,
                       &c->blocks32, &c->blk_off, &c->ws_sigma, &c->ws_y, &c->pinv32, &c->pinv64, &c->tc_blk_hi,
                       &c->tc_blk_lo, &c->tc_pinv_hi, &c->tc_pinv_lo, &c->tc_bt})
    qams_dev_free(c, b);
  c->assembled = false;
  c->have_precond = false;
  c->tc_blk_ok = c->tc_pinv_ok = false;
  c->tc_groups.clear();
  c->bodies = std::move(bh);
  int rc = qams_build_nodes(c);
  if (rc) return rc;
  const long long N = c->N;
  const int nb = n_bodies;
  std::vector<double> x4(4 * N), n4(4 * N), cen(4 * nb);
  std::vector<float> xl(4 * N), nl(4 * N), xlo(4 * N, 0.0f), nlo(4 * N, 0.0f);
  std::vector<long long> off(nb + 1);
  for (int b = 0; b < nb; ++b) {
    const BodyHost& B = c->bodies[b];
    off[b] = B.offset;
    for (int r = 0; r < 3; ++r) cen[4 * b + r] = B.d.center[r];
    cen[4 * b + 3] = 0.0;
    for (long long t = B.offset; t < B.offset + B.n; ++t) {
      for (int r = 0; r < 3; ++r) {
        x4[4 * t + r] = c->hx[3 * t + r];
        n4[4 * t + r] = c->hn[3 * t + r];
        const double xr = c->hx[3 * t + r] - B.d.center[r];
        xl[4 * t + r] = (float)xr;
        nl[4 * t + r] = (float)c->hn[3 * t + r];
        xlo[4 * t + r] = (float)(xr - (double)xl[4 * t + r]);
        nlo[4 * t + r] = (float)(c->hn[3 * t + r] - (double)nl[4 * t + r]);
      }
      x4[4 * t + 3] = c->hw[t];
      n4[4 * t + 3] = 0.0;
      xl[4 * t + 3] = (float)c->hw[t];
      nl[4 * t + 3] = 0.0f;
    }
  }
  off[nb] = N;
  if ((rc = qams_dev_alloc(c, &c->x64, sizeof(double) * 4 * N))) return rc;
  if ((rc = qams_dev_alloc(c, &c->n64, sizeof(double) * 4 * N))) return rc;
  if ((rc = qams_dev_alloc(c, &c->x32, sizeof(float) * 4 * N))) return rc;
  if ((rc = qams_dev_alloc(c, &c->n32, sizeof(float) * 4 * N))) return rc;
  if ((rc = qams_dev_alloc(c, &c->x32lo, sizeof(float) * 4 * N))) return rc;
  if ((rc = qams_dev_alloc(c, &c->n32lo, sizeof(float) * 4 * N))) return rc;
  if ((rc = qams_dev_alloc(c, &c->centers, sizeof(double) * 4 * nb))) return rc;
  if ((rc = qams_dev_alloc(c, &c->boff, sizeof(long long) * (nb + 1)))) return rc;
  if ((rc = qams_dev_alloc(c, &c->jac64, sizeof(double) * N))) return rc;
  // classes of congruent bodies; every body's block offset is its class's
  c->body_class.assign(nb, 0);
  c->class_rep.clear();
  c->class_blk.clear();
  std::map<std::string, int> cls;
  long long blk = 0;
  for (int b = 0; b < nb; ++b) {
    auto ins = cls.emplace(qams_shape_key(c->bodies[b]), (int)c->class_rep.size());
    if (ins.second) {
      c->class_rep.push_back(b);
      c->class_blk.push_back(blk);
      blk += (long long)c->bodies[b].n * c->bodies[b].n;
    }
    c->body_class[b] = ins.first->second;
  }
  std::vector<long long> boffs(nb + 1, blk);
  for (int b = 0; b < nb; ++b) boffs[b] = c->class_blk[c->body_class[b]];
  if ((rc = qams_dev_alloc(c, &c->blk_off, sizeof(long long) * (nb + 1)))) return rc;
  QAMS_CUDA(cudaMemcpy(c->blk_off.p, boffs.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->jac64.p, c->hj.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->x64.p, x4.data(), sizeof(double) * 4 * N, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->n64.p, n4.data(), sizeof(double) * 4 * N, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->x32.p, xl.data(), sizeof(float) * 4 * N, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->n32.p, nl.data(), sizeof(float) * 4 * N, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->x32lo.p, xlo.data(), sizeof(float) * 4 * N, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->n32lo.p, nlo.data(), sizeof(float) * 4 * N, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->centers.p, cen.data(), sizeof(double) * 4 * nb, cudaMemcpyHostToDevice));
  QAMS_CUDA(cudaMemcpy(c->boff.p, off.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice));
  return qams_pairsum_prepare(c);
}

int qams_set_lattice(qams_ctx* c, const qams_body_desc* body, const int* dims, const double* basis, double min_gap) {
  if (!c || !body || !dims || !basis) return QAMS_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || dims[a] > 32) return QAMS_EINVAL;
  for (int a = 0; a < 9; ++a)
    if (!std::isfinite(basis[a])) return QAMS_EINVAL;
  const int nb = dims[0] * dims[1] * dims[2];
  std::vector<qams_body_desc> d(nb, *body);
  for (int p = 0; p < dims[0]; ++p)
    for (int q = 0; q < dims[1]; ++q)
      for (int r = 0; r < dims[2]; ++r) {
        qams_body_desc& b = d[(p * dims[1] + q) * dims[2] + r];
        for (int x = 0; x < 3; ++x) b.center[x] = body->center[x] + p * basis[x] + q * basis[3 + x] + r * basis[6 + x];
      }
  int rc = qams_set_bodies(c, nb, d.data(), min_gap);
  if (rc) return rc;
  LatticeState& L = c->lat;
  L.on = true;
  L.ready = false;
  L.n = c->bodies[0].n;
  for (int a = 0; a < 3; ++a) {
    L.P[a] = dims[a];
    L.L[a] = 2 * dims[a] - 1;
  }
  std::copy(basis, basis + 9, L.basis);
  return QAMS_OK;
}

int qams_lattice_prepare(qams_ctx* c, void* stream) {
  if (!c || !c->lat.on || !c->have_k) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  int rc = qams_lattice_prepare_launch(c, (cudaStream_t)stream);
  if (rc) return rc;
  QAMS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return QAMS_OK;
}

int qams_node_count(const qams_ctx* c, long long* n) {
  if (!c || !n) return QAMS_EINVAL;
  *n = c->N;
  return QAMS_OK;
}

int qams_body_offsets(const qams_ctx* c, long long* off) {
  if (!c || !off || c->bodies.empty()) return QAMS_EINVAL;
  for (size_t b = 0; b < c->bodies.size(); ++b) off[b] = c->bodies[b].offset;
  off[c->bodies.size()] = c->N;
  return QAMS_OK;
}

int qams_get_nodes(const qams_ctx* c, double* x, double* n, double* w) {
  if (!c || c->bodies.empty()) return QAMS_EINVAL;
  if (x) std::memcpy(x, c->hx.data(), sizeof(double) * 3 * c->N);
  if (n) std::memcpy(n, c->hn.data(), sizeof(double) * 3 * c->N);
  if (w) std::memcpy(w, c->hw.data(), sizeof(double) * c->N);
  return QAMS_OK;
}

int qams_set_wavenumber(qams_ctx* c, double k, double eta) {
  if (!c || !(k > 0) || !std::isfinite(k) || !std::isfinite(eta)) return QAMS_EINVAL;
  c->k = k;
  c->eta = eta;
  c->have_k = true;
  c->lat.ready = false;
  return QAMS_OK;
}

int qams_pairsum(qams_ctx* c, int R, const void* sigma, void* y, int precision, void* stream) {
  if (!c || R < 1 || !sigma || !y || c->bodies.empty() || !c->have_k) return QAMS_EINVAL;
  if (precision != QAMS_PREC_FP64 && precision != QAMS_PREC_FP32 && precision != QAMS_PREC_FF) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  return qams_pairsum_launch(c, R, sigma, y, precision, (cudaStream_t)stream);
}

int qams_assemble(qams_ctx* c, void* stream) {
  if (!c || c->bodies.empty() || !c->have_k) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  c->assembled = false;
  c->have_precond = false;
  int rc = qams_assemble_launch(c, (cudaStream_t)stream);
  if (rc) return rc;
  rc = qams_blocks_to_fp32(c, (cudaStream_t)stream);
  if (rc) return rc;
  if (c->lat.on && c->lat.use && (rc = qams_lattice_prepare_launch(c, (cudaStream_t)stream))) return rc;
  c->assembled = true;
  return QAMS_OK;
}

int qams_assembly_counts(const qams_ctx* c, long long* counts) {
  if (!c || !c->assembled || !counts) return QAMS_EINVAL;
  counts[0] = c->asm_counts[0];
  counts[1] = c->asm_counts[1];
  return QAMS_OK;
}

int qams_copy_selfblock(const qams_ctx* c, int body, void* dst, void* stream) {
  if (!c || !c->assembled || body < 0 || body >= (int)c->bodies.size() || !dst) return QAMS_EINVAL;
  const long long off = c->class_blk[c->body_class[body]];
  const long long n = c->bodies[body].n;
  QAMS_CUDA(cudaSetDevice(c->device));
  QAMS_CUDA(cudaMemcpyAsync(dst, (const double2*)c->blocks64.p + off, sizeof(double2) * n * n,
                            cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return QAMS_OK;
}

int qams_build_preconditioner(qams_ctx* c, void* stream) {
  if (!c || !c->assembled) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  c->have_precond = false;
  int rc = qams_precond_launch(c, (cudaStream_t)stream);
  if (rc) return rc;
  c->have_precond = true;
  return QAMS_OK;
}

int qams_copy_preconditioner(const qams_ctx* c, int body, void* dst, void* stream) {
  if (!c || !c->have_precond || body < 0 || body >= (int)c->bodies.size() || !dst) return QAMS_EINVAL;
  const long long off = c->class_blk[c->body_class[body]];
  const long long n = c->bodies[body].n;
  QAMS_CUDA(cudaSetDevice(c->device));
  QAMS_CUDA(cudaMemcpyAsync(dst, (const double2*)c->pinv64.p + off, sizeof(double2) * n * n,
                            cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return QAMS_OK;
}

int qams_apply(qams_ctx* c, int R, const void* x, void* y, int precision, void* stream) {
  if (!c || R < 1 || !x || !y || !c->assembled) return QAMS_EINVAL;
  if (precision != QAMS_PREC_FP64 && precision != QAMS_PREC_FP32 && precision != QAMS_PREC_FF) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  return qams_apply_launch(c, R, x, y, precision, (cudaStream_t)stream);
}

static int block_apply_diag(qams_ctx* c, int which, int R, const void* x, void* y, int precision, void* stream) {
  if (!c || R < 1 || !x || !y || !c->assembled || (which != 0 && which != 1)) return QAMS_EINVAL;
  if (precision != QAMS_PREC_FP64 && precision != QAMS_PREC_FP32) return QAMS_EINVAL;
  if (which == 1 && !c->have_precond) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  const void* blocks = which == 0 ? (precision == QAMS_PREC_FP64 ? c->blocks64.p : c->blocks32.p)
                                  : (precision == QAMS_PREC_FP64 ? c->pinv64.p : c->pinv32.p);
  return qams_block_apply_ptr(c, blocks, R, x, y, precision, false, (cudaStream_t)stream);
}

int qams_selfblock_apply(qams_ctx* c, int R, const void* x, void* y, int precision, void* stream) {
  return block_apply_diag(c, 0, R, x, y, precision, stream);
}

int qams_precond_apply(qams_ctx* c, int R, const void* x, void* y, int precision, void* stream) {
  return block_apply_diag(c, 1, R, x, y, precision, stream);
}

int qams_incident_plane(qams_ctx* c, int R, const double* dirs, void* rhs, void* stream) {
  if (!c || R < 1 || !dirs || !rhs || c->bodies.empty() || !c->have_k) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  return qams_incident_launch(c, R, dirs, rhs, (cudaStream_t)stream);
}

int qams_farfield(qams_ctx* c, int R, const void* mu, int M, const double* dirs, void* uinf, void* stream) {
  if (!c || R < 1 || M < 1 || !mu || !dirs || !uinf || c->bodies.empty() || !c->have_k) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  return qams_farfield_launch(c, R, mu, M, dirs, uinf, (cudaStream_t)stream);
}

int qams_field_near_pairs(const qams_ctx* c, long long* pairs) {
  if (!c || !pairs) return QAMS_EINVAL;
  *pairs = c->near_pairs;
  return QAMS_OK;
}

int qams_field(qams_ctx* c, int R, const void* mu, int M, const double* points, void* u, void* stream) {
  if (!c || R < 1 || M < 1 || !mu || !points || !u || c->bodies.empty() || !c->have_k) return QAMS_EINVAL;
  QAMS_CUDA(cudaSetDevice(c->device));
  return qams_field_launch(c, R, mu, M, points, u, (cudaStream_t)stream);
}

}  // extern "C"
