// server.cpp -- the request loop (ilu_server_*): interior solves submitted
// one by one, run concurrently on one device.
//
// Continuous batching: a request becomes a slot as soon as a slot thread and
// device memory are free; each slot solves on its own CUDA stream, so the
// kernels of all admitted requests overlap on the GPU, and a finished slot
// takes the next request at once (no waiting for a batch to drain).
//
// Admission: the loop owns a device-memory budget (opts or 80% of the free
// memory at creation).  A request is charged its vectors plus, if its tet is
// not resident yet, the tet's tables, scratch and solver vectors (an upper
// estimate made before set-up).  Set-up tets stay resident, keyed by their
// geometry, level, coefficient and degree, so a request on a tet seen before
// (an outer Schur-complement or Steklov-Poincare iteration revisits the same
// macro-tets) skips the FP64 host set-up; idle resident tets are evicted,
// least recently used first, when a request does not fit.  A tet serves one
// request at a time (its scratch is shared); later requests on it wait while
// requests on other tets go ahead.  A request that cannot fit even in an
// empty device fails with ILU_ENOMEM.
//
// Multigrid requests (ILU_MG_VCYCLE, ILU_MG_PCG) are served by a resident
// multigrid hierarchy (ilu_mg) instead of a single tet handle, keyed
// separately; their solves take a handful of V-cycles at any level.
//
// Every request runs the same kernels on its own vectors whatever else is
// admitted, so its result does not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ilu.h"
#include "hooks.h"

namespace ilu {
void set_last_error(const std::string &msg);
}

namespace {

using Clock = std::chrono::steady_clock;

ilu_status fail(ilu_status s, const std::string &msg) {
  ilu::set_last_error(msg);
  return s;
}

// identity of a set-up tet
struct Key {
  double P[12];
  int level, kind, ipow, degree, mg, orient, boundary;
  double c0, amp;
  bool operator<(const Key &o) const {
    int c = std::memcmp(P, o.P, sizeof(P));
    if (c) return c < 0;
    if (level != o.level) return level < o.level;
    if (kind != o.kind) return kind < o.kind;
    if (ipow != o.ipow) return ipow < o.ipow;
    if (degree != o.degree) return degree < o.degree;
    if (mg != o.mg) return mg < o.mg;
    if (orient != o.orient) return orient < o.orient;
    if (boundary != o.boundary) return boundary < o.boundary;
    c = std::memcmp(&c0, &o.c0, sizeof(double));
    if (c) return c < 0;
    return std::memcmp(&amp, &o.amp, sizeof(double)) < 0;
  }
};

// a resident set-up: one tet handle, or a multigrid hierarchy
struct Handle {
  ilu_tet t = nullptr;
  ilu_mg m = nullptr;
  explicit operator bool() const { return t || m; }
  void destroy() {
    if (t) ilu_destroy(t);
    if (m) ilu_mg_destroy(m);
    t = nullptr;
    m = nullptr;
  }
};

struct Resident {
  Handle t;
  size_t bytes = 0;
  bool busy = false;
  std::list<Key>::iterator lru;  // position in the idle list (valid when !busy)
};

struct Job {
  ilu_request req = {};
  std::vector<double> b, x0;
  Key key = {};
  size_t vec_bytes = 0, tet_bytes = 0;
  bool done = false, released = false;
  ilu_result res = {};
  std::vector<double> x;
  Clock::time_point t_submit, t_done;
};

constexpr int kMaxLevel = 10;

size_t num_nodes(int level) {
  const size_t N = (size_t)1 << level;
  return (N + 1) * (N + 2) * (N + 3) / 6;
}

// upper estimate of a tet's device memory: row tables, scratch, kappa and
// its stored stencils, Krylov vectors of ilu_solve, reduction buffers and
// launch bookkeeping
size_t estimate_tet_bytes(int level, int precision, int degree, bool var) {
  const size_t N = (size_t)1 << level, nn = num_nodes(level);
  const size_t ew = precision == ILU_F64 ? 8 : 4, ex = precision == ILU_F32 ? 4 : 8;
  const size_t rstride = degree + 1 <= 4 ? 4 : (degree + 1 <= 8 ? 8 : 16);
  const size_t rows = N * N / 2 + N;
  size_t b = rows * 15 * rstride * ew;  // forward + backward row tables
  b += nn * ew;                         // scratch w
  if (var) b += nn * 8;                 // kappa
  if (var && 14 * nn * 8 <= ((size_t)4 << 30)) b += 14 * nn * 8;  // stored stencils (ILU_STENCIL_AUTO)
  if (precision == ILU_F64 && level <= 9) b += 16 * nn * 8;  // tabulated surrogate values (ILU_VALUES_AUTO)
  b += 5 * nn * ex;                     // Krylov vectors
  b += (N * N / 8 + 4096) * 8;          // partial sums, flags, norms
  return b + (1u << 20);                // allocation granularity
}

}  // namespace

struct ilu_server_s {
  ilu_server_opts opts = {};
  size_t budget = 0, used = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Job> jobs;
  std::map<Key, Resident> resident;
  std::list<Key> idle;  // resident and not busy, least recently used first
  std::vector<std::thread> slots;
  int active = 0, max_active = 0;
  long long submitted = 0, completed = 0, failed = 0;
  std::vector<double> latencies;
  bool have_first = false;
  Clock::time_point first_submit, last_done;

  // pick the first queued job that can run now; evicts idle tets to make
  // room; fails jobs that can never fit.  Called with mu held.
  bool pick(uint64_t *out, std::vector<Handle> *evict) {
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Job &j = jobs[*it];
      auto r = resident.find(j.key);
      if (r != resident.end() && r->second.busy) continue;  // its tet is serving another request
      const size_t need = j.vec_bytes + (r == resident.end() ? j.tet_bytes : 0);
      // evict idle tets (never this job's own) until it fits
      auto lit = idle.begin();
      while (used + need > budget && lit != idle.end()) {
        if (r != resident.end() && !(*lit < j.key) && !(j.key < *lit)) {
          ++lit;
          continue;
        }
        auto v = resident.find(*lit);
        used -= v->second.bytes;
        evict->push_back(v->second.t);
        resident.erase(v);
        lit = idle.erase(lit);
      }
      if (used + need <= budget) {
        *out = *it;
        queue.erase(it);
        return true;
      }
      if (active == 0 && used + need > budget) {
        // nothing running and nothing left to evict: it can never fit
        const uint64_t tk = *it;
        queue.erase(it);
        finish(tk, ILU_ENOMEM, 0, 0.0);
        return pick(out, evict);
      }
      return false;  // first come first served on memory: wait for running slots
    }
    return false;
  }

  // mark a job done (mu held)
  void finish(uint64_t tk, ilu_status st, int iters, double rel) {
    Job &j = jobs[tk];
    j.done = true;
    j.t_done = Clock::now();
    j.res.status = st;
    j.res.iters = iters;
    j.res.rel_res = rel;
    j.res.latency_ms = std::chrono::duration<double, std::milli>(j.t_done - j.t_submit).count();
    j.res.x = st == ILU_OK || st == ILU_ENOTCONV ? j.x.data() : nullptr;
    j.res.n = j.res.x ? j.x.size() : 0;
    if (st == ILU_OK) {
      ++completed;
      latencies.push_back(j.res.latency_ms);
    } else {
      ++failed;
    }
    last_done = j.t_done;
    j.b.clear();
    j.b.shrink_to_fit();
    j.x0.clear();
    j.x0.shrink_to_fit();
    cv_done.notify_all();
  }

  void slot_main();
  ilu_status run(Job &j, Handle t, cudaStream_t st, int *iters, double *rel);
};

// one request on its tet: vectors in, ilu_solve, solution out; the vectors
// are stream-ordered allocations returned when the request ends
ilu_status ilu_server_s::run(Job &j, Handle t, cudaStream_t st, int *iters, double *rel) {
  const size_t nn = num_nodes(j.req.level);
  const bool f32 = opts.precision == ILU_F32;
  const size_t es = f32 ? sizeof(float) : sizeof(double);
  void *dxp = nullptr, *dbp = nullptr;
  if (cudaMallocAsync(&dxp, nn * es, st) != cudaSuccess) return fail(ILU_ENOMEM, "device vectors");
  if (cudaMallocAsync(&dbp, nn * es, st) != cudaSuccess) {
    cudaFreeAsync(dxp, st);
    return fail(ILU_ENOMEM, "device vectors");
  }
  struct Free {
    void *a, *b;
    cudaStream_t s;
    ~Free() {
      cudaFreeAsync(a, s);
      cudaFreeAsync(b, s);
      cudaStreamSynchronize(s);
    }
  } guard{dxp, dbp, st};
  void **dx = &dxp, **db = &dbp;
  std::vector<float> tmp;
  auto put = [&](void *dst, const std::vector<double> &src) -> bool {
    if (!f32) return cudaMemcpyAsync(dst, src.data(), nn * es, cudaMemcpyHostToDevice, st) == cudaSuccess;
    tmp.assign(src.begin(), src.end());
    if (cudaMemcpyAsync(dst, tmp.data(), nn * es, cudaMemcpyHostToDevice, st) != cudaSuccess) return false;
    return cudaStreamSynchronize(st) == cudaSuccess;  // tmp is reused
  };
  if (!put(*db, j.b) || !put(*dx, j.x0)) return fail(ILU_ECUDA, "upload of b or x0");
  ilu_status s = t.m ? ilu_mg_solve(t.m, *dx, *db, j.req.method == ILU_MG_PCG ? ILU_PCG : ILU_RICHARDSON, j.req.rtol,
                                    j.req.max_iter, st, iters, rel)
                     : ilu_solve(t.t, *dx, *db, j.req.method, j.req.rtol, j.req.max_iter, st, iters, rel);
  if (s != ILU_OK && s != ILU_ENOTCONV) return s;
  j.x.resize(nn);
  if (!f32) {
    if (cudaMemcpyAsync(j.x.data(), *dx, nn * es, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return fail(ILU_ECUDA, "download of x");
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(ILU_ECUDA, "download of x");
  } else {
    std::vector<float> xf(nn);
    if (cudaMemcpyAsync(xf.data(), *dx, nn * es, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(ILU_ECUDA, "download of x");
    std::copy(xf.begin(), xf.end(), j.x.begin());
  }
  return s;
}

void ilu_server_s::slot_main() {
  cudaStream_t st = nullptr;
  bool have_dev = cudaSetDevice(opts.device) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  for (;;) {
    uint64_t tk = 0;
    std::vector<Handle> evict;
    Handle t;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) break;
        if (pick(&tk, &evict)) break;
        if (!evict.empty()) {  // free what was evicted before sleeping
          lk.unlock();
          for (Handle &e : evict) e.destroy();
          evict.clear();
          lk.lock();
          continue;
        }
        cv_work.wait(lk);
      }
      if (tk == 0) break;
      Job &j = jobs[tk];
      auto r = resident.find(j.key);
      if (r != resident.end()) {
        idle.erase(r->second.lru);
        r->second.busy = true;
        t = r->second.t;
        used += j.vec_bytes;
      } else {
        used += j.vec_bytes + j.tet_bytes;  // charged now, set up below
      }
      ++active;
      max_active = std::max(max_active, active);
    }
    for (Handle &e : evict) e.destroy();
    Job &j = jobs[tk];  // stable: unordered_map references survive rehashing
    ilu_status s = ILU_OK;
    int iters = 0;
    double rel = 0.0;
    bool fresh = false;
    if (!have_dev) s = fail(ILU_ENODEV, "no usable CUDA device for the request loop");
    if (s == ILU_OK && !t) {
      ilu_opts o;
      ilu_opts_default(&o);
      o.precision = opts.precision;
      o.device = opts.device;
      o.orient = j.req.orient;
      o.boundary = j.req.boundary;
      o.max_cluster = opts.max_cluster;
      if (j.key.mg)
        s = ilu_mg_setup(j.req.macro_tet, j.req.level, &j.req.coeff, j.req.poly_degree, 3, &o, &t.m);
      else
        s = ilu_setup(j.req.macro_tet, j.req.level, &j.req.coeff, j.req.poly_degree, &o, &t.t);
      fresh = true;
    }
    if (s == ILU_OK) s = run(j, t, st, &iters, &rel);
    {
      std::lock_guard<std::mutex> lk(mu);
      --active;
      used -= j.vec_bytes;
      const bool keep = t && (s == ILU_OK || s == ILU_ENOTCONV);
      if (fresh) {
        if (keep) {
          Resident rr;
          rr.t = t;
          rr.bytes = j.tet_bytes;
          rr.busy = false;
          rr.lru = idle.insert(idle.end(), j.key);
          resident[j.key] = rr;
        } else {
          used -= j.tet_bytes;
        }
      } else if (t) {
        auto r = resident.find(j.key);
        if (keep) {
          r->second.busy = false;
          r->second.lru = idle.insert(idle.end(), j.key);
        } else {  // a failed handle must be destroyed
          used -= r->second.bytes;
          resident.erase(r);
        }
      }
      if (!keep && t) evict.assign(1, t);
      else evict.clear();
      finish(tk, s, iters, rel);
    }
    for (Handle &e : evict) e.destroy();
    cv_work.notify_all();
  }
  if (st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
}

extern "C" {

ilu_status ilu_server_create(const ilu_server_opts *opts, ilu_server *out) {
  ilu::DeviceRestore keep_device;
  if (!out) return fail(ILU_EINVAL, "null output handle");
  *out = nullptr;
  if (!opts) return fail(ILU_EINVAL, "null options");
  if (opts->precision < ILU_F64 || opts->precision > ILU_MIXED) return fail(ILU_EINVAL, "unknown precision");
  if (opts->device < 0) return fail(ILU_ENODEV, "the request loop needs a CUDA device");
  ilu_server s = new (std::nothrow) ilu_server_s;
  if (!s) return fail(ILU_ENOMEM, "out of host memory");
  s->opts = *opts;
  if (s->opts.max_slots <= 0) s->opts.max_slots = 64;
  if (opts->hbm_budget_bytes > 0) {
    s->budget = (size_t)opts->hbm_budget_bytes;
  } else {
    size_t fr = 0, tot = 0;
    if (cudaSetDevice(opts->device) != cudaSuccess || cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete s;
      return fail(ILU_ENODEV, "cannot query device memory for the default budget");
    }
    s->budget = (size_t)(0.8 * (double)fr);
  }
  try {
    for (int i = 0; i < s->opts.max_slots; ++i) s->slots.emplace_back([s] { s->slot_main(); });
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &th : s->slots) th.join();
    delete s;
    return fail(ILU_ENOMEM, "cannot start slot threads");
  }
  *out = s;
  return ILU_OK;
}

ilu_status ilu_server_submit(ilu_server s, const ilu_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket) return fail(ILU_EINVAL, "null argument");
  if (req->level < 2 || req->level > kMaxLevel) return fail(ILU_EINVAL, "level out of [2, 10]");
  if (!req->b) return fail(ILU_EINVAL, "null right-hand side");
  if (req->method < ILU_RICHARDSON || req->method > ILU_MG_PCG) return fail(ILU_EINVAL, "unknown method");
  const bool mg = req->method == ILU_MG_VCYCLE || req->method == ILU_MG_PCG;
  if (mg && req->level < 3) return fail(ILU_EINVAL, "multigrid needs level >= 3");
  if (req->orient != ILU_ORIENT_GIVEN && req->orient != ILU_ORIENT_LFA) return fail(ILU_EINVAL, "unknown orientation");
  if (req->boundary != ILU_BOUNDARY_V2 && req->boundary != ILU_BOUNDARY_V1) return fail(ILU_EINVAL, "unknown boundary variant");
  if (!(req->rtol >= 0.0) || req->max_iter < 0) return fail(ILU_EINVAL, "bad tolerance or iteration limit");
  if (req->poly_degree < 0 || req->poly_degree > 12) return fail(ILU_EINVAL, "degree out of [0, 12]");
  const size_t nn = num_nodes(req->level);
  Job j;
  try {
    j.b.assign(req->b, req->b + nn);
    if (req->x0) j.x0.assign(req->x0, req->x0 + nn);
    else j.x0.assign(nn, 0.0);
  } catch (const std::bad_alloc &) {
    return fail(ILU_ENOMEM, "out of host memory");
  }
  j.req = *req;
  j.req.b = nullptr;
  j.req.x0 = nullptr;
  std::memcpy(j.key.P, req->macro_tet, sizeof(j.key.P));
  j.key.level = req->level;
  j.key.kind = req->coeff.kind;
  j.key.ipow = req->coeff.ipow;
  j.key.c0 = req->coeff.c0;
  j.key.amp = req->coeff.amp;
  j.key.degree = req->poly_degree;
  j.key.mg = mg ? 1 : 0;
  j.key.orient = req->orient;
  j.key.boundary = req->boundary;
  const size_t ex = s->opts.precision == ILU_F32 ? 4 : 8;
  j.vec_bytes = 2 * nn * ex;
  const bool var = req->coeff.kind != ILU_COEFF_CONST;
  if (mg) {  // a tet per level 3..L, and per level x, b, r plus five Krylov vectors at the finest
    j.tet_bytes = 0;
    for (int l = 3; l <= req->level; ++l)
      j.tet_bytes += estimate_tet_bytes(l, s->opts.precision, req->poly_degree, var) + 3 * num_nodes(l) * ex;
    j.tet_bytes += 5 * nn * ex;
  } else {
    j.tet_bytes = estimate_tet_bytes(req->level, s->opts.precision, req->poly_degree, var);
  }
  j.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(ILU_EBUSY, "the request loop is shutting down");
    const uint64_t tk = s->next_ticket++;
    s->jobs.emplace(tk, std::move(j));
    s->queue.push_back(tk);
    ++s->submitted;
    if (!s->have_first) {
      s->have_first = true;
      s->first_submit = s->jobs[tk].t_submit;
    }
    *ticket = tk;
  }
  s->cv_work.notify_all();
  return ILU_OK;
}

ilu_status ilu_server_wait(ilu_server s, uint64_t ticket, int timeout_ms, ilu_result *res) {
  if (!s || !res) return fail(ILU_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end() || it->second.released) return fail(ILU_EINVAL, "unknown ticket");
  auto ready = [&] { return it->second.done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return fail(ILU_ETIMEOUT, "request not finished yet");
  }
  *res = it->second.res;
  return ILU_OK;
}

ilu_status ilu_server_release(ilu_server s, uint64_t ticket) {
  if (!s) return fail(ILU_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(ILU_EINVAL, "unknown ticket");
  if (!it->second.done) return fail(ILU_EBUSY, "request still running");
  s->jobs.erase(it);
  return ILU_OK;
}

ilu_status ilu_server_stats(ilu_server s, ilu_stats *st) {
  if (!s || !st) return fail(ILU_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->max_concurrent = s->max_active;
  std::vector<double> v = s->latencies;
  std::sort(v.begin(), v.end());
  auto q = [&](double p) {  // nearest-rank percentile
    if (v.empty()) return 0.0;
    size_t k = (size_t)std::ceil(p * (double)v.size());
    k = std::min(std::max<size_t>(k, 1), v.size());
    return v[k - 1];
  };
  st->p50_ms = q(0.50);
  st->p99_ms = q(0.99);
  const double span = s->have_first && s->completed
                          ? std::chrono::duration<double>(s->last_done - s->first_submit).count()
                          : 0.0;
  st->solves_per_s = span > 0 ? (double)s->completed / span : 0.0;
  return ILU_OK;
}

ilu_status ilu_server_destroy(ilu_server s) {
  ilu::DeviceRestore keep_device;
  if (!s) return ILU_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // requests not admitted yet are cancelled
    for (uint64_t tk : s->queue) s->finish(tk, ILU_EBUSY, 0, 0.0);
    s->queue.clear();
  }
  s->cv_work.notify_all();
  for (auto &th : s->slots) th.join();
  for (auto &kv : s->resident) kv.second.t.destroy();
  delete s;
  return ILU_OK;
}

}  // extern "C"
