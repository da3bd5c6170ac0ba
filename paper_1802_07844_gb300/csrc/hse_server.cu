// hse_server.cu -- continuous-batching evaluation server (host runtime).
//
// Requests queue on submission.  Each worker slot (one thread, one
// non-blocking CUDA stream) takes the oldest queued request whose plan is
// resident and idle, or whose new plan fits the device-memory budget after
// evicting idle plans (least recently used); requests that do not fit, or
// whose plan is busy with another request, wait while later ones are admitted.  Plans are checked out exclusively
// (a plan is not re-entrant) and stay resident between requests with equal
// (kernel mask, precision, tol, box, xi).  Waits on the host are bounded.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hse_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct PlanKey {
  int mask, precision;
  double tol, box[3], xi;
  int df64_fourier = 0;  // HSE_MIXED: double-float Fourier part (see choose_df64_fourier)
  bool operator==(const PlanKey& o) const {
    return mask == o.mask && precision == o.precision && tol == o.tol && box[0] == o.box[0] &&
           box[1] == o.box[1] && box[2] == o.box[2] && xi == o.xi && df64_fourier == o.df64_fourier;
  }
};

struct PlanEntry {
  PlanKey key;
  hse_plan plan = nullptr;  // null while being built
  size_t bytes = 0;
  bool busy = false;
  uint64_t last_used = 0;
};

struct Record {
  hse_request req;
  PlanKey key;
  size_t est_bytes = 0;
  hse_status status = (hse_status)HSE_PENDING;
  Clock::time_point t_submit, t_done;
  bool done = false;
  bool have_params = false;
  hse_params params{};  // parameters of the plan that evaluated the request
  std::string error;
};

// xi from the source density, on a factor-sqrt(2) ladder so that requests of
// similar size share plans: xi = 0.7 (N / V)^(1/3).
double choose_xi(int64_t n, const double box[3]) {
  double v = box[0] * box[1] * box[2];
  double xi = 0.7 * std::cbrt((double)(n > 1 ? n : 1) / v);
  double k = std::round(2.0 * std::log2(xi));
  return std::exp2(k / 2.0);
}

size_t workspace_bytes(int64_t n) { return (size_t)(n > 1024 ? n : 1024) * 640; }

// HSE_MIXED half-space stokeslet requests: the FP32 rounding of the Fourier
// part is amplified where the wall's image system cancels the long-range field
// (low wave numbers, scaled by ~1/k^2), measured at ~2.5e-8 sqrt(N) of the
// velocity for sources spread through the box; when that exceeds a third of
// tol the request runs its Fourier part in double-float (the real space stays
// FP32).
bool choose_df64_fourier(int mask, int precision, double tol, int64_t n) {
  if (precision != HSE_MIXED || !(mask & HSE_STOKESLET) || hse::free_space(mask)) return false;
  return 2.5e-8 * std::sqrt((double)(n > 1 ? n : 1)) > tol / 3.0;
}

hse_status create_plan(const PlanKey& key, hse_plan* plan) {
  hse_status st = hse_plan_create(key.mask, key.box, key.xi, 0.0, 0, key.tol, key.precision, plan);
  if (st == HSE_OK && key.df64_fourier) {
    st = hse_plan_set_fft(*plan, HSE_FFT_DF64);
    if (st != HSE_OK) {
      hse_plan_destroy(*plan);
      *plan = nullptr;
    }
  }
  return st;
}

}  // namespace

struct hse_server_s {
  int device = 0;
  hse_server_config cfg{};
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Record> rec;
  std::vector<PlanEntry> pool;
  size_t resident = 0;
  uint64_t next_ticket = 1, use_clock = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  // statistics
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0, targets_done = 0, plans_created = 0, plans_evicted = 0;
  int64_t plan_hits = 0;     // admitted requests that found their plan resident
  double plan_build_s = 0;   // host time spent building plans (requests and prewarm)
  bool have_first = false;
  Clock::time_point t_first, t_last;

  // Picks an admissible request (caller holds m).  On success returns the
  // ticket and the pool index of the plan to use (-1: build a new one).
  bool pick(uint64_t* ticket, int* pool_idx) {
    for (auto it = queue.begin(); it != queue.end(); ++it) {
      Record& r = rec[*it];
      int idle = -1;
      bool in_use = false;
      for (size_t i = 0; i < pool.size(); ++i)
        if (pool[i].key == r.key) {
          if (!pool[i].busy && pool[i].plan) { idle = (int)i; break; }
          in_use = true;
        }
      if (idle >= 0) {
        *ticket = *it;
        *pool_idx = idle;
        queue.erase(it);
        return true;
      }
      // its plan exists but is evaluating (or being built): it is free again
      // within one evaluation, far sooner than a duplicate could be built, so
      // the request waits for it while later requests are admitted
      if (in_use) continue;
      // a new plan: evict idle plans (LRU) until it fits, if that can succeed
      size_t idle_bytes = 0;
      for (auto& e : pool)
        if (!e.busy && e.plan) idle_bytes += e.bytes;
      if (resident - idle_bytes + r.est_bytes > cfg.mem_budget_bytes) continue;  // does not fit now
      while (resident + r.est_bytes > cfg.mem_budget_bytes) {
        int lru = -1;
        for (size_t i = 0; i < pool.size(); ++i)
          if (!pool[i].busy && pool[i].plan && (lru < 0 || pool[i].last_used < pool[lru].last_used)) lru = (int)i;
        if (lru < 0) break;
        hse_plan_destroy(pool[lru].plan);
        resident -= pool[lru].bytes;
        pool.erase(pool.begin() + lru);
        ++plans_evicted;
      }
      *ticket = *it;
      *pool_idx = -1;
      queue.erase(it);
      return true;
    }
    return false;
  }

  void finish(uint64_t t, hse_status st, int64_t n_tgt) {
    Record& r = rec[t];
    r.status = st;
    r.done = true;
    r.t_done = Clock::now();
    if (st == HSE_OK) {
      ++completed;
      targets_done += n_tgt;
      lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
    } else {
      ++failed;
    }
    t_last = r.t_done;
  }

  void worker(int slot) {
    cudaSetDevice(device);
    cudaStream_t s = streams[slot];
    std::unique_lock<std::mutex> lk(m);
    for (;;) {
      uint64_t t = 0;
      int pi = -1;
      cv_work.wait(lk, [&] { return stop || pick(&t, &pi); });
      if (t == 0) return;  // stopping and nothing admitted
      Record& r = rec[t];
      if (pi >= 0) ++plan_hits;
      if (pi < 0) {  // reserve memory and a pool slot, build outside the lock
        PlanEntry e;
        e.key = r.key;
        e.bytes = r.est_bytes;
        e.busy = true;
        pool.push_back(e);
        pi = (int)pool.size() - 1;
        resident += r.est_bytes;
      } else {
        pool[pi].busy = true;
      }
      PlanKey key = r.key;
      hse_request req = r.req;
      hse_plan plan = pool[pi].plan;
      lk.unlock();
      hse_status st = HSE_OK;
      std::string err;
      double build_s = 0.0;
      if (!plan) {
        const Clock::time_point t0 = Clock::now();
        st = create_plan(key, &plan);
        build_s = std::chrono::duration<double>(Clock::now() - t0).count();
        if (st != HSE_OK) {
          plan = nullptr;
          err = std::string("plan: ") + hse_last_error(nullptr);
        }
      }
      hse_params used{};
      const bool have_params = plan && hse_plan_get_params(plan, &used) == HSE_OK;
      if (st == HSE_OK) {
        st = hse_eval(plan, req.n_src, req.src_xyz, req.strengths, req.n_tgt, req.tgt_xyz, req.vel, s);
        if (st != HSE_OK) err = std::string("eval: ") + hse_last_error(plan);
      }
      if (st == HSE_OK) {
        cudaError_t ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
          st = HSE_ERR_CUDA;
          err = std::string("stream: ") + cudaGetErrorString(ce);
        }
      }
      lk.lock();
      plan_build_s += build_s;
      rec[t].error = err;
      rec[t].have_params = have_params;
      rec[t].params = used;
      // the pool may have been compacted by evictions: find our busy entry by plan or reservation
      int idx = -1;
      for (size_t i = 0; i < pool.size(); ++i)
        if (pool[i].busy && pool[i].key == key && (pool[i].plan == plan || pool[i].plan == nullptr)) {
          idx = (int)i;
          break;
        }
      if (idx >= 0) {
        if (!pool[idx].plan && plan) {
          pool[idx].plan = plan;
          ++plans_created;
        }
        if (!pool[idx].plan) {  // creation failed: release the reservation
          resident -= pool[idx].bytes;
          pool.erase(pool.begin() + idx);
        } else {
          pool[idx].busy = false;
          pool[idx].last_used = ++use_clock;
        }
      }
      finish(t, st, req.n_tgt);
      cv_done.notify_all();
      cv_work.notify_all();
      if (stop && queue.empty()) return;
    }
  }
};

using hse::set_err;

extern "C" hse_status hse_server_create(const hse_server_config* cfg, hse_server* out) {
  if (!cfg || !out || cfg->n_slots < 1 || cfg->n_slots > 64) return set_err(nullptr, HSE_ERR_INVALID, "server config");
  *out = nullptr;
  hse_server srv = new (std::nothrow) hse_server_s();
  if (!srv) return set_err(nullptr, HSE_ERR_OOM, "host allocation");
  srv->cfg = *cfg;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    delete srv;
    return set_err(nullptr, HSE_ERR_CUDA, "cudaGetDevice");
  }
  if (srv->cfg.mem_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    srv->cfg.mem_budget_bytes = (size_t)(0.6 * (double)fr);
  }
  for (int i = 0; i < cfg->n_slots; ++i) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto x : srv->streams) cudaStreamDestroy(x);
      delete srv;
      return set_err(nullptr, HSE_ERR_CUDA, "cudaStreamCreate");
    }
    srv->streams.push_back(s);
  }
  for (int i = 0; i < cfg->n_slots; ++i) srv->workers.emplace_back([srv, i] { srv->worker(i); });
  *out = srv;
  return HSE_OK;
}

extern "C" hse_status hse_server_submit(hse_server srv, const hse_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return HSE_ERR_INVALID;
  if (!hse::valid_mask(req->kernel_mask) || !(req->tol > 0.0) || req->n_src < 0 || req->n_tgt < 0 ||
      !(req->box[0] > 0) || !(req->box[1] > 0) || !(req->box[2] > 0))
    return set_err(nullptr, HSE_ERR_INVALID, "hse_server_submit: bad request");
  Record r;
  r.req = *req;
  r.key.mask = req->kernel_mask;
  r.key.precision = req->precision;
  r.key.tol = req->tol;
  for (int d = 0; d < 3; ++d) r.key.box[d] = req->box[d];
  r.key.xi = choose_xi(req->n_src, req->box);
  r.key.df64_fourier = choose_df64_fourier(r.key.mask, r.key.precision, r.key.tol, req->n_src) ? 1 : 0;
  size_t grid = 0;
  hse_status st = hse::plan_estimate(r.key.mask, r.key.box, r.key.xi, r.key.tol, r.key.precision, &grid, nullptr,
                                     nullptr, r.key.df64_fourier);
  if (st != HSE_OK) return st;
  r.est_bytes = grid + workspace_bytes(req->n_src);
  std::lock_guard<std::mutex> lk(srv->m);
  if (srv->stop) return set_err(nullptr, HSE_ERR_INVALID, "server is stopping");
  if (r.est_bytes > srv->cfg.mem_budget_bytes)
    return set_err(nullptr, HSE_ERR_OOM, "request needs %zu bytes, above the budget %zu", r.est_bytes,
                   srv->cfg.mem_budget_bytes);
  r.t_submit = Clock::now();
  if (!srv->have_first) {
    srv->have_first = true;
    srv->t_first = r.t_submit;
  }
  uint64_t t = srv->next_ticket++;
  srv->rec.emplace(t, r);
  srv->queue.push_back(t);
  ++srv->submitted;
  *ticket = t;
  srv->cv_work.notify_one();
  return HSE_OK;
}

extern "C" hse_status hse_server_prewarm(hse_server srv, const hse_request* req) {
  if (!srv || !req) return HSE_ERR_INVALID;
  if (!hse::valid_mask(req->kernel_mask) || !(req->tol > 0.0) || req->n_src < 0 || !(req->box[0] > 0) ||
      !(req->box[1] > 0) || !(req->box[2] > 0))
    return set_err(nullptr, HSE_ERR_INVALID, "hse_server_prewarm: bad request");
  PlanKey key;
  key.mask = req->kernel_mask;
  key.precision = req->precision;
  key.tol = req->tol;
  for (int d = 0; d < 3; ++d) key.box[d] = req->box[d];
  key.xi = choose_xi(req->n_src, req->box);
  key.df64_fourier = choose_df64_fourier(key.mask, key.precision, key.tol, req->n_src) ? 1 : 0;
  size_t grid = 0;
  HSE_TRY(hse::plan_estimate(key.mask, key.box, key.xi, key.tol, key.precision, &grid, nullptr, nullptr,
                             key.df64_fourier));
  {
    std::lock_guard<std::mutex> lk(srv->m);
    if (srv->stop) return set_err(nullptr, HSE_ERR_INVALID, "server is stopping");
    for (auto& e : srv->pool)
      if (e.key == key) return HSE_OK;  // resident or being built
    if (srv->resident + grid > srv->cfg.mem_budget_bytes)
      return set_err(nullptr, HSE_ERR_OOM, "prewarm: plan of %zu bytes does not fit the budget", grid);
    PlanEntry e;
    e.key = key;
    e.bytes = grid;
    e.busy = true;  // reserved: no worker uses it until it is built
    srv->pool.push_back(e);
    srv->resident += grid;
  }
  int prev_dev = srv->device;
  cudaGetDevice(&prev_dev);
  cudaSetDevice(srv->device);
  hse_plan plan = nullptr;
  const Clock::time_point t0 = Clock::now();
  hse_status st = create_plan(key, &plan);
  const double build_s = std::chrono::duration<double>(Clock::now() - t0).count();
  cudaSetDevice(prev_dev);
  std::lock_guard<std::mutex> lk(srv->m);
  srv->plan_build_s += build_s;
  for (size_t i = 0; i < srv->pool.size(); ++i) {
    PlanEntry& e = srv->pool[i];
    if (e.key == key && e.busy && e.plan == nullptr) {
      if (st == HSE_OK) {
        e.plan = plan;
        e.busy = false;
        e.last_used = ++srv->use_clock;
        ++srv->plans_created;
      } else {
        srv->resident -= e.bytes;
        srv->pool.erase(srv->pool.begin() + i);
      }
      break;
    }
  }
  srv->cv_work.notify_all();
  return st;
}

extern "C" hse_status hse_server_request_params(hse_server srv, uint64_t ticket, hse_params* out) {
  if (!srv || !out) return HSE_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->m);
  auto it = srv->rec.find(ticket);
  if (it == srv->rec.end()) return HSE_ERR_INVALID;
  if (!it->second.done) return (hse_status)HSE_PENDING;
  if (!it->second.have_params) return set_err(nullptr, HSE_ERR_INVALID, "request %llu has no plan",
                                              (unsigned long long)ticket);
  *out = it->second.params;
  return HSE_OK;
}

extern "C" hse_status hse_server_poll(hse_server srv, uint64_t ticket) {
  if (!srv) return HSE_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->m);
  auto it = srv->rec.find(ticket);
  if (it == srv->rec.end()) return HSE_ERR_INVALID;
  return it->second.done ? it->second.status : (hse_status)HSE_PENDING;
}

extern "C" hse_status hse_server_wait(hse_server srv, uint64_t ticket, double timeout_s) {
  if (!srv) return HSE_ERR_INVALID;
  std::unique_lock<std::mutex> lk(srv->m);
  auto it = srv->rec.find(ticket);
  if (it == srv->rec.end()) return HSE_ERR_INVALID;
  auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(
                                     timeout_s > 0 ? timeout_s : 0.0));
  bool ok = srv->cv_done.wait_until(lk, deadline, [&] { return srv->rec[ticket].done; });
  if (!ok) return HSE_ERR_TIMEOUT;
  return srv->rec[ticket].status;
}

extern "C" const char* hse_server_error_text(hse_server srv, uint64_t ticket) {
  if (!srv) return "";
  std::lock_guard<std::mutex> lk(srv->m);
  auto it = srv->rec.find(ticket);
  return it == srv->rec.end() ? "" : it->second.error.c_str();
}

extern "C" hse_status hse_server_get_stats(hse_server srv, hse_server_stats* out) {
  if (!srv || !out) return HSE_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->m);
  *out = hse_server_stats{};
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->failed = srv->failed;
  out->in_flight = srv->submitted - srv->completed - srv->failed;
  out->plans_created = srv->plans_created;
  out->plans_evicted = srv->plans_evicted;
  out->plan_hits = srv->plan_hits;
  out->plan_build_s = srv->plan_build_s;
  out->resident_bytes = srv->resident;
  std::vector<double> v = srv->lat_ms;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)std::floor(f * (v.size() - 1) + 0.5))]; };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    double s = 0;
    for (double x : v) s += x;
    out->mean_ms = s / v.size();
  }
  if (srv->have_first && srv->completed > 0) {
    out->busy_s = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
    out->targets_per_s = out->busy_s > 0 ? srv->targets_done / out->busy_s : 0.0;
  }
  return HSE_OK;
}

extern "C" hse_status hse_server_reset_stats(hse_server srv) {
  if (!srv) return HSE_ERR_INVALID;
  std::lock_guard<std::mutex> lk(srv->m);
  srv->lat_ms.clear();
  srv->completed = srv->failed = srv->targets_done = srv->submitted = 0;
  srv->plan_hits = 0;
  srv->plan_build_s = 0.0;
  for (auto& kv : srv->rec)
    if (!kv.second.done) ++srv->submitted;
  srv->have_first = false;
  return HSE_OK;
}

extern "C" hse_status hse_server_destroy(hse_server srv) {
  if (!srv) return HSE_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(srv->m);
    srv->stop = true;
    for (uint64_t t : srv->queue) {
      Record& r = srv->rec[t];
      r.status = HSE_ERR_INVALID;
      r.done = true;
      ++srv->failed;
    }
    srv->queue.clear();
  }
  srv->cv_work.notify_all();
  srv->cv_done.notify_all();
  for (auto& th : srv->workers) th.join();
  cudaSetDevice(srv->device);
  for (auto& e : srv->pool)
    if (e.plan) hse_plan_destroy(e.plan);
  for (auto s : srv->streams) cudaStreamDestroy(s);
  delete srv;
  return HSE_OK;
}
