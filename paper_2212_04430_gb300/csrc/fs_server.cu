// Serving loop: continuous batching of FS-MLMC trace jobs on one GPU.
//
// Jobs (a gauge field and the parameters of one mlmc_level_trace call) are queued
// as they arrive. A job is admitted when an active slot is free and its
// device-memory estimate fits the budget next to the jobs already running. Among
// the queued jobs that fit, the one with the least work (solves x lattice sites)
// goes first by default; a job that has waited max_wait_ms goes next whatever its
// size, and no later job passes it, so none waits for ever. fs_server_set_admission
// selects first in, first out instead. Every active job runs on its own worker thread with its own context and
// CUDA stream, so the work of concurrent jobs overlaps on the device; inside a
// job the solves are continuously batched over the slots of its tile. A job's
// results depend only on its own inputs (per-system kernels, fixed-order
// reductions), so they are identical whether it runs alone or in a mix.
// Latency = completion - submission; the server reports p50 / p99 over the
// completed jobs.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "fs_engine.h"
#include "fsmlmc.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SJob {
  uint64_t ticket = 0;
  int dims[4] = {0, 0, 0, 0};
  int bc_t = -1;
  double c_sw = 0.0;
  std::vector<double> U, sigma, gamma;
  std::vector<int> nsamp;
  std::vector<int32_t> colors;  // probing colours, [V] (empty: no probing)
  fs_mlmc_params P{};
  size_t est = 0;
  double work = 0;  // solves x lattice sites: the admission order's measure of a job's size
  double t_submit = 0, t_start = 0, t_end = 0;
  bool done = false;
  fs_job_result res{};
};

size_t real_bytes(int prec) { return prec == FS_PREC_F64 ? 8 : (prec == FS_PREC_F32 ? 4 : 2); }

// Device memory a job needs: gauge copies, its solver tile, staging and contraction buffers.
size_t estimate(const SJob& j) {
  const size_t V = (size_t)j.dims[0] * j.dims[1] * j.dims[2] * j.dims[3];
  const size_t Vh = V / 2;
  const int prec = j.P.solve.prec;
  int tile = j.P.solve.rhs_tile > 0 ? j.P.solve.rhs_tile : 32;
  tile = std::max(tile, j.P.estimator == FS_EST_SPLIT_EVEN ? 2 : 1);
  const size_t f64 = 24 * Vh * tile * 8;
  const size_t fts = 24 * Vh * tile * real_bytes(prec);
  const size_t ftx = 24 * Vh * tile * (prec == FS_PREC_F64 ? 8 : 4);
  const size_t tile_bytes = 6 * f64 + (prec == FS_PREC_F64 ? 0 : f64) + ftx + 7 * fts + (8 + 3 + 3) * (size_t)tile * (Vh / 8) * 8;
  const size_t gauge = 8 * Vh * (18 * 8 + 20 * 4 + 12 * 4 + 24 * 2 + 16 * 2);
  const size_t stage = j.P.estimator == FS_EST_PRODUCT ? (size_t)tile * V * 24 * 8 : 0;
  const size_t contract = (size_t)tile * ((2 * Vh + 255) / 256) * 2 * 8 + (64u << 10) +
                          (j.P.p > 0 ? V * 18 * 8 : 0) +  // partial sums + the path products
                          (j.P.colors ? V * 4 : 0);       // + the probing colours
  // staging of finished solutions for groups of several systems (split-even pairs): 2 tile
  // columns of FP64 vectors, twice with the expansion's vectors
  const size_t staging = j.P.estimator == FS_EST_SPLIT_EVEN
                             ? (size_t)2 * tile * 24 * V * 8 * (j.P.hpe_order > 0 ? 2 : 1) : 0;
  const size_t lanes = (size_t)std::max(1, j.P.solve.lanes);
  // the clover table (2 x 114 reals per site in FP64 and FP32) and each tile's C x field
  const size_t clover = j.c_sw != 0.0 ? V * 2 * 114 * (8 + 4) + lanes * fts : 0;
  return lanes * (tile_bytes + stage + staging) + gauge + contract + clover + (32u << 20);
}

}  // namespace

struct fs_server {
  int device = 0;
  size_t budget = 0;
  int max_active = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<SJob*> queue;
  std::map<uint64_t, std::unique_ptr<SJob>> jobs;
  uint64_t next_ticket = 1;
  size_t reserved = 0;
  int active = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<double> latencies;
  long long completed = 0, solves = 0;
  long long gauge_reuses = 0;  // jobs that found their gauge field resident on their worker
  double t_first = -1, t_last = 0;
  // admission order: least work first among the jobs that fit the budget, except that a job
  // queued for max_wait_ms goes next (oldest first) and no job passes it; least_work_first = 0
  // is first in, first out
  int least_work_first = 1;
  double max_wait_ms = 10000.0;

  // index in `queue` of the job to admit now, or -1 (called with mu held)
  int pick() const {
    if (queue.empty()) return -1;
    if (!least_work_first) return reserved + queue.front()->est <= budget ? 0 : -1;
    const double t = now_ms();
    for (size_t i = 0; i < queue.size(); i++)
      if (t - queue[i]->t_submit >= max_wait_ms) return reserved + queue[i]->est <= budget ? (int)i : -1;
    int best = -1;
    for (size_t i = 0; i < queue.size(); i++)
      if (reserved + queue[i]->est <= budget && (best < 0 || queue[i]->work < queue[best]->work)) best = (int)i;
    return best;
  }

  void worker() {
    fs_ctx* ctx = nullptr;
    int cdims[4] = {0, 0, 0, 0}, cbc = 0;
    // the gauge field resident in ctx (the host copy of the last job that uploaded it): a later
    // job on this worker with the same lattice and a byte-identical field skips the upload, and
    // the context keeps its packed copies and contraction paths
    std::vector<double> resident;
    double resident_csw = 0.0;  // the clover coefficient of the context's operator
    cudaSetDevice(device);
    while (true) {
      SJob* j = nullptr;
      {
        std::unique_lock<std::mutex> lock(mu);
        int k = -1;
        // re-checked at least every 100 ms: a job reaching max_wait_ms changes the choice
        while (!(stop && queue.empty()) && (k = pick()) < 0) cv_work.wait_for(lock, std::chrono::milliseconds(100));
        if (queue.empty()) break;  // stopping and drained
        j = queue[k];
        queue.erase(queue.begin() + k);
        reserved += j->est;
        active += 1;
        j->t_start = now_ms();
      }
      // a context per worker, rebuilt when the lattice changes; tiles are released per job
      const bool same = ctx && cbc == j->bc_t && std::equal(cdims, cdims + 4, j->dims);
      int rc = FS_OK;
      if (!same) {
        if (ctx) fs_ctx_destroy(ctx);
        ctx = nullptr;
        resident.clear();
        resident_csw = 0.0;
        rc = fs_ctx_create(&ctx, j->dims, j->bc_t, device);
        if (rc == FS_OK) {
          std::copy(j->dims, j->dims + 4, cdims);
          cbc = j->bc_t;
        }
      }
      const bool gauge_resident = rc == FS_OK && !resident.empty() && resident.size() == j->U.size() &&
                                  std::memcmp(resident.data(), j->U.data(), j->U.size() * sizeof(double)) == 0;
      // the clover table belongs to (field, c_sw): built once for a new field (the coefficient
      // is dropped first so that the upload does not build a table for the old one)
      if (rc == FS_OK && !gauge_resident) {
        if (resident_csw != j->c_sw && resident_csw != 0.0) rc = fs_set_clover(ctx, 0.0);
        if (rc == FS_OK) rc = fs_set_gauge(ctx, j->U.data());
        if (rc == FS_OK) resident.swap(j->U);  // the job needs its host copy no longer
        else resident.clear();
        if (rc == FS_OK && resident_csw != j->c_sw) rc = fs_set_clover(ctx, j->c_sw);
      } else if (rc == FS_OK && resident_csw != j->c_sw) {
        rc = fs_set_clover(ctx, j->c_sw);
      }
      if (rc == FS_OK) resident_csw = j->c_sw;
      else resident.clear();
      if (gauge_resident) {
        std::lock_guard<std::mutex> lock(mu);
        gauge_reuses += 1;
      }
      fs_job_result r{};
      if (rc == FS_OK) {
        const int nsolve = fs_mlmc_num_solves(&j->P);
        std::vector<fs_sys_stats> st(std::max(nsolve, 1));
        double trace[FS_JOB_MAX_LEVELS * 2], var[FS_JOB_MAX_LEVELS];
        rc = mlmc_level_trace(ctx, &j->P, trace, var, nullptr, st.data());
        long long it = 0;
        for (int k = 0; k < nsolve; k++) {
          it += st[k].iters;
          r.max_iters = std::max(r.max_iters, st[k].iters);
          r.noconv += st[k].status != FS_SYS_CONVERGED;
          r.restarts += st[k].restarts;
        }
        for (int l = 0; l < j->P.nlev; l++) {
          r.trace[l][0] = trace[2 * l];
          r.trace[l][1] = trace[2 * l + 1];
          r.var[l] = var[l];
        }
        r.solves = nsolve;
        r.mean_iters = nsolve > 0 ? (double)it / nsolve : 0.0;
      }
      r.status = rc;
      r.nlev = j->P.nlev;
      if (ctx) ctx->c.tiles.clear();  // the tile memory goes back before the next admission
      {
        std::lock_guard<std::mutex> lock(mu);
        j->t_end = now_ms();
        r.latency_ms = j->t_end - j->t_submit;
        r.queue_ms = j->t_start - j->t_submit;
        j->res = r;
        j->done = true;
        reserved -= j->est;
        active -= 1;
        completed += 1;
        solves += r.solves;
        latencies.push_back(r.latency_ms);
        if (t_first < 0) t_first = j->t_submit;
        t_last = j->t_end;
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    if (ctx) fs_ctx_destroy(ctx);
  }
};

extern "C" {

int fs_server_create(fs_server** out, int device, size_t hbm_budget_bytes, int max_active) {
  if (!out) return FS_ERR_ARG;
  *out = nullptr;
  if (max_active < 1 || max_active > 64 || hbm_budget_bytes == 0) return FS_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return FS_ERR_CUDA;
  }
  fs_server* s = new fs_server();
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  for (int w = 0; w < max_active; w++) s->workers.emplace_back([s] { s->worker(); });
  *out = s;
  return FS_OK;
}

int fs_server_submit(fs_server* s, const fs_job* job, uint64_t* ticket) {
  if (!s || !job || !ticket) return FS_ERR_ARG;
  const fs_mlmc_params& P = job->params;
  if (P.nlev < 1 || P.nlev > FS_JOB_MAX_LEVELS || !P.sigma || !P.n_samples || !P.gamma || !job->U)
    return FS_ERR_ARG;
  long long V = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (job->dims[mu] < 2 || job->dims[mu] % 2) return FS_ERR_ARG;
    V *= job->dims[mu];
  }
  if (V >= (1LL << 27)) return FS_ERR_ARG;
  std::unique_ptr<SJob> j(new SJob());
  std::copy(job->dims, job->dims + 4, j->dims);
  j->bc_t = job->bc_t;
  if (!std::isfinite(job->c_sw)) return FS_ERR_INPUT;
  j->c_sw = job->c_sw;
  j->U.assign(job->U, job->U + (size_t)4 * V * 18);
  j->sigma.assign(P.sigma, P.sigma + P.nlev);
  j->nsamp.assign(P.n_samples, P.n_samples + P.nlev);
  j->gamma.assign(P.gamma, P.gamma + 32);
  if (P.colors) j->colors.assign(P.colors, P.colors + V);
  j->P = P;
  // the server overlaps whole jobs; one tile per job unless the caller asked for more lanes
  if (j->P.solve.lanes == 0) j->P.solve.lanes = 1;
  // the admission estimate assumes at most 32-system tiles where the caller left the choice
  // open; jobs are not autotuned (a trial holds candidate tiles beside the admitted jobs)
  if (j->P.solve.rhs_tile == 0) j->P.solve.rhs_tile = std::max(1, std::min(32, fs_mlmc_num_solves(&P)));
  j->P.sigma = j->sigma.data();
  j->P.n_samples = j->nsamp.data();
  j->P.gamma = j->gamma.data();
  j->P.colors = P.colors ? j->colors.data() : nullptr;
  j->est = estimate(*j);
  j->work = (double)std::max(0, fs_mlmc_num_solves(&j->P)) * (double)V;
  if (j->est > s->budget) return FS_ERR_BUDGET;
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return FS_ERR_STATE;
  j->ticket = s->next_ticket++;
  j->t_submit = now_ms();
  *ticket = j->ticket;
  s->queue.push_back(j.get());
  s->jobs[j->ticket] = std::move(j);
  s->cv_work.notify_all();
  return FS_OK;
}

int fs_server_poll(fs_server* s, uint64_t ticket, fs_job_result* out, int timeout_ms) {
  if (!s || !out) return FS_ERR_ARG;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return FS_ERR_ARG;
  SJob* j = it->second.get();
  const auto pred = [&] { return j->done; };
  if (timeout_ms < 0) s->cv_done.wait(lock, pred);
  else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), pred)) return FS_ERR_TIMEOUT;
  *out = j->res;
  s->jobs.erase(it);  // a result is handed out once
  return FS_OK;
}

int fs_server_set_admission(fs_server* s, int least_work_first, double max_wait_ms) {
  if (!s || (least_work_first != 0 && least_work_first != 1) || !(max_wait_ms >= 0.0)) return FS_ERR_ARG;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->least_work_first = least_work_first;
    s->max_wait_ms = max_wait_ms;
  }
  s->cv_work.notify_all();
  return FS_OK;
}

int fs_server_stats(fs_server* s, fs_server_report* out) {
  if (!s || !out) return FS_ERR_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->queued = (long long)s->queue.size();
  out->active = s->active;
  out->solves = s->solves;
  out->reserved_bytes = s->reserved;
  std::vector<double> l = s->latencies;
  std::sort(l.begin(), l.end());
  if (!l.empty()) {
    auto pct = [&](double q) {
      const size_t k = std::min(l.size() - 1, (size_t)(q * (double)(l.size() - 1) + 0.5));
      return l[k];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.back();
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_ms = sum / (double)l.size();
  }
  const double span = s->t_last - s->t_first;
  out->solves_per_s = span > 0 ? (double)s->solves / (span / 1e3) : 0.0;
  out->gauge_reuses = s->gauge_reuses;
  return FS_OK;
}

void fs_server_destroy(fs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

}  // extern "C"
