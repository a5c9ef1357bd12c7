// C ABI of the FS-MLMC library (declared in include/fsmlmc.h).
#include "fsmlmc.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <thread>
#include <cstring>
#include <vector>

#include "fs_engine.h"

namespace {

// Eq. (practical_variance) of n complex samples c[2k], c[2k+1]: (1/n) sum_k |c_k - t|^2 with the
// sample mean t = (tr, ti), the biased 1/n form the paper prints. Two passes (the mean first): the
// one-pass (1/n) sum |c_k|^2 - |t|^2 loses digits to cancellation when the mean is large next to
// the spread, and can even come out negative.
double practical_var(const double* c, int n, double& tr, double& ti) {
  double sr = 0.0, si = 0.0;
  for (int k = 0; k < n; k++) {
    sr += c[2 * k];
    si += c[2 * k + 1];
  }
  tr = sr / n;
  ti = si / n;
  double s2 = 0.0;
  for (int k = 0; k < n; k++) {
    const double dr = c[2 * k] - tr, di = c[2 * k + 1] - ti;
    s2 += dr * dr + di * di;
  }
  return s2 / n;
}

using fs::Ctx;

bool finite_array(const double* a, size_t n) {
  for (size_t i = 0; i < n; i++)
    if (!std::isfinite(a[i])) return false;
  return true;
}

int set_device(Ctx& c) {
  cudaError_t e = cudaSetDevice(c.device);
  return e ? c.cuda_fail(e, "cudaSetDevice") : 0;
}

// Frees what a context owns: a lane leaves the shared gauge copies and paths alone.
void release(Ctx& c) {
  cudaStreamSynchronize(c.stream);
  for (auto& l : c.lanes) release(*l);
  c.lanes.clear();
  c.tiles.clear();
  if (!c.shared) {
    if (c.gauge64) cudaFree(c.gauge64);
    if (c.wline) cudaFree(c.wline);
    for (auto& kv : c.gauge_lo) cudaFree(kv.second);
    if (c.clover64) cudaFree(c.clover64);
    if (c.clover32) cudaFree(c.clover32);
    fs::clover_inverses_free(&c);
  }
  if (c.colors_own && c.colors_d) cudaFree(c.colors_d);
  if (c.canon_d) cudaFree(c.canon_d);
  if (c.canon_h) cudaFreeHost(c.canon_h);
  for (auto& ev : c.prof.pending) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
  for (auto& ev : c.prof.pending64) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
  for (auto& ev : c.prof.pool) { cudaEventDestroy(ev.first); cudaEventDestroy(ev.second); }
  if (c.prof.work_d) cudaFree(c.prof.work_d);
  if (c.own_stream) cudaStreamDestroy(c.own_stream);
}

// Profiling state of one context: hop launches timed on its stream, (site, system) counters.
int prof_reset(Ctx& c, bool enable) {
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e) return c.cuda_fail(e, "fs_profile_enable");
  for (auto& ev : c.prof.pending) c.prof.pool.push_back(ev);
  for (auto& ev : c.prof.pending64) c.prof.pool.push_back(ev);
  c.prof.pending.clear();
  c.prof.pending64.clear();
  c.prof.launches = 0;
  c.prof.ms = 0;
  c.prof.bytes = 0;
  c.prof.pending_bytes = 0;
  c.prof.launches64 = 0;
  c.prof.ms64 = 0;
  if (!c.prof.work_d) {
    e = cudaMalloc(&c.prof.work_d, fs::PROF_SLOTS * sizeof(unsigned long long));
    if (e) return c.cuda_fail(e, "profile counters");
  }
  e = cudaMemset(c.prof.work_d, 0, fs::PROF_SLOTS * sizeof(unsigned long long));
  if (e) return c.cuda_fail(e, "profile counters");
  c.prof.enabled = enable;
  return 0;
}

// Folds the finished launches' event times into the totals (idempotent: the counters are read
// afresh each time) and adds this context's inner-precision hop figures (hi = false) or those of
// its FP64-arithmetic work-list hops (hi = true, bytes unused).
int prof_collect(Ctx& c, long long& launches, double& ms, double& bytes, double& pairs, bool hi = false) {
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e) return c.cuda_fail(e, "fs_profile_read");
  for (auto& ev : c.prof.pending) {
    float t = 0;
    if (cudaEventElapsedTime(&t, ev.first, ev.second) == cudaSuccess) c.prof.ms += t;
    c.prof.pool.push_back(ev);
  }
  c.prof.pending.clear();
  for (auto& ev : c.prof.pending64) {
    float t = 0;
    if (cudaEventElapsedTime(&t, ev.first, ev.second) == cudaSuccess) c.prof.ms64 += t;
    c.prof.pool.push_back(ev);
  }
  c.prof.pending64.clear();
  unsigned long long w[fs::PROF_SLOTS] = {0};
  if (c.prof.work_d) {
    e = cudaMemcpy(w, c.prof.work_d, sizeof(w), cudaMemcpyDeviceToHost);
    if (e) return c.cuda_fail(e, "profile counters");
  }
  if (hi) {
    launches += c.prof.launches64;
    ms += c.prof.ms64;
    pairs += (double)w[12];
    return 0;
  }
  const double real_bytes[4] = {8.0, 4.0, 2.0, 2.0};
  double b = c.prof.pending_bytes;
  for (int pr = 0; pr < 4; pr++)
    for (int k = 0; k < 3; k++) b += (double)w[pr * 3 + k] * (48.0 + 24.0 * k) * real_bytes[pr];
  launches += c.prof.launches;
  ms += c.prof.ms;
  bytes += b;
  for (int k = 0; k < 12; k++) pairs += (double)w[k];
  return 0;
}

fs::NoiseSpec noise_id(uint64_t seed, uint32_t job, uint32_t level, uint32_t sample, bool g5) {
  fs::NoiseSpec n{};
  n.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
  n.key1 = (uint32_t)(seed >> 32);
  n.job = job;
  n.level = level;
  n.sample = sample;
  n.flags = fs::NOISE_VALID | (g5 ? fs::NOISE_G5 : 0);
  return n;
}

struct Opts {
  fs::SolveOpts so;
  int tile;
  int lanes;  // tiles solved at the same time (mlmc_level_trace); 0 = library choice
};

int resolve_params(Ctx& c, const fs_solve_params* p, int nsys, double m, Opts& o) {
  fs_solve_params d{};
  if (p) d = *p;
  o.so.m = m;
  o.so.prec = d.prec;
  if (o.so.prec < FS_PREC_F64 || o.so.prec > FS_PREC_BF16) return c.fail(FS_ERR_ARG, "prec must be 0..3");
  o.so.tol = d.tol > 0 ? d.tol : (o.so.prec == FS_PREC_F64 ? 1e-10 : 1e-8);
  if (o.so.tol < 1e-14) return c.fail(FS_ERR_ARG, "tol below 1e-14 is not reachable in FP64");
  o.so.max_iter = d.max_iter > 0 ? d.max_iter : 20000;
  o.so.nr = d.link_compress == 0 ? 18 : d.link_compress;
  if (o.so.nr != 18 && o.so.nr != 12) return c.fail(FS_ERR_ARG, "link_compress must be 18 or 12");
  if (o.so.prec == FS_PREC_F64) o.so.nr = 18;  // FP64 path keeps full links
  if (d.delta > 0) o.so.delta = d.delta;
  // default reliable-update trigger: as deep as the storage precision lets the sloppy
  // residual fall before rounding stalls it (each update costs two FP64 hops per system)
  else o.so.delta = o.so.prec == FS_PREC_F64 ? 0.0 : (o.so.prec == FS_PREC_F32 ? 1e-5 : (o.so.prec == FS_PREC_F16 ? 3e-3 : 2e-2));
  if (o.so.delta >= 1.0) return c.fail(FS_ERR_ARG, "delta must be < 1");
  o.so.verify = d.verify;
  o.so.check_every = 4;
  if (d.fallback_iter < 0) o.so.cg_max_iter = 0;
  else if (d.fallback_iter > 0) o.so.cg_max_iter = d.fallback_iter;
  else o.so.cg_max_iter = (int)std::min<long long>(4LL * o.so.max_iter, 1 << 30);
  int tile = d.rhs_tile;
  if (tile < 0 || tile > fs::MAX_TILE) return c.fail(FS_ERR_ARG, "rhs_tile must be in [0, 64]");
  if (tile == 0) tile = std::min(32, std::max(1, nsys));
  o.tile = tile;
  if (d.lanes < 0 || d.lanes > 4) return c.fail(FS_ERR_ARG, "lanes must be in [0, 4]");
  o.lanes = d.lanes;
  if (d.rhs_tile == 0 && nsys >= 16 && c.have_gauge) {
    // library choice with enough systems to matter: the autotuned tile (measured once)
    if (int rc = set_device(c)) return rc;
    const int t = fs::autotune_tile(&c, o.so, std::min(nsys, fs::MAX_TILE));
    if (t > 0) o.tile = t;
  }
  return 0;
}

void fill_stats(const fs::SysState& s, fs_sys_stats* out, bool verify) {
  out->iters = s.iters;
  out->status = s.status == fs::SYS_CONVERGED ? FS_SYS_CONVERGED : FS_SYS_NOCONV;
  out->reliable_updates = s.updates;
  out->restarts = s.restarts;
  const double r2 = verify ? s.r2_full : s.r2_true;
  out->true_resid = s.b2 > 0 ? std::sqrt(r2 / s.b2) : 0.0;
  out->fallback_iters = s.cg_iters;
  out->pad = 0;
}

// Tile for a job list: at least the largest group, at most 64 systems.
fs::TileBase* tile_for(Ctx& c, const std::vector<fs::QJob>& jobs, const Opts& o) {
  int gmax = 1;
  for (auto& q : jobs) gmax = std::max(gmax, (int)q.sys.size());
  const int N = std::max(o.tile, gmax);
  if (N > fs::MAX_TILE) return nullptr;
  return c.tile(o.so.prec, N, o.so.nr);
}

// Solves the jobs on `nl` tiles at the same time, one per lane (a stream, tile and host thread
// of its own). A system's result does not depend on the tile it ran in, so lanes change only
// the schedule: while one tile runs its FP64 reliable updates, the other's FP16 iterations
// use the rest of the GPU. Jobs go to the lanes two at a time in turn, so every lane gets the
// same mix of shifts. Shared inputs (gauge copies, contraction paths) must exist beforehand.
int run_lanes(Ctx& c, const std::vector<fs::QJob>& jobs, const Opts& o, const fs::QOut& out, int nl, bool canon) {
  // every lane needs a tile: lanes beyond the first whose tile does not fit in device memory are
  // dropped (the jobs go to the others), so more lanes than memory allows never fail a call
  for (int l = 1; l < nl; l++) {
    Ctx* ln = c.lane(l);
    if (!ln) return FS_ERR_CUDA;
    if (!tile_for(*ln, jobs, o)) {
      cudaGetLastError();
      nl = l;
      break;
    }
  }
  std::vector<std::vector<fs::QJob>> part(nl);
  for (size_t i = 0; i < jobs.size(); i++) part[(i / 2) % nl].push_back(jobs[i]);
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e) return c.cuda_fail(e, "lane event");
  struct EvGuard {
    cudaEvent_t ev;
    ~EvGuard() { cudaEventDestroy(ev); }
  } guard{ev};
  // the lanes start after the work enqueued on the caller's stream so far
  if ((e = cudaEventRecord(ev, c.stream))) return c.cuda_fail(e, "lane start");
  std::vector<Ctx*> L(nl, nullptr);
  std::vector<fs::TileBase*> T(nl, nullptr);
  for (int l = 0; l < nl; l++) {
    if (part[l].empty()) continue;
    if (!(L[l] = c.lane(l))) return FS_ERR_CUDA;
    if (c.prof.enabled && !L[l]->prof.enabled)
      if (prof_reset(*L[l], true)) return c.fail(FS_ERR_CUDA, L[l]->err);
    if ((e = cudaStreamWaitEvent(L[l]->stream, ev, 0))) return c.cuda_fail(e, "lane start");
    if (!(T[l] = tile_for(*L[l], jobs, o)))  // the tile the check above allocated
      return c.fail(FS_ERR_OOM, "device allocation of a lane's solver tile failed");
    if (canon && L[l]->ensure_canon(T[l]->N)) return c.fail(FS_ERR_OOM, L[l]->err);
  }
  std::vector<int> lrc(nl, 0), nc(nl, 0);
  std::vector<std::thread> th;
  for (int l = 0; l < nl; l++) {
    if (!L[l]) continue;
    th.emplace_back([&, l] {
      if (cudaSetDevice(c.device) != cudaSuccess) {
        lrc[l] = L[l]->fail(FS_ERR_CUDA, "cudaSetDevice in a lane");
        return;
      }
      fs::QOut ol = out;  // result rows and state entries of different lanes are disjoint
      ol.noconv = &nc[l];
      lrc[l] = fs::run_queue(L[l], T[l], part[l], o.so, ol);
    });
  }
  for (auto& t : th) t.join();
  // the caller's stream continues after every lane
  for (int l = 0; l < nl && !e; l++) {
    if (!L[l]) continue;
    e = cudaEventRecord(ev, L[l]->stream);
    if (!e) e = cudaStreamWaitEvent(c.stream, ev, 0);
  }
  for (int l = 0; l < nl; l++) {
    if (!L[l]) continue;
    if (lrc[l]) return c.fail(lrc[l], L[l]->err);
    if (nc[l] && out.noconv) *out.noconv = 1;
  }
  if (e) return c.cuda_fail(e, "lane join");
  return 0;
}

}  // namespace

extern "C" {

int fs_ctx_create(fs_ctx** out, const int dims[4], int bc_t, int device) {
  if (!out || !dims) return FS_ERR_ARG;
  *out = nullptr;
  long long V = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (dims[mu] < 2 || dims[mu] % 2) return FS_ERR_ARG;
    V *= dims[mu];
  }
  if (V >= (1LL << 27)) return FS_ERR_ARG;
  if (bc_t != 1 && bc_t != -1) return FS_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return FS_ERR_CUDA; }
  fs_ctx* ctx = new fs_ctx();
  Ctx& c = ctx->c;
  c.device = device;
  for (int mu = 0; mu < 4; mu++) c.g.L[mu] = dims[mu];
  c.g.Lh0 = dims[0] / 2;
  c.g.V = (int)V;
  c.g.Vh = (int)(V / 2);
  c.g.bc_t = bc_t;
  fs::geom_init_div(c.g);
  if (cudaDeviceGetAttribute(&c.nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c.own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FS_ERR_CUDA;
  }
  c.stream = c.own_stream;
  *out = ctx;
  return FS_OK;
}

void fs_ctx_destroy(fs_ctx* ctx) {
  if (!ctx) return;
  Ctx& c = ctx->c;
  cudaSetDevice(c.device);
  release(c);
  delete ctx;
}


const char* fs_last_error(const fs_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

int fs_set_stream(fs_ctx* ctx, void* stream) {
  if (!ctx) return FS_ERR_ARG;
  ctx->c.stream = stream ? (cudaStream_t)stream : ctx->c.own_stream;
  return FS_OK;
}

size_t fs_ctx_device_bytes(const fs_ctx* ctx) { return ctx ? ctx->c.device_bytes() : 0; }

int fs_tuned_shape(const fs_ctx* ctx, int prec, int link_compress, int* tile, int* ring_depth, int* blocks_per_sm) {
  if (!ctx || !tile || !ring_depth || !blocks_per_sm) return FS_ERR_ARG;
  const int nr = prec == FS_PREC_F64 ? 18 : (link_compress == 0 ? 18 : link_compress);
  *tile = 0;
  *ring_depth = 0;
  *blocks_per_sm = 0;
  auto it = ctx->c.tuned_tile.find(prec * 100 + nr);
  if (it == ctx->c.tuned_tile.end()) return FS_OK;
  *tile = it->second;
  auto sh = ctx->c.tuned_shape.find((long long)(prec * 100 + nr) * 1000 + it->second);
  if (sh != ctx->c.tuned_shape.end()) {
    *ring_depth = sh->second.depth;
    *blocks_per_sm = sh->second.blocks;
  }
  return FS_OK;
}

int fs_tuned_tile(const fs_ctx* ctx, int prec, int link_compress) {
  if (!ctx) return 0;
  const int nr = prec == FS_PREC_F64 ? 18 : (link_compress == 0 ? 18 : link_compress);
  auto it = ctx->c.tuned_tile.find(prec * 100 + nr);
  return it == ctx->c.tuned_tile.end() ? 0 : it->second;
}

int fs_set_gauge(fs_ctx* ctx, const double* U) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (!U) return c.fail(FS_ERR_ARG, "null gauge field");
  if (int rc = set_device(c)) return rc;
  const size_t n = (size_t)4 * c.g.V * 18;
  if (!finite_array(U, n)) return c.fail(FS_ERR_INPUT, "gauge field holds a non-finite value");
  double* stage = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&stage, n * sizeof(double), c.stream);
  if (e) return c.cuda_fail(e, "gauge staging allocation");
  e = cudaMemcpyAsync(stage, U, n * sizeof(double), cudaMemcpyHostToDevice, c.stream);
  auto need = [&](void*& p, size_t bytes) -> cudaError_t {
    if (p) return cudaSuccess;
    cudaError_t r = cudaMalloc(&p, bytes);
    if (r == cudaSuccess) c.extra_bytes += bytes;
    return r;
  };
  const size_t nl = (size_t)8 * c.g.Vh;
  c.wline_mask = 0;  // the contraction's path products belong to the old field
  if (!e) e = need(c.gauge64, nl * 18 * sizeof(double));
  if (!e) e = fs::launch_gauge_pack<double>(c.gauge64, stage, c.g, 18, c.stream);
  struct LoCopy { int prec, nr; size_t bytes; };
  const LoCopy lo[] = {
      {FS_PREC_F32, 18, nl * fs::link_pad<float>(18) * sizeof(float)},
      {FS_PREC_F32, 12, nl * fs::link_pad<float>(12) * sizeof(float)},
      {FS_PREC_F16, 18, nl * fs::link_pad<__half>(18) * sizeof(__half)},
      {FS_PREC_F16, 12, nl * fs::link_pad<__half>(12) * sizeof(__half)},
  };
  for (const LoCopy& l : lo) {
    if (e) break;
    void*& p = c.gauge_lo[l.prec * 100 + l.nr];
    e = need(p, l.bytes);
    if (!e) {
      if (l.prec == FS_PREC_F32) e = fs::launch_gauge_pack<float>(p, stage, c.g, l.nr, c.stream);
      else e = fs::launch_gauge_pack<__half>(p, stage, c.g, l.nr, c.stream);
    }
  }
  cudaFreeAsync(stage, c.stream);
  if (!e) e = cudaStreamSynchronize(c.stream);
  if (e) return c.cuda_fail(e, "fs_set_gauge");
  c.have_gauge = true;
  if (c.c_sw != 0.0) {  // the clover table belongs to the field
    if (int rc = fs::clover_build(&c, c.c_sw)) {
      c.have_gauge = false;
      return rc;
    }
  }
  return FS_OK;
}

int fs_set_clover(fs_ctx* ctx, double c_sw) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (!std::isfinite(c_sw)) return c.fail(FS_ERR_INPUT, "non-finite c_sw");
  if (c.shared) return c.fail(FS_ERR_STATE, "a lane takes its owner's clover term");
  if (int rc = set_device(c)) return rc;
  if (cudaError_t e = cudaStreamSynchronize(c.stream)) return c.cuda_fail(e, "fs_set_clover");
  for (auto& l : c.lanes)
    if (cudaError_t e = cudaStreamSynchronize(l->stream)) return c.cuda_fail(e, "fs_set_clover");
  if (c_sw == 0.0) {
    fs::clover_inverses_free(&c);
    if (c.clover64) {
      cudaFree(c.clover64);
      cudaFree(c.clover32);
      c.extra_bytes -= (size_t)2 * c.g.Vh * 2 * fs::CLV_REALS * (sizeof(double) + sizeof(float));
    }
    c.clover64 = nullptr;
    c.clover32 = nullptr;
    c.c_sw = 0.0;
  } else if (c.have_gauge) {
    if (int rc = fs::clover_build(&c, c_sw)) return rc;
  } else {
    c.c_sw = c_sw;  // built with the gauge field
  }
  for (auto& l : c.lanes) {
    l->c_sw = c.c_sw;
    l->clover64 = c.clover64;
    l->clover32 = c.clover32;
  }
  return FS_OK;
}

int wilson_dslash(fs_ctx* ctx, double m, double sigma, const double* in, double* out, int nrhs, int prec,
                  int link_compress) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (nrhs < 0) return c.fail(FS_ERR_ARG, "nrhs must be >= 0");
  if (nrhs == 0) return FS_OK;
  if (!in || !out) return c.fail(FS_ERR_ARG, "null vector");
  if (prec < FS_PREC_F64 || prec > FS_PREC_BF16) return c.fail(FS_ERR_ARG, "prec must be 0..3");
  const int nr = link_compress == 0 ? 18 : link_compress;
  if (nr != 18 && nr != 12) return c.fail(FS_ERR_ARG, "link_compress must be 18 or 12");
  if (prec == FS_PREC_F64 && nr != 18) return c.fail(FS_ERR_ARG, "FP64 uses uncompressed links");
  if (!c.have_gauge) return c.fail(FS_ERR_STATE, "no gauge field set");
  if (!std::isfinite(m) || !std::isfinite(sigma)) return c.fail(FS_ERR_INPUT, "non-finite mass or shift");
  const size_t vlen = (size_t)c.g.V * 24;
  if (!finite_array(in, vlen * nrhs)) return c.fail(FS_ERR_INPUT, "input holds a non-finite value");
  if (int rc = set_device(c)) return rc;
  const int N = std::min(nrhs, fs::MAX_TILE);
  if (int rc = c.ensure_canon(N)) return rc;
  fs::TileBase* T = c.tile(prec, N, nr);
  if (!T) return c.fail(FS_ERR_OOM, "device allocation of the tile failed");
  cudaError_t e = cudaSuccess;
  for (int k0 = 0; k0 < nrhs && !e; k0 += N) {
    const int nb = std::min(N, nrhs - k0);
    for (int j = 0; j < N; j++) {
      fs::SysState& s = T->st_h[j];
      memset(&s, 0, sizeof(s));
      T->vec_h[j] = j < nb ? j : -1;
      if (j >= nb) continue;
      const double A = 4.0 + m + sigma;
      s.A = A;
      s.cd[fs::C_A] = A;
      s.cf[fs::C_A] = (float)A;
      s.flags = fs::FLAG_INIT;
    }
    e = cudaMemcpyAsync(T->st_d, T->st_h, sizeof(fs::SysState) * N, cudaMemcpyHostToDevice, c.stream);
    if (!e) e = cudaMemcpyAsync(T->vec_d, T->vec_h, sizeof(int) * N, cudaMemcpyHostToDevice, c.stream);
    if (!e) e = cudaMemcpyAsync(c.canon_d, in + k0 * vlen, nb * vlen * sizeof(double), cudaMemcpyHostToDevice,
                                c.stream);
    if (!e) e = T->enqueue_dslash(c.canon_d);
    if (!e) e = cudaMemcpyAsync(out + k0 * vlen, c.canon_d, nb * vlen * sizeof(double), cudaMemcpyDeviceToHost,
                                c.stream);
    if (!e) e = cudaStreamSynchronize(c.stream);
  }
  if (e) return c.cuda_fail(e, "wilson_dslash");
  return FS_OK;
}

int shifted_solve(fs_ctx* ctx, double m, const double* sigma, int nshift, const double* b, int nrhs, double* x,
                  const fs_solve_params* params, fs_sys_stats* stats) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (nshift < 0 || nrhs < 0) return c.fail(FS_ERR_ARG, "negative count");
  if (nshift == 0 || nrhs == 0) return FS_OK;
  if (!sigma || !b || !x) return c.fail(FS_ERR_ARG, "null pointer");
  if (!c.have_gauge) return c.fail(FS_ERR_STATE, "no gauge field set");
  if (!std::isfinite(m) || !finite_array(sigma, nshift)) return c.fail(FS_ERR_INPUT, "non-finite mass or shift");
  const size_t vlen = (size_t)c.g.V * 24;
  if (!finite_array(b, vlen * nrhs)) return c.fail(FS_ERR_INPUT, "right-hand side holds a non-finite value");
  for (int j = 0; j < nshift; j++)
    if (std::fabs(4.0 + m + sigma[j]) < 1e-12) return c.fail(FS_ERR_ARG, "4 + m + sigma must be nonzero");
  Opts o;
  const int S = nshift * nrhs;
  if (int rc = resolve_params(c, params, S, m, o)) return rc;
  if (int rc = set_device(c)) return rc;
  if (int rc = fs::clover_inverses(&c, m, sigma, nshift, o.so)) return rc;
  std::vector<fs::QJob> jobs(S);
  for (int i = 0; i < S; i++) {
    const int j = i / nrhs, k = i % nrhs;
    jobs[i].sys = {fs::SysSpec{sigma[j], 1, k, fs::NoiseSpec{}}};
    jobs[i].stat_index = {i};
    jobs[i].out_index = {i};
  }
  fs::TileBase* T = tile_for(c, jobs, o);
  if (!T) return c.fail(FS_ERR_OOM, "device allocation of the solver tile failed");
  const int N = T->N;
  if (int rc = c.ensure_canon((size_t)nrhs + N)) return rc;
  cudaError_t e = cudaMemcpyAsync(c.canon_d, b, nrhs * vlen * sizeof(double), cudaMemcpyHostToDevice, c.stream);
  if (e) return c.cuda_fail(e, "upload right-hand sides");
  int noconv = 0;
  std::vector<fs::SysState> st(S);
  fs::QOut out;
  out.states = &st;
  out.noconv = &noconv;
  out.x_host = x;
  out.canon_out_base = nrhs;
  if (int rc = fs::run_queue(&c, T, jobs, o.so, out)) return rc;
  if (stats)
    for (int i = 0; i < S; i++) fill_stats(st[i], &stats[i], o.so.verify != 0);
  return noconv ? c.fail(FS_ERR_NOCONV, "some systems reached max_iter") : FS_OK;
}

int shifted_solve_dev(fs_ctx* ctx, double m, const double* sigma, int nshift, const double* b, int nrhs, double* x,
                      const fs_solve_params* params, fs_sys_stats* stats) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (nshift < 0 || nrhs < 0) return c.fail(FS_ERR_ARG, "negative count");
  if (nshift == 0 || nrhs == 0) return FS_OK;
  if (!sigma || !b || !x) return c.fail(FS_ERR_ARG, "null pointer");
  if (!c.have_gauge) return c.fail(FS_ERR_STATE, "no gauge field set");
  if (!std::isfinite(m) || !finite_array(sigma, nshift)) return c.fail(FS_ERR_INPUT, "non-finite mass or shift");
  for (int j = 0; j < nshift; j++)
    if (std::fabs(4.0 + m + sigma[j]) < 1e-12) return c.fail(FS_ERR_ARG, "4 + m + sigma must be nonzero");
  if (int rc = set_device(c)) return rc;
  // both arrays must be device (or managed) memory of this context's GPU, 16-byte aligned
  for (const void* q : {(const void*)b, (const void*)x}) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
      cudaGetLastError();
      return c.fail(FS_ERR_ARG, "b and x must be device pointers");
    }
    if ((at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) || at.device != c.device)
      return c.fail(FS_ERR_ARG, "b and x must be device memory of the context's GPU");
    if (reinterpret_cast<uintptr_t>(q) % 16) return c.fail(FS_ERR_ARG, "b and x must be 16-byte aligned");
  }
  Opts o;
  const int S = nshift * nrhs;
  if ((long long)nshift * nrhs > 0x7FFFFFFF) return c.fail(FS_ERR_ARG, "too many systems");
  if (int rc = resolve_params(c, params, S, m, o)) return rc;
  if (int rc = set_device(c)) return rc;
  if (int rc = fs::clover_inverses(&c, m, sigma, nshift, o.so)) return rc;
  std::vector<fs::QJob> jobs(S);
  for (int i = 0; i < S; i++) {
    const int j = i / nrhs, k = i % nrhs;
    jobs[i].sys = {fs::SysSpec{sigma[j], 1, k, fs::NoiseSpec{}}};
    jobs[i].stat_index = {i};
    jobs[i].out_index = {i};
  }
  fs::TileBase* T = tile_for(c, jobs, o);
  if (!T) return c.fail(FS_ERR_OOM, "device allocation of the solver tile failed");
  int noconv = 0;
  std::vector<fs::SysState> st(S);
  fs::QOut out;
  out.states = &st;
  out.noconv = &noconv;
  out.rhs_canon = b;
  out.x_dev = x;
  if (int rc = fs::run_queue(&c, T, jobs, o.so, out)) return rc;
  if (stats)
    for (int i = 0; i < S; i++) fill_stats(st[i], &stats[i], o.so.verify != 0);
  return noconv ? c.fail(FS_ERR_NOCONV, "some systems reached max_iter") : FS_OK;
}

int fs_hpe_exact_trace(fs_ctx* ctx, double m, double sigma, const double* gamma, int p, int K, uint64_t seed,
                       const fs_solve_params* params, double* out) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (!gamma || !out) return c.fail(FS_ERR_ARG, "null pointer");
  if (!c.have_gauge) return c.fail(FS_ERR_STATE, "no gauge field set");
  if (K < 1 || K > 8) return c.fail(FS_ERR_ARG, "K must be in [1, 8]");
  if (p < 0 || p >= c.g.L[2]) return c.fail(FS_ERR_ARG, "p must be in [0, Lz)");
  if (!std::isfinite(m) || !std::isfinite(sigma) || !finite_array(gamma, 32))
    return c.fail(FS_ERR_INPUT, "non-finite mass, shift or Gamma");
  if (std::fabs(4.0 + m + sigma) < 1e-12) return c.fail(FS_ERR_ARG, "4 + m + sigma must be nonzero");
  Opts o;
  if (int rc = resolve_params(c, params, 12, m, o)) return rc;  // 12 < 16: no tile autotuning
  if (int rc = set_device(c)) return rc;
  if (int rc = fs::clover_inverses(&c, m, &sigma, 1, o.so)) return rc;
  if (!params || params->rhs_tile == 0) o.tile = fs::MAX_TILE;  // the probing pieces fill whole tiles
  if (int rc = set_device(c)) return rc;
  fs::TileBase* T = c.tile(o.so.prec, o.tile, o.so.nr);
  if (!T) return c.fail(FS_ERR_OOM, "device allocation of the solver tile failed");
  if (int rc = fs::ensure_wline(&c, 1 << p, p)) return rc;
  return fs::hpe_exact(&c, T, o.so, sigma, K, p, gamma, seed, out);
}

// Probing colours of a call: every site has a colour in [0, ncolors) and every colour is used
// (no piece of a sample has an empty support).
static int check_colors(Ctx& c, const int32_t* colors, int ncolors) {
  std::vector<char> used(ncolors, 0);
  for (long long x = 0; x < c.g.V; x++) {
    const int32_t j = colors[x];
    if (j < 0 || j >= ncolors) return c.fail(FS_ERR_ARG, "probing colour out of range");
    used[j] = 1;
  }
  for (int j = 0; j < ncolors; j++)
    if (!used[j]) return c.fail(FS_ERR_ARG, "every probing colour must be used");
  return 0;
}

// Pieces of one sample: probing colours times spin-colour components (Sec. 2.1, Sec. 3.1).
static int num_pieces(const fs_mlmc_params* p) {
  if (p->dilute != 0 && p->dilute != 1) return -1;
  if (p->colors && (p->ncolors < 1 || p->ncolors > (1 << 26))) return -1;
  return (p->colors ? p->ncolors : 1) * (p->dilute ? 12 : 1);
}

int fs_mlmc_num_solves(const fs_mlmc_params* p) {
  if (!p || p->nlev < 1 || !p->n_samples) return -1;
  const int pieces = num_pieces(p);
  if (pieces < 1) return -1;
  long long n = 0;
  for (int l = 0; l < p->nlev; l++) {
    if (p->n_samples[l] < 0) return -1;
    n += (long long)p->n_samples[l] * (l + 1 < p->nlev ? 2 : 1);
  }
  n *= pieces;
  return n > 0x7FFFFFFF ? -1 : (int)n;
}

namespace {

// Level traces for the displacements p_in[0..np) from the same solves (the contraction forms all of
// them in one pass); outputs per displacement in the caller's order: trace [np][nlev][2],
// var [np][nlev], samples [np][sum N_l][2].
int mlmc_impl(Ctx& c, const fs_mlmc_params* P, const int* p_in, int np, double* trace, double* var, double* samples,
              fs_sys_stats* stats) {
  if (!P || !trace || !var || !p_in) return c.fail(FS_ERR_ARG, "null pointer");
  if (P->nlev < 1 || !P->sigma || !P->n_samples || !P->gamma) return c.fail(FS_ERR_ARG, "bad level parameters");
  if (!c.have_gauge) return c.fail(FS_ERR_STATE, "no gauge field set");
  if (np < 1 || np > fs::CONTRACT_MAXP) return c.fail(FS_ERR_ARG, "np must be in [1, 16]");
  // displacements are contracted in increasing order; order[qs] is the caller's index of the
  // qs-th smallest
  std::vector<int> order(np);
  for (int k = 0; k < np; k++) {
    if (p_in[k] < 0 || p_in[k] > 30) return c.fail(FS_ERR_ARG, "p must be in [0, 30]");
    order[k] = k;
  }
  std::sort(order.begin(), order.end(), [&](int a, int b) { return p_in[a] < p_in[b]; });
  std::vector<int> plist(np);
  int pmask = 0, pmax = 0;
  for (int k = 0; k < np; k++) {
    plist[k] = p_in[order[k]];
    if (pmask & (1 << plist[k])) return c.fail(FS_ERR_ARG, "displacements must be distinct");
    pmask |= 1 << plist[k];
    pmax = std::max(pmax, plist[k]);
  }
  if (P->estimator < FS_EST_DIFF || P->estimator > FS_EST_PRODUCT) return c.fail(FS_ERR_ARG, "bad estimator");
  if (!std::isfinite(P->m) || !finite_array(P->sigma, P->nlev) || !finite_array(P->gamma, 32))
    return c.fail(FS_ERR_INPUT, "non-finite mass, shift or Gamma");
  const int L = P->nlev - 1;
  long long total = 0;
  for (int l = 0; l <= L; l++) {
    if (P->n_samples[l] < 1) return c.fail(FS_ERR_ARG, "every level needs at least one sample");
    total += P->n_samples[l];
    if (l < L && !(P->sigma[l + 1] > P->sigma[l])) return c.fail(FS_ERR_ARG, "shifts must increase");
    if (std::fabs(4.0 + P->m + P->sigma[l]) < 1e-12) return c.fail(FS_ERR_ARG, "4 + m + sigma must be nonzero");
  }
  const int nsolve = fs_mlmc_num_solves(P);
  if (nsolve < 0) return c.fail(FS_ERR_ARG, "too many solves, or bad ncolors / dilute");
  const int npieces = num_pieces(P);
  const int ncomp = P->dilute ? 12 : 1;
  if (P->hpe_order < 0 || P->hpe_order > 8) return c.fail(FS_ERR_ARG, "hpe_order must be in [0, 8]");
  // the expansion converges for A = 4 + m + sigma > 4 only (Sec. 3.1 uses it where m + s > 0)
  const bool hpe = P->hpe_order > 0 && P->m + P->sigma[L] > 0.0;
  // the exact low orders take Omega_0 = 1; a displacement of a whole period is a Polyakov loop
  if (hpe && pmax >= c.g.L[2]) return c.fail(FS_ERR_ARG, "hpe_order needs p < Lz");
  if (P->colors)
    if (int rc = check_colors(c, P->colors, P->ncolors)) return rc;
  Opts o;
  if (int rc = resolve_params(c, &P->solve, nsolve, P->m, o)) return rc;
  if (int rc = set_device(c)) return rc;
  if (int rc = fs::clover_inverses(&c, P->m, P->sigma, P->nlev, o.so)) return rc;
  std::vector<double> csum((size_t)np * total * 2, 0.0);  // per-sample values [np][level-major][2]
  std::vector<long long> off(L + 2, 0);
  for (int l = 0; l <= L; l++) off[l + 1] = off[l] + P->n_samples[l];
  std::vector<fs::SysState> st(nsolve);
  std::vector<int> solve_off(L + 2, 0);
  for (int l = 0; l <= L; l++) solve_off[l + 1] = solve_off[l] + P->n_samples[l] * npieces * (l < L ? 2 : 1);
  int noconv = 0;
  // the noise of one piece: the sample's Z4 vector restricted to a colour and a component
  auto piece_noise = [&](int l, int s, int piece, bool g5) {
    fs::NoiseSpec n = noise_id(P->seed, P->job, l, s, g5);
    if (P->colors) {
      n.flags |= fs::NOISE_COLOR;
      n.color = piece / ncomp;
    }
    if (P->dilute) {
      n.flags |= fs::NOISE_COMP;
      n.comp = piece % ncomp;
    }
    return n;
  };
  // one result row per solve; the level sample is combined from the rows below
  std::vector<fs::QJob> jobs;
  for (int l = 0; l <= L; l++) {
    for (int s = 0; s < P->n_samples[l]; s++) {
      for (int piece = 0; piece < npieces; piece++) {
        const int si = solve_off[l] + (s * npieces + piece) * (l < L ? 2 : 1);
        const fs::NoiseSpec z = piece_noise(l, s, piece, false);
        fs::QJob q;
        if (l == L) {
          q.sys = {fs::SysSpec{P->sigma[L], 0, -1, z}};
          q.stat_index = {si};
          q.pairs = {{0, 0, 0, si}};
          if (hpe) {  // z^dag Gamma Omega_p (kappa H)^K x; the exact low orders are added below
            q.sys[0].hpe = 1;
            q.pairs[0].right_kind = 1;
          }
          jobs.push_back(q);
        } else if (P->estimator == FS_EST_DIFF) {
          // the two solves of a DIFF sample are independent: one group each packs slots best
          fs::QJob q2;
          q.sys = {fs::SysSpec{P->sigma[l], 0, -1, z}};
          q.stat_index = {si};
          q.pairs = {{0, 0, 0, si}};
          q2.sys = {fs::SysSpec{P->sigma[l + 1], 0, -1, z}};
          q2.stat_index = {si + 1};
          q2.pairs = {{0, 0, 0, si + 1}};
          jobs.push_back(q);
          jobs.push_back(q2);
        } else if (P->estimator == FS_EST_SPLIT_EVEN) {
          q.sys = {fs::SysSpec{P->sigma[l], 0, -1, piece_noise(l, s, piece, true)},
                   fs::SysSpec{P->sigma[l + 1], 0, -1, z}};
          q.stat_index = {si, si + 1};
          q.pairs = {{1, 0, 1, si}};  // y^dag Gamma Omega_p x_{l+1}, y = gamma_5 x~_l
          jobs.push_back(q);
        } else {
          // PRODUCT: x1 = (D + s_{l+1})^-1 z, then (D + s_l)^-1 x1 in the same slot
          q.sys = {fs::SysSpec{P->sigma[l + 1], 0, -1, z}};
          q.chain = {P->sigma[l]};
          q.stat_index = {si};
          q.stat_index2 = {si + 1};
          q.pairs = {{0, 0, 0, si}};
          jobs.push_back(q);
        }
      }
    }
  }
  // several tiles at once when the job fills them (lanes = 0: three, as many as the job fills);
  // a system's result is the same in any lane
  const int nl = o.lanes > 0 ? o.lanes : std::max(1, std::min(3, nsolve / std::max(1, o.tile)));
  fs::TileBase* T = nullptr;
  if (nl == 1) {
    T = tile_for(c, jobs, o);
    if (!T) return c.fail(FS_ERR_OOM, "device allocation of the solver tile failed");
    if (P->estimator == FS_EST_PRODUCT)
      if (int rc = c.ensure_canon(T->N)) return rc;
  }
  // exact low orders of the expansion (probing colours of their own, so computed before the
  // caller's colours are uploaded), on the owner's tile
  std::vector<double> t_exact((size_t)np * 2, 0.0);  // per sorted displacement
  if (hpe) {
    fs::TileBase* TE = T ? T : tile_for(c, jobs, o);
    if (!TE) return c.fail(FS_ERR_OOM, "device allocation of the solver tile failed");
    if (int rc = fs::ensure_wline(&c, pmask, pmax)) return rc;
    for (int qs = 0; qs < np; qs++)
      if (int rc = fs::hpe_exact(&c, TE, o.so, P->sigma[L], P->hpe_order, plist[qs], P->gamma, P->seed,
                                 &t_exact[(size_t)qs * 2]))
        return rc;
  }
  if (P->colors)
    if (int rc = fs::upload_colors(&c, P->colors)) return rc;
  std::vector<double> res;
  res.assign((size_t)nsolve * np * 2, 0.0);
  fs::QOut out;
  out.gamma = P->gamma;
  out.plist = &plist;
  out.rows = nsolve;
  out.hpe_order = hpe ? P->hpe_order : 0;
  out.result = &res;
  out.states = &st;
  out.noconv = &noconv;
  out.canon_chain_base = 0;
  if (nl > 1) {
    if (int rc = fs::ensure_wline(&c, pmask, pmax)) return rc;
    if (int rc = run_lanes(c, jobs, o, out, nl, P->estimator == FS_EST_PRODUCT)) return rc;
  } else if (int rc = fs::run_queue(&c, T, jobs, o.so, out)) {
    return rc;
  }
  // a sample is the sum of its pieces' estimators, in piece order; res rows are [solve][np][2]
  auto r = [&](int si, int qs, int ri) { return res[((size_t)si * np + qs) * 2 + ri]; };
  for (int qs = 0; qs < np; qs++) {
    const size_t qo = (size_t)order[qs] * total;  // the caller's displacement index
    for (int l = 0; l <= L; l++) {
      for (int s = 0; s < P->n_samples[l]; s++) {
        double re = 0.0, im = 0.0;
        for (int piece = 0; piece < npieces; piece++) {
          const int si = solve_off[l] + (s * npieces + piece) * (l < L ? 2 : 1);
          if (l == L) {
            re += r(si, qs, 0); im += r(si, qs, 1);
          } else if (P->estimator == FS_EST_DIFF) {
            re += r(si, qs, 0) - r(si + 1, qs, 0);
            im += r(si, qs, 1) - r(si + 1, qs, 1);
          } else {
            const double ds = P->sigma[l + 1] - P->sigma[l];
            re += ds * r(si, qs, 0); im += ds * r(si, qs, 1);
          }
        }
        if (l == L && hpe) {
          re += t_exact[(size_t)qs * 2];
          im += t_exact[(size_t)qs * 2 + 1];
        }
        csum[(qo + off[l] + s) * 2] = re;
        csum[(qo + off[l] + s) * 2 + 1] = im;
      }
    }
  }
  // per-level mean and practical variance, Eq. (practical_variance)
  for (int q = 0; q < np; q++) {
    const size_t qo = (size_t)q * total;
    for (int l = 0; l <= L; l++) {
      double tr, ti;
      var[(size_t)q * P->nlev + l] = practical_var(&csum[(qo + off[l]) * 2], P->n_samples[l], tr, ti);
      trace[((size_t)q * P->nlev + l) * 2] = tr;
      trace[((size_t)q * P->nlev + l) * 2 + 1] = ti;
    }
  }
  if (samples) memcpy(samples, csum.data(), csum.size() * sizeof(double));
  if (stats)
    for (int k = 0; k < nsolve; k++) fill_stats(st[k], &stats[k], o.so.verify != 0);
  return noconv ? c.fail(FS_ERR_NOCONV, "some systems reached max_iter") : FS_OK;
}

}  // namespace

int mlmc_level_trace(fs_ctx* ctx, const fs_mlmc_params* P, double* trace, double* var, double* samples,
                     fs_sys_stats* stats) {
  if (!ctx) return FS_ERR_ARG;
  if (!P) return ctx->c.fail(FS_ERR_ARG, "null pointer");
  return mlmc_impl(ctx->c, P, &P->p, 1, trace, var, samples, stats);
}

int mlmc_level_traces(fs_ctx* ctx, const fs_mlmc_params* P, const int* p, int np, double* trace, double* var,
                      double* samples, fs_sys_stats* stats) {
  if (!ctx) return FS_ERR_ARG;
  return mlmc_impl(ctx->c, P, p, np, trace, var, samples, stats);
}

namespace {

// Variance sampling (Sec. 3.1 algorithm) with optional probed / diluted noise: a noise vector's
// a_i and b_ij are sums over its pieces. With full spin-colour dilution a piece lives on one spin
// s, so gamma_5 z = eps z (eps = +1 for s < 2, -1 otherwise) and the adjoint solution is
// y^(i) = gamma_5 (D+s_i)^-1 gamma_5 z = eps gamma_5 x^(i): no second solve (Sec. 3.1).
int variance_sample_impl(Ctx& c, double m, const double* s_hat, int ms, const double* gamma, const int* p, int np,
                         int Ns, uint64_t seed, uint32_t job, const fs_solve_params* params, const int32_t* colors,
                         int ncolors, int dilute, int hpe_order, double* VL, double* Vbar, double* a_out,
                         double* b_out, double* iters) {
  if (hpe_order < 0 || hpe_order > 8) return c.fail(FS_ERR_ARG, "hpe_order must be in [0, 8]");
  if (!s_hat || !gamma || !p || !VL || !Vbar) return c.fail(FS_ERR_ARG, "null pointer");
  if (ms < 1 || 2 * ms > fs::MAX_TILE) return c.fail(FS_ERR_ARG, "m_shifts must be in [1, 32]");
  if (np < 1 || np > fs::CONTRACT_MAXP) return c.fail(FS_ERR_ARG, "np must be in [1, 16]");
  if (Ns < 1) return c.fail(FS_ERR_ARG, "Ns must be >= 1");
  if (dilute != 0 && dilute != 1) return c.fail(FS_ERR_ARG, "dilute must be 0 or 1");
  if (colors && (ncolors < 1 || ncolors > (1 << 26))) return c.fail(FS_ERR_ARG, "bad ncolors");
  if (!c.have_gauge) return c.fail(FS_ERR_STATE, "no gauge field set");
  if (!std::isfinite(m) || !finite_array(s_hat, ms) || !finite_array(gamma, 32))
    return c.fail(FS_ERR_INPUT, "non-finite mass, shift or Gamma");
  for (int i = 0; i < ms; i++) {
    if (i > 0 && !(s_hat[i] > s_hat[i - 1])) return c.fail(FS_ERR_ARG, "sampling shifts must increase");
    if (std::fabs(4.0 + m + s_hat[i]) < 1e-12) return c.fail(FS_ERR_ARG, "4 + m + sigma must be nonzero");
  }
  if (colors)
    if (int rc = check_colors(c, colors, ncolors)) return rc;
  const int ncomp = dilute ? 12 : 1;
  const long long npieces_ll = (long long)(colors ? ncolors : 1) * ncomp;
  const int gsize = dilute ? ms : 2 * ms;  // systems per piece: x^(i), and y^(i) unless diluted
  if ((long long)Ns * npieces_ll * gsize > 0x7FFFFFFF) return c.fail(FS_ERR_ARG, "too many solves");
  const int npieces = (int)npieces_ll;
  // displacements are contracted in increasing order; map back to the caller's order
  std::vector<int> order(np);
  for (int k = 0; k < np; k++) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return p[a] < p[b]; });
  std::vector<int> plist(np);
  for (int k = 0; k < np; k++) plist[k] = p[order[k]];
  const int nsys = Ns * npieces * gsize;
  Opts o;
  if (int rc = resolve_params(c, params, nsys, m, o)) return rc;
  if (int rc = set_device(c)) return rc;
  if (int rc = fs::clover_inverses(&c, m, s_hat, ms, o.so)) return rc;
  if (colors)
    if (int rc = fs::upload_colors(&c, colors)) return rc;
  // keep the requested tile even where whole groups leave a few slots idle: a multiple of 32
  // systems runs the persistent FP16 hop, which outweighs the idle slots
  o.tile = std::max(gsize, o.tile);
  const int per = ms + ms * (ms + 1) / 2;  // contraction rows per piece
  const size_t ngroups = (size_t)Ns * npieces;
  std::vector<fs::QJob> groups(ngroups);
  for (int k = 0; k < Ns; k++) {
    for (int pc = 0; pc < npieces; pc++) {
      const size_t gi = (size_t)k * npieces + pc;
      fs::QJob& g = groups[gi];
      auto piece = [&](bool g5) {
        fs::NoiseSpec n = noise_id(seed, job, 0x80000000u, k, g5);
        if (colors) {
          n.flags |= fs::NOISE_COLOR;
          n.color = pc / ncomp;
        }
        if (dilute) {
          n.flags |= fs::NOISE_COMP;
          n.comp = pc % ncomp;
        }
        return n;
      };
      for (int i = 0; i < ms; i++) g.sys.push_back(fs::SysSpec{s_hat[i], 0, -1, piece(false)});
      if (!dilute)
        for (int i = 0; i < ms; i++) g.sys.push_back(fs::SysSpec{s_hat[i], 0, -1, piece(true)});
      for (int i = 0; i < gsize; i++) g.stat_index.push_back((int)(gi * gsize + i));
      int row = (int)(gi * per);
      for (int i = 0; i < ms; i++) {
        // a_i; with the expansion (m + s_i > 0) the remainder z^dag Gamma Omega_p (kappa H)^K x^(i),
        // whose variance is V_L (the exact low orders shift every sample alike)
        fs::ContractPair q{i, i, 0, row++};
        if (hpe_order > 0 && m + s_hat[i] > 0.0) {
          g.sys[i].hpe = 1;
          q.right_kind = 1;
        }
        g.pairs.push_back(q);
      }
      for (int i = 0; i < ms; i++)
        for (int j = i; j < ms; j++)  // b_ij: y^(i) = gamma_5 x~^(i), x~ solved for gamma_5 z (or eps x^(i))
          g.pairs.push_back({j, dilute ? i : ms + i, 1, row++});
    }
  }
  std::vector<double> res(ngroups * per * np * 2, 0.0);
  std::vector<fs::SysState> st((size_t)nsys);
  int noconv = 0;
  fs::TileBase* T = tile_for(c, groups, o);
  if (!T) return c.fail(FS_ERR_OOM, "device allocation of the solver tile failed");
  fs::QOut out;
  out.gamma = gamma;
  out.plist = &plist;
  out.rows = (int)(ngroups * per);
  out.result = &res;
  out.states = &st;
  out.noconv = &noconv;
  out.hpe_order = hpe_order;
  if (int rc = fs::run_queue(&c, T, groups, o.so, out)) return rc;
  // a noise vector's value of row r: the sum over its pieces (b rows carry eps with dilution)
  auto val = [&](int k, int r, int q, int ri) {
    double sum = 0.0;
    for (int pc = 0; pc < npieces; pc++) {
      const double sgn = (dilute && r >= ms && (pc % ncomp) / 3 >= 2) ? -1.0 : 1.0;
      sum += sgn * res[((((size_t)k * npieces + pc) * per + r) * np + q) * 2 + ri];
    }
    return sum;
  };
  for (int qs = 0; qs < np; qs++) {
    const int q = order[qs];  // caller's index of the qs-th smallest displacement
    std::vector<double> cs((size_t)Ns * 2);
    double tr, ti;
    for (int i = 0; i < ms; i++) {
      for (int k = 0; k < Ns; k++) {
        const double re = val(k, i, qs, 0), im = val(k, i, qs, 1);
        cs[(size_t)k * 2] = re;
        cs[(size_t)k * 2 + 1] = im;
        if (a_out) {
          a_out[(((size_t)k * np + q) * ms + i) * 2] = re;
          a_out[(((size_t)k * np + q) * ms + i) * 2 + 1] = im;
        }
      }
      VL[(size_t)q * ms + i] = practical_var(cs.data(), Ns, tr, ti);
    }
    int r = ms;
    for (int i = 0; i < ms; i++) {
      for (int j = 0; j < ms; j++) {
        if (j < i) {
          Vbar[((size_t)q * ms + i) * ms + j] = 0.0;
          if (b_out)
            for (int k = 0; k < Ns; k++) {
              b_out[((((size_t)k * np + q) * ms + i) * ms + j) * 2] = 0.0;
              b_out[((((size_t)k * np + q) * ms + i) * ms + j) * 2 + 1] = 0.0;
            }
          continue;
        }
        for (int k = 0; k < Ns; k++) {
          const double re = val(k, r, qs, 0), im = val(k, r, qs, 1);
          cs[(size_t)k * 2] = re;
          cs[(size_t)k * 2 + 1] = im;
          if (b_out) {
            b_out[((((size_t)k * np + q) * ms + i) * ms + j) * 2] = re;
            b_out[((((size_t)k * np + q) * ms + i) * ms + j) * 2 + 1] = im;
          }
        }
        Vbar[((size_t)q * ms + i) * ms + j] = practical_var(cs.data(), Ns, tr, ti);
        r++;
      }
    }
  }
  if (iters) {
    // mean iterations of every solve at shift i (x^(i), and y^(i) unless diluted)
    for (int i = 0; i < ms; i++) {
      double sum = 0;
      for (size_t gi = 0; gi < ngroups; gi++) {
        sum += st[gi * gsize + i].iters;
        if (!dilute) sum += st[gi * gsize + ms + i].iters;
      }
      iters[i] = sum / ((double)ngroups * (dilute ? 1 : 2));
    }
  }
  return noconv ? c.fail(FS_ERR_NOCONV, "some systems reached max_iter") : FS_OK;
}

}  // namespace

int variance_sample(fs_ctx* ctx, double m, const double* s_hat, int ms, const double* gamma, const int* p, int np,
                    int Ns, uint64_t seed, uint32_t job, const fs_solve_params* params, double* VL, double* Vbar,
                    double* a_out, double* b_out, double* iters) {
  if (!ctx) return FS_ERR_ARG;
  return variance_sample_impl(ctx->c, m, s_hat, ms, gamma, p, np, Ns, seed, job, params, nullptr, 0, 0, 0, VL,
                              Vbar, a_out, b_out, iters);
}

int variance_sample_probed(fs_ctx* ctx, double m, const double* s_hat, int ms, const double* gamma, const int* p,
                           int np, int Ns, uint64_t seed, uint32_t job, const fs_solve_params* params,
                           const int32_t* colors, int ncolors, int dilute, int hpe_order, double* VL, double* Vbar,
                           double* a_out, double* b_out, double* iters) {
  if (!ctx) return FS_ERR_ARG;
  return variance_sample_impl(ctx->c, m, s_hat, ms, gamma, p, np, Ns, seed, job, params, colors, ncolors, dilute,
                              hpe_order, VL, Vbar, a_out, b_out, iters);
}

int fs_noise_codes(fs_ctx* ctx, uint64_t seed, uint32_t job, uint32_t level, uint32_t sample, uint8_t* codes) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (!codes) return c.fail(FS_ERR_ARG, "null output");
  if (int rc = set_device(c)) return rc;
  const size_t n = (size_t)c.g.V * 12;
  uint8_t* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, n, c.stream);
  if (!e) e = fs::launch_noise_codes(d, noise_id(seed, job, level, sample, false), c.g.V, c.stream);
  if (!e) e = cudaMemcpyAsync(codes, d, n, cudaMemcpyDeviceToHost, c.stream);
  if (d) cudaFreeAsync(d, c.stream);
  if (!e) e = cudaStreamSynchronize(c.stream);
  return e ? c.cuda_fail(e, "fs_noise_codes") : FS_OK;
}

int fs_profile_enable(fs_ctx* ctx, int enable) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (int rc = set_device(c)) return rc;
  if (int rc = prof_reset(c, enable != 0)) return rc;
  for (auto& l : c.lanes)
    if (prof_reset(*l, enable != 0)) return c.fail(FS_ERR_CUDA, l->err);
  return FS_OK;
}

int fs_profile_read(fs_ctx* ctx, long long* launches, double* total_ms, double* bytes, double* site_systems) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (int rc = set_device(c)) return rc;
  long long n = 0;
  double ms = 0, b = 0, pairs = 0;
  if (int rc = prof_collect(c, n, ms, b, pairs)) return rc;
  for (auto& l : c.lanes)
    if (prof_collect(*l, n, ms, b, pairs)) return c.fail(FS_ERR_CUDA, l->err);
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (bytes) *bytes = b;
  if (site_systems) *site_systems = pairs;
  return FS_OK;
}

int fs_set_iteration_bound(fs_ctx* ctx, long long bound) {
  if (!ctx) return FS_ERR_ARG;
  if (bound < 0) return ctx->c.fail(FS_ERR_ARG, "negative iteration bound");
  ctx->c.iter_bound = bound;
  for (auto& l : ctx->c.lanes) l->iter_bound = bound;
  return FS_OK;
}

int fs_profile_read_fp64(fs_ctx* ctx, long long* launches, double* total_ms, double* site_systems) {
  if (!ctx) return FS_ERR_ARG;
  Ctx& c = ctx->c;
  if (int rc = set_device(c)) return rc;
  long long n = 0;
  double ms = 0, b = 0, pairs = 0;
  if (int rc = prof_collect(c, n, ms, b, pairs, true)) return rc;
  for (auto& l : c.lanes)
    if (prof_collect(*l, n, ms, b, pairs, true)) return c.fail(FS_ERR_CUDA, l->err);
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (site_systems) *site_systems = pairs;
  return FS_OK;
}

long long fs_kernel_launches(void) { return fs::launch_count(); }

}  // extern "C"
