// Continuous batching of shifted solves over the slots of one tile.
//
// Systems arrive as groups (systems whose solutions are contracted together).
// A group is admitted when enough slots are free; its slots are initialised
// (noise or caller right-hand side, even-odd preparation) while the other slots
// keep iterating, since every kernel masks by slot state. When all systems of a
// group have converged, the group is harvested (odd-site reconstruction, optional
// FP64 verification, contractions, outputs) and its slots are reused at once. A
// system with a follow-up shift (the nested solve of the product estimator) is
// re-initialised in place with its own solution as the next right-hand side.
#include "fs_engine.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "fsmlmc.h"

namespace fs {

namespace {

void set_coef_h(SysState& s, int k, double v) {
  s.cd[k] = v;
  s.cf[k] = (float)v;
}

void init_state(SysState& s, double sigma, const SolveOpts& o) {
  memset(&s, 0, sizeof(SysState));
  const double A = 4.0 + o.m + sigma;
  s.sigma = sigma;
  s.A = A;
  s.inv4A = 1.0 / (4.0 * A);
  set_coef_h(s, C_A, A);
  set_coef_h(s, C_MINV4A, -1.0 / (4.0 * A));
  set_coef_h(s, C_INV2A, 1.0 / (2.0 * A));
  set_coef_h(s, C_INVA, 1.0 / A);
  set_coef_h(s, C_INV4A, 1.0 / (4.0 * A));
  set_coef_h(s, C_MINVA, -A);
  set_coef_h(s, C_SCALE, 1.0);
  set_coef_h(s, C_INVSCALE, 1.0);
  s.tol2 = o.tol * o.tol;  // made absolute (x ||z||^2) on the device
  s.delta2 = o.delta * o.delta;
  s.max_iter = o.max_iter;
  s.status = SYS_IDLE;
  s.flags = FLAG_INIT;
  if (o.clv_inv != nullptr) {  // Wilson-clover: the packed inverse of this shift, where the call built one
    auto it = o.clv_inv->find(A);
    if (it != o.clv_inv->end()) {
      s.clv_inv64 = it->second.t64;
      s.clv_inv32 = it->second.t32;
    }
  }
}

cudaError_t upload_slots(Ctx* c, TileBase* T, const std::vector<int>& slots) {
  for (int j : slots) {
    cudaError_t e = cudaMemcpyAsync(T->st_d + j, T->st_h + j, sizeof(SysState), cudaMemcpyHostToDevice, c->stream);
    if (!e) e = cudaMemcpyAsync(T->spec_d + j, T->spec_h + j, sizeof(NoiseSpec), cudaMemcpyHostToDevice, c->stream);
    if (e) return e;
  }
  return cudaSuccess;
}

cudaError_t upload_vec(Ctx* c, TileBase* T) {
  return cudaMemcpyAsync(T->vec_d, T->vec_h, sizeof(int) * T->N, cudaMemcpyHostToDevice, c->stream);
}

// Every slot of T idle, on the host mirror and the device (the stream synchronised): a call that
// stops early (its iteration bound ran out) leaves no system running into the next call.
void idle_all(Ctx* c, TileBase* T) {
  for (int j = 0; j < T->N; j++) {
    T->st_h[j].status = SYS_IDLE;
    T->st_h[j].flags = 0;
  }
  if (cudaMemcpyAsync(T->st_d, T->st_h, sizeof(SysState) * T->N, cudaMemcpyHostToDevice, c->stream) == cudaSuccess)
    cudaStreamSynchronize(c->stream);
}

// CGNR fallback for the slots BiCGStab left unconverged: bounded host loop of
// device iterations; returns with the stream idle and st_h current.
int run_cg(Ctx* c, TileBase* T, const std::vector<int>& slots, const SolveOpts& o) {
  if (T->cg_alloc()) return c->fail(3, "device allocation of the CGNR fallback vectors failed");
  for (int j : slots) {
    SysState& s = T->st_h[j];
    s.status = SYS_ACTIVE;
    s.flags = FLAG_CG;
    s.cg_iters = 0;
    s.cg_max_iter = o.cg_max_iter;
  }
  cudaError_t e = upload_slots(c, T, slots);
  if (!e) e = T->enqueue_cg_init();
  if (e) return c->cuda_fail(e, "CGNR fallback initialisation");
  const int every = 16;
  const long long bound = c->iter_bound > 0 ? c->iter_bound : (long long)o.cg_max_iter + 2 * every;
  for (long long it = 0;; it += every) {
    for (int k = 0; k < every && !e; k++) e = T->enqueue_cg_iter();
    if (!e) e = cudaMemcpyAsync(T->st_h, T->st_d, sizeof(SysState) * T->N, cudaMemcpyDeviceToHost, c->stream);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) return c->cuda_fail(e, "CGNR fallback iteration");
    bool active = false;
    for (int j : slots) active |= T->st_h[j].status == SYS_ACTIVE;
    if (!active) return 0;
    if (it > bound) {
      idle_all(c, T);
      return c->fail(6, "CGNR fallback did not terminate within its iteration bound");
    }
  }
}

}  // namespace

// Tile autotuner. The tile size sets how many systems share each site's links in the hop
// kernels, which kernel variant runs (the persistent kernel for 32-system chunks, the
// prefetch kernel otherwise) and how many blocks the BLAS steps launch; the FP64 reliable
// updates run per system and do not depend on it. So the candidates (8, 16, 32, 64 systems)
// are compared by the time of a BiCGStab iteration per system: each tile is filled with Z4
// right-hand sides through the normal initialisation, iterated 4 times untimed and 8 times
// timed with CUDA events (the graph path the solver uses). A candidate that is not the best so
// far is released at once, and every slot of the chosen tile is left idle.
int autotune_tile(Ctx* c, const SolveOpts& o, int nmax) {
  const int key = o.prec * 100 + o.nr;
  auto it = c->tuned_tile.find(key);
  if (it != c->tuned_tile.end()) return std::min(it->second, nmax);
  static const int cand[] = {8, 16, 32, 64};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return 0;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return 0; }
  SolveOpts to = o;
  to.max_iter = 1 << 20;  // no system stops during the trial
  to.delta = 0.0;         // and none takes a reliable update (per system, the same for every tile)
  // fills T with Z4 right-hand sides, runs 4 untimed and 8 timed BiCGStab iterations on the graph
  // path and returns their milliseconds (every slot left idle afterwards); < 0 on failure
  auto trial = [&](TileBase* T) -> float {
    const int N = T->N;
    std::vector<int> all(N);
    for (int j = 0; j < N; j++) {
      all[j] = j;
      init_state(T->st_h[j], 0.1, to);
      NoiseSpec n{};
      n.key0 = 0x5EEDu;
      n.job = 0xFFFFFFFFu;
      n.sample = (uint32_t)j;
      n.flags = NOISE_VALID | NOISE_RHS;
      T->spec_h[j] = n;
    }
    cudaError_t e = upload_slots(c, T, all);
    if (!e) e = T->enqueue_noise();
    if (!e) e = T->enqueue_init();
    if (!e) e = T->enqueue_iters(4);  // eager (first use) or graph, untimed
    if (!e) e = T->enqueue_iters(4);
    if (!e) e = cudaEventRecord(e0, c->stream);
    if (!e) e = T->enqueue_iters(4);
    if (!e) e = T->enqueue_iters(4);
    if (!e) e = cudaEventRecord(e1, c->stream);
    if (!e) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    for (int j = 0; j < N; j++) {
      memset(&T->st_h[j], 0, sizeof(SysState));
      T->st_h[j].status = SYS_IDLE;
    }
    if (!e) e = upload_slots(c, T, all);
    if (!e) e = cudaStreamSynchronize(c->stream);
    if (e) {
      c->cuda_fail(e, "tile autotuner");
      return -1.f;
    }
    return ms;
  };
  auto done = [&](int r) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
  };
  double best_t = 0.0;
  int best = 0;
  for (int N : cand) {
    if (N > nmax) break;
    TileBase* T = c->tile(o.prec, N, o.nr);
    if (!T) break;  // no room for a tile this large
    const float ms = trial(T);
    if (ms < 0.f) return done(0);
    const double per = ms / (8.0 * N);
    // keep only the best tile so far: at most two candidates hold device memory at once
    if (best == 0 || per < best_t) {
      if (best) c->tiles.erase(((long long)o.prec * 1000 + best) * 100 + o.nr);
      best_t = per;
      best = N;
    } else {
      c->tiles.erase(((long long)o.prec * 1000 + N) * 100 + o.nr);
    }
  }
  // the launch shape of the persistent hop (tiles of 32-system chunks in the inner precision):
  // ring depth and resident blocks per SM, timed on the chosen tile in the same way
  if (best > 0 && best % 32 == 0 && o.prec != PREC_F64) {
    TileBase* T = c->tile(o.prec, best, o.nr);
    if (T) {
      static const PkShape shapes[] = {{0, 0}, {3, 0}, {0, 2}, {3, 2}};
      PkShape pick{};
      float pick_ms = 0.f;
      for (const PkShape& sh : shapes) {
        T->set_shape(sh);
        const float ms = trial(T);
        if (ms < 0.f) return done(0);
        if (pick_ms == 0.f || ms < pick_ms) {
          pick_ms = ms;
          pick = sh;
        }
      }
      T->set_shape(pick);
      c->tuned_shape[(long long)key * 1000 + best] = pick;
    }
  }
  if (best > 0) c->tuned_tile[key] = best;
  return done(best);
}

// Exact low orders of the hopping parameter expansion. D + s = A (1 - kappa H), so
// (D + s)^-1 = sum_{k<K} (kappa H)^k / A + (kappa H)^K (D + s)^-1, and the traces of the first K
// terms are deterministic. Order 0 is Tr(Gamma Omega_p) = 3 V tr(Gamma) for p = 0 (Omega_p moves
// every site otherwise). Orders 1..K-1 link site x only to sites within distance K - 1 of x + p z,
// so with displacement-p distance-(K-1) colours no two distinct sites of one colour are linked,
// and for the pieces e (one colour, one spin-colour index, unit-modulus Z4 entries)
// sum_e e^dag Gamma Omega_p (kappa H)^k e is the trace exactly. The pieces fill the tile N at a
// time; each power is one FP64 kappa H application (work list over the pieces) and one
// contraction.
int hpe_exact(Ctx* c, TileBase* T, const SolveOpts& o, double sigma, int K, int p, const double* gamma,
              uint64_t seed, double out[2]) {
  // Wilson-clover (the generalised expansion): T = sum_{k<K} Tr(Gamma Omega_p K^k A^-1), K = A(x)^-1 H / 2,
  // A(x) = A + C(x) per site, every order from the pieces (order 0 has no closed form), no 1/A
  const bool clv = c->c_sw != 0.0;
  const double A = clv ? 1.0 : 4.0 + o.m + sigma;
  double tr = 0.0, ti = 0.0;
  if (p < 0 || p >= c->g.L[2]) return c->fail(1, "the expansion's exact part needs 0 <= p < Lz");
  const int pz = p;
  if (pz == 0 && !clv)
    for (int s = 0; s < 4; s++) {
      tr += 3.0 * c->g.V * gamma[(s * 4 + s) * 2];
      ti += 3.0 * c->g.V * gamma[(s * 4 + s) * 2 + 1];
    }
  if (K > 1 || clv) {
    std::vector<int32_t> colors((size_t)c->g.V);
    int nc = 0;
    // (order 0 alone, with the clover term: distance-1 colours, finer than it needs)
    if (int rc = fs_probing_colors(c->g.L, std::max(K - 1, 1), pz, colors.data(), &nc))
      return c->fail(rc, "probing colours of the hopping parameter expansion");
    if (int rc = upload_colors(c, colors.data())) return rc;
    const int N = T->N;
    const long long npieces = 12LL * nc;
    const std::vector<int> plist = {p};
    std::vector<int> all(N);
    std::iota(all.begin(), all.end(), 0);
    cudaError_t e;
    for (long long base = 0; base < npieces; base += N) {
      const int nb = (int)std::min<long long>(N, npieces - base);
      // the host mirrors are rewritten below: every earlier upload must have executed
      if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "hopping parameter expansion");
      std::vector<ContractPair> pairs;
      for (int j = 0; j < N; j++) {
        if (j < nb) {
          init_state(T->st_h[j], sigma, o);  // FLAG_INIT: the noise kernel writes the piece
          T->st_h[j].flags |= FLAG_HPE;
          NoiseSpec n{};
          n.key0 = (uint32_t)(seed & 0xFFFFFFFFull);
          n.key1 = (uint32_t)(seed >> 32);
          n.level = 0x40000000u;
          n.flags = NOISE_VALID | NOISE_RHS | NOISE_COLOR | NOISE_COMP;
          n.color = (int)((base + j) / 12);
          n.comp = (int)((base + j) % 12);
          T->spec_h[j] = n;
          ContractPair q{j, j, 0, j};
          q.right_kind = 1;
          pairs.push_back(q);
        } else {
          memset(&T->st_h[j], 0, sizeof(SysState));
          memset(&T->spec_h[j], 0, sizeof(NoiseSpec));
        }
      }
      if ((e = upload_slots(c, T, all))) return c->cuda_fail(e, "hopping parameter expansion");
      if ((e = T->enqueue_noise())) return c->cuda_fail(e, "hopping parameter expansion");
      int from = PAIR_Z;
      if (clv) {
        // order 0: A(x)^-1 e
        if ((e = T->enqueue_site_inverse(PAIR_Z, PAIR_S))) return c->cuda_fail(e, "hopping parameter expansion");
        std::vector<double> part;
        if (int rc = contract_tile(c, T, pairs, gamma, plist, part, N, PAIR_S)) return rc;
        for (int j = 0; j < nb; j++) {
          tr += part[(size_t)j * 2];
          ti += part[(size_t)j * 2 + 1];
        }
        from = PAIR_S;
      }
      for (int k = 1; k < K; k++) {
        const int to = (from == PAIR_S) ? PAIR_X : PAIR_S;
        if ((e = T->enqueue_kappa_hop(from, to))) return c->cuda_fail(e, "hopping parameter expansion");
        std::vector<double> part;
        if (int rc = contract_tile(c, T, pairs, gamma, plist, part, N, to)) return rc;
        for (int j = 0; j < nb; j++) {
          tr += part[(size_t)j * 2];
          ti += part[(size_t)j * 2 + 1];
        }
        from = to;
      }
    }
    // leave the tile idle for the solves
    if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "hopping parameter expansion");
    for (int j = 0; j < N; j++) {
      memset(&T->st_h[j], 0, sizeof(SysState));
      memset(&T->spec_h[j], 0, sizeof(NoiseSpec));
    }
    if ((e = upload_slots(c, T, all))) return c->cuda_fail(e, "hopping parameter expansion");
    if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "hopping parameter expansion");
  }
  out[0] = tr / A;
  out[1] = ti / A;
  return 0;
}

int run_queue(Ctx* c, TileBase* T, const std::vector<QJob>& jobs, const SolveOpts& o, const QOut& out) {
  const int N = T->N;
  for (const QJob& q : jobs)
    if ((int)q.sys.size() > N) return c->fail(1, "a group of systems does not fit in one tile");
  const int np = out.plist ? (int)out.plist->size() : 0;
  const size_t vlen = (size_t)c->g.V * 24;

  // Staging (groups of several systems contracted together): a finished system leaves the tile at
  // once, its FP64 solution (and expanded vector) copied to a staging column reserved for it at
  // admission, and the group is contracted from staging when its last member arrives. Without it
  // a group holds all its slots until its slowest member converges (a variance-sampling group
  // spans five shifts). Not for follow-up solves or caller-requested solution vectors.
  bool staged = out.result && np > 0 && !out.x_host && !out.x_dev;
  int gmax = 1;
  for (const QJob& q : jobs) {
    gmax = std::max(gmax, (int)q.sys.size());
    for (double ch : q.chain)
      if (!std::isnan(ch)) staged = false;
  }
  if (gmax < 2) staged = false;
  const int S = 2 * N;  // reserved columns bound the groups in flight to twice the tile
  if (staged && T->stage_alloc(S, out.hpe_order > 0) != 0) staged = false;  // no room: groups keep their slots
  std::vector<int> stage_free;
  if (staged)
    for (int k = S - 1; k >= 0; k--) stage_free.push_back(k);
  std::vector<std::vector<int>> stage_col(staged ? jobs.size() : 0);
  const size_t colsz = (size_t)24 * c->g.Vh;  // doubles of one staged parity column

  struct Slot {
    int job = -1, member = -1, phase = 0;
    bool done = false;
    bool cg_tried = false;  // the CGNR fallback ran on this phase
  };
  std::vector<Slot> slot(N);
  std::vector<int> free_slots;
  for (int j = N - 1; j >= 0; j--) free_slots.push_back(j);
  std::vector<int> remaining(jobs.size(), 0);  // members not yet in their final state
  size_t next = 0, finished = 0;
  cudaError_t e;
  const int every = std::max(1, o.check_every);
  long long iters_run = 0;
  // every system stops at max_iter (FLAG_FINAL); a follow-up solve doubles that (the caller's
  // watchdog bound, fs_set_iteration_bound, replaces it)
  const long long bound =
      c->iter_bound > 0 ? c->iter_bound : ((long long)o.max_iter * 2 + 64) * (long long)(jobs.size() + 1);
  // no slot carries a system over from an earlier call that stopped early
  idle_all(c, T);

  // The host mirrors st_h / spec_h / vec_h are pinned and uploaded asynchronously: the host
  // must not write them again until the copies that read them have executed. Every batch
  // of uploads records `fence`; every host write waits on it first.
  cudaEvent_t fence;
  if ((e = cudaEventCreateWithFlags(&fence, cudaEventDisableTiming))) return c->cuda_fail(e, "event");
  struct FenceGuard {
    cudaEvent_t ev;
    ~FenceGuard() { cudaEventDestroy(ev); }
  } fence_guard{fence};
  bool fence_pending = false;
  auto mark = [&]() -> cudaError_t {
    fence_pending = true;
    return cudaEventRecord(fence, c->stream);
  };
  auto wait_fence = [&]() -> cudaError_t {
    if (!fence_pending) return cudaSuccess;
    fence_pending = false;
    return cudaEventSynchronize(fence);
  };

  auto admit_rhs = [&](const std::vector<int>& adm, bool any_vec, bool any_noise) -> int {
    if ((e = upload_slots(c, T, adm))) return c->cuda_fail(e, "upload slot state");
    if (any_vec && (e = upload_vec(c, T))) return c->cuda_fail(e, "upload vector map");
    if ((e = mark())) return c->cuda_fail(e, "upload fence");
    if (any_vec && (e = T->enqueue_rhs_from_canon(out.rhs_canon ? out.rhs_canon : c->canon_d)))
      return c->cuda_fail(e, "pack right-hand sides");
    if (any_noise && (e = T->enqueue_noise())) return c->cuda_fail(e, "noise");
    if ((e = T->enqueue_init())) return c->cuda_fail(e, "solver initialisation");
    return 0;
  };

  // groups completed and systems finished since the last harvest: kept across a pass that runs
  // the CGNR fallback first, so that no completion is lost
  std::vector<int> done_jobs;
  std::vector<int> newly_done;
  while (finished < jobs.size()) {
    if ((e = wait_fence())) return c->cuda_fail(e, "upload fence");
    // ---- admit whole groups into free slots
    std::vector<int> adm;
    bool any_vec = false, any_noise = false;
    for (int j = 0; j < N; j++) T->vec_h[j] = -1;
    while (next < jobs.size() && free_slots.size() >= jobs[next].sys.size() &&
           (!staged || stage_free.size() >= jobs[next].sys.size())) {
      const QJob& q = jobs[next];
      remaining[next] = (int)q.sys.size();
      if (staged)
        for (size_t k = 0; k < q.sys.size(); k++) {
          stage_col[next].push_back(stage_free.back());
          stage_free.pop_back();
        }
      for (size_t k = 0; k < q.sys.size(); k++) {
        const int j = free_slots.back();
        free_slots.pop_back();
        slot[j] = Slot{(int)next, (int)k, 0, false};
        const SysSpec& sp = q.sys[k];
        init_state(T->st_h[j], sp.sigma, o);
        T->spec_h[j] = sp.noise;
        if (sp.rhs_kind == 0) {
          T->spec_h[j].flags |= NOISE_RHS;
          any_noise = true;
        } else {
          T->vec_h[j] = sp.vec;
          any_vec = true;
        }
        adm.push_back(j);
      }
      next++;
    }
    if (!adm.empty())
      if (int rc = admit_rhs(adm, any_vec, any_noise)) return rc;

    // ---- iterate
    if ((e = T->enqueue_iters(every))) return c->cuda_fail(e, "solver iteration");
    iters_run += every;
    if ((e = cudaMemcpyAsync(T->st_h, T->st_d, sizeof(SysState) * N, cudaMemcpyDeviceToHost, c->stream)))
      return c->cuda_fail(e, "download system state");
    if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "solver iteration");
    if (iters_run > bound) {
      idle_all(c, T);
      return c->fail(6, "solver did not terminate within its iteration bound");
    }

    // ---- find finished systems
    std::vector<int> chain_slots;
    std::vector<int> cg_slots;
    for (int j = 0; j < N; j++) {
      Slot& sl = slot[j];
      if (sl.job < 0 || sl.done) continue;
      const SysState& s = T->st_h[j];
      if (s.status != SYS_CONVERGED && s.status != SYS_NOCONV) continue;
      if (s.status == SYS_NOCONV && o.cg_max_iter > 0 && !sl.cg_tried) {
        cg_slots.push_back(j);
        continue;
      }
      const QJob& q = jobs[sl.job];
      const bool has_chain = !q.chain.empty() && !std::isnan(q.chain[sl.member]);
      if (s.status != SYS_CONVERGED && out.noconv) *out.noconv = 1;
      if (sl.phase == 0 && has_chain) {
        chain_slots.push_back(j);
        continue;
      }
      sl.done = true;
      newly_done.push_back(j);
      if (--remaining[sl.job] == 0) done_jobs.push_back(sl.job);
    }
    if (!cg_slots.empty()) {
      // BiCGStab failed on these systems: CGNR from their last reliable iterate; the next
      // pass through the loop harvests them with the fallback's verdict
      if (int rc = run_cg(c, T, cg_slots, o)) return rc;
      for (int j : cg_slots) slot[j].cg_tried = true;
      continue;
    }
    if (chain_slots.empty() && done_jobs.empty() && !(staged && !newly_done.empty())) continue;

    // ---- harvest: reconstruct the odd sites (and verify) of every slot leaving its phase
    // (staged: every finished system; else the systems of completed groups)
    std::vector<int> harvest = chain_slots;
    if (staged)
      harvest.insert(harvest.end(), newly_done.begin(), newly_done.end());
    else
      for (int j = 0; j < N; j++)
        if (slot[j].job >= 0 && slot[j].done &&
            std::find(done_jobs.begin(), done_jobs.end(), slot[j].job) != done_jobs.end())
          harvest.push_back(j);
    for (int j : harvest) T->st_h[j].flags |= FLAG_HARVEST;
    if ((e = upload_slots(c, T, harvest))) return c->cuda_fail(e, "upload harvest flags");
    if ((e = T->enqueue_recon())) return c->cuda_fail(e, "reconstruct odd sites");
    if (o.verify && (e = T->enqueue_verify())) return c->cuda_fail(e, "verify residual");
    if ((e = cudaMemcpyAsync(T->st_h, T->st_d, sizeof(SysState) * N, cudaMemcpyDeviceToHost, c->stream)))
      return c->cuda_fail(e, "download system state");
    if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "harvest");

    // statistics of every harvested phase
    for (int j : harvest) {
      const QJob& q = jobs[slot[j].job];
      const std::vector<int>& si = slot[j].phase == 0 ? q.stat_index : q.stat_index2;
      if (out.states && !si.empty() && si[slot[j].member] >= 0) (*out.states)[si[slot[j].member]] = T->st_h[j];
    }

    // hopping parameter expansion: y = (kappa H)^K x for the finished systems that take it
    // (their right-hand side and scratch pairs are free now; x stays for the other contractions)
    int right_pair = PAIR_X;
    std::vector<char> is_hpe(N, 0);
    if (out.hpe_order > 0 && (!done_jobs.empty() || (staged && !newly_done.empty()))) {
      std::vector<int> hpe_slots;
      for (int j = 0; j < N; j++) {
        if (slot[j].job < 0 || !slot[j].done || !jobs[slot[j].job].sys[slot[j].member].hpe) continue;
        const bool now = staged ? std::find(newly_done.begin(), newly_done.end(), j) != newly_done.end()
                                : std::find(done_jobs.begin(), done_jobs.end(), slot[j].job) != done_jobs.end();
        if (!now) continue;
        T->st_h[j].flags |= FLAG_HPE;
        hpe_slots.push_back(j);
        is_hpe[j] = 1;
      }
      if (!hpe_slots.empty()) {
        if ((e = upload_slots(c, T, hpe_slots))) return c->cuda_fail(e, "upload expansion flags");
        int from = PAIR_X;
        for (int k = 0; k < out.hpe_order; k++) {
          const int to = (k % 2 == 0) ? PAIR_S : PAIR_Z;
          if ((e = T->enqueue_kappa_hop(from, to))) return c->cuda_fail(e, "hopping parameter expansion");
          from = to;
        }
        right_pair = hpe_result_pair(out.hpe_order);
      }
    }

    // staged: the finished systems' vectors go to their columns and their slots are free at once
    if (staged && !newly_done.empty()) {
      const size_t cb = colsz * sizeof(double);
      for (int j : newly_done) {
        const size_t col = (size_t)stage_col[slot[j].job][slot[j].member];
        const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
        e = cudaMemcpyAsync(T->stage_x_e + col * colsz, T->x_hi + (size_t)j * colsz, cb, d2d, c->stream);
        if (!e) e = cudaMemcpyAsync(T->stage_x_o + col * colsz, T->x_o + (size_t)j * colsz, cb, d2d, c->stream);
        if (!e && is_hpe[j]) {
          e = cudaMemcpyAsync(T->stage_y_e + col * colsz, T->field_pair(right_pair, 0) + (size_t)j * colsz, cb, d2d,
                              c->stream);
          if (!e)
            e = cudaMemcpyAsync(T->stage_y_o + col * colsz, T->field_pair(right_pair, 1) + (size_t)j * colsz, cb,
                                d2d, c->stream);
        }
        T->stage_spec_h[col] = T->spec_h[j];
        if (!e)
          e = cudaMemcpyAsync(T->stage_spec_d + col, T->stage_spec_h + col, sizeof(NoiseSpec), cudaMemcpyHostToDevice,
                              c->stream);
        if (e) return c->cuda_fail(e, "stage solutions");
      }
      for (int j : newly_done) {
        memset(&T->st_h[j], 0, sizeof(SysState));
        memset(&T->spec_h[j], 0, sizeof(NoiseSpec));
        slot[j] = Slot{};
        free_slots.push_back(j);
      }
      if ((e = upload_slots(c, T, newly_done))) return c->cuda_fail(e, "release slots");
      if ((e = mark())) return c->cuda_fail(e, "upload fence");
    }

    // contractions of the completed groups
    if (out.result && np > 0 && !done_jobs.empty()) {
      std::vector<ContractPair> pairs;
      for (int g : done_jobs) {
        std::vector<int> member_slot(jobs[g].sys.size(), -1);
        if (staged)
          member_slot = stage_col[g];
        else
          for (int j = 0; j < N; j++)
            if (slot[j].job == g) member_slot[slot[j].member] = j;
        for (ContractPair p : jobs[g].pairs) {
          p.right = member_slot[p.right];
          p.left = member_slot[p.left];
          pairs.push_back(p);
        }
      }
      if (!pairs.empty()) {
        std::vector<double> part;
        const StageView sv{T->stage_x_e, T->stage_x_o, T->stage_y_e, T->stage_y_o, T->stage_spec_d, S};
        if (int rc = contract_tile(c, T, pairs, out.gamma, *out.plist, part, out.rows, right_pair,
                                   staged ? &sv : nullptr))
          return rc;
        for (const ContractPair& p : pairs)
          for (int q2 = 0; q2 < np * 2; q2++)
            (*out.result)[(size_t)p.out * np * 2 + q2] = part[(size_t)p.out * np * 2 + q2];
      }
    }

    // solution vectors requested by the caller: unpacked straight into the caller's device array
    if (out.x_dev) {
      for (int j = 0; j < N; j++) T->vec_h[j] = -1;
      bool any = false;
      for (int j : harvest) {
        if (slot[j].phase != 0 || std::find(chain_slots.begin(), chain_slots.end(), j) != chain_slots.end())
          continue;
        const QJob& q = jobs[slot[j].job];
        if (q.out_index.empty() || q.out_index[slot[j].member] < 0) continue;
        T->vec_h[j] = q.out_index[slot[j].member];
        any = true;
      }
      if (any) {
        if ((e = upload_vec(c, T))) return c->cuda_fail(e, "upload vector map");
        if ((e = T->enqueue_solution_to_canon(out.x_dev))) return c->cuda_fail(e, "unpack solutions");
        // the map upload must land before the host rewrites vec_h
        if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "unpack solutions");
      }
    } else if (out.x_host) {
      std::vector<std::pair<int, int>> copies;  // slot, output index
      for (int j = 0; j < N; j++) T->vec_h[j] = -1;
      int used = 0;
      for (int j : harvest) {
        if (slot[j].phase != 0 || std::find(chain_slots.begin(), chain_slots.end(), j) != chain_slots.end())
          continue;
        const QJob& q = jobs[slot[j].job];
        if (q.out_index.empty() || q.out_index[slot[j].member] < 0) continue;
        T->vec_h[j] = out.canon_out_base + used;
        copies.push_back({used, q.out_index[slot[j].member]});
        used++;
      }
      if (used) {
        if ((e = upload_vec(c, T))) return c->cuda_fail(e, "upload vector map");
        if ((e = T->enqueue_solution_to_canon(c->canon_d))) return c->cuda_fail(e, "unpack solutions");
        for (auto& cp : copies) {
          e = cudaMemcpyAsync(out.x_host + (size_t)cp.second * vlen,
                              c->canon_d + (size_t)(out.canon_out_base + cp.first) * vlen, vlen * sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream);
          if (e) return c->cuda_fail(e, "download solutions");
        }
        if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "download solutions");
      }
    }

    // release the slots of completed groups (staged: their columns; the slots are free already)
    std::vector<int> released;
    for (int g : done_jobs) {
      if (staged) {
        for (int col : stage_col[g]) stage_free.push_back(col);
        stage_col[g].clear();
        finished++;
        continue;
      }
      for (int j = 0; j < N; j++) {
        if (slot[j].job != g) continue;
        memset(&T->st_h[j], 0, sizeof(SysState));
        memset(&T->spec_h[j], 0, sizeof(NoiseSpec));
        slot[j] = Slot{};
        free_slots.push_back(j);
        released.push_back(j);
      }
      finished++;
    }
    if (!released.empty()) {
      if ((e = upload_slots(c, T, released))) return c->cuda_fail(e, "release slots");
      if ((e = mark())) return c->cuda_fail(e, "upload fence");
    }
    done_jobs.clear();
    newly_done.clear();

    // follow-up solves: the phase-0 solution becomes the right-hand side of the same slot
    if (!chain_slots.empty()) {
      if ((e = wait_fence())) return c->cuda_fail(e, "upload fence");
      for (int j = 0; j < N; j++) T->vec_h[j] = -1;
      for (int j : chain_slots) T->vec_h[j] = out.canon_chain_base + j;
      if ((e = upload_vec(c, T))) return c->cuda_fail(e, "upload vector map");
      if ((e = T->enqueue_solution_to_canon(c->canon_d))) return c->cuda_fail(e, "stage follow-up rhs");
      // the map upload above must land before the host reuses vec_h (same map, re-sent below)
      if ((e = cudaStreamSynchronize(c->stream))) return c->cuda_fail(e, "stage follow-up rhs");
      for (int j : chain_slots) {
        const QJob& q = jobs[slot[j].job];
        const NoiseSpec keep = T->spec_h[j];
        init_state(T->st_h[j], q.chain[slot[j].member], o);
        T->spec_h[j] = keep;
        T->spec_h[j].flags &= ~(uint32_t)NOISE_RHS;  // the noise stays the contraction's left vector
        slot[j].phase = 1;
        slot[j].cg_tried = false;
      }
      if (int rc = admit_rhs(chain_slots, true, false)) return rc;
    }
  }
  return 0;
}

}  // namespace fs
