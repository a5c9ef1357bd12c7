// Engine: context services, the Tile kernel sequences and the batched solve loop.
#define FS_ENGINE_KERNELS 1
#include "fs_engine.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

namespace fs {

static std::atomic<long long> g_launches{0};
static thread_local bool t_capturing = false;  // launches recorded into a graph are counted per replay
void note_launch(int n) {
  if (!t_capturing) g_launches.fetch_add(n, std::memory_order_relaxed);
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

Shape make_shape(int N, int Vh) {
  Shape s;
  s.N = N;
  int NB = N;
  if (N > 32) {
    NB = 1;
    for (int d = 32; d >= 1; d--)
      if (N % d == 0) { NB = d; break; }
  }
  s.NB = NB;
  int SB = (256 / NB) / 8 * 8;
  if (SB < 8) SB = 8;
  s.SB = SB;
  s.nchunk = (Vh + SB - 1) / SB;
  return s;
}

double* pinned_alloc(size_t bytes) {
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) return nullptr;
  return (double*)p;
}

int Ctx::cuda_fail(cudaError_t e, const char* where) {
  err = std::string(where) + ": " + cudaGetErrorString(e);
  return 7;  // FS_ERR_CUDA
}

Launch Ctx::launch_for(const Shape& sh) const {
  Launch l;
  l.grid_y = (sh.N + sh.NB - 1) / sh.NB;
  l.block = sh.SB * sh.NB;
  const int target = std::max(1, (nsm * 8) / l.grid_y);
  l.grid_x = std::min(sh.nchunk, target);
  l.stream = stream;
  return l;
}

void* Ctx::gauge_for(int prec, int nr) {
  if (prec == PREC_F64) return gauge64;
  const int key = (prec == PREC_BF16 ? PREC_F16 : prec) * 100 + nr;
  auto it = gauge_lo.find(key);
  return it == gauge_lo.end() ? nullptr : it->second;
}

int Ctx::ensure_canon(size_t nvec) {
  if (nvec <= canon_cap) return 0;
  if (canon_d) cudaFree(canon_d);
  canon_d = nullptr;
  canon_cap = 0;
  if (cudaMalloc(&canon_d, nvec * (size_t)g.V * 24 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(3, "device allocation of the vector staging buffer failed");
  }
  canon_cap = nvec;
  return 0;
}

int Ctx::ensure_canon_host(size_t nvec) {
  if (nvec <= canon_h_cap) return 0;
  if (canon_h) cudaFreeHost(canon_h);
  canon_h = pinned_alloc(nvec * (size_t)g.V * 24 * sizeof(double));
  canon_h_cap = canon_h ? nvec : 0;
  return canon_h ? 0 : fail(3, "pinned host allocation failed");
}

size_t Ctx::device_bytes() const {
  size_t b = extra_bytes + canon_cap * (size_t)g.V * 24 * sizeof(double);
  for (auto& kv : tiles) b += kv.second->bytes;
  for (auto& l : lanes) b += l->device_bytes();
  return b;
}

Ctx* Ctx::lane(int i) {
  while ((int)lanes.size() <= i) {
    std::unique_ptr<Ctx> l(new Ctx());
    l->device = device;
    l->nsm = nsm;
    l->g = g;
    l->shared = true;
    cudaError_t e = cudaStreamCreateWithFlags(&l->own_stream, cudaStreamNonBlocking);
    if (e) {
      cuda_fail(e, "lane stream");
      return nullptr;
    }
    l->stream = l->own_stream;
    lanes.push_back(std::move(l));
  }
  Ctx* l = lanes[i].get();
  l->iter_bound = iter_bound;
  l->tuned_shape = tuned_shape;
  l->have_gauge = have_gauge;
  l->gauge64 = gauge64;
  l->gauge_lo = gauge_lo;
  l->wline = wline;
  l->wline_mask = wline_mask;
  l->wline_cap = 0;  // never reallocated or freed by the lane
  l->colors_d = colors_d;
  l->colors_own = false;
  l->c_sw = c_sw;
  l->clover64 = clover64;
  l->clover32 = clover32;
  return l;
}

// ---------------------------------------------------------------------------
template <typename Ts>
class Tile : public TileBase {
 public:
  using Tx = typename XOf<Ts>::T;
  Ctx* c = nullptr;
  Shape sh{};
  Launch L{};
  // system-major: a block covers SYS_SITES sites of ONE system (uniform per-block masks). 128-site
  // blocks: 4 resident per SM at 128 registers, finer than 256-site blocks for the few
  // flagged systems of a reliable update (measured 7% faster FP64 hops).
  static constexpr int SYS_SITES = 128;
  Shape sh1{};
  Launch L1{};
  Launch LW{};   // system-major work-list launches: resident blocks sweep (selected system, chunk) items
  // the FP64 hop's work list: three resident 128-site blocks per SM (its launch bounds), since
  // items go to blocks in turn and a block beyond the resident ones would run its share last
  Launch lwh() const {
    Launch l = LW;
    l.grid_x = std::max(1, 3 * c->nsm);
    return l;
  }
  Launch LH{};   // hopping kernels: one site chunk per block, so resident blocks sweep the
                 // lattice in order and neighbour spinors are re-read from L2, not DRAM
  int ngroups = 0;
  double *bhat = nullptr, *r_hi = nullptr, *tmp64 = nullptr;
  void *x_lo = nullptr, *r = nullptr, *rhat = nullptr, *p = nullptr, *v = nullptr, *s = nullptr, *t = nullptr,
       *tmp = nullptr;
  double *pa = nullptr, *pb = nullptr, *pc = nullptr;
  int* gate = nullptr;
  double* fin_slice = nullptr;   // finalize slice sums [MAX_TILE][FIN_SPLIT][FIN_MAXV]
  unsigned* fin_count = nullptr; // finalize arrival tickets [MAX_TILE], zero between finalizes
  double *cg_p = nullptr, *cg_q = nullptr, *cg_g = nullptr, *cg_w = nullptr, *cg_r = nullptr;  // CGNR fallback
  void* cw = nullptr;            // C x of the Wilson-clover operator (inner precision, tile layout)
  std::vector<void*> owned;
  // K BiCGStab iterations captured once and replayed (launch overhead dominates small lattices)
  cudaGraphExec_t gexec = nullptr;
  int gk = 0;
  size_t gnodes = 0;

  ~Tile() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    for (void* q : owned) cudaFree(q);
    if (st_h) cudaFreeHost(st_h);
    if (spec_h) cudaFreeHost(spec_h);
    if (stage_spec_h) cudaFreeHost(stage_spec_h);
    if (vec_h) cudaFreeHost(vec_h);
  }

  void* dalloc(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, n) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    owned.push_back(q);
    bytes += n;
    return q;
  }

  int alloc(Ctx* ctx, int n, int nr_) override {
    c = ctx;
    N = n;
    nr = nr_;
    sh = make_shape(N, c->g.Vh);
    L = c->launch_for(sh);
    sh1 = sh;
    sh1.NB = 1;
    sh1.SB = SYS_SITES;
    sh1.nchunk = (c->g.Vh + SYS_SITES - 1) / SYS_SITES;
    L1.grid_y = N;
    L1.block = SYS_SITES;
    L1.grid_x = std::min(sh1.nchunk, std::max(1, 8 * c->nsm));
    L1.stream = c->stream;
    LW.stream = c->stream;
    LW = L1;
    LW.grid_y = 1;
    LW.grid_x = std::max(1, 4 * c->nsm);  // 4 resident 128-site blocks per SM
    LH = L;
    LH.grid_x = sh.nchunk;
    ngroups = c->g.Vh / 8;
    const size_t f64 = (size_t)24 * c->g.Vh * N * sizeof(double);
    const size_t fts = (size_t)24 * c->g.Vh * N * sizeof(Ts);
    const size_t ftx = (size_t)24 * c->g.Vh * N * sizeof(Tx);
    z_e = (double*)dalloc(f64); z_o = (double*)dalloc(f64); bhat = (double*)dalloc(f64);
    x_hi = (double*)dalloc(f64); x_o = (double*)dalloc(f64); r_hi = (double*)dalloc(f64);
    x_lo = dalloc(ftx);
    r = dalloc(fts); rhat = dalloc(fts); p = dalloc(fts); v = dalloc(fts); s = dalloc(fts); t = dalloc(fts);
    tmp = dalloc(fts);
    tmp64 = std::is_same<Ts, double>::value ? (double*)tmp : (double*)dalloc(f64);
    // pa holds up to 8 values per (system, 8-site group) (the t = M s dots), pb and pc up to 3
    const size_t pbytes = (size_t)N * 3 * ngroups * sizeof(double);
    pa = (double*)dalloc((size_t)N * 8 * ngroups * sizeof(double));
    pb = (double*)dalloc(pbytes); pc = (double*)dalloc(pbytes);
    gate = (int*)dalloc(sizeof(int));
    fin_slice = (double*)dalloc(sizeof(double) * MAX_TILE * FIN_SPLIT * FIN_MAXV);
    fin_count = (unsigned*)dalloc(sizeof(unsigned) * MAX_TILE);
    st_d = (SysState*)dalloc(sizeof(SysState) * MAX_TILE);
    spec_d = (NoiseSpec*)dalloc(sizeof(NoiseSpec) * MAX_TILE);
    vec_d = (int*)dalloc(sizeof(int) * MAX_TILE);
    const void* req[] = {z_e, z_o, bhat, x_hi, x_o, r_hi, x_lo, r, rhat, p, v, s, t, tmp, tmp64,
                         pa, pb, pc, gate, fin_slice, fin_count, st_d, spec_d, vec_d};
    for (const void* q : req)
      if (!q) return 3;
    if (cudaMallocHost(&st_h, sizeof(SysState) * MAX_TILE) != cudaSuccess) return 3;
    if (cudaMallocHost(&spec_h, sizeof(NoiseSpec) * MAX_TILE) != cudaSuccess) return 3;
    if (cudaMallocHost(&vec_h, sizeof(int) * MAX_TILE) != cudaSuccess) return 3;
    memset(st_h, 0, sizeof(SysState) * MAX_TILE);
    cudaMemsetAsync(gate, 0, sizeof(int), c->stream);
    cudaMemsetAsync(fin_count, 0, sizeof(unsigned) * MAX_TILE, c->stream);
    return 0;
  }

  int clover_alloc() override {
    if (cw) return 0;
    cw = dalloc((size_t)24 * c->g.Vh * N * sizeof(Ts));
    return cw ? 0 : 3;
  }
  bool clv() const { return c->c_sw != 0.0; }
  // A clover pass over the systems of `mask`: the tile layout in the storage precision, or the
  // FP64 system-major work list (sysmajor).
  // f32: the FP64 work list in FP32 arithmetic (the FP32-arithmetic reliable updates).
  cudaError_t clover_pass(int mode, void* out, const void* in, const void* Y, int parity, int mask, bool gated,
                          bool sysmajor, bool f32 = false) {
    ClovArgs a{};
    a.out = out; a.in = in; a.Y = Y;
    a.table = ((sysmajor && !f32) || std::is_same<Ts, double>::value) ? (const void*)c->clover64
                                                                      : (const void*)c->clover32;
    a.st = st_d; a.gate = gated ? gate : nullptr;
    a.g = c->g; a.sh = sysmajor ? sh1 : sh; a.parity = parity; a.mask = mask;
    a.sysmajor = sysmajor ? 1 : 0;
    if (sysmajor) return f32 ? launch_clover64_f32(mode, a, LW) : launch_clover<double>(mode, a, LW);
    return launch_clover<Ts>(mode, a, L);
  }

  // Both site factors of a Wilson-clover M-hat in one tile-layout launch over the active systems:
  // out = (A + C_oo)^-1 in (odd sites), out2 = C_ee in2 (even sites).
  cudaError_t clover_pass2(void* out, const void* in, void* out2, const void* in2) {
    ClovArgs a{};
    a.out = out; a.in = in; a.out2 = out2; a.in2 = in2;
    a.table = std::is_same<Ts, double>::value ? (const void*)c->clover64 : (const void*)c->clover32;
    a.st = st_d; a.gate = nullptr;
    a.g = c->g; a.sh = sh; a.parity = 1; a.mask = MASK_ACTIVE;
    return launch_clover<Ts>(CLV_INV_MUL, a, L);
  }

  HopArgs hop(void* out, const void* in, const void* X, const void* Y, const void* R, double* part, int p_out,
              int mask, bool gated, bool hi, bool sysmajor = false) {
    HopArgs a{};
    a.clover = clv() ? 1 : 0;
    a.out = out; a.in = in; a.X = X; a.Y = Y; a.R = R;
    a.gauge = hi ? c->gauge64 : c->gauge_for(prec, nr);
    a.st = st_d; a.partial = part; a.gate = gated ? gate : nullptr; a.work = nullptr;
    a.g = c->g; a.sh = sysmajor ? sh1 : sh; a.p_out = p_out; a.mask = mask;
    a.sysmajor = sysmajor ? 1 : 0;  // one system per block <-> the FP64 fields' system-major layout
    return a;
  }
  BlasArgs blas(int mask, const double* src, double* part, bool gated, bool sysmajor = false) {
    BlasArgs b{};
    b.x_lo = x_lo; b.r = r; b.rhat = rhat; b.p = p; b.v = v; b.s = s; b.t = t;
    b.x_hi = x_hi; b.src = src; b.st = st_d; b.partial = part; b.gate = gated ? gate : nullptr;
    b.Vh = c->g.Vh; b.sh = sysmajor ? sh1 : sh; b.mask = mask;
    b.sysmajor = sysmajor ? 1 : 0;
    return b;
  }
  cudaError_t fin(int op, int mask, const double* a_, const double* b_ = nullptr, const double* c_ = nullptr) {
    FinArgs f{};
    f.st = st_d; f.pa = a_; f.pb = b_; f.pc = c_; f.gate = gate;
    f.slice = fin_slice; f.count = fin_count;
    f.N = N; f.ngroups = ngroups; f.mask = mask;
    f.target = 0.25;  // rms of a scaled residual entry (keeps FP16 away from both range limits)
    f.nreal = 24.0 * c->g.Vh;
    f.max_restarts = 8;
    // (the Wilson-clover updates leave A_oo^-1 H_oe x_e in the scratch, not H_oe x_e)
    f.first_approx = std::is_same<Ts, double>::value ? 0 : 1;
    // tmp64 is a buffer of its own in the mixed precisions (FP64 storage shares it with tmp,
    // which the other systems' iterations overwrite)
    f.hx_kept = std::is_same<Ts, double>::value || clv() ? 0 : 1;
    const dim3 grid(N, FIN_SPLIT);
    switch (fin_values(op)) {
      case 1: fin_kernel<1><<<grid, 256, 0, c->stream>>>(f, op); break;
      case 2: fin_kernel<2><<<grid, 256, 0, c->stream>>>(f, op); break;
      case 3: fin_kernel<3><<<grid, 256, 0, c->stream>>>(f, op); break;
      case 8: fin_kernel<8><<<grid, 256, 0, c->stream>>>(f, op); break;
      default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
  }

  void set_shape(const PkShape& s) override {
    if (s.depth == shape.depth && s.blocks == shape.blocks) return;
    shape = s;
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
    gk = 0;
  }

  // Timed hop launch in the inner precision (the kernel the roofline is about).
  cudaError_t hop_lo(int coef, int dot, const HopArgs& a, int nextra) {
    HopProfile& pf = c->prof;
    LH.stream = c->stream;
    LH.pk_depth = shape.depth;
    LH.pk_blocks = shape.blocks;
    if (!pf.enabled) return launch_hop<Ts>(coef, dot, nr, a, LH);
    cudaEvent_t e0, e1;
    if (!pf.pool.empty()) {
      e0 = pf.pool.back().first; e1 = pf.pool.back().second; pf.pool.pop_back();
    } else {
      cudaEventCreate(&e0); cudaEventCreate(&e1);
    }
    HopArgs b = a;
    b.work = pf.work_d + prec * 3 + nextra;
    cudaEventRecord(e0, c->stream);
    cudaError_t e = launch_hop<Ts>(coef, dot, nr, b, LH);
    cudaEventRecord(e1, c->stream);
    pf.pending.push_back({e0, e1});
    pf.launches += 1;
    // links: every link once per launch (algorithmic), nr reals each
    pf.pending_bytes += (double)c->g.Vh * 8.0 * nr * sizeof(typename GaugeOf<Ts>::T);
    return e;
  }

  // An FP64-arithmetic hop on the system-major work list, timed while profiling is on.
  cudaError_t hop_hi(int coef, int dot, const HopArgs& a, const Launch& l) {
    HopProfile& pf = c->prof;
    if (!pf.enabled) return launch_hop<double>(coef, dot, 18, a, l);
    cudaEvent_t e0, e1;
    if (!pf.pool.empty()) {
      e0 = pf.pool.back().first; e1 = pf.pool.back().second; pf.pool.pop_back();
    } else {
      cudaEventCreate(&e0); cudaEventCreate(&e1);
    }
    HopArgs b = a;
    b.work = pf.work_d + 12;
    cudaEventRecord(e0, l.stream);
    cudaError_t e = launch_hop<double>(coef, dot, 18, b, l);
    cudaEventRecord(e1, l.stream);
    pf.pending64.push_back({e0, e1});
    pf.launches64 += 1;
    return e;
  }

  cudaError_t enqueue_rhs_from_canon(const double* canon) override {
    L.stream = c->stream;
    L1.stream = c->stream;
    LW.stream = c->stream;
    return launch_pack<double>(z_e, z_o, canon, vec_d, c->g, sh1, L1, true);
  }

  cudaError_t enqueue_noise() override {
    L1.stream = c->stream;
    LW.stream = c->stream;
    noise_kernel<<<dim3(std::min(2 * sh1.nchunk, 2 * L1.grid_x), N), SYS_SITES, 0, c->stream>>>(
        z_e, z_o, spec_d, st_d, c->colors_d, c->g, sh1);
    note_launch();
    return cudaGetLastError();
  }

  // Initialisation of the INIT slots; FP64 work on the system-major shape so that
  // refilling a few slots costs only their own systems.
  cudaError_t enqueue_init() override {
    L1.stream = c->stream;
    LW.stream = c->stream;
    cudaError_t e;
    // bhat_e = z_e - D_eo A^-1 z_o, ||bhat||^2 (Wilson-clover: A_oo^-1 z_o by a clover pass first)
    const double* zin = z_o;
    if (clv()) {
      if ((e = clover_pass(CLV_INV, tmp64, z_o, nullptr, 1, MASK_INIT, false, true))) return e;
      zin = tmp64;
    }
    if ((e = hop_hi(COEF_PREP, DOT_NORM, hop(bhat, zin, z_e, nullptr, nullptr, pa, 0, MASK_INIT, false, true, true),
                    lwh()))) return e;
    if ((e = launch_blas<Ts>(OP_NORM64, blas(MASK_INIT, z_e, pb, false, true), LW))) return e;
    if ((e = launch_blas<Ts>(OP_NORM64, blas(MASK_INIT, z_o, pc, false, true), LW))) return e;
    if ((e = launch_blas<Ts>(OP_ZEROX, blas(MASK_INIT, nullptr, nullptr, false, true), LW))) return e;
    if ((e = fin(FIN_NORM, MASK_INIT, pa, pb, pc))) return e;
    if ((e = launch_blas<Ts>(OP_SETR, blas(MASK_INIT, bhat, pa, false, true), LW))) return e;
    return fin(FIN_INIT, MASK_INIT, pa);
  }

  cudaError_t enqueue_iter() override {
    L.stream = c->stream;
    cudaError_t e;
    const bool cl = clv();
    // p was set by the previous iteration's OP_XRP, or by OP_SETR at a (re)start
    if ((e = hop_lo(COEF_PLAIN, DOT_NONE, hop(tmp, p, nullptr, nullptr, nullptr, nullptr, 1, MASK_ACTIVE, false,
                                              false), 0))) return e;
    // Wilson-clover: M-hat p = (A + C_ee) p - H_eo (A + C_oo)^-1 H_oe p / 4, the site factors by passes
    if (cl && (e = clover_pass2(tmp, tmp, cw, p))) return e;
    if ((e = hop_lo(COEF_MHAT, DOT_R, hop(v, tmp, p, cl ? cw : nullptr, rhat, pa, 0, MASK_ACTIVE, false, false), 2)))
      return e;
    if ((e = fin(FIN_ALPHA, MASK_ACTIVE, pa))) return e;
    if ((e = launch_blas<Ts>(OP_S, blas(MASK_ACTIVE, nullptr, nullptr, false), L))) return e;
    if ((e = hop_lo(COEF_PLAIN, DOT_NONE, hop(tmp, s, nullptr, nullptr, nullptr, nullptr, 1, MASK_ACTIVE, false,
                                              false), 0))) return e;
    if (cl && (e = clover_pass2(tmp, tmp, cw, s))) return e;
    if ((e = hop_lo(COEF_MHAT, DOT_TS, hop(t, tmp, s, cl ? cw : nullptr, rhat, pa, 0, MASK_ACTIVE, false, false), 2)))
      return e;
    if ((e = fin(FIN_OMEGA, MASK_ACTIVE, pa))) return e;
    if ((e = launch_blas<Ts>(OP_XRP, blas(MASK_ACTIVE, nullptr, nullptr, false), L))) return e;
    // Reliable update of the systems flagged by FIN_OMEGA, in FP64. These kernels use the
    // system-major shape: a block serves one system, so unflagged systems cost one flag
    // read per block instead of occupying FP64 issue slots inside mixed warps.
    L1.stream = c->stream;
    LW.stream = c->stream;
    // Mixed precision: FP32 arithmetic (FP32 links, FP64 fields, the FP32 pipe) where it meets
    // the update's need, FP64 where the residual decides convergence.
    //  - update 0 restarts from a residual of about delta ||b||: r = bhat - M x_hi in FP32
    //    arithmetic errs by about eps32 A ||x||, a small fraction of it;
    //  - odd updates: the full residual in FP64 (and only these end a solve);
    //  - even updates k >= 2: r = r_prev - M dx, dx = x_lo / scale the iterate's change since the
    //    previous (FP64) update, held in x_o (free until the odd sites are reconstructed); the
    //    FP32 error is about eps32 A ||dx||, relative to the small dx instead of x.
    // The FP64 storage mode keeps FP64 throughout.
    constexpr bool mixed = !std::is_same<Ts, double>::value;
    if ((e = launch_blas<Ts>(OP_ACCX, blas(MASK_UPDATE, mixed ? x_o : nullptr, nullptr, true, true), LW))) return e;
    if (cl) {
      // Wilson-clover: r = bhat - C_ee x - A x + H_eo A_oo^-1 H_oe x / 4, the clover parts by passes, in the
      // same three forms as below (x_o holds bhat - C_ee x for a full residual, dx for a correction,
      // whose r_prev - C_ee dx is formed in place)
      int lat = MASK_UPDATE;
      if constexpr (mixed) {
        lat = MASK_UPDATE_LATER;
        void* g32 = c->gauge_for(PREC_F32, 18);
        HopArgs h1 = hop(tmp64, x_hi, nullptr, nullptr, nullptr, nullptr, 1, MASK_UPDATE_FIRST, true, true, true);
        HopArgs h2 = hop(r_hi, tmp64, x_hi, x_o, nullptr, pa, 0, MASK_UPDATE_FIRST, true, true, true);
        HopArgs h3 = hop(tmp64, x_o, nullptr, nullptr, nullptr, nullptr, 1, MASK_UPDATE_CORR, true, true, true);
        HopArgs h4 = hop(r_hi, tmp64, x_o, r_hi, nullptr, pa, 0, MASK_UPDATE_CORR, true, true, true);
        h1.gauge = h2.gauge = h3.gauge = h4.gauge = g32;
        if ((e = launch_hop64_f32(COEF_PLAIN, DOT_NONE, h1, lwh()))) return e;
        if ((e = clover_pass(CLV_INV, tmp64, tmp64, nullptr, 1, MASK_UPDATE_FIRST, true, true, true))) return e;
        if ((e = clover_pass(CLV_SUB, x_o, x_hi, bhat, 0, MASK_UPDATE_FIRST, true, true, true))) return e;
        if ((e = launch_hop64_f32(COEF_TRUERES, DOT_NORM, h2, lwh()))) return e;
        if ((e = launch_hop64_f32(COEF_PLAIN, DOT_NONE, h3, lwh()))) return e;
        if ((e = clover_pass(CLV_INV, tmp64, tmp64, nullptr, 1, MASK_UPDATE_CORR, true, true, true))) return e;
        if ((e = clover_pass(CLV_SUB, r_hi, x_o, r_hi, 0, MASK_UPDATE_CORR, true, true, true))) return e;
        if ((e = launch_hop64_f32(COEF_TRUERES, DOT_NORM, h4, lwh()))) return e;
      }
      if ((e = hop_hi(COEF_PLAIN, DOT_NONE,
                      hop(tmp64, x_hi, nullptr, nullptr, nullptr, nullptr, 1, lat, true, true, true), lwh())))
        return e;
      if ((e = clover_pass(CLV_INV, tmp64, tmp64, nullptr, 1, lat, true, true))) return e;
      if ((e = clover_pass(CLV_SUB, x_o, x_hi, bhat, 0, lat, true, true))) return e;
      if ((e = hop_hi(COEF_TRUERES, DOT_NORM, hop(r_hi, tmp64, x_hi, x_o, nullptr, pa, 0, lat, true, true, true),
                      lwh())))
        return e;
      if ((e = fin(FIN_TRUE, MASK_UPDATE, pa))) return e;
      if ((e = launch_blas<Ts>(OP_SETR, blas(MASK_UPDATE, r_hi, pa, true, true), LW))) return e;
      return fin(FIN_UPDATE, MASK_UPDATE, pa);
    }
    int later = MASK_UPDATE;
    if constexpr (mixed) {
      later = MASK_UPDATE_LATER;
      void* g32 = c->gauge_for(PREC_F32, 18);
      HopArgs h1 = hop(tmp64, x_hi, nullptr, nullptr, nullptr, nullptr, 1, MASK_UPDATE_FIRST, true, true, true);
      HopArgs h2 = hop(r_hi, tmp64, x_hi, bhat, nullptr, pa, 0, MASK_UPDATE_FIRST, true, true, true);
      HopArgs h3 = hop(tmp64, x_o, nullptr, nullptr, nullptr, nullptr, 1, MASK_UPDATE_CORR, true, true, true);
      HopArgs h4 = hop(r_hi, tmp64, x_o, r_hi, nullptr, pa, 0, MASK_UPDATE_CORR, true, true, true);
      h1.gauge = h2.gauge = h3.gauge = h4.gauge = g32;
      if ((e = launch_hop64_f32(COEF_PLAIN, DOT_NONE, h1, lwh()))) return e;
      if ((e = launch_hop64_f32(COEF_TRUERES, DOT_NORM, h2, lwh()))) return e;
      if ((e = launch_hop64_f32(COEF_PLAIN, DOT_NONE, h3, lwh()))) return e;
      if ((e = launch_hop64_f32(COEF_TRUERES, DOT_NORM, h4, lwh()))) return e;
    }
    if ((e = hop_hi(COEF_PLAIN, DOT_NONE,
                    hop(tmp64, x_hi, nullptr, nullptr, nullptr, nullptr, 1, later, true, true, true), lwh())))
      return e;
    if ((e = hop_hi(COEF_TRUERES, DOT_NORM, hop(r_hi, tmp64, x_hi, bhat, nullptr, pa, 0, later, true, true, true),
                    lwh())))
      return e;
    if ((e = fin(FIN_TRUE, MASK_UPDATE, pa))) return e;
    if ((e = launch_blas<Ts>(OP_SETR, blas(MASK_UPDATE, r_hi, pa, true, true), LW))) return e;
    return fin(FIN_UPDATE, MASK_UPDATE, pa);
  }

  cudaError_t enqueue_iters(int k) override {
    const bool graphs = !c->prof.enabled && c->stream != nullptr && c->stream != cudaStreamLegacy &&
                        c->stream != cudaStreamPerThread;
    cudaError_t e = cudaSuccess;
    if (!graphs || iters_eager < 1) {
      // eager launches (always the first time, so every one-time kernel set-up is done)
      for (int i = 0; i < k && !e; i++) e = enqueue_iter();
      iters_eager++;
      return e;
    }
    if (!gexec || gk != k || gclv != (int)clv()) {
      if (gexec) cudaGraphExecDestroy(gexec);
      gexec = nullptr;
      cudaGraph_t graph = nullptr;
      t_capturing = true;
      e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
      for (int i = 0; i < k && !e; i++) e = enqueue_iter();
      cudaError_t e2 = cudaStreamEndCapture(c->stream, &graph);
      t_capturing = false;
      if (!e) e = e2;
      if (!e) e = cudaGraphGetNodes(graph, nullptr, &gnodes);
      if (!e) e = cudaGraphInstantiate(&gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e) return e;
      gk = k;
      gclv = (int)clv();
    }
    note_launch((int)gnodes);
    return cudaGraphLaunch(gexec, c->stream);
  }
  int iters_eager = 0;
  int gclv = -1;  // the clover term's state when the graph was captured

  cudaError_t enqueue_recon() override {
    L1.stream = c->stream;
    LW.stream = c->stream;
    // x_o = A^-1 (z_o - D_oe x_e): from the H_oe x_e that the final FP64 residual left in tmp64 where
    // it is still there (a vector operation), else by an FP64 hop
    cudaError_t e;
    if (clv()) {
      // x_o = (A + C_oo)^-1 (z_o + H_oe x_e / 2)
      if ((e = hop_hi(COEF_RECON, DOT_NONE,
                      hop(x_o, x_hi, z_o, nullptr, nullptr, nullptr, 1, MASK_HARVEST, false, true, true), lwh())))
        return e;
      return clover_pass(CLV_INV, x_o, x_o, nullptr, 1, MASK_HARVEST, false, true);
    }
    BlasArgs b = blas(MASK_HARVEST_HX, tmp64, nullptr, false, true);
    b.x_hi = x_o;
    b.src2 = z_o;
    if ((e = launch_blas<Ts>(OP_RECON, b, LW))) return e;
    return hop_hi(COEF_RECON, DOT_NONE,
                  hop(x_o, x_hi, z_o, nullptr, nullptr, nullptr, 1, MASK_HARVEST_HOP, false, true, true), lwh());
  }

  cudaError_t enqueue_verify() override {
    L1.stream = c->stream;
    LW.stream = c->stream;
    cudaError_t e;
    // r = z - (D + sigma) x on both parities; Wilson-clover: z - C x first, by a pass
    const double *ye = z_e, *yo = z_o;
    if (clv()) {
      if ((e = clover_pass(CLV_SUB, r_hi, x_hi, z_e, 0, MASK_HARVEST, false, true))) return e;
      if ((e = clover_pass(CLV_SUB, tmp64, x_o, z_o, 1, MASK_HARVEST, false, true))) return e;
      ye = r_hi;
      yo = tmp64;
    }
    if ((e = hop_hi(COEF_FULLRES, DOT_NORM, hop(r_hi, x_o, x_hi, ye, nullptr, pa, 0, MASK_HARVEST, false, true, true),
                    lwh())))
      return e;
    if ((e = hop_hi(COEF_FULLRES, DOT_NORM, hop(tmp64, x_hi, x_o, yo, nullptr, pb, 1, MASK_HARVEST, false, true, true),
                    lwh())))
      return e;
    return fin(FIN_VERIFY, MASK_HARVEST, pa, pb);
  }

  double* field_pair(int id, int parity) override {
    if (id == PAIR_X) return parity ? x_o : x_hi;
    if (id == PAIR_Z) return parity ? z_o : z_e;
    return parity ? tmp64 : r_hi;
  }

  int stage_alloc(int S, bool with_y) override {
    if (S <= stage_cols && (!with_y || stage_y_e)) return 0;
    const int cols = std::max(S, stage_cols);
    const size_t col = (size_t)24 * c->g.Vh * sizeof(double);
    double* xe = (double*)dalloc(col * cols);
    double* xo = (double*)dalloc(col * cols);
    double* ye = (with_y || stage_y_e) ? (double*)dalloc(col * cols) : nullptr;
    double* yo = (with_y || stage_y_e) ? (double*)dalloc(col * cols) : nullptr;
    NoiseSpec* sd = (NoiseSpec*)dalloc(sizeof(NoiseSpec) * cols);
    NoiseSpec* sh_ = nullptr;
    if (cudaMallocHost(&sh_, sizeof(NoiseSpec) * cols) != cudaSuccess) sh_ = nullptr;
    if (!xe || !xo || !sd || !sh_ || ((with_y || stage_y_e) && (!ye || !yo))) {
      if (sh_) cudaFreeHost(sh_);
      return 3;  // the partial allocations stay owned by the tile and are freed with it
    }
    if (stage_spec_h) cudaFreeHost(stage_spec_h);
    stage_x_e = xe; stage_x_o = xo; stage_y_e = ye; stage_y_o = yo;
    stage_spec_d = sd; stage_spec_h = sh_;
    memset(stage_spec_h, 0, sizeof(NoiseSpec) * cols);
    stage_cols = cols;
    return 0;
  }

  cudaError_t enqueue_kappa_hop(int from, int to) override {
    L1.stream = c->stream;
    LW.stream = c->stream;
    // even <- kappa H_eo (odd), odd <- kappa H_oe (even); FP64 work list over the FLAG_HPE slots
    // (Wilson-clover: H / 2, then A(x)^-1 in place)
    cudaError_t e = launch_hop<double>(COEF_KAPPA, DOT_NONE, 18,
                                       hop(field_pair(to, 0), field_pair(from, 1), nullptr, nullptr, nullptr, nullptr,
                                           0, MASK_HPE, false, true, true), lwh());
    if (e) return e;
    if ((e = launch_hop<double>(COEF_KAPPA, DOT_NONE, 18,
                                hop(field_pair(to, 1), field_pair(from, 0), nullptr, nullptr, nullptr, nullptr, 1,
                                    MASK_HPE, false, true, true), lwh())))
      return e;
    return clv() ? enqueue_site_inverse(to, to) : cudaSuccess;
  }

  cudaError_t enqueue_site_inverse(int from, int to) override {
    if (!clv()) return cudaErrorInvalidValue;
    L1.stream = c->stream;
    LW.stream = c->stream;
    cudaError_t e = clover_pass(CLV_INV, field_pair(to, 0), field_pair(from, 0), nullptr, 0, MASK_HPE, false, true);
    if (e) return e;
    return clover_pass(CLV_INV, field_pair(to, 1), field_pair(from, 1), nullptr, 1, MASK_HPE, false, true);
  }

  cudaError_t enqueue_dslash(double* canon) override {
    L.stream = c->stream;
    // in: canon[vec[j]] -> (p, tmp) ; out = (D + sigma) in -> (v, s) -> canon[vec[j]]
    cudaError_t e;
    if ((e = launch_pack<Ts>(p, tmp, canon, vec_d, c->g, sh, L, false))) return e;
    const bool f64 = std::is_same<Ts, double>::value;
    const bool cl = clv();
    // Wilson-clover: C x of each parity by a pass, added through Y (the field cw)
    HopArgs he = hop(v, tmp, p, cl ? cw : nullptr, nullptr, nullptr, 0, MASK_INIT, false, f64);
    HopArgs ho = hop(s, p, tmp, cl ? cw : nullptr, nullptr, nullptr, 1, MASK_INIT, false, f64);
    if (cl && (e = clover_pass(CLV_MUL, cw, p, nullptr, 0, MASK_INIT, false, false))) return e;
    if ((e = hop_lo(COEF_DSLASH, DOT_NONE, he, 1))) return e;
    if (cl && (e = clover_pass(CLV_MUL, cw, tmp, nullptr, 1, MASK_INIT, false, false))) return e;
    if ((e = hop_lo(COEF_DSLASH, DOT_NONE, ho, 1))) return e;
    return launch_unpack<Ts>(canon, v, s, vec_d, c->g, sh, L, false);
  }

  // ---- CGNR fallback on M^dag M, FP64, system-major (only the FLAG_CG slots work) ----
  int cg_alloc() override {
    if (cg_p) return 0;
    const size_t f64 = (size_t)24 * c->g.Vh * N * sizeof(double);
    cg_p = (double*)dalloc(f64); cg_q = (double*)dalloc(f64); cg_g = (double*)dalloc(f64);
    cg_w = (double*)dalloc(f64); cg_r = (double*)dalloc(f64);
    return (cg_p && cg_q && cg_g && cg_w && cg_r) ? 0 : 3;
  }
  CgArgs cga(int mask, double* part) {
    CgArgs a{};
    a.x = x_hi; a.s = r_hi; a.p = cg_p; a.q = cg_q; a.g = cg_g; a.w = cg_w; a.r = cg_r;
    a.st = st_d; a.partial = part; a.Vh = c->g.Vh; a.sh = sh1; a.mask = mask;
    return a;
  }
  template <int OP>
  cudaError_t cg_op(int mask, double* part = nullptr) {
    cg_kernel<OP><<<dim3(LW.grid_x, 1), SYS_SITES, 0, c->stream>>>(cga(mask, part));
    note_launch();
    return cudaGetLastError();
  }
  // out = M-hat in on the FP64 work list over mask, ||out||^2 -> part when part != nullptr. The
  // Wilson-clover M-hat takes its clover passes, with C_ee in in x_o (free until the reconstruction).
  cudaError_t mhat64(double* out, const double* in, int mask, double* part) {
    cudaError_t e;
    if ((e = launch_hop<double>(COEF_PLAIN, DOT_NONE, 18,
                                hop(tmp64, in, nullptr, nullptr, nullptr, nullptr, 1, mask, false, true, true), lwh())))
      return e;
    const bool cl = clv();
    if (cl && ((e = clover_pass(CLV_INV, tmp64, tmp64, nullptr, 1, mask, false, true)) ||
               (e = clover_pass(CLV_MUL, x_o, in, nullptr, 0, mask, false, true))))
      return e;
    return launch_hop<double>(COEF_MHAT, part ? DOT_NORM : DOT_NONE, 18,
                              hop(out, tmp64, in, cl ? x_o : nullptr, nullptr, part, 0, mask, false, true, true), lwh());
  }
  // r = M^dag s = gamma5 M gamma5 s, ||r||^2 -> part
  cudaError_t cg_normal_residual(int mask, double* part) {
    cudaError_t e;
    if ((e = cg_op<CG_G5>(mask))) return e;
    if ((e = mhat64(cg_w, cg_g, mask, nullptr))) return e;
    return cg_op<CG_R>(mask, part);
  }
  // s = bhat - M x (into r_hi), ||s||^2 -> part
  cudaError_t cg_true_residual(int mask, double* part) {
    cudaError_t e;
    if ((e = launch_hop<double>(COEF_PLAIN, DOT_NONE, 18,
                                hop(tmp64, x_hi, nullptr, nullptr, nullptr, nullptr, 1, mask, false, true, true), lwh())))
      return e;
    const double* y = bhat;
    if (clv()) {  // bhat - C_ee x - A x + H_eo A_oo^-1 H_oe x / 4
      if ((e = clover_pass(CLV_INV, tmp64, tmp64, nullptr, 1, mask, false, true))) return e;
      if ((e = clover_pass(CLV_SUB, x_o, x_hi, bhat, 0, mask, false, true))) return e;
      y = x_o;
    }
    return launch_hop<double>(COEF_TRUERES, DOT_NORM, 18,
                              hop(r_hi, tmp64, x_hi, y, nullptr, part, 0, mask, false, true, true), lwh());
  }
  cudaError_t enqueue_cg_init() override {
    L1.stream = c->stream;
    LW.stream = c->stream;
    cudaError_t e;
    if ((e = cg_true_residual(MASK_CG, pa))) return e;
    if ((e = cg_normal_residual(MASK_CG, pb))) return e;
    if ((e = fin(FIN_CG_INIT, MASK_CG, pa, pb))) return e;
    return cg_op<CG_P0>(MASK_CG);
  }
  cudaError_t enqueue_cg_iter() override {
    L1.stream = c->stream;
    LW.stream = c->stream;
    cudaError_t e;
    // q = M p, alpha = <r, r> / ||q||^2
    if ((e = mhat64(cg_q, cg_p, MASK_CG, pa))) return e;
    if ((e = fin(FIN_CG_ALPHA, MASK_CG, pa))) return e;
    if ((e = cg_op<CG_XS>(MASK_CG, pa))) return e;   // x += alpha p, s -= alpha q
    if ((e = cg_normal_residual(MASK_CG, pb))) return e;
    if ((e = fin(FIN_CG_BETA, MASK_CG, pa, pb))) return e;
    // true residual of the systems due a check (every 64 iterations, apparent convergence, the last)
    if ((e = cg_true_residual(MASK_CG_CHECK, pc))) return e;
    if ((e = fin(FIN_CG_TRUE, MASK_CG_CHECK, pc))) return e;
    return cg_op<CG_P>(MASK_CG);
  }

  cudaError_t enqueue_solution_to_canon(double* canon) override {
    L.stream = c->stream;
    L1.stream = c->stream;
    LW.stream = c->stream;
    return launch_unpack<double>(canon, x_hi, x_o, vec_d, c->g, sh1, L1, true);
  }
};

TileBase* Ctx::tile(int prec, int N, int nr) {
  const long long key = ((long long)prec * 1000 + N) * 100 + nr;
  auto it = tiles.find(key);
  if (it != tiles.end()) {
    if (c_sw != 0.0 && it->second->clover_alloc() != 0) {
      fail(3, "device allocation of the clover field failed");
      return nullptr;
    }
    return it->second.get();
  }
  std::unique_ptr<TileBase> t;
  switch (prec) {
    case PREC_F64: t.reset(new Tile<double>()); break;
    case PREC_F32: t.reset(new Tile<float>()); break;
    case PREC_F16: t.reset(new Tile<__half>()); break;
    case PREC_BF16: t.reset(new Tile<__nv_bfloat16>()); break;
    default: return nullptr;
  }
  t->prec = prec;
  if (t->alloc(this, N, nr) != 0) {
    // release other cached tiles and retry once
    tiles.clear();
    switch (prec) {
      case PREC_F64: t.reset(new Tile<double>()); break;
      case PREC_F32: t.reset(new Tile<float>()); break;
      case PREC_F16: t.reset(new Tile<__half>()); break;
      default: t.reset(new Tile<__nv_bfloat16>()); break;
    }
    t->prec = prec;
    if (t->alloc(this, N, nr) != 0) return nullptr;
  }
  TileBase* raw = t.get();
  if (c_sw != 0.0 && raw->clover_alloc() != 0) {
    fail(3, "device allocation of the clover field failed");
    return nullptr;
  }
  auto sh = tuned_shape.find((long long)(prec * 100 + nr) * 1000 + N);
  if (sh != tuned_shape.end()) raw->set_shape(sh->second);
  tiles[key] = std::move(t);
  return raw;
}

int ensure_wline(Ctx* c, int pmask, int pmax) {
  const int wmask = pmask & ~1;
  if (!wmask || c->wline_mask == wmask) return 0;
  if (c->shared) return c->fail(1, "contraction paths of a lane must be built by its owner");
  cudaError_t e;
  // the path products depend on the gauge field and the displacements only: built once
  const size_t need_w = (size_t)__builtin_popcount(wmask) * 18 * 2 * c->g.Vh * sizeof(double);
  if (need_w > c->wline_cap) {
    if (c->wline) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->wline);
      c->extra_bytes -= c->wline_cap;
      c->wline = nullptr;
      c->wline_cap = 0;
    }
    if ((e = cudaMalloc((void**)&c->wline, need_w))) return c->cuda_fail(e, "contraction path products");
    c->wline_cap = need_w;
    c->extra_bytes += need_w;
  }
  transport_kernel<<<(2 * c->g.Vh + 255) / 256, 256, 0, c->stream>>>(c->wline, (const double*)c->gauge64, c->g,
                                                                    wmask, pmax);
  note_launch();
  if ((e = cudaGetLastError())) return c->cuda_fail(e, "contraction path products");
  c->wline_mask = wmask;
  return 0;
}

int upload_colors(Ctx* c, const int* colors) {
  if (c->shared) return c->fail(1, "the probing colours of a lane are set by its owner");
  cudaError_t e;
  if (!c->colors_d) {
    if ((e = cudaMalloc((void**)&c->colors_d, (size_t)c->g.V * sizeof(int)))) {
      c->colors_d = nullptr;
      return c->cuda_fail(e, "probing colours");
    }
    c->colors_own = true;
    c->extra_bytes += (size_t)c->g.V * sizeof(int);
  }
  if ((e = cudaMemcpyAsync(c->colors_d, colors, (size_t)c->g.V * sizeof(int), cudaMemcpyHostToDevice, c->stream)))
    return c->cuda_fail(e, "probing colours");
  return 0;
}

int contract_tile(Ctx* c, TileBase* T, const std::vector<ContractPair>& pairs, const double* gamma,
                  const std::vector<int>& plist, std::vector<double>& result, int rows, int right_pair,
                  const StageView* sv) {
  const int np = (int)plist.size();
  const int npairs = (int)pairs.size();
  if (npairs == 0) return 0;
  if (np <= 0 || np > CONTRACT_MAXP) return c->fail(1, "between 1 and 16 displacements are supported");
  ContractArgs a{};
  int pmask = 0, pmax = 0;
  for (int q : plist) {
    if (q < 0 || q > 30) return c->fail(1, "displacement p must be in [0, 30]");
    if (pmask & (1 << q)) return c->fail(1, "displacements must be distinct");
    pmask |= 1 << q;
    pmax = std::max(pmax, q);
  }
  // results come back in increasing p; callers pass plist sorted
  for (int k = 1; k < np; k++)
    if (plist[k] <= plist[k - 1]) return c->fail(1, "displacements must be increasing");
  cudaError_t e;
  if (int rc = ensure_wline(c, pmask, pmax)) return rc;
  a.x_e = T->x_hi; a.x_o = T->x_o; a.wline = c->wline; a.spec = T->spec_d; a.colors = c->colors_d;
  a.y_e = T->field_pair(right_pair, 0);
  a.y_o = T->field_pair(right_pair, 1);
  a.N = T->N;
  if (sv) {  // staged vectors: system-major columns addressed like the tile's FP64 fields
    a.x_e = sv->x_e; a.x_o = sv->x_o; a.y_e = sv->y_e; a.y_o = sv->y_o; a.spec = sv->spec; a.N = sv->N;
  }
  for (int k = 0; k < 32; k++) a.gamma[k] = gamma[k];
  // detect a monomial Gamma (one entry per row, each +-1 or +-i): applied as a permutation
  a.gmono = 1;
  for (int r = 0; r < 4 && a.gmono; r++) {
    int found = -1;
    for (int t = 0; t < 4; t++) {
      const double re = gamma[(r * 4 + t) * 2], im = gamma[(r * 4 + t) * 2 + 1];
      if (re == 0.0 && im == 0.0) continue;
      if (found >= 0) { a.gmono = 0; break; }
      found = t;
      if (re == 1.0 && im == 0.0) a.gphase[r] = 0;
      else if (re == 0.0 && im == 1.0) a.gphase[r] = 1;
      else if (re == -1.0 && im == 0.0) a.gphase[r] = 2;
      else if (re == 0.0 && im == -1.0) a.gphase[r] = 3;
      else a.gmono = 0;
    }
    if (found < 0) a.gmono = 0;
    a.gperm[r] = found;
  }
  a.g = c->g; a.pmask = pmask; a.pmax = pmax; a.np = np;
  a.nblk = (2 * c->g.Vh + 255) / 256;
  const size_t part_n = (size_t)npairs * np * 2 * a.nblk;
  const size_t res_n = (size_t)rows * np * 2;
  const size_t need = part_n * sizeof(double) + res_n * sizeof(double) + npairs * sizeof(ContractPair) + 256;
  char* buf = nullptr;
  if ((e = cudaMallocAsync((void**)&buf, need, c->stream))) return c->cuda_fail(e, "contraction buffers");
  double* part = (double*)buf;
  double* res = part + part_n;
  ContractPair* pr = (ContractPair*)(res + res_n);
  a.partial = part;
  a.pairs = pr;
  e = cudaMemcpyAsync(pr, pairs.data(), npairs * sizeof(ContractPair), cudaMemcpyHostToDevice, c->stream);
  if (!e) e = cudaMemsetAsync(res, 0, res_n * sizeof(double), c->stream);
  if (!e) {
    contract_kernel<<<dim3(a.nblk, npairs), 256, 0, c->stream>>>(a);
    note_launch();
    e = cudaGetLastError();
  }
  if (!e) {
    contract_finalize<<<npairs * np, 256, 0, c->stream>>>(part, pr, res, np, a.nblk);
    note_launch();
    e = cudaGetLastError();
  }
  result.assign(res_n, 0.0);
  if (!e) e = cudaMemcpyAsync(result.data(), res, res_n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaFreeAsync(buf, c->stream);
  if (!e) e = cudaStreamSynchronize(c->stream);
  if (e) return c->cuda_fail(e, "contraction");
  return 0;
}

// entry points used by the API translation unit
cudaError_t launch_noise_codes(uint8_t* codes, NoiseSpec n, int V, cudaStream_t s) {
  noise_codes_kernel<<<(V + 255) / 256, 256, 0, s>>>(codes, n, V);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fs
