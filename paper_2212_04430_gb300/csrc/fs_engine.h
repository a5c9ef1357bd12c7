// Host-side engine: the context (device, geometry, gauge copies, stream, buffers)
// and the Tile, a batch of up to 64 shifted systems solved together by
// even-odd preconditioned BiCGStab with per-system convergence masks and
// mixed-precision reliable updates.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <string>
#include <vector>

#include "fs_aux.cuh"
#include "fs_blas.cuh"
#include "fs_clover.cuh"
#include "fs_hop.cuh"

namespace fs {

constexpr int MAX_TILE = 64;

// ---- kernel launchers (one translation unit per storage precision) ----
template <typename Ts> struct GaugeOf { using T = Ts; };
template <> struct GaugeOf<__nv_bfloat16> { using T = __half; };
template <typename Ts> struct XOf { using T = float; };
template <> struct XOf<double> { using T = double; };

struct Launch {
  int grid_x;
  int grid_y;
  int block;
  cudaStream_t stream;
  int pk_depth = 0;   // persistent FP16/BF16/FP32 hop: ring depth (0: the default of its storage)
  int pk_blocks = 0;  // its resident blocks per SM (0: as many as fit)
};

// Launch shape of the persistent hop picked by the autotuner for a (precision, link format, tile).
struct PkShape {
  int depth = 0, blocks = 0;
};

template <typename Ts> cudaError_t launch_hop(int coef, int dot, int nr, const HopArgs& a, const Launch& l);
// FP64 fields, FP32 links (18 reals) and FP32 arithmetic, system-major work list: the true residual
// of a system's first reliable update (fs_kern_f32.cu); COEF_PLAIN / DOT_NONE and COEF_TRUERES /
// DOT_NORM only.
cudaError_t launch_hop64_f32(int coef, int dot, const HopArgs& a, const Launch& l);
// The clover passes of those updates: FP64 fields, the FP32 table and FP32 arithmetic, system-major
// work list (fs_kern_f32.cu); CLV_SUB and CLV_INV only.
cudaError_t launch_clover64_f32(int mode, const ClovArgs& a, const Launch& l);
template <typename Ts> cudaError_t launch_blas(int op, const BlasArgs& a, const Launch& l);
// Clover passes (fs_clover.cuh): tile layout in the storage precision (FP32 table and arithmetic
// for the inner precisions), or the FP64 system-major work list when a.sysmajor (Ts = double).
template <typename Ts> cudaError_t launch_clover(int mode, const ClovArgs& a, const Launch& l);
template <typename Ts> cudaError_t launch_pack(void* fe, void* fo, const double* canon, const int* vec,
                                               const Geom& g, const Shape& sh, const Launch& l, bool sysmajor);
template <typename Ts> cudaError_t launch_unpack(double* canon, const void* fe, const void* fo, const int* vec,
                                                 const Geom& g, const Shape& sh, const Launch& l, bool sysmajor);
template <typename Tg> cudaError_t launch_gauge_pack(void* out, const double* canon, const Geom& g, int nr,
                                                     cudaStream_t s);

Shape make_shape(int N, int Vh);

struct Ctx;

// Profiling of the hopping kernel launches (CUDA events on the context stream).
struct HopProfile {
  bool enabled = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  long long launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
  double pending_bytes = 0.0;
  unsigned long long* work_d = nullptr;  // (site, system) pairs per [precision][extra fields read], then
                                         // [12] those of the FP64-arithmetic work-list hops
  // the FP64-arithmetic work-list hops (preparation, reliable-update residuals, reconstruction,
  // verification), timed separately: they run on the FP64 pipe
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending64;
  long long launches64 = 0;
  double ms64 = 0.0;
};
constexpr int PROF_SLOTS = 13;

class TileBase {
 public:
  virtual ~TileBase() {}
  // the persistent hop's launch shape; a change drops the captured iteration graph
  virtual void set_shape(const PkShape& s) = 0;
  PkShape shape;
  int N = 0;
  int nr = 18;
  int prec = 0;
  size_t bytes = 0;
  SysState* st_d = nullptr;
  SysState* st_h = nullptr;  // pinned mirror
  NoiseSpec* spec_d = nullptr;
  NoiseSpec* spec_h = nullptr;
  int* vec_d = nullptr;      // slot -> canonical vector index (pack / unpack)
  int* vec_h = nullptr;
  double* z_e = nullptr;     // full right-hand side (FP64)
  double* z_o = nullptr;
  double* x_hi = nullptr;    // solution, even sites (FP64)
  double* x_o = nullptr;     // solution, odd sites (FP64, after reconstruction)
  virtual int alloc(Ctx* c, int N, int nr) = 0;
  // the field that holds C x for the Wilson-clover operator, allocated when the clover term is on
  virtual int clover_alloc() = 0;
  virtual cudaError_t enqueue_rhs_from_canon(const double* canon) = 0;  // z <- canon[vec[j]] for INIT slots
  virtual cudaError_t enqueue_noise() = 0;  // z <- Z4 noise for INIT slots with a noise rhs
  virtual cudaError_t enqueue_init() = 0;
  virtual cudaError_t enqueue_iter() = 0;
  virtual cudaError_t enqueue_iters(int k) = 0;  // k iterations, from a captured CUDA graph when possible
  virtual cudaError_t enqueue_recon() = 0;
  virtual cudaError_t enqueue_verify() = 0;
  virtual cudaError_t enqueue_solution_to_canon(double* canon) = 0;  // canon[vec[j]] <- x for all j with vec >= 0
  virtual cudaError_t enqueue_dslash(double* canon) = 0;  // canon[vec[j]] <- (D + sigma_j) canon[vec[j]], INIT slots
  // FP64 field pairs (even, odd) of every slot: PAIR_X the solution (x_hi, x_o), PAIR_Z the
  // right-hand side (z_e, z_o), PAIR_S scratch (r_hi and the FP64 temporary); the last two are
  // free once a system has finished
  virtual double* field_pair(int id, int parity) = 0;
  // pair `to` <- kappa H (pair `from`), full lattice, FP64, for the FLAG_HPE slots (Wilson-clover:
  // to <- A(x)^-1 H from / 2, the generalised expansion)
  virtual cudaError_t enqueue_kappa_hop(int from, int to) = 0;
  // pair `to` <- A(x)^-1 (pair `from`) with A(x) = 4 + m + sigma + C(x), FP64, for the FLAG_HPE slots
  // (the Wilson-clover operator only)
  virtual cudaError_t enqueue_site_inverse(int from, int to) = 0;
  // Staging of finished solutions (run_queue): S columns laid out like the tile's FP64 fields
  // (system-major, one column = one system's parity, 24 Vh doubles, contiguous), so a slot's
  // solution moves with plain device copies and its slot is free at once. y holds the
  // expansion's (kappa H)^K x when requested. Allocated on first use; 0 or 3 (out of memory).
  double *stage_x_e = nullptr, *stage_x_o = nullptr, *stage_y_e = nullptr, *stage_y_o = nullptr;
  NoiseSpec* stage_spec_d = nullptr;
  NoiseSpec* stage_spec_h = nullptr;  // pinned mirror
  int stage_cols = 0;
  virtual int stage_alloc(int S, bool with_y) = 0;
  // CGNR fallback (FP64) for the slots flagged FLAG_CG; its vectors are allocated on first use
  virtual int cg_alloc() = 0;
  virtual cudaError_t enqueue_cg_init() = 0;
  virtual cudaError_t enqueue_cg_iter() = 0;
};

// The packed (A + C(x))^-1 of one shift (Wilson-clover), [2][Vh][2][CLV_PACKED] reals.
struct ClvInv {
  double* t64 = nullptr;
  float* t32 = nullptr;
};

struct Ctx {
  int device = 0;
  int nsm = 0;
  Geom g{};
  cudaStream_t own_stream = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
  bool have_gauge = false;
  void* gauge64 = nullptr;              // [2][4][Vh][18] doubles
  std::map<int, void*> gauge_lo;        // key: prec * 100 + nr
  double* wline = nullptr;              // straight z-paths W(x, x + q z) of the contraction
  size_t wline_cap = 0;                 // bytes allocated
  int wline_mask = 0;                   // the q > 0 they hold (bit q); 0: none or stale
  int* colors_d = nullptr;              // probing colour per canonical site, [V] (probed noise)
  bool colors_own = false;              // colors_d allocated by this context
  std::map<long long, std::unique_ptr<TileBase>> tiles;
  double* canon_d = nullptr;            // staging for canonical vectors
  size_t canon_cap = 0;                 // in vectors
  double* canon_h = nullptr;            // pinned host staging
  size_t canon_h_cap = 0;
  HopProfile prof;
  size_t extra_bytes = 0;

  int fail(int code, const std::string& msg) {
    err = msg;
    return code;
  }
  int cuda_fail(cudaError_t e, const char* where);
  Launch launch_for(const Shape& sh) const;
  void* gauge_for(int prec, int nr);    // builds the copy on demand; nullptr on failure
  TileBase* tile(int prec, int N, int nr);
  int ensure_canon(size_t nvec);
  int ensure_canon_host(size_t nvec);
  size_t device_bytes() const;
  // Lanes: contexts of their own (stream, tiles, staging, profile) that share this context's
  // gauge copies and contraction paths (read-only while they run), so that tiles in different
  // lanes can run at the same time. lane(i) creates lane i on first use and refreshes the shared
  // pointers; nullptr on failure (message in err).
  std::vector<std::unique_ptr<Ctx>> lanes;
  bool shared = false;  // a lane: the gauge copies and contraction paths are not its own
  Ctx* lane(int i);
  std::map<int, int> tuned_tile;  // autotuned systems per tile, key: prec * 100 + nr
  std::map<long long, PkShape> tuned_shape;  // autotuned hop shape, key: (prec * 100 + nr) * 1000 + N
  long long iter_bound = 0;       // watchdog of the host solve loops (iterations); 0: built-in bound
  // the clover term (Wilson-clover operator) when c_sw != 0: per-site tables of the gauge field
  double c_sw = 0.0;
  double* clover64 = nullptr;     // [2][Vh][2][CLV_REALS]
  float* clover32 = nullptr;
  std::map<double, ClvInv> clv_inv;  // packed inverses per A = 4 + m + sigma, built per call (owner only)
};

// Builds c's clover tables from its FP64 gauge copy (fs_clover.cu); 0 or an error code.
int clover_build(Ctx* c, double c_sw);
// Frees every packed inverse (their table changed).
void clover_inverses_free(Ctx* c);

// The contraction's straight z-paths W(x, x + q z) for the displacements q > 0 in pmask,
// built once per gauge field (fs_engine.cu); 0 or an error code (message in c->err).
int ensure_wline(Ctx* c, int pmask, int pmax);

// Copies the probing colours (host, [V] in canonical site order) to c->colors_d, on c's stream.
int upload_colors(Ctx* c, const int* colors);

enum { PAIR_X = 0, PAIR_Z = 1, PAIR_S = 2 };

// One system to solve.
struct SysSpec {
  double sigma;
  int rhs_kind;        // 0: Z4 noise, 1: canonical vector `vec` (device staging)
  int vec;             // canonical vector index for rhs_kind 1
  NoiseSpec noise;     // noise identity (the right-hand side and/or the contraction's left vector)
  int hpe = 0;         // 1: the solution takes QOut::hpe_order kappa H applications (into the field
                       // pair of hpe_result_pair) before the contractions that read it (right_kind 1)
};

struct SolveOpts {
  const std::map<double, ClvInv>* clv_inv = nullptr;  // per A = 4 + m + sigma; read-only during a call
  double m;
  double tol;
  int max_iter;
  int prec;
  int nr;
  double delta;
  int verify;
  int check_every;
  int cg_max_iter;  // CGNR fallback iterations; 0: no fallback
};

// The packed (A + C(x))^-1 for every shift sigma[0..n) of a call (A = 4 + m + sigma), built from
// the eigen-decomposed table where missing and kept for later calls (beyond 32 in all, the kept
// tables of shifts the call does not name are dropped first); o.clv_inv then points at them. A
// no-op without the clover term. 0 or an error code (3: no device memory for them) (fs_clover.cu).
int clover_inverses(Ctx* c, double m, const double* sigma, int n, SolveOpts& o);

// A group of systems whose solutions are contracted together (they share the tile
// until all of them have converged).
struct QJob {
  std::vector<SysSpec> sys;
  std::vector<double> chain;           // per system: NaN = none, else the follow-up shift
  std::vector<ContractPair> pairs;     // right / left are group-local; out is a global result row
  std::vector<int> stat_index;         // per system: stats row of its (first) solve, -1 none
  std::vector<int> stat_index2;        // per system: stats row of the follow-up solve
  std::vector<int> out_index;          // per system: host output vector index (-1 none)
};

struct QOut {
  const double* gamma = nullptr;
  const std::vector<int>* plist = nullptr;
  int rows = 0;
  std::vector<double>* result = nullptr;    // [rows][np][2]
  std::vector<SysState>* states = nullptr;
  int* noconv = nullptr;
  double* x_host = nullptr;                 // solutions, [out_index][V][24]
  int canon_out_base = 0;                   // staging vectors [base, base + N) for outputs
  int canon_chain_base = 0;                 // staging vectors [base, base + N) for follow-up rhs
  int hpe_order = 0;                        // K of the hopping parameter expansion (SysSpec::hpe)
  const double* rhs_canon = nullptr;        // caller's device right-hand sides [vec][V][24] (else staging)
  double* x_dev = nullptr;                  // caller's device solutions [out_index][V][24]
};

// Field pair that holds (kappa H)^K x after the expansion's K hops from PAIR_X (alternating
// between PAIR_S and PAIR_Z).
inline int hpe_result_pair(int K) { return (K % 2) ? PAIR_S : PAIR_Z; }

// Continuous batching of the jobs over the slots of tile T (fs_driver.cu).
int run_queue(Ctx* c, TileBase* T, const std::vector<QJob>& jobs, const SolveOpts& o, const QOut& out);

// Tile autotuner (fs_driver.cu): systems per tile for (o.prec, o.nr) on this lattice, at most
// nmax; measured once per context and format, then cached in c->tuned_tile. 0 on failure.
int autotune_tile(Ctx* c, const SolveOpts& o, int nmax);

// Where contract_tile reads its vectors when they are not the tile's own: the staging columns.
struct StageView {
  const double *x_e, *x_o, *y_e, *y_o;
  const NoiseSpec* spec;
  int N;
};

// Contractions over the solutions held in a tile (or, with sv, in its staging columns); pairs
// with right_kind 1 read their right vector from field pair `right_pair` (sv: the staged y).
int contract_tile(Ctx* c, TileBase* T, const std::vector<ContractPair>& pairs, const double* gamma,
                  const std::vector<int>& plist, std::vector<double>& result /* [rows][np][2] */, int rows,
                  int right_pair = PAIR_X, const StageView* sv = nullptr);

// Exact low orders of the hopping parameter expansion (Sec. 3.1, the remark after
// Eq. (sampled_single)): T = sum_{k<K} Tr(Gamma Omega_p (kappa H)^k) / A, A = 4 + m + sigma,
// from displacement-p distance-(K-1) probing vectors with full spin-colour dilution on the idle
// tile T (fs_driver.cu). out = {re, im}; 0 or an error code (message in c->err).
int hpe_exact(Ctx* c, TileBase* T, const SolveOpts& o, double sigma, int K, int p, const double* gamma,
              uint64_t seed, double out[2]);

double* pinned_alloc(size_t bytes);
void note_launch(int n = 1);          // library-wide count of kernel launches
long long launch_count();
cudaError_t launch_noise_codes(uint8_t* codes, NoiseSpec n, int V, cudaStream_t s);

}  // namespace fs

// The opaque context handle of the C ABI.
struct fs_ctx {
  fs::Ctx c;
};
