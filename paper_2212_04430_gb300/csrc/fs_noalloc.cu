// wilson_dslash_noalloc: the Wilson operator (D + sigma I) on device buffers, with
// no device allocation at all.
//
// Who needs it: code that must not call cudaMalloc / cudaFree (or any allocator
// that wraps them) while it runs: work recorded inside a CUDA stream capture
// region, where allocating calls are not permitted; callers that run under a
// fixed device-memory budget set up in advance (a serving process that has
// carved up the GPU, an embedding application that owns the allocator); and
// latency-critical loops where an allocation's implicit synchronisation or
// failure is not acceptable. The regular wilson_dslash allocates its context
// buffers on demand, so it cannot serve them.
//
// How: the even-odd packed gauge field, the packed input and output spinors, the
// per-system coefficients and the slot map live in one file-scope
// `static __device__` scratch array of FS_NOALLOC_SCRATCH_BYTES. Every GPU that
// loads this library holds that array until the process exits. Host code never
// dereferences the array's symbol: on the first call on a device (that device
// current) the library asks the runtime for its device address with
// cudaGetSymbolAddress, checks the result, caches it per device and passes it to
// the kernels. Because that first call performs this set-up, it should happen
// before any stream capture on the device.
//
// All calls on a device share the one array and it keeps the contents of the
// last call: every field a call reads is rewritten by that call first (nothing
// relies on a zeroed array), and calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on the array and corrupt each other.
// The cached address belongs to the device's current context: after a
// cudaDeviceReset it is stale and the entry point must not be called again in
// that process.
//
// Errors: a CUDA error already pending when the call starts (left by unrelated
// work) makes it return FS_ERR_CUDA at once, without touching or clearing that
// error; otherwise each of its own launches is checked.
#include <algorithm>
#include <mutex>

#include "fs_engine.h"
#include "fsmlmc.h"

#define FS_NOALLOC_SCRATCH_BYTES (32u << 20)  // 32 MiB per device
#define FS_NOALLOC_MAX_DEVICES 64

namespace {

static __device__ __align__(256) unsigned char fs_noalloc_scratch[FS_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_addr[FS_NOALLOC_MAX_DEVICES] = {nullptr};

// Per-system state of the scratch run: coefficient A = 4 + m + sigma, all
// systems selected, slot j <-> vector j. Written in full by the kernel itself.
__global__ void noalloc_init_kernel(fs::SysState* st, int* vec, int n, double A) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  fs::SysState s;
  unsigned char* b = reinterpret_cast<unsigned char*>(&s);
  for (size_t k = 0; k < sizeof(fs::SysState); k++) b[k] = 0;
  s.A = A;
  s.cd[fs::C_A] = A;
  s.cf[fs::C_A] = (float)A;
  s.flags = fs::FLAG_INIT;
  st[j] = s;
  vec[j] = j;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int wilson_dslash_noalloc(const int dims[4], int bc_t, double m, double sigma, const double* U,
                                     const double* in, double* out, int nrhs, void* stream) {
  if (!dims || !U || !in || !out) return FS_ERR_ARG;
  if (nrhs < 0 || nrhs > fs::MAX_TILE) return FS_ERR_ARG;
  if (bc_t != 1 && bc_t != -1) return FS_ERR_ARG;
  long long V = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (dims[mu] < 2 || dims[mu] % 2) return FS_ERR_ARG;
    V *= dims[mu];
  }
  if (nrhs == 0) return FS_OK;
  if (V >= (1LL << 27)) return FS_ERR_BUDGET;
  const size_t Vh = (size_t)V / 2;
  const size_t gauge_bytes = align256(8 * Vh * 18 * sizeof(double));
  const size_t field_bytes = align256(Vh * 24 * (size_t)nrhs * sizeof(double));
  const size_t state_bytes = align256((size_t)nrhs * sizeof(fs::SysState));
  const size_t vec_bytes = align256((size_t)nrhs * sizeof(int));
  const size_t need = gauge_bytes + 4 * field_bytes + state_bytes + vec_bytes;
  if (need > FS_NOALLOC_SCRATCH_BYTES) return FS_ERR_BUDGET;  // lattice x nrhs beyond the fixed scratch

  // an error left pending by other work is not ours to clear: refuse before launching anything
  if (cudaPeekAtLastError() != cudaSuccess) return FS_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= FS_NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return FS_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, fs_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return FS_ERR_CUDA;
      }
      g_addr[dev] = p;
    }
    base = (unsigned char*)g_addr[dev];
  }
  double* gauge = (double*)base;
  double* in_e = (double*)(base + gauge_bytes);
  double* in_o = (double*)(base + gauge_bytes + field_bytes);
  double* out_e = (double*)(base + gauge_bytes + 2 * field_bytes);
  double* out_o = (double*)(base + gauge_bytes + 3 * field_bytes);
  fs::SysState* st = (fs::SysState*)(base + gauge_bytes + 4 * field_bytes);
  int* vec = (int*)(base + gauge_bytes + 4 * field_bytes + state_bytes);

  fs::Geom g{};
  for (int mu = 0; mu < 4; mu++) g.L[mu] = dims[mu];
  g.Lh0 = dims[0] / 2;
  g.V = (int)V;
  g.Vh = (int)Vh;
  g.bc_t = bc_t;
  fs::geom_init_div(g);
  cudaStream_t s = (cudaStream_t)stream;
  const fs::Shape sh = fs::make_shape(nrhs, g.Vh);
  const int gy = (nrhs + sh.NB - 1) / sh.NB;
  const int block = sh.SB * sh.NB;

  // no error was pending on entry, so an error read here comes from this call's own launches
  int launched = 0;
  auto launched_ok = [&]() {
    launched++;
    return cudaGetLastError() == cudaSuccess;
  };
  noalloc_init_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(st, vec, nrhs, 4.0 + m + sigma);
  bool ok = launched_ok();
  if (ok) {
    fs::gauge_pack_kernel<double, 18><<<(8 * g.Vh + 255) / 256, 256, 0, s>>>(gauge, U, g);
    ok = launched_ok();
  }
  if (ok) {
    fs::pack_kernel<double><<<dim3(std::min(2 * sh.nchunk, 65535), gy), block, 0, s>>>(in_e, in_o, in, vec, g, sh,
                                                                                     false);
    ok = launched_ok();
  }
  fs::HopArgs a{};
  a.gauge = gauge;
  a.st = st;
  a.g = g;
  a.sh = sh;
  a.mask = fs::MASK_INIT;
  // out_e = A in_e - H_eo in_o / 2 ; out_o = A in_o - H_oe in_e / 2
  if (ok) {
    a.out = out_e; a.in = in_o; a.X = in_e; a.p_out = 0;
    fs::hop_kernel<double, double, double, 18, fs::COEF_DSLASH, fs::DOT_NONE><<<dim3(sh.nchunk, gy), block, 0, s>>>(a);
    ok = launched_ok();
  }
  if (ok) {
    a.out = out_o; a.in = in_e; a.X = in_o; a.p_out = 1;
    fs::hop_kernel<double, double, double, 18, fs::COEF_DSLASH, fs::DOT_NONE><<<dim3(sh.nchunk, gy), block, 0, s>>>(a);
    ok = launched_ok();
  }
  if (ok) {
    fs::unpack_kernel<double><<<dim3(std::min(2 * sh.nchunk, 65535), gy), block, 0, s>>>(out, out_e, out_o, vec, g,
                                                                                       sh, false);
    ok = launched_ok();
  }
  fs::note_launch(launched);
  return ok ? FS_OK : FS_ERR_CUDA;
}
