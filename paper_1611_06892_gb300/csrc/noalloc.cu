// bidiag_band_noalloc: the band reduction for callers that must not allocate device memory.
//
// Everything the reduction needs besides the caller's input and output (the zero-padded tile copy of
// A, the R copy of R-BiDiag, the T factors, the executor's task program, its completion flags and its
// control words) is carved out of one fixed array in device global memory, g_scratch, declared below
// with a static size.  Every GPU that loads the library holds this array until the process exits.
// Host code cannot use the name g_scratch as a device address: the first call in each CUDA context
// (normally one per device: the device's primary context) looks up the array's device address with
// cudaGetSymbolAddress, with that device current, and keeps it for that context.  The address is
// keyed by the context's unique ID, so a context created after cudaDeviceReset, or a non-primary
// context made current by the caller, gets its own lookup instead of a stale address.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/bidiag.h"
#include "kernels.cuh"
#include "plan.h"

namespace {

constexpr size_t kScratchBytes = (size_t)BIDIAG_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
// (context ID, device address of g_scratch in that context), one entry per context seen
std::vector<std::pair<unsigned long long, unsigned char*>> g_addr;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique ID of the calling thread's current context (the runtime makes the device's primary context
// current when there is none).  False if the driver does not offer the query.
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  CUcontext ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_scratch in the current context (device `dev` current), looked up once per
// context.  Before the runtime has initialised the device there may be no current context: the
// lookup itself initialises it, and the address is then keyed by the context it was found in.
cudaError_t scratch_address(int dev, unsigned char** out) {
  (void)dev;
  unsigned long long id = 0;
  bool keyed = current_context_id(&id);
  std::lock_guard<std::mutex> lock(g_mu);
  if (keyed) {
    for (const auto& kv : g_addr)
      if (kv.first == id) {
        *out = kv.second;
        return cudaSuccess;
      }
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  if (!keyed) keyed = current_context_id(&id);
  if (keyed) g_addr.emplace_back(id, static_cast<unsigned char*>(p));
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int cuda_status(cudaError_t e) { return e == cudaSuccess ? BIDIAG_OK : BIDIAG_ERR_CUDA; }

}  // namespace

extern "C" int bidiag_band_noalloc(int64_t m, int64_t n, const double* d_A, int64_t lda, int nb, int ib, int tree,
                                   int variant, double* d_ab, int64_t ldab, void* cuda_stream) {
  if (m < 1) return -1;
  if (n < 1) return -2;
  if (!d_A) return -3;
  if (lda < m) return -4;
  if (nb < 1 || nb > bd::kMaxNb) return -5;
  if (ib < 1 || ib > (nb < 64 ? nb : 64) || nb % ib) return -6;
  if (tree < 0 || tree > 3) return -7;
  if (variant < 0 || variant > 1) return -8;
  if (!d_ab) return -9;
  if (ldab < nb + 1) return -10;
  if (m < n) return BIDIAG_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

  int dev = 0, nsm = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return BIDIAG_ERR_CUDA;
  if (dev >= kMaxDevices) return BIDIAG_ERR_UNSUPPORTED;

  const int w = bd::choose_strip_width(nb, ib, 32, (size_t)optin - 64, 8);
  if (!w) return BIDIAG_ERR_UNSUPPORTED;
  const size_t smem = bd::exec_smem_bytes(nb, ib, w, 8);

  // The task program is planned on the host (host memory only).
  bd::Plan pl;
  try {
    const char* env = std::getenv("BIDIAG_AUTO_RES");
    const int64_t R = env && std::atoll(env) > 0 ? std::atoll(env) : std::max<int64_t>(1, (int64_t)nsm * w / nb);
    bd::build_plan(pl, m, n, nb, ib, tree, variant, R, w);
  } catch (const std::bad_alloc&) {
    return BIDIAG_ERR_NOMEM;
  } catch (...) {
    return BIDIAG_ERR_UNSUPPORTED;
  }
  const size_t ntask = pl.dev.size();
  const size_t tile = (size_t)nb * nb * sizeof(double);

  // Carve the scratch: control words, completion flags, task program, tiles, R copy, T factors.
  size_t off = 0;
  const size_t o_ctrl = off;   off = align256(off + 4 * sizeof(int));
  const size_t o_done = off;   off = align256(off + (ntask + 1) * sizeof(int));
  const size_t o_task = off;   off = align256(off + ntask * sizeof(bd::DevTask));
  const size_t o_deps = off;   off = align256(off + pl.deps.size() * sizeof(int32_t));
  const size_t o_tiles = off;  off = align256(off + (size_t)pl.p * pl.q * tile);
  const size_t o_tiles2 = off; off = align256(off + (variant == BIDIAG_RBIDIAG ? (size_t)pl.q * pl.q * tile : 0));
  const size_t o_T = off;      off = align256(off + (size_t)(pl.npanels > 0 ? pl.npanels : 1) * ib * nb * sizeof(double));
  if (off > kScratchBytes) return BIDIAG_ERR_SCRATCH;

  unsigned char* base = nullptr;
  if ((e = scratch_address(dev, &base)) != cudaSuccess) return BIDIAG_ERR_CUDA;
  int* ctrl = reinterpret_cast<int*>(base + o_ctrl);
  int* done = reinterpret_cast<int*>(base + o_done);
  double* tiles = reinterpret_cast<double*>(base + o_tiles);
  double* tiles2 = variant == BIDIAG_RBIDIAG ? reinterpret_cast<double*>(base + o_tiles2) : nullptr;

  // The array keeps the previous call's contents: clear what must start at zero.
  if ((e = cudaMemsetAsync(base, 0, o_task, st)) != cudaSuccess) return cuda_status(e);
  if (tiles2 && (e = cudaMemsetAsync(tiles2, 0, (size_t)pl.q * pl.q * tile, st)) != cudaSuccess) return cuda_status(e);
  if (ntask && (e = cudaMemcpyAsync(base + o_task, pl.dev.data(), ntask * sizeof(bd::DevTask), cudaMemcpyHostToDevice,
                                    st)) != cudaSuccess)
    return cuda_status(e);
  if (!pl.deps.empty() && (e = cudaMemcpyAsync(base + o_deps, pl.deps.data(), pl.deps.size() * sizeof(int32_t),
                                               cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_status(e);
  if ((e = bd::launch_pack(d_A, lda, m, n, nb, tiles, pl.p, pl.q, st)) != cudaSuccess) return cuda_status(e);

  if (ntask) {
    bd::ExecParams prm{};
    prm.tasks = reinterpret_cast<const bd::DevTask*>(base + o_task);
    prm.deps = reinterpret_cast<const int32_t*>(base + o_deps);
    prm.ntasks = (int32_t)ntask;
    prm.nflags = (int32_t)ntask + 1;
    prm.done = done;
    prm.head = ctrl;
    prm.err = ctrl + 1;
    prm.buf[0] = tiles;
    prm.ntiles[0] = (int64_t)pl.p * pl.q;
    prm.buf[1] = tiles2;
    prm.ntiles[1] = tiles2 ? (int64_t)pl.q * pl.q : 0;
    prm.T = reinterpret_cast<double*>(base + o_T);
    prm.npanels = pl.npanels;
    prm.nb = nb;
    prm.ib = ib;
    prm.w = w;
    const char* wl = std::getenv("BIDIAG_WAIT_LIMIT_NS");
    prm.wait_ns = wl ? std::strtoull(wl, nullptr, 10) : 20000000000ull;
    prm.esize = 8;
    prm.window = tiles2 ? 0 : bd::kWindowF64BiDiag;
    if ((e = bd::exec_set_smem(smem, 8)) != cudaSuccess) return cuda_status(e);
    int per_sm = bd::exec_max_ctas_per_sm(smem, 8);
    if (per_sm < 1) per_sm = 1;
    const int64_t grid = (int64_t)nsm * per_sm < (int64_t)ntask ? (int64_t)nsm * per_sm : (int64_t)ntask;
    if ((e = bd::launch_exec(prm, (int)grid, smem, st)) != cudaSuccess) return cuda_status(e);
  }
  if ((e = bd::launch_extract(tiles2 ? tiles2 : tiles, tiles2 ? pl.q : pl.p, nb, n, d_ab, ldab, st)) != cudaSuccess)
    return cuda_status(e);

  int err[3] = {0, 0, 0};
  if ((e = cudaMemcpyAsync(err, ctrl + 1, sizeof(err), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_status(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e);
  if (err[0] == bd::DERR_TIMEOUT) return BIDIAG_ERR_TIMEOUT;
  if (err[0] != bd::DERR_OK) return BIDIAG_ERR_CUDA;
  return BIDIAG_OK;
}
