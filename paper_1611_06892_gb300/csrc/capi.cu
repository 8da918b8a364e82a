// C ABI of the library (declared in include/bidiag.h): handles, results, argument checks, the plan
// cache, buffer management and the launches of the pack / executor / extract kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <set>
#include <stdexcept>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/bidiag.h"
#include "kernels.cuh"
#include "plan.h"

namespace {

struct BwdDev;

struct PlanDev {
  bd::Plan plan;
  std::shared_ptr<BwdDev> bwd[2];   // adjoint program of this plan (FP64, FP32 storage), built on first use
  bd::DevTask* d_tasks = nullptr;
  int32_t* d_deps = nullptr;
  int* d_done = nullptr;
  int nflags = 0;
  int64_t ndeps = 0;           // entries of d_deps
  std::vector<int32_t> dump;   // canonical task list, 6 int32 per task
  ~PlanDev() {
    if (d_tasks) cudaFree(d_tasks);
    if (d_deps) cudaFree(d_deps);
    if (d_done) cudaFree(d_done);
  }
};

// Adjoint program (reverse sweep) of a plan and its slot tables on the device.
struct BwdDev {
  bd::BwdPlan bp;
  PlanDev prog;                  // only the device program arrays are used
  int64_t* d_slot_off = nullptr;
  int32_t* d_pinfo = nullptr;
  ~BwdDev() {
    if (d_slot_off) cudaFree(d_slot_off);
    if (d_pinfo) cudaFree(d_pinfo);
  }
};

using PlanKey = std::tuple<int64_t, int64_t, int, int, int, int, int64_t, int, int, int>;   // ..., strip width, esize, priority weights

// Everything about a batch that depends only on its shapes and options: per-matrix configurations and
// plans, the storage layout and the merged device program (cached on the handle, reused by later calls
// with the same shapes).
struct BatchPlan {
  struct One {
    int nb, ib, tree, variant, w;
    std::shared_ptr<PlanDev> pd;
  };
  std::vector<One> mats;
  std::vector<bd::MatInfo> info;
  int64_t tot0 = 0, tot1 = 0, totT = 0, tiles_all = 0, cols_all = 0;
  size_t smem = 0;
  int ntasks = 0;
  PlanDev prog;                 // the merged device program
  void* d_mats = nullptr;       // info on the device
  ~BatchPlan() {
    if (d_mats) cudaFree(d_mats);
  }
};

// Device storage shared by the results of one batched reduction (freed with the last of them).
struct BatchStore {
  void* tiles = nullptr;
  void* tiles2 = nullptr;
  void* T = nullptr;
  void* d_desc = nullptr;
  std::shared_ptr<BatchPlan> plan;   // keeps the program alive while results exist
  ~BatchStore() {
    for (void* p : {tiles, tiles2, T, d_desc})
      if (p) cudaFree(p);
  }
};

}  // namespace

struct bidiag_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int nsm = 0;
  size_t smem_optin = 0;
  std::string err;
  std::map<PlanKey, std::shared_ptr<PlanDev>> cache;
  int* d_ctrl = nullptr;         // [0] queue head, [1..3] device error word
  uint64_t wait_ns = 20000000000ull;
  int64_t auto_res = -1;
  int debug_unset = 0;
  int strip_w = 0;                 // update strip width; 0: 64 for one FP32-storage matrix, else 32
  int timing = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool timed = false;
  std::set<bidiag_result*> live;   // results made on this handle and not yet freed
  int tracing = 0;
  int f32_simt = 0;                // FP32 storage: updates by FFMA instead of 3xTF32 tensor-core products
  int f32_scalars64 = 0;           // FP32 storage: reflector scalars in FP64 instead of float pairs
  int window = -1;                 // executor look-ahead (queue entries scanned); -1: by precision and variant
  int prio = 1;                    // priority weights of the device program: 1 calibrated per kind, 0 flops
  int64_t* d_trace = nullptr;      // per-task trace of the last traced reduction
  std::map<std::tuple<int, int, int, int64_t>, int> splits;   // best three-step split per (p, q, tree, R)
  std::map<std::vector<int64_t>, std::shared_ptr<BatchPlan>> batches;   // batch programs by shapes / options
  int64_t trace_cap = 0, trace_len = 0;
  std::vector<bd::DevTask> trace_dev;   // device program of the last traced launch (queue order)
  std::vector<int32_t> trace_deps;
};

struct bidiag_result {
  bidiag_ctx* h = nullptr;
  std::shared_ptr<PlanDev> pd;
  int64_t m = 0, n = 0;
  int nb = 0, ib = 0, tree = 0, variant = 0, p = 0, q = 0;
  int esize = 8;                  // 8: FP64 storage, 4: FP32 storage (split-precision updates)
  std::shared_ptr<BatchStore> store;   // batched results: tiles, tiles2 and T point into it
  void* tiles = nullptr;
  void* tiles2 = nullptr;
  void* T = nullptr;
  void* ab = nullptr;
  int64_t ldab = 0;
};

namespace {

int fail(bidiag_handle h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(bidiag_handle h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? BIDIAG_ERR_NOMEM : BIDIAG_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                 \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

void dump_tasks(const std::vector<bd::Task>& tasks, std::vector<int32_t>& out) {
  out.resize(tasks.size() * 6);
  for (size_t x = 0; x < tasks.size(); ++x) {
    const bd::Task& t = tasks[x];
    int32_t* o = &out[x * 6];
    o[0] = t.type; o[1] = t.phase; o[2] = t.k; o[3] = t.i; o[4] = t.piv; o[5] = t.j;
  }
}

int upload_program(bidiag_handle h, PlanDev& pd, const std::vector<bd::DevTask>& dev, const std::vector<int32_t>& deps,
                   int extra_flags) {
  const size_t nt = dev.size();
  pd.nflags = (int)nt + extra_flags;
  pd.ndeps = (int64_t)deps.size();
  CK(h, cudaMalloc(&pd.d_tasks, std::max<size_t>(1, nt) * sizeof(bd::DevTask)));
  CK(h, cudaMalloc(&pd.d_deps, std::max<size_t>(1, deps.size()) * sizeof(int32_t)));
  CK(h, cudaMalloc(&pd.d_done, std::max<size_t>(1, pd.nflags) * sizeof(int)));
  if (nt) CK(h, cudaMemcpy(pd.d_tasks, dev.data(), nt * sizeof(bd::DevTask), cudaMemcpyHostToDevice));
  if (!deps.empty()) CK(h, cudaMemcpy(pd.d_deps, deps.data(), deps.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  return BIDIAG_OK;
}

// Resources R of the Auto tree (Sec. 5 "nbcores"): the number of workers that each take one tile
// task.  A tile update is spread over nb / w SMs (one column strip each), so the default is
// SMs * w / nb for FP64 storage.  With FP32 storage the updates are about ten times faster while the
// panels are not, so more, smaller groups pay: SMs * 64 / nb (twice the FP64 value at w = 32; with the
// 64-column FP32 strips the same R): 8192^2 took 190 ms with it against 232 ms with SMs * 32 / nb
// (FP64: 1398 vs 1386 ms, and 4096^2 prefers the smaller R).  BIDIAG_OPT_AUTO_RESOURCES overrides it.
int64_t resources_of(bidiag_handle h, int nb, int w, int esize) {
  if (h->auto_res > 0) return h->auto_res;
  return std::max<int64_t>(1, (int64_t)h->nsm * (esize == 4 ? 64 : w) / nb);
}

// Executor launch of a program held in pd with the given buffers.
int run_exec(bidiag_handle h, const PlanDev& pd, int ntasks, void* b0, int64_t n0, void* b1, int64_t n1, void* b2,
             int64_t n2, void* T, int npanels, int nb, int ib, int w, int esize, bool timed = false,
             const bd::MatInfo* d_mats = nullptr, int nmats = 0, size_t smem_batch = 0,
             const void* const* bx = nullptr, const int64_t* nx = nullptr, const bd::BwdParams* bwd = nullptr,
             int auto_window = 0) {
  if (ntasks == 0) return BIDIAG_OK;
  size_t smem = d_mats ? smem_batch : (bwd ? bd::bwd_smem_bytes(nb, ib, bwd->hw, esize) : bd::exec_smem_bytes(nb, ib, w, esize));
  // tcgen05 updates (FP32 forward, one CTA per SM): TMEM for one accumulator of N = max(w, ib) (rounded to
  // 16) columns per 128-row chunk of the tile and per k-step of 8, allocated as a power of two of at
  // least 32 columns, and the shared memory of that path's layout
  int umma_cols = 0;
  if (esize == 4 && !bwd && !d_mats && h->f32_simt == 0 && nb % 16 == 0 && ib == 32 && w <= 64) {
    const int need = ((nb + 127) / 128) * (ib / 8) * ((std::max(w, ib) + 15) / 16 * 16);
    int cols = 32;
    while (cols < need) cols *= 2;
    const size_t su = std::max(smem, bd::umma_smem_bytes(nb, ib, w));
    if (cols <= 512 && su <= h->smem_optin && bd::exec_set_smem(su, esize, false) == cudaSuccess &&
        bd::exec_max_ctas_per_sm(su, esize, false) == 1) {
      umma_cols = cols;
      smem = su;
    }
  }
  CK(h, bd::exec_set_smem(smem, esize, bwd != nullptr));
  const int per_sm = std::max(1, bd::exec_max_ctas_per_sm(smem, esize, bwd != nullptr));
  bd::ExecParams prm{};
  prm.tasks = pd.d_tasks;
  prm.deps = pd.d_deps;
  prm.ntasks = ntasks;
  prm.nflags = pd.nflags;
  prm.done = pd.d_done;
  prm.head = h->d_ctrl;
  prm.err = h->d_ctrl + 1;
  prm.buf[0] = b0; prm.ntiles[0] = n0;
  prm.buf[1] = b1; prm.ntiles[1] = n1;
  prm.buf[2] = b2; prm.ntiles[2] = n2;
  for (int i = 0; i < 3; ++i) {   // buffers 3..5 (adjoint only)
    prm.buf[3 + i] = bx ? const_cast<void*>(bx[i]) : nullptr;
    prm.ntiles[3 + i] = nx ? nx[i] : 0;
  }
  if (bwd) prm.bwd = *bwd;
  prm.T = T;
  prm.npanels = npanels;
  prm.nb = nb;
  prm.ib = ib;
  prm.w = w;
  prm.wait_ns = h->wait_ns;
  prm.esize = esize;
  prm.f32_simt = h->f32_simt;
  prm.f32_scalars64 = h->f32_scalars64;
  prm.window = h->window >= 0 ? h->window : auto_window;
  prm.umma_cols = umma_cols;
  prm.mats = d_mats;
  prm.nmats = nmats;
  prm.trace = nullptr;
  if (timed && h->tracing) {
    if (h->trace_cap < ntasks) {
      if (h->d_trace) CK(h, cudaFree(h->d_trace));
      h->d_trace = nullptr;
      CK(h, cudaMalloc(&h->d_trace, sizeof(int64_t) * 4 * (size_t)ntasks));
      h->trace_cap = ntasks;
    }
    prm.trace = h->d_trace;
    h->trace_len = ntasks;
    // keep the program this trace belongs to (its queue order and dependencies)
    h->trace_dev.resize((size_t)ntasks);
    h->trace_deps.resize((size_t)pd.ndeps);
    CK(h, cudaMemcpy(h->trace_dev.data(), pd.d_tasks, sizeof(bd::DevTask) * (size_t)ntasks, cudaMemcpyDeviceToHost));
    if (pd.ndeps)
      CK(h, cudaMemcpy(h->trace_deps.data(), pd.d_deps, sizeof(int32_t) * (size_t)pd.ndeps, cudaMemcpyDeviceToHost));
  }
  CK(h, cudaMemsetAsync(pd.d_done, 0, sizeof(int) * (size_t)pd.nflags, h->stream));
  CK(h, cudaMemsetAsync(h->d_ctrl, 0, sizeof(int), h->stream));
  const int grid = std::min<int64_t>((int64_t)h->nsm * per_sm, ntasks);
  if (timed) CK(h, cudaEventRecord(h->ev[0], h->stream));
  CK(h, bd::launch_exec(prm, grid, smem, h->stream));
  if (timed) CK(h, cudaEventRecord(h->ev[1], h->stream));
  return BIDIAG_OK;
}

// Strip width of a one-matrix reduction: with FP32 storage 64 columns by default (each inner block of
// V staged in shared memory then serves twice the columns; 8192^2: 162 -> 150 ms), else 32.
int choose_strip(bidiag_handle h, int nb, int ib, int esize, int* w) {
  const int pref = h->strip_w > 0 ? h->strip_w : (esize == 4 ? 64 : 32);
  *w = bd::choose_strip_width(nb, ib, pref, h->smem_optin, esize);
  if (*w) return BIDIAG_OK;
  return fail(h, BIDIAG_ERR_UNSUPPORTED, "tile size / inner blocking need more shared memory than the device has");
}

int get_plan(bidiag_handle h, int64_t m, int64_t n, int nb, int ib, int tree, int variant, int w, int esize,
             std::shared_ptr<PlanDev>* out) {
  const int64_t R = resources_of(h, nb, w, esize);
  const bool debug = h->debug_unset != 0;
  PlanKey key{m, n, nb, ib, tree, variant, R, w, esize, h->prio};
  if (!debug) {
    auto it = h->cache.find(key);
    if (it != h->cache.end()) {
      *out = it->second;
      return BIDIAG_OK;
    }
  }
  auto pd = std::make_shared<PlanDev>();
  try {
    bd::build_plan(pd->plan, m, n, nb, ib, tree, variant, R, w, esize, h->prio);
  } catch (const std::bad_alloc&) {
    return fail(h, BIDIAG_ERR_NOMEM, "host allocation failed while planning");
  } catch (const std::exception& e) {
    return fail(h, BIDIAG_ERR_UNSUPPORTED, std::string("planner: ") + e.what());
  }
  dump_tasks(pd->plan.tasks, pd->dump);
  std::vector<int32_t> deps = pd->plan.deps;
  std::vector<bd::DevTask> dev = pd->plan.dev;
  int extra = 1;
  if (debug && !dev.empty()) {
    // failure-path test: the first queued task also waits for a flag that nothing sets
    const int32_t never = (int32_t)dev.size();
    std::vector<int32_t> nd;
    nd.push_back(never);
    for (size_t y = 0; y < dev.size(); ++y) {
      const int32_t b = (int32_t)nd.size();
      if (y == 0) {
        for (int32_t d = dev[y].dep_begin; d < dev[y].dep_end; ++d) nd.push_back(deps[d]);
        dev[y].dep_begin = 0;
        dev[y].dep_end = (int32_t)nd.size();
        continue;
      }
      for (int32_t d = dev[y].dep_begin; d < dev[y].dep_end; ++d) nd.push_back(deps[d]);
      dev[y].dep_begin = b;
      dev[y].dep_end = (int32_t)nd.size();
    }
    deps.swap(nd);
    h->debug_unset = 0;
  }
  int rc = upload_program(h, *pd, dev, deps, extra);
  if (rc) return rc;
  if (!debug) h->cache[key] = pd;
  *out = pd;
  return BIDIAG_OK;
}

template <typename T>
int dev_alloc(bidiag_handle h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return BIDIAG_OK;
  cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMallocAsync");
  return BIDIAG_OK;
}

void free_result_buffers(bidiag_result* r) {
  cudaStream_t s = r->h ? r->h->stream : nullptr;
  if (!r->store) {
    if (r->tiles) cudaFreeAsync(r->tiles, s);
    if (r->tiles2) cudaFreeAsync(r->tiles2, s);
    if (r->T) cudaFreeAsync(r->T, s);
  }
  if (r->ab) cudaFreeAsync(r->ab, s);
  r->tiles = r->tiles2 = r->T = r->ab = nullptr;
  r->store.reset();
}

// Replays the panel tasks of one side (QR side: left = true; LQ side: left = false) on a tiled copy of C.
template <typename E>
int apply_side(bidiag_handle h, bidiag_result_t r, bool left, int trans, int64_t other, E* C, int64_t ldc) {
  const bd::Plan& pl = r->pd->plan;
  const int nb = r->nb, ib = r->ib;
  const int64_t crow = left ? r->m : other, ccol = left ? other : r->n;
  if (crow == 0 || ccol == 0) return BIDIAG_OK;
  const int64_t rows_t = (crow + nb - 1) / nb, cols_t = (ccol + nb - 1) / nb;
  const int64_t nblk = left ? cols_t : rows_t;   // independent tile columns of the oriented C
  int w = 0;
  int rc = choose_strip(h, nb, ib, (int)sizeof(E), &w);
  if (rc) return rc;
  const int S = (nb + w - 1) / w;
  // panel tasks of this side, in application order
  std::vector<int32_t> panels;
  for (size_t x = 0; x < pl.tasks.size(); ++x) {
    const bd::Task& t = pl.tasks[x];
    if (!(t.type == bd::GEQRT || t.type == bd::TSQRT || t.type == bd::TTQRT)) continue;
    if ((t.phase == bd::PH_LQ) == left) continue;
    panels.push_back((int32_t)x);
  }
  // left: Q^T C forward (trans = 1) / Q C backward.  right: C P forward with Q^T-mode on C^T (trans = 0),
  // C P^T backward with Q-mode.
  const bool forward = left ? (trans == 1) : (trans == 0);
  const bool notrans = !forward;
  if (!forward) std::reverse(panels.begin(), panels.end());
  std::vector<bd::DevTask> dev;
  std::vector<int32_t> deps;
  std::vector<int32_t> last((size_t)rows_t * cols_t * S, -1);   // last writer per (C tile, strip)
  auto cref = [&](int64_t orow, int64_t ocol) {                  // oriented C tile -> buffer-2 reference
    const int64_t a = left ? orow : ocol, b = left ? ocol : orow;
    return std::make_pair(bd::tile_ref(2, b * rows_t + a), b * rows_t + a);
  };
  for (int32_t x : panels) {
    const bd::Task& t = pl.tasks[x];
    const int buf = bd::task_buffer(t.phase, t.k, r->variant);
    const int grid_rows = buf == 0 ? r->p : r->q;
    const bool lq = t.phase == bd::PH_LQ;
    const int ax = lq ? t.k : t.i, ay = lq ? t.i : t.k;     // actual tile of oriented (i, k)
    const int32_t vref = bd::tile_ref(buf, (int64_t)ay * grid_rows + ax);
    const int utype = t.type == bd::GEQRT ? bd::UNMQR : (t.type == bd::TSQRT ? bd::TSMQR : bd::TTMQR);
    for (int64_t b = 0; b < nblk; ++b) {
      auto ci = cref(t.i, b);
      std::pair<int32_t, int64_t> cp{-1, -1};
      if (utype != bd::UNMQR) cp = cref(t.piv, b);
      for (int s = 0; s < S; ++s) {
        bd::DevTask d{};
        d.op = utype | ((lq ? 1 : 0) << 4) | ((notrans ? 1 : 0) << 5) | (s << 8);
        d.x = vref;
        d.a = cp.first;
        d.c = ci.first;
        d.tslot = pl.tslot[x];
        d.flags = 0;
        d.dep_begin = (int32_t)deps.size();
        const int32_t me = (int32_t)dev.size();
        int32_t& lc = last[(size_t)ci.second * S + s];
        if (lc >= 0) deps.push_back(lc);
        if (cp.second >= 0) {
          int32_t& lp = last[(size_t)cp.second * S + s];
          if (lp >= 0 && lp != lc) deps.push_back(lp);
          lp = me;
        }
        lc = me;
        d.dep_end = (int32_t)deps.size();
        dev.push_back(d);
      }
    }
  }
  if (dev.empty()) return BIDIAG_OK;
  PlanDev prog;
  rc = upload_program(h, prog, dev, deps, 1);
  if (rc) return rc;
  E* Ct = nullptr;
  rc = dev_alloc(h, &Ct, (size_t)rows_t * cols_t * nb * nb);
  if (rc) return rc;
  CK(h, bd::launch_pack(C, ldc, crow, ccol, nb, Ct, rows_t, cols_t, h->stream));
  rc = run_exec(h, prog, (int)dev.size(), r->tiles, (int64_t)r->p * r->q, r->tiles2,
                r->tiles2 ? (int64_t)r->q * r->q : 0, Ct, rows_t * cols_t, r->T, pl.npanels, nb, ib, w,
                (int)sizeof(E));
  if (rc) return rc;
  CK(h, bd::launch_unpack(Ct, rows_t, nb, crow, ccol, C, ldc, h->stream));
  CK(h, cudaFreeAsync(Ct, h->stream));
  // the program buffers are freed by ~PlanDev; wait for the stream so that they outlive the launch
  CK(h, cudaStreamSynchronize(h->stream));
  return BIDIAG_OK;
}

template <typename E>
int band_impl(bidiag_handle h, int64_t m, int64_t n, const E* d_A, int64_t lda, int nb, int ib, int tree,
              int variant, bidiag_result_t* out) {
  if (!h) return -1;
  if (m < 1) return fail(h, -2, "m < 1");
  if (n < 1) return fail(h, -3, "n < 1");
  if (!d_A) return fail(h, -4, "A is NULL");
  if (lda < m) return fail(h, -5, "lda < m");
  if (nb < 1 || nb > bd::kMaxNb) return fail(h, -6, "nb out of range");
  if (ib < 1 || ib > std::min(nb, 64) || nb % ib) return fail(h, -7, "ib out of range or does not divide nb");
  if (tree < 0 || tree > 3) return fail(h, -8, "unknown tree");
  if (variant < 0 || (variant > BIDIAG_THREESTEP && variant - BIDIAG_THREESTEP_SPLIT(0) >= (n + nb - 1) / nb))
    return fail(h, -9, "unknown variant or three-step split >= q");
  if (!out) return fail(h, -10, "out is NULL");
  *out = nullptr;
  if (m < n) return fail(h, BIDIAG_ERR_UNSUPPORTED, "m < n: reduce the transpose");
  CK(h, cudaSetDevice(h->device));
  int w = 0;
  int rc = choose_strip(h, nb, ib, (int)sizeof(E), &w);
  if (rc) return rc;
  if (variant == BIDIAG_AUTO_VARIANT || variant == BIDIAG_THREESTEP) {
    const int p = (int)((m + nb - 1) / nb), q = (int)((n + nb - 1) / nb);
    const int64_t R = resources_of(h, nb, w, (int)sizeof(E));
    try {
      if (variant == BIDIAG_AUTO_VARIANT) {
        variant = bd::choose_variant(p, q, tree, R, nullptr, nullptr);
      } else {
        const auto key = std::make_tuple(p, q, tree, R);
        auto it = h->splits.find(key);
        const int sp = it != h->splits.end() ? it->second : bd::best_split(p, q, tree, R, nullptr);
        h->splits[key] = sp;
        variant = BIDIAG_THREESTEP_SPLIT(sp);
      }
    } catch (...) {
      return fail(h, BIDIAG_ERR_NOMEM, "host allocation failed while choosing the variant");
    }
  }
  if (variant == BIDIAG_THREESTEP_SPLIT(0)) variant = BIDIAG_RBIDIAG;   // the same task list
  std::shared_ptr<PlanDev> pd;
  rc = get_plan(h, m, n, nb, ib, tree, variant, w, (int)sizeof(E), &pd);
  if (rc) return rc;
  bidiag_result* r = new (std::nothrow) bidiag_result();
  if (!r) return fail(h, BIDIAG_ERR_NOMEM, "host allocation failed");
  r->h = h;
  r->pd = pd;
  r->m = m;
  r->n = n;
  r->nb = nb;
  r->ib = ib;
  r->tree = tree;
  r->variant = variant;
  r->p = pd->plan.p;
  r->q = pd->plan.q;
  r->ldab = nb + 1;
  r->esize = (int)sizeof(E);
  const size_t tile_elems = (size_t)nb * nb;
  E *tiles = nullptr, *tiles2 = nullptr, *Tst = nullptr, *ab = nullptr;
  rc = dev_alloc(h, &tiles, (size_t)r->p * r->q * tile_elems);
  if (!rc && bd::split_of(variant) >= 0) rc = dev_alloc(h, &tiles2, (size_t)r->q * r->q * tile_elems);
  if (!rc) rc = dev_alloc(h, &Tst, (size_t)std::max(1, pd->plan.npanels) * ib * nb);
  if (!rc) rc = dev_alloc(h, &ab, (size_t)(nb + 1) * n);
  r->tiles = tiles;
  r->tiles2 = tiles2;
  r->T = Tst;
  r->ab = ab;
  if (rc) {
    free_result_buffers(r);
    delete r;
    return rc;
  }
  auto bail = [&](int code) {
    free_result_buffers(r);
    delete r;
    return code;
  };
  cudaError_t e = bd::launch_pack(d_A, lda, m, n, nb, tiles, r->p, r->q, h->stream);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "pack"));
  if (r->tiles2) {
    e = cudaMemsetAsync(r->tiles2, 0, (size_t)r->q * r->q * tile_elems * sizeof(E), h->stream);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "memset"));
  }
  const bool timed = h->timing != 0 || h->tracing != 0;
  if (timed && !h->ev[0]) {
    e = cudaEventCreate(&h->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev[1]);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaEventCreate"));
  }
  rc = run_exec(h, *pd, (int)pd->plan.dev.size(), r->tiles, (int64_t)r->p * r->q, r->tiles2,
                r->tiles2 ? (int64_t)r->q * r->q : 0, nullptr, 0, r->T, pd->plan.npanels, nb, ib, w, (int)sizeof(E),
                timed, nullptr, 0, 0, nullptr, nullptr, nullptr,
                (sizeof(E) == 8 && !r->tiles2) ? bd::kWindowF64BiDiag : 0);
  h->timed = timed;
  if (rc) return bail(rc);
  if (tiles2 && variant != BIDIAG_RBIDIAG) {
    // three-step: the band's first s tile rows come from the BiDiag steps on A, the rest from the R copy
    e = bd::launch_extract_split(tiles, r->p, tiles2, r->q, (int64_t)bd::split_of(variant) * nb, nb, n, ab, r->ldab,
                                 h->stream);
  } else {
    e = bd::launch_extract(tiles2 ? tiles2 : tiles, tiles2 ? r->q : r->p, nb, n, ab, r->ldab, h->stream);
  }
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "extract"));
  h->live.insert(r);
  *out = r;
  return BIDIAG_OK;
}


// Adjoint of a reduction: dL/dA from dL/dB (band storage) by the reverse sweep over the result's
// reflectors.  The working state starts as [B; 0] and the gradient as the band gradient, both tiled
// like A; after the sweep they hold the reconstruction of A and dL/dA.
// Adjoint program of a result (built and uploaded on first use, cached on its plan) and the sizes of
// one adjoint call's device workspace.
struct AdjointSizes {
  int hw = 0;            // column chunk of the update adjoints
  int red_ctas = 0;      // executor CTAs (each gets nb x ib elements of panel-adjoint scratch)
  int64_t bytes = 0;     // state + gradient tiles, partial-slot storage, panel-adjoint scratch
};

int adjoint_setup(bidiag_handle h, bidiag_result_t r, int esize, AdjointSizes* z) {
  const bd::Plan& pl = r->pd->plan;
  const int nb = r->nb, ib = r->ib;
  const int bi = esize == 8 ? 0 : 1;
  if (!r->pd->bwd[bi]) {
    auto bw = std::make_shared<BwdDev>();
    try {
      bd::build_backward(pl, bw->bp, esize == 8);
    } catch (const std::bad_alloc&) {
      return fail(h, BIDIAG_ERR_NOMEM, "host allocation failed while planning the adjoint");
    } catch (const std::exception& e) {
      return fail(h, BIDIAG_ERR_UNSUPPORTED, std::string("adjoint planner: ") + e.what());
    }
    int rc = upload_program(h, bw->prog, bw->bp.dev, bw->bp.deps, 1);
    if (rc) return rc;
    CK(h, cudaMalloc(&bw->d_slot_off, bw->bp.slot_off.size() * sizeof(int64_t)));
    CK(h, cudaMalloc(&bw->d_pinfo, bw->bp.pinfo.size() * sizeof(int32_t)));
    CK(h, cudaMemcpy(bw->d_slot_off, bw->bp.slot_off.data(), bw->bp.slot_off.size() * sizeof(int64_t),
                     cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(bw->d_pinfo, bw->bp.pinfo.data(), bw->bp.pinfo.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    r->pd->bwd[bi] = bw;
  }
  const BwdDev& bw = *r->pd->bwd[bi];
  z->hw = bd::choose_bwd_chunk(nb, ib, bw.bp.strip_w, h->smem_optin, esize);
  if (!z->hw) return fail(h, BIDIAG_ERR_UNSUPPORTED, "the adjoint of this tile size / inner blocking needs more shared memory");
  const size_t smem = bd::bwd_smem_bytes(nb, ib, z->hw, esize);
  CK(h, bd::exec_set_smem(smem, esize, true));
  z->red_ctas = h->nsm * std::max(1, bd::exec_max_ctas_per_sm(smem, esize, true));
  const int64_t tiles = (int64_t)r->p * r->q + (r->tiles2 ? (int64_t)r->q * r->q : 0);
  z->bytes = (int64_t)esize * (2 * tiles * nb * nb + std::max<int64_t>(1, bw.bp.slot_off.back()) +
                               (int64_t)z->red_ctas * nb * ib);
  return BIDIAG_OK;
}

template <typename E>
int backward_impl(bidiag_handle h, bidiag_result_t r, const E* d_abbar, int64_t ldab, E* d_Abar, int64_t ldabar,
                  E* d_Arec, int64_t ldarec) {
  if (!h) return -1;
  if (!r || !r->pd) return fail(h, -2, "result is NULL");
  if (r->h != h) return fail(h, -2, "result belongs to another handle");
  if (r->esize != (int)sizeof(E)) return fail(h, -2, "result has the other storage precision");
  if (!d_abbar) return fail(h, -3, "band gradient is NULL");
  if (ldab < r->nb + 1) return fail(h, -4, "ldab < nb + 1");
  if (!d_Abar) return fail(h, -5, "A_bar is NULL");
  if (ldabar < r->m) return fail(h, -6, "ldabar < m");
  if (d_Arec && ldarec < r->m) return fail(h, -8, "ldarec < m");
  CK(h, cudaSetDevice(h->device));
  const bd::Plan& pl = r->pd->plan;
  const int nb = r->nb, ib = r->ib, esize = (int)sizeof(E);
  AdjointSizes z{};
  int rc0 = adjoint_setup(h, r, esize, &z);
  if (rc0) return rc0;
  const BwdDev& bw = *r->pd->bwd[esize == 8 ? 0 : 1];
  const int hw = z.hw;
  // Working state and gradient, tiled like the forward's buffers: S / G mirror the A tiles (p x q);
  // for R-BiDiag, S2 / G2 mirror the R copy (q x q).  Start: the band lives in the last buffer the
  // forward wrote (A tiles for BiDiag, the R copy for R-BiDiag); for R-BiDiag the A tiles' state is the
  // pre-QR's R factor, which the forward leaves in the upper part of its tiles.
  const bool rb = r->tiles2 != nullptr;
  const int split = std::max(0, bd::split_of(r->variant));      // three-step: first-phase tile rows
  const int64_t srow = (int64_t)split * nb;
  const int64_t ntiles = (int64_t)r->p * r->q, ntiles2 = rb ? (int64_t)r->q * r->q : 0;
  const size_t tile_elems = (size_t)nb * nb;
  E *S = nullptr, *G = nullptr, *S2 = nullptr, *G2 = nullptr, *part = nullptr, *red = nullptr;
  int rc = dev_alloc(h, &S, (size_t)ntiles * tile_elems);
  if (!rc) rc = dev_alloc(h, &G, (size_t)ntiles * tile_elems);
  if (!rc && rb) rc = dev_alloc(h, &S2, (size_t)ntiles2 * tile_elems);
  if (!rc && rb) rc = dev_alloc(h, &G2, (size_t)ntiles2 * tile_elems);
  if (!rc) rc = dev_alloc(h, &part, (size_t)std::max<int64_t>(1, bw.bp.slot_off.back()));
  if (!rc) rc = dev_alloc(h, &red, (size_t)z.red_ctas * nb * ib);
  auto release = [&]() {
    for (E* x : {S, G, S2, G2, part, red})
      if (x) cudaFreeAsync(x, h->stream);
  };
  if (rc) {
    release();
    return rc;
  }
  // band rows [0, srow) belong to the A tiles (BiDiag, or the first phase of a three-step), the others
  // to the R copy; the A tiles of a two-phase reduction also hold the pre-QR's R factor (tiles from s on)
  const E* abE = static_cast<const E*>(r->ab);
  const int64_t arows = rb ? srow : r->n;
  cudaError_t e = cudaMemsetAsync(G, 0, (size_t)ntiles * tile_elems * esize, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, (size_t)ntiles * tile_elems * esize, h->stream);
  if (e == cudaSuccess && rb) e = cudaMemsetAsync(S2, 0, (size_t)ntiles2 * tile_elems * esize, h->stream);
  if (e == cudaSuccess && rb) e = cudaMemsetAsync(G2, 0, (size_t)ntiles2 * tile_elems * esize, h->stream);
  if (e == cudaSuccess && rb)
    e = bd::launch_r_part(static_cast<const E*>(r->tiles), S, r->p, r->q, nb, split, h->stream);
  if (e == cudaSuccess && arows > 0) e = bd::launch_scatter_band(abE, r->ldab, nb, r->n, S, r->p, 0, arows, h->stream);
  if (e == cudaSuccess && rb) e = bd::launch_scatter_band(abE, r->ldab, nb, r->n, S2, r->q, srow, r->n, h->stream);
  if (e == cudaSuccess && arows > 0) e = bd::launch_scatter_band(d_abbar, ldab, nb, r->n, G, r->p, 0, arows, h->stream);
  if (e == cudaSuccess && rb) e = bd::launch_scatter_band(d_abbar, ldab, nb, r->n, G2, r->q, srow, r->n, h->stream);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(h, e, "adjoint set-up");
  }
  const bool timed = h->timing != 0 || h->tracing != 0;
  if (timed && !h->ev[0]) {
    e = cudaEventCreate(&h->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev[1]);
    if (e != cudaSuccess) {
      release();
      return cuda_fail(h, e, "cudaEventCreate");
    }
  }
  bd::BwdParams bp{};
  bp.part = part;
  bp.slot_off = bw.d_slot_off;
  bp.nslots = (int32_t)(bw.bp.slot_off.size() - 1);
  bp.pinfo = bw.d_pinfo;
  bp.red = red;
  bp.red_ctas = z.red_ctas;
  bp.hw = hw;
  bp.pu_split = bw.bp.pu_split;
  const void* bx[3] = {S2, G, G2};
  const int64_t nx[3] = {ntiles2, ntiles, ntiles2};
  rc = run_exec(h, bw.prog, (int)bw.bp.dev.size(), r->tiles, ntiles, r->tiles2, ntiles2, S, ntiles, r->T, pl.npanels,
                nb, ib, bw.bp.strip_w, esize, timed, nullptr, 0, 0, bx, nx, &bp);
  h->timed = timed;
  if (rc) {
    release();
    return rc;
  }
  e = bd::launch_unpack(G, r->p, nb, r->m, r->n, d_Abar, ldabar, h->stream);
  if (e == cudaSuccess && d_Arec) e = bd::launch_unpack(S, r->p, nb, r->m, r->n, d_Arec, ldarec, h->stream);
  release();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint unpack");
  return BIDIAG_OK;
}

// Batched form: `count` independent reductions in one persistent launch.  Each matrix keeps its own
// plan (tile size, tree, variant); the device programs are merged by critical-path priority and every
// sub-task finds its matrix's offsets and tile size in a per-matrix table.
template <typename E>
int band_batched_impl(bidiag_handle h, int64_t count, const int64_t* m, const int64_t* n, const E* const* d_A,
                      const int64_t* lda, const int* nb_in, const int* ib_in, const int* tree_in, const int* var_in,
                      bidiag_result_t* out) {
  if (!h) return -1;
  if (count < 0) return fail(h, -2, "count < 0");
  if (count == 0) return BIDIAG_OK;
  if (!m || !n || !d_A || !lda) return fail(h, -3, "m, n, A and lda arrays are required");
  if (!out) return fail(h, -11, "out is NULL");
  CK(h, cudaSetDevice(h->device));
  const int esize = (int)sizeof(E);
  for (int64_t b = 0; b < count; ++b) {
    out[b] = nullptr;
    if (m[b] < 1 || n[b] < 1 || m[b] < n[b] || lda[b] < m[b] || !d_A[b])
      return fail(h, -3, "matrix " + std::to_string(b) + ": need m >= n >= 1, lda >= m and A != NULL");
  }
  // the batch program depends only on the shapes and options: look it up first
  std::vector<int64_t> key;
  key.reserve(6 * (size_t)count + 4);
  key.push_back(esize);
  key.push_back(h->strip_w);
  key.push_back(h->auto_res);
  key.push_back(h->prio);
  key.push_back(count);
  for (int64_t b = 0; b < count; ++b) {
    key.push_back(m[b]);
    key.push_back(n[b]);
    key.push_back(nb_in ? nb_in[b] : -1);
    key.push_back(ib_in ? ib_in[b] : -1);
    key.push_back(tree_in ? tree_in[b] : -1);
    key.push_back(var_in ? var_in[b] : -1);
  }
  std::shared_ptr<BatchPlan> bp;
  {
    auto it = h->batches.find(key);
    if (it != h->batches.end()) bp = it->second;
  }
  if (!bp) {
    bp = std::make_shared<BatchPlan>();
    auto& mats = bp->mats;
    mats.resize((size_t)count);
  // configuration (autotuned when nb is NULL) and plan of every matrix, in parallel on the host
  std::vector<int> bad((size_t)count, 0);   // 0 ok, else the error code of that matrix
  {
    const unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::atomic<int64_t> next(0);
    auto worker = [&]() {
      for (int64_t b = next++; b < count; b = next++) {
        BatchPlan::One& o = mats[(size_t)b];
        try {
          if (nb_in) {
            o.nb = nb_in[b];
            o.ib = ib_in ? ib_in[b] : std::min(o.nb, 32);
            o.tree = tree_in ? tree_in[b] : BIDIAG_AUTO;
            o.variant = var_in ? var_in[b] : BIDIAG_AUTO_VARIANT;
          } else {
            bd::autotune(m[b], n[b], h->nsm, esize, &o.nb, &o.ib, &o.tree, &o.variant);
            if (tree_in) o.tree = tree_in[b];
            if (var_in) o.variant = var_in[b];
          }
          if (o.nb < 1 || o.nb > bd::kMaxNb || o.ib < 1 || o.ib > std::min(o.nb, 64) || o.nb % o.ib) {
            bad[(size_t)b] = -7;
            continue;
          }
          if (o.tree < 0 || o.tree > 3 || o.variant < 0 || o.variant > 2) {   // no three-step in batches
            bad[(size_t)b] = -9;
            continue;
          }
          o.w = bd::choose_strip_width(o.nb, o.ib, h->strip_w > 0 ? h->strip_w : 32, h->smem_optin, esize);
          if (!o.w) {
            bad[(size_t)b] = BIDIAG_ERR_UNSUPPORTED;
            continue;
          }
          const int p = (int)((m[b] + o.nb - 1) / o.nb), q = (int)((n[b] + o.nb - 1) / o.nb);
          const int64_t R = resources_of(h, o.nb, o.w, esize);
          if (o.variant == BIDIAG_AUTO_VARIANT) o.variant = bd::choose_variant(p, q, o.tree, R, nullptr, nullptr);
          o.pd = std::make_shared<PlanDev>();
          bd::build_plan(o.pd->plan, m[b], n[b], o.nb, o.ib, o.tree, o.variant, R, o.w, esize, h->prio);
          dump_tasks(o.pd->plan.tasks, o.pd->dump);
        } catch (const std::bad_alloc&) {
          bad[(size_t)b] = BIDIAG_ERR_NOMEM;
        } catch (...) {
          bad[(size_t)b] = BIDIAG_ERR_UNSUPPORTED;
        }
      }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nthr && (int64_t)t < count; ++t) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
  }
  for (int64_t b = 0; b < count; ++b) {
    if (bad[(size_t)b]) {
      const int code = bad[(size_t)b];
      const char* what = code == -7 ? "invalid nb / ib" : code == -9 ? "invalid tree / variant"
                       : code == BIDIAG_ERR_NOMEM ? "host allocation failed" : "unsupported configuration";
      return fail(h, code, "matrix " + std::to_string(b) + ": " + what);
    }
    const BatchPlan::One& o = mats[(size_t)b];
    bp->smem = std::max(bp->smem, bd::exec_smem_bytes(o.nb, o.ib, o.w, esize));
  }
  // storage layout
  bp->info.resize((size_t)count);
  for (int64_t b = 0; b < count; ++b) {
    const bd::Plan& pl = mats[(size_t)b].pd->plan;
    bd::MatInfo& mi = bp->info[(size_t)b];
    const int64_t t2 = (int64_t)pl.nb * pl.nb;
    mi.off[0] = bp->tot0;
    mi.ntiles[0] = (int64_t)pl.p * pl.q;
    bp->tot0 += mi.ntiles[0] * t2;
    mi.off[1] = bp->tot1;
    mi.ntiles[1] = pl.variant == BIDIAG_RBIDIAG ? (int64_t)pl.q * pl.q : 0;
    bp->tot1 += mi.ntiles[1] * t2;
    mi.offT = bp->totT;
    bp->totT += (int64_t)std::max(1, pl.npanels) * pl.ib * pl.nb;
    mi.nb = pl.nb;
    mi.ib = pl.ib;
    mi.w = pl.strip_w;
    mi.npanels = pl.npanels;
    mi.pad = 0;
    bp->tiles_all += mi.ntiles[0];
    bp->cols_all += n[b];
  }
  std::vector<const bd::Plan*> plans;
  for (auto& o : mats) plans.push_back(&o.pd->plan);
  std::vector<bd::DevTask> dev;
  std::vector<int32_t> deps;
  try {
    bd::merge_programs(plans, &dev, &deps);
  } catch (const std::exception& ex) {
    return fail(h, BIDIAG_ERR_UNSUPPORTED, std::string("merge: ") + ex.what());
  }
  int rc0 = upload_program(h, bp->prog, dev, deps, 1);
  if (rc0) return rc0;
  bp->ntasks = (int)dev.size();
  CK(h, cudaMalloc(&bp->d_mats, sizeof(bd::MatInfo) * (size_t)count));
  CK(h, cudaMemcpy(bp->d_mats, bp->info.data(), sizeof(bd::MatInfo) * (size_t)count, cudaMemcpyHostToDevice));
  if (h->batches.size() >= 8) h->batches.clear();
  h->batches[key] = bp;
  }
  const auto& mats = bp->mats;
  const auto& info = bp->info;
  const int64_t tot0 = bp->tot0, tot1 = bp->tot1, totT = bp->totT, tiles_all = bp->tiles_all, cols_all = bp->cols_all;
  const size_t smem = bp->smem;
  auto store = std::make_shared<BatchStore>();
  store->plan = bp;
  int rc = 0;
  CK(h, cudaMalloc(&store->tiles, (size_t)std::max<int64_t>(1, tot0) * esize));
  if (tot1) CK(h, cudaMalloc(&store->tiles2, (size_t)tot1 * esize));
  CK(h, cudaMalloc(&store->T, (size_t)std::max<int64_t>(1, totT) * esize));
  CK(h, cudaMalloc(&store->d_desc, sizeof(bd::PackDesc) * 2 * (size_t)count));
  // results and their bands
  std::vector<bidiag_result*> res((size_t)count, nullptr);
  auto bail = [&](int code) {
    for (bidiag_result* r : res)
      if (r) {
        free_result_buffers(r);
        delete r;
      }
    return code;
  };
  std::vector<bd::PackDesc> pk((size_t)count), ex((size_t)count);
  int64_t first_tile = 0, first_col = 0;
  for (int64_t b = 0; b < count; ++b) {
    const bd::Plan& pl = mats[(size_t)b].pd->plan;
    bidiag_result* r = new (std::nothrow) bidiag_result();
    if (!r) return bail(fail(h, BIDIAG_ERR_NOMEM, "host allocation failed"));
    res[(size_t)b] = r;
    r->h = h;
    r->pd = mats[(size_t)b].pd;
    r->m = m[b];
    r->n = n[b];
    r->nb = pl.nb;
    r->ib = pl.ib;
    r->tree = pl.tree;
    r->variant = pl.variant;
    r->p = pl.p;
    r->q = pl.q;
    r->esize = esize;
    r->ldab = pl.nb + 1;
    r->store = store;
    r->tiles = static_cast<E*>(store->tiles) + info[(size_t)b].off[0];
    r->tiles2 = info[(size_t)b].ntiles[1] ? static_cast<E*>(store->tiles2) + info[(size_t)b].off[1] : nullptr;
    r->T = static_cast<E*>(store->T) + info[(size_t)b].offT;
    E* ab = nullptr;
    if ((rc = dev_alloc(h, &ab, (size_t)(pl.nb + 1) * n[b]))) return bail(rc);
    r->ab = ab;
    pk[(size_t)b] = bd::PackDesc{d_A[b], r->tiles, lda[b], m[b], n[b], (int64_t)pl.p, first_tile, pl.nb, 0};
    ex[(size_t)b] = bd::PackDesc{r->tiles2 ? r->tiles2 : r->tiles, ab, r->ldab, 0, n[b],
                                 (int64_t)(r->tiles2 ? pl.q : pl.p), first_col, pl.nb, 0};
    first_tile += (int64_t)pl.p * pl.q;
    first_col += n[b];
  }
  bd::PackDesc* d_pk = static_cast<bd::PackDesc*>(store->d_desc);
  bd::PackDesc* d_ex = d_pk + count;
  cudaError_t e = cudaMemcpyAsync(d_pk, pk.data(), sizeof(bd::PackDesc) * (size_t)count, cudaMemcpyHostToDevice,
                                  h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ex, ex.data(), sizeof(bd::PackDesc) * (size_t)count, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && tot1) e = cudaMemsetAsync(store->tiles2, 0, (size_t)tot1 * esize, h->stream);
  if (e == cudaSuccess) e = bd::launch_pack_batched(d_pk, (int)count, tiles_all, esize, h->stream);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "batched pack"));
  const bool timed = h->timing != 0 || h->tracing != 0;
  if (timed && !h->ev[0]) {
    e = cudaEventCreate(&h->ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev[1]);
    if (e != cudaSuccess) return bail(cuda_fail(h, e, "cudaEventCreate"));
  }
  rc = run_exec(h, bp->prog, bp->ntasks, store->tiles, tiles_all, store->tiles2, tot1 ? 1 : 0, nullptr, 0, store->T,
                0, 0, 1, 1, esize, timed, static_cast<const bd::MatInfo*>(bp->d_mats), (int)count, smem);
  if (rc) return bail(rc);
  h->timed = timed;
  e = bd::launch_extract_batched(d_ex, (int)count, cols_all, esize, h->stream);
  if (e != cudaSuccess) return bail(cuda_fail(h, e, "batched extract"));
  for (int64_t b = 0; b < count; ++b) {
    h->live.insert(res[(size_t)b]);
    out[b] = res[(size_t)b];
  }
  return BIDIAG_OK;
}

}  // namespace

extern "C" {

int bidiag_create(bidiag_handle* h, int device, void* cuda_stream) {
  if (!h) return -1;
  *h = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return -2;
  bidiag_ctx* c = new (std::nothrow) bidiag_ctx();
  if (!c) return BIDIAG_ERR_NOMEM;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, device);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_ctrl, 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(c->d_ctrl, 0, 4 * sizeof(int));
  if (e != cudaSuccess) {
    delete c;
    return e == cudaErrorMemoryAllocation ? BIDIAG_ERR_NOMEM : BIDIAG_ERR_CUDA;
  }
  c->smem_optin = (size_t)optin - 64;   // headroom for the executor's static shared memory
  if (const char* s = std::getenv("BIDIAG_WAIT_LIMIT_NS")) c->wait_ns = std::strtoull(s, nullptr, 10);
  if (const char* s = std::getenv("BIDIAG_AUTO_RES")) c->auto_res = std::atoll(s);
  *h = c;
  return BIDIAG_OK;
}

int bidiag_set_option(bidiag_handle h, int option, int64_t value) {
  if (!h) return -1;
  switch (option) {
    case BIDIAG_OPT_WAIT_LIMIT_NS:
      if (value <= 0) return -3;
      h->wait_ns = (uint64_t)value;
      return BIDIAG_OK;
    case BIDIAG_OPT_AUTO_RESOURCES:
      if (value < 0) return -3;
      h->auto_res = value;
      return BIDIAG_OK;
    case BIDIAG_OPT_DEBUG_UNSET_DEP:
      h->debug_unset = value != 0;
      return BIDIAG_OK;
    case BIDIAG_OPT_STRIP:
      if (value != 16 && value != 32 && value != 64) return -3;
      h->strip_w = (int)value;
      return BIDIAG_OK;
    case BIDIAG_OPT_TIMING:
      h->timing = value != 0;
      return BIDIAG_OK;
    case BIDIAG_OPT_TRACE:
      h->tracing = value != 0;
      return BIDIAG_OK;
    case BIDIAG_OPT_F32_UPDATES:
      if (value < 0 || value > 2) return -3;
      h->f32_simt = (int)value;
      return BIDIAG_OK;
    case BIDIAG_OPT_F32_SCALARS:
      if (value != 0 && value != 1) return -3;
      h->f32_scalars64 = (int)value;
      return BIDIAG_OK;
    case BIDIAG_OPT_WINDOW:
      if (value < -1 || value > 1024) return -3;
      h->window = (int)value;
      return BIDIAG_OK;
    case BIDIAG_OPT_PRIORITY:
      if (value != 0 && value != 1) return -3;
      h->prio = (int)value;
      return BIDIAG_OK;
    default:
      return -2;
  }
}

int bidiag_band(bidiag_handle h, int64_t m, int64_t n, const double* d_A, int64_t lda, int nb, int ib, int tree,
                int variant, bidiag_result_t* out) {
  return band_impl(h, m, n, d_A, lda, nb, ib, tree, variant, out);
}

int bidiag_band_f32(bidiag_handle h, int64_t m, int64_t n, const float* d_A, int64_t lda, int nb, int ib, int tree,
                    int variant, bidiag_result_t* out) {
  return band_impl(h, m, n, d_A, lda, nb, ib, tree, variant, out);
}

int bidiag_band_batched(bidiag_handle h, int64_t count, const int64_t* m, const int64_t* n, const double* const* d_A,
                        const int64_t* lda, const int* nb, const int* ib, const int* tree, const int* variant,
                        bidiag_result_t* out) {
  return band_batched_impl(h, count, m, n, d_A, lda, nb, ib, tree, variant, out);
}

int bidiag_band_batched_f32(bidiag_handle h, int64_t count, const int64_t* m, const int64_t* n,
                            const float* const* d_A, const int64_t* lda, const int* nb, const int* ib, const int* tree,
                            const int* variant, bidiag_result_t* out) {
  return band_batched_impl(h, count, m, n, d_A, lda, nb, ib, tree, variant, out);
}

int bidiag_autotune(int64_t m, int64_t n, int nsm, int elem_bytes, int* nb, int* ib, int* tree, int* variant) {
  if (m < 1 || n < 1 || m < n) return -1;
  if (nsm < 1) return -3;
  if (elem_bytes != 4 && elem_bytes != 8) return -4;
  if (!nb || !ib || !tree || !variant) return -5;
  try {
    bd::autotune(m, n, nsm, elem_bytes, nb, ib, tree, variant);
  } catch (...) {
    return BIDIAG_ERR_NOMEM;
  }
  return BIDIAG_OK;
}

int bidiag_band_host(bidiag_handle h, int64_t m, int64_t n, const double* h_A, int64_t lda, int nb, int ib, int tree,
                     int variant, double* h_ab, int64_t ldab, bidiag_result_t* out) {
  if (!h) return -1;
  if (out) *out = nullptr;
  if (!h_A) return fail(h, -4, "A is NULL");
  if (lda < m) return fail(h, -5, "lda < m");
  if (!h_ab) return fail(h, -11, "ab is NULL");
  if (ldab < nb + 1) return fail(h, -12, "ldab < nb + 1");
  if (m < 1) return fail(h, -2, "m < 1");
  if (n < 1) return fail(h, -3, "n < 1");
  CK(h, cudaSetDevice(h->device));
  double* dA = nullptr;
  int rc = dev_alloc(h, &dA, (size_t)lda * n);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(dA, h_A, sizeof(double) * (size_t)lda * n, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    cudaFreeAsync(dA, h->stream);
    return cuda_fail(h, e, "copy A to device");
  }
  bidiag_result_t r = nullptr;
  rc = bidiag_band(h, m, n, dA, lda, nb, ib, tree, variant, &r);
  cudaFreeAsync(dA, h->stream);
  if (rc) return rc;
  e = cudaMemcpy2DAsync(h_ab, sizeof(double) * ldab, r->ab, sizeof(double) * r->ldab, sizeof(double) * (nb + 1), n,
                        cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) {
    bidiag_result_free(r);
    return cuda_fail(h, e, "copy band to host");
  }
  rc = bidiag_sync(h);
  if (rc || !out) {
    bidiag_result_free(r);
    return rc;
  }
  *out = r;
  return BIDIAG_OK;
}

int bidiag_result_band(bidiag_result_t r, const double** ab, int64_t* ldab, int64_t* n, int* nb) {
  if (!r) return -1;
  if (r->esize != 8) return BIDIAG_ERR_UNSUPPORTED;
  if (ab) *ab = static_cast<const double*>(r->ab);
  if (ldab) *ldab = r->ldab;
  if (n) *n = r->n;
  if (nb) *nb = r->nb;
  return BIDIAG_OK;
}

int bidiag_result_band_f32(bidiag_result_t r, const float** ab, int64_t* ldab, int64_t* n, int* nb) {
  if (!r) return -1;
  if (r->esize != 4) return BIDIAG_ERR_UNSUPPORTED;
  if (ab) *ab = static_cast<const float*>(r->ab);
  if (ldab) *ldab = r->ldab;
  if (n) *n = r->n;
  if (nb) *nb = r->nb;
  return BIDIAG_OK;
}

int bidiag_result_tasks(bidiag_result_t r, const int32_t** tasks, int64_t* ntasks) {
  if (!r) return -1;
  if (tasks) *tasks = r->pd->dump.data();
  if (ntasks) *ntasks = (int64_t)r->pd->plan.tasks.size();
  return BIDIAG_OK;
}

int bidiag_result_reflectors(bidiag_result_t r, bidiag_reflectors* desc) {
  if (!r) return -1;
  if (!desc) return -2;
  desc->tiles = r->tiles;
  desc->tiles2 = r->tiles2;
  desc->T = r->T;
  desc->elem_bytes = r->esize;
  desc->tree = r->tree;
  desc->tslot = r->pd->plan.tslot.data();
  desc->ntasks = (int64_t)r->pd->plan.tasks.size();
  desc->m = r->m;
  desc->n = r->n;
  desc->nb = r->nb;
  desc->ib = r->ib;
  desc->p = r->p;
  desc->q = r->q;
  desc->npanels = r->pd->plan.npanels;
  desc->variant = r->variant;
  return BIDIAG_OK;
}

int bidiag_apply_q(bidiag_handle h, bidiag_result_t r, int trans, int64_t ncols, double* d_C, int64_t ldc) {
  if (!h) return -1;
  if (!r) return fail(h, -2, "result is NULL");
  if (r->h != h) return fail(h, -2, "result was made on another handle or its handle was destroyed");
  if (r->esize != 8) return fail(h, -2, "FP32 result: use bidiag_apply_q_f32");
  if (trans != 0 && trans != 1) return fail(h, -3, "trans must be 0 or 1");
  if (ncols < 0) return fail(h, -4, "ncols < 0");
  if (!d_C && ncols > 0) return fail(h, -5, "C is NULL");
  if (ldc < r->m) return fail(h, -6, "ldc < m");
  CK(h, cudaSetDevice(h->device));
  return apply_side(h, r, true, trans, ncols, d_C, ldc);
}

int bidiag_apply_q_f32(bidiag_handle h, bidiag_result_t r, int trans, int64_t ncols, float* d_C, int64_t ldc) {
  if (!h) return -1;
  if (!r) return fail(h, -2, "result is NULL");
  if (r->h != h) return fail(h, -2, "result was made on another handle or its handle was destroyed");
  if (r->esize != 4) return fail(h, -2, "FP64 result: use bidiag_apply_q");
  if (trans != 0 && trans != 1) return fail(h, -3, "trans must be 0 or 1");
  if (ncols < 0) return fail(h, -4, "ncols < 0");
  if (!d_C && ncols > 0) return fail(h, -5, "C is NULL");
  if (ldc < r->m) return fail(h, -6, "ldc < m");
  CK(h, cudaSetDevice(h->device));
  return apply_side(h, r, true, trans, ncols, d_C, ldc);
}

int bidiag_band_backward(bidiag_handle h, bidiag_result_t r, const double* d_abbar, int64_t ldab, double* d_Abar,
                         int64_t ldabar, double* d_Arec, int64_t ldarec) {
  return backward_impl<double>(h, r, d_abbar, ldab, d_Abar, ldabar, d_Arec, ldarec);
}

int bidiag_band_backward_f32(bidiag_handle h, bidiag_result_t r, const float* d_abbar, int64_t ldab, float* d_Abar,
                             int64_t ldabar, float* d_Arec, int64_t ldarec) {
  return backward_impl<float>(h, r, d_abbar, ldab, d_Abar, ldabar, d_Arec, ldarec);
}

int bidiag_apply_p(bidiag_handle h, bidiag_result_t r, int trans, int64_t nrows, double* d_C, int64_t ldc) {
  if (!h) return -1;
  if (!r) return fail(h, -2, "result is NULL");
  if (r->h != h) return fail(h, -2, "result was made on another handle or its handle was destroyed");
  if (r->esize != 8) return fail(h, -2, "FP32 result: use bidiag_apply_p_f32");
  if (trans != 0 && trans != 1) return fail(h, -3, "trans must be 0 or 1");
  if (nrows < 0) return fail(h, -4, "nrows < 0");
  if (!d_C && nrows > 0) return fail(h, -5, "C is NULL");
  if (ldc < std::max<int64_t>(1, nrows)) return fail(h, -6, "ldc < nrows");
  CK(h, cudaSetDevice(h->device));
  return apply_side(h, r, false, trans, nrows, d_C, ldc);
}

int bidiag_apply_p_f32(bidiag_handle h, bidiag_result_t r, int trans, int64_t nrows, float* d_C, int64_t ldc) {
  if (!h) return -1;
  if (!r) return fail(h, -2, "result is NULL");
  if (r->h != h) return fail(h, -2, "result was made on another handle or its handle was destroyed");
  if (r->esize != 4) return fail(h, -2, "FP64 result: use bidiag_apply_p");
  if (trans != 0 && trans != 1) return fail(h, -3, "trans must be 0 or 1");
  if (nrows < 0) return fail(h, -4, "nrows < 0");
  if (!d_C && nrows > 0) return fail(h, -5, "C is NULL");
  if (ldc < std::max<int64_t>(1, nrows)) return fail(h, -6, "ldc < nrows");
  CK(h, cudaSetDevice(h->device));
  return apply_side(h, r, false, trans, nrows, d_C, ldc);
}

int bidiag_sync(bidiag_handle h) {
  if (!h) return -1;
  CK(h, cudaSetDevice(h->device));
  CK(h, cudaStreamSynchronize(h->stream));
  int err[3] = {0, 0, 0};
  CK(h, cudaMemcpy(err, h->d_ctrl + 1, sizeof(err), cudaMemcpyDeviceToHost));
  if (err[0] != bd::DERR_OK) {
    CK(h, cudaMemset(h->d_ctrl + 1, 0, sizeof(err)));
    if (err[0] == bd::DERR_TIMEOUT)
      return fail(h, BIDIAG_ERR_TIMEOUT, "device dependency wait ran out at queue position " +
                                             std::to_string(err[1]) + " waiting for " + std::to_string(err[2]));
    return fail(h, BIDIAG_ERR_CUDA, "executor rejected an invalid task at queue position " + std::to_string(err[1]));
  }
  h->err.clear();
  return BIDIAG_OK;
}

int bidiag_last_exec_ms(bidiag_handle h, float* ms) {
  if (!h) return -1;
  if (!ms) return -2;
  if (!h->timed || !h->ev[0]) return fail(h, BIDIAG_ERR_UNSUPPORTED, "timing was off for the last reduction");
  CK(h, cudaEventElapsedTime(ms, h->ev[0], h->ev[1]));
  return BIDIAG_OK;
}

int bidiag_backward_workspace(bidiag_handle h, bidiag_result_t r, int64_t* bytes) {
  if (!h) return -1;
  if (!r || !r->pd) return fail(h, -2, "result is NULL");
  if (r->h != h) return fail(h, -2, "result belongs to another handle");
  if (!bytes) return -3;
  CK(h, cudaSetDevice(h->device));
  AdjointSizes z{};
  const int rc = adjoint_setup(h, r, r->esize, &z);
  if (rc) return rc;
  *bytes = z.bytes;
  return BIDIAG_OK;
}

int bidiag_trace_program(bidiag_handle h, int32_t* program, int64_t cap, int64_t* count, int32_t* deps, int64_t dcap,
                         int64_t* ndeps) {
  if (!h) return -1;
  if (!count) return -4;
  if (!ndeps) return -7;
  *count = (int64_t)h->trace_dev.size();
  *ndeps = (int64_t)h->trace_deps.size();
  if (h->trace_dev.empty()) return fail(h, BIDIAG_ERR_UNSUPPORTED, "no traced reduction");
  if (program && cap >= *count) std::memcpy(program, h->trace_dev.data(), sizeof(bd::DevTask) * (size_t)*count);
  if (deps && dcap >= *ndeps && *ndeps) std::memcpy(deps, h->trace_deps.data(), sizeof(int32_t) * (size_t)*ndeps);
  return BIDIAG_OK;
}

int bidiag_trace(bidiag_handle h, int64_t* out, int64_t cap, int64_t* count) {
  if (!h) return -1;
  if (!count) return -4;
  *count = h->trace_len;
  if (!h->d_trace || !h->trace_len) return fail(h, BIDIAG_ERR_UNSUPPORTED, "no traced reduction");
  if (out && cap >= h->trace_len)
    CK(h, cudaMemcpy(out, h->d_trace, sizeof(int64_t) * 4 * (size_t)h->trace_len, cudaMemcpyDeviceToHost));
  return BIDIAG_OK;
}

const char* bidiag_last_error(bidiag_handle h) { return h ? h->err.c_str() : "null handle"; }

int bidiag_result_free(bidiag_result_t r) {
  if (!r) return -1;
  if (r->h) {
    cudaSetDevice(r->h->device);
    r->h->live.erase(r);
    free_result_buffers(r);
  }
  delete r;
  return BIDIAG_OK;
}

int bidiag_destroy(bidiag_handle h) {
  if (!h) return -1;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  // results still alive lose their buffers now; freeing them later only releases the host object
  for (bidiag_result* r : h->live) {
    free_result_buffers(r);
    r->h = nullptr;
  }
  h->live.clear();
  cudaStreamSynchronize(h->stream);
  h->cache.clear();
  if (h->d_ctrl) cudaFree(h->d_ctrl);
  if (h->d_trace) cudaFree(h->d_trace);
  if (h->ev[0]) cudaEventDestroy(h->ev[0]);
  if (h->ev[1]) cudaEventDestroy(h->ev[1]);
  delete h;
  return BIDIAG_OK;
}

int bidiag_plan_eliminations(int64_t p, int64_t q, int tree, int variant, int64_t resources, int32_t* out, int64_t cap,
                             int64_t* count) {
  if (p < 1 || q < 1 || q > p) return -1;
  if (tree < 0 || tree > 3) return -3;
  if (variant < 0 || variant == 2 || variant == 3 || variant - BIDIAG_THREESTEP_SPLIT(0) >= q) return -4;
  if (!count) return -8;
  try {
    auto el = bd::make_eliminations((int)p, (int)q, tree, variant, resources);
    *count = (int64_t)el.size();
    if (out && cap >= (int64_t)el.size()) {
      for (size_t x = 0; x < el.size(); ++x) {
        out[5 * x + 0] = el[x].phase; out[5 * x + 1] = el[x].k; out[5 * x + 2] = el[x].i;
        out[5 * x + 3] = el[x].piv; out[5 * x + 4] = el[x].kind;
      }
    }
  } catch (...) {
    return BIDIAG_ERR_NOMEM;
  }
  return BIDIAG_OK;
}

int bidiag_plan_tasks(int64_t p, int64_t q, int tree, int variant, int64_t resources, int32_t* tasks, int32_t* level,
                      int64_t cap, int64_t* count, int64_t* cp) {
  if (p < 1 || q < 1 || q > p) return -1;
  if (tree < 0 || tree > 3) return -3;
  if (variant < 0 || variant == 2 || variant == 3 || variant - BIDIAG_THREESTEP_SPLIT(0) >= q) return -4;
  if (!count) return -9;
  try {
    auto ts = bd::make_tasks((int)p, (int)q, tree, variant, resources);
    *count = (int64_t)ts.size();
    const bool fits = cap >= (int64_t)ts.size();
    if (level || cp) {
      std::vector<int32_t> lv;
      int64_t c = 0;
      bd::make_dag(ts, (int)p, (int)q, variant, nullptr, &lv, &c);
      if (cp) *cp = c;
      if (level && fits) std::copy(lv.begin(), lv.end(), level);
    }
    if (tasks && fits) {
      std::vector<int32_t> d;
      dump_tasks(ts, d);
      std::copy(d.begin(), d.end(), tasks);
    }
  } catch (...) {
    return BIDIAG_ERR_NOMEM;
  }
  return BIDIAG_OK;
}

int bidiag_plan_choose_variant(int64_t p, int64_t q, int tree, int64_t resources, int* variant, int64_t* cp_bidiag,
                               int64_t* cp_rbidiag) {
  if (p < 1 || q < 1 || q > p) return -1;
  if (tree < 0 || tree > 3) return -3;
  if (!variant) return -5;
  try {
    *variant = bd::choose_variant((int)p, (int)q, tree, resources, cp_bidiag, cp_rbidiag);
  } catch (...) {
    return BIDIAG_ERR_NOMEM;
  }
  return BIDIAG_OK;
}

int bidiag_plan_best_split(int64_t p, int64_t q, int tree, int64_t resources, int* split, int64_t* cp) {
  if (q < 1 || p < q) return -1;
  if (tree < 0 || tree > 3) return -3;
  if (!split) return -5;
  try {
    *split = bd::best_split((int)p, (int)q, tree, resources, cp);
  } catch (const std::bad_alloc&) {
    return BIDIAG_ERR_NOMEM;
  } catch (...) {
    return BIDIAG_ERR_UNSUPPORTED;
  }
  return BIDIAG_OK;
}

int bidiag_plan_program(int64_t m, int64_t n, int nb, int ib, int tree, int variant, int64_t resources, int strip_w,
                        int32_t* program, int64_t cap, int64_t* count, int32_t* deps, int64_t dcap, int64_t* ndeps,
                        int32_t* strip_w_used) {
  if (m < 1 || n < 1 || m < n) return -1;
  if (nb < 1 || nb > bd::kMaxNb) return -3;
  if (ib < 1 || nb % ib) return -4;
  if (tree < 0 || tree > 3) return -5;
  if (variant < 0 || variant == 2 || variant == 3 || variant - BIDIAG_THREESTEP_SPLIT(0) >= (n + nb - 1) / nb)
    return -6;
  if (!count || !ndeps) return -9;
  int w = std::max(ib, (strip_w / ib) * ib);
  w = std::min(w, nb);
  try {
    bd::Plan pl;
    bd::build_plan(pl, m, n, nb, ib, tree, variant, resources, w);
    *count = (int64_t)pl.dev.size();
    *ndeps = (int64_t)pl.deps.size();
    if (strip_w_used) *strip_w_used = pl.strip_w;
    if (program && cap >= *count) std::memcpy(program, pl.dev.data(), pl.dev.size() * sizeof(bd::DevTask));
    if (deps && dcap >= *ndeps) std::memcpy(deps, pl.deps.data(), pl.deps.size() * sizeof(int32_t));
  } catch (const std::bad_alloc&) {
    return BIDIAG_ERR_NOMEM;
  } catch (...) {
    return BIDIAG_ERR_UNSUPPORTED;
  }
  return BIDIAG_OK;
}

int bidiag_plan_backward(int64_t m, int64_t n, int nb, int ib, int tree, int variant, int64_t resources, int strip_w,
                         int32_t* program, int32_t* fwd, int64_t cap, int64_t* count, int32_t* deps, int64_t dcap,
                         int64_t* ndeps, int64_t* slot_off, int64_t scap, int64_t* nslot_off, int32_t* pinfo,
                         int64_t pcap, int64_t* npinfo, int32_t* strip_w_used) {
  if (m < 1 || n < 1 || m < n) return -1;
  if (nb < 1 || nb > bd::kMaxNb) return -3;
  if (ib < 1 || nb % ib) return -4;
  if (tree < 0 || tree > 3) return -5;
  if (variant < 0 || variant == 2 || variant == 3 || variant - BIDIAG_THREESTEP_SPLIT(0) >= (n + nb - 1) / nb)
    return -6;
  if (!count || !ndeps || !nslot_off || !npinfo) return -10;
  int w = std::max(ib, (strip_w / ib) * ib);
  w = std::min(w, nb);
  try {
    bd::Plan pl;
    bd::build_plan(pl, m, n, nb, ib, tree, variant, resources, w);
    bd::BwdPlan bp;
    bd::build_backward(pl, bp);
    *count = (int64_t)bp.dev.size();
    *ndeps = (int64_t)bp.deps.size();
    *nslot_off = (int64_t)bp.slot_off.size();
    *npinfo = (int64_t)bp.pinfo.size();
    if (strip_w_used) *strip_w_used = bp.strip_w;
    if (program && cap >= *count) std::memcpy(program, bp.dev.data(), bp.dev.size() * sizeof(bd::DevTask));
    if (fwd && cap >= *count) std::memcpy(fwd, bp.fwd.data(), bp.fwd.size() * sizeof(int32_t));
    if (deps && dcap >= *ndeps) std::memcpy(deps, bp.deps.data(), bp.deps.size() * sizeof(int32_t));
    if (slot_off && scap >= *nslot_off) std::memcpy(slot_off, bp.slot_off.data(), bp.slot_off.size() * sizeof(int64_t));
    if (pinfo && pcap >= *npinfo) std::memcpy(pinfo, bp.pinfo.data(), bp.pinfo.size() * sizeof(int32_t));
  } catch (const std::bad_alloc&) {
    return BIDIAG_ERR_NOMEM;
  } catch (...) {
    return BIDIAG_ERR_UNSUPPORTED;
  }
  return BIDIAG_OK;
}

}  // extern "C"
