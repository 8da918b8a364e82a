// Host planner of the tiled BiDiag / R-BiDiag reduction: reduction trees -> canonical task list ->
// task DAG -> device sub-tasks in a topological priority order for the persistent executor.
#pragma once
#include <cstdint>
#include <vector>

namespace bd {

enum TaskType : int { GEQRT = 0, UNMQR = 1, TSQRT = 2, TSMQR = 3, TTQRT = 4, TTMQR = 5, COPY = 6 };
// Device-only sub-task types: factor one inner block of a panel (PF), apply it to a later column block
// of the panel (PU).  Their op word carries the panel kind (0 GE, 1 TS, 2 TT) in bits 24-25.
enum SubType : int { PF = 7, PU = 8 };
// Sub-tasks of the adjoint program (reverse sweep): BPF / BPU undo PF / PU, BUPD undoes an update strip
// (kind bits 24-25: 0 UNMQR, 1 TSMQR, 2 TTMQR), BCOPY undoes a COPY (adds the gradient of the copied
// part of an R tile to the pre-QR tile it was copied from).
enum BwdType : int { BPF = 9, BPU = 10, BUPD = 11, BCOPY = 12, BRED = 13 };
// BRED: sums, in slot order, the update-strip partials of one block of a panel task over a chunk of
// kRedElems / ib rows (strip field = chunk index, blk = block, kind = panel kind) into the panel's
// reduced slot, so that the factor sub-task of the block reads one slot instead of all of them.
// Panels with fewer than kRedMinSlots update strips keep the direct sum.
constexpr int kRedElems = 2048;
constexpr int kRedMinSlots = 8;
enum Phase : int { PH_QR = 0, PH_LQ = 1, PH_PQR = 2 };
enum Tree : int { FLATTS = 0, FLATTT = 1, GREEDY = 2, AUTO = 3 };
enum Variant : int { V_BIDIAG = 0, V_RBIDIAG = 1 };
// Three-step (Sec. 4.5) with split s: s BiDiag steps on A, then R-BiDiag on the trailing tiles.
// Encoded as variant V_THREESTEP + s; R-BiDiag is the split s = 0.
constexpr int V_THREESTEP = 4;
// Number of BiDiag steps before the switch to R-BiDiag (-1 for BiDiag: no second phase).
inline int split_of(int variant) { return variant == V_BIDIAG ? -1 : (variant == V_RBIDIAG ? 0 : variant - V_THREESTEP); }
// Matrix a task works on: 0 = A, 1 = the R copy of the second phase (its LQ steps k >= s and QR steps
// k >= s + 1; QR(s) belongs to the pre-QR).
inline int task_buffer(int phase, int k, int variant) {
  const int s = split_of(variant);
  if (s < 0 || phase == 2) return 0;
  return ((phase == 1 && k >= s) || (phase == 0 && k > s)) ? 1 : 0;
}
enum Kind : int { K_TS = 0, K_TT = 1 };

struct Task {
  int type, phase, k, i, piv, j;
};
struct Elim {
  int phase, k, i, piv, kind;
};

// One unit of work of the persistent executor (32 bytes).  Tile references pack a buffer id in the
// top 4 bits and the tile index (column-major tile grid of that buffer) in the low 28 bits.
struct DevTask {
  int32_t op;        // type | tr << 4 | notrans << 5 | strip << 8 | block << 16 | kind << 24
  int32_t x;         // reflector / panel tile (COPY: source tile)
  int32_t a;         // pivot tile (TS/TT panels) or top C tile (TSMQR/TTMQR)
  int32_t c;         // C tile of UNMQR / bottom C tile of TSMQR, TTMQR (COPY: destination tile)
  int32_t tslot;     // T slot of the panel task
  int32_t dep_begin; // deps in [dep_begin, dep_end) of the dependency array
  int32_t dep_end;
  int32_t flags;     // bit 0: diagonal COPY (upper triangle only); bits 8-31: matrix of a batch
};

inline int32_t tile_ref(int buf, int64_t idx) { return (int32_t)(((uint32_t)buf << 28) | (uint32_t)idx); }

struct Plan {
  int64_t m = 0, n = 0;
  int nb = 0, ib = 0, tree = 0, variant = 0, p = 0, q = 0, strip_w = 32, nstrips = 1;
  int64_t resources = 0;
  std::vector<Elim> elims;
  std::vector<Task> tasks;
  std::vector<int32_t> level;
  std::vector<int32_t> tslot;      // per task
  std::vector<int32_t> owner;      // per update task: panel task index
  int npanels = 0;
  int64_t critical_path = 0;       // Table 1 units
  // device program
  std::vector<DevTask> dev;        // in queue (priority) order
  std::vector<int32_t> deps;       // indices into dev (queue positions)
  std::vector<int64_t> prio;       // bottom level of each queued sub-task (flop-proportional weights)
};

// Adjoint program of a plan (the reverse sweep).  Sub-task y of the forward program becomes its
// adjoint; every dependency is reversed, priorities are the bottom levels of the reversed DAG.  Tile
// references: x = reflector tile of the forward result (buffers 0 / 1 as in the forward program),
// a / c = working-state tiles: buffer 2 mirrors the forward's tile buffer 0 (p x q grid), buffer 3 its
// R copy (q x q, R-BiDiag); the gradients are buffers 4 and 5 with the same indices.  BCOPY: x = the
// pre-QR state tile, c = the R state tile, flags bit 0 = diagonal tile.  Update sub-tasks write their
// contributions to the reflectors' derivatives into partial slots (flags = slot index); the factor
// sub-task of a block sums them, or reads their sum from the panel's reduced slot (pinfo[3] >= 0),
// written by the BRED sub-tasks of the block.
struct BwdPlan {
  std::vector<DevTask> dev;
  std::vector<int32_t> deps;
  std::vector<int64_t> slot_off;   // element offset of each partial slot; last entry = total elements
  std::vector<int32_t> pinfo;      // per panel task (T slot): first update slot, number, first PU slot,
                                   // reduced slot (-1: none)
  std::vector<int32_t> fwd;        // forward queue position of each adjoint sub-task
  int strip_w = 0;                 // column width of the adjoint update strips
  int pu_split = 1;                // BPU sub-tasks per panel-block update (column pieces of ib / pu_split)
};
// split_strips: undo each update strip of >= 16 columns as two column halves with a partial slot each
// (shorter critical path; worth it when the arithmetic dominates, FP64, not with FP32 storage).  Panel-
// block updates with ib >= 16 are always undone as two halves (bit 5 of op, notrans, = the half).
void build_backward(const Plan& pl, BwdPlan& bp, bool split_strips = true);

// Trees and task lists (independent of any device state).
std::vector<Elim> make_eliminations(int p, int q, int tree, int variant, int64_t resources);
std::vector<Task> make_tasks(int p, int q, int tree, int variant, int64_t resources);
// Task DAG: predecessor lists, levels and the Table 1 critical path.
void make_dag(const std::vector<Task>& tasks, int p, int q, int variant,
              std::vector<std::vector<int32_t>>* preds, std::vector<int32_t>* level, int64_t* cp);
// Variant with the shorter critical path (Sec. 4.3.3: BiDiag for square-ish, R-BiDiag for tall
// matrices, switching at p/q = delta_s).  The Auto tree is compared through Greedy, whose critical path
// the paper studies (Auto's has no meaning without a resource model).  Ties keep BiDiag.
int choose_variant(int p, int q, int tree, int64_t resources, int64_t* cp_bidiag, int64_t* cp_rbidiag);
// Sec. 4.5: the three-step split with the shortest critical path, trying every s in [0, q) (ties keep
// the smallest s); returns s and, if cp is not null, its critical path.
int best_split(int p, int q, int tree, int64_t resources, int64_t* cp);
// Full plan for a reduction: tasks, DAG, device sub-tasks ordered by critical-path priority.  esize
// (8: FP64, 4: FP32 storage) and prio (1: calibrated per-kind times, 0: flop counts) only set the
// priority weights.
void build_plan(Plan& pl, int64_t m, int64_t n, int nb, int ib, int tree, int variant, int64_t resources,
                int strip_w, int esize = 8, int prio = 1);

// Several independent plans as one device program: the queues are merged by decreasing bottom level
// (each plan's own order is kept, so the result is topological), matrix b's sub-tasks carry b in
// flags bits 8-31 and their dependencies are renumbered to the merged queue.
void merge_programs(const std::vector<const Plan*>& plans, std::vector<DevTask>* dev, std::vector<int32_t>* deps);

// Tile size, inner blocking, tree and variant for one m x n matrix of a batch (the batched form's
// autotuner), for FP64 (esize 8) or FP32 (esize 4) storage: a search over the calibrated (nb, ib) pairs
// (nb in {32, 64, 128}, ib in {8, 16, 32}) and the FlatTS, Greedy and Auto trees, minimising the
// calibrated busy time of the matrix's sub-tasks (plus its critical path over nsm / 8); the variant by
// critical path.  Falls back to a Table 1 work model when the table has no row for the precision.
void autotune(int64_t m, int64_t n, int nsm, int esize, int* nb, int* ib, int* tree, int* variant);

}  // namespace bd
