// Host planner: reduction trees, canonical task lists and the task DAG of tiled BiDiag / R-BiDiag,
// and the device program (sub-tasks + dependencies in a topological priority order).
//
// Trees (Sec. 3.3 and Sec. 5 of Faverge, Langou, Robert, Dongarra, arXiv 1611.06892):
//  * FlatTS / FlatTT: the pivot is the first panel tile; every other tile is eliminated into it in
//    order, with TS (Algorithm 2) or TT (Algorithm 3) kernels.
//  * Greedy: halving rule - with ready rows r_0 < ... < r_{z-1} and h = floor(z/2), r_{z-h+t} is
//    eliminated into r_{z-2h+t}; repeated on the survivors (depth ceil(log2 z), Sec. 4).  For the
//    multi-column QR(p,q) of R-BiDiag it is time-stepped: at time s the rows ready in column k are
//    those eliminated in column k-1 at a time < s (all rows for k = 0) and not yet eliminated in k.
//  * Auto (Sec. 5): FlatTS groups of a consecutive tiles, heads joined by the halving Greedy rule with
//    TT kernels; a is the largest value in [1, u] with ceil(u/a) * v >= 2 * R (else 1), u and v being
//    the live numbers of panel tiles and trailing tiles of the step.
// Sequences: BiDiag QR(1); LQ(1); ...; LQ(q-1); QR(q) (Sec. 3.4); R-BiDiag QR(p,q); LQ(1); QR(2); ...
// on a separate copy of R (Sec. 3.5 and 3.6).  A tile already in triangle form is not factored again
// (end of Sec. 3.2).
#include "plan.h"

#include <algorithm>
#include <cstdio>
#include <deque>
#include <functional>
#include <map>
#include <stdexcept>

namespace bd {

namespace {

struct Pair {
  int i, piv;
};

// Halving Greedy: list of rounds of (eliminated, pivot).
std::vector<std::vector<Pair>> halving_rounds(std::vector<int> rows) {
  std::vector<std::vector<Pair>> rounds;
  while (rows.size() > 1) {
    const int z = (int)rows.size(), h = z / 2;
    std::vector<Pair> rnd;
    std::vector<char> gone(z, 0);
    for (int t = 0; t < h; ++t) {
      rnd.push_back({rows[z - h + t], rows[z - 2 * h + t]});
      gone[z - h + t] = 1;
    }
    std::vector<int> keep;
    for (int x = 0; x < z; ++x)
      if (!gone[x]) keep.push_back(rows[x]);
    rows.swap(keep);
    rounds.push_back(rnd);
  }
  return rounds;
}

int auto_a(int u, int v, int64_t R) {
  for (int a = u; a >= 1; --a) {
    const int64_t groups = (u + a - 1) / a;
    if (groups * (int64_t)v >= 2 * R) return a;
  }
  return 1;
}

struct El {
  int i, piv, kind;
};

std::vector<El> one_step(const std::vector<int>& rows, int v, int tree, int64_t R) {
  std::vector<El> out;
  if (rows.size() < 2) return out;
  if (tree == FLATTS || tree == FLATTT) {
    for (size_t x = 1; x < rows.size(); ++x) out.push_back({rows[x], rows[0], tree == FLATTS ? K_TS : K_TT});
  } else if (tree == GREEDY) {
    for (auto& rnd : halving_rounds(rows))
      for (auto& pr : rnd) out.push_back({pr.i, pr.piv, K_TT});
  } else if (tree == AUTO) {
    const int u = (int)rows.size();
    const int a = auto_a(u, v, R);
    std::vector<int> heads;
    for (int s = 0; s < u; s += a) {
      heads.push_back(rows[s]);
      for (int x = s + 1; x < std::min(u, s + a); ++x) out.push_back({rows[x], rows[s], K_TS});
    }
    for (auto& rnd : halving_rounds(heads))
      for (auto& pr : rnd) out.push_back({pr.i, pr.piv, K_TT});
  } else {
    throw std::invalid_argument("tree");
  }
  return out;
}

// Time-stepped greedy over all columns of QR(p, q): (k, i, piv) in (time, column) order.
struct CEl {
  int k, i, piv;
};
std::vector<CEl> greedy_columns(int p, int q) {
  const int kmax = std::min(p, q);
  std::vector<int> t_elim((size_t)p * kmax, -1);  // time at which row i was eliminated in column k
  auto T = [&](int i, int k) -> int& { return t_elim[(size_t)k * p + i]; };
  std::vector<int> remaining(kmax);
  int total = 0;
  for (int k = 0; k < kmax; ++k) total += (remaining[k] = p - 1 - k);
  std::vector<CEl> out;
  for (int s = 0; total > 0; ++s) {
    for (int k = 0; k < kmax; ++k) {
      if (!remaining[k]) continue;
      std::vector<int> ready;
      for (int i = k; i < p; ++i) {
        if (T(i, k) >= 0) continue;
        if (k == 0 || (T(i, k - 1) >= 0 && T(i, k - 1) < s)) ready.push_back(i);
      }
      const int z = (int)ready.size(), h = z / 2;
      for (int t = 0; t < h; ++t) {
        const int i = ready[z - h + t], piv = ready[z - 2 * h + t];
        T(i, k) = s;
        out.push_back({k, i, piv});
        --remaining[k];
        --total;
      }
    }
  }
  return out;
}

struct Step {
  int phase, k;
  std::vector<int> rows;
  int ntrail;
};

// Steps of the first phase (BiDiag on A: all of them for BiDiag, the first s for a split s) and of
// the second (BiDiag of the trailing R after the pre-QR).
void steps_of(int p, int q, int variant, std::vector<Step>* first, std::vector<Step>* second) {
  auto range = [](int a, int b) {
    std::vector<int> r;
    for (int x = a; x < b; ++x) r.push_back(x);
    return r;
  };
  const int s = split_of(variant);
  if (s >= q || s < -1) throw std::invalid_argument("three-step split must be in [0, q)");
  first->clear();
  second->clear();
  for (int k = 0; k < (s < 0 ? q : s); ++k) {
    first->push_back({PH_QR, k, range(k, p), q - k - 1});
    if (k < q - 1) first->push_back({PH_LQ, k, range(k + 1, q), p - k - 1});
  }
  if (s >= 0) {
    for (int k = s; k + 1 < q; ++k) {
      second->push_back({PH_LQ, k, range(k + 1, q), q - k - 1});
      second->push_back({PH_QR, k + 1, range(k + 1, q), q - k - 2});
    }
  }
}

// Eliminations of the pre-QR of tiles s..p-1 x s..q-1 in program order.
std::vector<Elim> preqr_eliminations(int p, int q, int s, int tree, int64_t R) {
  std::vector<Elim> out;
  if (tree == GREEDY) {
    for (auto& e : greedy_columns(p - s, q - s)) out.push_back({PH_PQR, e.k + s, e.i + s, e.piv + s, K_TT});
  } else {
    for (int k = s; k < q; ++k) {
      std::vector<int> rows;
      for (int r = k; r < p; ++r) rows.push_back(r);
      for (auto& e : one_step(rows, q - k - 1, tree, R)) out.push_back({PH_PQR, k, e.i, e.piv, e.kind});
    }
  }
  return out;
}

// Expansion of eliminations into kernel tasks (Algorithms 2 and 3).
struct Expander {
  std::vector<Task>& out;
  std::vector<char> tri;  // (phase, k, row) already triangular
  int p;
  Expander(std::vector<Task>& o, int p_) : out(o), tri((size_t)3 * (p_ + 1) * (p_ + 1), 0), p(p_) {}
  char& flag(int phase, int k, int r) { return tri[((size_t)phase * (p + 1) + k) * (p + 1) + r]; }
  bool factor(int phase, int k, int r) {
    if (flag(phase, k, r)) return false;
    flag(phase, k, r) = 1;
    out.push_back({GEQRT, phase, k, r, -1, -1});
    return true;
  }
  void elim(int phase, int k, const El& e, int ntrail) {
    if (e.kind == K_TS) {
      const bool fp = factor(phase, k, e.piv);
      out.push_back({TSQRT, phase, k, e.i, e.piv, -1});
      for (int j = k + 1; j <= k + ntrail; ++j) {
        if (fp) out.push_back({UNMQR, phase, k, e.piv, -1, j});
        out.push_back({TSMQR, phase, k, e.i, e.piv, j});
      }
    } else {
      const bool fp = factor(phase, k, e.piv);
      const bool fi = factor(phase, k, e.i);
      for (int j = k + 1; j <= k + ntrail; ++j) {
        if (fp) out.push_back({UNMQR, phase, k, e.piv, -1, j});
        if (fi) out.push_back({UNMQR, phase, k, e.i, -1, j});
      }
      out.push_back({TTQRT, phase, k, e.i, e.piv, -1});
      for (int j = k + 1; j <= k + ntrail; ++j) out.push_back({TTMQR, phase, k, e.i, e.piv, j});
    }
  }
  void single(int phase, int k, int row, int ntrail) {
    if (!factor(phase, k, row)) return;
    for (int j = k + 1; j <= k + ntrail; ++j) out.push_back({UNMQR, phase, k, row, -1, j});
  }
};

}  // namespace

std::vector<Elim> make_eliminations(int p, int q, int tree, int variant, int64_t R) {
  std::vector<Elim> out;
  std::vector<Step> first, second;
  steps_of(p, q, variant, &first, &second);
  for (auto& st : first)
    for (auto& e : one_step(st.rows, st.ntrail, tree, R)) out.push_back({st.phase, st.k, e.i, e.piv, e.kind});
  const int s = split_of(variant);
  if (s >= 0)
    for (auto& e : preqr_eliminations(p, q, s, tree, R)) out.push_back(e);
  for (auto& st : second)
    for (auto& e : one_step(st.rows, st.ntrail, tree, R)) out.push_back({st.phase, st.k, e.i, e.piv, e.kind});
  return out;
}

std::vector<Task> make_tasks(int p, int q, int tree, int variant, int64_t R) {
  if (!(p >= q && q >= 1)) throw std::invalid_argument("need p >= q >= 1");
  std::vector<Task> tasks;
  Expander ex(tasks, p);
  std::vector<Step> first, second;
  steps_of(p, q, variant, &first, &second);
  auto run = [&](const std::vector<Step>& steps) {
    for (auto& st : steps) {
      auto el = one_step(st.rows, st.ntrail, tree, R);
      if (el.empty()) ex.single(st.phase, st.k, st.rows[0], st.ntrail);
      for (auto& e : el) ex.elim(st.phase, st.k, e, st.ntrail);
    }
  };
  run(first);
  const int s = split_of(variant);
  if (s >= 0) {
    if (tree == GREEDY) {
      std::vector<char> seen(q, 0);
      for (auto& e : preqr_eliminations(p, q, s, tree, R)) {
        ex.elim(PH_PQR, e.k, {e.i, e.piv, K_TT}, q - e.k - 1);
        seen[e.k] = 1;
      }
      for (int k = s; k < q; ++k)
        if (!seen[k]) ex.single(PH_PQR, k, k, q - k - 1);
    } else {
      for (int k = s; k < q; ++k) {
        std::vector<int> rows;
        for (int r = k; r < p; ++r) rows.push_back(r);
        auto el = one_step(rows, q - k - 1, tree, R);
        if (el.empty()) ex.single(PH_PQR, k, k, q - k - 1);
        for (auto& e : el) ex.elim(PH_PQR, k, e, q - k - 1);
      }
    }
    for (int a = s; a < q; ++a)
      for (int b = a; b < q; ++b) tasks.push_back({COPY, PH_PQR, -1, a, -1, b});
  }
  run(second);
  return tasks;
}

// ---------------------------------------------------------------------------------------------
// Task DAG.  Data items: strict upper (SU), diagonal (D) and strict lower (SL) part of every tile of
// A (buffer 0) and of the R copy (buffer 1), plus the reflector object (V, T) of each panel task.
// Edges: read-after-write, write-after-write, write-after-read.
// ---------------------------------------------------------------------------------------------
namespace {
enum Part { SU = 0, D = 1, SL = 2 };

struct Access {
  int rd[6], nrd = 0;
  int wr[9], nwr = 0;
};

struct ItemMap {
  int p, q;
  int id(int buf, int a, int b, int part) const { return ((buf * q + b) * p + a) * 3 + part; }
  int size() const { return 2 * q * p * 3; }
};

Access access_of(const Task& t, int variant, const ItemMap& im) {
  Access ac;
  const int buf = task_buffer(t.phase, t.k, variant);
  const bool lq = t.phase == PH_LQ;
  auto put = [&](int* arr, int& n, int a, int b, int part) {
    const int x = lq ? b : a, y = lq ? a : b;
    arr[n++] = im.id(buf, x, y, part);
  };
  auto up = [&](int* arr, int& n, int a, int b) {
    put(arr, n, a, b, D);
    put(arr, n, a, b, lq ? SL : SU);  // oriented strict upper
  };
  auto lo = [&](int* arr, int& n, int a, int b) { put(arr, n, a, b, lq ? SU : SL); };
  auto full = [&](int* arr, int& n, int a, int b) {
    put(arr, n, a, b, SU);
    put(arr, n, a, b, D);
    put(arr, n, a, b, SL);
  };
  switch (t.type) {
    case GEQRT: full(ac.wr, ac.nwr, t.i, t.k); break;
    case UNMQR: lo(ac.rd, ac.nrd, t.i, t.k); full(ac.wr, ac.nwr, t.i, t.j); break;
    case TSQRT: up(ac.wr, ac.nwr, t.piv, t.k); full(ac.wr, ac.nwr, t.i, t.k); break;
    case TSMQR: full(ac.rd, ac.nrd, t.i, t.k); full(ac.wr, ac.nwr, t.piv, t.j); full(ac.wr, ac.nwr, t.i, t.j); break;
    case TTQRT: up(ac.wr, ac.nwr, t.piv, t.k); up(ac.wr, ac.nwr, t.i, t.k); break;
    case TTMQR: up(ac.rd, ac.nrd, t.i, t.k); full(ac.wr, ac.nwr, t.piv, t.j); full(ac.wr, ac.nwr, t.i, t.j); break;
    case COPY: {
      const int a = t.i, b = t.j;
      if (a == b) {
        ac.rd[ac.nrd++] = im.id(0, a, a, D);
        ac.rd[ac.nrd++] = im.id(0, a, a, SU);
      } else {
        for (int part = 0; part < 3; ++part) ac.rd[ac.nrd++] = im.id(0, a, b, part);
      }
      for (int part = 0; part < 3; ++part) ac.wr[ac.nwr++] = im.id(1, a, b, part);
      break;
    }
    default: throw std::invalid_argument("task type");
  }
  return ac;
}

const int kWeight[7] = {4, 6, 6, 12, 2, 6, 0};  // Table 1
}  // namespace

void make_dag(const std::vector<Task>& tasks, int p, int q, int variant, std::vector<std::vector<int32_t>>* preds,
              std::vector<int32_t>* level, int64_t* cp) {
  ItemMap im{p, q};
  std::vector<int32_t> last_w(im.size(), -1);
  std::vector<std::vector<int32_t>> readers(im.size());
  // owner panel of each update (reflector object)
  std::vector<int32_t> owner(tasks.size(), -1);
  {
    // key (type, phase, k, i) -> last panel index
    std::vector<int32_t> last_panel((size_t)3 * 3 * (q + 1) * (p + 1), -1);
    auto key = [&](int ptype, int phase, int k, int i) {
      return (((size_t)ptype * 3 + phase) * (q + 1) + k) * (p + 1) + i;
    };
    for (size_t x = 0; x < tasks.size(); ++x) {
      const Task& t = tasks[x];
      switch (t.type) {
        case GEQRT: last_panel[key(0, t.phase, t.k, t.i)] = (int32_t)x; break;
        case TSQRT: last_panel[key(1, t.phase, t.k, t.i)] = (int32_t)x; break;
        case TTQRT: last_panel[key(2, t.phase, t.k, t.i)] = (int32_t)x; break;
        case UNMQR: owner[x] = last_panel[key(0, t.phase, t.k, t.i)]; break;
        case TSMQR: owner[x] = last_panel[key(1, t.phase, t.k, t.i)]; break;
        case TTMQR: owner[x] = last_panel[key(2, t.phase, t.k, t.i)]; break;
        default: break;
      }
    }
  }
  std::vector<int32_t> lv(tasks.size(), 0);
  std::vector<int64_t> fin(tasks.size(), 0);
  if (preds) preds->assign(tasks.size(), {});
  int64_t best = 0;
  std::vector<int32_t> pr;
  for (size_t x = 0; x < tasks.size(); ++x) {
    const Access ac = access_of(tasks[x], variant, im);
    pr.clear();
    for (int r = 0; r < ac.nrd; ++r)
      if (last_w[ac.rd[r]] >= 0) pr.push_back(last_w[ac.rd[r]]);
    for (int w = 0; w < ac.nwr; ++w) {
      if (last_w[ac.wr[w]] >= 0) pr.push_back(last_w[ac.wr[w]]);
      for (int32_t rr : readers[ac.wr[w]]) pr.push_back(rr);
    }
    if (owner[x] >= 0) pr.push_back(owner[x]);
    std::sort(pr.begin(), pr.end());
    pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
    int32_t l = 0;
    int64_t f = 0;
    for (int32_t d : pr) {
      if (d == (int32_t)x) continue;
      l = std::max(l, lv[d] + 1);
      f = std::max(f, fin[d]);
    }
    lv[x] = l;
    fin[x] = f + kWeight[tasks[x].type];
    best = std::max(best, fin[x]);
    if (preds) (*preds)[x] = pr;
    for (int r = 0; r < ac.nrd; ++r) readers[ac.rd[r]].push_back((int32_t)x);
    for (int w = 0; w < ac.nwr; ++w) {
      last_w[ac.wr[w]] = (int32_t)x;
      readers[ac.wr[w]].clear();
    }
  }
  if (level) *level = lv;
  if (cp) *cp = best;
}

int choose_variant(int p, int q, int tree, int64_t R, int64_t* cp_bidiag, int64_t* cp_rbidiag) {
  const int t = tree == AUTO ? GREEDY : tree;
  int64_t cb = 0, cr = 0;
  make_dag(make_tasks(p, q, t, V_BIDIAG, R), p, q, V_BIDIAG, nullptr, nullptr, &cb);
  make_dag(make_tasks(p, q, t, V_RBIDIAG, R), p, q, V_RBIDIAG, nullptr, nullptr, &cr);
  if (cp_bidiag) *cp_bidiag = cb;
  if (cp_rbidiag) *cp_rbidiag = cr;
  return cr < cb ? V_RBIDIAG : V_BIDIAG;
}

int best_split(int p, int q, int tree, int64_t R, int64_t* cp) {
  int best = 0;
  int64_t best_cp = -1;
  for (int s = 0; s < q; ++s) {
    int64_t c = 0;
    make_dag(make_tasks(p, q, tree, V_THREESTEP + s, R), p, q, V_THREESTEP + s, nullptr, nullptr, &c);
    if (best_cp < 0 || c < best_cp) {
      best_cp = c;
      best = s;
    }
  }
  if (cp) *cp = best_cp;
  return best;
}

// ---------------------------------------------------------------------------------------------
// Device program.
//  * A panel task (GEQRT / TSQRT / TTQRT) becomes, for each inner block b of ib reflectors, a factor
//    sub-task PF(b) on column block b, followed by update sub-tasks PU(b, s) that apply block b to the
//    later column blocks s of the panel (and of the pivot's top rows for TS / TT).  Block b + 1 can be
//    factored as soon as PU(b, b + 1) is done (look-ahead inside the tile), and consecutive eliminations
//    into the same pivot overlap block by block.
//  * An update task (UNMQR / TSMQR / TTMQR) becomes one sub-task per column strip of w columns (w a
//    multiple of ib) of its C tiles.
// Dependencies come from the data each sub-task reads and writes, tracked per ib x ib block of every
// tile (a diagonal block is split into its strict upper part, diagonal and strict lower part) and per
// T block: read-after-write, write-after-write and write-after-read.  An update strip depends on the
// last sub-task of its panel task for the reflectors it applies (the panel's sub-tasks are chained, and
// a factored region is never written again).  Sub-tasks are queued by decreasing bottom level (longest
// weighted path to the end), a topological order since every weight is positive.
// ---------------------------------------------------------------------------------------------
namespace {

struct Items {
  int p = 0, q = 0, nblk = 0;
  int64_t per_tile = 0, tbase = 0;
  int64_t tile(int buf, int x, int y) const { return (((int64_t)buf * q + y) * p + x) * per_tile; }
  int64_t blk(int buf, int x, int y, int bi, int bj) const { return tile(buf, x, y) + (int64_t)bi * nblk + bj; }
  int64_t dsu(int buf, int x, int y, int b) const { return tile(buf, x, y) + (int64_t)nblk * nblk + 2 * b; }
  int64_t dsl(int buf, int x, int y, int b) const { return dsu(buf, x, y, b) + 1; }
  int64_t t(int slot, int b) const { return tbase + (int64_t)slot * nblk + b; }
  int64_t size(int npanels) const { return tbase + (int64_t)npanels * nblk; }
};

// Item sets of an oriented tile (oa, ob) of buffer `buf` in a step of orientation lq.
struct OTile {
  const Items* it;
  int buf, x, y;
  bool lq;
  OTile(const Items* i, int b, int oa, int ob, bool l) : it(i), buf(b), x(l ? ob : oa), y(l ? oa : ob), lq(l) {}
  void full(std::vector<int64_t>& v, int br, int bc) const {
    if (br != bc) {
      v.push_back(lq ? it->blk(buf, x, y, bc, br) : it->blk(buf, x, y, br, bc));
    } else {
      v.push_back(it->blk(buf, x, y, br, br));
      v.push_back(it->dsu(buf, x, y, br));
      v.push_back(it->dsl(buf, x, y, br));
    }
  }
  void up(std::vector<int64_t>& v, int b) const {   // oriented diagonal + strict upper of block (b, b)
    v.push_back(it->blk(buf, x, y, b, b));
    v.push_back(lq ? it->dsl(buf, x, y, b) : it->dsu(buf, x, y, b));
  }
  void lo(std::vector<int64_t>& v, int b) const {   // oriented strict lower of block (b, b)
    v.push_back(lq ? it->dsu(buf, x, y, b) : it->dsl(buf, x, y, b));
  }
};

enum PanelKind : int { PK_GE = 0, PK_TS = 1, PK_TT = 2 };

struct SubDag {
  std::vector<int32_t> last_w;
  std::vector<std::vector<int32_t>> readers;
  std::vector<DevTask> sub;
  std::vector<int64_t> weight;
  std::vector<std::vector<int32_t>> deps;
  std::vector<int32_t> tmp;

  explicit SubDag(int64_t nitems) : last_w(nitems, -1), readers(nitems) {}

  int32_t add(const DevTask& d, int64_t w, const std::vector<int64_t>& rd, const std::vector<int64_t>& wr,
              int32_t extra_dep) {
    const int32_t me = (int32_t)sub.size();
    tmp.clear();
    for (int64_t i : rd)
      if (last_w[i] >= 0) tmp.push_back(last_w[i]);
    for (int64_t i : wr) {
      if (last_w[i] >= 0) tmp.push_back(last_w[i]);
      for (int32_t r : readers[i]) tmp.push_back(r);
    }
    if (extra_dep >= 0) tmp.push_back(extra_dep);
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    for (int64_t i : rd) readers[i].push_back(me);
    for (int64_t i : wr) {
      last_w[i] = me;
      readers[i].clear();
    }
    sub.push_back(d);
    weight.push_back(w > 0 ? w : 1);
    deps.push_back(tmp);
    return me;
  }
};

inline int32_t make_op(int type, bool tr, bool notrans, int strip, int blk, int kind) {
  return type | ((tr ? 1 : 0) << 4) | ((notrans ? 1 : 0) << 5) | (strip << 8) | (blk << 16) | (kind << 24);
}

}  // namespace

// Priority weight of a sub-task: its Table 1 flops times the time per flop of its kind relative to a
// TSMQR strip, in percent (mode 1), measured from per-sub-task traces of the executor on a GB300 (nb 256,
// ib 32; FP32 storage at 8192^2 with the tcgen05 updates, FP64 at 4096^2).  Mode 0 is the flop count
// alone, with FP32-storage panel factors counted twice.
enum WeightClass { W_PF_GE, W_PF_TS, W_PF_TT, W_PU_GE, W_PU_TS, W_PU_TT, W_UNMQR, W_TSMQR, W_TTMQR };
static int64_t prio_weight(int64_t flops, int cls, int esize, int mode) {
  static const int64_t kF32[9] = {640, 400, 650, 125, 115, 210, 135, 100, 150};
  static const int64_t kF64[9] = {71, 51, 74, 71, 70, 79, 117, 100, 119};
  if (mode == 0) return (cls <= W_PF_TT && esize == 4 ? 2 : 1) * flops;
  return std::max<int64_t>(1, flops * (esize == 4 ? kF32[cls] : kF64[cls]) / 100);
}

void build_plan(Plan& pl, int64_t m, int64_t n, int nb, int ib, int tree, int variant, int64_t R, int strip_w,
                int esize, int prio) {
  pl.m = m;
  pl.n = n;
  pl.nb = nb;
  pl.ib = ib;
  pl.tree = tree;
  pl.variant = variant;
  pl.resources = R;
  pl.p = (int)((m + nb - 1) / nb);
  pl.q = (int)((n + nb - 1) / nb);
  pl.strip_w = std::min(strip_w, nb);
  pl.nstrips = (nb + pl.strip_w - 1) / pl.strip_w;
  if (pl.strip_w % ib) throw std::invalid_argument("strip width must be a multiple of ib");
  const int p = pl.p, q = pl.q, S = pl.nstrips, w = pl.strip_w, nblk = nb / ib;
  if (S > 255 || nblk > 255) throw std::invalid_argument("too many strips or inner blocks");
  pl.elims = make_eliminations(p, q, tree, variant, R);
  pl.tasks = make_tasks(p, q, tree, variant, R);
  make_dag(pl.tasks, p, q, variant, nullptr, &pl.level, &pl.critical_path);
  const size_t nt = pl.tasks.size();

  // T slots and the panel task whose reflectors each update applies
  pl.tslot.assign(nt, -1);
  pl.owner.assign(nt, -1);
  pl.npanels = 0;
  {
    std::vector<int32_t> lastp((size_t)3 * 3 * (q + 1) * (p + 1), -1);
    auto key = [&](int ptype, int phase, int k, int i) {
      return (((size_t)ptype * 3 + phase) * (q + 1) + k) * (p + 1) + i;
    };
    for (size_t x = 0; x < nt; ++x) {
      const Task& t = pl.tasks[x];
      if (t.type == GEQRT || t.type == TSQRT || t.type == TTQRT) pl.tslot[x] = pl.npanels++;
      if (t.type == GEQRT) lastp[key(0, t.phase, t.k, t.i)] = (int32_t)x;
      if (t.type == TSQRT) lastp[key(1, t.phase, t.k, t.i)] = (int32_t)x;
      if (t.type == TTQRT) lastp[key(2, t.phase, t.k, t.i)] = (int32_t)x;
      if (t.type == UNMQR) pl.owner[x] = lastp[key(0, t.phase, t.k, t.i)];
      if (t.type == TSMQR) pl.owner[x] = lastp[key(1, t.phase, t.k, t.i)];
      if (t.type == TTMQR) pl.owner[x] = lastp[key(2, t.phase, t.k, t.i)];
    }
  }

  Items it;
  it.p = p;
  it.q = q;
  it.nblk = nblk;
  it.per_tile = (int64_t)nblk * nblk + 2 * nblk;
  it.tbase = 2 * (int64_t)q * p * it.per_tile;
  SubDag g(it.size(pl.npanels));
  std::vector<int32_t> panel_last(nt, -1);   // last sub-task of each panel task
  std::vector<int64_t> rd, wr;
  const int64_t ib2 = (int64_t)ib * ib;

  auto tref = [&](int buf, int oa, int ob, bool lq) {
    const int x = lq ? ob : oa, y = lq ? oa : ob;
    const int rows = buf == 0 ? p : q;
    return tile_ref(buf, (int64_t)y * rows + x);
  };

  for (size_t x = 0; x < nt; ++x) {
    const Task& t = pl.tasks[x];
    const int buf = task_buffer(t.phase, t.k, variant);
    const bool lq = t.phase == PH_LQ;
    if (t.type == GEQRT || t.type == TSQRT || t.type == TTQRT) {
      const int kind = t.type == GEQRT ? PK_GE : (t.type == TSQRT ? PK_TS : PK_TT);
      const OTile X(&it, buf, t.i, t.k, lq);
      const OTile A(&it, buf, kind == PK_GE ? t.i : t.piv, t.k, lq);
      const int slot = pl.tslot[x];
      DevTask d{};
      d.x = tref(buf, t.i, t.k, lq);
      d.a = kind == PK_GE ? -1 : tref(buf, t.piv, t.k, lq);
      d.c = -1;
      d.tslot = slot;
      int32_t last = -1;
      for (int b = 0; b < nblk; ++b) {
        // PF(b)
        rd.clear();
        wr.clear();
        if (kind == PK_GE) {
          X.full(wr, b, b);
          for (int br = b + 1; br < nblk; ++br) X.full(wr, br, b);
        } else if (kind == PK_TS) {
          A.up(wr, b);
          for (int br = 0; br < nblk; ++br) X.full(wr, br, b);
        } else {
          A.up(wr, b);
          for (int br = 0; br < b; ++br) X.full(wr, br, b);
          X.up(wr, b);
        }
        wr.push_back(it.t(slot, b));
        const int64_t rows = kind == PK_GE ? nb - (int64_t)b * ib : (kind == PK_TS ? nb : (int64_t)(b + 1) * ib);
        d.op = make_op(PF, lq, false, 0, b, kind);
        last = g.add(d, prio_weight(12 * ib2 * rows, W_PF_GE + kind, esize, prio), rd, wr, -1);
        // PU(b, s)
        for (int s = b + 1; s < nblk; ++s) {
          rd.clear();
          wr.clear();
          if (kind == PK_GE) {
            X.lo(rd, b);
            for (int br = b + 1; br < nblk; ++br) X.full(rd, br, b);
            for (int br = b; br < nblk; ++br) X.full(wr, br, s);
          } else if (kind == PK_TS) {
            for (int br = 0; br < nblk; ++br) X.full(rd, br, b);
            A.full(wr, b, s);
            for (int br = 0; br < nblk; ++br) X.full(wr, br, s);
          } else {
            for (int br = 0; br < b; ++br) X.full(rd, br, b);
            X.up(rd, b);
            A.full(wr, b, s);
            for (int br = 0; br <= b; ++br) X.full(wr, br, s);
          }
          rd.push_back(it.t(slot, b));
          d.op = make_op(PU, lq, false, s, b, kind);
          last = g.add(d, prio_weight(6 * ib2 * rows, W_PU_GE + kind, esize, prio), rd, wr, -1);
        }
      }
      panel_last[x] = last;
    } else if (t.type == UNMQR || t.type == TSMQR || t.type == TTMQR) {
      const int owner = pl.owner[x];
      DevTask d{};
      d.x = tref(buf, t.i, t.k, lq);
      d.a = t.type == UNMQR ? -1 : tref(buf, t.piv, t.j, lq);
      d.c = tref(buf, t.i, t.j, lq);
      d.tslot = pl.tslot[owner];
      const OTile C(&it, buf, t.i, t.j, lq);
      const OTile Cp(&it, buf, t.type == UNMQR ? t.i : t.piv, t.j, lq);
      const int64_t per_strip = (t.type == TSMQR ? 4 : 2) * (int64_t)nb * nb * w;
      for (int s = 0; s < S; ++s) {
        rd.clear();
        wr.clear();
        const int cb0 = s * (w / ib), cb1 = std::min(nblk, (s + 1) * (w / ib));
        for (int cb = cb0; cb < cb1; ++cb) {
          for (int br = 0; br < nblk; ++br) {
            C.full(wr, br, cb);
            if (t.type != UNMQR) Cp.full(wr, br, cb);
          }
        }
        d.op = make_op(t.type, lq, false, s, 0, 0);
        g.add(d, prio_weight(per_strip, t.type == UNMQR ? W_UNMQR : (t.type == TSMQR ? W_TSMQR : W_TTMQR), esize, prio),
              rd, wr, panel_last[owner]);
      }
    } else {   // COPY(i, j): R part of A's tile (i, j) into the second phase's tile (i, j)
      DevTask d{};
      d.x = tile_ref(0, (int64_t)t.j * p + t.i);
      d.a = -1;
      d.c = tile_ref(1, (int64_t)t.j * q + t.i);
      d.tslot = -1;
      d.flags = t.i == t.j ? 1 : 0;
      d.op = make_op(COPY, false, false, 0, 0, 0);
      rd.clear();
      wr.clear();
      const OTile src(&it, 0, t.i, t.j, false), dst(&it, 1, t.i, t.j, false);
      for (int br = 0; br < nblk; ++br) {
        for (int bc = 0; bc < nblk; ++bc) {
          dst.full(wr, br, bc);
          if (t.i < t.j) src.full(rd, br, bc);
          else if (br < bc) src.full(rd, br, bc);
          else if (br == bc) src.up(rd, br);
        }
      }
      g.add(d, (int64_t)nb * nb, rd, wr, -1);
    }
  }

  // bottom levels (sub-task numbering is a topological order: dependencies point backwards)
  const int32_t nsub = (int32_t)g.sub.size();
  std::vector<int64_t> bottom(nsub, 0);
  for (int32_t y = nsub - 1; y >= 0; --y) {
    bottom[y] += g.weight[y];
    for (int32_t dd : g.deps[y]) bottom[dd] = std::max(bottom[dd], bottom[y]);
  }
  std::vector<int32_t> order(nsub);
  for (int32_t y = 0; y < nsub; ++y) order[y] = y;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return bottom[a] > bottom[b]; });
  std::vector<int32_t> pos(nsub);
  for (int32_t y = 0; y < nsub; ++y) pos[order[y]] = y;
  pl.dev.resize(nsub);
  pl.deps.clear();
  pl.prio.resize(nsub);
  for (int32_t y = 0; y < nsub; ++y) {
    pl.prio[y] = bottom[order[y]];
    DevTask e = g.sub[order[y]];
    e.dep_begin = (int32_t)pl.deps.size();
    for (int32_t dd : g.deps[order[y]]) {
      if (pos[dd] >= y) throw std::logic_error("priority order is not topological");
      pl.deps.push_back(pos[dd]);
    }
    e.dep_end = (int32_t)pl.deps.size();
    pl.dev[y] = e;
  }
}

// ---------------------------------------------------------------------------------------------
// Adjoint program.  The reverse sweep undoes the forward sub-tasks in an order compatible with the
// reversed DAG: a sub-task's adjoint reads the state and gradient its forward counterpart wrote and
// writes those its counterpart read, so every forward hazard edge, reversed, orders the adjoints.  The
// derivatives of the reflectors of panel block b are sums over every column block the block was
// applied to: each BUPD strip (all blocks of its panel task) and each BPU(b, s) writes its part into a
// partial slot of its own, and BPF(b) -- which depends on all of them through the reversed edges
// (update strip -> last sub-task of its panel; PU(b, s) -> PF(b)) -- sums the slots in a fixed order.
// Slot layout: an update strip's slot holds, for every block beta, a nb x ib block (rows of the
// reflector tails) then an ib x ib block per beta; a PU slot holds the two blocks of its one block.
// ---------------------------------------------------------------------------------------------
void build_backward(const Plan& pl, BwdPlan& bp, bool split_strips) {
  const int nb = pl.nb, ib = pl.ib, nblk = nb / ib;
  const int32_t nsub = (int32_t)pl.dev.size();
  // An update strip's adjoint has three times its flops; with split_strips it is undone as two column
  // halves (each with its own partial slot) when the strip is at least 16 wide, which halves its
  // latency on the critical path.
  const int w = pl.strip_w, split = (split_strips && w >= 16 && w % 2 == 0) ? 2 : 1, wb = w / split;
  bp.strip_w = wb;
  const int pus = (ib >= 16 && ib % 2 == 0) ? 2 : 1;   // BPU column pieces (both storage precisions)
  bp.pu_split = pus;
  auto state_ref = [&](int32_t ref) -> int32_t {   // forward buffer 0 / 1 -> state buffer 2 / 3
    if (ref < 0) return -1;
    const int buf = (int)((uint32_t)ref >> 28);
    return tile_ref(buf + 2, ref & 0x0fffffff);
  };
  auto is_upd = [](int type) { return type == UNMQR || type == TSMQR || type == TTMQR; };
  auto pieces = [&](const DevTask& f) {   // adjoint strips of a forward update strip
    const int strip = (f.op >> 8) & 0xff;
    int n = 0;
    for (int h = 0; h < split; ++h)
      if ((int64_t)(strip * split + h) * wb < nb) ++n;
    return n;
  };
  // slots: per panel task, its adjoint update strips first (in program order), then its PU sub-tasks
  const int npu = nblk * (nblk - 1) / 2 * pus;
  std::vector<int32_t> nupd(std::max(1, pl.npanels), 0);
  for (const DevTask& f : pl.dev) {
    if (is_upd(f.op & 15)) {
      if (f.tslot < 0 || f.tslot >= pl.npanels) throw std::logic_error("update without a panel");
      nupd[f.tslot] += pieces(f);
    }
  }
  bp.pinfo.assign((size_t)4 * std::max(1, pl.npanels), 0);
  bp.slot_off.clear();
  int64_t off = 0;
  const int64_t upd_size = (int64_t)nb * nb + (int64_t)nb * ib, pu_size = (int64_t)nb * ib + (int64_t)ib * ib;
  for (int t = 0; t < pl.npanels; ++t) {
    bp.pinfo[4 * t + 0] = (int32_t)bp.slot_off.size();
    bp.pinfo[4 * t + 1] = nupd[t];
    for (int u = 0; u < nupd[t]; ++u) {
      bp.slot_off.push_back(off);
      off += upd_size;
    }
    bp.pinfo[4 * t + 2] = (int32_t)bp.slot_off.size();
    for (int u = 0; u < npu; ++u) {
      bp.slot_off.push_back(off);
      off += pu_size;
    }
    bp.pinfo[4 * t + 3] = -1;
    if (nupd[t] >= kRedMinSlots) {   // reduced slot, laid out as an update slot
      bp.pinfo[4 * t + 3] = (int32_t)bp.slot_off.size();
      bp.slot_off.push_back(off);
      off += upd_size;
    }
  }
  bp.slot_off.push_back(off);
  if (bp.slot_off.size() >= (1u << 31)) throw std::invalid_argument("too many partial slots");
  std::vector<int32_t> next_upd(std::max(1, pl.npanels), 0);
  auto pu_index = [&](int b, int s, int h) { return (b * nblk - b * (b + 1) / 2 + (s - b - 1)) * pus + h; };

  // adjoint nodes: one per forward sub-task, `split` per forward update strip
  std::vector<DevTask> sub;
  std::vector<int64_t> wt;
  std::vector<int32_t> fwd_of;
  std::vector<int32_t> first(nsub + 1, 0);
  std::vector<std::vector<int32_t>> bupd_of(std::max(1, pl.npanels));   // adjoint update strips per panel
  const int64_t ib2 = (int64_t)ib * ib;
  for (int32_t y = 0; y < nsub; ++y) {
    first[y] = (int32_t)sub.size();
    const DevTask& f = pl.dev[y];
    const int type = f.op & 15, tr = (f.op >> 4) & 1, strip = (f.op >> 8) & 0xff, blk = (f.op >> 16) & 0xff;
    const int kind = (f.op >> 24) & 3;
    DevTask d{};
    d.x = f.x;
    d.tslot = f.tslot;
    d.flags = 0;
    if (type == PF || type == PU) {
      d.a = state_ref(f.a);
      d.c = state_ref(f.x);
      const int64_t rows = kind == PK_GE ? nb - (int64_t)blk * ib : (kind == PK_TS ? nb : (int64_t)(blk + 1) * ib);
      if (type == PF) {
        d.op = make_op(BPF, tr, false, 0, blk, kind);
        // 10 ib^2 rows flops, weighted x2: its per-reflector chain runs at about half the rate of the
        // block sub-tasks (measured per-sub-task times on a GB300)
        wt.push_back(20 * ib2 * rows);
        sub.push_back(d);
        fwd_of.push_back(y);
      } else {
        for (int h = 0; h < pus; ++h) {
          DevTask e = d;
          e.op = make_op(BPU, tr, h == 1, strip, blk, kind);
          e.flags = bp.pinfo[4 * f.tslot + 2] + pu_index(blk, strip, h);
          wt.push_back(14 * ib2 * rows / pus);
          sub.push_back(e);
          fwd_of.push_back(y);
        }
      }
    } else if (is_upd(type)) {
      d.a = state_ref(f.a);
      d.c = state_ref(f.c);
      const int uk = type == UNMQR ? 0 : (type == TSMQR ? 1 : 2);
      for (int h = 0; h < split; ++h) {
        const int sb = strip * split + h;
        if ((int64_t)sb * wb >= nb) continue;
        if (sb > 255) throw std::invalid_argument("too many adjoint strips");
        DevTask e = d;
        e.op = make_op(BUPD, tr, false, sb, 0, uk);
        e.flags = bp.pinfo[4 * f.tslot + 0] + next_upd[f.tslot]++;
        bupd_of[f.tslot].push_back((int32_t)sub.size());
        sub.push_back(e);
        wt.push_back(3 * (type == TSMQR ? 4 : 2) * (int64_t)nb * nb * wb);
        fwd_of.push_back(y);
      }
    } else {
      d.x = state_ref(f.x);
      d.a = -1;
      d.c = state_ref(f.c);
      d.flags = f.flags & 1;
      d.op = make_op(BCOPY, false, false, 0, 0, 0);
      wt.push_back((int64_t)nb * nb);
      sub.push_back(d);
      fwd_of.push_back(y);
    }
  }
  first[nsub] = (int32_t)sub.size();
  // reduction sub-tasks: per block of a panel with a reduced slot, chunks of kRedElems / ib rows
  std::vector<std::pair<int32_t, int32_t>> red_edge;   // (BRED node, BPF node it feeds)
  const int red_rows = std::max(1, kRedElems / ib);
  for (int32_t y = 0; y < nsub; ++y) {
    const DevTask& f = pl.dev[y];
    if ((f.op & 15) != PF || bp.pinfo[4 * f.tslot + 3] < 0) continue;
    const int tr = (f.op >> 4) & 1, blk = (f.op >> 16) & 0xff, kind = (f.op >> 24) & 3;
    const int64_t vrows = kind == PK_GE ? nb - (int64_t)blk * ib : (kind == PK_TS ? nb : (int64_t)(blk + 1) * ib);
    const int nchunk = (int)((vrows + red_rows - 1) / red_rows);
    if (nchunk > 255) throw std::invalid_argument("too many reduction chunks");
    const int64_t nu = nupd[f.tslot];
    for (int c = 0; c < nchunk; ++c) {
      DevTask e{};
      e.op = make_op(BRED, tr, false, c, blk, kind);
      e.x = state_ref(f.x);
      e.a = -1;
      e.c = -1;
      e.tslot = f.tslot;
      e.flags = 0;
      red_edge.push_back({(int32_t)sub.size(), first[y]});
      sub.push_back(e);
      wt.push_back(nu * std::min<int64_t>(red_rows, vrows - (int64_t)c * red_rows) * ib + (c == 0 ? nu * ib2 : 0));
      fwd_of.push_back(y);
    }
  }
  const int32_t nnode = (int32_t)sub.size();
  // reversed DAG: forward y depends on d  ->  every adjoint node of d depends on every node of y
  std::vector<std::vector<int32_t>> rdeps(nnode);
  for (int32_t y = 0; y < nsub; ++y)
    for (int32_t k = pl.dev[y].dep_begin; k < pl.dev[y].dep_end; ++k) {
      const int32_t d = pl.deps[k];
      for (int32_t a = first[d]; a < first[d + 1]; ++a)
        for (int32_t b = first[y]; b < first[y + 1]; ++b) rdeps[a].push_back(b);
    }
  // a reduction waits for every update strip of its panel; the factor sub-task waits for its reductions
  for (const auto& re : red_edge) {
    rdeps[re.first] = bupd_of[sub[re.first].tslot];
    rdeps[re.second].push_back(re.first);
  }
  // bottom levels of the reversed DAG, over a topological order (Kahn)
  std::vector<std::vector<int32_t>> succ(nnode);
  std::vector<int32_t> indeg(nnode, 0), topo;
  topo.reserve(nnode);
  for (int32_t a = 0; a < nnode; ++a)
    for (int32_t b : rdeps[a]) {
      succ[b].push_back(a);
      ++indeg[a];
    }
  for (int32_t a = nnode - 1; a >= 0; --a)
    if (indeg[a] == 0) topo.push_back(a);
  for (size_t h = 0; h < topo.size(); ++h)
    for (int32_t a : succ[topo[h]])
      if (--indeg[a] == 0) topo.push_back(a);
  if ((int32_t)topo.size() != nnode) throw std::logic_error("adjoint DAG has a cycle");
  std::vector<int64_t> bottom(nnode, 0);
  for (int32_t h = nnode - 1; h >= 0; --h) {
    const int32_t a = topo[h];
    int64_t mx = 0;
    for (int32_t b : succ[a]) mx = std::max(mx, bottom[b]);
    bottom[a] = wt[a] + mx;
  }
  std::vector<int32_t> order(nnode);
  for (int32_t z = 0; z < nnode; ++z) order[z] = nnode - 1 - z;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return bottom[a] > bottom[b]; });
  std::vector<int32_t> pos(nnode);
  for (int32_t z = 0; z < nnode; ++z) pos[order[z]] = z;

  // Partial-slot storage is recycled in queue order.  A panel's slots are read by its factor adjoints
  // and reductions only; the factor adjoint of its block 0 follows all of them in the reversed DAG
  // (BPF(b) waits for BPU(b, s), which waits for BPF(s), s > b; BPF(b) waits for its reductions and
  // PU slots, the reductions for every update strip), so once that sub-task has run the panel's
  // storage is free.  Walking the queue, each logical slot takes, at its first writer, the storage of
  // its size released longest ago (or new storage), and every writer of that slot also waits for the
  // releasing BPF(0), which is earlier in the queue: the order stays topological, each storage region
  // has one owner at a time, and the sums keep their fixed order (the result is bitwise the same as
  // with private slots).  Peak storage is what the queue order keeps live (8192^2 Auto, nb = 256:
  // 6.8 GB instead of 222 GB).
  {
    const int32_t nlog = (int32_t)bp.slot_off.size() - 1;
    std::vector<int64_t> ssize(nlog);
    for (int32_t l = 0; l < nlog; ++l) ssize[l] = bp.slot_off[l + 1] - bp.slot_off[l];
    std::vector<int32_t> slot_panel(nlog, -1);
    const int npu_all = nblk * (nblk - 1) / 2 * pus;
    for (int t = 0; t < pl.npanels; ++t) {
      const int32_t* pi = &bp.pinfo[4 * t];
      for (int32_t l = pi[0]; l < pi[0] + pi[1]; ++l) slot_panel[l] = t;
      for (int32_t l = pi[2]; l < pi[2] + npu_all; ++l) slot_panel[l] = t;
      if (pi[3] >= 0) slot_panel[pi[3]] = t;
    }
    std::vector<int64_t> phys(nlog, -1);
    std::vector<int32_t> rel(nlog, -1);                    // node whose completion frees the storage
    std::map<int64_t, std::deque<std::pair<int64_t, int32_t>>> free_list;   // size -> (offset, releasing node)
    std::vector<std::vector<int32_t>> held(std::max(1, pl.npanels));
    int64_t pool = 0;
    for (int32_t z = 0; z < nnode; ++z) {
      const int32_t y = order[z];
      const DevTask& e = sub[y];
      const int type = e.op & 15;
      int32_t l = -1;
      if (type == BUPD || type == BPU) l = e.flags;
      else if (type == BRED) l = bp.pinfo[4 * e.tslot + 3];
      if (l >= 0) {
        if (l >= nlog || slot_panel[l] != e.tslot) throw std::logic_error("partial slot of another panel");
        if (phys[l] < 0) {
          auto& fl = free_list[ssize[l]];
          if (!fl.empty()) {
            phys[l] = fl.front().first;
            rel[l] = fl.front().second;
            fl.pop_front();
          } else {
            phys[l] = pool;
            pool += ssize[l];
          }
          held[e.tslot].push_back(l);
        }
        if (rel[l] >= 0) rdeps[y].push_back(rel[l]);
      }
      if (type == BPF && ((e.op >> 16) & 0xff) == 0 && e.tslot >= 0 && e.tslot < pl.npanels) {
        for (int32_t h : held[e.tslot]) free_list[ssize[h]].push_back({phys[h], y});
        held[e.tslot].clear();
      }
    }
    for (int32_t l = 0; l < nlog; ++l) {
      if (phys[l] < 0) {   // never written (not expected): storage of its own
        phys[l] = pool;
        pool += ssize[l];
      }
      bp.slot_off[l] = phys[l];
    }
    bp.slot_off[nlog] = pool;
  }
  bp.dev.resize(nnode);
  bp.fwd.resize(nnode);
  bp.deps.clear();
  for (int32_t z = 0; z < nnode; ++z) {
    const int32_t y = order[z];
    DevTask e = sub[y];
    e.dep_begin = (int32_t)bp.deps.size();
    for (int32_t dd : rdeps[y]) {
      if (pos[dd] >= z) throw std::logic_error("adjoint order is not topological");
      bp.deps.push_back(pos[dd]);
    }
    e.dep_end = (int32_t)bp.deps.size();
    bp.dev[z] = e;
    bp.fwd[z] = fwd_of[y];
  }
}

void merge_programs(const std::vector<const Plan*>& plans, std::vector<DevTask>* dev, std::vector<int32_t>* deps) {
  const size_t np = plans.size();
  if (np >= (1u << 23)) throw std::invalid_argument("too many matrices in a batch");
  size_t total = 0;
  for (const Plan* pl : plans) total += pl->dev.size();
  std::vector<size_t> head(np, 0);
  std::vector<std::vector<int32_t>> gpos(np);
  for (size_t b = 0; b < np; ++b) gpos[b].resize(plans[b]->dev.size());
  // k-way merge by decreasing priority (ties: lower matrix index first)
  using Item = std::pair<int64_t, int64_t>;   // (-prio, b)
  std::vector<Item> heap;
  auto push = [&](size_t b) {
    if (head[b] < plans[b]->dev.size()) {
      heap.push_back({-plans[b]->prio[head[b]], (int64_t)b});
      std::push_heap(heap.begin(), heap.end(), std::greater<Item>());
    }
  };
  for (size_t b = 0; b < np; ++b) push(b);
  dev->clear();
  dev->reserve(total);
  std::vector<std::pair<int32_t, int32_t>> src;   // (matrix, local queue position) per global position
  src.reserve(total);
  while (!heap.empty()) {
    std::pop_heap(heap.begin(), heap.end(), std::greater<Item>());
    const size_t b = (size_t)heap.back().second;
    heap.pop_back();
    const int32_t y = (int32_t)head[b]++;
    gpos[b][y] = (int32_t)src.size();
    src.push_back({(int32_t)b, y});
    push(b);
  }
  deps->clear();
  for (size_t g = 0; g < src.size(); ++g) {
    const Plan* pl = plans[src[g].first];
    DevTask e = pl->dev[src[g].second];
    const int32_t b0 = e.dep_begin, b1 = e.dep_end;
    e.dep_begin = (int32_t)deps->size();
    for (int32_t d = b0; d < b1; ++d) {
      const int32_t gd = gpos[src[g].first][pl->deps[d]];
      if (gd >= (int32_t)g) throw std::logic_error("merged order is not topological");
      deps->push_back(gd);
    }
    e.dep_end = (int32_t)deps->size();
    e.flags = (e.flags & 0xff) | (src[g].first << 8);
    dev->push_back(e);
  }
}

namespace {

// Measured mean sub-task times of the executor, per storage precision and (nb, ib): see
// autotune_table.inc for the command that writes them.  Classes: PF GE / TS / TT, PU GE / TS / TT,
// UNMQR / TSMQR / TTMQR update strips.
struct AutotuneRow {
  int esize, nb, ib;
  double us[9];
};
const AutotuneRow kAutotuneTable[] = {
#include "autotune_table.inc"
    {0, 0, 0, {0, 0, 0, 0, 0, 0, 0, 0, 0}},   // end marker
};

// Fallback model when the table has no row for this precision: padded Table 1 work over the relative
// efficiency of the tile size in batches (FP64, GB300: FlatTS batches of nb = 32 / 64 / 128 ran at
// 0.19 / 0.48 / 0.62 of the FP64 rate the nb = 128 batch reached), plus the critical path over the
// number of SMs a matrix competes with; FlatTS, ib = 16 for nb = 32, else 32.
void autotune_model(int64_t m, int64_t n, int nsm, int* nb_out, int* ib_out, int* tree_out, int* variant_out) {
  const int cands[3] = {32, 64, 128};
  const double eff[3] = {0.30, 0.75, 1.0};
  double best = -1.0;
  for (int c = 0; c < 3; ++c) {
    const int nb = cands[c];
    if (c > 0 && cands[c - 1] >= n) break;          // a larger tile would only add padding
    const int p = (int)((m + nb - 1) / nb), q = (int)((n + nb - 1) / nb);
    const int variant = choose_variant(p, q, FLATTS, 1, nullptr, nullptr);
    const std::vector<Task> ts = make_tasks(p, q, FLATTS, variant, 1);
    int64_t work = 0, cp = 0;
    const int kw[7] = {4, 6, 6, 12, 2, 6, 0};
    for (const Task& t : ts) work += kw[t.type];
    make_dag(ts, p, q, variant, nullptr, nullptr, &cp);
    const double unit = (double)nb * nb * nb / 3.0;
    const double cost = (double)work * unit / eff[c] + (double)cp * unit / std::max(1, nsm / 8);
    if (best < 0 || cost < best) {
      best = cost;
      *nb_out = nb;
      *ib_out = nb == 32 ? 16 : 32;
      *tree_out = FLATTS;
      *variant_out = variant;
    }
  }
}

}  // namespace

void autotune(int64_t m, int64_t n, int nsm, int esize, int* nb_out, int* ib_out, int* tree_out, int* variant_out) {
  // Candidates: every calibrated (nb, ib) of this precision x {FlatTS, Greedy, Auto}, the variant by
  // critical path (Sec. 4.3.3).  A candidate's cost is the time its sub-tasks keep SMs busy (the
  // calibrated times summed over its device program: a panel task is nb/ib factor sub-tasks and
  // (nb/ib)(nb/ib - 1)/2 panel updates, an update task nb/w strips) plus its critical path with the same
  // times over nsm / 8 (in a batch the other matrices supply the parallelism, so the busy time decides
  // and the critical path only breaks near-ties).  The critical path is evaluated only for candidates
  // within 10 % of the best busy time.
  struct Cand {
    int nb, ib, tree, variant;
    double busy;
    const AutotuneRow* row;
  };
  std::vector<Cand> cands;
  int64_t smallest_fit = -1;   // smallest calibrated nb >= n: larger tiles would only add padding
  for (const AutotuneRow* r = kAutotuneTable; r->esize; ++r)
    if (r->esize == esize && r->nb >= n && (smallest_fit < 0 || r->nb < smallest_fit)) smallest_fit = r->nb;
  for (const AutotuneRow* r = kAutotuneTable; r->esize; ++r) {
    if (r->esize != esize || r->ib < 1 || r->nb % r->ib) continue;
    if (smallest_fit > 0 && r->nb > smallest_fit) continue;
    const int nb = r->nb, ib = r->ib, nblk = nb / ib;
    const int w = std::min(nb, std::max(ib, 32 / ib * ib));     // the executor's default strip width
    const int64_t R = std::max<int64_t>(1, (int64_t)nsm * w * (esize == 4 ? 2 : 1) / nb);
    const int p = (int)((m + nb - 1) / nb), q = (int)((n + nb - 1) / nb);
    const int nstrip = (nb + w - 1) / w;
    for (int tree : {FLATTS, GREEDY, AUTO}) {
      const int variant = choose_variant(p, q, tree, R, nullptr, nullptr);
      double busy = 0.0;
      for (const Task& t : make_tasks(p, q, tree, variant, R)) {
        const int kind = t.type == GEQRT ? 0 : (t.type == TSQRT ? 1 : (t.type == TTQRT ? 2 : -1));
        if (kind >= 0) busy += nblk * r->us[kind] + nblk * (nblk - 1) / 2 * r->us[3 + kind];
        else if (t.type == UNMQR) busy += nstrip * r->us[6];
        else if (t.type == TSMQR) busy += nstrip * r->us[7];
        else if (t.type == TTMQR) busy += nstrip * r->us[8];
      }
      cands.push_back({nb, ib, tree, variant, busy, r});
    }
  }
  if (cands.empty()) {
    autotune_model(m, n, nsm, nb_out, ib_out, tree_out, variant_out);
    return;
  }
  double best_busy = cands[0].busy;
  for (const Cand& c : cands) best_busy = std::min(best_busy, c.busy);
  double best = -1.0;
  for (const Cand& c : cands) {
    if (c.busy > 1.1 * best_busy) continue;
    const int nb = c.nb, nblk = nb / c.ib;
    const int w = std::min(nb, std::max(c.ib, 32 / c.ib * c.ib));
    const int64_t R = std::max<int64_t>(1, (int64_t)nsm * w * (esize == 4 ? 2 : 1) / nb);
    const int p = (int)((m + nb - 1) / nb), q = (int)((n + nb - 1) / nb);
    const std::vector<Task> ts = make_tasks(p, q, c.tree, c.variant, R);
    std::vector<std::vector<int32_t>> preds;
    make_dag(ts, p, q, c.variant, &preds, nullptr, nullptr);
    std::vector<double> fin(ts.size(), 0.0);
    double cp = 0.0;
    for (size_t x = 0; x < ts.size(); ++x) {
      const Task& t = ts[x];
      const int kind = t.type == GEQRT ? 0 : (t.type == TSQRT ? 1 : (t.type == TTQRT ? 2 : -1));
      double wt = 0.0;
      if (kind >= 0) wt = nblk * c.row->us[kind] + (nblk - 1) * c.row->us[3 + kind];   // the factor chain
      else if (t.type == UNMQR) wt = c.row->us[6];
      else if (t.type == TSMQR) wt = c.row->us[7];
      else if (t.type == TTMQR) wt = c.row->us[8];
      double st = 0.0;
      for (int32_t d : preds[x]) st = std::max(st, fin[d]);
      fin[x] = st + wt;
      cp = std::max(cp, fin[x]);
    }
    const double cost = c.busy + cp * 8.0 / std::max(1, nsm);
    if (best < 0 || cost < best) {
      best = cost;
      *nb_out = c.nb;
      *ib_out = c.ib;
      *tree_out = c.tree;
      *variant_out = c.variant;
    }
  }
}

}  // namespace bd
