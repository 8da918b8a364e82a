// Tile kernels of the tiled QR / LQ steps and the persistent dataflow executor (sm_103a), for FP64
// and for FP32 storage (the split-precision form).
//
// Kernels (Table 1, Sec. 3.2 of Faverge, Langou, Robert, Dongarra, arXiv 1611.06892):
//   GEQRT  QR of one tile                      UNMQR  apply its Q^T to a tile of the same row
//   TSQRT  triangle on top of square           TSMQR  apply to the pair of tile rows
//   TTQRT  triangle on top of triangle         TTMQR  apply to the pair of tile rows
// An LQ step (Algorithm 4) runs the same kernels on transposed tiles: every tile access goes through
// an orientation flag `tr`, so GELQT/UNMLQ/... are GEQRT/UNMQR/... on the transposed geometry.
//
// FP64: GB300's FP64 units deliver 2 FMA/clock/SM (about 1.2 TFLOP/s per GPU, measured) and FP64 MMA
// is not faster than DFMA on this part, so the contractions are register-blocked DFMA loops.
// FP32 storage: the contractions of the updates run on the tensor cores as three TF32 products,
// a_hi b_hi + a_hi b_lo + a_lo b_hi with a = a_hi + a_lo (a_hi = TF32 round-to-nearest of a, a_lo =
// TF32 of the remainder), accumulated in FP32 (Markidis et al. 2018; Ootomo and Yokota 2022); the
// reflector norms, beta, tau (the T diagonal) and the scaling of the reflector vectors are computed in
// FP64.  Each task stages its operands in shared memory, reads and writes global memory through L2
// only (ld/st.cg: tiles written by other SMs are never served stale from L1), and applies reflectors
// in compact-WY blocks of ib (the paper's inner blocking): W = op(T) (C_top + V^T C), C_top -= W,
// C -= V W.
//
// Householder convention (LAPACK style): for x = [alpha; tail], sigma2 = tail . tail; sigma2 == 0 gives
// H = I (tau = 0, beta = alpha); otherwise beta = -sgn(alpha) sqrt(alpha^2 + sigma2) with sgn(alpha) = -1
// only for alpha < 0, tau = (beta - alpha) / beta, v = [1; tail / (alpha - beta)].
#include <cstdio>

#include "kernels.cuh"

namespace bd {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarps = kThreads / 32;

template <typename E> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

__device__ __forceinline__ double ldg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldg(const float* p) { return __ldcg(p); }
__device__ __forceinline__ void stg(double* p, double v) { __stcg(p, v); }
__device__ __forceinline__ void stg(float* p, float v) { __stcg(p, v); }

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__host__ __device__ inline int odd_ld(int rows) { return rows | 1; }
// Leading dimension of a row-major shared buffer with n columns.  FP64: even, with ld/2 odd, so that
// the 16-byte pairs of consecutive rows read by consecutive lanes fall in distinct bank groups.  FP32:
// n rounded up to 8, plus 8, so that the 4 x 8 (row x column) patterns of the MMA fragments hit 32
// distinct banks.
__host__ __device__ inline int rm_ld(int n, int esize) {
  if (esize == 8) {
    int l = n + (n & 1);
    if (((l >> 1) & 1) == 0) l += 2;
    return l;
  }
  return ((n + 7) & ~7) + 8;
}

// Shared-memory layout: a header of doubles (tau, block reduction scratch) followed by arrays of the
// element type at offsets (in elements) that keep 16-byte alignment.
struct Layout {
  int lp, lv, lc;            // col-major panel ld; row-major V ld; row-major C / W ld
  int P, V, Vh, B, Cs, Ct, Rt, Tb, G, W, W2, total;
};
// tau[<= 64], red[32]; the adjoint panel also uses three more arrays of 64 doubles
constexpr int kHeaderDoubles = 64 + 32 + 3 * 64;
__host__ __device__ inline int align4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline int align32(int x) { return (x + 31) & ~31; }
__host__ __device__ inline Layout layout_panel(int nb, int ib, int esize) {
  Layout L{};
  L.lp = odd_ld(nb);
  L.lv = L.lc = 0;
  int o = 0;
  L.P = o;   o = align4(o + L.lp * ib);
  L.Rt = o;  o = align4(o + ib * ib);
  L.Tb = o;  o = align4(o + ib * ib);
  L.G = o;   o = align4(o + 2 * ib * ib);   // Gram matrix and a scratch block for T
  L.V = L.Vh = L.B = L.Cs = L.Ct = L.W = L.W2 = -1;
  L.total = o;
  return L;
}
__host__ __device__ inline Layout layout_update(int nb, int ib, int w, int esize) {
  Layout L{};
  L.lp = odd_ld(nb);
  L.lv = rm_ld(ib, esize);
  L.lc = rm_ld(w, esize);
  int o = 0;
  L.Cs = o;  o = align4(o + nb * L.lc);
  L.Ct = o;  o = align32(o + ib * L.lc);
  L.V = o;   o = align32(o + nb * L.lv);     // MMA operand regions start on 128-byte boundaries
  L.Tb = o;  o = align4(o + ib * (ib + 4));  // T (ld ib, or ib + 4 in the tcgen05 path)
  L.W = o;   o = align4(o + ib * L.lc);
  L.W2 = o;  o = align32(o + ib * L.lc);
  L.Vh = L.B = -1;
  if (esize == 4) {          // FP32 storage: TF32 high parts of V (V itself then holds the low parts),
                             // and the split -W2 operand of the tcgen05 phase (2 x ib x up to 64 rows)
    L.Vh = o;  o = align32(o + nb * L.lv);
    L.B = o;   o = align32(o + 2 * ib * ((w > ib ? w : ib) + 15) / 16 * 16);
  }
  L.P = L.Rt = L.G = -1;
  L.total = o;
  return L;
}

// Adjoint sub-tasks.  Update adjoint: state and gradient rows of a column chunk (hw columns), the
// top rows of both, one reflector block and T, and three ib x hw products.  Panel adjoint: reflector
// tails, state and gradient of one column block (column-major, ld lp), the top triangles and S.
struct BwdLayout {
  int lc, lv, lp;
  int Cs, Cg, Cts, Ctg, V, Vh, Tb, W, W2s, W2g, Ms, Mg, Rts, Rtg, Sb, Sc, total;
};
__host__ __device__ inline BwdLayout layout_bwd_update(int nb, int ib, int hw, int esize) {
  BwdLayout L{};
  L.lc = rm_ld(hw, esize);
  L.lv = rm_ld(ib, esize);
  L.lp = 0;
  int o = 0;
  L.Cs = o;  o = align4(o + nb * L.lc);
  L.Cg = o;  o = align4(o + nb * L.lc);
  L.Cts = o; o = align4(o + ib * L.lc);
  L.Ctg = o; o = align4(o + ib * L.lc);
  L.V = o;   o = align4(o + nb * L.lv);
  L.Tb = o;  o = align4(o + ib * ib);
  L.W = o;   o = align4(o + ib * L.lc);
  L.W2s = o; o = align4(o + ib * L.lc);
  L.W2g = o; o = align4(o + ib * L.lc);
  L.Vh = -1;
  if (esize == 4) {          // FP32 storage: TF32 high parts of V
    L.Vh = o;  o = align4(o + nb * L.lv);
  }
  L.Ms = L.Mg = L.Rts = L.Rtg = L.Sb = L.Sc = -1;
  L.total = o;
  return L;
}
__host__ __device__ inline BwdLayout layout_bwd_panel(int nb, int ib, int esize) {
  BwdLayout L{};
  L.lp = odd_ld(nb);
  L.lc = L.lv = 0;
  int o = 0;
  L.V = o;   o = align4(o + L.lp * ib);
  L.Ms = o;  o = align4(o + L.lp * ib);
  L.Mg = o;  o = align4(o + L.lp * ib);
  L.Rts = o; o = align4(o + ib * ib);
  L.Rtg = o; o = align4(o + ib * ib);
  L.Sb = o;  o = align4(o + ib * ib);
  L.Sc = o;  o = align4(o + (2 * ib + kThreads) * (8 / esize));   // doubles: reciprocals, row-sum partials
  L.Cs = L.Cg = L.Cts = L.Ctg = L.Tb = L.W = L.W2s = L.W2g = L.Vh = -1;
  L.total = o;
  return L;
}

__device__ __forceinline__ int toff(int r, int c, int nb, int tr) { return tr ? r * nb + c : r + c * nb; }

enum Mask : int { M_NONE = 0, M_UPPER = 1, M_UNITLOWER = 2 };

template <typename E>
__device__ __forceinline__ E masked_ld(const E* g, int R, int C, int nb, int tr, int mask) {
  if (mask == M_UPPER && R > C) return E(0);
  if (mask == M_UNITLOWER && R <= C) return (R == C) ? E(1) : E(0);
  return ldg(g + toff(R, C, nb, tr));
}

__device__ __forceinline__ uint32_t tf32_round(float x);
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo);

// Stores v at index i of s, or (FP32 storage, hi != null) its TF32 high part at hi[i] and low part at
// s[i] (the operands of the three-product tensor-core contraction).
template <typename E>
__device__ __forceinline__ void put(E* s, E* hi, int i, E v) {
  if constexpr (sizeof(E) == 4) {
    if (hi) {
      uint32_t h, l;
      split_tf32(v, h, l);
      hi[i] = __uint_as_float(h);
      s[i] = __uint_as_float(l);
      return;
    }
  }
  s[i] = v;
}

// Up to 256 x 32 elements: all of a thread's loads (up to 32) are issued before the first shared store, so
// that one L2 latency covers the whole block.  Lanes run along the contiguous direction of global memory.
template <typename E>
__device__ __forceinline__ void load_block32(E* s, int rs, int cs, const E* g, int nb, int tr, int r0, int c0,
                                             int rows, int cols, int mask, E* hi) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  E v[32];
  if (!tr) {   // c = warp + 8 kc, r = lane + 32 kr
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
      for (int kr = 0; kr < 8; ++kr) {
        const int c = warp + 8 * kc, r = lane + 32 * kr;
        v[kc * 8 + kr] = (c < cols && r < rows) ? masked_ld(g, r0 + r, c0 + c, nb, tr, mask) : E(0);
      }
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
      for (int kr = 0; kr < 8; ++kr) {
        const int c = warp + 8 * kc, r = lane + 32 * kr;
        if (c < cols && r < rows) put(s, hi, r * rs + c * cs, v[kc * 8 + kr]);
      }
    }
  } else {     // r = warp + 8 kr, c = lane
#pragma unroll
    for (int kr = 0; kr < 32; ++kr) {
      const int r = warp + 8 * kr;
      v[kr] = (lane < cols && r < rows) ? masked_ld(g, r0 + r, c0 + lane, nb, tr, mask) : E(0);
    }
#pragma unroll
    for (int kr = 0; kr < 32; ++kr) {
      const int r = warp + 8 * kr;
      if (lane < cols && r < rows) put(s, hi, r * rs + lane * cs, v[kr]);
    }
  }
}

// Shared element (r, c) at s[r * rs + c * cs] <- oriented X(r0 + r, c0 + c).  M_UPPER zeroes entries
// below the diagonal, M_UNITLOWER gives the unit lower trapezoid.  Blocks of at most 256 x 32 go through
// load_block32.  With hi != null (FP32) the block is stored split: TF32 high parts in hi, low parts in s
// (same indexing).
template <typename E>
__device__ void load_tile(E* s, int rs, int cs, const E* g, int nb, int tr, int r0, int c0, int rows, int cols,
                          int mask, E* hi = nullptr) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (rows <= 256 && cols <= 32) {
    load_block32(s, rs, cs, g, nb, tr, r0, c0, rows, cols, mask, hi);
    return;
  }
  if (!tr) {
    for (int c = warp; c < cols; c += kWarps) {
#pragma unroll 4
      for (int r = lane; r < rows; r += 32) put(s, hi, r * rs + c * cs, masked_ld(g, r0 + r, c0 + c, nb, tr, mask));
    }
  } else {
#pragma unroll 4
    for (int r = warp; r < rows; r += kWarps) {
      for (int c = lane; c < cols; c += 32) put(s, hi, r * rs + c * cs, masked_ld(g, r0 + r, c0 + c, nb, tr, mask));
    }
  }
}
// Oriented X(r0 + r, c0 + c) <- s[r * rs + c * cs]; M_UPPER writes only entries on or above the diagonal.
template <typename E>
__device__ void store_tile(const E* s, int rs, int cs, E* g, int nb, int tr, int r0, int c0, int rows, int cols,
                           int mask) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!tr) {
    for (int c = warp; c < cols; c += kWarps) {
#pragma unroll 4
      for (int r = lane; r < rows; r += 32) {
        if (mask == M_UPPER && r0 + r > c0 + c) continue;
        stg(g + toff(r0 + r, c0 + c, nb, tr), s[r * rs + c * cs]);
      }
    }
  } else {
#pragma unroll 4
    for (int r = warp; r < rows; r += kWarps) {
      for (int c = lane; c < cols; c += 32) {
        if (mask == M_UPPER && r0 + r > c0 + c) continue;
        stg(g + toff(r0 + r, c0 + c, nb, tr), s[r * rs + c * cs]);
      }
    }
  }
}

template <typename E>
__device__ __forceinline__ E warp_sum(E v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

enum PanelMode : int { PM_GE = 0, PM_TS = 1, PM_TT = 2 };

// Error-free transformations of FP32 numbers (the _rn intrinsics keep the compiler from contracting
// them into FMAs): TwoSum (Knuth; Moller 1965) s + e = a + b exactly; FastTwoSum (Dekker 1971) the same
// for |a| >= |b|.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// beta, tau and the tail scale 1 / (alpha - beta) of a reflector with FP32 storage, from alpha and the
// tail's squared norm sh + sl (an unevaluated float pair), in float-pair arithmetic (about 44 bits):
//   n2 = alpha^2 + sigma^2 (exact square by FMA), nrm = sqrt(n2) as y + (n2 - y^2) / (2 y) with y the
//   rounded FP32 root (one Newton correction), beta = -sgn(alpha) nrm, d = alpha - beta (|d| = |alpha| +
//   nrm, no cancellation), tau = (beta - alpha) / beta = 1 + |alpha| / nrm and 1 / d, each reciprocal as
//   r0 (1 + e) with r0 the rounded FP32 reciprocal and e = 1 - x r0 its residual (one Newton step).
// Returns the FP32 roundings of beta and tau and the scale as a float pair.  sigma^2 = 0: H = I.
__device__ __forceinline__ void reflector_scalars_pair(float alpha, float sh, float sl, float& beta, float& tau,
                                                       float& sch, float& scl) {
  float s2h, s2l;
  two_sum(sh, sl, s2h, s2l);
  if (s2h == 0.0f) {
    beta = alpha;
    tau = 0.0f;
    sch = scl = 0.0f;
    return;
  }
  const float a2h = __fmul_rn(alpha, alpha), a2l = fmaf(alpha, alpha, -a2h);
  float nh, nl;
  two_sum(a2h, s2h, nh, nl);
  nl = __fadd_rn(nl, __fadd_rn(a2l, s2l));
  fast_two_sum(nh, nl, nh, nl);
  const float y = __fsqrt_rn(nh);
  const float res = __fadd_rn(fmaf(-y, y, nh), nl);             // n2 - y^2 (the FMA residual is exact)
  float rh, rl;
  fast_two_sum(y, __fmul_rn(res, __fmul_rn(0.5f, __frcp_rn(y))), rh, rl);
  const bool neg = alpha < 0.0f;
  const float bh = neg ? rh : -rh, bl = neg ? rl : -rl;
  float dh, dl;
  two_sum(alpha, -bh, dh, dl);
  dl = __fsub_rn(dl, bl);
  fast_two_sum(dh, dl, dh, dl);
  const float q0 = __frcp_rn(rh);                                // 1 / nrm = q0 (1 + eq)
  const float eq = __fsub_rn(fmaf(-rh, q0, 1.0f), __fmul_rn(rl, q0));
  const float aa = fabsf(alpha);
  const float ph = __fmul_rn(aa, q0);
  const float pl = __fadd_rn(fmaf(aa, q0, -ph), __fmul_rn(ph, eq));
  float th, tl;
  fast_two_sum(1.0f, ph, th, tl);                                // |alpha| / nrm <= 1
  tau = __fadd_rn(th, __fadd_rn(tl, pl));
  const float r0 = __frcp_rn(dh);                                // 1 / d = r0 (1 + er)
  const float er = __fsub_rn(fmaf(-dh, r0, 1.0f), __fmul_rn(dl, r0));
  fast_two_sum(r0, __fmul_rn(r0, er), sch, scl);
  beta = __fadd_rn(bh, bl);
}

// Unblocked factorization of kb panel columns held in P (ld lp).
//  GE: reflector jj has alpha = P[jj, jj] and tail P[jj+1 .. rows-1, jj].
//  TS: alpha = Rt[jj, jj] (top triangle), tail P[0 .. rows-1, jj].
//  TT: as TS with tail P[0 .. min(rows, voff + jj + 1) - 1, jj] (the eliminated tile is a triangle).
// FP64 storage: the squared norm, beta, tau and the scaling of the tail are computed in FP64.  FP32
// storage: the squared norm is a compensated float-pair sum (FP64-level accuracy); beta, tau and the
// scale follow in FP64 (pair_scalars false) or in float-pair arithmetic (pair_scalars true,
// reflector_scalars_pair), both giving the FP32 values the reduction stores to within their rounding.
template <typename E>
__device__ void factor_panel(int mode, E* P, int lp, int rows, int kb, E* Rt, int lrt, int voff, double* tau_s,
                             double* red, bool pair_scalars = false) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* scale_s = tau_s + 96;          // 1 / (alpha - beta) of each reflector (header scratch)
  // float-pair scalars (FP32 storage): tau and the scale pair per reflector (header doubles 160..255)
  float* tauf_s = reinterpret_cast<float*>(tau_s + 160);
  float* sch_s = tauf_s + 64;
  float* scl_s = sch_s + 64;
  const bool pairs = sizeof(E) == 4 && pair_scalars;
  auto tail = [&](int j, int& t0, int& t1) {
    if (mode == PM_GE) {
      t0 = j + 1;
      t1 = rows;
    } else {
      t0 = 0;
      t1 = (mode == PM_TT) ? min(rows, voff + j + 1) : rows;
    }
  };
  // beta, tau and the tail scaling 1/(alpha - beta) of column j from its tail's squared norm sigma2, by
  // one thread (FP64 issues at 2 FMA / clock / SM on this part: the scalar chain is done once, with one
  // division: inv = 1 / (beta d), d = alpha - beta, scale = beta inv, tau = -d^2 inv = (beta - alpha)/beta).
  auto scalars = [&](int j, double sigma2) {
    E* alpha_p = (mode == PM_GE) ? &P[j + j * lp] : &Rt[j + j * lrt];
    const double alpha = (double)*alpha_p;
    double beta = alpha, tau = 0.0, scale = 0.0;
    if (sigma2 != 0.0) {
      const double nrm = sqrt(alpha * alpha + sigma2);
      beta = alpha < 0.0 ? nrm : -nrm;
      const double d = alpha - beta;
      const double inv = 1.0 / (beta * d);
      scale = beta * inv;
      tau = -d * d * inv;
    }
    *alpha_p = (E)beta;
    tau_s[j] = tau;
    scale_s[j] = scale;
  };
  auto scalars_pair = [&](int j, float sh, float sl) {
    E* alpha_p = (mode == PM_GE) ? &P[j + j * lp] : &Rt[j + j * lrt];
    float beta, tau, sch, scl;
    reflector_scalars_pair((float)*alpha_p, sh, sl, beta, tau, sch, scl);
    *alpha_p = (E)beta;
    tauf_s[j] = tau;
    sch_s[j] = sch;
    scl_s[j] = scl;
  };
  // The tails stay unscaled during the factorization (v = [1; scale x]): applying H_j to column c is
  // w = c_top + scale (x . c_tail), c_top -= tau w, c_tail -= (tau w scale) x, and the scaling of all
  // tails is one parallel pass at the end, off the critical chain.  Warp 0 applies H_jj to column jj + 1
  // and forms reflector jj + 1 (its squared norm accumulated while updating), warps 1..7 update the
  // later columns: one barrier per column.
  if (warp == 0) {
    int t0, t1;
    tail(0, t0, t1);
    if (pairs) {
      float sh = 0.0f, sl = 0.0f;
      for (int r = t0 + lane; r < t1; r += 32) {
        const float x = (float)P[r];
        const float p = __fmul_rn(x, x);
        float s2, e2;
        two_sum(sh, p, s2, e2);
        sl = __fadd_rn(sl, __fadd_rn(e2, fmaf(x, x, -p)));
        sh = s2;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(kFull, sh, o), ol = __shfl_xor_sync(kFull, sl, o);
        float s2, e2;
        two_sum(sh, oh, s2, e2);
        sl = __fadd_rn(__fadd_rn(sl, ol), e2);
        sh = s2;
      }
      if (lane == 0) scalars_pair(0, sh, sl);
    } else {
      double part = 0.0;
      for (int r = t0 + lane; r < t1; r += 32) {
        const double x = (double)P[r];
        part += x * x;
      }
      part = warp_sum(part);
      if (lane == 0) scalars(0, part);
    }
  }
  __syncthreads();
  for (int jj = 0; jj < kb; ++jj) {
    // tau and the tail scale of reflector jj in the storage type (FP32 storage: rounded from the FP64
    // values, or from the float-pair ones)
    E tauE, se;
    if (pairs) {
      tauE = (E)tauf_s[jj];
      se = (E)__fadd_rn(sch_s[jj], scl_s[jj]);
    } else {
      tauE = (E)tau_s[jj];
      se = (E)scale_s[jj];
    }
    const bool refl = tauE != E(0);
    int t0, t1;
    tail(jj, t0, t1);
    if (warp == 0) {
      if (jj + 1 < kb) {
        const int c = jj + 1;
        int n0, n1;                      // tail of reflector c
        tail(c, n0, n1);
        double part = 0.0;
        if constexpr (sizeof(E) == 4) {
          // FP32 storage: the squared norm is summed as an unevaluated pair of floats (exact products
          // by FMA, error-free two-sums: the Sum2 / Dot2 scheme of Ogita, Rump and Oishi, "Accurate
          // sum and dot product", SIAM J. Sci. Comput. 26, 2005), about 2^-48 relative for these
          // lengths, and turned into FP64 once per column: the FP64 pipe (2 FMA / clock / SM) would
          // otherwise take a conversion and an FMA per element on the chain every column waits for.
          float sh = 0.0f, sl = 0.0f;
          auto add_sq = [&](float x) {
            const float p = __fmul_rn(x, x), e = fmaf(x, x, -p);   // __fmul_rn: never contracted into an FMA
            const float s2 = sh + p, bb = s2 - sh;
            sl += ((sh - (s2 - bb)) + (p - bb)) + e;
            sh = s2;
          };
          if (refl) {
            float sum = 0.0f;
#pragma unroll 4
            for (int r = t0 + lane; r < t1; r += 32) sum += P[r + jj * lp] * P[r + c * lp];
            sum = warp_sum(sum);
            float* top = (mode == PM_GE) ? &P[jj + c * lp] : &Rt[jj + c * lrt];
            const float wv = *top + (float)se * sum;
            __syncwarp();
            if (lane == 0) *top = *top - (float)tauE * wv;
            const float tw = (float)tauE * wv * (float)se;
#pragma unroll 4
            for (int r = t0 + lane; r < t1; r += 32) {
              const float x = P[r + c * lp] - P[r + jj * lp] * tw;
              P[r + c * lp] = x;
              if (r >= n0 && r < n1) add_sq(x);
            }
          } else {
            for (int r = t0 + lane; r < t1; r += 32)
              if (r >= n0 && r < n1) add_sq(P[r + c * lp]);
          }
          for (int r = max(n0, t1) + lane; r < n1; r += 32) add_sq(P[r + c * lp]);   // rows of tail c outside tail jj
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(kFull, sh, o), ol = __shfl_xor_sync(kFull, sl, o);
            const float s2 = sh + oh, bb = s2 - sh;
            sl = sl + ol + ((sh - (s2 - bb)) + (oh - bb));
            sh = s2;
          }
          if (pairs) {
            __syncwarp();
            if (lane == 0) scalars_pair(c, sh, sl);
          } else {
            part = (double)sh + (double)sl;
          }
        } else {
          if (refl) {
            E sum = E(0);
            for (int r = t0 + lane; r < t1; r += 32) sum += P[r + jj * lp] * P[r + c * lp];
            sum = warp_sum(sum);
            E* top = (mode == PM_GE) ? &P[jj + c * lp] : &Rt[jj + c * lrt];
            const E wv = *top + se * sum;
            __syncwarp();
            if (lane == 0) *top = *top - tauE * wv;
            const E tw = tauE * wv * se;
            for (int r = t0 + lane; r < t1; r += 32) {
              const E x = P[r + c * lp] - P[r + jj * lp] * tw;
              P[r + c * lp] = x;
              if (r >= n0 && r < n1) part += (double)x * (double)x;
            }
          } else {
            for (int r = t0 + lane; r < t1; r += 32) {
              const double x = (double)P[r + c * lp];
              if (r >= n0 && r < n1) part += x * x;
            }
          }
          for (int r = max(n0, t1) + lane; r < n1; r += 32) {   // rows of tail c outside tail jj
            const double x = (double)P[r + c * lp];
            part += x * x;
          }
          part = warp_sum(part);
        }
        __syncwarp();
        if (lane == 0 && !pairs) scalars(c, part);
      }
    } else if (refl && sizeof(E) == 8) {   // FP64: one column per pass (the FP64 pipe is the limit)
      const E taue = tauE;
      for (int c = jj + 2 + (warp - 1); c < kb; c += kWarps - 1) {
        E sum = E(0);
        for (int r = t0 + lane; r < t1; r += 32) sum += P[r + jj * lp] * P[r + c * lp];
        sum = warp_sum(sum);
        E* top = (mode == PM_GE) ? &P[jj + c * lp] : &Rt[jj + c * lrt];
        const E wv = *top + se * sum;
        __syncwarp();
        if (lane == 0) *top = *top - taue * wv;
        const E tw = taue * wv * se;
        for (int r = t0 + lane; r < t1; r += 32) P[r + c * lp] -= P[r + jj * lp] * tw;
      }
    } else if (refl) {
      // FP32: two columns c and c + 7 per pass (independent, so their reductions overlap; a lone last
      // column is reduced twice); each column's arithmetic is the single-column form's
      const E taue = tauE;
      for (int c = jj + 2 + (warp - 1); c < kb; c += 2 * (kWarps - 1)) {
        const int c2 = c + (kWarps - 1);
        const bool two = c2 < kb;
        const int cb = two ? c2 : c;
        E sum = E(0), sum2 = E(0);
#pragma unroll 4
        for (int r = t0 + lane; r < t1; r += 32) {
          const E v = P[r + jj * lp];
          sum += v * P[r + c * lp];
          sum2 += v * P[r + cb * lp];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sum += __shfl_xor_sync(kFull, sum, o);
          sum2 += __shfl_xor_sync(kFull, sum2, o);
        }
        E* top = (mode == PM_GE) ? &P[jj + c * lp] : &Rt[jj + c * lrt];
        E* top2 = (mode == PM_GE) ? &P[jj + cb * lp] : &Rt[jj + cb * lrt];
        const E wv = *top + se * sum, wv2 = *top2 + se * sum2;
        __syncwarp();
        if (lane == 0) {
          *top = *top - taue * wv;
          if (two) *top2 = *top2 - taue * wv2;
        }
        const E tw = taue * wv * se, tw2 = taue * wv2 * se;
#pragma unroll 4
        for (int r = t0 + lane; r < t1; r += 32) {
          const E v = P[r + jj * lp];
          P[r + c * lp] -= v * tw;
          if (two) P[r + c2 * lp] -= v * tw2;
        }
      }
    }
    __syncthreads();
  }
  // scale the tails (float-pair scalars: x (sh + sl) rounded once, by an FMA residual; their tau also
  // goes to the FP64 array the T factor reads)
  for (int jj = warp; jj < kb; jj += kWarps) {
    int t0, t1;
    tail(jj, t0, t1);
    if (pairs) {
      const float sh = sch_s[jj], sl = scl_s[jj];
      if (lane == 0) tau_s[jj] = (double)tauf_s[jj];
      for (int r = t0 + lane; r < t1; r += 32) {
        const float x = (float)P[r + jj * lp], p = __fmul_rn(x, sh);
        P[r + jj * lp] = (E)__fadd_rn(p, fmaf(x, sl, fmaf(x, sh, -p)));
      }
    } else {
      const double sc = scale_s[jj];
      for (int r = t0 + lane; r < t1; r += 32) P[r + jj * lp] = (E)((double)P[r + jj * lp] * sc);
    }
  }
  __syncthreads();
}

// T factor (kb x kb, upper) of the kb reflectors in P, Q = H_0 ... H_{kb-1} = I - V T V^T.  G is
// 2 kb x kb scratch (the Gram matrix V^T V, then a work block).  The Gram entries are computed in 2 x 2
// blocks per thread (no cross-lane reductions).  T itself: the forward recurrence T[l,l] = tau_l,
// T[0:l, l] = -tau_l T[0:l, 0:l] G[0:l, l] inside diagonal blocks of 8 columns (all blocks at once),
// then blocks are merged pairwise, [T11 T12; 0 T22] with T12 = -T11 G12 T22 (the product of two compact
// WY blocks), so the sequential depth is 8 + 2 log2(kb/8) barrier steps instead of kb.
template <typename E>
__device__ void build_t(int mode, const E* P, int lp, int rows, int kb, int voff, const double* tau_s, E* Tb, int ldt,
                        E* G) {
  // reflector tail values: GE unit lower trapezoid, TS the full tail, TT the tail up to row voff + c
  auto vval = [&](int r, int c) -> E {
    if (mode == PM_GE) return r > c ? P[r + c * lp] : (r == c ? E(1) : E(0));
    if (mode == PM_TT && r > voff + c) return E(0);
    return P[r + c * lp];
  };
  const int nbk = (kb + 1) >> 1;
  const int nblocks = nbk * (nbk + 1) / 2;      // 2 x 2 blocks (bi <= bj) of the upper triangle
  for (int u = threadIdx.x; u < nblocks; u += kThreads) {
    int bj = 0, rem = u;
    while (rem > bj) { rem -= bj + 1; ++bj; }
    const int bi = rem;
    const int a0 = 2 * bi, l0 = 2 * bj;
    const int a1 = min(a0 + 1, kb - 1), l1 = min(l0 + 1, kb - 1);
    const int rlo = (mode == PM_GE) ? a0 : 0;
    const int rhi = (mode == PM_TT) ? min(rows, voff + l1 + 1) : rows;
    const int rplain = (mode == PM_GE) ? l1 + 1 : (mode == PM_TT ? min(rhi, voff + a0 + 1) : rhi);
    E s00 = E(0), s01 = E(0), s10 = E(0), s11 = E(0);
    int r = rlo;
    if (mode == PM_GE) {
      for (; r < min(rplain, rhi); ++r) {
        const E va0 = vval(r, a0), va1 = vval(r, a1), vl0 = vval(r, l0), vl1 = vval(r, l1);
        s00 += va0 * vl0; s01 += va0 * vl1; s10 += va1 * vl0; s11 += va1 * vl1;
      }
      for (; r < rhi; ++r) {
        const E va0 = P[r + a0 * lp], va1 = P[r + a1 * lp], vl0 = P[r + l0 * lp], vl1 = P[r + l1 * lp];
        s00 += va0 * vl0; s01 += va0 * vl1; s10 += va1 * vl0; s11 += va1 * vl1;
      }
    } else {
      for (; r < rplain; ++r) {
        const E va0 = P[r + a0 * lp], va1 = P[r + a1 * lp], vl0 = P[r + l0 * lp], vl1 = P[r + l1 * lp];
        s00 += va0 * vl0; s01 += va0 * vl1; s10 += va1 * vl0; s11 += va1 * vl1;
      }
      for (; r < rhi; ++r) {
        const E va0 = vval(r, a0), va1 = vval(r, a1), vl0 = vval(r, l0), vl1 = vval(r, l1);
        s00 += va0 * vl0; s01 += va0 * vl1; s10 += va1 * vl0; s11 += va1 * vl1;
      }
    }
    if (a0 < l0) G[a0 + l0 * kb] = s00;
    if (a0 < l1 && l1 != l0) G[a0 + l1 * kb] = s01;
    if (a1 < l0 && a1 != a0) G[a1 + l0 * kb] = s10;
    if (a1 < l1 && a1 != a0 && l1 != l0) G[a1 + l1 * kb] = s11;
  }
  __syncthreads();
  E* Y = G + kb * kb;
  constexpr int kB0 = 8;
  for (int o = threadIdx.x; o < kb * kb; o += kThreads) Tb[(o % kb) + (o / kb) * ldt] = E(0);
  __syncthreads();
  // diagonal blocks of kB0 columns: the forward recurrence, all blocks in parallel
  const int nblk0 = (kb + kB0 - 1) / kB0;
  for (int step = 0; step < kB0; ++step) {
    for (int u = threadIdx.x; u < nblk0 * kB0; u += kThreads) {
      const int d = u / kB0, a = d * kB0 + u % kB0, l = d * kB0 + step;
      if (l >= kb || a > l) continue;
      if (a == l) {
        Tb[l + l * ldt] = (E)tau_s[l];
      } else {
        E acc = E(0);
        for (int t = a; t < l; ++t) acc += Tb[a + t * ldt] * G[t + l * kb];
        Tb[a + l * ldt] = -(E)tau_s[l] * acc;
      }
    }
    __syncthreads();
  }
  // pairwise merges: T12 = -T11 (G12 T22) for blocks [c0, c0 + h) and [c0 + h, c1)
  for (int h = kB0; h < kb; h *= 2) {
    const int npair = (kb + 2 * h - 1) / (2 * h);
    for (int u = threadIdx.x; u < npair * h * h; u += kThreads) {     // Y = G12 T22
      const int pr = u / (h * h), i = (u % (h * h)) % h, j = (u % (h * h)) / h;
      const int c0 = pr * 2 * h, c1 = min(c0 + 2 * h, kb);
      if (c0 + h + j >= c1) continue;
      const int col = c0 + h + j;
      E acc = E(0);
      for (int t = c0 + h; t <= col; ++t) acc += G[(c0 + i) + t * kb] * Tb[t + col * ldt];
      Y[(c0 + i) + col * kb] = acc;
    }
    __syncthreads();
    for (int u = threadIdx.x; u < npair * h * h; u += kThreads) {     // T12 = -T11 Y
      const int pr = u / (h * h), i = (u % (h * h)) % h, j = (u % (h * h)) / h;
      const int c0 = pr * 2 * h, c1 = min(c0 + 2 * h, kb);
      if (c0 + h + j >= c1) continue;
      const int row = c0 + i, col = c0 + h + j;
      E acc = E(0);
      for (int t = row; t < c0 + h; ++t) acc += Tb[row + t * ldt] * Y[t + col * kb];
      Tb[row + col * ldt] = -acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------------
// Three-TF32 products on the tensor cores (mma.sync m16n8k8): x = hi + lo with hi the TF32 rounding of
// x and lo the TF32 rounding of x - hi; A B ~ A_lo B_hi + A_hi B_lo + A_hi B_hi in FP32.
// Fragment layout (lane = 4 g + t): A (16 x 8, row) a0 (g, t), a1 (g+8, t), a2 (g, t+4), a3 (g+8, t+4);
// B (8 x 8, col) b0 (t, g), b1 (t+4, g); C (16 x 8) c0 (g, 2t), c1 (g, 2t+1), c2 (g+8, 2t), c3 (g+8, 2t+1).
// ---------------------------------------------------------------------------------------------
// TF32 rounding of an FP32 value: round to nearest with ties away from zero to the 10 explicit mantissa
// bits of TF32, i.e. add half the weight of the 13 dropped bits to the magnitude and clear them.  Done
// on the integer units (the conversion instruction is a low-throughput one, and the split operands of
// an update strip make it the bottleneck of the contraction).  Finite inputs only (tile data).
__device__ __forceinline__ uint32_t tf32_round(float x) { return (__float_as_uint(x) + 0x1000u) & 0xffffe000u; }
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_round(x);
  lo = tf32_round(x - __uint_as_float(hi));    // x - hi is exact in FP32
}
__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// The tensor core's FP32 accumulation truncates, so one k8-step's three products go into a fresh
// accumulator that is then added to the running sum with a correctly rounded FP32 add: the truncation
// error stays relative to one step's partial sum instead of growing with K.
// A operand already split (hi / lo TF32 words), B split here.
__device__ __forceinline__ void mma_3xtf32(float* acc, const uint32_t* ah, const uint32_t* al, const float* b) {
  uint32_t bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) split_tf32(b[i], bh[i], bl[i]);
  float part[4] = {0.f, 0.f, 0.f, 0.f};
  mma_tf32(part, al, bh);
  mma_tf32(part, ah, bl);
  mma_tf32(part, ah, bh);
#pragma unroll
  for (int i = 0; i < 4; ++i) acc[i] += part[i];
}


// Block reflector application on row-major shared operands:
//   W = op(T) (Ct + V^T C),  Ct -= W,  C -= V W
// V: vrows x kb (ld lv), C: vrows x ncols, Ct: kb x ncols or null, W/W2: kb x ncols (ld lc); T is kb x kb
// column-major (ld kb).  op(T) = T^T applies Q^T (reflectors in increasing order), op(T) = T applies Q.
// FP64: register-blocked DFMA (phase 1: 1 column x 4 reflectors per thread, phase 3: 1 row x 8
// columns).  FP32: phases 1 and 3 on the tensor cores (three TF32 products) when kb and vrows are
// multiples of 16 and ncols of 8, register-blocked FFMA otherwise.
// Zero structure of an update block's V (oriented rows 0 .. vrows - 1, reflectors 0 .. kb - 1): none, unit
// lower triangle on top (GEQRT reflectors: V(r, a) = 0 for r < a), or upper triangle at the bottom (TTQRT
// reflectors: V(r, a) = 0 for r > vrows - kb + a).  The FP64 / FFMA phases skip those zeros.
enum TriShape : int { TRI_NONE = 0, TRI_UNITLOWER = 1, TRI_UPPER = 2 };

template <typename E>
__device__ void apply_phase1_simt(const E* V, int lv, int vrows, int kb, const E* Ct, const E* C, int lc, int ncols,
                                  E* W, int tri = TRI_NONE) {
  using V2 = typename Vec2<E>::type;
  if ((kb & 3) == 0) {
    const int nunits = ncols * (kb >> 2);
    for (int u = threadIdx.x; u < nunits; u += kThreads) {
      const int c = u % ncols, a0 = (u / ncols) << 2;
      E s0 = E(0), s1 = E(0), s2 = E(0), s3 = E(0);
      if (Ct) {
        s0 = Ct[a0 * lc + c]; s1 = Ct[(a0 + 1) * lc + c]; s2 = Ct[(a0 + 2) * lc + c]; s3 = Ct[(a0 + 3) * lc + c];
      }
      const E* vp = V + a0;
      const E* cp = C + c;
      // rows where reflectors a0 .. a0 + 3 are all zero are skipped (their terms are exact zeros)
      const int rb = tri == TRI_UNITLOWER ? a0 : 0;
      const int re = tri == TRI_UPPER ? vrows - kb + a0 + 4 : vrows;
#pragma unroll 4
      for (int r = rb; r < re; ++r) {
        const V2 v01 = *reinterpret_cast<const V2*>(vp + r * lv);
        const V2 v23 = *reinterpret_cast<const V2*>(vp + r * lv + 2);
        const E x = cp[r * lc];
        s0 = fma(v01.x, x, s0);
        s1 = fma(v01.y, x, s1);
        s2 = fma(v23.x, x, s2);
        s3 = fma(v23.y, x, s3);
      }
      W[a0 * lc + c] = s0;
      W[(a0 + 1) * lc + c] = s1;
      W[(a0 + 2) * lc + c] = s2;
      W[(a0 + 3) * lc + c] = s3;
    }
  } else {
    for (int u = threadIdx.x; u < ncols * kb; u += kThreads) {
      const int c = u % ncols, a = u / ncols;
      E s = Ct ? Ct[a * lc + c] : E(0);
      for (int r = 0; r < vrows; ++r) s = fma(V[r * lv + a], C[r * lc + c], s);
      W[a * lc + c] = s;
    }
  }
}

template <typename E>
__device__ void apply_phase3_simt(const E* V, int lv, int vrows, int kb, E* C, int lc, int ncols, const E* W2,
                                  int tri = TRI_NONE) {
  using V2 = typename Vec2<E>::type;
  if ((ncols & 7) == 0 && (kb & 1) == 0) {
    const int nunits = vrows * (ncols >> 3);
    for (int u = threadIdx.x; u < nunits; u += kThreads) {
      const int r = u % vrows, c0 = (u / vrows) << 3;
      V2* cp = reinterpret_cast<V2*>(C + r * lc + c0);
      V2 a0 = cp[0], a1 = cp[1], a2 = cp[2], a3 = cp[3];
      const E* vp = V + r * lv;
      // pairs of reflectors whose entries in row r are both zero are skipped
      const int ab = tri == TRI_UPPER ? max(0, r - (vrows - kb)) & ~1 : 0;
      const int ae = tri == TRI_UNITLOWER ? min(kb, (r + 2) & ~1) : kb;
#pragma unroll 2
      for (int a = ab; a < ae; a += 2) {
        const V2 v = *reinterpret_cast<const V2*>(vp + a);
        const V2* w0 = reinterpret_cast<const V2*>(W2 + a * lc + c0);
        const V2* w1 = reinterpret_cast<const V2*>(W2 + (a + 1) * lc + c0);
        const V2 x0 = w0[0], x1 = w0[1], x2 = w0[2], x3 = w0[3];
        const V2 y0 = w1[0], y1 = w1[1], y2 = w1[2], y3 = w1[3];
        a0.x = fma(-v.x, x0.x, a0.x); a0.y = fma(-v.x, x0.y, a0.y);
        a1.x = fma(-v.x, x1.x, a1.x); a1.y = fma(-v.x, x1.y, a1.y);
        a2.x = fma(-v.x, x2.x, a2.x); a2.y = fma(-v.x, x2.y, a2.y);
        a3.x = fma(-v.x, x3.x, a3.x); a3.y = fma(-v.x, x3.y, a3.y);
        a0.x = fma(-v.y, y0.x, a0.x); a0.y = fma(-v.y, y0.y, a0.y);
        a1.x = fma(-v.y, y1.x, a1.x); a1.y = fma(-v.y, y1.y, a1.y);
        a2.x = fma(-v.y, y2.x, a2.x); a2.y = fma(-v.y, y2.y, a2.y);
        a3.x = fma(-v.y, y3.x, a3.x); a3.y = fma(-v.y, y3.y, a3.y);
      }
      cp[0] = a0; cp[1] = a1; cp[2] = a2; cp[3] = a3;
    }
  } else {
    for (int u = threadIdx.x; u < vrows * ncols; u += kThreads) {
      const int r = u % vrows, c = u / vrows;
      E s = C[r * lc + c];
      for (int a = 0; a < kb; ++a) s = fma(-V[r * lv + a], W2[a * lc + c], s);
      C[r * lc + c] = s;
    }
  }
}

// Tensor-core phase 1 (FP32): W[a][c] = Ct[a][c] + sum_r V[r][a] C[r][c]; M = kb, N = ncols, K = vrows.
// Vh / Vl: the TF32 high / low parts of V (split_v_tf32).
__device__ void apply_phase1_tc(const float* Vh, const float* Vl, int lv, int vrows, int kb, const float* Ct,
                                const float* C, int lc, int ncols, float* W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt_n = kb >> 4, nt_n = ncols >> 3;
  for (int tile = warp; tile < mt_n * nt_n; tile += kWarps) {
    const int m0 = (tile % mt_n) << 4, n0 = (tile / mt_n) << 3;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (Ct) {
      acc[0] = Ct[(m0 + g) * lc + n0 + 2 * t];
      acc[1] = Ct[(m0 + g) * lc + n0 + 2 * t + 1];
      acc[2] = Ct[(m0 + g + 8) * lc + n0 + 2 * t];
      acc[3] = Ct[(m0 + g + 8) * lc + n0 + 2 * t + 1];
    }
#pragma unroll 4
    for (int k0 = 0; k0 < vrows; k0 += 8) {   // the three-product chains of 4 k-steps overlap
      const int i0 = (k0 + t) * lv + m0 + g, i1 = (k0 + t + 4) * lv + m0 + g;
      const uint32_t ah[4] = {__float_as_uint(Vh[i0]), __float_as_uint(Vh[i0 + 8]), __float_as_uint(Vh[i1]),
                              __float_as_uint(Vh[i1 + 8])};
      const uint32_t al[4] = {__float_as_uint(Vl[i0]), __float_as_uint(Vl[i0 + 8]), __float_as_uint(Vl[i1]),
                              __float_as_uint(Vl[i1 + 8])};
      const float b[2] = {C[(k0 + t) * lc + n0 + g], C[(k0 + t + 4) * lc + n0 + g]};
      mma_3xtf32(acc, ah, al, b);
    }
    W[(m0 + g) * lc + n0 + 2 * t] = acc[0];
    W[(m0 + g) * lc + n0 + 2 * t + 1] = acc[1];
    W[(m0 + g + 8) * lc + n0 + 2 * t] = acc[2];
    W[(m0 + g + 8) * lc + n0 + 2 * t + 1] = acc[3];
  }
}

// Tensor-core phase 3 (FP32): C[r][c] -= sum_a V[r][a] W2[a][c]; M = vrows, N = ncols, K = kb.  The
// product is formed as V (-W2), so the split V parts serve unchanged (TF32 rounding is symmetric).
__device__ void apply_phase3_tc(const float* Vh, const float* Vl, int lv, int vrows, int kb, float* C, int lc,
                                int ncols, const float* W2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt_n = vrows >> 4, np_n = (ncols + 15) >> 4;      // m-tiles, pairs of n-tiles
  // unit = one m-tile x two n-tiles: the A fragments of a k-step serve both n-tiles
  for (int u = warp; u < mt_n * np_n; u += kWarps) {
    const int m0 = (u % mt_n) << 4, n0 = (u / mt_n) << 4;
    const bool two = n0 + 8 < ncols;
    float* c00 = C + (m0 + g) * lc + n0 + 2 * t;
    float* c10 = C + (m0 + g + 8) * lc + n0 + 2 * t;
    float acc0[4] = {c00[0], c00[1], c10[0], c10[1]};
    float acc1[4] = {0.f, 0.f, 0.f, 0.f};
    if (two) {
      acc1[0] = c00[8]; acc1[1] = c00[9]; acc1[2] = c10[8]; acc1[3] = c10[9];
    }
#pragma unroll 4
    for (int k0 = 0; k0 < kb; k0 += 8) {
      const int i0 = (m0 + g) * lv + k0 + t, i1 = (m0 + g + 8) * lv + k0 + t;
      const uint32_t ah[4] = {__float_as_uint(Vh[i0]), __float_as_uint(Vh[i1]), __float_as_uint(Vh[i0 + 4]),
                              __float_as_uint(Vh[i1 + 4])};
      const uint32_t al[4] = {__float_as_uint(Vl[i0]), __float_as_uint(Vl[i1]), __float_as_uint(Vl[i0 + 4]),
                              __float_as_uint(Vl[i1 + 4])};
      const float b0[2] = {-W2[(k0 + t) * lc + n0 + g], -W2[(k0 + t + 4) * lc + n0 + g]};
      mma_3xtf32(acc0, ah, al, b0);
      if (two) {
        const float b1[2] = {-W2[(k0 + t) * lc + n0 + 8 + g], -W2[(k0 + t + 4) * lc + n0 + 8 + g]};
        mma_3xtf32(acc1, ah, al, b1);
      }
    }
    c00[0] = acc0[0];
    c00[1] = acc0[1];
    c10[0] = acc0[2];
    c10[1] = acc0[3];
    if (two) {
      c00[8] = acc1[0];
      c00[9] = acc1[1];
      c10[8] = acc1[2];
      c10[9] = acc1[3];
    }
  }
}

// FP32 storage applies a block on the tensor cores when the fragment shapes tile it exactly.
template <typename E>
__device__ __forceinline__ bool use_tc(bool simt, int kb, int vrows, int ncols) {
  return sizeof(E) == 4 && !simt && (kb & 15) == 0 && (vrows & 15) == 0 && (ncols & 7) == 0;
}

// Vh != null (FP32 storage, V loaded split by load_tile): phases 1 and 3 on the tensor cores with V = TF32 low parts and
// Vh = high parts; otherwise V holds the values and the phases run on the FMA units.
template <typename E>
__device__ void apply_rm(const E* V, const E* Vh, int lv, int vrows, int kb, const E* Tb, bool notrans, E* Ct, E* C,
                         int lc, int ncols, E* W, E* W2, int tri = TRI_NONE) {
  constexpr bool kF32 = sizeof(E) == 4;
  const bool tc = kF32 && Vh != nullptr;
  // phase 1
  if constexpr (kF32) {
    if (tc) apply_phase1_tc(Vh, V, lv, vrows, kb, Ct, C, lc, ncols, W);
    else apply_phase1_simt(V, lv, vrows, kb, Ct, C, lc, ncols, W, tri);
  } else {
    apply_phase1_simt(V, lv, vrows, kb, Ct, C, lc, ncols, W, tri);
  }
  __syncthreads();
  // phase 2: W2 = op(T) W, then Ct -= W2.  For kb = 32 and ncols = 32 each thread takes the rows
  // g, 31 - g, g + 8, 23 - g of one column (g = warp), so that every thread does 66 FMAs.
  if (kb == 32 && ncols == 32) {
    const int c = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int arow[4] = {g, 31 - g, g + 8, 23 - g};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int a = arow[q];
      E s = E(0);
      if (!notrans) {
        for (int t = 0; t <= a; ++t) s = fma(Tb[t + a * kb], W[t * lc + c], s);
      } else {
        for (int t = a; t < kb; ++t) s = fma(Tb[a + t * kb], W[t * lc + c], s);
      }
      W2[a * lc + c] = s;
      if (Ct) Ct[a * lc + c] -= s;
    }
  } else {
    for (int u = threadIdx.x; u < ncols * kb; u += kThreads) {
      const int c = u % ncols, a = u / ncols;
      E s = E(0);
      if (!notrans) {
        for (int t = 0; t <= a; ++t) s = fma(Tb[t + a * kb], W[t * lc + c], s);
      } else {
        for (int t = a; t < kb; ++t) s = fma(Tb[a + t * kb], W[t * lc + c], s);
      }
      W2[a * lc + c] = s;
      if (Ct) Ct[a * lc + c] -= s;
    }
  }
  __syncthreads();
  // phase 3: C -= V W2
  if constexpr (kF32) {
    if (tc) apply_phase3_tc(Vh, V, lv, vrows, kb, C, lc, ncols, W2);
    else apply_phase3_simt(V, lv, vrows, kb, C, lc, ncols, W2, tri);
  } else {
    apply_phase3_simt(V, lv, vrows, kb, C, lc, ncols, W2, tri);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Phase 3 of an FP32-storage block application on the 5th-generation tensor cores (tcgen05, kind::tf32):
// P = V (-W2) with V (vrows x kb) and -W2 (kb x ncols) split into TF32 high / low parts in shared memory
// in the K-major core-matrix layout (8 rows x 16 bytes per core matrix; element (row, k) at
// (row / 8) SBO + (k / 4) 128 B + (row % 8) 16 B + (k % 4) 4 B, SBO = kb / 4 x 128 B), the products
// accumulated in TMEM.  As in the warp-level form, each k-step of 8 gets its own accumulator holding its
// three products (lo hi, hi lo, hi hi), and the epilogue adds the k-steps to C with rounded FP32 adds in
// increasing k.  One thread issues the MMAs (M = 128 rows per chunk, N = ncols rounded up to 16) and
// commits them to an mbarrier; every thread waits (bounded), then each warp reads its 32 TMEM lanes.
// ---------------------------------------------------------------------------------------------
struct Umma {
  uint32_t tmem;      // TMEM base address of this CTA's allocation
  uint32_t mbar;      // shared-memory address of the completion mbarrier
  uint32_t phase;     // parity of the next completion
  uint32_t ncols_alloc;
  int failed;         // a completion wait ran out (the MMAs may still be in flight)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading-dimension byte offset >> 4
// (16-29: the step between core matrices along K), stride-dimension byte offset >> 4 (32-45: the step
// between 8-row groups), descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (7-9 and 10-12 = 2), both
// K-major, N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// Bounded wait for the mbarrier phase with the given parity; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = gtime();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (gtime() - t0 > limit_ns) return false;
  }
}
// 32 consecutive TMEM columns of this warp's 32 lanes into v (one column per register).
// 32 consecutive TMEM columns of this warp's 32 lanes into r (no wait: call tmem_wait_ld before use).
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Core-matrix index (in floats) of element (row, k) of a K-major operand with kb columns of K.
__device__ __forceinline__ int core_idx(int row, int k, int kb) {
  return (row >> 3) * (kb << 3) + ((k >> 2) << 5) + ((row & 7) << 2) + (k & 3);
}

// Phase 1 (warp-level tensor cores) reading V from the core-matrix layout: W = Ct + V^T C, with the C
// strip column-major (leading dimension ldc) and Ct, W row-major (lc).
__device__ void apply_phase1_tc_core(const float* Vh, const float* Vl, int vrows, int kb, const float* Ct,
                                     const float* C, int ldc, int lc, int ncols, float* W) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt_n = kb >> 4, nt_n = ncols >> 3, ntile = mt_n * nt_n;
  // kb = 32 (mt_n = 2 divides kWarps): tiles warp and warp + 8 share their 16 reflectors, so their V
  // fragments are read once per k-step; each tile keeps its own accumulation order.  Fragment rows g and
  // g + 8 stand for reflectors m0 + 2 g and m0 + 2 g + 1, adjacent in the core-matrix layout, so that each
  // pair of A registers is one 8-byte load (the row order of an MMA does not change its sums).
  for (int tile = warp; tile < ntile; tile += 2 * kWarps) {
    const int m0 = (tile % mt_n) << 4, n0 = (tile / mt_n) << 3;
    const int tile2 = tile + kWarps;
    const bool two = tile2 < ntile;
    const int n1 = two ? (tile2 / mt_n) << 3 : n0;
    const int ra = m0 + 2 * g, rb = ra + 1;   // reflectors of fragment rows g and g + 8
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, acc2[4] = {0.f, 0.f, 0.f, 0.f};
    if (Ct) {
      acc[0] = Ct[ra * lc + n0 + 2 * t];
      acc[1] = Ct[ra * lc + n0 + 2 * t + 1];
      acc[2] = Ct[rb * lc + n0 + 2 * t];
      acc[3] = Ct[rb * lc + n0 + 2 * t + 1];
      acc2[0] = Ct[ra * lc + n1 + 2 * t];
      acc2[1] = Ct[ra * lc + n1 + 2 * t + 1];
      acc2[2] = Ct[rb * lc + n1 + 2 * t];
      acc2[3] = Ct[rb * lc + n1 + 2 * t + 1];
    }
#pragma unroll 2
    for (int k0 = 0; k0 < vrows; k0 += 8) {
      const int i0 = core_idx(k0 + t, ra, kb), i1 = core_idx(k0 + t + 4, ra, kb);
      const uint2 h0 = *reinterpret_cast<const uint2*>(Vh + i0), h1 = *reinterpret_cast<const uint2*>(Vh + i1);
      const uint2 l0 = *reinterpret_cast<const uint2*>(Vl + i0), l1 = *reinterpret_cast<const uint2*>(Vl + i1);
      const uint32_t ah[4] = {h0.x, h0.y, h1.x, h1.y};
      const uint32_t al[4] = {l0.x, l0.y, l1.x, l1.y};
      const float b[2] = {C[(k0 + t) + (n0 + g) * ldc], C[(k0 + t + 4) + (n0 + g) * ldc]};
      mma_3xtf32(acc, ah, al, b);
      if (two) {
        const float b2[2] = {C[(k0 + t) + (n1 + g) * ldc], C[(k0 + t + 4) + (n1 + g) * ldc]};
        mma_3xtf32(acc2, ah, al, b2);
      }
    }
    W[ra * lc + n0 + 2 * t] = acc[0];
    W[ra * lc + n0 + 2 * t + 1] = acc[1];
    W[rb * lc + n0 + 2 * t] = acc[2];
    W[rb * lc + n0 + 2 * t + 1] = acc[3];
    if (two) {
      W[ra * lc + n1 + 2 * t] = acc2[0];
      W[ra * lc + n1 + 2 * t + 1] = acc2[1];
      W[rb * lc + n1 + 2 * t] = acc2[2];
      W[rb * lc + n1 + 2 * t + 1] = acc2[3];
    }
  }
}

// The whole block application W = op(T) (Ct + V^T C), Ct -= W, C -= V W with V in the core-matrix layout
// (Tb: op(T) column-major with leading dimension kb + 4, see phase 2)
// (load_v_core) and the C strip column-major (ldc; one row per lane in the epilogue is then free of bank
// conflicts): phase 1 on the warp-level tensor cores, phase 2 on the FMA units, phase 3 with tcgen05.
// Bh / Bl: kb x 64 floats each for the split -W2 operand.  Returns false if the MMA completion wait ran
// out (the error word is then set and C is left as it was).
__device__ bool apply_rm_umma(const float* Vh, const float* Vl, int vrows, int kb, const float* Tb, bool notrans,
                              float* Ct, float* C, int ldc, int lc, int ncols, float* W, float* W2, float* Bh,
                              float* Bl, Umma& um, const ExecParams& prm) {
  apply_phase1_tc_core(Vh, Vl, vrows, kb, Ct, C, ldc, lc, ncols, W);
  __syncthreads();
  // phase 2: S = op(T) W, then Ct -= S and -S, split, into the B operand of the tcgen05 phase (ncols rows
  // of K = kb, core-matrix layout).  Tb holds op(T) (T^T for Q^T, T for Q) column-major with leading
  // dimension kb + 4, its zeros included; a thread forms 4 consecutive rows a0..a0+3 of one column c, so
  // that op(T)(a0..a0+3, t) is one float4 and the 4 split values are one 16-byte store per part.  Each
  // sum runs in increasing t over the triangle's range (the extra terms multiply stored zeros).
  const int npad = (ncols + 15) & ~15;
  {
    const int lt = kb + 4, lg = 31 - __clz(ncols);            // ncols in {32, 64}
    for (int u = threadIdx.x; u < ncols * (kb >> 2); u += kThreads) {
      const int c = u & (ncols - 1), a0 = (u >> lg) << 2;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const int tlo = notrans ? a0 : 0, thi = notrans ? kb : a0 + 4;
      for (int t = tlo; t < thi; ++t) {
        const float wv = W[t * lc + c];
        const float4 tv = *reinterpret_cast<const float4*>(Tb + a0 + t * lt);
        acc[0] = fmaf(tv.x, wv, acc[0]);
        acc[1] = fmaf(tv.y, wv, acc[1]);
        acc[2] = fmaf(tv.z, wv, acc[2]);
        acc[3] = fmaf(tv.w, wv, acc[3]);
      }
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (Ct) Ct[(a0 + k) * lc + c] -= acc[k];
        split_tf32(-acc[k], hi[k], lo[k]);
      }
      const int bi = core_idx(c, a0, kb);
      *reinterpret_cast<uint4*>(Bh + bi) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(Bl + bi) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
  }
  for (int u = threadIdx.x; u < (npad - ncols) * kb; u += kThreads) {   // zero rows of the padded N
    const int c = ncols + u / kb, a = u % kb;
    Bl[core_idx(c, a, kb)] = 0.f;
    Bh[core_idx(c, a, kb)] = 0.f;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy smem writes -> MMA reads
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int nks = kb >> 3, mch = (vrows + 127) >> 7;
  if (threadIdx.x == 0) {
    const uint32_t sbo = (uint32_t)(kb >> 2) * 128u, idesc = umma_idesc_tf32(128, npad);
    const uint32_t vh = smem_u32(Vh), vl = smem_u32(Vl), bh = smem_u32(Bh), bl = smem_u32(Bl);
    for (int mc = 0; mc < mch; ++mc)
      for (int ks = 0; ks < nks; ++ks) {
        const uint32_t d = um.tmem + (uint32_t)((mc * nks + ks) * npad);
        const uint32_t ao = (uint32_t)mc * 16u * sbo + (uint32_t)ks * 256u, bo = (uint32_t)ks * 256u;
        umma_tf32(d, umma_desc(vl + ao, 128, sbo), umma_desc(bh + bo, 128, sbo), idesc, 0);
        umma_tf32(d, umma_desc(vh + ao, 128, sbo), umma_desc(bl + bo, 128, sbo), idesc, 1);
        umma_tf32(d, umma_desc(vh + ao, 128, sbo), umma_desc(bh + bo, 128, sbo), idesc, 1);
      }
    umma_commit(um.mbar);
  }
  const bool ok = __syncthreads_and(mbar_wait(um.mbar, um.phase, prm.wait_ns) ? 1 : 0) != 0;
  um.phase ^= 1u;
  if (!ok) {
    if (threadIdx.x == 0) atomicCAS(prm.err, 0, DERR_TIMEOUT);
    um.failed = 1;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, mc = warp >> 2, q = warp & 3;
  if (ok && mc < mch) {
    const int r = mc * 128 + q * 32 + lane;
    for (int cg = 0; cg < ncols; cg += 32) {
      float acc[32];
      const int nc = min(32, ncols - cg);
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = (r < vrows && j < nc) ? C[r + (cg + j) * ldc] : 0.f;
      // two k-steps per TMEM round trip; the adds stay in increasing k
      for (int ks = 0; ks < nks; ks += 2) {
        const uint32_t ta = um.tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((mc * nks + ks) * npad + cg);
        uint32_t p0[32], p1[32];
        tmem_ld32_nowait(ta, p0);
        if (ks + 1 < nks) tmem_ld32_nowait(ta + (uint32_t)npad, p1);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += __uint_as_float(p0[j]);
        if (ks + 1 < nks) {
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[j] += __uint_as_float(p1[j]);
        }
      }
      if (r < vrows) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nc) C[r + (cg + j) * ldc] = acc[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  return ok;
}

// ---------------------------------------------------------------------------------------------
// Panel factor sub-task PF(b): factors inner block b (columns b*ib .. b*ib + ib - 1) of a panel task
// and writes its reflectors in place and its T block.  GE: rows b*ib .. nb-1 of tile X.  TS: the
// triangle of pivot tile A's diagonal block b over all rows of X.  TT: the same triangle over the upper
// part of X (rows 0 .. b*ib + ib - 1).  The later column blocks are updated by PU sub-tasks.
// ---------------------------------------------------------------------------------------------
template <typename E>
__device__ void task_panel_factor(unsigned char* smb, int kind, E* X, E* A, int tr, E* Tg, int nb, int ib, int b,
                                  bool pair_scalars) {
  const Layout L = layout_panel(nb, ib, (int)sizeof(E));
  double* tau = reinterpret_cast<double*>(smb);
  double* red = tau + 64;
  E* sm = reinterpret_cast<E*>(smb + kHeaderDoubles * sizeof(double));
  E *P = sm + L.P, *Rt = sm + L.Rt, *Tb = sm + L.Tb, *G = sm + L.G;
  const int c0 = b * ib, kb = ib;
  if (kind == PM_GE) {
    const int rows = nb - c0;
    load_tile(P, 1, L.lp, X, nb, tr, c0, c0, rows, kb, M_NONE);
    __syncthreads();
    factor_panel(PM_GE, P, L.lp, rows, kb, (E*)nullptr, 0, 0, tau, red, pair_scalars);
    build_t(PM_GE, P, L.lp, rows, kb, 0, tau, Tb, kb, G);
    store_tile(P, 1, L.lp, X, nb, tr, c0, c0, rows, kb, M_NONE);
  } else {
    const bool tt = kind == PM_TT;
    const int vrows = tt ? c0 + kb : nb;
    load_tile(Rt, 1, kb, A, nb, tr, c0, c0, kb, kb, M_UPPER);
    load_tile(P, 1, L.lp, X, nb, tr, 0, c0, vrows, kb, tt ? M_UPPER : M_NONE);
    __syncthreads();
    factor_panel(kind, P, L.lp, vrows, kb, Rt, kb, c0, tau, red, pair_scalars);
    build_t(kind, P, L.lp, vrows, kb, c0, tau, Tb, kb, G);
    store_tile(Rt, 1, kb, A, nb, tr, c0, c0, kb, kb, M_UPPER);
    store_tile(P, 1, L.lp, X, nb, tr, 0, c0, vrows, kb, tt ? M_UPPER : M_NONE);
  }
  for (int o = threadIdx.x; o < kb * kb; o += kThreads) stg(Tg + (size_t)c0 * ib + o, Tb[o]);
}

// Applies reflector blocks [blk0, blk1) of V tile X (UNMQR: GEQRT reflectors; TSMQR: TSQRT reflectors
// over [Cp; C]; TTMQR: TTQRT reflectors) to columns [col0, col0 + ncols) of the C tiles (oriented), in
// increasing block order for Q^T and decreasing for Q.  Only the rows the blocks touch are loaded and
// written: rows blk0*ib .. nb-1 of C (UNMQR), all rows of C (TSMQR), rows 0 .. blk1*ib - 1 of C
// (TTMQR), and rows b*ib .. b*ib + ib - 1 of Cp for each block b.  The C rows stay in shared memory.
// With blk0 = b, blk1 = b + 1 and C = X this is the PU(b, s) sub-task of a panel.
template <typename E>
__device__ void task_update(unsigned char* smb, int type, const E* X, E* Cp, E* C, int tr, bool notrans, const E* Tg,
                            int nb, int ib, int w, int blk0, int blk1, int col0, int ncols, bool simt) {
  const Layout L = layout_update(nb, ib, w, (int)sizeof(E));
  E* sm = reinterpret_cast<E*>(smb + kHeaderDoubles * sizeof(double));
  E *Cs = sm + L.Cs, *Ct = sm + L.Ct, *V = sm + L.V, *Tb = sm + L.Tb, *W = sm + L.W, *W2 = sm + L.W2;
  const int row_lo = (type == UNMQR) ? blk0 * ib : 0;
  const int row_hi = (type == TTMQR) ? blk1 * ib : nb;
  load_tile(Cs + row_lo * L.lc, L.lc, 1, C, nb, tr, row_lo, col0, row_hi - row_lo, ncols, M_NONE);
  const int nbk = blk1 - blk0;
  for (int bb = 0; bb < nbk; ++bb) {
    const int b = notrans ? blk1 - 1 - bb : blk0 + bb;
    const int c0 = b * ib, kb = ib;
    int vrows;
    E* Cb;
    E* Ctop = nullptr;
    // T's loads are issued first so that their latency overlaps the loads of V
    E tv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int o = threadIdx.x + k * kThreads;
      tv[k] = o < kb * kb ? ldg(Tg + (size_t)c0 * ib + o) : E(0);
    }
    vrows = (type == UNMQR) ? nb - c0 : ((type == TSMQR) ? nb : c0 + kb);
    E* Vh = (L.Vh >= 0 && use_tc<E>(simt, kb, vrows, ncols)) ? sm + L.Vh : nullptr;
    if (type == UNMQR) {
      load_tile(V, L.lv, 1, X, nb, tr, c0, c0, vrows, kb, M_UNITLOWER, Vh);
      Cb = Cs + c0 * L.lc;
    } else {
      load_tile(V, L.lv, 1, X, nb, tr, 0, c0, vrows, kb, type == TSMQR ? M_NONE : M_UPPER, Vh);
      load_tile(Ct, L.lc, 1, Cp, nb, tr, c0, col0, kb, ncols, M_NONE);
      Ctop = Ct;
      Cb = Cs;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int o = threadIdx.x + k * kThreads;
      if (o < kb * kb) Tb[o] = tv[k];
    }
    for (int o = threadIdx.x + 4 * kThreads; o < kb * kb; o += kThreads) Tb[o] = ldg(Tg + (size_t)c0 * ib + o);
    __syncthreads();
    apply_rm(V, Vh, L.lv, vrows, kb, Tb, notrans, Ctop, Cb, L.lc, ncols, W, W2,
             type == UNMQR ? TRI_UNITLOWER : (type == TTMQR ? TRI_UPPER : TRI_NONE));
    if (Ctop) {
      store_tile(Ct, L.lc, 1, Cp, nb, tr, c0, col0, kb, ncols, M_NONE);
      __syncthreads();
    }
  }
  store_tile(Cs + row_lo * L.lc, L.lc, 1, C, nb, tr, row_lo, col0, row_hi - row_lo, ncols, M_NONE);
}

// Shared-memory layout of the tcgen05 update path (FP32 storage): the C strip column-major (ldc = nb + 4),
// Ct and W row-major (lc), V split into TF32 high / low parts in the core-matrix layout, op(T) (ld ib + 4),
// the split -op(T) W operand, and staging buffers that receive the next block's raw V (column-major ld nb,
// or row-major ld ib + 4 for transposed tiles), T (ib x ib, as stored) and Ct (column-major ld ib + 4, or
// row-major lc for transposed tiles) while the current block is applied.  Offsets in floats.
struct UmmaLayout {
  int ldc, lc, Cs, Ct, Vl, Vh, Vr, Tb, W, B, Tr, Cr, total;
};
__host__ __device__ inline UmmaLayout layout_umma(int nb, int ib, int w) {
  UmmaLayout L{};
  const int wc = w > ib ? w : ib;
  L.ldc = nb + 4;
  L.lc = rm_ld(wc, 4);
  int o = 0;
  L.Cs = o;  o = align32(o + L.ldc * wc);
  L.Ct = o;  o = align32(o + ib * L.lc);
  L.Vl = o;  o = align32(o + nb * ib);
  L.Vh = o;  o = align32(o + nb * ib);
  L.Vr = o;  o = align32(o + nb * (ib + 4));
  L.Tb = o;  o = align32(o + ib * (ib + 4));
  L.W = o;   o = align32(o + ib * L.lc);
  L.B = o;   o = align32(o + 2 * ib * ((wc + 15) / 16 * 16));
  L.Tr = o;  o = align32(o + ib * ib);
  L.Cr = o;  o = align32(o + max(wc * (ib + 4), ib * L.lc));
  L.total = o;
  return L;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Starts the copy of V block (oriented X(r0 + r, c0 + a), r < vrows, a < kb) into the staging buffer Vr in
// 16-byte pieces (one commit group): column-major (ld nb) for tr = 0, row-major (ld kb + 4) for tr = 1.
__device__ void prefetch_v(float* Vr, const float* X, int nb, int tr, int r0, int c0, int vrows, int kb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!tr) {   // warp per column, lanes along the rows (kb = 32: 4 columns per warp)
    for (int a = warp; a < kb; a += kWarps)
      for (int r = lane << 2; r < vrows; r += 128) cp_async16(Vr + a * nb + r, X + (r0 + r) + (size_t)(c0 + a) * nb);
  } else {     // 8 threads per row of kb = 32 columns
    const int a = (threadIdx.x & 7) << 2;
    for (int r = threadIdx.x >> 3; r < vrows; r += kThreads >> 3)
      cp_async16(Vr + r * (kb + 4) + a, X + (size_t)(r0 + r) * nb + c0 + a);
  }
}

// Starts the copies of a block's T (kb x kb, contiguous) into Tr and of Ct = oriented Cp(c0 + r, col0 + c),
// r < kb, c < ncols, into Cr: column-major ld kb + 4 for tr = 0 (16-byte pieces along r), row-major ld lc
// for tr = 1 (pieces along c).
__device__ void prefetch_t_ct(float* Tr, const float* T, float* Cr, const float* Cp, int nb, int tr, int c0, int col0,
                              int kb, int ncols, int lc) {
  for (int q = threadIdx.x; q < (kb * kb) >> 2; q += kThreads) cp_async16(Tr + 4 * q, T + 4 * q);
  if (!Cp) return;
  const int nch = (kb * ncols) >> 2;            // kb = 32, ncols 32 or 64
  const int lq = ncols == 64 ? 4 : 3;           // log2(ncols / 4)
  for (int q = threadIdx.x; q < nch; q += kThreads) {
    if (!tr) {
      const int c = q >> 3, r = (q & 7) << 2;
      cp_async16(Cr + c * (kb + 4) + r, Cp + (c0 + r) + (size_t)(col0 + c) * nb);
    } else {
      const int r = q >> lq, c = (q & ((1 << lq) - 1)) << 2;
      cp_async16(Cr + r * lc + c, Cp + (size_t)(c0 + r) * nb + col0 + c);
    }
  }
}

// Starts the copy of the C strip (oriented C(r, col0 + c), r0 <= r < r1, c < ncols) into Cs column-major
// (ld ldc): 16-byte pieces along r for tr = 0, 4-byte pieces (coalesced along c) for tr = 1.
__device__ void prefetch_c(float* Cs, int ldc, const float* C, int nb, int tr, int r0, int r1, int col0, int ncols) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!tr) {   // warp per column, lanes along the rows
    for (int c = warp; c < ncols; c += kWarps)
      for (int r = r0 + (lane << 2); r < r1; r += 128) cp_async16(Cs + c * ldc + r, C + r + (size_t)(col0 + c) * nb);
  } else {     // warp per row, lanes along the columns
    for (int r = r0 + warp; r < r1; r += kWarps)
      for (int c = lane; c < ncols; c += 32) cp_async4(Cs + c * ldc + r, C + (size_t)r * nb + col0 + c);
  }
}

// Staged V block -> TF32 high / low parts in the core-matrix layout, with the mask of load_tile applied in
// oriented coordinates (R = r0 + r, C = c0 + a).  A thread handles 4 consecutive a of one row: one
// 16-byte core row per part.
__device__ void split_v_core(const float* Vr, float* Vl, float* Vh, int nb, int tr, int r0, int c0, int vrows,
                             int kb, int mask) {
  // kb = 32: warp w takes columns a0 = 4 w .. 4 w + 3, lanes along the rows
  const int a0 = (threadIdx.x >> 5) << 2;
  for (int r = threadIdx.x & 31; r < vrows; r += 32) {
    float x[4];
    if (tr) {
      const float4 v = *reinterpret_cast<const float4*>(Vr + r * (kb + 4) + a0);
      x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = Vr[(a0 + k) * nb + r];
    }
    uint32_t hi[4], lo[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int R = r0 + r, C = c0 + a0 + k;
      if (mask == M_UPPER && R > C) x[k] = 0.f;
      if (mask == M_UNITLOWER && R <= C) x[k] = (R == C) ? 1.f : 0.f;
      split_tf32(x[k], hi[k], lo[k]);
    }
    const int ci = core_idx(r, a0, kb);
    *reinterpret_cast<uint4*>(Vh + ci) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(Vl + ci) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

// FP32-storage update (strip or panel-block update, as task_update) with phase 3 on tcgen05; the next
// block's V is copied (cp.async) while the current block is applied.  Used when the CTA holds TMEM for it
// (ExecParams::umma_cols) and the shapes fit (ib 32, 32 or 64 columns: the epilogue reads TMEM 32
// columns at a time); returns false when it does not apply (the caller then runs task_update).
__device__ bool task_update_umma(unsigned char* smb, int type, const float* X, float* Cp, float* C, int tr,
                                 bool notrans, const float* Tg, int nb, int ib, int w, int blk0, int blk1, int col0,
                                 int ncols, Umma& um, const ExecParams& prm) {
  const int kb = ib;
  const int npad = (ncols + 15) & ~15;
  if (um.ncols_alloc == 0 || kb != 32 || (nb & 15) || (ncols & 31) || ncols > 64 || ncols > (w > ib ? w : ib) ||
      ((nb + 127) >> 7) * (kb >> 3) * npad > (int)um.ncols_alloc)
    return false;
  const UmmaLayout L = layout_umma(nb, ib, w);
  float* sm = reinterpret_cast<float*>(smb + kHeaderDoubles * sizeof(double));
  float *Cs = sm + L.Cs, *Ct = sm + L.Ct, *Vl = sm + L.Vl, *Vh = sm + L.Vh, *Vr = sm + L.Vr, *Tb = sm + L.Tb;
  float *W = sm + L.W, *Bl = sm + L.B, *Bh = Bl + kb * npad, *Tr = sm + L.Tr, *Cr = sm + L.Cr;
  if ((smem_u32(Vl) | smem_u32(Vh) | smem_u32(Bl) | smem_u32(Bh)) & 127) return false;
  const int ldc = L.ldc, lc = L.lc;
  const int row_lo = (type == UNMQR) ? blk0 * ib : 0;
  const int row_hi = (type == TTMQR) ? blk1 * ib : nb;
  const int nbk = blk1 - blk0;
  const bool top = type != UNMQR;   // TSMQR / TTMQR: the pivot tile's rows of the block are updated too
  auto blk_of = [&](int bb) { return notrans ? blk1 - 1 - bb : blk0 + bb; };
  auto rows_of = [&](int c0) { return (type == UNMQR) ? nb - c0 : ((type == TSMQR) ? nb : c0 + kb); };
  auto r0_of = [&](int c0) { return (type == UNMQR) ? c0 : 0; };
  auto prefetch_block = [&](int c0) {
    prefetch_v(Vr, X, nb, tr, r0_of(c0), c0, rows_of(c0), kb);
    prefetch_t_ct(Tr, Tg + (size_t)c0 * ib, Cr, top ? Cp : nullptr, nb, tr, c0, col0, kb, ncols, lc);
    cp_async_commit();
  };
  prefetch_c(Cs, ldc, C, nb, tr, row_lo, row_hi, col0, ncols);
  prefetch_block(blk_of(0) * ib);
  for (int bb = 0; bb < nbk; ++bb) {
    const int b = blk_of(bb);
    const int c0 = b * ib, vrows = rows_of(c0);
    cp_async_wait_all();
    __syncthreads();                       // this block's V, T, Ct (and the C strip) are staged
    split_v_core(Vr, Vl, Vh, nb, tr, r0_of(c0), c0, vrows, kb,
                 type == UNMQR ? M_UNITLOWER : (type == TSMQR ? M_NONE : M_UPPER));
    for (int o = threadIdx.x; o < kb * kb; o += kThreads) {   // op(T) column-major, ld kb + 4 (kb = 32)
      const int r = o & 31, c = o >> 5;
      Tb[notrans ? r + c * (kb + 4) : c + r * (kb + 4)] = Tr[o];
    }
    if (top) {   // lanes along the columns: the row-major stores are conflict-free
      const int lgc = ncols == 64 ? 6 : 5;
      for (int o = threadIdx.x; o < kb * ncols; o += kThreads) {
        const int c = o & (ncols - 1), r = o >> lgc;
        Ct[r * lc + c] = tr ? Cr[r * lc + c] : Cr[c * (kb + 4) + r];
      }
    }
    __syncthreads();                       // the staging buffers are free again
    if (bb + 1 < nbk) prefetch_block(blk_of(bb + 1) * ib);
    if (!apply_rm_umma(Vh, Vl, vrows, kb, Tb, notrans, top ? Ct : nullptr, top ? Cs : Cs + c0, ldc, lc, ncols, W, W,
                       Bh, Bl, um, prm)) {
      // the MMA completion wait ran out (the error word is set): no further MMA is issued, the copies
      // in flight are waited for, and nothing is written back
      cp_async_wait_all();
      __syncthreads();
      return true;
    }
    if (top) {
      store_tile(Ct, lc, 1, Cp, nb, tr, c0, col0, kb, ncols, M_NONE);
      __syncthreads();
    }
  }
  store_tile(Cs + row_lo, 1, ldc, C, nb, tr, row_lo, col0, row_hi - row_lo, ncols, M_NONE);
  return true;
}

// ---------------------------------------------------------------------------------------------
// Adjoint of the reduction (reverse sweep).  Each Householder step of the forward sweep is
// M' = H(x) M on the rows it acts on, H = I - tau v v^T, x its pivot column, H x = beta e_1.  Going
// backwards with the gradient G' of M':  M = H M' (H is its own inverse), G = H G', and the
// reflector's derivatives  tau_bar = -a.b,  v_bar = -tau (G' a + M b)  with a = M^T v, b = G'^T v,
// summed over every column the reflector was applied to, then pushed through house() into the pivot
// column.  For a compact-WY block (V, T) applied to columns C as C' = Q^T C, Q = I - V T V^T:
//   undoing it is C = Q C' (T applied as T: W2s = T V^T C' = -Z with Z_k = tau_k v_k^T M_k),
//   the gradient is G = Q G' (W2g = T V^T G' = Y with Y_k = tau_k v_k^T G_k),
// where M_k / G_k are the column states around reflector k.  Writing M_k and G_k through V, Z, Y
// gives, for the reflectors of the block,
//   v_bar_k = -(P')_k + sum_{l <= k} v_l D_lk,   tau_bar_k = -S_kk / tau_k^2,
//   P' = C W2g^T - G W2s^T (pre-step state and gradient),  S = -W2g W2s^T,
//   D_lk = S_kl - S_lk (l < k),  D_kk = -S_kk,
// all sums over columns, so every column chunk adds its P' and S to a partial slot.
// ---------------------------------------------------------------------------------------------
template <typename E>
__device__ void bwd_partial(const E* Cs, const E* Cg, int lc, int vrows, int kb, int nc, const E* W2s, const E* W2g,
                            E* P, E* S, bool accumulate) {
  if ((kb & 3) == 0) {
    const int nunits = vrows * (kb >> 2);
    for (int u = threadIdx.x; u < nunits; u += kThreads) {
      const int r = u % vrows, k0 = (u / vrows) << 2;
      E a0 = E(0), a1 = E(0), a2 = E(0), a3 = E(0);
      const E* cs = Cs + r * lc;
      const E* cg = Cg + r * lc;
      for (int c = 0; c < nc; ++c) {
        const E x = cs[c], y = -cg[c];
        a0 = fma(x, W2g[k0 * lc + c], fma(y, W2s[k0 * lc + c], a0));
        a1 = fma(x, W2g[(k0 + 1) * lc + c], fma(y, W2s[(k0 + 1) * lc + c], a1));
        a2 = fma(x, W2g[(k0 + 2) * lc + c], fma(y, W2s[(k0 + 2) * lc + c], a2));
        a3 = fma(x, W2g[(k0 + 3) * lc + c], fma(y, W2s[(k0 + 3) * lc + c], a3));
      }
      E* pp = P + (size_t)r * kb + k0;
      if (accumulate) {
        a0 += ldg(pp); a1 += ldg(pp + 1); a2 += ldg(pp + 2); a3 += ldg(pp + 3);
      }
      stg(pp, a0); stg(pp + 1, a1); stg(pp + 2, a2); stg(pp + 3, a3);
    }
  } else {
    for (int u = threadIdx.x; u < vrows * kb; u += kThreads) {
      const int r = u % vrows, k = u / vrows;
      E a = E(0);
      for (int c = 0; c < nc; ++c) a = fma(Cs[r * lc + c], W2g[k * lc + c], fma(-Cg[r * lc + c], W2s[k * lc + c], a));
      E* pp = P + (size_t)r * kb + k;
      if (accumulate) a += ldg(pp);
      stg(pp, a);
    }
  }
  for (int u = threadIdx.x; u < kb * kb; u += kThreads) {
    const int a = u / kb, k = u % kb;
    E v = E(0);
    for (int c = 0; c < nc; ++c) v = fma(-W2g[a * lc + c], W2s[k * lc + c], v);
    if (accumulate) v += ldg(S + u);
    stg(S + u, v);
  }
}

// Sum of the update-strip partials of panel block b over rows [chunk R, (chunk + 1) R) of its P'
// (R = kRedElems / ib, clipped to the block's vrows rows) and, with chunk 0, of its S block, in slot
// order and in FP64, into the panel's reduced slot `out` (laid out as an update slot).  Each thread
// keeps kRedPer independent sums, so that kRedPer loads per slot are in flight at once.
constexpr int kRedPer = kRedElems / kThreads;
template <typename E>
__device__ void task_bwd_reduce(int nb, int ib, int b, int chunk, int vrows, const E* part, const int64_t* slot_off,
                                int u0, int nu, E* out) {
  const int kb = ib, nblk = nb / ib, rows = max(1, kRedElems / kb);
  const int r0 = chunk * rows, r1 = min(vrows, r0 + rows);
  const size_t pblk = (size_t)b * nb * ib, sblk = (size_t)nblk * nb * ib + (size_t)b * kb * kb;
  const int o0 = r0 * kb, o1 = r1 * kb;    // element (r, k) of the block at pblk + r kb + k
  double acc[kRedPer];
#pragma unroll
  for (int j = 0; j < kRedPer; ++j) acc[j] = 0.0;
  for (int i = 0; i < nu; ++i) {
    const E* src = part + slot_off[u0 + i] + pblk;
#pragma unroll
    for (int j = 0; j < kRedPer; ++j) {
      const int o = o0 + (int)threadIdx.x + j * kThreads;
      if (o < o1) acc[j] += (double)ldg(src + o);
    }
  }
#pragma unroll
  for (int j = 0; j < kRedPer; ++j) {
    const int o = o0 + (int)threadIdx.x + j * kThreads;
    if (o < o1) stg(out + pblk + o, (E)acc[j]);
  }
  if (chunk == 0) {
    for (int o = threadIdx.x; o < kb * kb; o += kThreads) {
      double s = 0.0;
      for (int i = 0; i < nu; ++i) s += (double)ldg(part + slot_off[u0 + i] + sblk + o);
      stg(out + sblk + o, (E)s);
    }
  }
}

// Adjoint of an update (UNMQR / TSMQR / TTMQR strip, or PU(b, s) with C = the panel tile): blocks
// [blk0, blk1) are undone in decreasing order on the state (C_s, Cp_s) and the gradient (C_g, Cp_g) of
// columns [col0, col0 + ncols), chunk by chunk, and each block's P' (vrows x ib, row-major) and S
// (ib x ib) go to the slot: block beta at (beta - blk0) nb ib, its S after all P blocks.
template <typename E>
__device__ void task_bwd_update(unsigned char* smb, int type, const E* X, E* Cp_s, E* C_s, E* Cp_g, E* C_g, int tr,
                                const E* Tg, int nb, int ib, int hw, int blk0, int blk1, int col0, int ncols, E* slot,
                                bool simt) {
  const BwdLayout L = layout_bwd_update(nb, ib, hw, (int)sizeof(E));
  E* sm = reinterpret_cast<E*>(smb + kHeaderDoubles * sizeof(double));
  E *Cs = sm + L.Cs, *Cg = sm + L.Cg, *Cts = sm + L.Cts, *Ctg = sm + L.Ctg, *V = sm + L.V, *Tb = sm + L.Tb;
  E *W = sm + L.W, *W2s = sm + L.W2s, *W2g = sm + L.W2g;
  const int lc = L.lc, lv = L.lv;
  const int row_lo = (type == UNMQR) ? blk0 * ib : 0;
  const int row_hi = (type == TTMQR) ? blk1 * ib : nb;
  const int nbk = blk1 - blk0;
  const size_t pstride = (size_t)nb * ib, sbase = (size_t)nbk * nb * ib;
  for (int ch = 0; ch < ncols; ch += hw) {
    const int nc = min(hw, ncols - ch);
    load_tile(Cs + row_lo * lc, lc, 1, C_s, nb, tr, row_lo, col0 + ch, row_hi - row_lo, nc, M_NONE);
    load_tile(Cg + row_lo * lc, lc, 1, C_g, nb, tr, row_lo, col0 + ch, row_hi - row_lo, nc, M_NONE);
    for (int bb = 0; bb < nbk; ++bb) {
      const int b = blk1 - 1 - bb;
      const int c0 = b * ib, kb = ib;
      E *Cbs, *Cbg, *Tops = nullptr, *Topg = nullptr;
      const int vrows = (type == UNMQR) ? nb - c0 : ((type == TSMQR) ? nb : c0 + kb);
      E* Vh = (L.Vh >= 0 && use_tc<E>(simt, kb, vrows, nc)) ? sm + L.Vh : nullptr;
      if (type == UNMQR) {
        load_tile(V, lv, 1, X, nb, tr, c0, c0, vrows, kb, M_UNITLOWER, Vh);
        Cbs = Cs + c0 * lc;
        Cbg = Cg + c0 * lc;
      } else {
        load_tile(V, lv, 1, X, nb, tr, 0, c0, vrows, kb, type == TSMQR ? M_NONE : M_UPPER, Vh);
        load_tile(Cts, lc, 1, Cp_s, nb, tr, c0, col0 + ch, kb, nc, M_NONE);
        load_tile(Ctg, lc, 1, Cp_g, nb, tr, c0, col0 + ch, kb, nc, M_NONE);
        Tops = Cts;
        Topg = Ctg;
        Cbs = Cs;
        Cbg = Cg;
      }
      for (int o = threadIdx.x; o < kb * kb; o += kThreads) Tb[o] = ldg(Tg + (size_t)c0 * ib + o);
      __syncthreads();
      apply_rm(V, Vh, lv, vrows, kb, Tb, true, Tops, Cbs, lc, nc, W, W2s);
      apply_rm(V, Vh, lv, vrows, kb, Tb, true, Topg, Cbg, lc, nc, W, W2g);
      bwd_partial(Cbs, Cbg, lc, vrows, kb, nc, W2s, W2g, slot + (size_t)(b - blk0) * pstride,
                  slot + sbase + (size_t)(b - blk0) * kb * kb, ch > 0);
      if (Tops) {
        store_tile(Cts, lc, 1, Cp_s, nb, tr, c0, col0 + ch, kb, nc, M_NONE);
        store_tile(Ctg, lc, 1, Cp_g, nb, tr, c0, col0 + ch, kb, nc, M_NONE);
      }
      __syncthreads();
    }
    store_tile(Cs + row_lo * lc, lc, 1, C_s, nb, tr, row_lo, col0 + ch, row_hi - row_lo, nc, M_NONE);
    store_tile(Cg + row_lo * lc, lc, 1, C_g, nb, tr, row_lo, col0 + ch, row_hi - row_lo, nc, M_NONE);
    __syncthreads();
  }
}

// Adjoint of PF(b): sums the block's partial slots (every update strip of the panel task, and the
// PU(b, s) sub-tasks), forms the tails' derivative from the columns right of the block (written to
// red, column-major, ld nb) and tau_bar, then undoes the block's reflectors one at a time on its own
// columns, pushing (v_bar, tau_bar) through house():
//   x = beta (e_1 - tau v), alpha = beta (1 - tau), g = -(v_bar . v_tail) / (beta tau),
//   alpha_bar = -tau_bar / beta - g,  beta_bar = tau_bar alpha / beta^2 + g,
//   x_bar = [alpha_bar + beta_bar alpha / beta;  -v_bar / (beta tau) - beta_bar tau v_tail].
// The post-step state of the block is its R triangle (GE: rows c0.. of X; TS / TT: the pivot's
// triangle) with the eliminated entries exactly zero, and so is the gradient there.
template <typename E>
__device__ void task_bwd_panel(unsigned char* smb, int kind, const E* X, E* A_s, E* X_s, E* A_g, E* X_g, int tr,
                               const E* Tg, int nb, int ib, int b, const E* part, const int64_t* slot_off, int u0,
                               int nu, int pu0, int pus, E* red) {
  const BwdLayout L = layout_bwd_panel(nb, ib, (int)sizeof(E));
  double* tau = reinterpret_cast<double*>(smb);
  double* rsc = tau + 64;
  double* wsA = tau + 96;
  double* bA = tau + 160;
  double* tbt = tau + 224;
  E* sm = reinterpret_cast<E*>(smb + kHeaderDoubles * sizeof(double));
  E *V = sm + L.V, *Ms = sm + L.Ms, *Mg = sm + L.Mg, *Rts = sm + L.Rts, *Rtg = sm + L.Rtg, *Sb = sm + L.Sb;
  const int lp = L.lp, c0 = b * ib, kb = ib, nblk = nb / ib;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool ge = kind == PM_GE, tt = kind == PM_TT;
  const int vrows = ge ? nb - c0 : (kind == PM_TS ? nb : c0 + kb);
  E* redb = red;            // this CTA's nb x ib scratch
  if (ge) load_tile(V, 1, lp, X, nb, tr, c0, c0, vrows, kb, M_UNITLOWER);
  else load_tile(V, 1, lp, X, nb, tr, 0, c0, vrows, kb, tt ? M_UPPER : M_NONE);
  for (int k = threadIdx.x; k < kb; k += kThreads) tau[k] = (double)ldg(Tg + (size_t)c0 * ib + k + k * ib);
  // partial sums, in slot order (deterministic); Ms holds P' meanwhile
  const size_t pblk = (size_t)b * nb * ib, sblk = (size_t)nblk * nb * ib + (size_t)b * kb * kb;
  // panel-block update slots of this block: (s - b - 1) pus + h for the later blocks s, pieces h
  const int pu_first = pu0 + (b * nblk - b * (b + 1) / 2) * pus, npu_b = (nblk - 1 - b) * pus;
  // (kRedPer independent sums per thread, so that as many loads per slot are in flight; element
  // (r, k) of P' at r kb + k in every slot)
  const int nsrc = nu + npu_b, np = vrows * kb;
  for (int o0 = 0; o0 < np; o0 += kRedPer * kThreads) {
    double acc[kRedPer];
#pragma unroll
    for (int j = 0; j < kRedPer; ++j) acc[j] = 0.0;
    for (int i = 0; i < nsrc; ++i) {
      const E* src = part + (i < nu ? slot_off[u0 + i] + pblk : slot_off[pu_first + i - nu]);
#pragma unroll
      for (int j = 0; j < kRedPer; ++j) {
        const int o = o0 + (int)threadIdx.x + j * kThreads;
        if (o < np) acc[j] += (double)ldg(src + o);
      }
    }
#pragma unroll
    for (int j = 0; j < kRedPer; ++j) {
      const int o = o0 + (int)threadIdx.x + j * kThreads;
      if (o < np) Ms[o / kb + (o % kb) * lp] = (E)acc[j];
    }
  }
  for (int o0 = 0; o0 < kb * kb; o0 += kRedPer * kThreads) {
    double acc[kRedPer];
#pragma unroll
    for (int j = 0; j < kRedPer; ++j) acc[j] = 0.0;
    for (int i = 0; i < nsrc; ++i) {
      const E* src = part + (i < nu ? slot_off[u0 + i] + sblk : slot_off[pu_first + i - nu] + (size_t)nb * kb);
#pragma unroll
      for (int j = 0; j < kRedPer; ++j) {
        const int o = o0 + (int)threadIdx.x + j * kThreads;
        if (o < kb * kb) acc[j] += (double)ldg(src + o);
      }
    }
#pragma unroll
    for (int j = 0; j < kRedPer; ++j) {
      const int o = o0 + (int)threadIdx.x + j * kThreads;
      if (o < kb * kb) Sb[o] = (E)acc[j];
    }
  }
  __syncthreads();
  // tau_bar needs S_kk; then S becomes D in place: D_lk = S_kl - S_lk at [k kb + l] (l < k), D_kk = -S_kk
  // (a pass writes only entries with k >= l and reads the ones with l < k, so the pass is race-free)
  for (int k = threadIdx.x; k < kb; k += kThreads)
    tbt[k] = tau[k] != 0.0 ? -(double)Sb[k * kb + k] / (tau[k] * tau[k]) : 0.0;
  __syncthreads();
  for (int o = threadIdx.x; o < kb * kb; o += kThreads) {
    const int k = o / kb, l = o % kb;
    if (l < k) Sb[o] = (E)((double)Sb[o] - (double)Sb[l * kb + k]);
    else if (l == k) Sb[o] = -Sb[o];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < vrows * kb; o += kThreads) {
    const int r = o % vrows, k = o / vrows;
    double s = -(double)Ms[r + k * lp];
    for (int l = 0; l <= k; ++l) s += (double)V[r + l * lp] * (double)Sb[k * kb + l];
    stg(redb + (size_t)k * nb + r, (E)s);
  }
  __syncthreads();
  if (ge) {
    load_tile(Ms, 1, lp, X_s, nb, tr, c0, c0, vrows, kb, M_UPPER);
    load_tile(Mg, 1, lp, X_g, nb, tr, c0, c0, vrows, kb, M_UPPER);
  } else {
    load_tile(Rts, 1, kb, A_s, nb, tr, c0, c0, kb, kb, M_UPPER);
    load_tile(Rtg, 1, kb, A_g, nb, tr, c0, c0, kb, kb, M_UPPER);
    for (int o = threadIdx.x; o < vrows * kb; o += kThreads) {
      const int r = o % vrows, k = o / vrows;
      Ms[r + k * lp] = E(0);
      Mg[r + k * lp] = E(0);
    }
  }
  __syncthreads();
  const int lts = ge ? lp : kb;
  // Per-reflector scalars are formed by warp 0 (FP64 issues at 2 FMA / clock / SM, so a serial chain
  // of FP64 operations on one thread is slow): the eight warp partials are combined by a 3-level
  // shuffle, and the divisions by beta_k and beta_k tau_k are replaced by reciprocals formed up front
  // for all k in parallel (beta_k, the top entry of column k, is not changed before step k).
  static_assert(kWarps == 8, "warp-partial reductions assume 8 warps");
  double* sc = rsc + kWarps;       // sc[0..3]: om, tau_bar, -1 / (beta tau), -beta_bar tau
  double* wbp = rsc + 16;          // per warp: sum_j wsA_j bA_j over its columns
  double* vbp = rsc + 24;          // per warp: v_bar . v
  double* rinv = reinterpret_cast<double*>(sm + L.Sc);   // [k]: 1 / beta_k, [kb + k]: 1 / (beta_k tau_k)
  double* pbuf = rinv + 2 * kb;    // row-sum partials of the column groups 1..G-1
  // Row update layout: G groups of RP threads, group g takes the later columns j = k + 1 + g (mod G),
  // so that short blocks keep all warps busy; group 0 owns the row (its v_bar and column k).
  const int RP = vrows <= 32 ? 32 : (vrows <= 64 ? 64 : (vrows <= 128 ? 128 : kThreads));
  const int G = kThreads / RP, gq = threadIdx.x / RP, ri = threadIdx.x % RP;
  for (int k = threadIdx.x; k < kb; k += kThreads) {
    const double beta = ge ? (double)Ms[k + k * lp] : (double)Rts[k + k * kb];
    const bool ok = tau[k] != 0.0 && beta != 0.0;
    rinv[k] = ok ? 1.0 / beta : 0.0;
    rinv[kb + k] = ok ? 1.0 / (beta * tau[k]) : 0.0;
  }
  __syncthreads();
  for (int k = kb - 1; k >= 0; --k) {
    const double t = tau[k];
    if (t == 0.0) continue;
    const int t0 = ge ? k + 1 : 0;
    const int t1 = ge ? vrows : (tt ? min(vrows, c0 + k + 1) : vrows);
    E* ts = ge ? Ms + k : Rts + k;      // top entries of column j at ts[j * lts]
    E* tg = ge ? Mg + k : Rtg + k;
    const double beta = (double)ts[k * lts];
    const int r = t0 + ri;
    const bool row = r < t1, own = row && gq == 0;
    const double vbtr = own ? (double)ldg(redb + (size_t)k * nb + r) : 0.0;
    const double v = row ? (double)V[r + k * lp] : 0.0;
    // A: |v_tail|^2 (warp partials) and, per later column j, v^T M' and v^T G'
    const double vvp = warp_sum(own ? v * v : 0.0);
    if (lane == 0) rsc[warp] = vvp;
    double wb = 0.0;
    for (int j = k + 1 + warp; j < kb; j += kWarps) {
      double s1 = 0.0, s2 = 0.0;
      for (int rr = t0 + lane; rr < t1; rr += 32) {
        const double vr = (double)V[rr + k * lp];
        s1 += vr * (double)Ms[rr + j * lp];
        s2 += vr * (double)Mg[rr + j * lp];
      }
      s1 = warp_sum(s1);
      s2 = warp_sum(s2);
      const double wa = (double)ts[j * lts] + s1, ba = (double)tg[j * lts] + s2;
      wb += wa * ba;
      if (lane == 0) {
        wsA[j] = wa;
        bA[j] = ba;
      }
    }
    if (lane == 0) wbp[warp] = wb;
    __syncthreads();
    if (warp == 0) {
      double vv = lane < kWarps ? rsc[lane] : 0.0, sw = lane < kWarps ? wbp[lane] : 0.0;
#pragma unroll
      for (int o = kWarps / 2; o > 0; o >>= 1) {
        vv += __shfl_xor_sync(kFull, vv, o);
        sw += __shfl_xor_sync(kFull, sw, o);
      }
      if (lane == 0) {
        const double om = 1.0 - t * (1.0 + vv);   // a_j = om (v^T M')_j, a_k = om beta (v^T v = 1 + |tail|^2)
        const double bk = (double)tg[k * lts];
        bA[k] = bk;
        sc[0] = om;
        sc[1] = tbt[k] - om * (beta * bk + sw);
      }
    }
    __syncthreads();
    const double om = sc[0];
    double vbar = 0.0;
    if (row) {
      double sG = 0.0, sM = 0.0;
      for (int j = k + 1 + gq; j < kb; j += G) {
        const double g = (double)Mg[r + j * lp];
        const double mpre = (double)Ms[r + j * lp] - t * v * wsA[j];
        sG += g * wsA[j];
        sM += mpre * bA[j];
        Ms[r + j * lp] = (E)mpre;
        Mg[r + j * lp] = (E)(g - t * v * bA[j]);
      }
      if (gq == 0) {
        const double mk = -beta * t * v;
        sM += mk * bA[k];
        Ms[r + k * lp] = (E)mk;
        Mg[r + k * lp] = (E)(-t * v * bA[k]);
      }
      vbar = om * sG + sM;
      if (gq > 0) pbuf[(gq - 1) * RP + ri] = vbar;
    }
    if (G > 1) __syncthreads();
    if (own) {
      for (int g = 1; g < G; ++g) vbar += pbuf[(g - 1) * RP + ri];
      vbar = vbtr - t * vbar;
    } else {
      vbar = 0.0;
    }
    if (threadIdx.x < kb - k) {
      const int j = k + threadIdx.x;
      if (j == k) {
        ts[k * lts] = (E)(beta * (1.0 - t));
      } else {
        ts[j * lts] = (E)((double)ts[j * lts] - t * wsA[j]);
        tg[j * lts] = (E)((double)tg[j * lts] - t * bA[j]);
      }
    }
    const double vbvp = warp_sum(vbar * v);
    if (lane == 0) vbp[warp] = vbvp;
    __syncthreads();
    if (warp == 0) {
      double vbv = lane < kWarps ? vbp[lane] : 0.0;
#pragma unroll
      for (int o = kWarps / 2; o > 0; o >>= 1) vbv += __shfl_xor_sync(kFull, vbv, o);
      if (lane == 0) {
        // alpha = beta (1 - tau): alpha / beta^2 = (1 - tau) / beta, alpha / beta = 1 - tau
        const double tb = sc[1];
        const double g = -vbv * rinv[kb + k];
        const double abar = -tb * rinv[k] - g;
        const double bbar = tb * (1.0 - t) * rinv[k] + g;
        tg[k * lts] = (E)((double)tg[k * lts] - t * bA[k] + abar + bbar * (1.0 - t));
        sc[2] = -rinv[kb + k];
        sc[3] = -bbar * t;
      }
    }
    __syncthreads();
    if (own) Mg[r + k * lp] = (E)((double)Mg[r + k * lp] + vbar * sc[2] + sc[3] * v);
    __syncthreads();
  }
  if (ge) {
    store_tile(Ms, 1, lp, X_s, nb, tr, c0, c0, vrows, kb, M_NONE);
    store_tile(Mg, 1, lp, X_g, nb, tr, c0, c0, vrows, kb, M_NONE);
  } else {
    store_tile(Rts, 1, kb, A_s, nb, tr, c0, c0, kb, kb, M_UPPER);
    store_tile(Rtg, 1, kb, A_g, nb, tr, c0, c0, kb, kb, M_UPPER);
    store_tile(Ms, 1, lp, X_s, nb, tr, 0, c0, vrows, kb, tt ? M_UPPER : M_NONE);
    store_tile(Mg, 1, lp, X_g, nb, tr, 0, c0, vrows, kb, tt ? M_UPPER : M_NONE);
  }
}

template <typename E>
__device__ void task_copy(const E* src, E* dst, int nb, bool diag) {
  for (int o = threadIdx.x; o < nb * nb; o += kThreads) {
    const int r = o % nb, c = o / nb;
    stg(dst + o, (diag && r > c) ? E(0) : ldg(src + o));
  }
}

// Tile reference (buffer << 28 | tile index) -> address, with the matrix's offsets and tile size.
struct MatView {
  int nb, ib, w, npanels;
  int64_t off[6], offT, nt[6];
};
template <typename E>
__device__ __forceinline__ E* tile_ptr(const ExecParams& prm, const MatView& mv, int32_t ref, bool& ok) {
  if (ref < 0) { ok = false; return nullptr; }
  const int buf = (int)((uint32_t)ref >> 28);
  const int64_t idx = ref & 0x0fffffff;
  if (buf > 5) { ok = false; return nullptr; }
  // selects instead of indexing, so that the small arrays stay in registers
  void* base = nullptr;
  int64_t nt = 0, off = 0;
#pragma unroll
  for (int i = 0; i < 6; ++i)
    if (buf == i) {
      base = prm.buf[i];
      nt = mv.nt[i];
      off = mv.off[i];
    }
  if (base == nullptr || idx >= nt) { ok = false; return nullptr; }
  return static_cast<E*>(base) + off + (size_t)idx * mv.nb * mv.nb;
}
// The adjoint's gradient tile at the same position as a state tile (buffer 2 / 3 -> 4 / 5).
__device__ __forceinline__ int32_t grad_ref(int32_t ref) {
  const int buf = (int)((uint32_t)ref >> 28);
  return (ref < 0 || buf < 2 || buf > 3) ? -1 : ref + (2 << 28);
}

// Next sub-task of a CTA (warp 0; the result is valid in lane 0).  Each sub-task's flag word is 0 while
// unclaimed, 2 once a CTA has claimed it and 1 when it is done.  First the CTA scans the `window` queue
// entries from the head and claims the first one whose dependencies are all done (it then runs without
// waiting); the head moves over a prefix found claimed.  If none is ready, it takes the head's entry
// (atomic increment, skipping entries claimed out of order) and waits for it.  Deadlock-free whatever
// the number of resident CTAs: a waiting CTA holds the lowest entry it could get in queue order, so
// everything before it is claimed, and the lowest unfinished claimed sub-task always has its
// dependencies done.  Returns ntasks when the queue is exhausted or the error word is set.
__device__ int next_task(const ExecParams& prm) {
  const int lane = threadIdx.x & 31;
  const int n = prm.ntasks;
  int err = 0;
  if (lane == 0) err = ld_relaxed(prm.err);
  if (__shfl_sync(kFull, err, 0) != 0) return n;   // warp-uniform exit
  int h = 0;
  if (lane == 0) h = ld_relaxed(prm.head);
  h = __shfl_sync(kFull, h, 0);     // one head value for the whole warp and the whole scan
  if (h >= n) return n;
  for (int base = 0; base < prm.window; base += 32) {
    const int i = h + base + lane;
    int st = 0;                     // entries not inspected (past the window or the queue) stop the skip
    bool ready = false;
    if (i < n && base + lane < prm.window) {
      st = ld_relaxed(prm.done + i);
      if (st == 0) {
        const DevTask& t = prm.tasks[i];
        const int d0 = t.dep_begin, d1 = t.dep_end;
        ready = true;
        for (int d = d0; d < d1; ++d) {
          const int dep = prm.deps[d];
          if (dep < 0 || dep >= prm.nflags || ld_acquire(prm.done + dep) != 1) { ready = false; break; }
        }
      }
    }
    if (base == 0) {   // move the head over entries already claimed
      const unsigned open = __ballot_sync(kFull, st == 0);
      const int skip = open ? __ffs(open) - 1 : 32;
      if (lane == 0 && skip > 0 && h + skip <= n) atomicCAS(prm.head, h, h + skip);
    }
    unsigned rm = __ballot_sync(kFull, ready);
    while (rm) {
      const int l = __ffs(rm) - 1;
      int got = 0;
      if (lane == l) got = atomicCAS(prm.done + i, 0, 2) == 0;
      got = __shfl_sync(kFull, got, l);
      if (got) return __shfl_sync(kFull, i, l);
      rm &= rm - 1;
    }
  }
  int idx = n;
  if (lane == 0) {
    for (;;) {
      if (ld_relaxed(prm.err) != 0) { idx = n; break; }
      idx = atomicAdd(prm.head, 1);
      if (idx >= n) { idx = n; break; }
      if (atomicCAS(prm.done + idx, 0, 2) == 0) break;
    }
  }
  return idx;
}

// Persistent dataflow executor: CTAs take sub-tasks from a queue in topological priority order
// (next_task), wait (bounded) until the sub-tasks they depend on are done, run them and publish
// completion.
template <typename E, bool kBwd>
__global__ void __launch_bounds__(kThreads, 1) exec_kernel(const ExecParams prm) {
  extern __shared__ __align__(128) unsigned char smb[];
  __shared__ int s_idx;
  __shared__ int s_abort;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ uint32_t s_tmem;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // FP32 storage: TMEM columns for the tcgen05 phase of the updates, held for the whole launch (the host
  // enables it only with one CTA per SM, so the allocation never waits), and the MMA completion barrier
  Umma um{0u, 0u, 0u, 0u, 0};
  if constexpr (sizeof(E) == 4 && !kBwd) {
    if (prm.umma_cols > 0) {
      if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"((uint32_t)prm.umma_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
      }
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      um.tmem = s_tmem;
      um.mbar = smem_u32(&s_mbar);
      um.ncols_alloc = (uint32_t)prm.umma_cols;
    }
  }
  for (;;) {
    if (warp == 0) {
      const int nt = next_task(prm);
      if (lane == 0) {
        s_idx = nt;
        s_abort = 0;
      }
    }
    __syncthreads();
    const int idx = s_idx;
    if (idx >= prm.ntasks) break;
    const DevTask t = prm.tasks[idx];
    if (warp == 0) {
      int bad = 0;
      for (int d = t.dep_begin + lane; d < t.dep_end; d += 32) {
        const int dep = prm.deps[d];
        if (dep < 0 || dep >= prm.nflags) {
          // record it now, so that lanes spinning on other dependencies see the error word and stop
          if (atomicCAS(prm.err, 0, DERR_BADTASK) == 0) { prm.err[1] = idx; prm.err[2] = -1; }
          bad = 2;
          break;
        }
        const uint64_t t0 = gtime();
        while (ld_acquire(prm.done + dep) != 1) {
          if (ld_relaxed(prm.err) != 0) { bad = 3; break; }
          if (gtime() - t0 > prm.wait_ns) {
            if (atomicCAS(prm.err, 0, DERR_TIMEOUT) == 0) {
              prm.err[1] = idx;
              prm.err[2] = dep;
            }
            bad = 1;
            break;
          }
          __nanosleep(256);
        }
        if (bad) break;
      }
      bad = __reduce_max_sync(kFull, bad);
      if (lane == 0 && bad) {
        s_abort = 1;
      }
    }
    __threadfence();
    __syncthreads();
    if (s_abort) break;

    uint64_t t_start = 0;
    if (prm.trace && threadIdx.x == 0) t_start = gtime();
    const int type = t.op & 15;
    const int tr = (t.op >> 4) & 1;
    const bool notrans = (t.op >> 5) & 1;
    const int strip = (t.op >> 8) & 0xff;
    const int blk = (t.op >> 16) & 0xff;
    const int kind = (t.op >> 24) & 3;
    bool ok = true;
    bool on_tc5 = false;      // the update ran its C -= V W product on tcgen05 (recorded in the trace)
    MatView mv;
    if (prm.mats) {
      const int mat = (t.flags >> 8) & 0xffffff;
      if (mat >= prm.nmats) {
        ok = false;
        mv = MatView{prm.nb, prm.ib, prm.w, 0, {0, 0, 0, 0, 0, 0}, 0, {0, 0, 0, 0, 0, 0}};
      } else {
        const MatInfo mi = prm.mats[mat];
        mv = MatView{mi.nb, mi.ib, mi.w, mi.npanels, {mi.off[0], mi.off[1], 0, 0, 0, 0}, mi.offT,
                     {mi.ntiles[0], mi.ntiles[1], 0, 0, 0, 0}};
      }
    } else {
      mv = MatView{prm.nb, prm.ib, prm.w, prm.npanels, {0, 0, 0, 0, 0, 0}, 0,
                   {prm.ntiles[0], prm.ntiles[1], prm.ntiles[2], prm.ntiles[3], prm.ntiles[4], prm.ntiles[5]}};
    }
    const int nb = mv.nb, ib = mv.ib, wst = mv.w;
    const int nblk = nb / ib;
    E* X = tile_ptr<E>(prm, mv, t.x, ok);
    E* Tg = (ok && t.tslot >= 0 && t.tslot < mv.npanels)
                ? static_cast<E*>(prm.T) + mv.offT + (size_t)t.tslot * ib * nb
                : nullptr;
    if constexpr (!kBwd) {
    switch (type) {
      case PF: {
        E* A = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        if (ok && Tg && blk < nblk && kind <= PM_TT)
          task_panel_factor(smb, kind, X, A, tr, Tg, nb, ib, blk, prm.f32_scalars64 == 0);
        else ok = false;
        break;
      }
      case PU: {
        E* A = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        const int utype = kind == PM_GE ? UNMQR : (kind == PM_TS ? TSMQR : TTMQR);
        if (ok && Tg && blk < strip && strip < nblk && kind <= PM_TT) {
          bool done = false;
          if constexpr (sizeof(E) == 4)
            if (prm.f32_simt == 0)
              done = task_update_umma(smb, utype, X, A, X, tr, false, Tg, nb, ib, wst, blk, blk + 1, strip * ib, ib,
                                      um, prm);
          on_tc5 = done;
          if (!done)
            task_update(smb, utype, X, A, X, tr, false, Tg, nb, ib, wst, blk, blk + 1, strip * ib, ib,
                        prm.f32_simt == 1);
        } else {
          ok = false;
        }
        break;
      }
      case UNMQR:
      case TSMQR:
      case TTMQR: {
        E* A = (type == UNMQR) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        E* C = tile_ptr<E>(prm, mv, t.c, ok);
        const int col0 = strip * wst;
        if (ok && Tg && col0 < nb) {
          bool done = false;
          if constexpr (sizeof(E) == 4)
            if (prm.f32_simt == 0)
              done = task_update_umma(smb, type, X, A, C, tr, notrans, Tg, nb, ib, wst, 0, nblk, col0,
                                      min(wst, nb - col0), um, prm);
          on_tc5 = done;
          if (!done)
            task_update(smb, type, X, A, C, tr, notrans, Tg, nb, ib, wst, 0, nblk, col0, min(wst, nb - col0),
                        prm.f32_simt == 1);
        } else {
          ok = false;
        }
        break;
      }
      case COPY: {
        E* C = tile_ptr<E>(prm, mv, t.c, ok);
        if (ok) task_copy(X, C, nb, t.flags & 1);
        break;
      }
      default:
        ok = false;
    }
    } else {
    switch (type) {
      case BPF: {
        const BwdParams& bw = prm.bwd;
        E* As = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        E* Ag = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, grad_ref(t.a), ok);
        E* Xs = tile_ptr<E>(prm, mv, t.c, ok);
        E* Xg = tile_ptr<E>(prm, mv, grad_ref(t.c), ok);
        if (ok && Tg && blk < nblk && kind <= PM_TT && bw.part && bw.red && (int)blockIdx.x < bw.red_ctas) {
          const int32_t* pi = bw.pinfo + 4 * t.tslot;
          // the update strips' sum comes from the reduced slot when the panel has one
          const int u0 = pi[3] >= 0 ? pi[3] : pi[0], nu = pi[3] >= 0 ? 1 : pi[1], pu0 = pi[2];
          const int pus = bw.pu_split;
          if (u0 < 0 || nu < 0 || u0 + nu > bw.nslots || pu0 < 0 || (pus != 1 && pus != 2) ||
              pu0 + nblk * (nblk - 1) / 2 * pus > bw.nslots) {
            ok = false;
          } else {
            task_bwd_panel(smb, kind, X, As, Xs, Ag, Xg, tr, Tg, nb, ib, blk, static_cast<const E*>(bw.part),
                           bw.slot_off, u0, nu, pu0, pus, static_cast<E*>(bw.red) + (size_t)blockIdx.x * nb * ib);
          }
        } else {
          ok = false;
        }
        break;
      }
      case BPU: {
        const BwdParams& bw = prm.bwd;
        E* As = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        E* Ag = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, grad_ref(t.a), ok);
        E* Xs = tile_ptr<E>(prm, mv, t.c, ok);
        E* Xg = tile_ptr<E>(prm, mv, grad_ref(t.c), ok);
        const int utype = kind == PM_GE ? UNMQR : (kind == PM_TS ? TSMQR : TTMQR);
        const int pus = bw.pu_split, half = notrans ? 1 : 0, pw = ib / max(1, pus);
        if (ok && Tg && blk < strip && strip < nblk && kind <= PM_TT && bw.part && t.flags >= 0 &&
            t.flags < bw.nslots && (pus == 1 || pus == 2) && half < pus && pw * pus == ib)
          task_bwd_update(smb, utype, X, As, Xs, Ag, Xg, tr, Tg, nb, ib, bw.hw, blk, blk + 1, strip * ib + half * pw,
                          pw, static_cast<E*>(bw.part) + bw.slot_off[t.flags], prm.f32_simt == 1);
        else
          ok = false;
        break;
      }
      case BUPD: {
        const BwdParams& bw = prm.bwd;
        const int utype = kind == 0 ? UNMQR : (kind == 1 ? TSMQR : TTMQR);
        E* Cps = (utype == UNMQR) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        E* Cpg = (utype == UNMQR) ? nullptr : tile_ptr<E>(prm, mv, grad_ref(t.a), ok);
        E* Cs = tile_ptr<E>(prm, mv, t.c, ok);
        E* Cg = tile_ptr<E>(prm, mv, grad_ref(t.c), ok);
        const int col0 = strip * wst;
        if (ok && Tg && col0 < nb && kind <= 2 && bw.part && t.flags >= 0 && t.flags < bw.nslots)
          task_bwd_update(smb, utype, X, Cps, Cs, Cpg, Cg, tr, Tg, nb, ib, bw.hw, 0, nblk, col0, min(wst, nb - col0),
                          static_cast<E*>(bw.part) + bw.slot_off[t.flags], prm.f32_simt == 1);
        else
          ok = false;
        break;
      }
      case BRED: {
        const BwdParams& bw = prm.bwd;
        const int vrows = kind == PM_GE ? nb - blk * ib : (kind == PM_TS ? nb : (blk + 1) * ib);
        if (ok && blk < nblk && kind <= PM_TT && bw.part && t.tslot >= 0 && t.tslot < mv.npanels &&
            strip * max(1, kRedElems / ib) < vrows) {
          const int32_t* pi = bw.pinfo + 4 * t.tslot;
          const int u0 = pi[0], nu = pi[1], r = pi[3];
          if (u0 < 0 || nu < 0 || u0 + nu > bw.nslots || r < 0 || r >= bw.nslots) {
            ok = false;
          } else {
            task_bwd_reduce(nb, ib, blk, strip, vrows, static_cast<const E*>(bw.part), bw.slot_off, u0, nu,
                            static_cast<E*>(bw.part) + bw.slot_off[r]);
          }
        } else {
          ok = false;
        }
        break;
      }
      case BCOPY: {   // gradient of the copied part of R tile c back onto pre-QR tile x
        E* Ga = tile_ptr<E>(prm, mv, grad_ref(t.x), ok);
        E* Gr = tile_ptr<E>(prm, mv, grad_ref(t.c), ok);
        if (ok) {
          const bool diag = t.flags & 1;
          for (int o = threadIdx.x; o < nb * nb; o += kThreads) {
            const int r = o % nb, c = o / nb;
            if (!diag || r <= c) stg(Ga + o, ldg(Ga + o) + ldg(Gr + o));
          }
        }
        break;
      }
      default:
        ok = false;
    }
    }
    if (!ok && threadIdx.x == 0 && atomicCAS(prm.err, 0, DERR_BADTASK) == 0) {
      prm.err[1] = idx;
      prm.err[2] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(prm.done + idx, 1);
      if (prm.trace) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        int64_t* rec = prm.trace + 4 * (size_t)idx;
        rec[0] = (int64_t)t_start;
        rec[1] = (int64_t)gtime();
        rec[2] = smid;
        rec[3] = (int64_t)(uint32_t)t.op | ((int64_t)on_tc5 << 32);
      }
    }
  }
  if constexpr (sizeof(E) == 4 && !kBwd) {
    if (prm.umma_cols > 0) {
      // every MMA was waited for, except after a wait that ran out: wait (bounded) once more for it
      if (um.failed) mbar_wait(um.mbar, um.phase ^ 1u, prm.wait_ns);
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(um.tmem), "r"(um.ncols_alloc)
                     : "memory");
    }
  }
}

template <typename E>
__global__ void r_part_kernel(const E* __restrict__ src, E* __restrict__ dst, int64_t rows_t, int64_t cols_t, int nb,
                              int s0) {
  const int64_t tile = blockIdx.x;
  const int64_t a = tile % rows_t, b = tile / rows_t;
  const E* s = src + (size_t)tile * nb * nb;
  E* d = dst + (size_t)tile * nb * nb;
  // tiles outside the trailing block keep what is already in dst (the first phase's band)
  if (a < s0) return;
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    const int r = o % nb, c = o / nb;
    const bool keep = a < cols_t && (a < b || (a == b && r <= c));
    d[o] = keep ? s[o] : E(0);
  }
}

// Band rows [r0, r1) into a zeroed tile buffer: tile (i / nb, j / nb) entry (i % nb, j % nb) =
// ab(nb + i - j, j).
template <typename E>
__global__ void scatter_band_kernel(const E* __restrict__ ab, int64_t ldab, int nb, int64_t n, E* __restrict__ tiles,
                                    int64_t rows_t, int64_t r0, int64_t r1) {
  const int64_t j = blockIdx.x;
  for (int d = threadIdx.x; d <= nb; d += blockDim.x) {
    const int64_t i = j + d - nb;
    if (i < r0 || i >= r1 || i < 0) continue;
    tiles[(size_t)((j / nb) * rows_t + i / nb) * nb * nb + (i % nb) + (j % nb) * nb] = ab[d + j * ldab];
  }
}

template <typename E>
__global__ void extract_split_kernel(const E* __restrict__ A, int64_t pa, const E* __restrict__ R, int64_t pr,
                                     int64_t srow, int nb, int64_t n, E* __restrict__ ab, int64_t ldab) {
  const int64_t j = blockIdx.x;
  for (int d = threadIdx.x; d <= nb; d += blockDim.x) {
    const int64_t i = j + d - nb;
    E v = E(0);
    if (i >= 0) {
      const E* t = i < srow ? A : R;
      const int64_t rows_t = i < srow ? pa : pr;
      v = t[(size_t)((j / nb) * rows_t + i / nb) * nb * nb + (i % nb) + (j % nb) * nb];
    }
    ab[d + j * ldab] = v;
  }
}

template <typename E>
__global__ void pack_kernel(const E* __restrict__ A, int64_t lda, int64_t m, int64_t n, int nb, E* __restrict__ tiles,
                            int64_t rows_t) {
  const int64_t tile = blockIdx.x;
  const int64_t a = tile % rows_t, b = tile / rows_t;
  E* dst = tiles + (size_t)tile * nb * nb;
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    const int r = o % nb, c = o / nb;
    const int64_t gi = a * nb + r, gj = b * nb + c;
    dst[o] = (gi < m && gj < n) ? A[gi + gj * lda] : E(0);
  }
}

template <typename E>
__global__ void unpack_kernel(const E* __restrict__ tiles, int64_t rows_t, int nb, int64_t m, int64_t n,
                              E* __restrict__ A, int64_t lda) {
  const int64_t tile = blockIdx.x;
  const int64_t a = tile % rows_t, b = tile / rows_t;
  const E* src = tiles + (size_t)tile * nb * nb;
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    const int r = o % nb, c = o / nb;
    const int64_t gi = a * nb + r, gj = b * nb + c;
    if (gi < m && gj < n) A[gi + gj * lda] = src[o];
  }
}

// ab(d, j) = B(j + d - nb, j) for d = 0..nb: the diagonal tile's upper triangle and the super-diagonal
// tile's lower triangle are exactly the band entries; rows < 0 are zero.
template <typename E>
__global__ void extract_kernel(const E* __restrict__ tiles, int64_t rows_t, int nb, int64_t n, E* __restrict__ ab,
                               int64_t ldab) {
  const int64_t j = blockIdx.x;
  for (int d = threadIdx.x; d <= nb; d += blockDim.x) {
    const int64_t i = j + d - nb;
    E v = E(0);
    if (i >= 0) {
      const int64_t a = i / nb, b = j / nb;
      v = tiles[(size_t)(b * rows_t + a) * nb * nb + (i % nb) + (j % nb) * nb];
    }
    ab[d + j * ldab] = v;
  }
}

__device__ __forceinline__ int find_matrix(const PackDesc* d, int count, int64_t x) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {   // last b with d[b].first <= x
    const int mid = (lo + hi + 1) >> 1;
    if (d[mid].first <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <typename E>
__global__ void pack_batched_kernel(const PackDesc* __restrict__ d, int count) {
  const int b = find_matrix(d, count, blockIdx.x);
  const PackDesc pd = d[b];
  const int64_t tile = blockIdx.x - pd.first;
  const int nb = pd.nb;
  const int64_t a = tile % pd.rows_t, c = tile / pd.rows_t;
  const E* A = static_cast<const E*>(pd.A);
  E* dst = static_cast<E*>(pd.out) + (size_t)tile * nb * nb;
  for (int o = threadIdx.x; o < nb * nb; o += blockDim.x) {
    const int r = o % nb, cc = o / nb;
    const int64_t gi = a * nb + r, gj = c * nb + cc;
    dst[o] = (gi < pd.m && gj < pd.n) ? A[gi + gj * pd.ld] : E(0);
  }
}

template <typename E>
__global__ void extract_batched_kernel(const PackDesc* __restrict__ d, int count) {
  const int b = find_matrix(d, count, blockIdx.x);
  const PackDesc pd = d[b];
  const int64_t j = blockIdx.x - pd.first;
  const int nb = pd.nb;
  const E* tiles = static_cast<const E*>(pd.A);
  E* ab = static_cast<E*>(pd.out);
  for (int dd = threadIdx.x; dd <= nb; dd += blockDim.x) {
    const int64_t i = j + dd - nb;
    E v = E(0);
    if (i >= 0) {
      const int64_t a = i / nb, c = j / nb;
      v = tiles[(size_t)(c * pd.rows_t + a) * nb * nb + (i % nb) + (j % nb) * nb];
    }
    ab[dd + j * pd.ld] = v;
  }
}

template <typename E>
cudaError_t pack_t(const E* A, int64_t lda, int64_t m, int64_t n, int nb, E* tiles, int64_t rows_t, int64_t cols_t,
                   cudaStream_t st) {
  if (rows_t * cols_t == 0) return cudaSuccess;
  pack_kernel<E><<<(unsigned)(rows_t * cols_t), 256, 0, st>>>(A, lda, m, n, nb, tiles, rows_t);
  return cudaGetLastError();
}
template <typename E>
cudaError_t unpack_t(const E* tiles, int64_t rows_t, int nb, int64_t m, int64_t n, E* A, int64_t lda, cudaStream_t st) {
  const int64_t cols_t = (n + nb - 1) / nb;
  if (rows_t * cols_t == 0) return cudaSuccess;
  unpack_kernel<E><<<(unsigned)(rows_t * cols_t), 256, 0, st>>>(tiles, rows_t, nb, m, n, A, lda);
  return cudaGetLastError();
}
template <typename E>
cudaError_t extract_t(const E* tiles, int64_t rows_t, int nb, int64_t n, E* ab, int64_t ldab, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  extract_kernel<E><<<(unsigned)n, 256, 0, st>>>(tiles, rows_t, nb, n, ab, ldab);
  return cudaGetLastError();
}

}  // namespace

size_t exec_smem_bytes(int nb, int ib, int w, int esize) {
  const Layout a = layout_panel(nb, ib, esize), b = layout_update(nb, ib, w, esize);
  return kHeaderDoubles * sizeof(double) + (size_t)esize * (size_t)(a.total > b.total ? a.total : b.total);
}

size_t umma_smem_bytes(int nb, int ib, int w) {
  return kHeaderDoubles * sizeof(double) + sizeof(float) * (size_t)layout_umma(nb, ib, w).total;
}

size_t bwd_smem_bytes(int nb, int ib, int hw, int esize) {
  const BwdLayout a = layout_bwd_update(nb, ib, hw, esize), b = layout_bwd_panel(nb, ib, esize);
  return kHeaderDoubles * sizeof(double) + (size_t)esize * (size_t)(a.total > b.total ? a.total : b.total);
}

int choose_bwd_chunk(int nb, int ib, int w, size_t smem_limit, int esize) {
  if (ib > 64 || nb > kThreads) return 0;
  if (kHeaderDoubles * sizeof(double) + (size_t)esize * layout_bwd_panel(nb, ib, esize).total > smem_limit) return 0;
  for (int hw = w; hw >= 1; hw /= 2) {
    if (bwd_smem_bytes(nb, ib, hw, esize) <= smem_limit) return hw;
    if (hw <= 8) break;
  }
  return 0;
}

int choose_strip_width(int nb, int ib, int preferred, size_t smem_limit, int esize) {
  if (ib > 64) return 0;
  for (int want = preferred; want >= 1; want /= 2) {
    int w = want < ib ? ib : (want / ib) * ib;
    if (w > nb) w = nb;
    if (exec_smem_bytes(nb, ib, w, esize) <= smem_limit) return w;
    if (w == ib) break;
  }
  return 0;
}

namespace {
template <typename E>
const void* exec_fn(bool bwd) {
  return bwd ? reinterpret_cast<const void*>(exec_kernel<E, true>) : reinterpret_cast<const void*>(exec_kernel<E, false>);
}
}  // namespace

cudaError_t exec_set_smem(size_t smem, int esize, bool bwd) {
  return cudaFuncSetAttribute(esize == 4 ? exec_fn<float>(bwd) : exec_fn<double>(bwd),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int exec_max_ctas_per_sm(size_t smem, int esize, bool bwd) {
  int n = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &n, esize == 4 ? exec_fn<float>(bwd) : exec_fn<double>(bwd), kThreads, smem);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_exec(const ExecParams& prm, int grid, size_t smem, cudaStream_t st) {
  const bool bwd = prm.bwd.part != nullptr;
  if (prm.esize == 4) {
    if (bwd) exec_kernel<float, true><<<grid, kThreads, smem, st>>>(prm);
    else exec_kernel<float, false><<<grid, kThreads, smem, st>>>(prm);
  } else {
    if (bwd) exec_kernel<double, true><<<grid, kThreads, smem, st>>>(prm);
    else exec_kernel<double, false><<<grid, kThreads, smem, st>>>(prm);
  }
  return cudaGetLastError();
}

cudaError_t launch_pack_batched(const PackDesc* d, int count, int64_t total_tiles, int esize, cudaStream_t st) {
  if (total_tiles == 0) return cudaSuccess;
  if (esize == 4) pack_batched_kernel<float><<<(unsigned)total_tiles, 256, 0, st>>>(d, count);
  else pack_batched_kernel<double><<<(unsigned)total_tiles, 256, 0, st>>>(d, count);
  return cudaGetLastError();
}

cudaError_t launch_extract_batched(const PackDesc* d, int count, int64_t total_cols, int esize, cudaStream_t st) {
  if (total_cols == 0) return cudaSuccess;
  if (esize == 4) extract_batched_kernel<float><<<(unsigned)total_cols, 256, 0, st>>>(d, count);
  else extract_batched_kernel<double><<<(unsigned)total_cols, 256, 0, st>>>(d, count);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* A, int64_t lda, int64_t m, int64_t n, int nb, double* tiles, int64_t rows_t,
                        int64_t cols_t, cudaStream_t st) {
  return pack_t(A, lda, m, n, nb, tiles, rows_t, cols_t, st);
}
cudaError_t launch_pack(const float* A, int64_t lda, int64_t m, int64_t n, int nb, float* tiles, int64_t rows_t,
                        int64_t cols_t, cudaStream_t st) {
  return pack_t(A, lda, m, n, nb, tiles, rows_t, cols_t, st);
}
cudaError_t launch_unpack(const double* tiles, int64_t rows_t, int nb, int64_t m, int64_t n, double* A, int64_t lda,
                          cudaStream_t st) {
  return unpack_t(tiles, rows_t, nb, m, n, A, lda, st);
}
cudaError_t launch_unpack(const float* tiles, int64_t rows_t, int nb, int64_t m, int64_t n, float* A, int64_t lda,
                          cudaStream_t st) {
  return unpack_t(tiles, rows_t, nb, m, n, A, lda, st);
}
cudaError_t launch_extract(const double* tiles, int64_t rows_t, int nb, int64_t n, double* ab, int64_t ldab,
                           cudaStream_t st) {
  return extract_t(tiles, rows_t, nb, n, ab, ldab, st);
}
template <typename E>
cudaError_t r_part_t(const E* src, E* dst, int64_t rows_t, int64_t cols_t, int nb, int s, cudaStream_t st) {
  if (rows_t * cols_t == 0) return cudaSuccess;
  r_part_kernel<E><<<(unsigned)(rows_t * cols_t), 256, 0, st>>>(src, dst, rows_t, cols_t, nb, s);
  return cudaGetLastError();
}
cudaError_t launch_r_part(const double* src, double* dst, int64_t rows_t, int64_t cols_t, int nb, int s,
                          cudaStream_t st) {
  return r_part_t(src, dst, rows_t, cols_t, nb, s, st);
}
cudaError_t launch_r_part(const float* src, float* dst, int64_t rows_t, int64_t cols_t, int nb, int s, cudaStream_t st) {
  return r_part_t(src, dst, rows_t, cols_t, nb, s, st);
}
template <typename E>
cudaError_t scatter_t(const E* ab, int64_t ldab, int nb, int64_t n, E* tiles, int64_t rows_t, int64_t r0, int64_t r1,
                      cudaStream_t st) {
  if (n == 0 || r1 <= r0) return cudaSuccess;
  scatter_band_kernel<E><<<(unsigned)n, 256, 0, st>>>(ab, ldab, nb, n, tiles, rows_t, r0, r1);
  return cudaGetLastError();
}
cudaError_t launch_scatter_band(const double* ab, int64_t ldab, int nb, int64_t n, double* tiles, int64_t rows_t,
                                int64_t r0, int64_t r1, cudaStream_t st) {
  return scatter_t(ab, ldab, nb, n, tiles, rows_t, r0, r1, st);
}
cudaError_t launch_scatter_band(const float* ab, int64_t ldab, int nb, int64_t n, float* tiles, int64_t rows_t,
                                int64_t r0, int64_t r1, cudaStream_t st) {
  return scatter_t(ab, ldab, nb, n, tiles, rows_t, r0, r1, st);
}
template <typename E>
cudaError_t extract_split_t(const E* A, int64_t pa, const E* R, int64_t pr, int64_t srow, int nb, int64_t n, E* ab,
                            int64_t ldab, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  extract_split_kernel<E><<<(unsigned)n, 256, 0, st>>>(A, pa, R, pr, srow, nb, n, ab, ldab);
  return cudaGetLastError();
}
cudaError_t launch_extract_split(const double* A, int64_t pa, const double* R, int64_t pr, int64_t srow, int nb,
                                 int64_t n, double* ab, int64_t ldab, cudaStream_t st) {
  return extract_split_t(A, pa, R, pr, srow, nb, n, ab, ldab, st);
}
cudaError_t launch_extract_split(const float* A, int64_t pa, const float* R, int64_t pr, int64_t srow, int nb,
                                 int64_t n, float* ab, int64_t ldab, cudaStream_t st) {
  return extract_split_t(A, pa, R, pr, srow, nb, n, ab, ldab, st);
}
cudaError_t launch_extract(const float* tiles, int64_t rows_t, int nb, int64_t n, float* ab, int64_t ldab,
                           cudaStream_t st) {
  return extract_t(tiles, rows_t, nb, n, ab, ldab, st);
}

}  // namespace bd
