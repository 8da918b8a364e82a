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
  int P, V, Cs, Ct, Rt, Tb, G, W, W2, total;
};
constexpr int kHeaderDoubles = 64 + 32;   // tau[<= 64], red[32]
__host__ __device__ inline int align4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline Layout layout_panel(int nb, int ib, int esize) {
  Layout L{};
  L.lp = odd_ld(nb);
  L.lv = L.lc = 0;
  int o = 0;
  L.P = o;   o = align4(o + L.lp * ib);
  L.Rt = o;  o = align4(o + ib * ib);
  L.Tb = o;  o = align4(o + ib * ib);
  L.G = o;   o = align4(o + ib * ib);
  L.V = L.Cs = L.Ct = L.W = L.W2 = -1;
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
  L.Ct = o;  o = align4(o + ib * L.lc);
  L.V = o;   o = align4(o + nb * L.lv);
  L.Tb = o;  o = align4(o + ib * ib);
  L.W = o;   o = align4(o + ib * L.lc);
  L.W2 = o;  o = align4(o + ib * L.lc);
  L.P = L.Rt = L.G = -1;
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

// Shared element (r, c) at s[r * rs + c * cs] <- oriented X(r0 + r, c0 + c).  M_UPPER zeroes entries
// below the diagonal, M_UNITLOWER gives the unit lower trapezoid.  Lanes run along the contiguous
// direction of global memory (rows for tr = 0, columns for tr = 1).  Blocks of at most 256 x 32 (every
// block the sub-tasks move) issue all of a thread's loads (up to 32) before the first shared store, so
// that one L2 latency covers the whole block.
template <typename E>
__device__ void load_tile(E* s, int rs, int cs, const E* g, int nb, int tr, int r0, int c0, int rows, int cols,
                          int mask) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (rows <= 256 && cols <= 32) {
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
          if (c < cols && r < rows) s[r * rs + c * cs] = v[kc * 8 + kr];
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
        if (lane < cols && r < rows) s[r * rs + lane * cs] = v[kr];
      }
    }
    return;
  }
  if (!tr) {
    for (int c = warp; c < cols; c += kWarps) {
#pragma unroll 4
      for (int r = lane; r < rows; r += 32) s[r * rs + c * cs] = masked_ld(g, r0 + r, c0 + c, nb, tr, mask);
    }
  } else {
#pragma unroll 4
    for (int r = warp; r < rows; r += kWarps) {
      for (int c = lane; c < cols; c += 32) s[r * rs + c * cs] = masked_ld(g, r0 + r, c0 + c, nb, tr, mask);
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

// Sum over the CTA, the same value (same order) in every thread.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) s += red[w];
  return s;
}

enum PanelMode : int { PM_GE = 0, PM_TS = 1, PM_TT = 2 };

// Unblocked factorization of kb panel columns held in P (ld lp).
//  GE: reflector jj has alpha = P[jj, jj] and tail P[jj+1 .. rows-1, jj].
//  TS: alpha = Rt[jj, jj] (top triangle), tail P[0 .. rows-1, jj].
//  TT: as TS with tail P[0 .. min(rows, voff + jj + 1) - 1, jj] (the eliminated tile is a triangle).
// The squared norm, beta, tau and the scaling of the tail are computed in FP64 whatever the storage.
template <typename E>
__device__ void factor_panel(int mode, E* P, int lp, int rows, int kb, E* Rt, int lrt, int voff, double* tau_s,
                             double* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int jj = 0; jj < kb; ++jj) {
    int t0, t1;
    E* alpha_p;
    if (mode == PM_GE) {
      t0 = jj + 1; t1 = rows; alpha_p = &P[jj + jj * lp];
    } else {
      t0 = 0; t1 = (mode == PM_TT) ? min(rows, voff + jj + 1) : rows; alpha_p = &Rt[jj + jj * lrt];
    }
    double part = 0.0;
    for (int r = t0 + threadIdx.x; r < t1; r += kThreads) {
      const double x = (double)P[r + jj * lp];
      part += x * x;
    }
    const double sigma2 = block_sum(part, red);
    const double alpha = (double)*alpha_p;
    double beta, tau, denom;
    if (sigma2 == 0.0) {
      beta = alpha; tau = 0.0; denom = 1.0;
    } else {
      const double nrm = sqrt(alpha * alpha + sigma2);
      beta = alpha < 0.0 ? nrm : -nrm;
      tau = (beta - alpha) / beta;
      denom = alpha - beta;
    }
    for (int r = t0 + threadIdx.x; r < t1; r += kThreads)
      P[r + jj * lp] = (tau != 0.0) ? (E)((double)P[r + jj * lp] / denom) : E(0);
    __syncthreads();
    if (threadIdx.x == 0) {
      *alpha_p = (E)beta;
      tau_s[jj] = tau;
    }
    if (tau != 0.0) {
      const E taue = (E)tau;
      for (int c = jj + 1 + warp; c < kb; c += kWarps) {
        E s = E(0);
        for (int r = t0 + lane; r < t1; r += 32) s += P[r + jj * lp] * P[r + c * lp];
        s = warp_sum(s);
        E* top = (mode == PM_GE) ? &P[jj + c * lp] : &Rt[jj + c * lrt];
        const E wv = *top + s;
        __syncwarp();
        if (lane == 0) *top = *top - taue * wv;
        const E tw = taue * wv;
        for (int r = t0 + lane; r < t1; r += 32) P[r + c * lp] -= P[r + jj * lp] * tw;
      }
    }
    __syncthreads();
  }
}

// T factor (kb x kb, upper) of the kb reflectors in P: T[l,l] = tau_l,
// T[0:l, l] = -tau_l T[0:l, 0:l] (V[:, 0:l]^T v_l).  G is kb x kb scratch.
template <typename E>
__device__ void build_t(int mode, const E* P, int lp, int rows, int kb, int voff, const double* tau_s, E* Tb, int ldt,
                        E* G) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int pr = warp; pr < kb * kb; pr += kWarps) {
    const int a = pr % kb, l = pr / kb;
    if (a >= l) continue;
    E s = E(0);
    if (mode == PM_GE) {
      for (int r = l + 1 + lane; r < rows; r += 32) s += P[r + a * lp] * P[r + l * lp];
      s = warp_sum(s) + P[l + a * lp];
    } else {
      const int r1 = (mode == PM_TT) ? min(rows, voff + a + 1) : rows;
      for (int r = lane; r < r1; r += 32) s += P[r + a * lp] * P[r + l * lp];
      s = warp_sum(s);
    }
    if (lane == 0) G[a + l * kb] = s;
  }
  __syncthreads();
  for (int l = 0; l < kb; ++l) {
    for (int a = threadIdx.x; a < kb; a += kThreads) {
      E v = E(0);
      if (a == l) {
        v = (E)tau_s[l];
      } else if (a < l) {
        E s = E(0);
        for (int t = a; t < l; ++t) s += Tb[a + t * ldt] * G[t + l * kb];
        v = -(E)tau_s[l] * s;
      }
      Tb[a + l * ldt] = v;
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
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  const float r = x - __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
  hi = h;
  lo = l;
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
__device__ __forceinline__ void mma_3xtf32(float* acc, const float* a, const float* b) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_tf32(a[i], ah[i], al[i]);
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
template <typename E>
__device__ void apply_phase1_simt(const E* V, int lv, int vrows, int kb, const E* Ct, const E* C, int lc, int ncols,
                                  E* W) {
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
#pragma unroll 4
      for (int r = 0; r < vrows; ++r) {
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
__device__ void apply_phase3_simt(const E* V, int lv, int vrows, int kb, E* C, int lc, int ncols, const E* W2) {
  using V2 = typename Vec2<E>::type;
  if ((ncols & 7) == 0 && (kb & 1) == 0) {
    const int nunits = vrows * (ncols >> 3);
    for (int u = threadIdx.x; u < nunits; u += kThreads) {
      const int r = u % vrows, c0 = (u / vrows) << 3;
      V2* cp = reinterpret_cast<V2*>(C + r * lc + c0);
      V2 a0 = cp[0], a1 = cp[1], a2 = cp[2], a3 = cp[3];
      const E* vp = V + r * lv;
#pragma unroll 2
      for (int a = 0; a < kb; a += 2) {
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
__device__ void apply_phase1_tc(const float* V, int lv, int vrows, int kb, const float* Ct, const float* C, int lc,
                                int ncols, float* W) {
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
    for (int k0 = 0; k0 < vrows; k0 += 8) {
      float a[4], b[2];
      a[0] = V[(k0 + t) * lv + m0 + g];
      a[1] = V[(k0 + t) * lv + m0 + g + 8];
      a[2] = V[(k0 + t + 4) * lv + m0 + g];
      a[3] = V[(k0 + t + 4) * lv + m0 + g + 8];
      b[0] = C[(k0 + t) * lc + n0 + g];
      b[1] = C[(k0 + t + 4) * lc + n0 + g];
      mma_3xtf32(acc, a, b);
    }
    W[(m0 + g) * lc + n0 + 2 * t] = acc[0];
    W[(m0 + g) * lc + n0 + 2 * t + 1] = acc[1];
    W[(m0 + g + 8) * lc + n0 + 2 * t] = acc[2];
    W[(m0 + g + 8) * lc + n0 + 2 * t + 1] = acc[3];
  }
}

// Tensor-core phase 3 (FP32): C[r][c] -= sum_a V[r][a] W2[a][c]; M = vrows, N = ncols, K = kb.
__device__ void apply_phase3_tc(const float* V, int lv, int vrows, int kb, float* C, int lc, int ncols,
                                const float* W2) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int mt_n = vrows >> 4, nt_n = ncols >> 3;
  for (int tile = warp; tile < mt_n * nt_n; tile += kWarps) {
    const int m0 = (tile % mt_n) << 4, n0 = (tile / mt_n) << 3;
    float* c0p = C + (m0 + g) * lc + n0 + 2 * t;
    float* c1p = C + (m0 + g + 8) * lc + n0 + 2 * t;
    float acc[4] = {c0p[0], c0p[1], c1p[0], c1p[1]};
    for (int k0 = 0; k0 < kb; k0 += 8) {
      float a[4], b[2];
      a[0] = -V[(m0 + g) * lv + k0 + t];
      a[1] = -V[(m0 + g + 8) * lv + k0 + t];
      a[2] = -V[(m0 + g) * lv + k0 + t + 4];
      a[3] = -V[(m0 + g + 8) * lv + k0 + t + 4];
      b[0] = W2[(k0 + t) * lc + n0 + g];
      b[1] = W2[(k0 + t + 4) * lc + n0 + g];
      mma_3xtf32(acc, a, b);
    }
    c0p[0] = acc[0];
    c0p[1] = acc[1];
    c1p[0] = acc[2];
    c1p[1] = acc[3];
  }
}

template <typename E>
__device__ void apply_rm(const E* V, int lv, int vrows, int kb, const E* Tb, bool notrans, E* Ct, E* C, int lc,
                         int ncols, E* W, E* W2, bool simt) {
  constexpr bool kF32 = sizeof(E) == 4;
  const bool tc = kF32 && !simt && (kb & 15) == 0 && (vrows & 15) == 0 && (ncols & 7) == 0;
  // phase 1
  if constexpr (kF32) {
    if (tc) apply_phase1_tc(V, lv, vrows, kb, Ct, C, lc, ncols, W);
    else apply_phase1_simt(V, lv, vrows, kb, Ct, C, lc, ncols, W);
  } else {
    apply_phase1_simt(V, lv, vrows, kb, Ct, C, lc, ncols, W);
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
    if (tc) apply_phase3_tc(V, lv, vrows, kb, C, lc, ncols, W2);
    else apply_phase3_simt(V, lv, vrows, kb, C, lc, ncols, W2);
  } else {
    apply_phase3_simt(V, lv, vrows, kb, C, lc, ncols, W2);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// Panel factor sub-task PF(b): factors inner block b (columns b*ib .. b*ib + ib - 1) of a panel task
// and writes its reflectors in place and its T block.  GE: rows b*ib .. nb-1 of tile X.  TS: the
// triangle of pivot tile A's diagonal block b over all rows of X.  TT: the same triangle over the upper
// part of X (rows 0 .. b*ib + ib - 1).  The later column blocks are updated by PU sub-tasks.
// ---------------------------------------------------------------------------------------------
template <typename E>
__device__ void task_panel_factor(unsigned char* smb, int kind, E* X, E* A, int tr, E* Tg, int nb, int ib, int b) {
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
    factor_panel(PM_GE, P, L.lp, rows, kb, (E*)nullptr, 0, 0, tau, red);
    build_t(PM_GE, P, L.lp, rows, kb, 0, tau, Tb, kb, G);
    store_tile(P, 1, L.lp, X, nb, tr, c0, c0, rows, kb, M_NONE);
  } else {
    const bool tt = kind == PM_TT;
    const int vrows = tt ? c0 + kb : nb;
    load_tile(Rt, 1, kb, A, nb, tr, c0, c0, kb, kb, M_UPPER);
    load_tile(P, 1, L.lp, X, nb, tr, 0, c0, vrows, kb, tt ? M_UPPER : M_NONE);
    __syncthreads();
    factor_panel(kind, P, L.lp, vrows, kb, Rt, kb, c0, tau, red);
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
    if (type == UNMQR) {
      vrows = nb - c0;
      load_tile(V, L.lv, 1, X, nb, tr, c0, c0, vrows, kb, M_UNITLOWER);
      Cb = Cs + c0 * L.lc;
    } else {
      vrows = (type == TSMQR) ? nb : c0 + kb;
      load_tile(V, L.lv, 1, X, nb, tr, 0, c0, vrows, kb, type == TSMQR ? M_NONE : M_UPPER);
      load_tile(Ct, L.lc, 1, Cp, nb, tr, c0, col0, kb, ncols, M_NONE);
      Ctop = Ct;
      Cb = Cs;
    }
    for (int o = threadIdx.x; o < kb * kb; o += kThreads) Tb[o] = ldg(Tg + (size_t)c0 * ib + o);
    __syncthreads();
    apply_rm(V, L.lv, vrows, kb, Tb, notrans, Ctop, Cb, L.lc, ncols, W, W2, simt);
    if (Ctop) {
      store_tile(Ct, L.lc, 1, Cp, nb, tr, c0, col0, kb, ncols, M_NONE);
      __syncthreads();
    }
  }
  store_tile(Cs + row_lo * L.lc, L.lc, 1, C, nb, tr, row_lo, col0, row_hi - row_lo, ncols, M_NONE);
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
  int64_t off[3], offT, nt[3];
};
template <typename E>
__device__ __forceinline__ E* tile_ptr(const ExecParams& prm, const MatView& mv, int32_t ref, bool& ok) {
  if (ref < 0) { ok = false; return nullptr; }
  const int buf = (int)((uint32_t)ref >> 28);
  const int64_t idx = ref & 0x0fffffff;
  if (buf > 2) { ok = false; return nullptr; }
  void* base = buf == 0 ? prm.buf[0] : (buf == 1 ? prm.buf[1] : prm.buf[2]);
  const int64_t nt = buf == 0 ? mv.nt[0] : (buf == 1 ? mv.nt[1] : mv.nt[2]);
  const int64_t off = buf == 0 ? mv.off[0] : (buf == 1 ? mv.off[1] : mv.off[2]);
  if (base == nullptr || idx >= nt) { ok = false; return nullptr; }
  return static_cast<E*>(base) + off + (size_t)idx * mv.nb * mv.nb;
}

// Persistent dataflow executor: CTAs take sub-tasks from a queue in topological priority order,
// wait (bounded) until the sub-tasks they depend on are done, run them and publish completion.
// Taking tasks in queue order makes the scheme deadlock-free whatever the number of resident CTAs.
template <typename E>
__global__ void __launch_bounds__(kThreads, 1) exec_kernel(const ExecParams prm) {
  extern __shared__ __align__(16) unsigned char smb[];
  __shared__ int s_idx;
  __shared__ int s_abort;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) {
      s_idx = (ld_relaxed(prm.err) != 0) ? prm.ntasks : atomicAdd(prm.head, 1);
      s_abort = 0;
    }
    __syncthreads();
    const int idx = s_idx;
    if (idx >= prm.ntasks) break;
    const DevTask t = prm.tasks[idx];
    if (warp == 0) {
      int bad = 0;
      for (int d = t.dep_begin + lane; d < t.dep_end; d += 32) {
        const int dep = prm.deps[d];
        if (dep < 0 || dep >= prm.nflags) { bad = 2; break; }
        const uint64_t t0 = gtime();
        while (ld_acquire(prm.done + dep) == 0) {
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
        if (bad == 2 && atomicCAS(prm.err, 0, DERR_BADTASK) == 0) { prm.err[1] = idx; prm.err[2] = -1; }
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
    MatView mv;
    if (prm.mats) {
      const int mat = (t.flags >> 8) & 0xffffff;
      if (mat >= prm.nmats) {
        ok = false;
        mv = MatView{prm.nb, prm.ib, prm.w, 0, {0, 0, 0}, 0, {0, 0, 0}};
      } else {
        const MatInfo mi = prm.mats[mat];
        mv = MatView{mi.nb, mi.ib, mi.w, mi.npanels, {mi.off[0], mi.off[1], 0}, mi.offT,
                     {mi.ntiles[0], mi.ntiles[1], 0}};
      }
    } else {
      mv = MatView{prm.nb, prm.ib, prm.w, prm.npanels, {0, 0, 0}, 0, {prm.ntiles[0], prm.ntiles[1], prm.ntiles[2]}};
    }
    const int nb = mv.nb, ib = mv.ib, wst = mv.w;
    const int nblk = nb / ib;
    E* X = tile_ptr<E>(prm, mv, t.x, ok);
    E* Tg = (ok && t.tslot >= 0 && t.tslot < mv.npanels)
                ? static_cast<E*>(prm.T) + mv.offT + (size_t)t.tslot * ib * nb
                : nullptr;
    switch (type) {
      case PF: {
        E* A = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        if (ok && Tg && blk < nblk && kind <= PM_TT) task_panel_factor(smb, kind, X, A, tr, Tg, nb, ib, blk);
        else ok = false;
        break;
      }
      case PU: {
        E* A = (kind == PM_GE) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        const int utype = kind == PM_GE ? UNMQR : (kind == PM_TS ? TSMQR : TTMQR);
        if (ok && Tg && blk < strip && strip < nblk && kind <= PM_TT)
          task_update(smb, utype, X, A, X, tr, false, Tg, nb, ib, wst, blk, blk + 1, strip * ib, ib,
                      prm.f32_simt != 0);
        else
          ok = false;
        break;
      }
      case UNMQR:
      case TSMQR:
      case TTMQR: {
        E* A = (type == UNMQR) ? nullptr : tile_ptr<E>(prm, mv, t.a, ok);
        E* C = tile_ptr<E>(prm, mv, t.c, ok);
        const int col0 = strip * wst;
        if (ok && Tg && col0 < nb)
          task_update(smb, type, X, A, C, tr, notrans, Tg, nb, ib, wst, 0, nblk, col0, min(wst, nb - col0),
                      prm.f32_simt != 0);
        else
          ok = false;
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
        rec[3] = t.op;
      }
    }
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

cudaError_t exec_set_smem(size_t smem, int esize) {
  if (esize == 4) return cudaFuncSetAttribute(exec_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaFuncSetAttribute(exec_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

int exec_max_ctas_per_sm(size_t smem, int esize) {
  int n = 0;
  cudaError_t e = esize == 4
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, exec_kernel<float>, kThreads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, exec_kernel<double>, kThreads, smem);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_exec(const ExecParams& prm, int grid, size_t smem, cudaStream_t st) {
  if (prm.esize == 4) exec_kernel<float><<<grid, kThreads, smem, st>>>(prm);
  else exec_kernel<double><<<grid, kThreads, smem, st>>>(prm);
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
cudaError_t launch_extract(const float* tiles, int64_t rows_t, int nb, int64_t n, float* ab, int64_t ldab,
                           cudaStream_t st) {
  return extract_t(tiles, rows_t, nb, n, ab, ldab, st);
}

}  // namespace bd
