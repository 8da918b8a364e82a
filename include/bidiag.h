/*
 * bidiag.h - C ABI of the GB300 tiled band-bidiagonalization library.
 *
 * The library reduces a dense real m x n matrix A (m >= n) to upper band-bidiagonal form
 *     B = Q^T A P,   Q (m x m) and P (n x n) orthogonal,  B with nb super-diagonals,
 * with the tiled BiDiag and R-BiDiag algorithms (Faverge, Langou, Robert, Dongarra, "Bidiagonalization
 * with parallel tiled algorithms", Sec. 3.4 and 3.5), whose QR and LQ steps eliminate tiles with the
 * GEQRT/TSQRT/TTQRT panel kernels and UNMQR/TSMQR/TTMQR update kernels of Table 1 (Sec. 3.2, Algorithms
 * 2 and 3; LQ steps use the same kernels on the transposed geometry, Algorithm 4), scheduled by the
 * FlatTS, FlatTT, Greedy (Sec. 3.3) or Auto (Sec. 5) reduction tree.
 *
 * Conventions for every entry point:
 *  - Matrices are column-major, FP64, sizes are int64_t.  Pointers named d_* are device pointers on the
 *    handle's device; pointers named h_* are host pointers.
 *  - Return value: BIDIAG_OK (0) on success; a negative value -i when argument i (1-based) is invalid
 *    (LAPACK "info" style); a positive BIDIAG_ERR_* code otherwise.  No function throws across the ABI.
 *    bidiag_last_error() returns a text for the last failure on a handle.
 *  - Work is stream-ordered on the handle's stream; results are valid once bidiag_sync() returned
 *    BIDIAG_OK (bidiag_band_host synchronises by itself).
 *  - Tile indices are 0-based.  Tile (a, b) covers rows [a nb, min((a+1) nb, m)) and columns
 *    [b nb, min((b+1) nb, n)); the last tile row/column may be ragged.
 */
#ifndef BIDIAG_H
#define BIDIAG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bidiag_ctx* bidiag_handle;
typedef struct bidiag_result* bidiag_result_t;

/* Reduction trees: Sec. 3.3 (FlatTS, FlatTT, Greedy) and Sec. 5 (Auto). */
enum { BIDIAG_FLATTS = 0, BIDIAG_FLATTT = 1, BIDIAG_GREEDY = 2, BIDIAG_AUTO = 3 };
/* Variants: Sec. 3.4 (BiDiag) and Sec. 3.5 (R-BiDiag = QR(p,q) then BiDiag of the top square).
 * BIDIAG_AUTO_VARIANT picks the one with the shorter critical path (Sec. 4.3.3, the delta_s switch;
 * see bidiag_plan_choose_variant); the result records the variant used.
 * Three-step (Sec. 4.5, partial BiDiag + pre-QR + BiDiag): BIDIAG_THREESTEP_SPLIT(s), 0 <= s < q, runs
 * the first s BiDiag steps (QR(k), LQ(k), k < s) on A, then R-BiDiag on the trailing (p-s) x (q-s)
 * tiles (pre-QR, copy of its R, BiDiag of that R); s = 0 is R-BiDiag (recorded as such), s = q-1 has
 * BiDiag's critical path.  BIDIAG_THREESTEP picks the split with the shortest critical path by trying
 * every s (the paper's brute force; see bidiag_plan_best_split).  Not available in the batched and
 * allocation-free forms. */
enum { BIDIAG_BIDIAG = 0, BIDIAG_RBIDIAG = 1, BIDIAG_AUTO_VARIANT = 2, BIDIAG_THREESTEP = 3 };
#define BIDIAG_THREESTEP_SPLIT(s) (4 + (s))
/* Status codes. */
enum {
  BIDIAG_OK = 0,
  BIDIAG_ERR_CUDA = 1,        /* a CUDA runtime call failed; text in bidiag_last_error */
  BIDIAG_ERR_NOMEM = 2,       /* device or host allocation failed */
  BIDIAG_ERR_TIMEOUT = 3,     /* a device-side dependency wait ran out (see bidiag_set_option) */
  BIDIAG_ERR_UNSUPPORTED = 4, /* valid but unsupported request, e.g. m < n */
  BIDIAG_ERR_SCRATCH = 5      /* bidiag_band_noalloc: the problem needs more than its fixed scratch */
};

/* Size of the fixed device scratch array behind bidiag_band_noalloc (bytes). */
#define BIDIAG_NOALLOC_SCRATCH_BYTES (8u << 20)
/* Options for bidiag_set_option. */
enum {
  BIDIAG_OPT_WAIT_LIMIT_NS = 1,   /* bound of every device-side dependency wait, ns (default 2e10) */
  BIDIAG_OPT_AUTO_RESOURCES = 2,  /* "nbcores" R of the Auto tree (default: SMs * w / nb with w = 32, the
                                     number of tile updates that run at once when each spreads over
                                     nb / w SMs; FP32 storage SMs * 64 / nb) */
  BIDIAG_OPT_DEBUG_UNSET_DEP = 3, /* 1: the next bidiag_band adds to its first task a dependency on a
                                     flag nothing sets, so that its wait runs out (failure-path test) */
  BIDIAG_OPT_STRIP = 4,           /* column-strip width of the update tasks (16, 32 or 64; default 32, and
                                     64 for a one-matrix reduction with FP32 storage) */
  BIDIAG_OPT_TIMING = 5,          /* 1: time the executor launch of each bidiag_band with CUDA events */
  BIDIAG_OPT_TRACE = 6,           /* 1: record a per-task trace of each bidiag_band (see bidiag_trace) */
  BIDIAG_OPT_F32_UPDATES = 7,     /* FP32 storage: 0 = updates as three TF32 tensor-core products, the
                                     C -= V W product on tcgen05 (one matrix; default), 1 = updates by FP32
                                     FMA on the CUDA cores (FP32-exact products), 2 = three TF32 products on
                                     the warp-level MMA only */
  BIDIAG_OPT_F32_SCALARS = 8,     /* FP32 storage: each reflector's beta, tau and tail scale from alpha and
                                     the tail's squared norm (always a compensated sum, FP64-level accuracy)
                                     0 = in float-pair arithmetic, about 44 bits (default), 1 = in FP64.
                                     Both give the FP32 values the reduction stores to within their
                                     rounding; FP64 costs ~1.7K cycles of serial FP64 latency per column */
  BIDIAG_OPT_WINDOW = 9,          /* executor look-ahead, -1..1024: a CTA looking for work scans this many
                                     queue entries from the head and takes the first whose dependencies
                                     are done; only when none is ready does it take the head's entry and
                                     wait for it.  0 = strict queue order; -1 (default) = 1024 for a
                                     one-matrix FP64 BiDiag reduction, else 0 (measured on 8192^2 and
                                     4096^2: 3.2 / 4.1 % faster; FP32 storage, R-BiDiag and batches are
                                     not faster).  Results do not depend on it: the program orders every
                                     access to shared data, the window only changes timing */
  BIDIAG_OPT_PRIORITY = 10        /* queue order of the device program, by bottom level (longest weighted
                                     path to the end) with sub-task weights 1 = Table 1 flops times the
                                     measured time per flop of each sub-task kind (default), 0 = flops
                                     alone (FP32-storage panel factors twice).  Results do not depend on
                                     it */
};

/* Task type codes of the canonical task list (GELQT etc. are the same codes in LQ phases). */
enum { BIDIAG_T_GEQRT = 0, BIDIAG_T_UNMQR = 1, BIDIAG_T_TSQRT = 2, BIDIAG_T_TSMQR = 3,
       BIDIAG_T_TTQRT = 4, BIDIAG_T_TTMQR = 5, BIDIAG_T_COPY = 6 };
/* Phase codes: QR / LQ steps of BiDiag (R-BiDiag: of the second phase), PQR = R-BiDiag's QR(p,q). */
enum { BIDIAG_PH_QR = 0, BIDIAG_PH_LQ = 1, BIDIAG_PH_PQR = 2 };

/*
 * Reflector store of a result (Sec. 3.6 "Memory usage": R-BiDiag keeps its pre-QR reflectors apart).
 * All pointers are device pointers owned by the result.
 *  tiles   : p*q tiles of nb*nb elements, tile (a, b) at tiles + (b*p + a)*nb*nb, column-major inside
 *            with leading dimension nb, zero padded beyond m / n.  After the reduction it holds the
 *            Householder vectors of every tile kernel in the positions they eliminated (GEQRT/GELQT:
 *            strict lower/upper triangle; TSQRT: the whole eliminated tile; TTQRT: the upper/lower
 *            triangle of the eliminated tile) and, for BiDiag, the band entries.
 *  tiles2  : R-BiDiag only (else NULL): q*q tiles, same layout, holding the second phase.
 *  T       : one block of ib*nb elements per panel task (tslot order): the ib x ib upper-triangular T
 *            factors of the compact WY form of each group of ib reflectors side by side
 *            (block b at T + slot*ib*nb + b*ib*ib, column-major, ld ib); tau_j = diag(T).
 *  tslot   : host array, one entry per canonical task: its T slot for a panel task, -1 otherwise.
 */
typedef struct bidiag_reflectors {
  const void* tiles;           /* double or float elements, see elem_bytes */
  const void* tiles2;
  const void* T;
  const int32_t* tslot;
  int64_t ntasks;
  int64_t m, n;
  int32_t nb, ib, p, q, npanels, variant;
  int32_t elem_bytes;          /* 8: tiles and T in FP64; 4: in FP32 (bidiag_band_f32) */
  int32_t tree;                /* tree the reduction used */
} bidiag_reflectors;

/* Creates a handle bound to CUDA device `device` and stream `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  Owns the plan cache and the scheduler workspace.
 * Errors: -1 (h NULL), -2 (bad device), BIDIAG_ERR_CUDA, BIDIAG_ERR_NOMEM. */
int bidiag_create(bidiag_handle* h, int device, void* cuda_stream);

/* Sets an option (BIDIAG_OPT_*) on the handle.  Errors: -2 unknown option, -3 bad value. */
int bidiag_set_option(bidiag_handle h, int option, int64_t value);

/*
 * GE2BND: reduces the m x n matrix at d_A (device, column-major, leading dimension lda; read only) to
 * band form with tile size nb, inner blocking ib (Sec. 6.2: internal blocking of the TS/TT kernels),
 * tree and variant.  Preconditions (else -i): m >= 1 (-2), 1 <= n (-3), d_A != NULL (-4), lda >= m
 * (-5), 1 <= nb <= 256 (-6), 1 <= ib <= min(nb, 64) and nb % ib == 0 (-7), tree in 0..3 (-8), variant
 * in 0..2 (-9), out != NULL (-10).  m < n returns BIDIAG_ERR_UNSUPPORTED (Sec. 3.6: the transposed
 * problem).  *out receives a new result object (free with bidiag_result_free) that owns the band, the
 * reflector store and the canonical task list.  The call enqueues the work and returns.
 */
int bidiag_band(bidiag_handle h, int64_t m, int64_t n, const double* d_A, int64_t lda,
                int nb, int ib, int tree, int variant, bidiag_result_t* out);

/*
 * Split-precision form of bidiag_band: FP32 storage (d_A, the tiles, T factors and band are float);
 * the trailing updates run on the tensor cores as three TF32 products (hi*hi + hi*lo + lo*hi, each
 * operand split into a TF32 part and a TF32 remainder) accumulated in FP32, while the reflector norms,
 * beta, tau (the T diagonal) and the scaling of the reflector vectors are computed in FP64.  Arguments,
 * errors and ownership as bidiag_band; read the band with bidiag_result_band_f32 and apply Q, P with
 * bidiag_apply_q_f32 / bidiag_apply_p_f32.  Sec. 3.6: the method holds for single precision.
 */
int bidiag_band_f32(bidiag_handle h, int64_t m, int64_t n, const float* d_A, int64_t lda,
                    int nb, int ib, int tree, int variant, bidiag_result_t* out);

/*
 * Batched form: reduces `count` independent matrices (each m[b] x n[b], m >= n, column-major at device
 * pointer d_A[b] with leading dimension lda[b]) in ONE persistent launch.  Per-matrix tile size nb[b],
 * inner blocking ib[b], tree[b] and variant[b] (BIDIAG_AUTO_VARIANT allowed); when nb is NULL the
 * library's autotuner (bidiag_autotune) picks all four per matrix; when only ib / tree / variant is NULL
 * the defaults are min(nb, 32), Auto and BIDIAG_AUTO_VARIANT.  The host arrays are read during the call.
 * out[b] receives one result per matrix (free each with bidiag_result_free; they share one device
 * allocation that is released with the last of them) usable like any other result (band, tasks,
 * reflectors, apply_q / apply_p).  Errors: -2 count, -3 a matrix's sizes or pointer, -7 nb/ib, -9 tree or
 * variant, -11 out; the text names the matrix.  No counterpart in the paper's experiments (Sec. 5's
 * runtime reduces one matrix); the per-matrix algorithm is the same.
 */
int bidiag_band_batched(bidiag_handle h, int64_t count, const int64_t* m, const int64_t* n,
                        const double* const* d_A, const int64_t* lda, const int* nb, const int* ib,
                        const int* tree, const int* variant, bidiag_result_t* out);
/* The same for FP32 storage (split-precision form of bidiag_band_f32). */
int bidiag_band_batched_f32(bidiag_handle h, int64_t count, const int64_t* m, const int64_t* n,
                            const float* const* d_A, const int64_t* lda, const int* nb, const int* ib,
                            const int* tree, const int* variant, bidiag_result_t* out);

/* Autotuner of the batched form (host only): for an m x n matrix of a batch on a device with nsm SMs and
 * storage of elem_bytes (8: FP64, 4: FP32), searches the calibrated tile sizes and inner blockings
 * (nb in {32, 64, 128}, ib in {8, 16, 32}) and the FlatTS, Greedy and Auto trees (Sec. 3.3, Sec. 5), the
 * variant by critical path (Sec. 4.3.3), minimising the time the matrix's sub-tasks keep SMs busy (mean
 * sub-task times measured on a GB300, compiled into the library) plus its critical path with the same
 * times over nsm / 8.  The paper tunes nb and ib by hand (Sec. 6.2); its Auto tree adapts the reduction
 * tree to the resources (Sec. 5).  Errors: -1 sizes, -3 nsm, -4 elem_bytes, -5 NULL output. */
int bidiag_autotune(int64_t m, int64_t n, int nsm, int elem_bytes, int* nb, int* ib, int* tree, int* variant);

/*
 * Same reduction for host buffers: copies h_A (column-major, lda) to the device, reduces it, copies the
 * band back into h_ab (LAPACK upper-band storage, (nb+1) x n, leading dimension ldab >= nb+1) and
 * synchronises.  h_A and h_ab should be pinned for full copy speed.  The result object is kept in *out
 * when out != NULL (else freed).  Errors as bidiag_band, plus -11 (h_ab NULL) and -12 (ldab).
 */
int bidiag_band_host(bidiag_handle h, int64_t m, int64_t n, const double* h_A, int64_t lda,
                     int nb, int ib, int tree, int variant, double* h_ab, int64_t ldab,
                     bidiag_result_t* out);

/*
 * The same reduction without any device allocation, for callers that may not allocate device memory:
 * code embedded in an application whose GPU memory is wholly owned by another allocator (a framework's
 * caching allocator that has reserved the device, say), or a service that forbids device allocation
 * after start-up because cudaMalloc can stall the whole device and can fail at an unpredictable moment.
 * The paper has no counterpart: this is a deployment convenience of this library.
 *
 * The caller passes the input d_A (m x n, column-major, lda; read only) and the output d_ab (the band in
 * LAPACK upper-band storage, (nb+1) x n, leading dimension ldab >= nb+1), both device pointers on the
 * current device, and a stream (NULL = legacy default stream).  Every other buffer (tile copy of A,
 * R copy, T factors, task program, flags) lives in one array of BIDIAG_NOALLOC_SCRATCH_BYTES (8 MiB) in
 * device global memory that the library declares statically; every GPU that loads the library holds
 * it until the process exits.  A problem that does not fit returns BIDIAG_ERR_SCRATCH before any work
 * is enqueued (a 512 x 512 BiDiag with nb = 64 needs about 3.3 MiB).  No cudaMalloc, cudaFree or
 * allocating library routine is called; the task program is planned in host memory.
 *
 * The first call in each CUDA context (normally once per device, in its primary context) looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it for that context; a context made
 * after cudaDeviceReset, or another context the caller makes current, gets a lookup of its own.  Make
 * that first call before any stream capture on the device.  All calls share the one array
 * and each call leaves its contents behind, so calls whose work overlaps on the GPU (other threads or
 * other streams at the same time) race and corrupt each other's results: serialise them.  The call
 * enqueues the work, waits for the stream and returns the device-side status (BIDIAG_OK,
 * BIDIAG_ERR_TIMEOUT, BIDIAG_ERR_CUDA).  No reflectors are kept (only the band is returned).
 * Argument errors: -1 m, -2 n, -3 d_A, -4 lda, -5 nb, -6 ib, -7 tree, -8 variant, -9 d_ab, -10 ldab;
 * m < n returns BIDIAG_ERR_UNSUPPORTED.
 */
int bidiag_band_noalloc(int64_t m, int64_t n, const double* d_A, int64_t lda, int nb, int ib, int tree,
                        int variant, double* d_ab, int64_t ldab, void* cuda_stream);

/* Band B in LAPACK upper-band storage (device): B(i, j) at ab[(nb + i - j) + j*ldab] for
 * max(0, j-nb) <= i <= j < n, ldab = nb + 1.  B is n x n (rows n..m-1 of Q^T A P are zero); every
 * entry outside the band is an exact zero by construction. */
int bidiag_result_band(bidiag_result_t r, const double** ab, int64_t* ldab, int64_t* n, int* nb);

/* Band of an FP32 result (bidiag_band_f32), same layout as bidiag_result_band; BIDIAG_ERR_UNSUPPORTED
 * for an FP64 result (and bidiag_result_band returns it for an FP32 result). */
int bidiag_result_band_f32(bidiag_result_t r, const float** ab, int64_t* ldab, int64_t* n, int* nb);

/* Canonical task list (host memory owned by the result): ntasks records of 6 int32
 * (type, phase, k, i, piv, j) in program order, oriented coordinates (an LQ step's oriented tile (a,b)
 * is tile (b,a)); -1 where a field is unused.  COPY(i, j) copies tile (i, j)'s R into the second
 * phase of R-BiDiag. */
int bidiag_result_tasks(bidiag_result_t r, const int32_t** tasks, int64_t* ntasks);

/* Fills *desc with the reflector store (see bidiag_reflectors). */
int bidiag_result_reflectors(bidiag_result_t r, bidiag_reflectors* desc);

/* Applies Q from the result to the m x ncols device matrix d_C (leading dimension ldc >= m):
 * trans = 0: C <- Q C, trans = 1: C <- Q^T C.  Errors: -3 trans, -4 ncols < 0, -5 d_C, -6 ldc. */
int bidiag_apply_q(bidiag_handle h, bidiag_result_t r, int trans, int64_t ncols, double* d_C,
                   int64_t ldc);

/* Applies P from the result to the nrows x n device matrix d_C (leading dimension ldc >= nrows):
 * trans = 0: C <- C P, trans = 1: C <- C P^T.  Errors: -3 trans, -4 nrows < 0, -5 d_C, -6 ldc. */
int bidiag_apply_p(bidiag_handle h, bidiag_result_t r, int trans, int64_t nrows, double* d_C,
                   int64_t ldc);

/* FP32 forms of bidiag_apply_q / bidiag_apply_p for results of bidiag_band_f32 (float C, same layout
 * and errors; -2 when the result's precision does not match). */
int bidiag_apply_q_f32(bidiag_handle h, bidiag_result_t r, int trans, int64_t ncols, float* d_C,
                       int64_t ldc);
int bidiag_apply_p_f32(bidiag_handle h, bidiag_result_t r, int trans, int64_t nrows, float* d_C,
                       int64_t ldc);

/*
 * Adjoint (reverse-mode derivative) of a reduction: given dL/dB in band storage (d_abbar, (nb+1) x n,
 * leading dimension ldab >= nb+1, the layout of bidiag_result_band; entries with row index < 0 are
 * ignored), writes dL/dA to d_Abar (m x n, column-major, ldabar >= m).  If d_Arec is not NULL it also
 * receives the reconstruction of A from the band and the reflectors (ldarec >= m), a by-product.
 * The reduction of Sec. 3.4 / 3.5 is a sequence of Householder steps M <- H(x) M (LQ steps on M^T); the
 * adjoint walks them backwards over the result's stored reflectors (V tiles and T), undoing each step on
 * a working copy of the state (H is its own inverse) and applying the chain rule through H and through
 * the reflector's construction from its pivot column.  The paper has no derivative; this is its exact
 * reverse mode, with a reflector of tau = 0 (a zero column, where the Householder map switches branch)
 * held constant.  The result must come from this handle and is not modified; FP64 results only
 * (FP32 ones: bidiag_band_backward_f32).  Device memory (bidiag_backward_workspace gives the exact
 * figure): two copies of the tiled matrix, the partial sums of the update adjoints (nb^2 + nb ib
 * elements per update strip, in storage recycled once the panel's factor adjoint has consumed them:
 * 1.0 GB for 4096 x 1024 and 6.8 GB for 8192^2 with nb = 256, FP64) and nb ib elements of scratch per
 * executor CTA, allocated and freed on the handle's stream.  Bitwise deterministic (no atomics).
 * Errors: -2 result, -3 d_abbar NULL, -4 ldab, -5 d_Abar NULL, -6 ldabar, -8 ldarec,
 * BIDIAG_ERR_UNSUPPORTED when nb / ib need more shared memory than a block has (nb = 256 needs
 * ib <= 32), BIDIAG_ERR_NOMEM, BIDIAG_ERR_CUDA.  Stream-ordered: call bidiag_sync before reading.
 */
int bidiag_band_backward(bidiag_handle h, bidiag_result_t r, const double* d_abbar, int64_t ldab,
                         double* d_Abar, int64_t ldabar, double* d_Arec, int64_t ldarec);
/* Device bytes one bidiag_band_backward(_f32) call on result r allocates (state and gradient tiles,
 * partial-sum storage, panel-adjoint scratch), in *bytes.  Plans and uploads the adjoint program if this
 * result's plan has none yet (the backward call then reuses it).  Errors: -1 h, -2 result, -3 bytes NULL,
 * BIDIAG_ERR_UNSUPPORTED, BIDIAG_ERR_NOMEM, BIDIAG_ERR_CUDA. */
int bidiag_backward_workspace(bidiag_handle h, bidiag_result_t r, int64_t* bytes);
/* The same for a result with FP32 storage (band_f32 / band_batched_f32); the reflector derivatives
 * and the Householder-construction step are evaluated in FP64, the updates as in the forward. */
int bidiag_band_backward_f32(bidiag_handle h, bidiag_result_t r, const float* d_abbar, int64_t ldab,
                             float* d_Abar, int64_t ldabar, float* d_Arec, int64_t ldarec);

/* Waits for the handle's stream and returns the device-side status of the work enqueued since the
 * last call: BIDIAG_OK, BIDIAG_ERR_TIMEOUT (a dependency wait ran out; the context stays usable) or
 * BIDIAG_ERR_CUDA. */
int bidiag_sync(bidiag_handle h);

/* Duration (ms, CUDA events on the handle's stream) of the executor kernel of the last bidiag_band
 * enqueued with BIDIAG_OPT_TIMING on; call after bidiag_sync.  Errors: -2 ms NULL, BIDIAG_ERR_UNSUPPORTED
 * when timing was off. */
int bidiag_last_exec_ms(bidiag_handle h, float* ms);

/* Per-task trace of the last bidiag_band enqueued with BIDIAG_OPT_TRACE on (call after bidiag_sync):
 * *count records of 4 int64 in queue order: start and end (%globaltimer ns), SM id, and the task's op
 * word (type | orientation << 4 | strip << 8, as bidiag_plan_program) in the low 32 bits, bit 32 set
 * when an FP32-storage update ran its C -= V W product on tcgen05.  Copied to host `out` when
 * cap >= *count. */
int bidiag_trace(bidiag_handle h, int64_t* out, int64_t cap, int64_t* count);

/* Device program of the last traced launch (host memory, for analysing its trace): *count sub-tasks
 * of 8 int32 in queue order (the layout of bidiag_plan_program: op, x, a, c, tslot, dep_begin, dep_end,
 * flags) and *ndeps dependency entries (queue positions).  Copied when cap >= *count and dcap >= *ndeps
 * respectively.  Errors: -1 h, -4 count NULL, -7 ndeps NULL, BIDIAG_ERR_UNSUPPORTED before any traced
 * launch. */
int bidiag_trace_program(bidiag_handle h, int32_t* program, int64_t cap, int64_t* count, int32_t* deps,
                         int64_t dcap, int64_t* ndeps);

/* Text of the last failure on the handle ("" if none).  Valid until the next call on h. */
const char* bidiag_last_error(bidiag_handle h);

/* Releases a result (stream-ordered on the handle's stream that made it). */
int bidiag_result_free(bidiag_result_t r);

/* Releases the handle (synchronises its stream first).  Results made on it that are still alive lose
 * their device buffers; bidiag_result_free must still be called on them to release the host object. */
int bidiag_destroy(bidiag_handle h);

/* ---------------------------------------------------------------------------------------------
 * Host-only planner queries (no device work; usable without a GPU).  They expose the planner's
 * elimination list, task list and task DAG so that they can be checked against the paper's critical
 * path formulas (Sec. 4) and an independent implementation.  `resources` is the Auto tree's R.
 * `variant` is BIDIAG_BIDIAG, BIDIAG_RBIDIAG or BIDIAG_THREESTEP_SPLIT(s) with s < q.
 * --------------------------------------------------------------------------------------------- */

/* Canonical elimination list: records of 5 int32 (phase, k, i, piv, kind[0 = TS, 1 = TT]).  When
 * out == NULL or cap is too small only *count is set. */
int bidiag_plan_eliminations(int64_t p, int64_t q, int tree, int variant, int64_t resources,
                             int32_t* out, int64_t cap, int64_t* count);

/* Canonical task list, 6 int32 per task as in bidiag_result_tasks, plus its DAG: level[t] (0 without
 * predecessors, else 1 + max level of its predecessors) when level != NULL, and the critical path in
 * Table 1 units (GEQRT 4, UNMQR 6, TSQRT 6, TSMQR 12, TTQRT 2, TTMQR 6, COPY 0) in *cp when cp != NULL. */
int bidiag_plan_tasks(int64_t p, int64_t q, int tree, int variant, int64_t resources,
                      int32_t* tasks, int32_t* level, int64_t cap, int64_t* count, int64_t* cp);

/* BiDiag or R-BiDiag for a p x q tile matrix, whichever has the shorter critical path in the task-DAG
 * model (Table 1 weights, unbounded resources; Sec. 4.3.3 shows the switch ratio delta_s = p/q
 * oscillates in [5, 8], e.g. 5.67 for q = 100).  The Auto tree is compared through Greedy.  Ties keep
 * BiDiag.  *variant receives BIDIAG_BIDIAG or BIDIAG_RBIDIAG; the two critical paths are returned when
 * the pointers are not NULL.  Errors: -1 (p, q), -3 (tree), -5 (variant NULL). */
int bidiag_plan_choose_variant(int64_t p, int64_t q, int tree, int64_t resources, int* variant,
                               int64_t* cp_bidiag, int64_t* cp_rbidiag);

/* Host-only: the three-step split s with the shortest critical path for p x q tiles (Table 1 weights,
 * unbounded resources; ties keep the smallest s) and, if cp is not NULL, that critical path.
 * Errors: -1 sizes (need p >= q >= 1), -3 tree, -5 split NULL. */
int bidiag_plan_best_split(int64_t p, int64_t q, int tree, int64_t resources, int* split, int64_t* cp);

/* The device program the executor runs for a reduction (host-only, for validation): *count sub-tasks
 * of 8 int32 in queue order (op word: type | orientation << 4 | Q-instead-of-Q^T << 5 | strip << 8 |
 * inner block << 16 | panel kind << 24; V/panel tile, pivot/top tile, C tile references (buffer << 28 |
 * tile index); T slot; first and one-past-last dependency; flags) and *ndeps dependency entries
 * (queue positions).  Sub-task types: 1, 3, 5 = update strips (UNMQR, TSMQR, TTMQR), 6 = COPY,
 * 7 = factor one inner block of a panel, 8 = apply it to a later column block of the panel.
 * *strip_w receives the update strip width.  Arrays are filled when their capacities suffice. */
int bidiag_plan_program(int64_t m, int64_t n, int nb, int ib, int tree, int variant, int64_t resources,
                        int strip_w, int32_t* program, int64_t cap, int64_t* count, int32_t* deps,
                        int64_t dcap, int64_t* ndeps, int32_t* strip_w_used);

/* Host-only query of the FP64 adjoint program bidiag_band_backward runs for these arguments (same rules
 * as bidiag_plan_program; strip_w is rounded to a multiple of ib): *count sub-tasks of 8 int32 in queue
 * order (op, x, a, c, tslot, dep_begin, dep_end, flags; op type 9 = undo a panel block, 10 = undo a
 * panel-block update (with ib >= 16 as two column halves, op bit 5 = the half), 11 = undo an update
 * strip, 12 = gradient of a COPY, 13 = sum the update-strip partials of one panel block over a chunk of
 * 2048 / ib rows (op bits 8-15 = chunk) into the panel's reduced slot; x = reflector tile of the forward
 * result, a / c = state tiles of the m x n grid, flags = partial slot), fwd[y] = the forward queue
 * position it undoes (a type-13 sub-task: the panel block it serves), *ndeps dependency indices,
 * *nslot_off slot offsets (the last one is the total number of elements) and *npinfo = 4 per panel
 * task (first update slot, number of update slots, first panel-update slot, reduced slot or -1; panels
 * with at least 8 update strips have one), and *strip_w_used = the column width of its update strips
 * (half the forward's when that is at least 16: each forward strip is undone as two sub-tasks).
 * Arrays are filled only when their capacity suffices.  Errors as bidiag_plan_program, -10 for a NULL
 * count pointer. */
int bidiag_plan_backward(int64_t m, int64_t n, int nb, int ib, int tree, int variant, int64_t resources,
                         int strip_w, int32_t* program, int32_t* fwd, int64_t cap, int64_t* count,
                         int32_t* deps, int64_t dcap, int64_t* ndeps, int64_t* slot_off, int64_t scap,
                         int64_t* nslot_off, int32_t* pinfo, int64_t pcap, int64_t* npinfo,
                         int32_t* strip_w_used);

/* Measurement support (the paper has no counterpart; no reduction uses it): the FP64 throughput of
 * the GPU `device`, the denominators of the FP64 reduction's roofline.  *gflops_fma receives the rate of
 * a loop of independent DFMA chains (the unit the reduction's contractions run on), *gflops_mma that of
 * a loop of mma.sync m8n8k4 f64 (the ISA's FP64 tensor-core path), both best of five launches of a few
 * tens of milliseconds on cuda_stream (NULL = legacy default stream), in GFLOP/s.  Allocates and frees a
 * small device buffer; makes `device` current.  Errors: -1 device, -3 / -4 NULL outputs,
 * BIDIAG_ERR_NOMEM, BIDIAG_ERR_CUDA. */
int bidiag_measure_fp64_peaks(int device, void* cuda_stream, double* gflops_fma, double* gflops_mma);

#ifdef __cplusplus
}
#endif

#endif /* BIDIAG_H */
