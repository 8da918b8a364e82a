// Device-side interface shared by the C ABI (capi.cu) and the kernels (kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "plan.h"

namespace bd {

constexpr int kThreads = 256;       // threads of every executor CTA
constexpr int kMaxNb = 256;

// Error word layout written by the executor: err[0] = code (0 ok, 1 wait ran out, 2 bad task),
// err[1] = queue position of the failing task, err[2] = dependency it waited for.
enum DevErr : int { DERR_OK = 0, DERR_TIMEOUT = 1, DERR_BADTASK = 2 };

// Per-matrix parameters of a batched program (sub-task flags bits 8-31 select the entry).
struct MatInfo {
  int64_t off[2];       // element offsets of the matrix's tiles in buf[0] (A) and buf[1] (R copy)
  int64_t offT;         // element offset of its T slots
  int64_t ntiles[2];
  int32_t nb, ib, w, npanels;
  int64_t pad;
};

// Matrix b of a batched pack / extract.
struct PackDesc {
  const void* A;        // column-major input (pack) or tile buffer of the band's source (extract)
  void* out;            // tile buffer base of the matrix (pack) or its band (extract)
  int64_t ld, m, n, rows_t, first;   // ld: lda (pack) / ldab (extract); first: first tile / column
  int32_t nb, pad;
};

// Extra arguments of the adjoint program (reverse sweep).
struct BwdParams {
  void* part;               // partial slots (element type by esize)
  const int64_t* slot_off;  // element offset of each slot
  int32_t nslots;
  const int32_t* pinfo;     // per panel task: first update slot, number of update slots, first PU slot,
                            // reduced slot (-1: none)
  void* red;                // per executor CTA nb x ib: scratch of a panel-block adjoint (the summed
                            // derivative of its reflector tails, written and read by that sub-task)
  int red_ctas;             // CTAs the scratch covers (the launch's grid)
  int hw;                   // column chunk of the update adjoints
  int pu_split;             // column pieces of a panel-block update adjoint (1 or 2)
};

// Executor look-ahead of one-matrix FP64 BiDiag reductions (queue entries scanned for a ready sub-task):
// 8192^2 1374 -> 1330 ms, 4096^2 232 -> 222 ms against strict queue order; FP32 storage, R-BiDiag and
// batches were not faster with it and keep strict order.
constexpr int kWindowF64BiDiag = 1024;

struct ExecParams {
  const DevTask* tasks;
  const int32_t* deps;
  int32_t ntasks;
  int32_t nflags;       // number of entries of done[] (>= ntasks; extra entries are never set)
  int* done;
  int* head;
  int* err;
  void* buf[6];         // tile buffers (element type by esize): A tiles, R copy (R-BiDiag), apply target;
                        // the adjoint uses 2 / 3 as the state of A / R and 4 / 5 as their gradients
  int64_t ntiles[6];
  void* T;
  int32_t npanels;
  int nb, ib, w;        // tile size, inner blocking, strip width
  uint64_t wait_ns;
  int64_t* trace;       // optional: 4 int64 per task (start ns, end ns, SM id, op), queue order
  int esize;            // 8: FP64 tiles; 4: FP32 tiles (split-precision updates)
  const MatInfo* mats;  // batched program: per-matrix parameters (null for one matrix)
  int nmats;
  int f32_simt;         // FP32 tiles only: 0 = three-TF32 tensor-core updates (tcgen05 where umma_cols > 0),
                        // 1 = updates by FP32 FFMA, 2 = three-TF32 updates on the warp-level MMA only
  int umma_cols;        // FP32 forward program: TMEM columns each CTA allocates for the tcgen05 phase (0: none)
  int f32_scalars64;    // FP32 tiles only: 1 = reflector beta / tau / scale in FP64 instead of float pairs
  int window;           // queue entries from the head a CTA scans for a ready sub-task (0: strict queue order)
  BwdParams bwd;        // adjoint program only
};

// Shared memory (bytes) the executor needs for (nb, ib, w) and element size esize (8 or 4).
size_t exec_smem_bytes(int nb, int ib, int w, int esize);
// Dynamic shared memory of the FP32 forward executor when its updates take the tcgen05 path (ib 32).
size_t umma_smem_bytes(int nb, int ib, int w);
// Column-strip width of the update sub-tasks: a multiple of ib, at most nb, as close to `preferred`
// as the shared-memory limit allows; 0 if even w = ib does not fit.
int choose_strip_width(int nb, int ib, int preferred, size_t smem_limit, int esize);

// Shared memory of the adjoint program and the column chunk of its update sub-tasks (0 if the panel
// adjoint does not fit).
size_t bwd_smem_bytes(int nb, int ib, int hw, int esize);
int choose_bwd_chunk(int nb, int ib, int w, size_t smem_limit, int esize);

// Executor launch: the adjoint instantiation when prm.bwd.part is set (bwd below must match).
cudaError_t launch_exec(const ExecParams& prm, int grid, size_t smem, cudaStream_t st);
cudaError_t exec_set_smem(size_t smem, int esize, bool bwd = false);
int exec_max_ctas_per_sm(size_t smem, int esize, bool bwd = false);

// Column-major (ld) matrix <-> zero-padded tile buffer (grid of rows_t x cols_t tiles of nb x nb).
cudaError_t launch_pack(const double* A, int64_t lda, int64_t m, int64_t n, int nb, double* tiles, int64_t rows_t,
                        int64_t cols_t, cudaStream_t st);
cudaError_t launch_pack(const float* A, int64_t lda, int64_t m, int64_t n, int nb, float* tiles, int64_t rows_t,
                        int64_t cols_t, cudaStream_t st);
cudaError_t launch_unpack(const double* tiles, int64_t rows_t, int nb, int64_t m, int64_t n, double* A, int64_t lda,
                          cudaStream_t st);
cudaError_t launch_unpack(const float* tiles, int64_t rows_t, int nb, int64_t m, int64_t n, float* A, int64_t lda,
                          cudaStream_t st);
// Batched pack / extract over `count` matrices described on the device (total = tiles / columns).
cudaError_t launch_pack_batched(const PackDesc* d, int count, int64_t total_tiles, int esize, cudaStream_t st);
cudaError_t launch_extract_batched(const PackDesc* d, int count, int64_t total_cols, int esize, cudaStream_t st);
// R-BiDiag adjoint start: dst = the R factor of the pre-QR held in src (tiles (a, b) with a <= b < q:
// upper triangle of diagonal tiles, whole tiles above), zero elsewhere; grid rows_t x cols_t.
// Only tiles with a >= s (the trailing block of a three-step) are kept.
cudaError_t launch_r_part(const double* src, double* dst, int64_t rows_t, int64_t cols_t, int nb, int s,
                          cudaStream_t st);
cudaError_t launch_r_part(const float* src, float* dst, int64_t rows_t, int64_t cols_t, int nb, int s, cudaStream_t st);
// Band rows [r0, r1) of ab ((nb+1) x n, ld ldab) into a zeroed tile buffer (grid rows rows_t): the
// inverse of extraction.
cudaError_t launch_scatter_band(const double* ab, int64_t ldab, int nb, int64_t n, double* tiles, int64_t rows_t,
                                int64_t r0, int64_t r1, cudaStream_t st);
cudaError_t launch_scatter_band(const float* ab, int64_t ldab, int nb, int64_t n, float* tiles, int64_t rows_t,
                                int64_t r0, int64_t r1, cudaStream_t st);
// Three-step band extraction: band rows < srow from tiles A (grid rows pa), the others from tiles R.
cudaError_t launch_extract_split(const double* A, int64_t pa, const double* R, int64_t pr, int64_t srow, int nb,
                                 int64_t n, double* ab, int64_t ldab, cudaStream_t st);
cudaError_t launch_extract_split(const float* A, int64_t pa, const float* R, int64_t pr, int64_t srow, int nb,
                                 int64_t n, float* ab, int64_t ldab, cudaStream_t st);
// Band extraction: ab((nb+1) x n, ld ldab) from the tile buffer (grid rows rows_t).
cudaError_t launch_extract(const double* tiles, int64_t rows_t, int nb, int64_t n, double* ab, int64_t ldab,
                           cudaStream_t st);
cudaError_t launch_extract(const float* tiles, int64_t rows_t, int nb, int64_t n, float* ab, int64_t ldab,
                           cudaStream_t st);

}  // namespace bd
