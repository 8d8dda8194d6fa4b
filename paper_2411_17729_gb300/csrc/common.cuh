// common.cuh -- shared declarations of the cascade library (host + device).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <array>
#include <string>
#include <vector>

#include "../../include/cascade.h"

namespace cascade {

// ---------------------------------------------------------------- host side
extern long long g_launches;                      // kernels launched (host count)
void set_global_error(const std::string& msg);
std::string global_error();

#define CASCADE_LAUNCHED() (++::cascade::g_launches)

// Tile of one stage: BM consecutive time steps of one sequence.
struct Tile {
  int64_t seq_row0;   // packed row of the sequence's first time step
  int32_t t0;         // first time step of the tile within the sequence
  int32_t len;        // sequence length L_i
  int32_t sys;        // system index
  int32_t flags;      // TILE_FINAL_FUSED: last stage with y = Cv + Du fused
  int32_t fbuf;       // workspace state buffer that holds the sequence's final states
  int32_t pad1;
};
static_assert(sizeof(Tile) == 32, "Tile is 32 bytes");
enum { TILE_FINAL_FUSED = 1 };

// Window of the fused first stages (stage_fused.cu): 128 time steps of one
// sequence from step r0 on (r0 may be negative: steps before the sequence are
// zero); the pass stores its rows from H on.
struct FusedWindow {
  int64_t seq_row0;   // packed row of the sequence's first time step
  int32_t r0;
  int32_t len;        // sequence length
  int32_t sys;
  int32_t pad;
};
static_assert(sizeof(FusedWindow) == 24, "FusedWindow is 24 bytes");

// Sequence record (output kernel, recursion, backward).
struct Seq {
  int64_t row0;
  int32_t len;
  int32_t sys;
  int32_t N;          // last stage index run for this sequence
  int32_t flags;      // SEQ_FUSED: output already written by the last stage
};
enum { SEQ_FUSED = 1 };

// Everything a stage launch needs besides tensor maps.
// Caller row buffers (u, y, dy, du) are read and written with 16-byte vector
// accesses on some paths; the entry points check this alignment before any launch.
constexpr uintptr_t ROW_ALIGN = 16;
inline bool row_aligned(const void* ptr) {
  return (reinterpret_cast<uintptr_t>(ptr) & (ROW_ALIGN - 1)) == 0;
}

struct StageArgs {
  const Tile* tiles;
  int32_t ntiles;
  int32_t nblocks;        // m / BN
  int32_t m, p, q;
  int32_t BN;
  int32_t stages;         // SMEM pipeline depth
  int32_t ring;           // residual staging slots of the epilogue
  int32_t shift;          // 2^k
  int32_t reverse;        // 1: adjoint stage (source l + s, transposed power)
  int32_t k;              // stage index
  int32_t kmax1;          // power-table entries per system
  int32_t keep_v;         // fused last stage also writes v (the backward reads it)
  int32_t S;              // 0: a tile is BM consecutive rows.  S > 0 (work-efficient
                          // schedule): a tile is BM rows S apart, tile.seq_row0 the
                          // first destination row, tile.len the rows in the tile,
                          // sources shift rows earlier, in place; the state maps are
                          // 3-D (column, row in group of S, group)
  const void* vin_hi;     // residual planes (row-major [rows, m])
  const void* vin_lo;
  void* vout_hi;
  void* vout_lo;
  const float* C32;       // [nsys, q, m]   (fused output)
  const float* D32;       // [nsys, q, p]
  const float* u;         // [rows, p]
  float* y;               // [rows, q]
  int32_t gen;            // stage 1 with v^(1) formed on chip from u (vin not read)
  const float* Bb;        // [nsys, m, p] Bbar            (gen)
  const float* ABb;       // [nsys, m, p] Abar Bbar       (gen)
  int32_t* err;           // device error word
  int32_t* diag;          // where the first bounded wait gave up (5 words) or null
  unsigned long long timeout_ns;
};

// ---------------------------------------------------------------- device side
#ifdef __CUDACC__
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#endif

// Time-reduction chunk list (backward): offsets into Plan::d_chunk_data.
struct ChunkList {
  int n = 0;
  size_t off_chunks = 0;
  size_t off_begin = 0;
};

// ------------------------------------------------------------- plan (host)
struct Plan {
  cascade_desc_t d;
  int device = 0;
  int num_sms = 0;
  std::string last_error;
  // systems
  bool have_system = false;
  bool continuous = false;
  int kmax1 = 0;                 // entries in the power table per system
  double* P64 = nullptr;         // [nsys, kmax1, m, m]
  void* Phi = nullptr;           // operand planes [nsys, kmax1, m, m] (bf16 or fp32)
  void* Plo = nullptr;
  void* PThi = nullptr;          // transposed powers (adjoint stages), same format
  void* PTlo = nullptr;
  double* PT64 = nullptr;        // transposed FP64 powers (FP64 adjoint stages)
  double* Minv64 = nullptr;      // (I - delta/2 A)^-1 per system (discretisation adjoint)
  float* P32 = nullptr;          // FP32 copies for the backward's small algebra
  float* Minv32 = nullptr;
  double* Bbar64 = nullptr;      // [nsys, m, p]
  double* ABbar64 = nullptr;     // [nsys, m, p]   Abar * Bbar (first stage fused with Bbar u)
  double* C64 = nullptr;         // [nsys, q, m]
  double* D64 = nullptr;         // [nsys, q, p]
  float* Bbar32 = nullptr;
  float* ABbar32 = nullptr;
  float* C32 = nullptr;
  float* D32 = nullptr;
  // (hi, lo) BF16 planes of the small matrices for the tensor-core projections
  // (PC_* below, all systems of each matrix contiguous; null unless supported)
  void* pc_hi = nullptr;
  void* pc_lo = nullptr;
  int64_t pc_off[8] = {};
  double* A64 = nullptr;         // continuous A (for the discretisation adjoint) [nsys,m,m]
  double* B64 = nullptr;         // continuous B [nsys,m,p]
  double* delta64 = nullptr;     // [nsys]
  double* scale64 = nullptr;     // [nsys] or null
  // zero-order hold (CASCADE_FLAG_ZOH): squarings of the forward exponential and
  // of the adjoint's block exponential, per system, and their scale factors
  std::vector<int> zoh_sq, zoh_sq_adj;
  double* zoh_f_adj = nullptr;   // [nsys] 2^-zoh_sq_adj
  std::vector<int32_t> N_sys;
  bool lower_powers = false;     // every Abar lower-triangular: triangular squaring chain
  int32_t* err = nullptr;        // device error word, then 7 diagnostic words
  // batch
  bool have_batch = false;
  int64_t rows = 0;
  int nseq = 0;
  int maxN = -1;                 // largest per-sequence N in the batch
  std::vector<int64_t> offsets;
  std::vector<int32_t> sys_of_seq;
  std::vector<int32_t> seq_N;
  std::vector<std::vector<Tile>> h_tiles;   // per stage k = 1..maxN
  std::vector<Tile*> d_tiles;                // device copies
  std::vector<int32_t> n_tiles;
  std::vector<std::vector<Tile>> h_adj_tiles;   // adjoint stage k = 1..maxN (all tiles)
  std::vector<Tile*> d_adj_tiles;
  std::vector<int32_t> n_adj_tiles;
  Tile* d_all_tiles = nullptr;               // every tile of every sequence (flags = N_i,
                                             // fbuf = buffer of its final states)
  int n_all_tiles = 0;
  int all_fbuf = -1;                         // fbuf shared by every tile, or -1
  std::vector<ChunkList> chunk_lists;        // [0]: every tile; [k]: tiles of stage k
  int32_t* d_chunk_data = nullptr;           // chunks [n][3] (first tile, count, system) and
                                             // per-system chunk ranges [nsys + 1] of each list
  int max_chunks = 0;                        // chunks of the largest stage list
  int chunks_all = 0;                        // chunks of the list of all tiles
  void* d_red_scratch = nullptr;             // group sums of the chunk reductions
  size_t red_scratch_bytes = 0;
  const void* saved_ws = nullptr;            // workspace of the last forward that kept states
  int64_t saved_batch = -1;
  Seq* d_seqs = nullptr;                     // all sequences
  int n_out_tiles = 0;                       // tiles of sequences whose output is not fused
  Tile* d_out_tiles = nullptr;               // (fbuf = workspace buffer of the final states)
  std::vector<std::array<int, 3>> out_segs;  // output tiles grouped by fbuf: (buf, first, count)
  Tile* d_stage0_tiles = nullptr;            // tiles for the first stage (all rows)
  int n_stage0_tiles = 0;
  bool fuse_output = false;
  // y = C v + D u formed on the tensor cores in the last stage (BF16 pairs, p and
  // q multiples of 16, q <= 64, §3 schedule), where fuse_output does not apply
  bool fuse_output_mma = false;
  std::vector<char> stage_fused;   // stage k of the §3 schedule holds fused tiles (per batch)
  // stages 1 .. fused_J of the §3 schedule run as one pass over overlapping
  // windows with the states on chip (0: not used; set per batch)
  int fused_J = 0;
  FusedWindow* d_fwin = nullptr;
  int n_fwin = 0;
  // stage 1 forms v^(1) = Bbar u_l + Abar Bbar u_(l-1) on chip; the first-stage
  // kernel does not run (set per batch)
  bool fuse_first = false;
  // work-efficient schedule: the first level stores only odd rows (and row 0),
  // the last down-sweep level forms its even rows' v^(1) from u (set per batch)
  bool scan_even_on_chip = false;
  // work-efficient schedule (CASCADE_FLAG_SCAN): its launches in order, each
  // one level k of the up-sweep or the down-sweep over rows 2^(k+1) apart
  struct ScanLevel {
    int k;
    int down;
    int n;            // tiles
    Tile* d_tiles;
  };
  std::vector<ScanLevel> scan;
  int64_t scan_rows_cap = 0;     // state rows allocated (a multiple of the largest 2^(k+1))
  int64_t* d_scan_rows = nullptr;  // rows l = 2^t - 1 of every sequence (never written by the
  int32_t* d_scan_rows_sys = nullptr;  // down-sweep) and their systems: their y when the
  int n_scan_rows = 0;                 // levels form y themselves
  int64_t matvecs = 0;           // products by powers in one forward of the batch
  // levels k >= scan_top_k0 (up and down) run in one launch, a block per sequence with
  // its compact rows in TMEM (-1: every level is its own launch); scan_top_pos: index in
  // `scan` of the first down-sweep level below k0 (the top launch runs before it)
  int scan_top_k0 = -1, scan_top_K = 0, scan_top_pos = 0;
  Seq* d_top_seqs = nullptr;
  int n_top_seqs = 0;
  // stage-output checkpoints (CASCADE_FLAG_RECOMPUTE): v^(j) is kept for
  // j = 1, 1 + ck_seg, 1 + 2 ck_seg, ... <= maxN; the backward recomputes the
  // others one segment at a time
  int ck_seg = 0, n_ck = 0;
  // tensor-core stage kernel shape: operand stages, epilogue ring slots,
  // chunks per epilogue step (0 = heuristic); set by cascade_autotune
  int tc_stages = 0, tc_ring = 0, tc_group = 0;
  // per stage k of the §3 schedule (forward, dense tiles), or per level of the
  // work-efficient schedule (entry k: up-sweep level k, 100 + k: down-sweep
  // level k): the autotuner's fastest shape, {0, 0, 0} where the plan-wide
  // shape applies
  std::vector<std::array<int32_t, 3>> tc_stage_shape;
  bool tuned = false;
  void* last_stream = nullptr;
  // per-launch stage timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;            // pairs per stage
  std::vector<int32_t> ev_k;
  int n_ev = 0;
  // host-buffer forward (cascade_forward_host): chunks of the first-stage and
  // output tile lists {first tile, tiles, first row, rows}, contiguous in rows, whose
  // copies overlap the projections; a plan-owned copy stream and its events
  std::vector<std::array<int64_t, 4>> io_in, io_out;
  cudaStream_t io_stream = nullptr;
  std::vector<cudaEvent_t> io_ev;
  // graph cache (recorded on a plan-owned stream: the legacy default stream
  // cannot be captured; the graph is then launched on the caller's stream)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  const void* graph_key[3] = {nullptr, nullptr, nullptr};
  int64_t graph_batch_id = -1;
  int64_t batch_id = 0;
};

// Geometry helpers shared by host code.
int tile_rows(const Plan& p);                 // BM for the plan's precision
int block_n(int m, int precision);            // BN for tensor-core precisions
size_t plane_elem_bytes(int precision);       // bytes per element per plane
size_t state_bytes_per_row(const Plan& p);    // bytes of one state row (all planes)

// Kernel launchers (defined in the .cu files).
cudaError_t launch_discretise(const double* A, const double* B, const double* delta,
                              const double* scale, double* Abar_out, int64_t abar_sys_stride,
                              double* Bbar_out, double* Minv_out, double* work, int nsys, int m,
                              int p, int32_t* singular, bool lower, cudaStream_t st);
// flag = 1 if a matrix of the batch has a non-zero above its diagonal
cudaError_t launch_upper_nonzero(const double* X, int64_t sys_stride, int ns, int m, int32_t* flag,
                                 cudaStream_t st);
// C = A B for lower-triangular n x n A, B (batched), skipping the exact zeros
cudaError_t launch_dgemm_lower(const double* A, const double* B, double* C, int n, int64_t sA,
                               int64_t sB, int64_t sC, int batch, cudaStream_t st);
cudaError_t launch_dgemm(const double* A, const double* B, double* C, int M, int N, int K,
                         int lda, int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC,
                         int batch, double alpha, double beta, bool transA, bool transB,
                         cudaStream_t st);
cudaError_t launch_frob_norms(const double* P, int nmat, int64_t elems, double* out,
                              cudaStream_t st);
cudaError_t launch_split_planes(const double* src, void* hi, void* lo, int64_t n, int precision,
                                cudaStream_t st);
cudaError_t launch_to_f32(const double* src, float* dst, int64_t n, cudaStream_t st);

cudaError_t launch_stage0(const Plan& p, const void* u, void* out_hi, void* out_lo,
                          cudaStream_t st);
cudaError_t launch_stage_f64(const Plan& p, int k, const double* vin, double* vout,
                             cudaStream_t st, bool reverse = false);
// u_hi, u_lo: u as (hi, lo) BF16 planes [rows, p], read by the last stage when
// it forms y = C v + D u on the tensor cores (Plan::fuse_output_mma).
cudaError_t launch_stage_tc(const Plan& p, int k, const void* vin_hi, const void* vin_lo,
                            void* vout_hi, void* vout_lo, const float* u, float* y,
                            cudaStream_t st, bool reverse = false, const void* u_hi = nullptr,
                            const void* u_lo = nullptr);
// In-place stage k over rows S apart (the work-efficient schedule); the state
// planes hold rows_cap rows, a multiple of S.  Tiles flagged TILE_FINAL_FUSED
// also form y = C v + D u for their rows (u, y may be null otherwise).
// even_resid: the destination rows are even rows of the work-efficient
// schedule's last level; their v^(1) = Bbar u is formed from u, not read, and
// only y is written.
cudaError_t launch_stage_tc_strided(const Plan& p, int k, int S, const Tile* tiles, int ntiles,
                                    uint64_t rows_cap, void* v_hi, void* v_lo, const float* u,
                                    float* y, cudaStream_t st, bool even_resid = false,
                                    int shape_key = -1);
// Workspace buffer j of a family of equally sized state buffers.
struct Bufs {
  uint8_t* base;
  size_t stride;      // bytes between buffers
  size_t lo_off;      // bytes from a buffer's hi plane to its lo plane (0: single plane)
  __host__ __device__ void* hi(int j) const { return base + (size_t)j * stride; }
  __host__ __device__ void* lo(int j) const {
    return lo_off ? base + (size_t)j * stride + lo_off : nullptr;
  }
};
cudaError_t launch_output(const Plan& p, const void* u, void* y, const Bufs& V, cudaStream_t st);

// Row-indexed operand of a time reduction (backward.cu).
struct TSrc {
  int kind;          // 0: workspace state buffer, 1: dense float [rows, ld], 2: dense double
  Bufs bufs;         // kind 0
  int buf_mode;      // 0: buffer buf_fixed; 1: buffer = tile.fbuf
  int buf_fixed;
  const void* dense; // kinds 1, 2
  int ld;
};
cudaError_t launch_treduce(const Plan& p, const Tile* tiles, const int32_t* chunks, int nchunks,
                           const int32_t* sys_begin, const TSrc& X, int a, const TSrc& Y, int b,
                           int shift, void* partial, void* out, bool out_f64,
                           int64_t out_sys_stride, int accumulate, cudaStream_t st);
cudaError_t launch_adj_init(const Plan& p, const void* G, const Bufs& W, cudaStream_t st);
// du and R1, R2 in one pass over W^(1) (p, q <= 4, ceil(m / 256) p <= 2)
bool first_adj_thin_supported(const Plan& p);
cudaError_t launch_first_adj_thin(const Plan& p, const Tile* tiles, const int32_t* chunks,
                                  int nchunks, const int32_t* sys_begin, const Bufs& W, int wbuf,
                                  const float* u, const float* G, float* du, float* partial,
                                  void* out, bool out_f64, int64_t out_sys_stride,
                                  int64_t seg_stride, cudaStream_t st);
// Wide-by-thin time reduction (one narrow side, see backward.cu); false if the
// shape is outside what the kernel handles (the caller then uses launch_treduce).
bool wtreduce_supported(const Plan& p, int a, int tc, int nsh);
cudaError_t launch_wtreduce(const Plan& p, const Tile* tiles, const int32_t* chunks, int nchunks,
                            const int32_t* sys_begin, const TSrc& X, int a, const void* T, int tc,
                            int nsh, int sh0, int sh1, bool thin_major, void* partial, void* out,
                            bool out_f64, int64_t out_sys_stride, int64_t seg_stride,
                            cudaStream_t st);
// Narrow projections as register-tiled GEMMs (proj.cu; tensor-core formats).
bool proj_supported(const Plan& p);
bool scan_top_supported(const Plan& p);
cudaError_t launch_scan_top(const Plan& p, void* v_hi, void* v_lo, uint64_t rows_cap,
                            const float* u, float* y, cudaStream_t st);
// Stages 1 .. fused_J in one pass from u (stage_fused.cu): BF16 split, p = 1,
// m = 128 or 256; writes v^(fused_J + 1).
bool fused_stages_supported(const Plan& p);
cudaError_t launch_fused_stages(const Plan& p, const float* u, void* vout_hi, void* vout_lo,
                                cudaStream_t st);
// Tensor-core projections (proj_tc.cu): BF16 split with p and q multiples of 16.
// The B operands are the PC_* matrices, split at set_system time.
enum { PC_B = 0, PC_AB, PC_C, PC_D, PC_CT, PC_BT, PC_ABT, PC_DT, PC_COUNT };
bool proj_tc_supported(const Plan& p);
size_t proj_coef_elems(const Plan& p, int64_t off[PC_COUNT]);
cudaError_t launch_proj_coef(const Plan& p, cudaStream_t st);
// FP32 rows of w entries -> (hi, lo) BF16 planes of rows of wp >= w entries (zero past w)
cudaError_t launch_split_rows(const float* x, int64_t rows, int w, int wp, void* hi, void* lo,
                              cudaStream_t st);
// U, G: (hi, lo) BF16 planes of u [rows, p] and G [rows, q] (buffer 0 of the Bufs)
// (tile0, ntiles: a range of the first-stage or output tile list; ntiles < 0: to
// its end)
cudaError_t launch_proj_tc_stage0(const Plan& p, const Bufs& U, const Bufs& V, int64_t v_rows,
                                  int buf, bool odd_only, cudaStream_t st, int tile0 = 0,
                                  int ntiles = -1);
cudaError_t launch_proj_tc_output(const Plan& p, const Bufs& U, float* y, const Bufs& V,
                                  int64_t v_rows, cudaStream_t st, int tile0 = 0,
                                  int ntiles = -1);
cudaError_t launch_proj_tc_adj_init(const Plan& p, const Bufs& G, const Bufs& W, cudaStream_t st);
cudaError_t launch_proj_tc_du(const Plan& p, const Bufs& G, const Bufs& W, int wbuf, float* du,
                              cudaStream_t st);
cudaError_t launch_proj_stage0(const Plan& p, const float* u, const Bufs& V, int buf,
                               int odd_mode, cudaStream_t st);
cudaError_t launch_proj_adj_init(const Plan& p, const float* G, const Bufs& W, cudaStream_t st);
cudaError_t launch_proj_output(const Plan& p, const float* u, float* y, const Bufs& V,
                               cudaStream_t st);
cudaError_t launch_proj_du(const Plan& p, const float* G, const Bufs& W, int wbuf, float* du,
                           cudaStream_t st);
// y = C v + D u for an explicit list of rows (state buffer `buf`).
cudaError_t launch_proj_rows_output(const Plan& p, const int64_t* rows, int nrows,
                                    const int32_t* row_sys, const float* u, float* y,
                                    const Bufs& V, int buf, cudaStream_t st);
cudaError_t launch_reduce_partials(const Plan& p, const float* partial, const int32_t* sys_begin,
                                   int64_t elems, void* out, bool out_f64, int64_t out_sys_stride,
                                   cudaStream_t st);
bool grad_tc_supported(const Plan& p);
int grad_tc_block_n(int m);
// The time reductions can run on the power-gradient kernel: BF16-split plans with m a
// multiple of 128 (u and G as planes of rows padded to multiples of 8 entries).
bool thin_tc_supported(const Plan& p);
cudaError_t launch_grad_tc_xy(const Plan& p, const Tile* tiles, const int32_t* chunks,
                              int nchunks, const void* x_hi, const void* x_lo, int ma, int ldx,
                              const void* y_hi, const void* y_lo, int nb, int ldy, int shift,
                              bool trans, float* partial, cudaStream_t st);
inline int pad8(int w) { return (w + 7) & ~7; }
cudaError_t launch_grad_tc(const Plan& p, const Tile* tiles, const int32_t* chunks, int nchunks,
                           const void* w_hi, const void* w_lo, const void* v_hi, const void* v_lo,
                           int shift, float* partial, cudaStream_t st);
cudaError_t launch_stage0_adj(const Plan& p, const void* G, const Bufs& W, int wbuf, void* du,
                              cudaStream_t st);
cudaError_t launch_transpose(const double* in, double* out, int n, int64_t stride, int batch,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_axpy_sys(const T* x, int64_t x_stride, T* y, int64_t y_stride, int64_t n,
                            int nsys, const double* scal, double factor, bool accumulate,
                            cudaStream_t st);
template <typename TI, typename TO>
cudaError_t launch_convert_sys(const TI* in, int64_t in_stride, TO* out, int64_t out_stride,
                               int64_t n, int nsys, cudaStream_t st);
// Batched GEMM in float (same contract as launch_dgemm).
cudaError_t launch_sgemm(const float* A, const float* B, float* C, int M, int N, int K, int lda,
                         int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC, int batch,
                         float alpha, float beta, bool transA, bool transB, cudaStream_t st);
// C = alpha (op(A1) op(B1) + op(A2) op(B2)) + beta C in FP32, batched; A2 = null: one
// product.  Both products share the leading dimensions and batch strides.  With
// few output tiles the K range is split over blocks when `scratch` (device
// floats) has room for the partial products; they are added in a fixed order.
cudaError_t launch_sgemm2(const float* A1, const float* B1, bool tA1, bool tB1, const float* A2,
                          const float* B2, bool tA2, bool tB2, float* C, int M, int N, int K,
                          int lda, int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC,
                          int batch, float alpha, float beta, cudaStream_t st,
                          float* scratch = nullptr, size_t scratch_floats = 0);
cudaError_t launch_recursion_f64(const Plan& p, const double* u, double* y, cudaStream_t st);
// Squaring-chain adjoint on the tensor cores (chain_tc.cu, BF16-split plans).
bool chain_tc_supported(const Plan& p);
size_t chain_tc_scratch_bytes(const Plan& p);
cudaError_t launch_chain_tc(const Plan& p, int k, bool first, float* dP, int64_t kst,
                            void* scratch, cudaStream_t st);
// Zero-order hold (zoh.cu): matrix exponentials by scaling and squaring, FP64.
size_t expm_scratch_doubles(int n, int ns);
int expm_squarings(double norm1);
cudaError_t expm_batched(double* X, int n, int ns, const std::vector<int>& sq, const double* d_f,
                         double* scratch, int32_t* singular, cudaStream_t st);
cudaError_t launch_zoh_block(const double* A, const double* B, const double* delta, double* Z,
                             int m, int p, int ns, bool transpose, cudaStream_t st);
cudaError_t launch_norms(const double* X, int n, int ns, double* n1, double* ninf,
                         cudaStream_t st);
cudaError_t launch_frechet_block(const double* ZT, const double* dAbar, const double* dBbar,
                                 const double* scale, double* W, double* gnorm, int m, int p,
                                 int ns, cudaStream_t st);
cudaError_t launch_block(const double* X, int n, int r0, int c0, int rows, int cols, double* out,
                         int64_t out_stride, const double* f, double c, int ns, cudaStream_t st);
cudaError_t launch_selftest_timeout(int32_t limit_us, int32_t* err, cudaStream_t st);

// Shape of the tensor-core stage kernel (see stage_tc.cu).
struct TcConfig {
  int stages;   // operand pipeline depth
  int ring;     // epilogue residual staging slots
  int group;    // column chunks per epilogue step
};
std::vector<TcConfig> tc_candidates(int m, int precision);
TcConfig tc_default(int m, int precision);

// Tensor-map encoder resolved through the runtime's driver entry point.
bool encode_tmap_2d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t inner,
                    uint64_t outer, uint32_t box_inner, uint32_t box_outer, std::string* err,
                    int swizzle_bytes = 128);
bool encode_tmap_colblocks(CUtensorMap* map, const void* base, int elem_bytes, uint64_t cols,
                           uint64_t rows, uint32_t box_rows, uint32_t box_blocks,
                           std::string* err, int swizzle_bytes = 64);
// Row-major [groups * S, inner] viewed as (inner, S, groups); box (box_inner, 1, box_groups).
bool encode_tmap_3d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t inner,
                    uint64_t S, uint64_t groups, uint32_t box_inner, uint32_t box_groups,
                    std::string* err, int swizzle_bytes = 128);

}  // namespace cascade
