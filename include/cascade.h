/*
 * cascade.h -- C ABI of the GB300 (sm_103a) cascade library.
 *
 * The library applies the transfer function of a discrete linear
 * time-invariant system,
 *
 *     H(z) = C (I - z^-1 Abar)^-1 Bbar + D                       (Eq. 1.3)
 *
 * to packed input sequences in the time domain, with the unconditionally
 * stable cascade of Beylkin, "Fast convolution algorithm for state space
 * models" (arXiv 2411.17729): the resolvent is truncated to the product of
 * N+1 factors I + (z^-1 Abar)^(2^k) (Eq. 2.2), the powers Abar^(2^k) are
 * formed by repeated squaring in FP64 (end of §2, §4), and the stages
 *
 *     v_l <- v_l + Abar^(2^k) v_(l - 2^k),   k = 0..N             (Eqs. 3.2-3.4)
 *
 * are applied to v^(0) = Bbar u, followed by y = C v + D u (end of §3).
 *
 * Conventions shared by every call:
 *   - Matrices are row-major (last index fastest).  System matrices carry a
 *     leading system axis: A is [nsys, m, m], B is [nsys, m, p], C is
 *     [nsys, q, m], D is [nsys, q, p], delta is [nsys].
 *   - Sequences are packed time-major: u is [rows, p], y is [rows, q], with
 *     rows = offsets[nseq]; sequence i occupies rows offsets[i]..offsets[i+1]-1.
 *   - Pointers named d_* are DEVICE pointers (caller-owned; the library never
 *     frees them); pointers named h_* are HOST pointers read during the call.
 *   - u/y/du/dy element type is double for CASCADE_FP64 plans and float
 *     otherwise.  System matrices and their gradients are always double.
 *   - `stream` is a cudaStream_t (0 = legacy default stream).  Calls that
 *     launch work are asynchronous on that stream unless stated otherwise.
 *     The tensor-core kernels are programmatic dependent launches: each may
 *     start its set-up while the previous kernel of the stream finishes, and
 *     waits for that kernel before touching memory.  Each also allows the next
 *     kernel to do the same; a caller's kernel launched without the
 *     programmatic-serialization attribute still starts after the library's
 *     last kernel has completed, as with any stream.
 *   - Every call returns a cascade_status_t; no call aborts or throws.  On
 *     failure the plan keeps its previous state and cascade_last_error()
 *     returns a one-line description.
 */
#ifndef GB300_CASCADE_H
#define GB300_CASCADE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CASCADE_OK = 0,
  CASCADE_ERR_INVALID_ARG = 1,   /* bad pointer, size, shape or layout        */
  CASCADE_ERR_UNSUPPORTED = 2,   /* valid request this build does not serve   */
  CASCADE_ERR_OOM = 3,           /* device allocation failed                  */
  CASCADE_ERR_CUDA = 4,          /* a CUDA runtime/driver call failed         */
  CASCADE_ERR_TIMEOUT = 5,       /* a bounded device wait expired             */
  CASCADE_ERR_STATE = 6          /* call order violated (e.g. no system set)  */
} cascade_status_t;

typedef enum {
  /* FP64 storage and FP64 arithmetic on the CUDA cores.                     */
  CASCADE_FP64 = 0,
  /* Stage contractions as three TF32 tensor-core products
     (hi*hi + hi*lo + lo*hi) with FP32 accumulation in TMEM; states stored
     as a pair of TF32-exact FP32 planes (hi + lo carries ~22 bits).  The
     tensor core adds each 8-term K step into the FP32 sum with a truncating
     add, so the error grows with m (about 1e-5 relative at m = 1024).       */
  CASCADE_FP32 = 1,
  /* Stage contractions as three BF16 tensor-core products with FP32
     accumulation in TMEM; states stored as a BF16 (hi, lo) pair.            */
  CASCADE_BF16_SPLIT = 2
} cascade_precision_t;

enum {
  /* Keep every stage output v^(k) in the workspace so that cascade_backward
     can run: maxN + 1 state buffers.                                        */
  CASCADE_FLAG_SAVE_STATES = 1,
  /* Keep only checkpoints v^(1), v^(1+c), v^(1+2c), ... and recompute the
     other stage outputs in cascade_backward, one segment of c stages at a
     time (c is chosen per batch to minimise the buffers; about 2 sqrt(N)
     state buffers instead of N + 1, for maxN - ceil(maxN / c) extra stage
     passes).  Results are bitwise equal to CASCADE_FLAG_SAVE_STATES.  Takes
     precedence when both flags are given.                                  */
  CASCADE_FLAG_RECOMPUTE = 2,
  /* Do not fuse y = C v + D u into the last stage (diagnostics).  The fused
     output is formed on the CUDA cores in the epilogue for q <= 4 when one
     tile spans all m columns, and on the tensor cores (a second tcgen05
     product of the finished state tile with C, plus D u) for BF16-split
     plans with p and q multiples of 16 and q <= 64.                         */
  CASCADE_FLAG_NO_FUSED_OUTPUT = 4,
  /* Record the forward launch sequence once per (u, y, workspace) triple in
     a CUDA graph and replay it on later calls.                             */
  CASCADE_FLAG_GRAPH = 8,
  /* Forward with the work-efficient schedule of the abstract and §6 instead
     of the §3 one: an up-sweep applies Abar^(2^k) to every 2^(k+1)-th entry
     (k = 0..K-1, K = ceil(log2 L)), a down-sweep fills the entries in between
     (k = K-2..0), about 2L products by powers per sequence instead of
     sum_k (L - 2^k).  In place on one state buffer.  The outputs equal the
     §3 cascade's up to rounding when 2^(N_i+1) >= L_i, which cascade_set_batch
     requires (CASCADE_ERR_UNSUPPORTED otherwise).  Tensor-core precisions
     only; no backward (CASCADE_ERR_INVALID_ARG with SAVE_STATES/RECOMPUTE). */
  CASCADE_FLAG_SCAN = 16,
  /* cascade_set_system_continuous discretises by the zero-order hold of §5,
     Abar = exp(delta A), Bbar = (delta A)^-1 (exp(delta A) - I) delta B (the
     printed last factor delta A read as delta B), instead of Eq. (4.2); both
     blocks come from one exponential of delta [[A, B], [0, 0]], so A need not
     be invertible.  FP64 scaling and squaring with a [13/13] Pade approximant.
     The backward's dA, dB go through the Frechet derivative of the
     exponential.                                                           */
  CASCADE_FLAG_ZOH = 32,
  /* Write v^(1) = Bbar u_l + Abar Bbar u_(l-1) (the first stage, §3) to
     device memory and read it back, instead of forming it on chip where it
     is used (diagnostics).  Forming it on chip applies to tensor-core plans
     with p = 1: on the §3 schedule (no stage outputs kept) inside stage 1,
     with sequences too short for a stage 1 (N_i = 0) still written since
     their output reads it; on the work-efficient schedule with the output
     fused, for the even rows in the last down-sweep level.  Results are the
     same bit for bit (cascade_get_first_fused).                           */
  CASCADE_FLAG_NO_FUSED_FIRST = 64,
  /* Discretise and square with the dense kernels even when every A (or Abar)
     is lower-triangular (diagnostics).  For lower-triangular systems, such as
     HiPPO-LegS, the set-up otherwise solves Eq. (4.2) by forward elimination
     without row exchanges (a triangular system needs none), over the non-zero
     triangle only, so Abar comes out exactly lower-triangular, and squares it
     with a triangular product that leaves out only exact zeros.  Where the
     dense elimination exchanges no rows either (small delta), the powers are
     the same bit for bit.                                                  */
  CASCADE_FLAG_DENSE_SETUP = 128,
  /* Form y = C v + D u on the tensor cores in the last stage also when m spans
     several column blocks of the stage kernel (m > 256): one block then takes
     a tile's column blocks one after the other and adds their partial y in a
     fixed order.  Off by default: at m = 1024, q = 64 the slots' K chunks of C
     leave room for only two operand stages, and the last stage with the output
     took 2.2 ms against 1.3 ms plus a 0.45 ms separate projection (GB300). */
  CASCADE_FLAG_FUSE_WIDE_OUTPUT = 256,
  /* Run stages 1, 2, 3 of the §3 schedule as separate launches through device
     memory (diagnostics).  By default forward-only plans with BF16 pairs,
     p = 1, m = 128 or 256, whose sequences all run more than 3 stages, run
     them as one pass over overlapping windows of 128 steps that keeps the
     states on chip (FP32 between the stages, so the results agree with the
     separate launches to rounding, not bit for bit); see
     cascade_get_fused_stages.                                              */
  CASCADE_FLAG_NO_FUSED_STAGES = 512
};

typedef struct cascade_plan_s* cascade_plan_t;

typedef struct {
  int32_t m, p, q;      /* state, input and output sizes, 1 <= p, q; m >= 1 (§1, Eq. 1.1) */
  int32_t nsys;         /* number of distinct systems (each sequence names one)          */
  int32_t N;            /* stages k = 0..N; N < 0 chooses N per system from eps          */
  int32_t precision;    /* cascade_precision_t                                            */
  int32_t max_len;      /* longest sequence the plan will see (sizes the power table)    */
  int32_t flags;        /* CASCADE_FLAG_*                                                 */
  int64_t max_rows;     /* most packed rows one batch may hold                            */
  double eps;           /* accuracy target when N < 0 (Lemma 1, remainder reading)        */
} cascade_desc_t;

/* Human-readable name of a status code.  Never NULL. */
const char* cascade_status_string(cascade_status_t status);

/* Last error message recorded on `plan` ("" if none).  Valid until the next
   call on the same plan.  plan may be NULL (returns the last global error). */
const char* cascade_last_error(cascade_plan_t plan);

/* Create a plan for the problem shape of §1 (Eq. 1.1) on the current CUDA
   device.  Validates the descriptor (INVALID_ARG) and the precision x m
   combination (UNSUPPORTED: the tensor-core precisions need m % 64 == 0 for
   BF16 and m % 32 == 0 for FP32, m <= 4096).  The plan owns the device
   copies of the discretised systems and their powers; nothing is allocated
   for sequences (see cascade_workspace_size).  *plan is NULL on failure. */
cascade_status_t cascade_plan_create(cascade_plan_t* plan, const cascade_desc_t* desc);

/* Release every resource the plan owns.  Synchronises the device first.
   NULL is ignored. */
void cascade_plan_destroy(cascade_plan_t plan);

/* Set continuous systems and discretise them with the trapezoidal rule of
   §1 (after Eq. 1.2) and Eq. (4.2):
       Abar = (I - delta/2 A)^-1 (I + delta/2 A),   Bbar = delta (I - delta/2 A)^-1 B,
   then multiply Abar by d_abar_scale[s] if that pointer is not NULL (used to
   place eigenvalues just outside the unit circle, §6).  Afterwards the powers
   Abar^(2^k) are formed by FP64 repeated squaring on the device (end of §2),
   N is chosen per system (desc.N, or from eps when desc.N < 0: the smallest
   N with 2^(N+1) >= max_len or ||Abar^(2^(N+1))||_F <= eps), and the powers
   are converted to the plan's operand format.
   Device inputs: d_A [nsys,m,m], d_B [nsys,m,p], d_delta [nsys],
   d_abar_scale [nsys] or NULL, d_C [nsys,q,m], d_D [nsys,q,p], all double.
   Synchronises `stream` before returning (N is read back to the host).
   Returns CASCADE_ERR_INVALID_ARG for a singular I - delta/2 A. */
cascade_status_t cascade_set_system_continuous(cascade_plan_t plan, const double* d_A,
                                               const double* d_B, const double* d_delta,
                                               const double* d_abar_scale, const double* d_C,
                                               const double* d_D, void* stream);

/* Set already-discrete systems (Eq. 1.2): d_Abar [nsys,m,m], d_Bbar
   [nsys,m,p], d_C, d_D as above, all double.  Then as the continuous call
   (powers, N, operand conversion).  Synchronises `stream`. */
cascade_status_t cascade_set_system_discrete(cascade_plan_t plan, const double* d_Abar,
                                             const double* d_Bbar, const double* d_C,
                                             const double* d_D, void* stream);

/* Copy the per-system N chosen by the last set_system call into h_N[nsys]. */
cascade_status_t cascade_get_N(cascade_plan_t plan, int32_t* h_N);

/* Copy the FP64 powers Abar^(2^k), k = 0..kmax, of system `sys` to the
   device buffer d_out [kmax+1, m, m] (double).  kmax may not exceed the
   plan's power-table size minus one (INVALID_ARG).  Asynchronous. */
cascade_status_t cascade_get_powers(cascade_plan_t plan, int32_t sys, int32_t kmax,
                                    double* d_out, void* stream);

/* Describe the packed batch the next forward/backward calls process:
   h_offsets [nseq+1] (int64, offsets[0] == 0, non-decreasing, last <=
   desc.max_rows, every length <= desc.max_len) and h_sys_of_seq [nseq]
   (each in 0..nsys-1; NULL means system 0 for every sequence).  Empty
   sequences are allowed.  Builds the per-stage tile schedules on the host
   and uploads them (synchronous).  Requires a system (CASCADE_ERR_STATE). */
cascade_status_t cascade_set_batch(cascade_plan_t plan, const int64_t* h_offsets, int32_t nseq,
                                   const int32_t* h_sys_of_seq);

/* Per-sequence N actually run (N of its system clipped so that 2^N < L):
   h_N [nseq]. */
cascade_status_t cascade_get_seq_N(cascade_plan_t plan, int32_t* h_N);

/* Products of a power Abar^(2^k) with a state vector that one forward over
   the current batch executes (summed over sequences): sum_k (L_i - 2^k)^+
   for the §3 schedule, about 2 L_i with CASCADE_FLAG_SCAN.  The input
   projection's Abar Bbar u term of the first stage counts as one per row it
   is applied to.  Host-side count of the schedule; *h_count. */
cascade_status_t cascade_get_matvec_count(cascade_plan_t plan, int64_t* h_count);

/* Whether the output y = C v + D u (§3) is formed in the epilogue of each
   sequence's last stage (the stage then reads v^(N_i) and u and writes y;
   it writes v^(N_i+1) only when the plan keeps its stage outputs), or by a
   separate projection after the last stage.  Fixed at plan creation: FP32
   or BF16-split plans with q <= 4 whose stage tiles span all m columns (y on
   the CUDA cores), and BF16-split plans on the §3 schedule with p and q
   multiples of 16, q <= 64 and m <= 256 (one column block; y on the tensor
   cores: the finished (hi, lo) state chunks times C, plus u times D,
   accumulated in TMEM), or any m with CASCADE_FLAG_FUSE_WIDE_OUTPUT, unless
   created with CASCADE_FLAG_NO_FUSED_OUTPUT.  *h_fused = 1 or 0. */
cascade_status_t cascade_get_output_fused(cascade_plan_t plan, int32_t* h_fused);

/* Whether first-stage values v^(1) = Bbar u_l + Abar Bbar u_(l-1) are formed
   on chip for the current batch instead of read from memory (p = 1, not
   disabled by CASCADE_FLAG_NO_FUSED_FIRST).  §3 schedule (no stage outputs
   kept): stage 1 reads u instead of v^(1), and the first-stage kernel runs
   only for sequences with N_i = 0.  Work-efficient schedule (fused output):
   the first level stores only the odd rows and row 0, and the last
   down-sweep level forms the even rows' v^(1) = Bbar u_l from u and writes
   only y.  *h_fused = 1 or 0; CASCADE_ERR_STATE before cascade_set_batch. */
cascade_status_t cascade_get_first_fused(cascade_plan_t plan, int32_t* h_fused);

/* Number of leading stages (1 .. J) of the §3 schedule that the current
   batch's forward runs as one pass from u with the states on chip, or 0
   (CASCADE_FLAG_NO_FUSED_STAGES).  *h_J; CASCADE_ERR_STATE before
   cascade_set_batch. */
cascade_status_t cascade_get_fused_stages(cascade_plan_t plan, int32_t* h_J);

/* Size of the fixed device scratch array behind cascade_forward_fixed_scratch. */
#define CASCADE_FIXED_SCRATCH_BYTES ((size_t)32 << 20)

/* Bytes of caller-provided device workspace that forward (and, for plans
   with CASCADE_FLAG_SAVE_STATES or CASCADE_FLAG_RECOMPUTE, backward) need for
   the current batch. */
cascade_status_t cascade_workspace_size(cascade_plan_t plan, size_t* bytes);

/* Apply the truncated transfer function to the current batch (§3):
   v^(0) = Bbar u, stages k = 0..N_i, y = C v + D u.  d_u [rows,p] and d_y
   [rows,q] in the plan's element type, 16-byte aligned (some paths move their
   rows in 16-byte words; CASCADE_ERR_INVALID_ARG otherwise); d_workspace of at
   least cascade_workspace_size bytes, 256-byte aligned.  Asynchronous on stream;
   device-side wait timeouts are reported by cascade_get_device_error. */
cascade_status_t cascade_forward(cascade_plan_t plan, const void* d_u, void* d_y,
                                 void* d_workspace, size_t workspace_bytes, void* stream);

/* cascade_forward with the input and the output in host memory (the call a
   host program makes): copies h_u [rows,p] to d_u, runs cascade_forward into
   d_y, copies d_y [rows,q] to h_y, and waits for the copy on `stream`.  d_u,
   d_y and the workspace are caller-owned device buffers as for
   cascade_forward; h_u, h_y should be page-locked for the copies to run at
   full speed.  When the plan projects u and y on the tensor cores in launches
   of their own (p, q multiples of 16, output not formed in the last stage, no
   CASCADE_FLAG_GRAPH), the copies run in row chunks on a plan-owned stream
   beside those projections; results are the same bit for bit.  The caller's
   stream then also waits for the copies.  Returns CASCADE_ERR_TIMEOUT when a
   bounded device wait of this forward gave up (the device error word stays
   set for cascade_get_device_error).  Synchronous, on errors too: when it
   returns, no copy it started still reads h_u or writes h_y. */
cascade_status_t cascade_forward_host(cascade_plan_t plan, const void* h_u, void* h_y, void* d_u,
                                      void* d_y, void* d_workspace, size_t workspace_bytes,
                                      void* stream);

/* cascade_forward without a workspace argument, for callers that cannot call
   cudaMalloc: for example a plugin that runs inside a host framework whose
   memory pool owns all device memory, or a latency-bound service path where
   a device allocation may synchronise the GPU.  (The paper has no
   counterpart: this is a deployment convenience of this library.)
   The workspace comes from a fixed array of CASCADE_FIXED_SCRATCH_BYTES
   (32 MiB) compiled into the library; every GPU that loads the library holds
   it until the process exits.  Batches whose workspace
   (cascade_workspace_size) exceeds it are rejected with
   CASCADE_ERR_UNSUPPORTED and a message giving both sizes; stage timing must
   be off (CASCADE_ERR_UNSUPPORTED otherwise).  The call makes no allocation
   of its own, but the array is a module variable: with lazy module loading
   (CUDA_MODULE_LOADING=LAZY, the default) the first call on each device
   loads it and commits its 32 MiB there, and a device that has no room
   left then fails with CASCADE_ERR_OOM; with eager loading the memory is
   committed when the library is loaded.  That first call resolves the
   array's device address (cudaGetSymbolAddress) with the device current;
   make it before any stream capture.  All calls share the one array, which
   keeps the last call's contents (the forward writes every byte it reads, so
   nothing needs clearing); calls whose executions overlap on the GPU, on any
   streams or plans, race on it and must be serialised by the caller.
   The call always launches the forward's kernels directly: a plan's
   CASCADE_FLAG_GRAPH applies to cascade_forward only.  Stage outputs that a
   CASCADE_FLAG_SAVE_STATES or CASCADE_FLAG_RECOMPUTE plan keeps are written
   into the shared array and are not available to cascade_backward, which
   still refers to the last cascade_forward with a caller workspace.
   Otherwise as cascade_forward: d_u [rows,p], d_y [rows,q], asynchronous. */
cascade_status_t cascade_forward_fixed_scratch(cascade_plan_t plan, const void* d_u, void* d_y,
                                               void* stream);

/* Reverse-mode derivative of sum(dy * y) for the last cascade_forward on
   this batch and workspace, which must come from a plan created with
   CASCADE_FLAG_SAVE_STATES or CASCADE_FLAG_RECOMPUTE (the forward then keeps
   every stage output, or checkpoints, in the workspace; CASCADE_ERR_STATE
   otherwise).  With checkpoints the call overwrites the forward's other state
   buffers; a second backward needs a new forward.  d_u is the forward's input,
   d_dy [rows,q] the output gradient (plan element type; d_u, d_dy and d_du
   16-byte aligned, the double outputs 8-byte aligned).  Writes d_du
   [rows,p] and, per system, d_dAbar [nsys,m,m], d_dBbar [nsys,m,p], d_dC
   [nsys,q,m], d_dD [nsys,q,p] (double): the gradients through the squaring
   chain (end of §2) and the stages (§3, derived adjoint: transposed powers,
   reversed shifts).  For continuous systems d_dA [nsys,m,m] and d_dB
   [nsys,m,p] are the gradients through Eq. (4.2).  Every entry of each
   requested output is written (not accumulated); a batch of no rows writes
   zeros and needs no u, dy or workspace.  Any output pointer may be NULL to
   skip it.  Asynchronous. */
cascade_status_t cascade_backward(cascade_plan_t plan, const void* d_u, const void* d_dy,
                                  void* d_du, double* d_dAbar, double* d_dBbar, double* d_dC,
                                  double* d_dD, double* d_dA, double* d_dB, void* d_workspace,
                                  size_t workspace_bytes, void* stream);

/* FP64 sequential recursion of Eq. (1.2), x_n = Abar x_(n-1) + Bbar u_n,
   y_n = C x_n + D u_n, one device thread block per sequence (the baseline
   the cascade replaces).  Uses the plan's systems and batch; d_u/d_y are
   double (8-byte aligned).  Asynchronous. */
cascade_status_t cascade_recursion_forward(cascade_plan_t plan, const double* d_u, double* d_y,
                                           void* stream);

/* Read and clear the device error word set by bounded waits in the plan's
   kernels (0 = none, otherwise a CASCADE_ERR_* code).  Synchronises the
   plan's last stream. */
cascade_status_t cascade_get_device_error(cascade_plan_t plan, int32_t* h_code);

/* Self-test of the bounded-wait path: launches one block that waits on an
   mbarrier no one arrives at, with a limit of `limit_us` microseconds, and
   returns CASCADE_ERR_TIMEOUT when the wait gave up (as it must).  The GPU
   context stays usable.  Synchronous. */
cascade_status_t cascade_selftest_timeout(int32_t limit_us);

/* Number of kernels this library launched since load (host-side count). */
int64_t cascade_launch_count(void);

/* Autotuner of the tensor-core stage kernel.  Runs the forward on the
   current batch once per candidate kernel shape (operand pipeline depth,
   epilogue staging ring, column chunks per epilogue step; every candidate
   fits shared and tensor memory), `reps` timed passes each after one
   warm-up, with CUDA events on `stream`, and keeps the fastest in the plan
   for later forwards.  On the §3 stage schedule each candidate also runs
   `reps` passes with every stage timed on its own, and each stage k keeps
   the candidate that ran it fastest (cascade_get_stage_shapes); the
   fastest whole forward's shape serves the adjoint stages and the scan
   levels.  d_u, d_y and d_workspace are as for cascade_forward (d_y is
   overwritten).  h_choice (NULL or int32[3]) receives the plan-wide
   stages, ring slots and chunks per step.  Synchronous; a no-op for FP64
   plans. */
cascade_status_t cascade_autotune(cascade_plan_t plan, const void* d_u, void* d_y,
                                  void* d_workspace, size_t workspace_bytes, void* stream,
                                  int32_t reps, int32_t* h_choice);

/* Set the tensor-core stage kernel shape directly (e.g. a shape saved from
   an earlier cascade_autotune): h_shape = {stages, ring slots, chunks per
   step}.  The kernel's two epilogue groups take alternate steps and each ring
   slot must always serve the same group, so ring slots must be a multiple of
   2 x chunks per step.  CASCADE_ERR_INVALID_ARG if that fails or the shape
   does not fit shared/tensor memory for this plan's m and precision.  The
   shape then applies to every stage (per-stage choices are cleared).  A
   no-op for FP64 plans. */
cascade_status_t cascade_set_kernel_shape(cascade_plan_t plan, const int32_t* h_shape);

/* Per-stage kernel shapes chosen by cascade_autotune: h_shape[3 k + j],
   j = stages, ring slots, chunks per step, for entry k < min(cap, *n);
   {0, 0, 0} where the plan-wide shape applies.  Entry k is stage k of the §3
   schedule; with CASCADE_FLAG_SCAN it is up-sweep level k, and entry 100 + k
   down-sweep level k.  *n = the number of entries the plan holds (0 before
   tuning or after cascade_set_kernel_shape). */
cascade_status_t cascade_get_stage_shapes(cascade_plan_t plan, int32_t cap, int32_t* h_shape,
                                          int32_t* n);

/* Set per-stage kernel shapes (e.g. saved from cascade_get_stage_shapes):
   n entries laid out as there.  Every non-zero entry must be a shape
   cascade_set_kernel_shape accepts for this plan, at an entry the current
   batch's schedule launches (§3: stages 1..maxN; work-efficient: its up- and
   down-sweep levels), and n may not exceed the entries that schedule has
   (maxN + 1, or 100 + maxN + 2): CASCADE_ERR_INVALID_ARG otherwise, nothing
   changed.  Needs a batch (CASCADE_ERR_STATE) unless n = 0, which clears
   them.  A no-op for FP64 plans. */
cascade_status_t cascade_set_stage_shapes(cascade_plan_t plan, int32_t n, const int32_t* h_shape);

/* Per-launch timing of the stage kernels.  When enabled, every later
   forward records a CUDA event pair on its stream around each tensor-core
   (or FP64) stage launch.  cascade_get_stage_times synchronises that stream
   and copies up to `cap` entries (stage index k, milliseconds) of the LAST
   forward into h_k / h_ms, returning the count in *n. */
cascade_status_t cascade_enable_stage_timing(cascade_plan_t plan, int32_t enable);
cascade_status_t cascade_get_stage_times(cascade_plan_t plan, int32_t cap, int32_t* h_k,
                                         float* h_ms, int32_t* n);

#ifdef __cplusplus
}
#endif
#endif /* GB300_CASCADE_H */
