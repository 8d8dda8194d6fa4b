// api.cu -- the C ABI declared in include/cascade.h: plan lifecycle, system
// preparation (discretisation, squaring chain, accuracy rule, operand
// planes), the per-stage tile schedule of a packed batch, and the forward.
#include "common.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <mutex>
#include <utility>

namespace cascade {

long long g_launches = 0;
static std::mutex g_err_mu;
static std::string g_err;

void set_global_error(const std::string& msg) {
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = msg;
}
std::string global_error() {
  std::lock_guard<std::mutex> lk(g_err_mu);
  return g_err;
}

int tile_rows(const Plan& p) { return p.d.precision == CASCADE_FP64 ? 64 : 128; }

// N extent of one tensor-core tile.  BF16: up to 256 (one accumulator per
// tile, two tiles in flight = 512 TMEM columns).  FP32: up to 128, because
// that path keeps the two small correction products in a second accumulator.
int block_n(int m, int precision) {
  const int cap = precision == CASCADE_FP32 ? 128 : 256;
  if (m <= cap) return m;
  for (int bn : {256, 128, 64, 32})
    if (bn <= cap && m % bn == 0) return bn;
  return 0;
}

size_t plane_elem_bytes(int precision) {
  switch (precision) {
    case CASCADE_FP64: return 8;
    case CASCADE_FP32: return 4;
    default: return 2;
  }
}

size_t state_bytes_per_row(const Plan& p) {
  const size_t e = plane_elem_bytes(p.d.precision);
  return (size_t)p.d.m * e * (p.d.precision == CASCADE_FP64 ? 1 : 2);
}

// ----------------------------------------------------------------- tensor maps
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encoder() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(ptr);
  });
  return fn;
}

bool encode_tmap_2d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t inner,
                    uint64_t outer, uint32_t box_inner, uint32_t box_outer, std::string* err,
                    int swizzle_bytes) {
  EncodeTiledFn enc = get_encoder();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const CUtensorMapDataType dt =
      elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {inner * (uint64_t)elem_bytes};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[128];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled returned %d", (int)r);
    *err = buf;
    return false;
  }
  return true;
}

bool encode_tmap_3d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t inner,
                    uint64_t S, uint64_t groups, uint32_t box_inner, uint32_t box_groups,
                    std::string* err, int swizzle_bytes) {
  EncodeTiledFn enc = get_encoder();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const CUtensorMapDataType dt =
      elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[3] = {inner, S, groups};
  cuuint64_t strides[2] = {inner * (uint64_t)elem_bytes, S * inner * (uint64_t)elem_bytes};
  cuuint32_t box[3] = {box_inner, 1, box_groups};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[128];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled (3-D) returned %d", (int)r);
    *err = buf;
    return false;
  }
  return true;
}

// Row-major [rows, cols] viewed as (32 entries, rows, cols / 32 column blocks):
// one box (32, box_rows, box_blocks) lands in shared memory as box_blocks
// consecutive [box_rows][32] tiles, the layout of box_blocks 2-D boxes.
bool encode_tmap_colblocks(CUtensorMap* map, const void* base, int elem_bytes, uint64_t cols,
                           uint64_t rows, uint32_t box_rows, uint32_t box_blocks,
                           std::string* err, int swizzle_bytes) {
  EncodeTiledFn enc = get_encoder();
  if (!enc) {
    *err = "cuTensorMapEncodeTiled unavailable";
    return false;
  }
  const CUtensorMapDataType dt =
      elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[3] = {32, rows, (cols + 31) / 32};
  cuuint64_t strides[2] = {cols * (uint64_t)elem_bytes, 32 * (uint64_t)elem_bytes};
  cuuint32_t box[3] = {32, box_rows, box_blocks};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    char buf[128];
    snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled (column blocks) returned %d", (int)r);
    *err = buf;
    return false;
  }
  return true;
}

}  // namespace cascade

using namespace cascade;

struct cascade_plan_s : public Plan {};

namespace {

cascade_status_t fail(Plan* p, cascade_status_t st, const std::string& msg) {
  if (p) p->last_error = msg;
  set_global_error(msg);
  return st;
}

cascade_status_t cuda_fail(Plan* p, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(p, e == cudaErrorMemoryAllocation ? CASCADE_ERR_OOM : CASCADE_ERR_CUDA, msg);
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return cuda_fail(p, _e, where); \
  } while (0)

template <typename T>
cudaError_t dalloc(T** ptr, size_t count) {
  *ptr = nullptr;
  if (count == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(ptr), count * sizeof(T));
}

void dfree(void* ptr) {
  if (ptr) cudaFree(ptr);
}

bool saves_states(const Plan& p) {
  return (p.d.flags & CASCADE_FLAG_SAVE_STATES) != 0 && !(p.d.flags & CASCADE_FLAG_RECOMPUTE);
}
bool recomputes(const Plan& p) { return (p.d.flags & CASCADE_FLAG_RECOMPUTE) != 0; }
bool scans(const Plan& p) { return (p.d.flags & CASCADE_FLAG_SCAN) != 0; }
bool zoh(const Plan& p) { return (p.d.flags & CASCADE_FLAG_ZOH) != 0; }
// The forward leaves what the backward needs (every stage output, or checkpoints).
bool keeps_states(const Plan& p) { return saves_states(p) || recomputes(p); }

// Workspace state buffer that holds v^(j) (j = 1..maxN+1, v^(j) = output of
// stage j-1) when the forward has finished.  Two buffers alternate; with
// CASCADE_FLAG_SAVE_STATES buffer j-1 keeps v^(j); with CASCADE_FLAG_RECOMPUTE
// the checkpoints v^(1), v^(1+c), v^(1+2c), ... (c = ck_seg) go to buffers
// 2, 3, ... and the other stage outputs alternate between buffers 0 and 1.
// A sequence's rows are written only by stages k <= N_i, so its final states
// v^(N_i+1) stay in fwd_buf(N_i+1).
int fwd_buf(const Plan& p, int j) {
  if (saves_states(p)) return j - 1;
  if (recomputes(p) && j <= p.maxN && (j - 1) % p.ck_seg == 0) return 2 + (j - 1) / p.ck_seg;
  return j & 1;
}

int ceil_log2(int64_t L) {
  int k = 0;
  while ((int64_t(1) << k) < L) ++k;
  return k;
}

// Stages with shift 2^k >= L do nothing; a sequence of length L runs k = 0..min(N, ceil(log2 L)-1).
// Largest p for which stage 1 forms v^(1) on chip: its row warps and epilogue
// form p-term dot products per element, which stays cheaper than the round
// trip of v^(1) through memory for p = 1 only (measured: p = 4 was slower).
constexpr int FUSE_FIRST_PMAX = 1;

int effective_N(int N, int64_t L) {
  if (L <= 1) return 0;
  return std::min(N, ceil_log2(L) - 1);
}

void free_batch(Plan* p) {
  for (Tile* t : p->d_tiles) dfree(t);
  p->d_tiles.clear();
  p->h_tiles.clear();
  p->n_tiles.clear();
  dfree(p->d_seqs);
  p->d_seqs = nullptr;
  dfree(p->d_out_tiles);
  p->d_out_tiles = nullptr;
  p->out_segs.clear();
  dfree(p->d_stage0_tiles);
  p->d_stage0_tiles = nullptr;
  dfree(p->d_all_tiles);
  p->d_all_tiles = nullptr;
  p->n_all_tiles = 0;
  dfree(p->d_chunk_data);
  p->d_chunk_data = nullptr;
  p->chunk_lists.clear();
  p->max_chunks = 0;
  p->chunks_all = 0;
  dfree(p->d_red_scratch);
  p->d_red_scratch = nullptr;
  p->red_scratch_bytes = 0;
  for (Tile* t : p->d_adj_tiles) dfree(t);
  p->d_adj_tiles.clear();
  p->n_adj_tiles.clear();
  p->saved_ws = nullptr;
  p->n_out_tiles = p->n_stage0_tiles = 0;
  dfree(p->d_fwin);
  p->d_fwin = nullptr;
  p->n_fwin = 0;
  p->fused_J = 0;
  for (Plan::ScanLevel& lv : p->scan) dfree(lv.d_tiles);
  p->scan.clear();
  dfree(p->d_scan_rows);
  dfree(p->d_scan_rows_sys);
  p->d_scan_rows = nullptr;
  p->d_scan_rows_sys = nullptr;
  p->n_scan_rows = 0;
  p->scan_rows_cap = 0;
  dfree(p->d_top_seqs);
  p->d_top_seqs = nullptr;
  p->n_top_seqs = 0;
  p->scan_top_k0 = -1;
  p->scan_top_K = 0;
  p->scan_top_pos = 0;
  p->matvecs = 0;
  p->have_batch = false;
  if (p->graph) {
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
}

void free_system(Plan* p) {
  void* ptrs[] = {p->P64, p->Phi, p->Plo, p->Bbar64, p->ABbar64, p->C64, p->D64, p->Bbar32,
                  p->ABbar32, p->C32, p->D32, p->A64, p->B64, p->delta64, p->scale64,
                  p->PThi, p->PTlo, p->PT64, p->Minv64, p->P32, p->Minv32};
  for (void* q : ptrs) dfree(q);
  dfree(p->pc_hi);
  dfree(p->pc_lo);
  p->pc_hi = p->pc_lo = nullptr;
  dfree(p->zoh_f_adj);
  p->zoh_f_adj = nullptr;
  p->P64 = nullptr;
  p->Phi = p->Plo = nullptr;
  p->Bbar64 = p->ABbar64 = p->C64 = p->D64 = nullptr;
  p->Bbar32 = p->ABbar32 = p->C32 = p->D32 = nullptr;
  p->A64 = p->B64 = p->delta64 = p->scale64 = nullptr;
  p->PThi = p->PTlo = nullptr;
  p->PT64 = p->Minv64 = nullptr;
  p->P32 = p->Minv32 = nullptr;
}

// Whether every one of the plan's nsys matrices X[s] (sys_stride apart) is
// lower-triangular (exact zeros above the diagonal).  Synchronises st; false on
// any CUDA error (the dense paths then run).
void check_lower(Plan* p, const double* X, int64_t sys_stride, bool* lower, cudaStream_t st) {
  *lower = false;
  if (p->d.flags & CASCADE_FLAG_DENSE_SETUP) return;
  int32_t* flag = nullptr;
  int32_t h = 1;
  cudaError_t e = cudaMalloc(&flag, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = launch_upper_nonzero(X, sys_stride, p->d.nsys, p->d.m, flag, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (flag) cudaFree(flag);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  *lower = (h == 0);
}

// Squaring chain, accuracy rule, Abar*Bbar, operand planes; P64[:,0] and
// Bbar64, C64, D64 are set.  Synchronises st.
cascade_status_t finish_system(Plan* p, cudaStream_t st) {
  const int m = p->d.m, pp = p->d.p, q = p->d.q, ns = p->d.nsys;
  const int64_t mm = (int64_t)m * m;
  const int64_t sys_stride = (int64_t)p->kmax1 * mm;
  // Lower-triangular Abar (the HiPPO-LegS systems): its powers are lower-triangular
  // too, and the squaring skips the zero triangle (same results bit for bit)
  bool lower = false;
  check_lower(p, p->P64, sys_stride, &lower, st);
  p->lower_powers = lower;
  // P_{k+1} = P_k P_k  (end of §2), batched over systems
  for (int k = 0; k + 1 < p->kmax1; ++k) {
    if (lower)
      CK(launch_dgemm_lower(p->P64 + k * mm, p->P64 + k * mm, p->P64 + (k + 1) * mm, m,
                            sys_stride, sys_stride, sys_stride, ns, st),
         "squaring chain");
    else
      CK(launch_dgemm(p->P64 + k * mm, p->P64 + k * mm, p->P64 + (k + 1) * mm, m, m, m, m, m, m,
                      sys_stride, sys_stride, sys_stride, ns, 1.0, 0.0, false, false, st),
         "squaring chain");
  }
  // Abar Bbar for the first stage fused with the input projection
  CK(launch_dgemm(p->P64, p->Bbar64, p->ABbar64, m, pp, m, m, pp, pp, sys_stride, (int64_t)m * pp,
                  (int64_t)m * pp, ns, 1.0, 0.0, false, false, st),
     "Abar*Bbar");
  // Accuracy rule
  const int Nmax = std::max(0, ceil_log2(p->d.max_len) - 1);
  p->N_sys.assign(ns, 0);
  if (p->d.N >= 0) {
    for (int s = 0; s < ns; ++s) p->N_sys[s] = std::min(p->d.N, Nmax);
  } else {
    double* d_norms = nullptr;
    CK(dalloc(&d_norms, (size_t)ns * p->kmax1), "norm buffer");
    cudaError_t e = launch_frob_norms(p->P64, ns * p->kmax1, mm, d_norms, st);
    std::vector<double> h((size_t)ns * p->kmax1);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h.data(), d_norms, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(d_norms);
    if (e != cudaSuccess) return cuda_fail(p, e, "norms");
    for (int s = 0; s < ns; ++s) {
      int N = Nmax;
      for (int n = 0; n <= Nmax; ++n) {
        if ((int64_t(1) << (n + 1)) >= (int64_t)p->d.max_len) { N = n; break; }
        if (p->d.eps > 0 && h[(size_t)s * p->kmax1 + n + 1] <= p->d.eps) { N = n; break; }
      }
      p->N_sys[s] = N;
    }
  }
  if (p->PT64)
    CK(launch_transpose(p->P64, p->PT64, m, mm, ns * p->kmax1, st), "transposed powers");
  // Operand formats
  if (p->d.precision != CASCADE_FP64) {
    CK(launch_split_planes(p->P64, p->Phi, p->Plo, (int64_t)ns * sys_stride, p->d.precision, st),
       "operand planes");
    if (p->PThi)
      CK(launch_split_planes(p->PT64, p->PThi, p->PTlo, (int64_t)ns * sys_stride, p->d.precision,
                             st),
         "transposed operand planes");
    if (p->P32) CK(launch_to_f32(p->P64, p->P32, (int64_t)ns * sys_stride, st), "FP32 powers");
    if (p->Minv32 && p->Minv64)
      CK(launch_to_f32(p->Minv64, p->Minv32, (int64_t)ns * mm, st), "FP32 M^-1");
    CK(launch_to_f32(p->Bbar64, p->Bbar32, (int64_t)ns * m * pp, st), "Bbar f32");
    CK(launch_to_f32(p->ABbar64, p->ABbar32, (int64_t)ns * m * pp, st), "ABbar f32");
    CK(launch_to_f32(p->C64, p->C32, (int64_t)ns * q * m, st), "C f32");
    CK(launch_to_f32(p->D64, p->D32, (int64_t)ns * q * pp, st), "D f32");
    if (p->pc_hi) CK(launch_proj_coef(*p, st), "projection operand planes");
  }
  CK(cudaStreamSynchronize(st), "set_system sync");
  p->have_system = true;
  if (p->have_batch) {   // the batch schedule depends on N: rebuild it
    std::vector<int64_t> offs = p->offsets;
    std::vector<int32_t> sys = p->sys_of_seq;
    free_batch(p);
    cascade_status_t r = cascade_set_batch(static_cast<cascade_plan_t>(p), offs.data(),
                                           (int32_t)(offs.size() - 1), sys.data());
    if (r != CASCADE_OK) return r;
  }
  return CASCADE_OK;
}

cascade_status_t alloc_system(Plan* p) {
  const int m = p->d.m, pp = p->d.p, q = p->d.q, ns = p->d.nsys;
  const size_t mm = (size_t)m * m;
  if (p->P64) return CASCADE_OK;
  CK(dalloc(&p->P64, (size_t)ns * p->kmax1 * mm), "alloc powers");
  CK(dalloc(&p->Bbar64, (size_t)ns * m * pp), "alloc Bbar");
  CK(dalloc(&p->ABbar64, (size_t)ns * m * pp), "alloc ABbar");
  CK(dalloc(&p->C64, (size_t)ns * q * m), "alloc C");
  CK(dalloc(&p->D64, (size_t)ns * q * pp), "alloc D");
  if (keeps_states(*p)) {   // the adjoint stages use the transposed powers
    CK(dalloc(&p->PT64, (size_t)ns * p->kmax1 * mm), "alloc transposed powers");
    if (p->d.precision != CASCADE_FP64) {
      CK(dalloc(&p->P32, (size_t)ns * p->kmax1 * mm), "alloc FP32 powers");
      CK(dalloc(&p->Minv32, (size_t)ns * mm), "alloc FP32 M^-1");
      const size_t e = plane_elem_bytes(p->d.precision);
      uint8_t* hi = nullptr;
      uint8_t* lo = nullptr;
      CK(dalloc(&hi, (size_t)ns * p->kmax1 * mm * e), "alloc transposed planes");
      CK(dalloc(&lo, (size_t)ns * p->kmax1 * mm * e), "alloc transposed planes");
      p->PThi = hi;
      p->PTlo = lo;
    }
  }
  if (p->d.precision != CASCADE_FP64) {
    const size_t e = plane_elem_bytes(p->d.precision);
    uint8_t* hi = nullptr;
    uint8_t* lo = nullptr;
    CK(dalloc(&hi, (size_t)ns * p->kmax1 * mm * e), "alloc planes");
    CK(dalloc(&lo, (size_t)ns * p->kmax1 * mm * e), "alloc planes");
    p->Phi = hi;
    p->Plo = lo;
    CK(dalloc(&p->Bbar32, (size_t)ns * m * pp), "alloc Bbar32");
    CK(dalloc(&p->ABbar32, (size_t)ns * m * pp), "alloc ABbar32");
    CK(dalloc(&p->C32, (size_t)ns * q * m), "alloc C32");
    CK(dalloc(&p->D32, (size_t)ns * q * pp), "alloc D32");
    if (proj_tc_supported(*p)) {
      const size_t n = proj_coef_elems(*p, p->pc_off);
      uint8_t* ch = nullptr;
      uint8_t* cl = nullptr;
      CK(dalloc(&ch, n * 2), "alloc projection planes");
      CK(dalloc(&cl, n * 2), "alloc projection planes");
      p->pc_hi = ch;
      p->pc_lo = cl;
    }
  }
  return CASCADE_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Workspace layout.  State buffers j = 0..nV-1 (each one FP64 plane or a
// (hi, lo) plane pair over all rows); with CASCADE_FLAG_SAVE_STATES buffer j
// keeps v^(j+1) of every stage, otherwise two buffers alternate.  Backward
// adds two adjoint buffers, the split-K partials, dP_k, and small FP64 scratch.
struct Layout {
  size_t plane = 0, buf_stride = 0, lo_off = 0;
  int nV = 2;
  size_t off_W = 0, off_part = 0, off_dP = 0, off_R = 0, off_T = 0, off_Z = 0, total = 0;
  // tensor-core projections: (hi, lo) BF16 planes of u [rows, p] and G [rows, q]
  size_t off_U = 0, u_plane = 0, off_G = 0, g_plane = 0;
};

Layout layout(const Plan& p) {
  Layout L;
  const int nplanes = p.d.precision == CASCADE_FP64 ? 1 : 2;
  const int64_t rows = scans(p) ? p.scan_rows_cap : p.rows;
  L.plane = align256((size_t)rows * p.d.m * plane_elem_bytes(p.d.precision));
  L.buf_stride = nplanes * L.plane;
  L.lo_off = nplanes == 2 ? L.plane : 0;
  const bool save = keeps_states(p);
  if (saves_states(p)) L.nV = std::max(p.maxN + 1, 1);
  else if (recomputes(p)) L.nV = 2 + p.n_ck + std::max(0, p.ck_seg - 3);   // + segment buffers
  else if (scans(p)) L.nV = 1;                                               // in place
  else L.nV = 2;
  size_t off = (size_t)L.nV * L.buf_stride;
  if (save) {
    const size_t m = p.d.m, pp = p.d.p, q = p.d.q, ns = p.d.nsys;
    const size_t acc = p.d.precision == CASCADE_FP64 ? 8 : 4;
    // partials: m x m per chunk of a stage list, q m, q p or 2 m p per chunk of
    // the list of all tiles
    const size_t elems0 = std::max(q * m, std::max(q * pp, 2 * m * pp));
    L.off_W = off;
    off += 2 * L.buf_stride;
    L.off_part = off;
    off += align256(std::max((size_t)std::max(p.max_chunks, 1) * m * m,
                             (size_t)std::max(p.chunks_all, 1) * elems0) *
                    acc);
    L.off_dP = off;
    off += align256(ns * p.kmax1 * m * m * 8);
    L.off_R = off;                                  // R1, R2, dBbar, dB: [nsys, m, p] each
    off += align256(4 * ns * m * pp * 8);
    L.off_T = off;                                  // T, dA: [nsys, m, m] each
    off += align256(2 * ns * m * m * 8);
    if (zoh(p) && p.continuous) {
      // adjoint of the zero-order hold: dAbar, dBbar in FP64, Z^T, the 2n x 2n
      // block matrices, the exponential's scratch, the G norms and a flag word
      const size_t n = m + pp, n2 = 2 * n;
      L.off_Z = off;
      off += align256(8 * (ns * m * m + ns * m * pp + ns * n * n + ns * n2 * n2 +
                           expm_scratch_doubles((int)n2, (int)ns) + ns) + 8);
    }
  }
  // (hi, lo) BF16 planes of u and G for the tensor-core projections and, in the
  // backward, the tensor-core time reductions (rows of pad8(p) and pad8(q) entries)
  const bool ptc = proj_tc_supported(p), thin = save && ptc && thin_tc_supported(p);
  if (ptc || thin) {
    L.u_plane = align256((size_t)p.rows * pad8(p.d.p) * 2);
    L.off_U = off;
    off += 2 * L.u_plane;
  }
  if (save && (ptc || thin)) {
    L.g_plane = align256((size_t)p.rows * pad8(p.d.q) * 2);
    L.off_G = off;
    off += 2 * L.g_plane;
  }
  L.total = off + 256;
  return L;
}

size_t forward_workspace(const Plan& p, int64_t) { return layout(p).total; }

cudaError_t ensure_events(Plan* p, int pairs) {
  while ((int)p->ev.size() < 2 * pairs) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    p->ev.push_back(e);
  }
  return cudaSuccess;
}

// The host side of cascade_forward_host when its copies overlap the projections:
// u comes from h_u chunk by chunk on the copy stream cs (in), y goes to h_y chunk
// by chunk (out), chunks as Plan::io_in / io_out.
struct HostIO {
  const void* h_u;
  void* h_y;
  size_t u_row_bytes, y_row_bytes;
  cudaStream_t cs;
  const cudaEvent_t* ev;   // io_in.size() + io_out.size() + 1 events
  bool in, out;
};

cascade_status_t run_forward(Plan* p, const void* u, void* y, void* ws, cudaStream_t st,
                             const HostIO* io = nullptr) {
  const Layout L = layout(*p);
  const Bufs V{static_cast<uint8_t*>(ws), L.buf_stride, L.lo_off};
  const bool save = keeps_states(*p);
  const bool timing = p->timing;
  // tensor-core projections read u as (hi, lo) BF16 planes
  const bool ptc = proj_tc_supported(*p);
  const Bufs U{static_cast<uint8_t*>(ws) + L.off_U, 0, L.u_plane};
  // (the copies overlap the tensor-core first-stage and output projections, when
  // those run as their own launches over every row)
  const bool io_in = io && io->in && ptc && !scans(*p) && p->fused_J == 0 && !p->fuse_first &&
                     !p->io_in.empty();
  const bool io_out = io && io->out && ptc && !scans(*p) && !p->io_out.empty();
  if (ptc && !io_in)
    CK(launch_split_rows(static_cast<const float*>(u), p->rows, p->d.p, p->d.p, U.hi(0), U.lo(0),
                         st),
       "input planes");
  if (timing) {
    CK(ensure_events(p, std::max(std::max(p->maxN, 1), (int)p->scan.size() + 1)), "timing events");
    p->ev_k.clear();
    p->n_ev = 0;
  }
  if (scans(*p)) {
    // work-efficient schedule, in place on buffer 0: the first up-sweep level
    // with the input projection, the other levels on the tensor cores, then
    // y = C x + D u for every row
    if (ptc)
      CK(launch_proj_tc_stage0(*p, U, V, p->scan_rows_cap, 0, true, st), "first level");
    else
      CK(launch_proj_stage0(*p, static_cast<const float*>(u), V, 0,
                            p->scan_even_on_chip ? 2 : 1, st),
         "first level");
    for (size_t li = 0; li <= p->scan.size(); ++li) {
      if ((int)li == p->scan_top_pos && p->scan_top_k0 >= 0 && p->n_top_seqs > 0) {
        // levels k >= k0, up and down, one block per sequence
        if (timing) CK(cudaEventRecord(p->ev[2 * p->n_ev], st), "event");
        CK(launch_scan_top(*p, V.hi(0), V.lo(0), (uint64_t)p->scan_rows_cap,
                           static_cast<const float*>(u), static_cast<float*>(y), st),
           "scan top levels");
        if (timing) {
          CK(cudaEventRecord(p->ev[2 * p->n_ev + 1], st), "event");
          p->ev_k.push_back(300 + p->scan_top_k0);
          p->n_ev++;
        }
      }
      if (li == p->scan.size()) break;
      const Plan::ScanLevel& lv = p->scan[li];
      if (timing && lv.n > 0) CK(cudaEventRecord(p->ev[2 * p->n_ev], st), "event");
      CK(launch_stage_tc_strided(*p, lv.k, 2 << lv.k, lv.d_tiles, lv.n,
                                 (uint64_t)p->scan_rows_cap, V.hi(0), V.lo(0),
                                 static_cast<const float*>(u), static_cast<float*>(y), st,
                                 p->scan_even_on_chip && lv.down && lv.k == 0,
                                 lv.down ? 100 + lv.k : lv.k),
         "scan level");
      if (timing && lv.n > 0) {
        CK(cudaEventRecord(p->ev[2 * p->n_ev + 1], st), "event");
        p->ev_k.push_back(lv.down ? 100 + lv.k : lv.k);
        p->n_ev++;
      }
    }
    if (p->fuse_output)
      CK(launch_proj_rows_output(*p, p->d_scan_rows, p->n_scan_rows, p->d_scan_rows_sys,
                                 static_cast<const float*>(u), static_cast<float*>(y), V, 0, st),
         "output projection (rows 2^t - 1)");
    else if (ptc)
      CK(launch_proj_tc_output(*p, U, static_cast<float*>(y), V, p->scan_rows_cap, st),
         "output projection");
    else
      CK(launch_proj_output(*p, static_cast<const float*>(u), static_cast<float*>(y), V, st),
         "output projection");
    return CASCADE_OK;
  }
  // buffer holding v^(k) read by stage k, and the one stage k writes
  auto in_buf = [&](int k) { return fwd_buf(*p, k); };
  auto out_buf = [&](int k) { return fwd_buf(*p, k + 1); };
  // stage 0 fused with v^(0) = Bbar u (formed inside stage 1 with fuse_first,
  // here only for the sequences without a stage 1)
  if (p->fused_J > 0) {
    // stages 1 .. fused_J in one pass from u (no first-stage launch: every
    // sequence runs past those stages); timed as stage 1
    const int J = p->fused_J;
    if (timing) CK(cudaEventRecord(p->ev[2 * p->n_ev], st), "event");
    CK(launch_fused_stages(*p, static_cast<const float*>(u), V.hi(in_buf(J + 1)),
                           V.lo(in_buf(J + 1)), st),
       "fused first stages");
    if (timing) {
      CK(cudaEventRecord(p->ev[2 * p->n_ev + 1], st), "event");
      p->ev_k.push_back(1);
      p->n_ev++;
    }
  } else if (p->fuse_first)
    CK(launch_proj_stage0(*p, static_cast<const float*>(u), V, out_buf(0), 0, st),
       "first stage");
  else if (ptc && io_in) {
    // each chunk of u is split and projected once its copy has landed, while the
    // next chunk is still on its way
    const size_t n = p->io_in.size();
    for (size_t c = 0; c < n; ++c) {
      const auto& ch = p->io_in[c];
      CK(cudaMemcpyAsync(static_cast<uint8_t*>(const_cast<void*>(u)) + ch[2] * io->u_row_bytes,
                         static_cast<const uint8_t*>(io->h_u) + ch[2] * io->u_row_bytes,
                         ch[3] * io->u_row_bytes, cudaMemcpyHostToDevice, io->cs),
         "copy u to the device");
      CK(cudaEventRecord(io->ev[c], io->cs), "event");
    }
    for (size_t c = 0; c < n; ++c) {
      const auto& ch = p->io_in[c];
      CK(cudaStreamWaitEvent(st, io->ev[c], 0), "wait for u");
      const size_t e0 = (size_t)ch[2] * p->d.p;   // first element of the chunk
      CK(launch_split_rows(static_cast<const float*>(u) + e0, ch[3], p->d.p, p->d.p,
                           static_cast<__nv_bfloat16*>(U.hi(0)) + e0,
                           static_cast<__nv_bfloat16*>(U.lo(0)) + e0, st),
         "input planes");
      CK(launch_proj_tc_stage0(*p, U, V, p->rows, out_buf(0), false, st, (int)ch[0], (int)ch[1]),
         "first stage");
    }
  } else if (ptc)
    CK(launch_proj_tc_stage0(*p, U, V, p->rows, out_buf(0), false, st), "first stage");
  else if (proj_supported(*p))
    CK(launch_proj_stage0(*p, static_cast<const float*>(u), V, out_buf(0), 0, st), "first stage");
  else
    CK(launch_stage0(*p, u, V.hi(out_buf(0)), V.lo(out_buf(0)), st), "first stage");
  for (int k = p->fused_J + 1; k <= p->maxN; ++k) {
    const int in = in_buf(k), out = out_buf(k);
    if (timing && p->n_tiles[k] > 0) CK(cudaEventRecord(p->ev[2 * p->n_ev], st), "event");
    if (p->d.precision == CASCADE_FP64) {
      CK(launch_stage_f64(*p, k, static_cast<const double*>(V.hi(in)),
                          static_cast<double*>(V.hi(out)), st),
         "stage (fp64)");
    } else {
      CK(launch_stage_tc(*p, k, V.hi(in), V.lo(in), V.hi(out), V.lo(out),
                         static_cast<const float*>(u), static_cast<float*>(y), st, false,
                         ptc ? U.hi(0) : nullptr, ptc ? U.lo(0) : nullptr),
         "stage (tensor core)");
    }
    if (timing && p->n_tiles[k] > 0) {
      CK(cudaEventRecord(p->ev[2 * p->n_ev + 1], st), "event");
      p->ev_k.push_back(k);
      p->n_ev++;
    }
  }
  if (ptc && io_out) {
    // y chunk by chunk: each chunk's copy to the host overlaps the next chunk's
    // projection; the stream then waits for the last copy
    const size_t n0 = p->io_in.size(), n = p->io_out.size();
    for (size_t c = 0; c < n; ++c) {
      const auto& ch = p->io_out[c];
      CK(launch_proj_tc_output(*p, U, static_cast<float*>(y), V, p->rows, st, (int)ch[0],
                               (int)ch[1]),
         "output projection");
      CK(cudaEventRecord(io->ev[n0 + c], st), "event");
      CK(cudaStreamWaitEvent(io->cs, io->ev[n0 + c], 0), "wait for y");
      CK(cudaMemcpyAsync(static_cast<uint8_t*>(io->h_y) + ch[2] * io->y_row_bytes,
                         static_cast<const uint8_t*>(y) + ch[2] * io->y_row_bytes,
                         ch[3] * io->y_row_bytes, cudaMemcpyDeviceToHost, io->cs),
         "copy y to the host");
    }
    CK(cudaEventRecord(io->ev[n0 + n], io->cs), "event");
    CK(cudaStreamWaitEvent(st, io->ev[n0 + n], 0), "wait for the copies");
  } else if (ptc)
    CK(launch_proj_tc_output(*p, U, static_cast<float*>(y), V, p->rows, st), "output projection");
  else if (proj_supported(*p))
    CK(launch_proj_output(*p, static_cast<const float*>(u), static_cast<float*>(y), V, st),
       "output projection");
  else
    CK(launch_output(*p, u, y, V, st), "output projection");
  if (save) {
    p->saved_ws = ws;
    p->saved_batch = p->batch_id;
  }
  return CASCADE_OK;
}

// GEMM in the backward's arithmetic type (FP32 for the tensor-core plans,
// FP64 for the FP64 plan).
cudaError_t gemm_t(const double* A, const double* B, double* C, int M, int N, int K, int lda,
                   int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC, int batch, double alpha,
                   double beta, bool tA, bool tB, cudaStream_t st, void* = nullptr, size_t = 0) {
  return launch_dgemm(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, alpha, beta, tA, tB, st);
}
// scratch (optional): room for a split-K of the long, narrow products
cudaError_t gemm_t(const float* A, const float* B, float* C, int M, int N, int K, int lda,
                   int ldb, int ldc, int64_t sA, int64_t sB, int64_t sC, int batch, double alpha,
                   double beta, bool tA, bool tB, cudaStream_t st, void* scratch = nullptr,
                   size_t scratch_bytes = 0) {
  // square-ish products, or any product with scratch for a split K: the
  // register-tiled kernel (128 x 128 tiles, or 64 x 64 with K slices)
  if ((M >= 128 && N >= 128) || scratch)
    return launch_sgemm2(A, B, tA, tB, nullptr, nullptr, false, false, C, M, N, K, lda, ldb, ldc,
                         sA, sB, sC, batch, (float)alpha, (float)beta, st,
                         static_cast<float*>(scratch), scratch_bytes / sizeof(float));
  return launch_sgemm(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, (float)alpha,
                      (float)beta, tA, tB, st);
}
// One level of the squaring-chain adjoint: dP_k += dP_(k+1) P_k^T + P_k^T dP_(k+1).
cudaError_t chain_step(const double* dPn, const double* P, double* dP, int m, int64_t stride,
                       int batch, cudaStream_t st, void*, size_t) {
  cudaError_t e = launch_dgemm(dPn, P, dP, m, m, m, m, m, m, stride, stride, stride, batch, 1.0,
                               1.0, false, true, st);
  if (e != cudaSuccess) return e;
  return launch_dgemm(P, dPn, dP, m, m, m, m, m, m, stride, stride, stride, batch, 1.0, 1.0, true,
                      false, st);
}
cudaError_t chain_step(const float* dPn, const float* P, float* dP, int m, int64_t stride,
                       int batch, cudaStream_t st, void* scratch, size_t scratch_bytes) {
  return launch_sgemm2(dPn, P, false, true, P, dPn, true, false, dP, m, m, m, m, m, m, stride,
                       stride, stride, batch, 1.0f, 1.0f, st, static_cast<float*>(scratch),
                       scratch_bytes / sizeof(float));
}
template <typename T>
cudaError_t to_f64(const T* src, int64_t src_stride, double* dst, int64_t dst_stride, int64_t n,
                   int nsys, cudaStream_t st);
template <>
cudaError_t to_f64<double>(const double* src, int64_t src_stride, double* dst, int64_t dst_stride,
                           int64_t n, int nsys, cudaStream_t st) {
  return cudaMemcpy2DAsync(dst, sizeof(double) * dst_stride, src, sizeof(double) * src_stride,
                           sizeof(double) * n, nsys, cudaMemcpyDeviceToDevice, st);
}
template <>
cudaError_t to_f64<float>(const float* src, int64_t src_stride, double* dst, int64_t dst_stride,
                          int64_t n, int nsys, cudaStream_t st) {
  return launch_convert_sys<float, double>(src, src_stride, dst, dst_stride, n, nsys, st);
}

// Reverse-mode derivative of sum(dy * y) after a forward that kept its stage
// outputs (see backward.cu for the equations).  T: arithmetic of the small
// m x m / m x p algebra at the end (squaring-chain and discretisation adjoints).
template <typename T>
cascade_status_t run_backward_t(Plan* p, const T* P, const T* Bbar, const T* Minv, const void* u,
                                const void* dy, void* du, double* dAbar, double* dBbar,
                                double* dC, double* dD, double* dA, double* dB, void* ws,
                                cudaStream_t st) {
  const Layout L = layout(*p);
  uint8_t* base = static_cast<uint8_t*>(ws);
  const Bufs V{base, L.buf_stride, L.lo_off};
  const Bufs W{base + L.off_W, L.buf_stride, L.lo_off};
  void* part = base + L.off_part;
  T* dP = reinterpret_cast<T*>(base + L.off_dP);
  const int m = p->d.m, pp = p->d.p, q = p->d.q, ns = p->d.nsys;
  const int64_t mm = (int64_t)m * m, mp = (int64_t)m * pp;
  const int64_t kst = (int64_t)p->kmax1 * mm;
  T* R1 = reinterpret_cast<T*>(base + L.off_R);
  T* R2 = R1 + ns * mp;
  T* dBb = R2 + ns * mp;
  T* dBt = dBb + ns * mp;
  T* Tm = reinterpret_cast<T*>(base + L.off_T);
  T* dAt = Tm + ns * mm;
  const bool f64 = p->d.precision == CASCADE_FP64;
  const bool tf64 = sizeof(T) == 8;
  const TSrc G{f64 ? 2 : 1, Bufs{}, 0, 0, dy, q};
  const TSrc U{f64 ? 2 : 1, Bufs{}, 0, 0, u, pp};
  auto chunks = [&](int li) { return p->d_chunk_data + p->chunk_lists[li].off_chunks; };
  auto sysbeg = [&](int li) { return p->d_chunk_data + p->chunk_lists[li].off_begin; };
  const int nall = p->chunk_lists[0].n;

  const bool proj = proj_supported(*p);
  // tensor-core projections read G as (hi, lo) BF16 planes
  const bool ptc = proj_tc_supported(*p);
  const Bufs Gp{base + L.off_G, 0, L.g_plane};
  const Bufs Up{base + L.off_U, 0, L.u_plane};
  // p and q multiples of 16 with m of 128: the time reductions of dC, dD, R1 and R2
  // run on the tensor cores like the power gradients.  (Narrower p and q were
  // measured on the same kernel with zero-padded planes: no faster than the
  // wide-by-thin CUDA-core kernels, whose one pass forms R1 and R2 together.)
  const bool thin_tc = ptc && thin_tc_supported(*p);
  const int ppad = pad8(pp), qpad = pad8(q);
  if (ptc || thin_tc)
    CK(launch_split_rows(static_cast<const float*>(dy), p->rows, q, qpad, Gp.hi(0), Gp.lo(0), st),
       "adjoint planes");
  if (thin_tc)
    CK(launch_split_rows(static_cast<const float*>(u), p->rows, pp, ppad, Up.hi(0), Up.lo(0), st),
       "input planes");

  // dC = sum G v^(N+1)^T: v^(N_i+1) sits in state buffer tile.fbuf.  This runs
  // first: with checkpoints, the recomputation below reuses those buffers.
  if (dC) {
    const TSrc VF{0, V, 1, 0, nullptr, 0};
    if (thin_tc && p->all_fbuf >= 0) {   // dC^T = sum v^(N+1)_l G_l^T, stored transposed
      CK(launch_grad_tc_xy(*p, p->d_all_tiles, chunks(0), nall, V.hi(p->all_fbuf),
                           V.lo(p->all_fbuf), m, m, Gp.hi(0), Gp.lo(0), q, qpad, 0, true,
                           static_cast<float*>(part), st),
         "dC (tensor core)");
      CK(launch_reduce_partials(*p, static_cast<const float*>(part), sysbeg(0), (int64_t)q * m,
                                dC, true, (int64_t)q * m, st),
         "dC reduction");
    } else if (wtreduce_supported(*p, m, q, 1))
      CK(launch_wtreduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), VF, m, dy, q, 1, 0, 0,
                         true, part, dC, true, (int64_t)q * m, 0, st),
         "dC");
    else
      CK(launch_treduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), G, q, VF, m, 0, part, dC,
                        true, (int64_t)q * m, 0, st),
         "dC");
  }
  if (dD) {   // dD = sum G u^T
    if (thin_tc) {
      CK(launch_grad_tc_xy(*p, p->d_all_tiles, chunks(0), nall, Gp.hi(0), Gp.lo(0), q, qpad,
                           Up.hi(0), Up.lo(0), pp, ppad, 0, false, static_cast<float*>(part), st),
         "dD (tensor core)");
      CK(launch_reduce_partials(*p, static_cast<const float*>(part), sysbeg(0), (int64_t)q * pp,
                                dD, true, (int64_t)q * pp, st),
         "dD reduction");
    } else if (wtreduce_supported(*p, q, pp, 1))
      CK(launch_wtreduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), G, q, u, pp, 1, 0, 0,
                         false, part, dD, true, (int64_t)q * pp, 0, st),
         "dD");
    else
      CK(launch_treduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), G, q, U, pp, 0, part, dD,
                        true, (int64_t)q * pp, 0, st),
         "dD");
  }
  // W^(N_i+1) = C^T G, in the adjoint buffer the stage N_i reads
  if (ptc)
    CK(launch_proj_tc_adj_init(*p, Gp, W, st), "adjoint init");
  else if (proj)
    CK(launch_proj_adj_init(*p, static_cast<const float*>(dy), W, st), "adjoint init");
  else
    CK(launch_adj_init(*p, dy, W, st), "adjoint init");
  CK(cudaMemsetAsync(dP, 0, sizeof(T) * ns * kst, st), "zero dP");

  // Adjoint of stage k (k >= 1) given v^(k) in state buffer vb:
  //   dP_k = sum_{l >= s} W^(k+1)_l v^(k)_(l-s)^T,  W^(k) = W^(k+1) + P_k^T shift(W^(k+1)).
  auto back_stage = [&](int k, int vb) -> cascade_status_t {
    const int win = (k + 1) & 1, wout = k & 1;
    const ChunkList& cl = p->chunk_lists[k];
    if (grad_tc_supported(*p)) {   // tensor cores, then the ordered per-system reduction
      CK(launch_grad_tc(*p, p->d_tiles[k], chunks(k), cl.n, W.hi(win), W.lo(win), V.hi(vb),
                        V.lo(vb), 1 << k, static_cast<float*>(part), st),
         "dP (tensor core)");
      CK(launch_reduce_partials(*p, static_cast<const float*>(part), sysbeg(k), mm,
                                dP + (int64_t)k * mm, tf64, kst, st),
         "dP reduction");
    } else {
      CK(launch_treduce(*p, p->d_tiles[k], chunks(k), cl.n, sysbeg(k),
                        TSrc{0, W, 0, win, nullptr, 0}, m, TSrc{0, V, 0, vb, nullptr, 0}, m,
                        1 << k, part, dP + (int64_t)k * mm, tf64, kst, 0, st),
         "dP");
    }
    if (f64) {
      CK(launch_stage_f64(*p, k, static_cast<const double*>(W.hi(win)),
                          static_cast<double*>(W.hi(wout)), st, true),
         "adjoint stage (fp64)");
    } else {
      CK(launch_stage_tc(*p, k, W.hi(win), W.lo(win), W.hi(wout), W.lo(wout), nullptr, nullptr,
                         st, true),
         "adjoint stage (tensor core)");
    }
    return CASCADE_OK;
  };
  // forward stage k from buffer a to buffer b (recomputation; no output projection)
  auto fwd_stage = [&](int k, int a, int b) -> cascade_status_t {
    if (f64)
      CK(launch_stage_f64(*p, k, static_cast<const double*>(V.hi(a)),
                          static_cast<double*>(V.hi(b)), st),
         "recomputed stage (fp64)");
    else
      CK(launch_stage_tc(*p, k, V.hi(a), V.lo(a), V.hi(b), V.lo(b), nullptr, nullptr, st),
         "recomputed stage (tensor core)");
    return CASCADE_OK;
  };
  if (!recomputes(*p)) {
    for (int k = p->maxN; k >= 1; --k) {   // v^(k) is state buffer k-1
      const cascade_status_t r = back_stage(k, k - 1);
      if (r != CASCADE_OK) return r;
    }
  } else {
    // Segments of c stages from the last checkpoint down: recompute v^(a+1) ..
    // v^(top) from the checkpoint v^(a) into buffers 0, 1, 2 + n_ck, ..., then
    // run their adjoint stages top .. a.
    const int c = p->ck_seg;
    for (int sgi = p->n_ck - 1; sgi >= 0; --sgi) {
      const int a = 1 + sgi * c;
      const int top = std::min(a + c - 1, p->maxN);
      auto buf_of = [&](int j) {
        if (j == a) return 2 + sgi;
        const int i = j - a - 1;
        return i < 2 ? i : 2 + p->n_ck + (i - 2);
      };
      for (int k = a; k < top; ++k) {
        const cascade_status_t r = fwd_stage(k, buf_of(k), buf_of(k + 1));
        if (r != CASCADE_OK) return r;
      }
      for (int k = top; k >= a; --k) {
        const cascade_status_t r = back_stage(k, buf_of(k));
        if (r != CASCADE_OK) return r;
      }
    }
  }
  // first stage (fused with Bbar u): W^(1) is adjoint buffer 1.  Narrow p and q: du,
  // R1 and R2 in one pass over W^(1)
  const bool fused_first = !f64 && !thin_tc && du && first_adj_thin_supported(*p);
  if (fused_first) {
    CK(launch_first_adj_thin(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), W, 1,
                             static_cast<const float*>(u), static_cast<const float*>(dy),
                             static_cast<float*>(du), static_cast<float*>(part), R1, tf64, mp,
                             (int64_t)ns * mp, st),
       "du, R1, R2");
  } else if (du) {
    if (ptc)
      CK(launch_proj_tc_du(*p, Gp, W, 1, static_cast<float*>(du), st), "du");
    else if (proj)
      CK(launch_proj_du(*p, static_cast<const float*>(dy), W, 1, static_cast<float*>(du), st),
         "du");
    else
      CK(launch_stage0_adj(*p, dy, W, 1, du, st), "du");
  }
  // R1 = sum W^(1)_l u_l^T,  R2 = sum W^(1)_l u_(l-1)^T
  const TSrc W1{0, W, 0, 1, nullptr, 0};
  if (fused_first) {
    // formed above
  } else if (thin_tc) {
    for (int sh = 0; sh < 2; ++sh) {
      CK(launch_grad_tc_xy(*p, p->d_all_tiles, chunks(0), nall, W.hi(1), W.lo(1), m, m, Up.hi(0),
                           Up.lo(0), pp, ppad, sh, false, static_cast<float*>(part), st),
         sh ? "R2 (tensor core)" : "R1 (tensor core)");
      CK(launch_reduce_partials(*p, static_cast<const float*>(part), sysbeg(0), mp,
                                sh ? R2 : R1, tf64, mp, st),
         "R1, R2 reduction");
    }
  } else if (wtreduce_supported(*p, m, pp, 2)) {
    CK(launch_wtreduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), W1, m, u, pp, 2, 0, 1,
                       false, part, R1, tf64, mp, (int64_t)ns * mp, st),
       "R1, R2");
  } else if (wtreduce_supported(*p, m, pp, 1)) {
    CK(launch_wtreduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), W1, m, u, pp, 1, 0, 0,
                       false, part, R1, tf64, mp, 0, st),
       "R1");
    CK(launch_wtreduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), W1, m, u, pp, 1, 1, 0,
                       false, part, R2, tf64, mp, 0, st),
       "R2");
  } else {
    CK(launch_treduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), W1, m, U, pp, 0, part, R1,
                      tf64, mp, 0, st),
       "R1");
    CK(launch_treduce(*p, p->d_all_tiles, chunks(0), nall, sysbeg(0), W1, m, U, pp, 1, part, R2,
                      tf64, mp, 0, st),
       "R2");
  }
  // dP_0 += R2 Bbar^T;  dBbar = R1 + Abar^T R2
  CK(gemm_t(R2, Bbar, dP, m, m, pp, pp, pp, m, mp, mp, kst, ns, 1.0, 1.0, false, true, st), "dP0");
  CK(cudaMemcpyAsync(dBb, R1, sizeof(T) * ns * mp, cudaMemcpyDeviceToDevice, st), "copy");
  CK(gemm_t(P, R2, dBb, m, pp, m, m, pp, pp, kst, mp, mp, ns, 1.0, 1.0, true, false, st, part,
            L.off_dP - L.off_part),
     "dBbar");
  // squaring chain P_(k+1) = P_k P_k:  dP_k += dP_(k+1) P_k^T + P_k^T dP_(k+1)
  // on the tensor cores for the BF16-split plans (the four split planes of
  // dP_(k+1) fit in the partial-sum region, free by now); FP32 / FP64 otherwise
  const bool chain_tc = sizeof(T) == 4 && chain_tc_supported(*p) &&
                        chain_tc_scratch_bytes(*p) <= L.off_dP - L.off_part;
  for (int k = p->kmax1 - 2; k >= 0; --k) {
    if (chain_tc)
      CK(launch_chain_tc(*p, k, k == p->kmax1 - 2, reinterpret_cast<float*>(dP), kst, part, st),
         "chain (tensor core)");
    else
      CK(chain_step(dP + (k + 1) * mm, P + k * mm, dP + k * mm, m, kst, ns, st, part,
                    L.off_dP - L.off_part),
         "chain");
  }
  if (dAbar) CK(to_f64<T>(dP, kst, dAbar, mm, mm, ns, st), "dAbar");
  if (dBbar) CK(to_f64<T>(dBb, mp, dBbar, mp, mp, ns, st), "dBbar");
  // trapezoidal discretisation (Eq. 4.2), Abar = c M^-1 (I + delta/2 A), Bbar = delta M^-1 B:
  // dA = delta/2 M^-T (c dAbar + dAbar Abar^T + dBbar Bbar^T),  dB = delta M^-T dBbar
  if (p->continuous && zoh(*p) && (dA || dB)) {
    // zero-order hold (§5): dZ = L(Z^T, G) is the upper right block of
    // exp([[Z^T, G/g], [0, Z^T]]) times g; dA = delta dZ[:m, :m], dB = delta dZ[:m, m:]
    const int n = m + pp;
    const int64_t nn = (int64_t)n * n;
    double* dA64 = reinterpret_cast<double*>(base + L.off_Z);
    double* dB64 = dA64 + ns * mm;
    double* ZT = dB64 + ns * mp;
    double* Wb = ZT + ns * nn;
    double* scr = Wb + 4 * ns * nn;
    double* gnorm = scr + expm_scratch_doubles(2 * n, ns);
    int32_t* sing = reinterpret_cast<int32_t*>(gnorm + ns);
    CK(to_f64<T>(dP, kst, dA64, mm, mm, ns, st), "dAbar (fp64)");
    CK(to_f64<T>(dBb, mp, dB64, mp, mp, ns, st), "dBbar (fp64)");
    CK(launch_zoh_block(p->A64, p->B64, p->delta64, ZT, m, pp, ns, true, st), "Z^T");
    CK(launch_frechet_block(ZT, dA64, dB64, p->scale64, Wb, gnorm, m, pp, ns, st), "W");
    CK(cudaMemsetAsync(sing, 0, sizeof(int32_t), st), "flag");
    CK(expm_batched(Wb, 2 * n, ns, p->zoh_sq_adj, p->zoh_f_adj, scr, sing, st), "exp(W)");
    if (dA) {
      CK(launch_block(Wb, 2 * n, 0, n, m, m, dA, mm, gnorm, 1.0, ns, st), "dA");
      CK(launch_axpy_sys<double>(dA, mm, dA, mm, mm, ns, p->delta64, 1.0, false, st), "dA");
    }
    if (dB) {
      CK(launch_block(Wb, 2 * n, 0, n + m, m, pp, dB, mp, gnorm, 1.0, ns, st), "dB");
      CK(launch_axpy_sys<double>(dB, mp, dB, mp, mp, ns, p->delta64, 1.0, false, st), "dB");
    }
  } else if (p->continuous && (dA || dB)) {
    CK(gemm_t(dP, P, Tm, m, m, m, m, m, m, kst, kst, mm, ns, 1.0, 0.0, false, true, st), "T");
    CK(gemm_t(dBb, Bbar, Tm, m, m, pp, pp, pp, m, mp, mp, mm, ns, 1.0, 1.0, false, true, st), "T");
    CK(launch_axpy_sys<T>(dP, kst, Tm, mm, mm, ns, p->scale64, 1.0, true, st), "T");
    if (dA) {
      CK(gemm_t(Minv, Tm, dAt, m, m, m, m, m, m, mm, mm, mm, ns, 1.0, 0.0, true, false, st), "dA");
      CK(launch_axpy_sys<T>(dAt, mm, dAt, mm, mm, ns, p->delta64, 0.5, false, st), "dA");
      CK(to_f64<T>(dAt, mm, dA, mm, mm, ns, st), "dA");
    }
    if (dB) {
      CK(gemm_t(Minv, dBb, dBt, m, pp, m, m, pp, pp, mm, mp, mp, ns, 1.0, 0.0, true, false, st,
                part, L.off_dP - L.off_part),
         "dB");
      CK(launch_axpy_sys<T>(dBt, mp, dBt, mp, mp, ns, p->delta64, 1.0, false, st), "dB");
      CK(to_f64<T>(dBt, mp, dB, mp, mp, ns, st), "dB");
    }
  }
  return CASCADE_OK;
}

cascade_status_t run_backward(Plan* p, const void* u, const void* dy, void* du, double* dAbar,
                              double* dBbar, double* dC, double* dD, double* dA, double* dB,
                              void* ws, cudaStream_t st) {
  if (p->d.precision == CASCADE_FP64)
    return run_backward_t<double>(p, p->P64, p->Bbar64, p->Minv64, u, dy, du, dAbar, dBbar, dC, dD,
                                  dA, dB, ws, st);
  return run_backward_t<float>(p, p->P32, p->Bbar32, p->Minv32, u, dy, du, dAbar, dBbar, dC, dD,
                               dA, dB, ws, st);
}

}  // namespace

namespace {
// Zero-order hold of every system (§5): Z = delta [[A, B], [0, 0]], E = exp(Z),
// Abar = scale * E[:m, :m] into P64[:, 0], Bbar = E[:m, m:].  Records, per
// system, the squarings of this exponential and of the adjoint's block
// exponential (whose 1-norm is at most ||Z||_inf + 1).  Synchronises st.
cascade_status_t discretise_zoh(Plan* p, cudaStream_t st) {
  const int m = p->d.m, pp = p->d.p, ns = p->d.nsys, n = m + pp;
  const size_t nn = (size_t)n * n;
  double* Z = nullptr;
  double* scratch = nullptr;
  double* nrm = nullptr;      // 1-norms, inf-norms, scale factors
  int32_t* sing = nullptr;
  cudaError_t e = dalloc(&Z, ns * nn);
  if (e == cudaSuccess) e = dalloc(&scratch, expm_scratch_doubles(n, ns));
  if (e == cudaSuccess) e = dalloc(&nrm, (size_t)3 * ns);
  if (e == cudaSuccess) e = dalloc(&sing, 1);
  if (e == cudaSuccess) e = cudaMemsetAsync(sing, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = launch_zoh_block(p->A64, p->B64, p->delta64, Z, m, pp, ns, false, st);
  if (e == cudaSuccess) e = launch_norms(Z, n, ns, nrm, nrm + ns, st);
  std::vector<double> h(2 * (size_t)ns);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), nrm, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  p->zoh_sq.assign(ns, 0);
  p->zoh_sq_adj.assign(ns, 0);
  std::vector<double> f(ns), fa(ns);
  for (int s = 0; s < ns; ++s) {
    p->zoh_sq[s] = expm_squarings(h[s]);
    p->zoh_sq_adj[s] = expm_squarings(h[ns + s] + 1.0);
    f[s] = ldexp(1.0, -p->zoh_sq[s]);
    fa[s] = ldexp(1.0, -p->zoh_sq_adj[s]);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(nrm + 2 * ns, f.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !p->zoh_f_adj) e = dalloc(&p->zoh_f_adj, (size_t)ns);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->zoh_f_adj, fa.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = expm_batched(Z, n, ns, p->zoh_sq, nrm + 2 * ns, scratch, sing, st);
  if (e == cudaSuccess)
    e = launch_block(Z, n, 0, 0, m, m, p->P64, (int64_t)p->kmax1 * m * m, p->scale64, 1.0, ns, st);
  if (e == cudaSuccess)
    e = launch_block(Z, n, 0, m, m, pp, p->Bbar64, (int64_t)m * pp, nullptr, 1.0, ns, st);
  int32_t h_sing = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_sing, sing, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // f, fa live on the host
  dfree(Z);
  dfree(scratch);
  dfree(nrm);
  dfree(sing);
  if (e != cudaSuccess) return cuda_fail(p, e, "zero-order hold");
  if (h_sing) return fail(p, CASCADE_ERR_INVALID_ARG, "singular Pade denominator in exp(delta A)");
  return CASCADE_OK;
}
}  // namespace

namespace cascade {
// Forward into a caller-chosen workspace (used by the fixed-scratch entry point).
cascade_status_t forward_with_workspace(Plan* p, const void* u, void* y, void* ws,
                                        cudaStream_t st) {
  p->last_stream = st;
  return run_forward(p, u, y, ws, st);
}
size_t forward_workspace_bytes(const Plan& p) { return forward_workspace(p, p.rows); }
}  // namespace cascade

// =================================================================== C ABI
// One forward with an event pair around every stage launch; adds each stage
// k's duration to acc[k].
static cascade_status_t timed_stages(Plan* p, const void* u, void* y, void* ws, cudaStream_t st,
                                     std::vector<float>& acc) {
  p->timing = true;
  const cascade_status_t r = run_forward(p, u, y, ws, st);
  p->timing = false;
  if (r != CASCADE_OK) return r;
  CK(cudaStreamSynchronize(st), "sync");
  for (int i = 0; i < p->n_ev; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]), "elapsed");
    const int k = p->ev_k[i];
    if (k >= 0 && k < (int)acc.size()) acc[k] += ms;
  }
  return CASCADE_OK;
}

extern "C" {

const char* cascade_status_string(cascade_status_t s) {
  switch (s) {
    case CASCADE_OK: return "ok";
    case CASCADE_ERR_INVALID_ARG: return "invalid argument";
    case CASCADE_ERR_UNSUPPORTED: return "unsupported";
    case CASCADE_ERR_OOM: return "out of device memory";
    case CASCADE_ERR_CUDA: return "CUDA error";
    case CASCADE_ERR_TIMEOUT: return "device wait timed out";
    case CASCADE_ERR_STATE: return "call order violated";
  }
  return "unknown status";
}

const char* cascade_last_error(cascade_plan_t plan) {
  static thread_local std::string tmp;
  if (plan) return plan->last_error.c_str();
  tmp = global_error();
  return tmp.c_str();
}

int64_t cascade_launch_count(void) { return g_launches; }

cascade_status_t cascade_plan_create(cascade_plan_t* out, const cascade_desc_t* desc) {
  Plan* p = nullptr;
  if (!out) return fail(p, CASCADE_ERR_INVALID_ARG, "plan output pointer is NULL");
  *out = nullptr;
  if (!desc) return fail(p, CASCADE_ERR_INVALID_ARG, "descriptor is NULL");
  const cascade_desc_t& d = *desc;
  if (d.m < 1 || d.p < 1 || d.q < 1 || d.nsys < 1 || d.max_len < 1 || d.max_rows < 0)
    return fail(p, CASCADE_ERR_INVALID_ARG, "m, p, q, nsys, max_len must be >= 1, max_rows >= 0");
  if (d.precision != CASCADE_FP64 && d.precision != CASCADE_FP32 &&
      d.precision != CASCADE_BF16_SPLIT)
    return fail(p, CASCADE_ERR_INVALID_ARG, "unknown precision");
  if (d.N < -1 || d.N > 40) return fail(p, CASCADE_ERR_INVALID_ARG, "N must be in -1..40");
  if (d.N < 0 && !(d.eps >= 0.0)) return fail(p, CASCADE_ERR_INVALID_ARG, "eps must be >= 0");
  if ((d.flags & CASCADE_FLAG_SCAN) &&
      (d.flags & (CASCADE_FLAG_SAVE_STATES | CASCADE_FLAG_RECOMPUTE)))
    return fail(p, CASCADE_ERR_INVALID_ARG,
                "the work-efficient schedule (CASCADE_FLAG_SCAN) has no backward: it cannot "
                "keep stage outputs");
  if ((d.flags & CASCADE_FLAG_SCAN) && d.precision == CASCADE_FP64)
    return fail(p, CASCADE_ERR_UNSUPPORTED,
                "the work-efficient schedule runs on the tensor-core precisions only");
  if (d.precision != CASCADE_FP64) {
    const int kc = d.precision == CASCADE_BF16_SPLIT ? 64 : 32;
    if (d.m % kc != 0 || d.m > 4096 || block_n(d.m, d.precision) == 0)
      return fail(p, CASCADE_ERR_UNSUPPORTED,
                  "tensor-core precisions need m a multiple of 64 (BF16) or 32 (FP32), m <= 4096");
    if (d.max_rows >= (int64_t(1) << 31))
      return fail(p, CASCADE_ERR_UNSUPPORTED, "max_rows must be < 2^31 (TMA coordinates)");
  } else if (d.m > 4096) {
    return fail(p, CASCADE_ERR_UNSUPPORTED, "m must be <= 4096");
  }
  p = new (std::nothrow) cascade_plan_s();
  if (!p) return fail(nullptr, CASCADE_ERR_OOM, "host allocation failed");
  p->d = d;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) {
    delete static_cast<cascade_plan_s*>(p);
    return fail(nullptr, CASCADE_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  const int Nmax = std::max(0, ceil_log2(d.max_len) - 1);
  p->kmax1 = (d.N >= 0) ? std::min(d.N, Nmax) + 1 : Nmax + 2;
  // y = C v + D u in the last stage's epilogue: one thread per row forms q dot
  // products of length m, which pays for q <= 4; wider outputs go to the
  // separate output GEMM
  p->fuse_output = d.precision != CASCADE_FP64 && !(d.flags & CASCADE_FLAG_NO_FUSED_OUTPUT) &&
                   block_n(d.m, d.precision) == d.m && d.q <= 4;
  // wider outputs of BF16-split plans whose projections run on the tensor cores
  // (p, q multiples of 16): y = C v + D u as a second tensor-core product in the
  // last stage, C v from the staged final state chunks (q <= 64: the y columns
  // fit inside one tile's accumulator); by default only where one tile spans all
  // m columns (measured slower than the separate pass at m = 1024)
  p->fuse_output_mma = !p->fuse_output && d.precision == CASCADE_BF16_SPLIT &&
                       !(d.flags & (CASCADE_FLAG_NO_FUSED_OUTPUT | CASCADE_FLAG_SCAN)) &&
                       d.m % 64 == 0 && d.p % 16 == 0 && d.q % 16 == 0 && d.q <= 64 &&
                       d.q <= block_n(d.m, d.precision) &&
                       (block_n(d.m, d.precision) >= d.m ||
                        (d.flags & CASCADE_FLAG_FUSE_WIDE_OUTPUT));
  e = cudaMalloc(&p->err, 8 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemset(p->err, 0, 8 * sizeof(int32_t));
  if (e != cudaSuccess) {
    delete static_cast<cascade_plan_s*>(p);
    return fail(nullptr, CASCADE_ERR_OOM, "device error word allocation failed");
  }
  *out = static_cast<cascade_plan_t>(p);
  return CASCADE_OK;
}

void cascade_plan_destroy(cascade_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : plan->ev) cudaEventDestroy(e);
  if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
  if (plan->io_stream) cudaStreamDestroy(plan->io_stream);
  for (cudaEvent_t e : plan->io_ev) cudaEventDestroy(e);
  free_batch(plan);
  free_system(plan);
  dfree(plan->err);
  delete plan;
}

cascade_status_t cascade_set_system_continuous(cascade_plan_t plan, const double* d_A,
                                               const double* d_B, const double* d_delta,
                                               const double* d_abar_scale, const double* d_C,
                                               const double* d_D, void* stream) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!d_A || !d_B || !d_delta || !d_C || !d_D)
    return fail(p, CASCADE_ERR_INVALID_ARG, "A, B, delta, C, D must be device pointers");
  cascade_status_t r = alloc_system(p);
  if (r != CASCADE_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int m = p->d.m, pp = p->d.p, q = p->d.q, ns = p->d.nsys;
  // keep the continuous system for the discretisation adjoint
  if (!p->A64) {
    CK(dalloc(&p->A64, (size_t)ns * m * m), "alloc A");
    CK(dalloc(&p->B64, (size_t)ns * m * pp), "alloc B");
    CK(dalloc(&p->delta64, (size_t)ns), "alloc delta");
    CK(dalloc(&p->scale64, (size_t)ns), "alloc scale");
  }
  CK(cudaMemcpyAsync(p->A64, d_A, sizeof(double) * ns * m * m, cudaMemcpyDeviceToDevice, st), "copy A");
  CK(cudaMemcpyAsync(p->B64, d_B, sizeof(double) * ns * m * pp, cudaMemcpyDeviceToDevice, st), "copy B");
  CK(cudaMemcpyAsync(p->delta64, d_delta, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st), "copy delta");
  if (d_abar_scale) {
    CK(cudaMemcpyAsync(p->scale64, d_abar_scale, sizeof(double) * ns, cudaMemcpyDeviceToDevice, st),
       "copy scale");
  } else {
    std::vector<double> ones(ns, 1.0);
    CK(cudaMemcpyAsync(p->scale64, ones.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st),
       "copy scale");
    CK(cudaStreamSynchronize(st), "sync");
  }
  CK(cudaMemcpyAsync(p->C64, d_C, sizeof(double) * ns * q * m, cudaMemcpyDeviceToDevice, st), "copy C");
  CK(cudaMemcpyAsync(p->D64, d_D, sizeof(double) * ns * q * pp, cudaMemcpyDeviceToDevice, st), "copy D");
  if (zoh(*p)) {
    r = discretise_zoh(p, st);
    if (r != CASCADE_OK) return r;
    p->continuous = true;
    return finish_system(p, st);
  }
  double* work = nullptr;
  int32_t* sing = nullptr;
  CK(dalloc(&work, (size_t)ns * m * (3 * m + pp)), "discretisation workspace");
  if (!p->Minv64) CK(dalloc(&p->Minv64, (size_t)ns * m * m), "alloc M^-1");
  cudaError_t e = cudaMalloc(&sing, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(sing, 0, sizeof(int32_t), st);
  // lower-triangular A (HiPPO-LegS): the elimination skips the zero triangle
  bool lower = false;
  if (e == cudaSuccess) check_lower(p, p->A64, (int64_t)m * m, &lower, st);
  if (e == cudaSuccess)
    e = launch_discretise(p->A64, p->B64, p->delta64, p->scale64, p->P64,
                          (int64_t)p->kmax1 * m * m, p->Bbar64, p->Minv64, work, ns, m, pp, sing,
                          lower, st);
  int32_t h_sing = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_sing, sing, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dfree(work);
  dfree(sing);
  if (e != cudaSuccess) return cuda_fail(p, e, "discretisation");
  if (h_sing) return fail(p, CASCADE_ERR_INVALID_ARG, "I - delta/2 A is singular for some system");
  p->continuous = true;
  return finish_system(p, st);
}

cascade_status_t cascade_set_system_discrete(cascade_plan_t plan, const double* d_Abar,
                                             const double* d_Bbar, const double* d_C,
                                             const double* d_D, void* stream) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!d_Abar || !d_Bbar || !d_C || !d_D)
    return fail(p, CASCADE_ERR_INVALID_ARG, "Abar, Bbar, C, D must be device pointers");
  cascade_status_t r = alloc_system(p);
  if (r != CASCADE_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int m = p->d.m, pp = p->d.p, q = p->d.q, ns = p->d.nsys;
  const size_t mm = (size_t)m * m;
  CK(cudaMemcpy2DAsync(p->P64, sizeof(double) * mm * p->kmax1, d_Abar, sizeof(double) * mm,
                       sizeof(double) * mm, ns, cudaMemcpyDeviceToDevice, st),
     "copy Abar");
  CK(cudaMemcpyAsync(p->Bbar64, d_Bbar, sizeof(double) * ns * m * pp, cudaMemcpyDeviceToDevice, st),
     "copy Bbar");
  CK(cudaMemcpyAsync(p->C64, d_C, sizeof(double) * ns * q * m, cudaMemcpyDeviceToDevice, st), "copy C");
  CK(cudaMemcpyAsync(p->D64, d_D, sizeof(double) * ns * q * pp, cudaMemcpyDeviceToDevice, st), "copy D");
  p->continuous = false;
  return finish_system(p, st);
}

cascade_status_t cascade_get_N(cascade_plan_t plan, int32_t* h_N) {
  Plan* p = plan;
  if (!p || !h_N) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_system) return fail(p, CASCADE_ERR_STATE, "no system set");
  memcpy(h_N, p->N_sys.data(), sizeof(int32_t) * p->N_sys.size());
  return CASCADE_OK;
}

cascade_status_t cascade_get_powers(cascade_plan_t plan, int32_t sys, int32_t kmax, double* d_out,
                                    void* stream) {
  Plan* p = plan;
  if (!p || !d_out) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_system) return fail(p, CASCADE_ERR_STATE, "no system set");
  if (sys < 0 || sys >= p->d.nsys || kmax < 0 || kmax >= p->kmax1)
    return fail(p, CASCADE_ERR_INVALID_ARG, "sys or kmax out of range");
  const size_t mm = (size_t)p->d.m * p->d.m;
  CK(cudaMemcpyAsync(d_out, p->P64 + (size_t)sys * p->kmax1 * mm, sizeof(double) * mm * (kmax + 1),
                     cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream)),
     "copy powers");
  return CASCADE_OK;
}

cascade_status_t cascade_set_batch(cascade_plan_t plan, const int64_t* h_offsets, int32_t nseq,
                                   const int32_t* h_sys_of_seq) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!p->have_system) return fail(p, CASCADE_ERR_STATE, "set a system before the batch");
  if (nseq < 0 || (nseq > 0 && !h_offsets))
    return fail(p, CASCADE_ERR_INVALID_ARG, "offsets missing or nseq < 0");
  if (nseq > 0 && h_offsets[0] != 0) return fail(p, CASCADE_ERR_INVALID_ARG, "offsets[0] != 0");
  for (int i = 0; i < nseq; ++i) {
    const int64_t L = h_offsets[i + 1] - h_offsets[i];
    if (L < 0) return fail(p, CASCADE_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (L > p->d.max_len) return fail(p, CASCADE_ERR_INVALID_ARG, "sequence longer than max_len");
    if (h_sys_of_seq && (h_sys_of_seq[i] < 0 || h_sys_of_seq[i] >= p->d.nsys))
      return fail(p, CASCADE_ERR_INVALID_ARG, "sys_of_seq out of range");
  }
  const int64_t rows = nseq > 0 ? h_offsets[nseq] : 0;
  if (rows > p->d.max_rows) return fail(p, CASCADE_ERR_INVALID_ARG, "more rows than max_rows");

  free_batch(p);
  p->nseq = nseq;
  p->rows = rows;
  p->offsets.assign(h_offsets, h_offsets + (nseq > 0 ? nseq + 1 : 0));
  if (nseq == 0) p->offsets.assign(1, 0);
  p->sys_of_seq.assign(nseq, 0);
  if (h_sys_of_seq) p->sys_of_seq.assign(h_sys_of_seq, h_sys_of_seq + nseq);
  p->seq_N.assign(nseq, -1);
  const bool save = keeps_states(*p);
  const int BM = tile_rows(*p);
  int maxN = -1;
  std::vector<Tile> t0s, outs, all;
  std::vector<Seq> seqs;
  for (int i = 0; i < nseq; ++i) {
    const int64_t L = h_offsets[i + 1] - h_offsets[i];
    const int sys = p->sys_of_seq[i];
    if (L == 0) continue;
    const int N = effective_N(p->N_sys[sys], L);
    p->seq_N[i] = N;
    maxN = std::max(maxN, N);
    seqs.push_back(Seq{h_offsets[i], (int32_t)L, sys, N, 0});
    for (int64_t t = 0; t < L; t += BM) {
      t0s.push_back(Tile{h_offsets[i], (int32_t)t, (int32_t)L, sys, 0, 0, 0});
      all.push_back(Tile{h_offsets[i], (int32_t)t, (int32_t)L, sys, N, 0, 0});   // flags = N_i
    }
  }
  p->maxN = maxN;
  // Stage 1 forms v^(1) on chip when nothing else needs it in memory; then
  // the first-stage kernel runs only for the sequences without a stage 1
  // (N_i = 0), whose output reads v^(1).
  p->fuse_first = p->d.precision != CASCADE_FP64 && !keeps_states(*p) && !scans(*p) &&
                  !(p->d.flags & CASCADE_FLAG_NO_FUSED_FIRST) && p->d.p <= FUSE_FIRST_PMAX &&
                  proj_supported(*p) && maxN >= 1;
  // The work-efficient schedule reads the even rows of v^(1) only in its last
  // down-sweep level, which with the output fused writes nothing but y: that
  // level forms them from u, and the first level stores only the odd rows and
  // row 0 (whose y the row-output kernel forms).
  p->scan_even_on_chip = scans(*p) && p->fuse_output &&
                         !(p->d.flags & CASCADE_FLAG_NO_FUSED_FIRST) &&
                         p->d.p <= FUSE_FIRST_PMAX && proj_supported(*p) &&
                         !proj_tc_supported(*p);
  if (p->fuse_first) {
    std::vector<Tile> keep;
    for (const Tile& t : t0s)
      if (effective_N(p->N_sys[t.sys], t.len) == 0) keep.push_back(t);
    t0s.swap(keep);
  }
  // products by powers: the Abar Bbar u term of the first stage on every row
  // l >= 1 (odd rows only in the work-efficient schedule), then the stages
  p->matvecs = 0;
  for (int i = 0; i < nseq; ++i) {
    const int64_t L = h_offsets[i + 1] - h_offsets[i];
    if (L == 0) continue;
    const int N = p->seq_N[i];
    if (scans(*p)) {
      if (N < ceil_log2(L) - 1) {
        free_batch(p);
        return fail(p, CASCADE_ERR_UNSUPPORTED,
                    "the work-efficient schedule needs 2^(N+1) >= L for every sequence "
                    "(truncated cascades use the stage schedule)");
      }
      p->matvecs += L / 2;
    } else {
      for (int k = 0; k <= N; ++k) p->matvecs += std::max<int64_t>(L - (int64_t(1) << k), 0);
    }
  }
  if (scans(*p)) {
    // Up-sweep level k (k = 1..K-1): rows l = (j+1) 2^(k+1) - 1 gain
    // Abar^(2^k) v_(l - 2^k); level 0 is the first-stage projection.
    // Down-sweep level k (k = K-2..0): rows l = (j+1) 2^(k+1) + 2^k - 1 gain
    // Abar^(2^k) v_(l - 2^k), whose prefix is complete.  One launch per level,
    // tiles of up to BM rows 2^(k+1) apart.
    const int K = maxN + 1;     // levels of the longest sequence
    int64_t cap = std::max<int64_t>(rows, 1);
    const int64_t Smax = int64_t(1) << std::max(K, 1);
    cap = (cap + Smax - 1) / Smax * Smax;
    if (cap >= (int64_t(1) << 31)) {
      free_batch(p);
      return fail(p, CASCADE_ERR_UNSUPPORTED, "rows rounded up to 2^K must stay below 2^31");
    }
    p->scan_rows_cap = cap;
    auto level = [&](int k, bool down) -> cascade_status_t {
      std::vector<Tile> tl;
      const int64_t S = int64_t(2) << k, d = down ? (int64_t(1) << k) : 0;
      for (int i = 0; i < nseq; ++i) {
        const int64_t L = h_offsets[i + 1] - h_offsets[i];
        const int64_t cnt = L > d ? (L - d) / S : 0;
        p->matvecs += cnt;
        for (int64_t j0 = 0; j0 < cnt; j0 += BM) {
          const int64_t R0 = h_offsets[i] + (j0 + 1) * S - 1 + d;
          // every row a down-sweep level writes is final: with the fused output its
          // epilogue also forms y for it
          tl.push_back(Tile{R0, 0, (int32_t)std::min<int64_t>(BM, cnt - j0), p->sys_of_seq[i],
                            (down && p->fuse_output) ? (int32_t)TILE_FINAL_FUSED : 0, 0, 0});
        }
      }
      Plan::ScanLevel lv{k, down ? 1 : 0, (int)tl.size(), nullptr};
      if (!tl.empty()) {
        CK(cudaMalloc(&lv.d_tiles, tl.size() * sizeof(Tile)), "alloc scan schedule");
        CK(cudaMemcpy(lv.d_tiles, tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice),
           "upload scan schedule");
      }
      p->scan.push_back(lv);
      return CASCADE_OK;
    };
    // Levels k >= k0 touch only rows (t+1) 2^k0 - 1 of each sequence; with at most
    // 128 such rows per sequence they run as one launch (a block per sequence,
    // states in TMEM) instead of one launch each.  k0: the smallest level with
    // L_i >> k0 <= 128 for every sequence; used when it replaces 3 or more launches.
    int64_t maxL = 0;
    for (int i = 0; i < nseq; ++i) maxL = std::max(maxL, h_offsets[i + 1] - h_offsets[i]);
    int k0 = 1;
    while ((maxL >> k0) > 128) ++k0;
    const bool top = scan_top_supported(*p) && K - k0 >= 2 &&
                     (K - k0) + (K - 1 - k0) >= 3;
    for (int k = 1; k <= K - 1; ++k) {
      if (top && k >= k0) {   // counted here, run by the top launch
        for (int i = 0; i < nseq; ++i) {
          const int64_t L = h_offsets[i + 1] - h_offsets[i];
          p->matvecs += L / (int64_t(2) << k);
        }
        continue;
      }
      const cascade_status_t r = level(k, false);
      if (r != CASCADE_OK) return r;
    }
    p->scan_top_pos = (int)p->scan.size();
    for (int k = K - 2; k >= 0; --k) {
      if (top && k >= k0) {
        const int64_t S = int64_t(2) << k, d = int64_t(1) << k;
        for (int i = 0; i < nseq; ++i) {
          const int64_t L = h_offsets[i + 1] - h_offsets[i];
          p->matvecs += L > d ? (L - d) / S : 0;
        }
        continue;
      }
      const cascade_status_t r = level(k, true);
      if (r != CASCADE_OK) return r;
    }
    if (top) {
      std::vector<Seq> ts;
      for (int i = 0; i < nseq; ++i) {
        const int64_t L = h_offsets[i + 1] - h_offsets[i];
        if ((L >> k0) >= 2)
          ts.push_back(Seq{h_offsets[i], (int32_t)L, p->sys_of_seq[i], p->seq_N[i], 0});
      }
      p->scan_top_k0 = k0;
      p->scan_top_K = K;
      p->n_top_seqs = (int)ts.size();
      if (!ts.empty()) {
        CK(cudaMalloc(&p->d_top_seqs, ts.size() * sizeof(Seq)), "alloc top schedule");
        CK(cudaMemcpy(p->d_top_seqs, ts.data(), ts.size() * sizeof(Seq), cudaMemcpyHostToDevice),
           "upload top schedule");
      }
    }
    if (p->fuse_output) {
      // rows l = 2^t - 1 are never written by the down-sweep: their y is formed
      // after the last level
      std::vector<int64_t> rws;
      std::vector<int32_t> rsys;
      for (int i = 0; i < nseq; ++i) {
        const int64_t L = h_offsets[i + 1] - h_offsets[i];
        for (int64_t l = 0; l < L; l = 2 * l + 1) {
          rws.push_back(h_offsets[i] + l);
          rsys.push_back(p->sys_of_seq[i]);
        }
      }
      p->n_scan_rows = (int)rws.size();
      if (!rws.empty()) {
        CK(cudaMalloc(&p->d_scan_rows, rws.size() * sizeof(int64_t)), "alloc scan rows");
        CK(cudaMalloc(&p->d_scan_rows_sys, rsys.size() * sizeof(int32_t)), "alloc scan rows");
        CK(cudaMemcpy(p->d_scan_rows, rws.data(), rws.size() * sizeof(int64_t),
                      cudaMemcpyHostToDevice), "upload scan rows");
        CK(cudaMemcpy(p->d_scan_rows_sys, rsys.data(), rsys.size() * sizeof(int32_t),
                      cudaMemcpyHostToDevice), "upload scan rows");
      }
    }
  }
  if (recomputes(*p)) {
    // segment length c: fewest state buffers 2 + ceil(maxN / c) + max(0, c - 3),
    // ties to the smaller c (more checkpoints, fewer recomputed stages)
    p->ck_seg = 2;
    int best = 1 << 30;
    for (int c = 2; c <= std::max(2, maxN); ++c) {
      const int nb = 2 + (std::max(maxN, 1) + c - 1) / c + std::max(0, c - 3);
      if (nb < best) { best = nb; p->ck_seg = c; }
    }
    p->n_ck = maxN >= 1 ? (maxN + p->ck_seg - 1) / p->ck_seg : 0;
  } else {
    p->ck_seg = 0;
    p->n_ck = 0;
  }
  for (Tile& t : all) t.fbuf = fwd_buf(*p, t.flags + 1);
  p->all_fbuf = all.empty() ? -1 : all[0].fbuf;
  for (const Tile& t : all)
    if (t.fbuf != p->all_fbuf) p->all_fbuf = -1;
  p->h_tiles.assign(std::max(maxN + 1, 1), {});
  p->stage_fused.assign(std::max(maxN + 1, 1), 0);
  for (int i = 0; i < nseq; ++i) {
    const int64_t L = h_offsets[i + 1] - h_offsets[i];
    if (L == 0) continue;
    const int N = p->seq_N[i], sys = p->sys_of_seq[i];
    const bool fused_last = (p->fuse_output || p->fuse_output_mma) && N >= 1 && !scans(*p);
    // (the work-efficient schedule forms y in its down-sweep levels instead)
    for (int k = 1; k <= N && !scans(*p); ++k) {   // stage schedule (§3)
      const bool fused = fused_last && k == N;
      if (fused) p->stage_fused[k] = 1;
      const int64_t prev_shift = int64_t(1) << (k - 1);
      for (int64_t t = 0; t < L; t += BM) {
        // Ping-pong buffers: rows below 2^(k-1) already hold their final value in the
        // output buffer.  Kept stage outputs or checkpoints: every stage writes every row.
        if (!save && !fused && k >= 2 && t + BM <= prev_shift) continue;
        p->h_tiles[k].push_back(Tile{h_offsets[i], (int32_t)t, (int32_t)L, sys,
                                     fused ? (int32_t)TILE_FINAL_FUSED : 0, 0, 0});
      }
    }
    if (!fused_last && !(scans(*p) && p->fuse_output)) {   // fbuf: buffer holding v^(N+1)
      const int buf = scans(*p) ? 0 : fwd_buf(*p, N + 1);
      for (int64_t t = 0; t < L; t += BM)
        outs.push_back(Tile{h_offsets[i], (int32_t)t, (int32_t)L, sys, 0, buf, 0});
    }
  }
  auto upload = [&](const std::vector<Tile>& v, Tile** d) -> cudaError_t {
    *d = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(d, v.size() * sizeof(Tile));
    if (e == cudaSuccess) e = cudaMemcpy(*d, v.data(), v.size() * sizeof(Tile), cudaMemcpyHostToDevice);
    return e;
  };
  p->d_tiles.assign(p->h_tiles.size(), nullptr);
  p->n_tiles.assign(p->h_tiles.size(), 0);
  for (size_t k = 0; k < p->h_tiles.size(); ++k) {
    CK(upload(p->h_tiles[k], &p->d_tiles[k]), "upload stage schedule");
    p->n_tiles[k] = (int32_t)p->h_tiles[k].size();
  }
  CK(upload(t0s, &p->d_stage0_tiles), "upload first-stage schedule");
  p->n_stage0_tiles = (int)t0s.size();
  // Stages 1 .. 3 in one pass over windows of 128 steps with the states on chip
  // (stage_fused.cu), for forward-only §3 plans with p = 1 at m = 128 or 256
  // whose sequences all run past stage 3 (none forms its output there).
  {
    const int J = 3, H = (2 << J) - 2;
    bool ok = fused_stages_supported(*p) && !scans(*p) &&
              !(p->d.flags & (CASCADE_FLAG_SAVE_STATES | CASCADE_FLAG_RECOMPUTE |
                              CASCADE_FLAG_NO_FUSED_STAGES));
    bool any = false;
    for (int i = 0; i < nseq && ok; ++i) {
      if (h_offsets[i + 1] == h_offsets[i]) continue;
      any = true;
      ok = p->seq_N[i] >= J + 1;
    }
    if (ok && any) {
      std::vector<FusedWindow> fw;
      for (int i = 0; i < nseq; ++i) {
        const int64_t L = h_offsets[i + 1] - h_offsets[i];
        for (int64_t o = 0; o < L; o += BM - H)
          fw.push_back(FusedWindow{h_offsets[i], (int32_t)(o - H), (int32_t)L,
                                   p->sys_of_seq[i], 0});
      }
      CK(cudaMalloc(&p->d_fwin, fw.size() * sizeof(FusedWindow)), "alloc fused windows");
      CK(cudaMemcpy(p->d_fwin, fw.data(), fw.size() * sizeof(FusedWindow),
                    cudaMemcpyHostToDevice),
         "upload fused windows");
      p->n_fwin = (int)fw.size();
      p->fused_J = J;
    }
  }
  // output tiles grouped by the buffer holding their final states (the
  // tensor-core output projection reads one buffer per launch)
  std::stable_sort(outs.begin(), outs.end(),
                   [](const Tile& a, const Tile& b) { return a.fbuf < b.fbuf; });
  p->out_segs.clear();
  for (int i = 0; i < (int)outs.size(); ++i) {
    if (p->out_segs.empty() || p->out_segs.back()[0] != outs[i].fbuf)
      p->out_segs.push_back({outs[i].fbuf, i, 0});
    p->out_segs.back()[2]++;
  }
  CK(upload(outs, &p->d_out_tiles), "upload output schedule");
  p->n_out_tiles = (int)outs.size();
  // Chunks of the first-stage and output tile lists for the host-buffer forward,
  // whose copies overlap the projections (tensor-core projections of one state
  // buffer: both lists then run in row order, so each chunk is a row range)
  p->io_in.clear();
  p->io_out.clear();
  if (proj_tc_supported(*p) && !scans(*p) && p->out_segs.size() <= 1) {
    auto chunk = [&](const std::vector<Tile>& v, std::vector<std::array<int64_t, 4>>& out) {
      const int n = (int)v.size(), CH = 4;
      for (int c = 0; c < CH && n > 0; ++c) {
        const int a = (int)((int64_t)n * c / CH), b = (int)((int64_t)n * (c + 1) / CH);
        if (b <= a) continue;
        const int64_t r0 = v[a].seq_row0 + v[a].t0;
        const int64_t r1 = v[b - 1].seq_row0 + std::min<int64_t>(v[b - 1].t0 + BM, v[b - 1].len);
        out.push_back({a, b - a, r0, r1 - r0});
      }
      // contiguous, covering every row in order
      int64_t next = 0;
      for (const auto& c : out) {
        if (c[2] != next) { out.clear(); return; }
        next = c[2] + c[3];
      }
      if (next != p->rows) out.clear();
    };
    chunk(t0s, p->io_in);
    chunk(outs, p->io_out);
  }
  if (!seqs.empty()) {
    CK(cudaMalloc(&p->d_seqs, seqs.size() * sizeof(Seq)), "alloc sequences");
    CK(cudaMemcpy(p->d_seqs, seqs.data(), seqs.size() * sizeof(Seq), cudaMemcpyHostToDevice),
       "upload sequences");
  }
  if (save) {
    // adjoint stage k walks the tiles of forward stage k (all tiles of the
    // sequences with N_i >= k) in reverse time order: its source rows l + s
    // then lie in tiles walked just before, and come from L2 as the forward's
    // sources l - s do (each tile's result does not depend on the order)
    p->d_adj_tiles.assign(p->d_tiles.size(), nullptr);
    p->n_adj_tiles = p->n_tiles;
    for (size_t k = 0; k < p->h_tiles.size(); ++k) {
      if (p->h_tiles[k].empty()) continue;
      const std::vector<Tile> rev(p->h_tiles[k].rbegin(), p->h_tiles[k].rend());
      CK(upload(rev, &p->d_adj_tiles[k]), "upload adjoint schedule");
    }
    CK(upload(all, &p->d_all_tiles), "upload tiles");
    p->n_all_tiles = (int)all.size();
    // Time-reduction chunks: runs of up to CH consecutive tiles of one system,
    // grouped by system (list 0: every tile; list k: the tiles of stage k).
    // Longer runs mean fewer partial sums to write and add; CH shrinks until
    // the reductions have at least three blocks per SM.  The tensor-core power
    // gradients of lists k >= 1 split each chunk further into (m / 128) x
    // (m / BN) output blocks, and each chunk leaves an m x m partial: their runs
    // grow (up to 64 tiles) while there are still three blocks per SM, and on
    // while the partials' write and read exceed 1/8 of the operand bytes the
    // chunk's blocks read (2 m^2 x 4 B against CH x 128 rows x 8m B, i.e. CH <
    // m / 16) and there are still 1.5 blocks per SM.  (Measured at m = 256:
    // six blocks per SM and no traffic rule took 4.82 ms per backward on 32 x
    // 8192 steps, p = q = 16, and 12.24 ms on 64 x 16384, p = q = 1; three
    // blocks, 4.61 and 12.10 ms; with the traffic rule, 4.44 and 12.10 ms.)
    int CH = 16;
    while (CH > 4 && (int64_t)all.size() < (int64_t)CH * 3 * p->num_sms) CH >>= 1;
    // the list of all tiles feeds the wide-by-thin reductions (one block per
    // chunk) unless they run on the tensor cores: then runs shrink to 4 tiles
    // while there are fewer than 8 blocks per SM
    int CH0 = CH;
    if (!(proj_tc_supported(*p) && thin_tc_supported(*p)))
      while (CH0 > 4 && (int64_t)all.size() < (int64_t)CH0 * 8 * p->num_sms) CH0 >>= 1;
    const int64_t grad_blocks =
        grad_tc_supported(*p) ? (int64_t)(p->d.m / 128) * (p->d.m / grad_tc_block_n(p->d.m)) : 0;
    std::vector<int32_t> data;
    p->chunk_lists.assign(std::max(maxN + 1, 1), ChunkList{});
    for (size_t li = 0; li < p->chunk_lists.size(); ++li) {
      const std::vector<Tile>& tl = li == 0 ? all : p->h_tiles[li];
      int CHl = li == 0 ? CH0 : CH;
      if (li > 0 && grad_blocks > 0) {
        CHl = 64;
        while (CHl > CH && (int64_t)tl.size() / CHl * grad_blocks < (int64_t)3 * p->num_sms)
          CHl >>= 1;
        while (CHl < 64 && CHl < p->d.m / 16 &&
               2 * ((int64_t)tl.size() / (2 * CHl) * grad_blocks) >= (int64_t)3 * p->num_sms)
          CHl <<= 1;
      }
      std::vector<std::array<int32_t, 3>> ch;
      for (int ti = 0; ti < (int)tl.size(); ++ti) {
        if (ch.empty() || ch.back()[2] != tl[ti].sys || ch.back()[1] == CHl ||
            ch.back()[0] + ch.back()[1] != ti)
          ch.push_back({ti, 0, tl[ti].sys});
        ch.back()[1]++;
      }
      std::stable_sort(ch.begin(), ch.end(),
                       [](const std::array<int32_t, 3>& a, const std::array<int32_t, 3>& b) {
                         return a[2] < b[2];
                       });
      ChunkList& cl = p->chunk_lists[li];
      cl.n = (int)ch.size();
      cl.off_chunks = data.size();
      for (auto& c : ch) data.insert(data.end(), c.begin(), c.end());
      cl.off_begin = data.size();
      size_t ci = 0;
      for (int sidx = 0; sidx <= p->d.nsys; ++sidx) {
        while (ci < ch.size() && ch[ci][2] < sidx) ++ci;
        data.push_back((int32_t)ci);
      }
      if (li == 0) p->chunks_all = cl.n;
      else p->max_chunks = std::max(p->max_chunks, cl.n);
    }
    // group sums for the reductions with little parallelism (fewer than
    // 2048 x SMs threads of one to four elements)
    p->red_scratch_bytes = (size_t)4 * 2048 * p->num_sms * sizeof(double);
    CK(cudaMalloc(&p->d_red_scratch, p->red_scratch_bytes), "alloc reduction scratch");
    CK(cudaMalloc(&p->d_chunk_data, data.size() * sizeof(int32_t)), "alloc chunks");
    CK(cudaMemcpy(p->d_chunk_data, data.data(), data.size() * sizeof(int32_t),
                  cudaMemcpyHostToDevice),
       "upload chunks");
  }
  p->have_batch = true;
  p->batch_id++;
  return CASCADE_OK;
}

cascade_status_t cascade_get_seq_N(cascade_plan_t plan, int32_t* h_N) {
  Plan* p = plan;
  if (!p || !h_N) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_batch) return fail(p, CASCADE_ERR_STATE, "no batch set");
  memcpy(h_N, p->seq_N.data(), sizeof(int32_t) * p->seq_N.size());
  return CASCADE_OK;
}

cascade_status_t cascade_get_matvec_count(cascade_plan_t plan, int64_t* h_count) {
  Plan* p = plan;
  if (!p || !h_count) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_batch) return fail(p, CASCADE_ERR_STATE, "no batch set");
  *h_count = p->matvecs;
  return CASCADE_OK;
}

cascade_status_t cascade_get_output_fused(cascade_plan_t plan, int32_t* h_fused) {
  Plan* p = plan;
  if (!p || !h_fused) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  *h_fused = (p->fuse_output || p->fuse_output_mma) ? 1 : 0;
  return CASCADE_OK;
}

cascade_status_t cascade_get_first_fused(cascade_plan_t plan, int32_t* h_fused) {
  Plan* p = plan;
  if (!p || !h_fused) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_batch) return fail(p, CASCADE_ERR_STATE, "no batch set");
  *h_fused = (p->fuse_first || p->scan_even_on_chip) ? 1 : 0;
  return CASCADE_OK;
}

cascade_status_t cascade_get_fused_stages(cascade_plan_t plan, int32_t* h_J) {
  Plan* p = plan;
  if (!p || !h_J) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_batch) return fail(p, CASCADE_ERR_STATE, "no batch set");
  *h_J = p->fused_J;
  return CASCADE_OK;
}

cascade_status_t cascade_workspace_size(cascade_plan_t plan, size_t* bytes) {
  Plan* p = plan;
  if (!p || !bytes) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (!p->have_batch) return fail(p, CASCADE_ERR_STATE, "no batch set");
  *bytes = forward_workspace(*p, p->rows);
  return CASCADE_OK;
}

cascade_status_t cascade_forward(cascade_plan_t plan, const void* d_u, void* d_y,
                                 void* d_workspace, size_t workspace_bytes, void* stream) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!p->have_system || !p->have_batch) return fail(p, CASCADE_ERR_STATE, "system and batch must be set");
  if (p->rows == 0) return CASCADE_OK;
  if (!d_u || !d_y || !d_workspace)
    return fail(p, CASCADE_ERR_INVALID_ARG, "u, y, workspace must be device pointers");
  if (!row_aligned(d_u) || !row_aligned(d_y))
    return fail(p, CASCADE_ERR_INVALID_ARG, "u and y must be 16-byte aligned");
  if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0)
    return fail(p, CASCADE_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (workspace_bytes < forward_workspace(*p, p->rows))
    return fail(p, CASCADE_ERR_INVALID_ARG, "workspace too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->last_stream = stream;
  if (p->d.flags & CASCADE_FLAG_GRAPH) {
    const bool hit = p->graph && p->graph_key[0] == d_u && p->graph_key[1] == d_y &&
                     p->graph_key[2] == d_workspace && p->graph_batch_id == p->batch_id;
    if (!hit) {
      if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
      }
      if (!p->cap_stream)
        CK(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking), "capture stream");
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      cascade_status_t r = run_forward(p, d_u, d_y, d_workspace, p->cap_stream);
      cudaError_t e = cudaStreamEndCapture(p->cap_stream, &g);
      if (r != CASCADE_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess) return cuda_fail(p, e, "end capture");
      e = cudaGraphInstantiate(&p->graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(p, e, "graph instantiate");
      p->graph_key[0] = d_u;
      p->graph_key[1] = d_y;
      p->graph_key[2] = d_workspace;
      p->graph_batch_id = p->batch_id;
    }
    CK(cudaGraphLaunch(p->graph, st), "graph launch");
    if (keeps_states(*p)) {
      p->saved_ws = d_workspace;
      p->saved_batch = p->batch_id;
    }
    return CASCADE_OK;
  }
  return run_forward(p, d_u, d_y, d_workspace, st);
}

cascade_status_t cascade_forward_host(cascade_plan_t plan, const void* h_u, void* h_y, void* d_u,
                                      void* d_y, void* d_workspace, size_t workspace_bytes,
                                      void* stream) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!p->have_system || !p->have_batch) return fail(p, CASCADE_ERR_STATE, "system and batch must be set");
  if (p->rows == 0) return CASCADE_OK;
  if (!h_u || !h_y || !d_u || !d_y)
    return fail(p, CASCADE_ERR_INVALID_ARG, "u and y need host and device buffers");
  if (!row_aligned(d_u) || !row_aligned(d_y))
    return fail(p, CASCADE_ERR_INVALID_ARG, "device u and y must be 16-byte aligned");
  const size_t es = p->d.precision == CASCADE_FP64 ? sizeof(double) : sizeof(float);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // With the tensor-core projections as launches of their own (and no graph), the
  // copies run chunk by chunk on a plan-owned stream beside them.
  const bool in = proj_tc_supported(*p) && !scans(*p) && p->fused_J == 0 && !p->fuse_first &&
                  !p->io_in.empty();
  const bool out = proj_tc_supported(*p) && !scans(*p) && !p->io_out.empty();
  if ((in || out) && !(p->d.flags & CASCADE_FLAG_GRAPH)) {
    if (!d_workspace) return fail(p, CASCADE_ERR_INVALID_ARG, "workspace must be a device pointer");
    if ((reinterpret_cast<uintptr_t>(d_workspace) & 255) != 0)
      return fail(p, CASCADE_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (workspace_bytes < forward_workspace(*p, p->rows))
      return fail(p, CASCADE_ERR_INVALID_ARG, "workspace too small");
    if (!p->io_stream)
      CK(cudaStreamCreateWithFlags(&p->io_stream, cudaStreamNonBlocking), "copy stream");
    const size_t nev = p->io_in.size() + p->io_out.size() + 2;
    while (p->io_ev.size() < nev) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
      p->io_ev.push_back(e);
    }
    // the copy stream starts after what the caller's stream has queued (which
    // may still read d_u or write d_y)
    CK(cudaEventRecord(p->io_ev[nev - 1], st), "event");
    CK(cudaStreamWaitEvent(p->io_stream, p->io_ev[nev - 1], 0), "wait");
    if (!in)
      CK(cudaMemcpyAsync(d_u, h_u, es * (size_t)p->rows * p->d.p, cudaMemcpyHostToDevice, st),
         "copy u to the device");
    const HostIO io{h_u, h_y, es * (size_t)p->d.p, es * (size_t)p->d.q, p->io_stream,
                    p->io_ev.data(), in, out};
    p->last_stream = stream;
    const cascade_status_t r = run_forward(p, d_u, d_y, d_workspace, st, &io);
    if (r != CASCADE_OK) {
      // the call is synchronous: no copy may still read h_u or write h_y
      cudaStreamSynchronize(p->io_stream);
      cudaStreamSynchronize(st);
      return r;
    }
    if (!out)
      CK(cudaMemcpyAsync(h_y, d_y, es * (size_t)p->rows * p->d.q, cudaMemcpyDeviceToHost, st),
         "copy y to the host");
  } else {
    CK(cudaMemcpyAsync(d_u, h_u, es * (size_t)p->rows * p->d.p, cudaMemcpyHostToDevice, st),
       "copy u to the device");
    const cascade_status_t r =
        cascade_forward(plan, d_u, d_y, d_workspace, workspace_bytes, stream);
    if (r != CASCADE_OK) {
      cudaStreamSynchronize(st);   // the copy of u has finished reading h_u
      return r;
    }
    CK(cudaMemcpyAsync(h_y, d_y, es * (size_t)p->rows * p->d.q, cudaMemcpyDeviceToHost, st),
       "copy y to the host");
  }
  CK(cudaStreamSynchronize(st), "synchronise");
  int32_t code = 0;
  CK(cudaMemcpy(&code, p->err, sizeof(code), cudaMemcpyDeviceToHost), "read error word");
  if (code != 0)
    return fail(p, CASCADE_ERR_TIMEOUT, "a bounded device wait gave up (cascade_get_device_error)");
  return CASCADE_OK;
}

cascade_status_t cascade_backward(cascade_plan_t plan, const void* d_u, const void* d_dy,
                                  void* d_du, double* d_dAbar, double* d_dBbar, double* d_dC,
                                  double* d_dD, double* d_dA, double* d_dB, void* d_workspace,
                                  size_t workspace_bytes, void* stream) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!keeps_states(*p))
    return fail(p, CASCADE_ERR_STATE,
                "backward needs a plan created with CASCADE_FLAG_SAVE_STATES or CASCADE_FLAG_RECOMPUTE");
  if (!p->have_system || !p->have_batch) return fail(p, CASCADE_ERR_STATE, "system and batch must be set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p->rows == 0) {   // no rows: every parameter gradient of sum(dy * y) is exactly zero
    const int m = p->d.m, pp = p->d.p, q = p->d.q, ns = p->d.nsys;
    const std::pair<double*, int64_t> outs[] = {
        {d_dAbar, (int64_t)m * m}, {d_dBbar, (int64_t)m * pp}, {d_dC, (int64_t)q * m},
        {d_dD, (int64_t)q * pp},   {p->continuous ? d_dA : nullptr, (int64_t)m * m},
        {p->continuous ? d_dB : nullptr, (int64_t)m * pp}};
    for (const auto& o : outs)
      if (o.first) CK(cudaMemsetAsync(o.first, 0, sizeof(double) * ns * o.second, st), "zero gradient");
    return CASCADE_OK;
  }
  if (!d_u || !d_dy || !d_workspace) return fail(p, CASCADE_ERR_INVALID_ARG, "u, dy, workspace required");
  if (!row_aligned(d_u) || !row_aligned(d_dy) || (d_du && !row_aligned(d_du)))
    return fail(p, CASCADE_ERR_INVALID_ARG, "u, dy and du must be 16-byte aligned");
  for (const double* g : {d_dAbar, d_dBbar, d_dC, d_dD, d_dA, d_dB})
    if (g && (reinterpret_cast<uintptr_t>(g) & (sizeof(double) - 1)) != 0)
      return fail(p, CASCADE_ERR_INVALID_ARG, "gradient outputs must be 8-byte aligned");
  if (p->saved_ws != d_workspace || p->saved_batch != p->batch_id)
    return fail(p, CASCADE_ERR_STATE, "run cascade_forward on this batch and workspace first");
  if (workspace_bytes < layout(*p).total) return fail(p, CASCADE_ERR_INVALID_ARG, "workspace too small");
  p->last_stream = stream;
  const cascade_status_t r =
      run_backward(p, d_u, d_dy, d_du, d_dAbar, d_dBbar, d_dC, d_dD, d_dA, d_dB, d_workspace, st);
  // recomputation reuses the buffers of the forward's final states
  if (recomputes(*p)) p->saved_ws = nullptr;
  return r;
}

cascade_status_t cascade_recursion_forward(cascade_plan_t plan, const double* d_u, double* d_y,
                                           void* stream) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!p->have_system || !p->have_batch) return fail(p, CASCADE_ERR_STATE, "system and batch must be set");
  if (p->rows == 0) return CASCADE_OK;
  if (!d_u || !d_y) return fail(p, CASCADE_ERR_INVALID_ARG, "u, y must be device pointers");
  if (((reinterpret_cast<uintptr_t>(d_u) | reinterpret_cast<uintptr_t>(d_y)) & 7) != 0)
    return fail(p, CASCADE_ERR_INVALID_ARG, "u and y must be 8-byte aligned");
  CK(launch_recursion_f64(*p, d_u, d_y, static_cast<cudaStream_t>(stream)), "recursion");
  return CASCADE_OK;
}

cascade_status_t cascade_get_device_error(cascade_plan_t plan, int32_t* h_code) {
  Plan* p = plan;
  if (!p || !h_code) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(p->last_stream);
  CK(cudaStreamSynchronize(st), "sync");
  int32_t words[8];
  CK(cudaMemcpy(words, p->err, sizeof(words), cudaMemcpyDeviceToHost), "read error word");
  CK(cudaMemset(p->err, 0, sizeof(words)), "clear error word");
  *h_code = words[0];
  if (words[0] != 0) {
    char buf[160];
    snprintf(buf, sizeof buf, "device wait gave up: site %d block %d counters %d %d stage %d",
             words[1], words[2], words[3], words[4], words[5]);
    p->last_error = buf;
  }
  return CASCADE_OK;
}

cascade_status_t cascade_autotune(cascade_plan_t plan, const void* d_u, void* d_y,
                                  void* d_workspace, size_t workspace_bytes, void* stream,
                                  int32_t reps, int32_t* h_choice) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (!p->have_system || !p->have_batch) return fail(p, CASCADE_ERR_STATE, "system and batch must be set");
  if (p->d.precision == CASCADE_FP64 || p->rows == 0) return CASCADE_OK;   // nothing to tune
  if (!d_u || !d_y || !d_workspace) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL buffer");
  if (workspace_bytes < forward_workspace(*p, p->rows))
    return fail(p, CASCADE_ERR_INVALID_ARG, "workspace too small");
  if (reps < 1) reps = 1;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  p->last_stream = stream;
  const bool timing = p->timing;
  p->timing = false;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  TcConfig best_c = tc_default(p->d.m, p->d.precision);
  cascade_status_t r = CASCADE_OK;
  // Each candidate's stages (or scan levels) are also timed one by one, and
  // every stage keeps the candidate that ran it fastest (the plan-wide shape,
  // the fastest whole forward, serves the adjoint stages and the top of the
  // scan tree).  Keys as the stage timings: k, or 100 + k for down-sweep levels.
  const bool per_stage = p->maxN >= 1;
  const int nkeys = scans(*p) ? 100 + p->maxN + 2 : p->maxN + 1;
  const std::vector<TcConfig> cands = tc_candidates(p->d.m, p->d.precision);
  std::vector<std::vector<float>> stage_ms;
  p->tc_stage_shape.clear();
  for (const TcConfig& c : cands) {
    p->tc_stages = c.stages;
    p->tc_ring = c.ring;
    p->tc_group = c.group;
    r = run_forward(p, d_u, d_y, d_workspace, st);             // warm-up
    if (r != CASCADE_OK) break;
    if (cudaEventRecord(e0, st) != cudaSuccess) { r = CASCADE_ERR_CUDA; break; }
    for (int i = 0; i < reps && r == CASCADE_OK; ++i) r = run_forward(p, d_u, d_y, d_workspace, st);
    if (r != CASCADE_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      r = cuda_fail(p, cudaGetLastError(), "autotune timing");
      break;
    }
    if (ms < best) { best = ms; best_c = c; }
    if (per_stage) {
      std::vector<float> acc(nkeys, 0.f);
      for (int i = 0; i < reps && r == CASCADE_OK; ++i)
        r = timed_stages(p, d_u, d_y, d_workspace, st, acc);
      if (r != CASCADE_OK) break;
      stage_ms.push_back(std::move(acc));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->timing = timing;
  p->tc_stages = best_c.stages;
  p->tc_ring = best_c.ring;
  p->tc_group = best_c.group;
  if (r == CASCADE_OK && per_stage && stage_ms.size() == cands.size() && !cands.empty()) {
    p->tc_stage_shape.assign(nkeys, {0, 0, 0});
    for (int k = 0; k < nkeys; ++k) {
      size_t bi = 0;
      for (size_t ci = 1; ci < cands.size(); ++ci)
        if (stage_ms[ci][k] < stage_ms[bi][k]) bi = ci;
      if (stage_ms[bi][k] > 0.f)
        p->tc_stage_shape[k] = {cands[bi].stages, cands[bi].ring, cands[bi].group};
    }
  }
  p->tuned = (r == CASCADE_OK);
  if (p->graph) {   // the recorded graph holds the old kernel shape
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  if (h_choice) {
    h_choice[0] = best_c.stages;
    h_choice[1] = best_c.ring;
    h_choice[2] = best_c.group;
  }
  return r;
}

cascade_status_t cascade_set_kernel_shape(cascade_plan_t plan, const int32_t* h_shape) {
  Plan* p = plan;
  if (!p || !h_shape) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  if (p->d.precision == CASCADE_FP64) return CASCADE_OK;
  bool ok = false;
  for (const TcConfig& c : tc_candidates(p->d.m, p->d.precision))
    ok = ok || (c.ring == h_shape[1] && c.group == h_shape[2] && h_shape[0] >= 2 &&
                h_shape[0] <= c.stages);
  if (!ok) return fail(p, CASCADE_ERR_INVALID_ARG, "kernel shape does not fit this plan");
  p->tc_stages = h_shape[0];
  p->tc_ring = h_shape[1];
  p->tc_group = h_shape[2];
  p->tc_stage_shape.clear();   // one shape for every stage
  if (p->graph) {
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  return CASCADE_OK;
}

cascade_status_t cascade_set_stage_shapes(cascade_plan_t plan, int32_t n,
                                          const int32_t* h_shape) {
  Plan* p = plan;
  if (!p || n < 0 || n > 4096 || (n > 0 && !h_shape))
    return fail(p, CASCADE_ERR_INVALID_ARG, "bad stage-shape array");
  if (p->d.precision == CASCADE_FP64) return CASCADE_OK;
  if (n > 0 && !p->have_batch)
    return fail(p, CASCADE_ERR_STATE, "per-stage shapes need a batch (their keys follow its schedule)");
  // keys: stage k = 1..maxN of the §3 schedule; up-sweep level k or 100 + k
  // for down-sweep level k of the work-efficient one (the levels it launches)
  const int nkeys = scans(*p) ? 100 + p->maxN + 2 : p->maxN + 1;
  if (n > nkeys)
    return fail(p, CASCADE_ERR_INVALID_ARG, "more stage-shape entries than this plan's schedule has");
  std::vector<char> launched(std::max(nkeys, 0), 0);
  if (scans(*p)) {
    for (const Plan::ScanLevel& lv : p->scan) {
      const int key = lv.down ? 100 + lv.k : lv.k;
      if (key >= 0 && key < nkeys) launched[key] = 1;
    }
  } else {
    for (int k = 1; k <= p->maxN; ++k) launched[k] = 1;
  }
  const std::vector<TcConfig> cands = tc_candidates(p->d.m, p->d.precision);
  std::vector<std::array<int32_t, 3>> sh(n, {0, 0, 0});
  for (int k = 0; k < n; ++k) {
    const int32_t* e = h_shape + 3 * k;
    if (e[0] == 0 && e[1] == 0 && e[2] == 0) continue;
    if (!launched[k])
      return fail(p, CASCADE_ERR_INVALID_ARG, "a stage shape names a stage or level this plan does not launch");
    bool ok = false;
    for (const TcConfig& c : cands)
      ok = ok || (c.ring == e[1] && c.group == e[2] && e[0] >= 2 && e[0] <= c.stages);
    if (!ok) return fail(p, CASCADE_ERR_INVALID_ARG, "a stage shape does not fit this plan");
    sh[k] = {e[0], e[1], e[2]};
  }
  p->tc_stage_shape.swap(sh);
  if (p->graph) {   // the recorded graph holds the old kernel shapes
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  return CASCADE_OK;
}

cascade_status_t cascade_get_stage_shapes(cascade_plan_t plan, int32_t cap, int32_t* h_shape,
                                          int32_t* n) {
  Plan* p = plan;
  if (!p || !n || (cap > 0 && !h_shape)) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  const int size = (int)p->tc_stage_shape.size();
  for (int k = 0; k < std::min<int>(cap, size); ++k)
    for (int j = 0; j < 3; ++j) h_shape[3 * k + j] = p->tc_stage_shape[k][j];
  *n = size;
  return CASCADE_OK;
}

cascade_status_t cascade_enable_stage_timing(cascade_plan_t plan, int32_t enable) {
  Plan* p = plan;
  if (!p) return fail(p, CASCADE_ERR_INVALID_ARG, "plan is NULL");
  if (enable && (p->d.flags & CASCADE_FLAG_GRAPH))
    return fail(p, CASCADE_ERR_UNSUPPORTED, "stage timing is not available with graph replay");
  p->timing = enable != 0;
  return CASCADE_OK;
}

cascade_status_t cascade_get_stage_times(cascade_plan_t plan, int32_t cap, int32_t* h_k,
                                         float* h_ms, int32_t* n) {
  Plan* p = plan;
  if (!p || !n || (cap > 0 && (!h_k || !h_ms))) return fail(p, CASCADE_ERR_INVALID_ARG, "NULL argument");
  CK(cudaStreamSynchronize(static_cast<cudaStream_t>(p->last_stream)), "sync");
  const int cnt = std::min(cap, p->n_ev);
  for (int i = 0; i < cnt; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p->ev[2 * i], p->ev[2 * i + 1]), "elapsed");
    h_k[i] = p->ev_k[i];
    h_ms[i] = ms;
  }
  *n = p->n_ev;
  return CASCADE_OK;
}

cascade_status_t cascade_selftest_timeout(int32_t limit_us) {
  Plan* p = nullptr;
  if (limit_us <= 0 || limit_us > 10000000)
    return fail(p, CASCADE_ERR_INVALID_ARG, "limit_us must be in 1..1e7");
  int32_t* d_err = nullptr;
  CK(cudaMalloc(&d_err, sizeof(int32_t)), "alloc");
  cudaError_t e = cudaMemset(d_err, 0, sizeof(int32_t));
  if (e == cudaSuccess) e = launch_selftest_timeout(limit_us, d_err, 0);
  int32_t h = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
  cudaFree(d_err);
  if (e != cudaSuccess) return cuda_fail(p, e, "self-test");
  return h == CASCADE_ERR_TIMEOUT ? CASCADE_ERR_TIMEOUT : CASCADE_OK;
}

}  // extern "C"
