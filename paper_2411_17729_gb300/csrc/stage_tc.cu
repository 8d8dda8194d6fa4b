// stage_tc.cu -- one cascade stage on the tcgen05 tensor cores (sm_103a).
//
// Stage k of §3 (Eqs. 3.2-3.4 and the general step) updates every time step
// l >= s = 2^k of every sequence:
//
//     v_l <- v_l + P v_(l - s),        P = Abar^(2^k),
//
// and leaves l < s unchanged (a source before the sequence start is zero:
// x_(-1) = 0).  With states stored time-major (row l of a [rows, m] matrix),
// the whole stage over all sequences is the dense contraction
//
//     Vout[tile rows] = Vin[tile rows] + Vin[tile rows - s] * P^T,
//
// an M = 128 (time) x N = BN (state) x K = m product per tile.  The shift is a
// TMA row offset; rows that fall before the sequence start are zeroed in
// shared memory before the tensor core reads them.
//
// Precision: P and V are carried as (hi, lo) pairs and the product is taken as
//     Vhi Phi^T + Vhi Plo^T + Vlo Phi^T
// (three passes over K), accumulated in FP32 in TMEM.  BF16 pairs (ELEM = 2)
// keep ~16 significant bits; TF32 pairs (ELEM = 4, FP32 storage) keep ~22.
// The tensor core's FP32 accumulation is not round-to-nearest (an emulation
// with truncating adds reproduces the measured error), so the TF32 path adds
// the two small correction products into a second TMEM accumulator and sums
// the two in the epilogue: the large partial sum is then rounded once per
// MMA instead of three times.
//
// Block layout (352 threads, or 480 when stage 1 forms v^(1) on chip; one
// block per SM, persistent over work items):
//   warp 0      TMA producer of the MMA operands (one elected lane)
//   warp 1      TMEM allocator and MMA issuer (one elected lane)
//   warps 2..5  epilogue group 0 and warps 7..10 epilogue group 1 (the two
//               take alternate column-chunk steps), thread = tile row = TMEM
//               lane: accumulator row + residual row -> new (hi, lo) row,
//               written back into the staging slot the residual arrived in
//   warp 6      staging-ring manager (one elected lane): TMA loads of the
//               residual column chunks RING chunks ahead (across tiles), TMA
//               stores of finished chunks, refill of each slot once its store
//               has read it
//   warps 11..14 (stage 1 on chip only) write the operand rows v^(1)_(l-s)
//               formed from u into the operand stages
// HBM traffic is whole lines in both directions, and the 64-byte swizzle of
// every shared tile keeps the thread-per-row accesses free of bank conflicts.
// No named barrier joins the epilogue warps: they signal a finished chunk
// with an mbarrier arrive and only ever wait (boundedly) for data.
// Pipelines: `stages` operand buffers (full/empty) producer -> MMA; two TMEM
// accumulators (acc_full/acc_empty) MMA -> epilogue, so tile i's epilogue
// overlaps tile i+1's MMAs; `ring` staging slots (res_full/res_done)
// manager <-> epilogue.
#include "common.cuh"
#include "ptx.cuh"

#include <cstring>

namespace cascade {
namespace {

constexpr int BM = 128;
// warps: 0 TMA producer, 1 MMA issuer, 6 ring manager, 2-5 and 7-10 epilogue
// (two groups of four, one warp per TMEM lane quadrant in each)
constexpr int NTHREADS = 352;
constexpr int GEN_THREADS = 128;              // first-stage row warps (stage 1 on chip)
constexpr int RING_MAX = 8;                   // staging slots (runtime ring <= 8)
constexpr uint32_t ROWB = 64;                 // bytes per row of every shared tile
constexpr uint32_t PLANE_TILE = BM * ROWB;    // one plane of a 128-row chunk: 8 KB
constexpr uint32_t SLOT_BYTES = 2 * PLANE_TILE;

// Tensor maps of the output on the tensor cores (YM): C and D (hi, lo) planes,
// [nsys q, m] and [nsys q, p], boxes of 32 K entries x q rows; u (hi, lo) planes
// [rows, p], boxes of 32 x 128 rows.
struct YMaps {
  CUtensorMap chi, clo, uhi, ulo, dhi, dlo;
};

template <int ELEM>
struct Fmt;

// BF16 pair: a 64-byte row chunk holds 32 elements; 16 bytes = 8 elements.
template <>
struct Fmt<2> {
  static constexpr int CW = 32;
  // a BF16 pair word as two FP32 lanes (a BF16 value is the top half of the
  // FP32 with the same bits)
  static __device__ __forceinline__ uint64_t widen(uint32_t w) {
    return ptx::f2_pack(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
  }
  // v += hi + lo, two lanes per operation
  static __device__ __forceinline__ void add16(uint4 h, uint4 l, float* v) {
    const uint32_t aw[4] = {h.x, h.y, h.z, h.w};
    const uint32_t bw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t t = ptx::f2_add(widen(aw[j]), widen(bw[j]));
      const float2 r = ptx::f2_unpack(ptx::f2_add(ptx::f2_pack(v[2 * j], v[2 * j + 1]), t));
      v[2 * j] = r.x;
      v[2 * j + 1] = r.y;
    }
  }
  // hi = RN_bf16(x), lo = RN_bf16(x - hi)
  static __device__ __forceinline__ void split16(const float* v, uint4& h, uint4& l) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      hw[j] = *reinterpret_cast<const uint32_t*>(&hh);
      const float2 d = ptx::f2_unpack(ptx::f2_sub(ptx::f2_pack(v[2 * j], v[2 * j + 1]), widen(hw[j])));
      const __nv_bfloat162 ll = __floats2bfloat162_rn(d.x, d.y);
      lw[j] = *reinterpret_cast<const uint32_t*>(&ll);
    }
    h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
};

// FP32 pair: hi = RN_tf32(x), lo = RN_tf32(x - hi), both TF32-exact, so the
// tensor core (which reads the top 19 bits of each operand) sees them unrounded
// and hi + lo carries x to ~2^-22 relative without bias.  16 bytes = 4 elements.
template <>
struct Fmt<4> {
  static constexpr int CW = 16;
  // v += hi + lo, two lanes per operation
  static __device__ __forceinline__ void add16(uint4 h, uint4 l, float* v) {
    const uint64_t t01 = ptx::f2_add(ptx::f2_pack(__uint_as_float(h.x), __uint_as_float(h.y)),
                                     ptx::f2_pack(__uint_as_float(l.x), __uint_as_float(l.y)));
    const uint64_t t23 = ptx::f2_add(ptx::f2_pack(__uint_as_float(h.z), __uint_as_float(h.w)),
                                     ptx::f2_pack(__uint_as_float(l.z), __uint_as_float(l.w)));
    const float2 r01 = ptx::f2_unpack(ptx::f2_add(ptx::f2_pack(v[0], v[1]), t01));
    const float2 r23 = ptx::f2_unpack(ptx::f2_add(ptx::f2_pack(v[2], v[3]), t23));
    v[0] = r01.x;
    v[1] = r01.y;
    v[2] = r23.x;
    v[3] = r23.y;
  }
  static __device__ __forceinline__ void split16(const float* v, uint4& h, uint4& l) {
    float hv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) hv[j] = ptx::tf32_rna(v[j]);
    const float2 d01 =
        ptx::f2_unpack(ptx::f2_sub(ptx::f2_pack(v[0], v[1]), ptx::f2_pack(hv[0], hv[1])));
    const float2 d23 =
        ptx::f2_unpack(ptx::f2_sub(ptx::f2_pack(v[2], v[3]), ptx::f2_pack(hv[2], hv[3])));
    h = make_uint4(__float_as_uint(hv[0]), __float_as_uint(hv[1]), __float_as_uint(hv[2]),
                   __float_as_uint(hv[3]));
    l = make_uint4(__float_as_uint(ptx::tf32_rna(d01.x)), __float_as_uint(ptx::tf32_rna(d01.y)),
                   __float_as_uint(ptx::tf32_rna(d23.x)), __float_as_uint(ptx::tf32_rna(d23.y)));
  }
};

// v[e] += Bbar[col0 + e] . x1 + (Abar Bbar)[col0 + e] . x0 for e < NV, with
// Bs, ABs the [m, p] coefficient matrices of one system and x1, x0 the p
// inputs u_l, u_(l-1): the first stage fused with the input projection, with
// the first-stage kernel's operation order (from v = 0 the same value).
template <int NV>
__device__ __forceinline__ void add_first_stage(const float* __restrict__ Bs,
                                                const float* __restrict__ ABs, int p, int col0,
                                                const float* x1, const float* x0, float* v) {
  if (p == 1) {
    // v += fma(ABbar, u_(l-1), Bbar * u_l), two lanes per operation
    const uint64_t u1 = ptx::f2_pack(x1[0], x1[0]), u0 = ptx::f2_pack(x0[0], x0[0]);
#pragma unroll
    for (int e = 0; e < NV; e += 4) {
      const float4 b = __ldg(reinterpret_cast<const float4*>(Bs + col0 + e));
      const float4 a = __ldg(reinterpret_cast<const float4*>(ABs + col0 + e));
      const uint64_t s01 =
          ptx::f2_fma(ptx::f2_pack(a.x, a.y), u0, ptx::f2_mul(ptx::f2_pack(b.x, b.y), u1));
      const uint64_t s23 =
          ptx::f2_fma(ptx::f2_pack(a.z, a.w), u0, ptx::f2_mul(ptx::f2_pack(b.z, b.w), u1));
      const float2 r01 = ptx::f2_unpack(ptx::f2_add(ptx::f2_pack(v[e], v[e + 1]), s01));
      const float2 r23 = ptx::f2_unpack(ptx::f2_add(ptx::f2_pack(v[e + 2], v[e + 3]), s23));
      v[e] = r01.x;
      v[e + 1] = r01.y;
      v[e + 2] = r23.x;
      v[e + 3] = r23.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < NV; ++e) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < p) {
          acc = fmaf(__ldg(Bs + (int64_t)(col0 + e) * p + j), x1[j], acc);
          acc = fmaf(__ldg(ABs + (int64_t)(col0 + e) * p + j), x0[j], acc);
        }
      v[e] += acc;
    }
  }
}

// Record the first bounded wait that gave up: the error word, and where
// (site, block, two counters of that wait) in the diagnostic words.
__device__ __forceinline__ void raise_timeout(const StageArgs& a, volatile int* abort_flag, int site,
                                              int x, int y) {
  if (atomicCAS(a.err, 0, (int32_t)CASCADE_ERR_TIMEOUT) == 0 && a.diag) {
    a.diag[0] = site;
    a.diag[1] = (int32_t)blockIdx.x;
    a.diag[2] = x;
    a.diag[3] = y;
    a.diag[4] = a.k;
  }
  *abort_flag = 1;
}

// Per-item facts every role derives identically from the tile table.
struct Item {
  Tile t;
  int nb;         // column block of the tile
  int n0;
  bool copy;      // every source row precedes the sequence: no MMA, output = residual
  bool fused;     // last stage with y = C v + D u formed in the epilogue
  bool ragged;    // last tile of a sequence: rows past its end must not be written
  bool acc;       // holds a TMEM accumulator (MMA items, and fused items with YM)
};

// Work items are (tile, column block) pairs, w = tile * nblocks + block.  The
// usual order gives block b the items b, b + grid, ...; with the output on the
// tensor cores (YM) a block takes whole tiles, their column blocks one after
// the other, so that it can sum a tile's partial outputs itself.
template <int YM>
__device__ __forceinline__ int first_item(const StageArgs& a) {
  return YM ? (int)blockIdx.x * a.nblocks : (int)blockIdx.x;
}
template <int YM>
__device__ __forceinline__ int next_item(const StageArgs& a, int w) {
  if (!YM) return w + (int)gridDim.x;
  return (w % a.nblocks != a.nblocks - 1) ? w + 1 : w + 1 + ((int)gridDim.x - 1) * a.nblocks;
}

template <int QMAX, int YM = 0>
__device__ __forceinline__ Item load_item(const StageArgs& a, int w) {
  Item it;
  it.t = a.tiles[w / a.nblocks];
  it.nb = w % a.nblocks;
  it.n0 = it.nb * a.BN;
  // every source row lies outside the sequence: before its start (forward
  // stages) or past its end (adjoint stages, source l + s)
  it.copy = a.S ? false
                 : a.reverse ? (it.t.t0 + a.shift >= it.t.len) : (it.t.t0 + BM <= a.shift);
  it.fused = (QMAX > 0 || YM) && (it.t.flags & TILE_FINAL_FUSED);
  it.ragged = it.t.t0 + BM > it.t.len;
  it.acc = !it.copy || (YM && it.fused);
  return it;
}

// Column chunks the staging ring carries for an item: the residual's, then,
// for the first column block of a tile whose output is formed on the tensor
// cores, the (u, D) chunks of the D u term.
template <int YM>
__device__ __forceinline__ int item_chunks(const StageArgs& a, const Item& it, int nch) {
  return nch + ((YM && it.fused && it.nb == 0) ? (a.p + 31) / 32 : 0);
}

// QMAX: 0 = never fuse the output; otherwise the largest q the fused
// epilogue handles (register accumulators for y).  G: column chunks the
// epilogue processes per step (their instructions interleave).
// GEN = 1 (stage 1 of the §3 schedule): no copy of v^(1) is read.  Four more
// warps form the operand rows v^(1)_(l-2) from u in shared memory, and the
// epilogue forms the residual v^(1)_l from u, so the first stage never goes
// through device memory.  GEN = 2 (the last down-sweep level of the
// work-efficient schedule, rows 2 apart): the destination rows are even, and
// an even row still holds v^(1)_l = Bbar u_l there; the epilogue forms that
// residual from u, the operand rows come by TMA as usual.  Both round v^(1) to
// the state format as the first-stage kernel does: the results equal those of
// the path through memory bit for bit.
// YM = 1 (BF16 pairs, p and q multiples of 16, q <= 64): tiles flagged
// TILE_FINAL_FUSED form y = C v + D u on the tensor cores.  The finished (hi,
// lo) state chunk the epilogue leaves in its staging slot is the A operand of a
// second product whose B operand, a 64-byte K chunk of C, the ring manager
// loads into the same slot next to the residual; the first column block of a
// tile adds D u from (u, D) chunks that follow its residual chunks.  One more
// warp (the y issuer) issues these products into TMEM columns [0, q) of the
// tile's own accumulator, once the epilogue has read those columns.  Epilogue
// group 0 reads the tile's y from there and, when m spans several column
// blocks (taken one after the other by the same block), adds them in order in
// its rows of y.
template <int ELEM, int QMAX, int G, int GEN, int YM>
__global__ void __launch_bounds__(GEN == 1 ? NTHREADS + GEN_THREADS : YM ? NTHREADS + 32 : NTHREADS, 1)
    stage_tc_kernel(const __grid_constant__ CUtensorMap tm_vhi,
                    const __grid_constant__ CUtensorMap tm_vlo,
                    const __grid_constant__ CUtensorMap tm_phi,
                    const __grid_constant__ CUtensorMap tm_plo,
                    const __grid_constant__ CUtensorMap tm_ohi,
                    const __grid_constant__ CUtensorMap tm_olo,
                    const __grid_constant__ YMaps ym, const StageArgs args) {
  constexpr int KC = (int)ROWB / ELEM;   // K elements per 64-byte operand row
  constexpr int UK = 32 / ELEM;          // K per tcgen05.mma
  constexpr int CW = Fmt<ELEM>::CW;      // epilogue chunk: columns per 64-byte row
  constexpr uint32_t FMT = (ELEM == 2) ? 1u : 2u;
  constexpr bool SEP = (ELEM == 4);      // separate accumulator for the correction products
  constexpr int QN = QMAX > 0 ? QMAX : 1;
  const int BN = args.BN;
  const int ACC = SEP ? 2 * args.BN : args.BN;   // TMEM columns of one tile's accumulators
  const int S = args.stages;
  const int RING = args.ring;                    // multiple of G, <= RING_MAX
  const int m = args.m;
  const int nkc = m / KC;
  const int nch = BN / CW;
  const int shift = args.shift;
  const int nwork = args.ntiles * args.nblocks;
  const int q = args.q;
  // a staging slot: the residual's (hi, lo) chunk, then (YM) a (hi, lo) K chunk
  // of C or D, q rows of 64 bytes each
  const uint32_t slot_bytes = YM ? SLOT_BYTES + 2u * (uint32_t)q * ROWB : SLOT_BYTES;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const uint32_t a_bytes = PLANE_TILE;
  const uint32_t b_bytes = (uint32_t)BN * ROWB;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  uint8_t* bufs = smem;
  uint8_t* ring = smem + (size_t)S * stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)RING * slot_bytes);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* res_full = acc_empty + 2;
  uint64_t* res_done = res_full + RING_MAX;
  uint64_t* drain = res_done + RING_MAX;
  uint64_t* ypart = drain + 1;      // group 1's partial y sums of a fused tile are ready
  uint64_t* yfree = ypart + 1;      // group 0 has taken them
  uint64_t* ymma_done = yfree + 1;  // [RING_MAX] (YM) the y issuer is done with a slot
  uint64_t* yfull = ymma_done + RING_MAX;   // [2] (YM) a tile's y products completed
  uint64_t* ydrain = yfull + 2;             // (YM) the y issuer's products completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ydrain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* ysum = reinterpret_cast<float*>(tmem_slot + 4);   // [QN][128]

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t tmem_cols = (ACC * 2 <= 32) ? 32u : (ACC * 2 <= 64) ? 64u : (ACC * 2 <= 128) ? 128u
                             : (ACC * 2 <= 256) ? 256u : 512u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(&full[s], GEN == 1 ? 2 : 1);   // the power copies and the row warps
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&acc_full[b], 1);
      ptx::mbar_init(&acc_empty[b], 256);    // both epilogue groups
    }
    for (int s = 0; s < RING; ++s) {
      ptx::mbar_init(&res_full[s], 1);
      ptx::mbar_init(&res_done[s], 128);
    }
    ptx::mbar_init(drain, 1);
    ptx::mbar_init(ypart, 128);
    ptx::mbar_init(yfree, 128);
    if (YM) {
      for (int s = 0; s < RING; ++s) ptx::mbar_init(&ymma_done[s], 1);
      ptx::mbar_init(&yfull[0], 1);
      ptx::mbar_init(&yfull[1], 1);
      ptx::mbar_init(ydrain, 1);
    }
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tm_vhi);
    ptx::prefetch_tmap(&tm_vlo);
    ptx::prefetch_tmap(&tm_phi);
    ptx::prefetch_tmap(&tm_plo);
    ptx::prefetch_tmap(&tm_ohi);
    ptx::prefetch_tmap(&tm_olo);
    if (YM) {
      ptx::prefetch_tmap(&ym.chi);
      ptx::prefetch_tmap(&ym.clo);
      ptx::prefetch_tmap(&ym.uhi);
      ptx::prefetch_tmap(&ym.ulo);
      ptx::prefetch_tmap(&ym.dhi);
      ptx::prefetch_tmap(&ym.dlo);
    }
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const unsigned long long limit = args.timeout_ns;
  // The next launch of the stream (launched as a programmatic dependent) may
  // start its prologue on SMs this grid leaves free; it waits for this grid's
  // completion before it touches the states.
  ptx::griddep_launch_dependents();

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued_parity[8];
      for (int s = 0; s < 8; ++s) issued_parity[s] = -1;
      bool waited = false;
      for (int w = first_item<YM>(args); w < nwork && !*abort_flag; w = next_item<YM>(args, w)) {
        const Item it = load_item<QMAX, YM>(args, w);
        if (it.copy) continue;                                   // no operands
        // source rows l - s (forward) or l + s (adjoint); may fall outside the
        // tensor (zero fill) or in a neighbouring sequence (zeroed below)
        const int src_row = (int)(it.t.seq_row0 + it.t.t0 + (args.reverse ? shift : -shift));
        // strided tiles: the same row as (row in group, group) of the 3-D map
        const int src_y = args.S ? src_row % args.S : src_row;
        const int src_z = args.S ? src_row / args.S : 0;
        const int prow = (it.t.sys * args.kmax1 + args.k) * m + it.n0;
        int c0 = 0;
        if (!waited) {
          // The powers do not depend on the previous launch: the first stages'
          // power chunks are requested before waiting for it, the state rows after.
          const int pre = min(S, nkc);
          int armed = 0;
          for (int c = 0; c < pre; ++c) {      // fresh stages: the empty waits pass at once
            if (!ptx::mbar_wait(&empty[c], 1u, limit, abort_flag)) {
              raise_timeout(args, abort_flag, 1, w, c);
              break;
            }
            uint8_t* sb_hi = bufs + (size_t)c * stage_bytes + 2 * a_bytes;
            ptx::mbar_arrive_expect_tx(&full[c], GEN == 1 ? 2 * b_bytes : stage_bytes);
            ptx::tma_load_2d(sb_hi, &tm_phi, &full[c], c * KC, prow);
            ptx::tma_load_2d(sb_hi + b_bytes, &tm_plo, &full[c], c * KC, prow);
            issued_parity[c] = 0;
            ++armed;
          }
          ptx::griddep_wait();
          waited = true;
          // every armed stage gets its state rows (its barrier expects them)
          for (int c = 0; c < armed && GEN != 1; ++c) {
            uint8_t* sa_hi = bufs + (size_t)c * stage_bytes;
            if (args.S) {
              ptx::tma_load_3d(sa_hi, &tm_vhi, &full[c], c * KC, src_y, src_z);
              ptx::tma_load_3d(sa_hi + a_bytes, &tm_vlo, &full[c], c * KC, src_y, src_z);
            } else {
              ptx::tma_load_2d(sa_hi, &tm_vhi, &full[c], c * KC, src_row);
              ptx::tma_load_2d(sa_hi + a_bytes, &tm_vlo, &full[c], c * KC, src_row);
            }
          }
          if (armed < pre) break;
          stage = pre;
          if (stage == S) { stage = 0; phase ^= 1u; }
          c0 = pre;
        }
        for (int c = c0; c < nkc; ++c) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, limit, abort_flag)) {
            raise_timeout(args, abort_flag, 1, w, stage);
            break;
          }
          uint8_t* sa_hi = bufs + (size_t)stage * stage_bytes;
          uint8_t* sa_lo = sa_hi + a_bytes;
          uint8_t* sb_hi = sa_lo + a_bytes;
          uint8_t* sb_lo = sb_hi + b_bytes;
          ptx::mbar_arrive_expect_tx(&full[stage], GEN == 1 ? 2 * b_bytes : stage_bytes);
          if (GEN == 1) {
            // the row warps write this stage's operand rows
          } else if (args.S) {
            ptx::tma_load_3d(sa_hi, &tm_vhi, &full[stage], c * KC, src_y, src_z);
            ptx::tma_load_3d(sa_lo, &tm_vlo, &full[stage], c * KC, src_y, src_z);
          } else {
            ptx::tma_load_2d(sa_hi, &tm_vhi, &full[stage], c * KC, src_row);
            ptx::tma_load_2d(sa_lo, &tm_vlo, &full[stage], c * KC, src_row);
          }
          ptx::tma_load_2d(sb_hi, &tm_phi, &full[stage], c * KC, prow);
          ptx::tma_load_2d(sb_lo, &tm_plo, &full[stage], c * KC, prow);
          issued_parity[stage] = (int)phase;
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
      if (!waited) ptx::griddep_wait();
      // Never leave the block with copies in flight.
      for (int s = 0; s < S; ++s)
        if (issued_parity[s] >= 0)
          ptx::mbar_wait(&full[s], (uint32_t)issued_parity[s], limit, nullptr);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = ptx::make_idesc(FMT, BM, BN);
    int stage = 0;
    uint32_t phase = 0;
    int acc_i = 0;
    for (int w = first_item<YM>(args); w < nwork && !*abort_flag; w = next_item<YM>(args, w)) {
      const Item it = load_item<QMAX, YM>(args, w);
      if (!it.acc) continue;
      const int abuf = acc_i & 1;
      const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
      // lane-uniform outcome: the warp leaves its loop as a whole
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&acc_empty[abuf], aph ^ 1u, limit, abort_flag))) {
        raise_timeout(args, abort_flag, 2, w, acc_i);
        break;
      }
      ptx::tc_fence_after();
      // tile rows [z0, z1) whose source lies outside the sequence read zero
      // (strided tiles: every source lies inside its sequence)
      const int z0 = args.reverse ? max(0, it.t.len - it.t.t0 - shift) : 0;
      const int z1 = args.S ? 0 : args.reverse ? BM : min(BM, shift - it.t.t0);
      const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * ACC);
      const uint32_t c_tmem = d_tmem + (SEP ? (uint32_t)BN : 0u);   // correction accumulator
      bool ok = true;
      // (YM: a fused copy item only takes the accumulator, for its y products)
      for (int c = 0; c < (it.copy ? 0 : nkc); ++c) {
        if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[stage], phase, limit, abort_flag))) {
          raise_timeout(args, abort_flag, 3, w, stage);
          ok = false;
          break;
        }
        uint8_t* sa_hi = bufs + (size_t)stage * stage_bytes;
        uint8_t* sa_lo = sa_hi + a_bytes;
        uint8_t* sb_hi = sa_lo + a_bytes;
        uint8_t* sb_lo = sb_hi + b_bytes;
        if (z1 > z0) {
          // row r occupies bytes [r * 64, r * 64 + 64) of each A buffer
          uint4* zh = reinterpret_cast<uint4*>(sa_hi);
          uint4* zl = reinterpret_cast<uint4*>(sa_lo);
          const uint4 z = make_uint4(0, 0, 0, 0);
          for (int i = z0 * 4 + lane; i < z1 * 4; i += 32) { zh[i] = z; zl[i] = z; }
          ptx::fence_proxy_async_smem();
          __syncwarp();
        }
        ptx::tc_fence_after();
        if (lane == 0) {
          const uint64_t dah = ptx::make_sdesc_sw64(ptx::smem_addr(sa_hi));
          const uint64_t dal = ptx::make_sdesc_sw64(ptx::smem_addr(sa_lo));
          const uint64_t dbh = ptx::make_sdesc_sw64(ptx::smem_addr(sb_hi));
          const uint64_t dbl = ptx::make_sdesc_sw64(ptx::smem_addr(sb_lo));
#pragma unroll
          for (int kk = 0; kk < KC / UK; ++kk) {
            const uint64_t adv = (uint64_t)((kk * UK * ELEM) >> 4);   // 32 bytes per step
            if (ELEM == 2) {
              ptx::mma_bf16(d_tmem, dah + adv, dbh + adv, idesc, (c | kk) != 0);
              ptx::mma_bf16(d_tmem, dah + adv, dbl + adv, idesc, 1u);
              ptx::mma_bf16(d_tmem, dal + adv, dbh + adv, idesc, 1u);
            } else {
              ptx::mma_tf32(d_tmem, dah + adv, dbh + adv, idesc, (c | kk) != 0);
              ptx::mma_tf32(c_tmem, dah + adv, dbl + adv, idesc, (c | kk) != 0);
              ptx::mma_tf32(c_tmem, dal + adv, dbh + adv, idesc, 1u);
            }
          }
          ptx::tc_commit(&empty[stage]);
        }
        __syncwarp();
        if (++stage == S) { stage = 0; phase ^= 1u; }
      }
      if (!ok) break;
      if (lane == 0) ptx::tc_commit(&acc_full[abuf]);
      __syncwarp();
      ++acc_i;
    }
    // Drain: every MMA this thread issued has completed before TMEM is freed.
    if (lane == 0) {
      ptx::tc_commit(drain);
      ptx::mbar_wait(drain, 0u, limit, nullptr);
    }
    __syncwarp();
  } else if (warp == 6) {
    // ------------------------------------------------------------ ring manager
    if (lane == 0) {
      ptx::griddep_wait();             // the residual rows are the previous launch's output
      int lw = first_item<YM>(args), lcc = 0;   // load cursor, RING chunks ahead of the epilogue
      uint32_t issued = 0;
      auto issue_next = [&](int slot) {
        if (lw >= nwork) return;
        const Item li = load_item<QMAX, YM>(args, lw);
        const Tile& lt = li.t;
        const int lnck = item_chunks<YM>(args, li, nch);
        const int x = li.n0 + lcc * CW;
        const int yrow = (int)(lt.seq_row0 + lt.t0);
        uint8_t* sh = ring + (size_t)slot * slot_bytes;
        if (YM && li.fused) {
          // the residual chunk and the matching K chunk of C, or a (u, D) chunk of
          // the D u term (K chunk j of u's p columns; past p, TMA fills zeros)
          const uint32_t cb = (uint32_t)q * ROWB;
          ptx::mbar_arrive_expect_tx(&res_full[slot], SLOT_BYTES + 2 * cb);
          const int crow = lt.sys * q;
          if (lcc < nch) {
            ptx::tma_load_2d(sh, &tm_vhi, &res_full[slot], x, yrow);
            ptx::tma_load_2d(sh + PLANE_TILE, &tm_vlo, &res_full[slot], x, yrow);
            ptx::tma_load_2d(sh + SLOT_BYTES, &ym.chi, &res_full[slot], x, crow);
            ptx::tma_load_2d(sh + SLOT_BYTES + cb, &ym.clo, &res_full[slot], x, crow);
          } else {
            const int ux = (lcc - nch) * 32;
            ptx::tma_load_2d(sh, &ym.uhi, &res_full[slot], ux, yrow);
            ptx::tma_load_2d(sh + PLANE_TILE, &ym.ulo, &res_full[slot], ux, yrow);
            ptx::tma_load_2d(sh + SLOT_BYTES, &ym.dhi, &res_full[slot], ux, crow);
            ptx::tma_load_2d(sh + SLOT_BYTES + cb, &ym.dlo, &res_full[slot], ux, crow);
          }
          ++issued;
          if (++lcc == lnck) { lcc = 0; lw = next_item<YM>(args, lw); }
          return;
        }
        if (GEN != 0) {
          ptx::mbar_arrive(&res_full[slot]);   // the epilogue forms the residual from u
        } else {
          ptx::mbar_arrive_expect_tx(&res_full[slot], SLOT_BYTES);
          if (args.S) {
            ptx::tma_load_3d(sh, &tm_vhi, &res_full[slot], x, yrow % args.S, yrow / args.S);
            ptx::tma_load_3d(sh + PLANE_TILE, &tm_vlo, &res_full[slot], x, yrow % args.S,
                             yrow / args.S);
          } else {
            ptx::tma_load_2d(sh, &tm_vhi, &res_full[slot], x, yrow);
            ptx::tma_load_2d(sh + PLANE_TILE, &tm_vlo, &res_full[slot], x, yrow);
          }
        }
        ++issued;
        if (++lcc == lnck) { lcc = 0; lw = next_item<YM>(args, lw); }
      };
      for (int s = 0; s < RING; ++s) issue_next(s);
      uint32_t g = 0;                  // chunks retired
      bool alive = true;
      // A slot is refilled one chunk after its store was issued, so that the
      // store of the newest chunk reads shared memory while the older one's
      // slot is reloaded (bulk wait with one group allowed in flight).
      int pend_slot = -1;
      for (int w = first_item<YM>(args); w < nwork && alive; w = next_item<YM>(args, w)) {
        const Item it = load_item<QMAX, YM>(args, w);
        const bool tma_out = (!it.fused || args.keep_v) && !it.ragged;
        const int ytile = (int)(it.t.seq_row0 + it.t.t0);
        const int nck = item_chunks<YM>(args, it, nch);
        for (int cc = 0; cc < nck; ++cc, ++g) {
          const int slot = (int)(g % RING);
          uint8_t* sh = ring + (size_t)slot * slot_bytes;
          // Every chunk passes through both barriers of its slot, also a pure
          // copy that the epilogue forwards untouched: a parity wait is then
          // never more than one phase ahead of the barrier it polls.  With YM
          // every chunk also passes the y issuer's release of the slot.
          if (!ptx::mbar_wait(&res_done[slot], (g / RING) & 1u, limit, abort_flag)) {
            raise_timeout(args, abort_flag, 5, w, (int)g);
            alive = false;
            break;
          }
          if (YM && !ptx::mbar_wait(&ymma_done[slot], (g / RING) & 1u, limit, abort_flag)) {
            raise_timeout(args, abort_flag, 14, w, (int)g);
            alive = false;
            break;
          }
          if (tma_out && cc < nch) {
            if (args.S) {
              ptx::tma_store_3d(&tm_ohi, sh, it.n0 + cc * CW, ytile % args.S, ytile / args.S);
              ptx::tma_store_3d(&tm_olo, sh + PLANE_TILE, it.n0 + cc * CW, ytile % args.S,
                                ytile / args.S);
            } else {
              ptx::tma_store_2d(&tm_ohi, sh, it.n0 + cc * CW, ytile);
              ptx::tma_store_2d(&tm_olo, sh + PLANE_TILE, it.n0 + cc * CW, ytile);
            }
            ptx::bulk_commit();
          }
          if (pend_slot >= 0) {
            // the previous chunk's store (if any) has read its slot: all bulk
            // groups but this chunk's (the newest, when it stored) are done reading
            if (tma_out && cc < nch) ptx::bulk_wait_read1();
            else ptx::bulk_wait_read0();
            issue_next(pend_slot);
          }
          pend_slot = slot;
        }
      }
      ptx::bulk_wait0();                // stores complete before the block exits
      // loads issued but not retired (only after an abort): let them land
      for (uint32_t h = g; h < issued; ++h)
        ptx::mbar_wait(&res_full[h % RING], (h / RING) & 1u, limit, nullptr);
    }
  } else if (YM && warp == NTHREADS / 32) {
    // ------------------------------------------------------------ y issuer (YM)
    // y = C v + D u of fused tiles: per staged chunk (A: the state chunk, or u;
    // B: the K chunk of C, or D, in the same slot) three BF16 products into TMEM
    // columns [0, q) of the tile's accumulator; the slot is released by a commit.
    // Chunks of other tiles pass through (plain arrive), so the release barrier
    // stays phase-locked with the slot.
    if (lane == 0) {
      const uint32_t idesc_y = ptx::make_idesc(FMT, BM, q);
      const int nq = min(nch, (q + CW - 1) / CW);   // chunks covering columns [0, q)
      const uint32_t cb = (uint32_t)q * ROWB;
      uint32_t g = 0;
      int acc_i = 0;
      bool alive = true;
      for (int w = first_item<YM>(args); w < nwork && alive; w = next_item<YM>(args, w)) {
        const Item it = load_item<QMAX, YM>(args, w);
        const int nck = item_chunks<YM>(args, it, nch);
        if (!it.fused) {
          for (int cc = 0; cc < nck; ++cc, ++g) {
            const int slot = (int)(g % RING);
            if (!ptx::mbar_wait(&res_done[slot], (g / RING) & 1u, limit, abort_flag)) {
              raise_timeout(args, abort_flag, 17, w, (int)g);
              alive = false;
              break;
            }
            ptx::mbar_arrive(&ymma_done[slot]);
          }
          if (it.acc) ++acc_i;
          continue;
        }
        const int abuf = acc_i & 1;
        const uint32_t ycol = tmem_base + (uint32_t)(abuf * ACC);
        // columns [0, q) are free once the epilogue has read chunks 0 .. nq - 1
        for (int h = 0; h < nq && alive; ++h) {
          const uint32_t gh = g + (uint32_t)h;
          if (!ptx::mbar_wait(&res_done[gh % RING], (gh / RING) & 1u, limit, abort_flag)) {
            raise_timeout(args, abort_flag, 13, w, (int)gh);
            alive = false;
          }
        }
        if (!alive) break;
        for (int cc = 0; cc < nck; ++cc, ++g) {
          const int slot = (int)(g % RING);
          if (cc >= nq && !ptx::mbar_wait(&res_done[slot], (g / RING) & 1u, limit, abort_flag)) {
            raise_timeout(args, abort_flag, 13, w, (int)g);
            alive = false;
            break;
          }
          ptx::tc_fence_after();
          uint8_t* sh = ring + (size_t)slot * slot_bytes;
          const uint64_t dah = ptx::make_sdesc_sw64(ptx::smem_addr(sh));
          const uint64_t dal = ptx::make_sdesc_sw64(ptx::smem_addr(sh + PLANE_TILE));
          const uint64_t dbh = ptx::make_sdesc_sw64(ptx::smem_addr(sh + SLOT_BYTES));
          const uint64_t dbl = ptx::make_sdesc_sw64(ptx::smem_addr(sh + SLOT_BYTES + cb));
#pragma unroll
          for (int kk = 0; kk < KC / UK; ++kk) {
            const uint64_t adv = (uint64_t)((kk * UK * ELEM) >> 4);
            ptx::mma_bf16(ycol, dah + adv, dbh + adv, idesc_y, (cc | kk) != 0);
            ptx::mma_bf16(ycol, dah + adv, dbl + adv, idesc_y, 1u);
            ptx::mma_bf16(ycol, dal + adv, dbh + adv, idesc_y, 1u);
          }
          ptx::tc_commit(&ymma_done[slot]);
        }
        if (!alive) break;
        ptx::tc_commit(&yfull[abuf]);
        ++acc_i;
      }
      // every product issued here has completed before TMEM is freed
      ptx::tc_commit(ydrain);
      ptx::mbar_wait(ydrain, 0u, limit, nullptr);
    }
    __syncwarp();
  } else if (GEN == 1 && warp >= NTHREADS / 32) {
    // ------------------------------------------------------------ first-stage rows
    // Operand rows v^(1)_(l-s) = Bbar u_(l-s) + Abar Bbar u_(l-s-1) of each K
    // chunk, written in the swizzled layout the TMA copy would give (zero where
    // the source precedes the sequence).  One thread per tile row; thread 0
    // waits for the stage and the others follow it through named barrier 1.
    const int r = threadIdx.x - NTHREADS;
    volatile int* gen_ok = reinterpret_cast<volatile int*>(tmem_slot + 2);
    ptx::griddep_wait();
    int stage = 0;
    uint32_t phase = 0;
    for (int w = first_item<YM>(args); w < nwork; w = next_item<YM>(args, w)) {
      const Item it = load_item<QMAX, YM>(args, w);
      if (it.copy) continue;
      const int src = it.t.t0 + r - shift;
      const bool live = it.t.t0 + r < it.t.len && src >= 0;
      float x1[4] = {0.f, 0.f, 0.f, 0.f}, x0[4] = {0.f, 0.f, 0.f, 0.f};
      if (live) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j < args.p) {
            x1[j] = __ldg(args.u + (it.t.seq_row0 + src) * args.p + j);
            if (src >= 1) x0[j] = __ldg(args.u + (it.t.seq_row0 + src - 1) * args.p + j);
          }
      }
      const float* Bs = args.Bb + (int64_t)it.t.sys * m * args.p;
      const float* ABs = args.ABb + (int64_t)it.t.sys * m * args.p;
      bool ok = true;
      for (int c = 0; c < nkc; ++c) {
        if (r == 0) *gen_ok = ptx::mbar_wait(&empty[stage], phase ^ 1u, limit, abort_flag) ? 1 : 0;
        ptx::named_bar_sync(1, GEN_THREADS);
        if (!*gen_ok) {
          if (r == 0) raise_timeout(args, abort_flag, 12, w, stage);
          ok = false;
          break;
        }
        float x[KC];
#pragma unroll
        for (int e = 0; e < KC; ++e) x[e] = 0.f;
        if (live) add_first_stage<KC>(Bs, ABs, args.p, c * KC, x1, x0, x);
        uint8_t* sa_hi = bufs + (size_t)stage * stage_bytes;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          uint4 hv, lv;
          Fmt<ELEM>::split16(x + q4 * (KC / 4), hv, lv);
          *reinterpret_cast<uint4*>(sa_hi + ptx::sw64_offset(r, q4)) = hv;
          *reinterpret_cast<uint4*>(sa_hi + a_bytes + ptx::sw64_offset(r, q4)) = lv;
        }
        ptx::fence_proxy_async_smem();          // visible to the tensor core's reads
        ptx::named_bar_sync(1, GEN_THREADS);
        if (r == 0) ptx::mbar_arrive(&full[stage]);
        if (++stage == S) { stage = 0; phase ^= 1u; }
      }
      if (!ok) break;
    }
  } else {
    // ------------------------------------------------------------ epilogue
    ptx::griddep_wait();                       // before any store to the states or y
    const int quad = warp & 3;                 // TMEM lane quadrant this warp may access
    const int r = quad * 32 + lane;            // tile row == TMEM lane
    // Two epilogue groups share the tiles: chunk g (counted over the whole
    // launch) belongs to group (g / G) % 2, so with ring % (2 G) == 0 every ring
    // slot is always served by the same group and a parity wait never runs two
    // phases ahead; each chunk still gets 128 arrivals on res_done.  For tiles
    // that form y, group 1 hands its partial sums to group 0 through ysum.
    const int egrp = warp >= 7 ? 1 : 0;
    uint32_t g = 0;                            // chunks consumed (by either group)
    int nfused = 0;                            // fused tiles seen (ypart / yfree phases)
    int acc_i = 0;
    int ycnt[2] = {0, 0};                      // (YM) fused tiles seen per accumulator
    bool alive = true;                         // warp-uniform
    for (int w = first_item<YM>(args); w < nwork && alive; w = next_item<YM>(args, w)) {
      const Item it = load_item<QMAX, YM>(args, w);
      const bool tma_out = (!it.fused || args.keep_v) && !it.ragged;
      const int tr = it.t.t0 + r;
      const bool valid = tr < it.t.len;
      const int64_t grow = args.S ? it.t.seq_row0 + (int64_t)r * args.S : it.t.seq_row0 + tr;
      const int abuf = acc_i & 1;
      float ur[4] = {0.f, 0.f, 0.f, 0.f}, ur1[4] = {0.f, 0.f, 0.f, 0.f};   // u_l, u_(l-1)
      const float* Bs = nullptr;
      const float* ABs = nullptr;
      if constexpr (GEN != 0) {
        Bs = args.Bb + (int64_t)it.t.sys * m * args.p;
        ABs = args.ABb + (int64_t)it.t.sys * m * args.p;
        if (valid) {
          // GEN = 2: an even row of the work-efficient schedule, v^(1) = Bbar u_l
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j < args.p) {
              ur[j] = __ldg(args.u + grow * args.p + j);
              if (GEN == 1 && tr >= 1) ur1[j] = __ldg(args.u + (grow - 1) * args.p + j);
            }
        }
      }
      if (it.copy && tma_out && !it.fused) {
        // the manager forwards the residual as is; acknowledge each chunk once
        // it has arrived, keeping both slot barriers phase-locked
        for (int cc = 0; cc < nch; ++cc, ++g) {
          if (((g / G) & 1) != (uint32_t)egrp) continue;
          const int slot = (int)(g % RING);
          if (!__all_sync(0xffffffffu,
                          ptx::mbar_wait(&res_full[slot], (g / RING) & 1u, limit, abort_flag))) {
            raise_timeout(args, abort_flag, 8, w, (int)g);
            alive = false;
            break;
          }
          ptx::mbar_arrive(&res_done[slot]);
        }
        continue;
      }
      if (it.acc) {
        const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
        if (!__all_sync(0xffffffffu, ptx::mbar_wait(&acc_full[abuf], aph, limit, abort_flag))) {
          raise_timeout(args, abort_flag, 6, w, acc_i);
          break;
        }
        ptx::tc_fence_after();
      }

      float yacc[QN];
#pragma unroll
      for (int qq = 0; qq < QN; ++qq) yacc[qq] = 0.f;
      const float* Cs = args.C32 + (int64_t)it.t.sys * args.q * m;
      const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(abuf * ACC);
      // G chunks per step (nch is always even): their TMEM loads, unpacking,
      // splitting and shared-memory traffic are independent.
      for (int cc = 0; cc < nch; cc += G, g += G) {
        if (((g / G) & 1) != (uint32_t)egrp) continue;   // the other group's step
        int slot[G];
        uint8_t* sh[G];
        bool got = true;
#pragma unroll
        for (int h = 0; h < G; ++h) {
          slot[h] = (int)((g + h) % RING);
          sh[h] = ring + (size_t)slot[h] * slot_bytes;
          got = got && ptx::mbar_wait(&res_full[slot[h]], ((g + h) / RING) & 1u, limit, abort_flag);
        }
        if (!__all_sync(0xffffffffu, got)) {     // tcgen05.ld below is warp-collective
          raise_timeout(args, abort_flag, 7, w, (int)g);
          alive = false;
          break;
        }
        if (YM && it.copy && it.fused) {
          // every source precedes the sequence: the slot already holds the final
          // (hi, lo) state, which is the y products' A operand as it stands
#pragma unroll
          for (int h = 0; h < G; ++h) ptx::mbar_arrive(&res_done[slot[h]]);
          continue;
        }
        // GEN = 2 (p = 1): the even rows' residual Bbar u_l, formed before the
        // TMEM load it does not depend on, so its coefficient loads overlap it
        float xr[GEN == 2 ? G : 1][GEN == 2 ? CW : 1];
        if constexpr (GEN == 2) {
#pragma unroll
          for (int h = 0; h < G; ++h) {
            const float4* b4 = reinterpret_cast<const float4*>(Bs + it.n0 + (cc + h) * CW);
#pragma unroll
            for (int e4 = 0; e4 < CW / 4; ++e4) {
              const float4 b = valid ? __ldg(b4 + e4) : make_float4(0.f, 0.f, 0.f, 0.f);
              xr[h][4 * e4] = b.x * ur[0];
              xr[h][4 * e4 + 1] = b.y * ur[0];
              xr[h][4 * e4 + 2] = b.z * ur[0];
              xr[h][4 * e4 + 3] = b.w * ur[0];
            }
          }
        }
        float v[G][CW];
        if (!it.copy) {
          uint32_t ra[G][CW];
#pragma unroll
          for (int h = 0; h < G; ++h) ptx::tmem_ld_nw<CW>(trow + (uint32_t)((cc + h) * CW), ra[h]);
          if (SEP) {
            uint32_t rb[G][CW];
#pragma unroll
            for (int h = 0; h < G; ++h)
              ptx::tmem_ld_nw<CW>(trow + (uint32_t)(BN + (cc + h) * CW), rb[h]);
            ptx::tmem_wait_ld();
#pragma unroll
            for (int h = 0; h < G; ++h)
#pragma unroll
              for (int j = 0; j < CW; ++j)
                v[h][j] = __uint_as_float(ra[h][j]) + __uint_as_float(rb[h][j]);
          } else {
            ptx::tmem_wait_ld();
#pragma unroll
            for (int h = 0; h < G; ++h)
#pragma unroll
              for (int j = 0; j < CW; ++j) v[h][j] = __uint_as_float(ra[h][j]);
          }
        } else {
#pragma unroll
          for (int h = 0; h < G; ++h)
#pragma unroll
            for (int j = 0; j < CW; ++j) v[h][j] = 0.f;
        }
        uint4 hq[G][4], lq[G][4];
        if constexpr (GEN == 2) {
          // rounded to the (hi, lo) pair the first level would have stored
#pragma unroll
          for (int h = 0; h < G; ++h)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              Fmt<ELEM>::split16(xr[h] + c * (CW / 4), hq[h][c], lq[h][c]);
              Fmt<ELEM>::add16(hq[h][c], lq[h][c], v[h] + c * (CW / 4));
            }
        } else if constexpr (GEN == 1) {
          // residual v^(1)_l of this row from u, rounded to the (hi, lo) pair the
          // first-stage kernel would have stored, so that results are the same
          // bit for bit (rows past the sequence end are not stored: zero)
#pragma unroll
          for (int h = 0; h < G; ++h)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float x[CW / 4];
#pragma unroll
              for (int e = 0; e < CW / 4; ++e) x[e] = 0.f;
              if (valid)
                add_first_stage<CW / 4>(Bs, ABs, args.p, it.n0 + (cc + h) * CW + c * (CW / 4), ur,
                                        ur1, x);
              Fmt<ELEM>::split16(x, hq[h][c], lq[h][c]);
              Fmt<ELEM>::add16(hq[h][c], lq[h][c], v[h] + c * (CW / 4));
            }
        } else {
#pragma unroll
          for (int h = 0; h < G; ++h)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              hq[h][c] = *reinterpret_cast<const uint4*>(sh[h] + ptx::sw64_offset(r, c));
              lq[h][c] =
                  *reinterpret_cast<const uint4*>(sh[h] + PLANE_TILE + ptx::sw64_offset(r, c));
            }
#pragma unroll
          for (int h = 0; h < G; ++h)
#pragma unroll
            for (int c = 0; c < 4; ++c) Fmt<ELEM>::add16(hq[h][c], lq[h][c], v[h] + c * (CW / 4));
        }
        if (QMAX > 0 && it.fused) {
          if (valid) {
#pragma unroll
            for (int qq = 0; qq < QN; ++qq) {
              if (qq < args.q) {
                // C row segment as 16-byte loads (m, n0 and CW are multiples of 4)
                const float4* crow =
                    reinterpret_cast<const float4*>(Cs + (int64_t)qq * m + it.n0 + cc * CW);
                float s = 0.f;
#pragma unroll
                for (int h = 0; h < G; ++h)
#pragma unroll
                  for (int j4 = 0; j4 < CW / 4; ++j4) {
                    const float4 c4 = __ldg(crow + h * (CW / 4) + j4);
                    s = fmaf(c4.x, v[h][4 * j4], s);
                    s = fmaf(c4.y, v[h][4 * j4 + 1], s);
                    s = fmaf(c4.z, v[h][4 * j4 + 2], s);
                    s = fmaf(c4.w, v[h][4 * j4 + 3], s);
                  }
                yacc[qq] += s;
              }
            }
          }
        }
        if (!it.fused || args.keep_v || YM) {
#pragma unroll
          for (int h = 0; h < G; ++h)
#pragma unroll
            for (int c = 0; c < 4; ++c) Fmt<ELEM>::split16(v[h] + c * (CW / 4), hq[h][c], lq[h][c]);
          // (YM: a fused tile's finished chunk is the A operand of its y products)
          if (tma_out || (YM && it.fused)) {
#pragma unroll
            for (int h = 0; h < G; ++h)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                *reinterpret_cast<uint4*>(sh[h] + ptx::sw64_offset(r, c)) = hq[h][c];
                *reinterpret_cast<uint4*>(sh[h] + PLANE_TILE + ptx::sw64_offset(r, c)) = lq[h][c];
              }
            ptx::fence_proxy_async_smem();      // visible to the TMA store and the MMA
          }
          if (!tma_out && valid && (!it.fused || args.keep_v)) {
#pragma unroll
            for (int h = 0; h < G; ++h) {
              const int64_t off = (grow * (int64_t)m + it.n0 + (cc + h) * CW) * ELEM;
              uint4* gh = reinterpret_cast<uint4*>(static_cast<uint8_t*>(args.vout_hi) + off);
              uint4* gl = reinterpret_cast<uint4*>(static_cast<uint8_t*>(args.vout_lo) + off);
#pragma unroll
              for (int c = 0; c < 4; ++c) { gh[c] = hq[h][c]; gl[c] = lq[h][c]; }
            }
          }
        }
        // (YM: the y issuer's products write TMEM columns this chunk's loads read)
        if (YM && it.fused) ptx::tc_fence_before();
#pragma unroll
        for (int h = 0; h < G; ++h) ptx::mbar_arrive(&res_done[slot[h]]);
      }
      if (!alive) break;
      if (YM && it.fused) {
        // the (u, D) chunks of the first column block go to the y issuer as they
        // are; each passes both slot barriers like any other chunk
        const int nck = item_chunks<YM>(args, it, nch);
        for (int cc = nch; cc < nck; ++cc, ++g) {
          if (((g / G) & 1) != (uint32_t)egrp) continue;
          const int slot = (int)(g % RING);
          if (!__all_sync(0xffffffffu,
                          ptx::mbar_wait(&res_full[slot], (g / RING) & 1u, limit, abort_flag))) {
            raise_timeout(args, abort_flag, 15, w, (int)g);
            alive = false;
            break;
          }
          ptx::mbar_arrive(&res_done[slot]);
        }
        if (!alive) break;
        if (egrp == 0) {
          // y of this column block from TMEM columns [0, q) of the tile's
          // accumulator; summed over the column blocks in order, plus D u (in
          // the first block's products), and stored by the last block
          // yfull[b] completes once per fused tile that used accumulator b
          const uint32_t yph = (uint32_t)(ycnt[abuf]++ & 1);
          if (!__all_sync(0xffffffffu, ptx::mbar_wait(&yfull[abuf], yph, limit, abort_flag))) {
            raise_timeout(args, abort_flag, 16, w, acc_i);
            break;
          }
          ptx::tc_fence_after();
          // (the partial sums of earlier column blocks wait in this thread's own
          // row of y: it wrote them, so it reads them back in program order)
          const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(abuf * ACC);
          // tcgen05.ld is warp-collective: every lane loads, rows past the
          // sequence end only skip the memory accesses
          for (int j0 = 0; j0 < q; j0 += 16) {
            float t[16];
            ptx::tmem_ld16(trow + (uint32_t)j0, t);
            if (!valid) continue;
            float4* yo = reinterpret_cast<float4*>(args.y + grow * q + j0);
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4) {
              if (it.nb > 0) {
                const float4 o = yo[e4];
                t[4 * e4] = o.x + t[4 * e4];
                t[4 * e4 + 1] = o.y + t[4 * e4 + 1];
                t[4 * e4 + 2] = o.z + t[4 * e4 + 2];
                t[4 * e4 + 3] = o.w + t[4 * e4 + 3];
              }
              yo[e4] = make_float4(t[4 * e4], t[4 * e4 + 1], t[4 * e4 + 2], t[4 * e4 + 3]);
            }
          }
        }
      }
      if (it.acc) {
        ptx::tc_fence_before();
        ptx::mbar_arrive(&acc_empty[abuf]);
        ++acc_i;
      }
      if (QMAX > 0 && it.fused) {
        // y sums over all columns: group 1 hands its partial sums to group 0
        const uint32_t fph = (uint32_t)(nfused & 1);
        ++nfused;
        if (egrp == 1) {
          if (nfused > 1 &&
              !__all_sync(0xffffffffu, ptx::mbar_wait(yfree, fph ^ 1u, limit, abort_flag))) {
            raise_timeout(args, abort_flag, 9, w, nfused);
            break;
          }
#pragma unroll
          for (int qq = 0; qq < QN; ++qq) ysum[qq * 128 + r] = yacc[qq];
          ptx::mbar_arrive(ypart);
          continue;
        }
        if (!__all_sync(0xffffffffu, ptx::mbar_wait(ypart, fph, limit, abort_flag))) {
          raise_timeout(args, abort_flag, 10, w, nfused);
          break;
        }
#pragma unroll
        for (int qq = 0; qq < QN; ++qq) yacc[qq] += ysum[qq * 128 + r];
        ptx::mbar_arrive(yfree);
      }
      if (QMAX > 0 && it.fused && valid) {
        const float* Ds = args.D32 + (int64_t)it.t.sys * args.q * args.p;
        const float* ur = args.u + grow * args.p;
#pragma unroll
        for (int qq = 0; qq < QN; ++qq) {
          if (qq < args.q) {
            float s = yacc[qq];
            for (int j = 0; j < args.p; ++j) s = fmaf(__ldg(Ds + qq * args.p + j), __ldg(ur + j), s);
            args.y[grow * args.q + qq] = s;
          }
        }
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem_base, tmem_cols);
}

template <int ELEM, int QMAX, int G, int GEN, int YM = 0>
cudaError_t launch_variant(const CUtensorMap* maps, const YMaps& ym, const StageArgs& a, int grid,
                           size_t smem, cudaStream_t st) {
  auto kern = stage_tc_kernel<ELEM, QMAX, G, GEN, YM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // programmatic dependent launch: the prologue (barriers, TMEM, the first
  // power chunks) overlaps the previous launch's tail on the SMs it leaves free
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(GEN == 1 ? NTHREADS + GEN_THREADS : YM ? NTHREADS + 32 : NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], ym, a);
  CASCADE_LAUNCHED();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

size_t stage_bytes_for(int BN) { return 2 * (size_t)PLANE_TILE + 2 * (size_t)BN * ROWB; }

// Shared memory besides the operand stages: alignment slack, the staging ring,
// the mbarriers (room for RING_MAX ring barriers of each kind), the TMEM slot and,
// when one tile spans all m columns (the output may be formed in the epilogue),
// the partial y sums.
// ym_q > 0 (output on the tensor cores): slots also carry a K chunk of C or D
// (q rows, both planes).
size_t fixed_smem_bytes(int S, int ring, bool ysum, int ym_q = 0) {
  const size_t slot = SLOT_BYTES + (ym_q > 0 ? 2 * (size_t)ym_q * ROWB : 0);
  return 1024 + (size_t)ring * slot + 8 * (2 * S + 10 + 3 * RING_MAX) + 16 +
         (ysum ? sizeof(float) * 4 * 128 : 0);
}

bool tc_config_fits(int m, int BN, const TcConfig& c, int ym_q = 0) {
  if (c.group != 1 && c.group != 2) return false;
  if (ym_q > 0 && c.group != 1) return false;
  // the y issuer waits for the chunks covering TMEM columns [0, q) before it
  // releases the first of them, and a slot is refilled one chunk after the
  // next one is retired: the ring needs one slot more than those chunks
  if (ym_q > 0 && c.ring < (ym_q + 31) / 32 + 1) return false;
  // each ring slot always serves the same epilogue group: ring % (2 group) == 0
  if (c.ring < 2 * c.group || c.ring > RING_MAX || c.ring % (2 * c.group) != 0) return false;
  if (c.stages < 2 || c.stages > 8) return false;
  return fixed_smem_bytes(c.stages, c.ring, BN >= m, ym_q) +
             (size_t)c.stages * stage_bytes_for(BN) <=
         227 * 1024;
}

}  // namespace

// Candidate kernel shapes for the autotuner: for each (chunks per step, ring
// slots), the deepest operand pipeline that fits.
std::vector<TcConfig> tc_candidates(int m, int precision) {
  const int BN = block_n(m, precision);
  std::vector<TcConfig> out;
  for (int g : {1, 2})
    for (int ring : {2, 4, 6, 8})
      for (int st = 6; st >= 2; --st) {
        TcConfig c{st, ring, g};
        if (tc_config_fits(m, BN, c)) { out.push_back(c); break; }
      }
  return out;
}

// Shape used when no tuning was done: one chunk per step, a 4-slot ring,
// the deepest operand pipeline (at most 4) that fits.
TcConfig tc_default(int m, int precision) {
  const int BN = block_n(m, precision);
  TcConfig c{4, 4, 1};
  while (c.stages > 2 && !tc_config_fits(m, BN, c)) --c.stages;
  return c;
}

namespace {

// One launch of the stage kernel over `tiles` (stage k).  S = 0: dense tiles,
// 2-D state maps; S > 0: strided in-place tiles (vin == vout), 3-D state maps
// over `rows_cap` rows (a multiple of S).  even_resid: the destination rows'
// residual is v^(1) = Bbar u of an even row, formed from u (the last
// down-sweep level), and only y is written.
cudaError_t stage_tc_core(const Plan& p, int k, const Tile* tiles, int ntiles, int S,
                          uint64_t rows_cap, const void* vin_hi, const void* vin_lo,
                          void* vout_hi, void* vout_lo, const float* u, float* y,
                          cudaStream_t st, bool reverse, bool even_resid = false,
                          int shape_key = -1, const void* u_hi = nullptr,
                          const void* u_lo = nullptr) {
  if (ntiles == 0) return cudaSuccess;
  if (!(reverse ? p.PThi : p.Phi) || !vin_hi || !vin_lo || !vout_hi || !vout_lo) {
    set_global_error("stage launch without its power or state planes");
    return cudaErrorInvalidValue;
  }
  const int m = p.d.m;
  const int elem = (int)plane_elem_bytes(p.d.precision);
  const int BN = block_n(m, p.d.precision);
  TcConfig cfg{p.tc_stages, p.tc_ring, p.tc_group};
  if (!tc_config_fits(m, BN, cfg)) cfg = tc_default(m, p.d.precision);
  // the autotuner's shape for this stage (§3: key k) or scan level (shape_key)
  const int key = S == 0 ? k : shape_key;
  if (!reverse && key >= 0 && key < (int)p.tc_stage_shape.size() &&
      p.tc_stage_shape[key][0] > 0) {
    const TcConfig ck{p.tc_stage_shape[key][0], p.tc_stage_shape[key][1],
                      p.tc_stage_shape[key][2]};
    if (tc_config_fits(m, BN, ck)) cfg = ck;
  }
  const uint32_t row_elems = ROWB / (uint32_t)elem;
  CUtensorMap maps[6];
  std::string err;
  const uint64_t prow = (uint64_t)p.d.nsys * p.kmax1 * m;
  auto state_map = [&](CUtensorMap* map, const void* base) {
    return S ? encode_tmap_3d(map, base, elem, m, (uint64_t)S, rows_cap / (uint64_t)S, row_elems,
                              BM, &err, 64)
             : encode_tmap_2d(map, base, elem, m, rows_cap, row_elems, BM, &err, 64);
  };
  if (!state_map(&maps[0], vin_hi) || !state_map(&maps[1], vin_lo) ||
      !encode_tmap_2d(&maps[2], reverse ? p.PThi : p.Phi, elem, m, prow, row_elems, BN, &err, 64) ||
      !encode_tmap_2d(&maps[3], reverse ? p.PTlo : p.Plo, elem, m, prow, row_elems, BN, &err, 64) ||
      !state_map(&maps[4], vout_hi) || !state_map(&maps[5], vout_lo)) {
    set_global_error("tensor map encode failed: " + err);
    return cudaErrorInvalidValue;
  }
  StageArgs a{};
  a.tiles = tiles;
  a.ntiles = ntiles;
  a.nblocks = m / BN;
  a.m = m;
  a.p = p.d.p;
  a.q = p.d.q;
  a.BN = BN;
  a.stages = cfg.stages;
  a.ring = cfg.ring;
  a.shift = 1 << k;
  a.reverse = reverse ? 1 : 0;
  a.k = k;
  a.kmax1 = p.kmax1;
  // fused tiles also write v when the backward reads it, and in the strided
  // schedule, where a row finished at down-sweep level k is a source below it
  a.keep_v = ((p.d.flags & (CASCADE_FLAG_SAVE_STATES | CASCADE_FLAG_RECOMPUTE)) || S > 0) ? 1 : 0;
  a.S = S;
  a.vin_hi = vin_hi;
  a.vin_lo = vin_lo;
  a.vout_hi = vout_hi;
  a.vout_lo = vout_lo;
  a.C32 = p.C32;
  a.D32 = p.D32;
  a.u = u;
  a.y = y;
  // stage 1 of a plan that forms v^(1) on chip (one column chunk per step:
  // the row warps' registers fit only that variant), or the last down-sweep
  // level forming its even rows' v^(1) (also one chunk per step: fewer
  // kernel variants)
  const bool fuse = p.fuse_output && !reverse && y != nullptr;
  // the output on the tensor cores (BF16 pairs, §3 schedule; u as (hi, lo)
  // planes), for the stages that are some sequence's last
  const bool ym = p.fuse_output_mma && !reverse && y != nullptr && S == 0 && k >= 0 &&
                  k < (int)p.stage_fused.size() && p.stage_fused[k];
  if (ym && (!u_hi || !u_lo || elem != 2 || !p.pc_hi)) {
    set_global_error("fused tensor-core output without its u or coefficient planes");
    return cudaErrorInvalidValue;
  }
  const int gen = (p.fuse_first && k == 1 && !reverse && S == 0 && u != nullptr) ? 1
                  : (even_resid && fuse && S > 0 && u != nullptr)               ? 2
                                                                               : 0;
  a.gen = gen;
  a.Bb = p.Bbar32;
  a.ABb = p.ABbar32;
  if (gen == 2) a.keep_v = 0;   // nothing reads these rows after the last level
  if (gen != 0 && cfg.group != 1) {
    const TcConfig c1{cfg.stages, cfg.ring, 1};
    cfg = tc_config_fits(m, BN, c1) ? c1 : tc_default(m, p.d.precision);
    a.stages = cfg.stages;
    a.ring = cfg.ring;
  }
  const int q = p.d.q;
  YMaps ymaps;
  memset(&ymaps, 0, sizeof(ymaps));
  if (ym) {
    // one chunk per step, and slots that also hold a K chunk of C or D: the
    // deepest shape at or below the chosen one that fits, with a slot more than
    // the chunks covering columns [0, q) that the y issuer waits for at once
    const int need = ((q + 31) / 32 + 2) & ~1;
    TcConfig c1{cfg.stages, std::max(cfg.ring, need), 1};
    while (!tc_config_fits(m, BN, c1, q) && c1.stages > 2) --c1.stages;
    while (!tc_config_fits(m, BN, c1, q) && c1.ring > need) c1.ring -= 2;
    if (!tc_config_fits(m, BN, c1, q)) {
      set_global_error("fused tensor-core output does not fit shared memory");
      return cudaErrorInvalidValue;
    }
    cfg = c1;
    a.stages = cfg.stages;
    a.ring = cfg.ring;
    const auto* ch = static_cast<const __nv_bfloat16*>(p.pc_hi) + p.pc_off[PC_C];
    const auto* cl = static_cast<const __nv_bfloat16*>(p.pc_lo) + p.pc_off[PC_C];
    const auto* dh = static_cast<const __nv_bfloat16*>(p.pc_hi) + p.pc_off[PC_D];
    const auto* dl = static_cast<const __nv_bfloat16*>(p.pc_lo) + p.pc_off[PC_D];
    const uint64_t crows = (uint64_t)p.d.nsys * q;
    if (!encode_tmap_2d(&ymaps.chi, ch, 2, m, crows, 32, q, &err, 64) ||
        !encode_tmap_2d(&ymaps.clo, cl, 2, m, crows, 32, q, &err, 64) ||
        !encode_tmap_2d(&ymaps.dhi, dh, 2, p.d.p, crows, 32, q, &err, 64) ||
        !encode_tmap_2d(&ymaps.dlo, dl, 2, p.d.p, crows, 32, q, &err, 64) ||
        !encode_tmap_2d(&ymaps.uhi, u_hi, 2, p.d.p, (uint64_t)p.rows, 32, BM, &err, 64) ||
        !encode_tmap_2d(&ymaps.ulo, u_lo, 2, p.d.p, (uint64_t)p.rows, 32, BM, &err, 64)) {
      set_global_error("tensor map encode failed: " + err);
      return cudaErrorInvalidValue;
    }
  }
  a.err = p.err;
  a.diag = p.err + 1;
  a.timeout_ns = 2000000000ull;
  const size_t smem = fixed_smem_bytes(a.stages, a.ring, BN >= m, ym ? q : 0) +
                      (size_t)a.stages * stage_bytes_for(BN);
  const int nwork = ntiles * a.nblocks;
  // YM: a block takes whole tiles
  const int nunits = ym ? ntiles : nwork;
  const int grid = nunits < p.num_sms ? nunits : p.num_sms;
  if (ym) return launch_variant<2, 0, 1, 0, 1>(maps, ymaps, a, grid, smem, st);
  // the fused output applies to forward stages that are given y (the stages
  // the backward recomputes are not)
  const int G = cfg.group;
#define CASCADE_TC_DISPATCH(E, Q, GEN2)                                               \
  return gen == 1 ? launch_variant<E, Q, 1, 1>(maps, ymaps, a, grid, smem, st)         \
         : gen == 2 ? launch_variant<E, Q, 1, GEN2>(maps, ymaps, a, grid, smem, st)    \
         : G == 2 ? launch_variant<E, Q, 2, 0>(maps, ymaps, a, grid, smem, st)         \
                  : launch_variant<E, Q, 1, 0>(maps, ymaps, a, grid, smem, st)
  // (mode 2 needs the fused output: the Q = 0 variants never take it)
  if (elem == 2) {
    if (!fuse) CASCADE_TC_DISPATCH(2, 0, 0);
    if (q == 1) CASCADE_TC_DISPATCH(2, 1, 2);
    CASCADE_TC_DISPATCH(2, 4, 2);
  } else {
    if (!fuse) CASCADE_TC_DISPATCH(4, 0, 0);
    if (q == 1) CASCADE_TC_DISPATCH(4, 1, 2);
    CASCADE_TC_DISPATCH(4, 4, 2);
  }
#undef CASCADE_TC_DISPATCH
}

}  // namespace

cudaError_t launch_stage_tc(const Plan& p, int k, const void* vin_hi, const void* vin_lo,
                            void* vout_hi, void* vout_lo, const float* u, float* y,
                            cudaStream_t st, bool reverse, const void* u_hi, const void* u_lo) {
  return stage_tc_core(p, k, reverse ? p.d_adj_tiles[k] : p.d_tiles[k],
                       reverse ? p.n_adj_tiles[k] : p.n_tiles[k], 0, (uint64_t)p.rows, vin_hi,
                       vin_lo, vout_hi, vout_lo, u, y, st, reverse, false, -1, u_hi, u_lo);
}

cudaError_t launch_stage_tc_strided(const Plan& p, int k, int S, const Tile* tiles, int ntiles,
                                    uint64_t rows_cap, void* v_hi, void* v_lo, const float* u,
                                    float* y, cudaStream_t st, bool even_resid, int shape_key) {
  if (S <= 0 || rows_cap % (uint64_t)S != 0) return cudaErrorInvalidValue;
  return stage_tc_core(p, k, tiles, ntiles, S, rows_cap, v_hi, v_lo, v_hi, v_lo, u, y, st, false,
                       even_resid, shape_key);
}

}  // namespace cascade
