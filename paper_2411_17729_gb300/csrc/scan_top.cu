// scan_top.cu -- the top of the work-efficient schedule's tree: one block per
// sequence, its states held in TMEM across all upper levels.
//
// Up-sweep level k updates rows l = (j+1) 2^(k+1) - 1 and down-sweep level k rows
// l = (j+1) 2^(k+1) + 2^k - 1, each by Abar^(2^k) v_(l - 2^k) (the ≤ 2L schedule
// built over the powers of §2-§3).  From level k0 up, every row involved is of the
// form l = (t+1) 2^k0 - 1.  Renumbered t = 0 .. L' - 1 (L' = L >> k0 <= 128), those
// rows form a complete scan of their own: level k is level k' = k - k0 of the
// compact sequence (up: rows (j+1) 2^(k'+1) - 1; down: rows (j+1) 2^(k'+1) + 2^k' - 1;
// source 2^k' rows earlier) with the power P_k.  Instead of one launch per level
// (each a few rows per sequence), one block per sequence keeps the L' compact
// states in TMEM as FP32 (lane t = compact row t, column = state entry) and runs
// every level >= k0, up and down, without returning to HBM:
//
//   each source row t reads its lane, splits it into a BF16 (hi, lo) pair and
//   writes it into row t + 2^k' of the A operand in shared memory (every other row
//   of A is zero); the tensor core then accumulates A P_k^T (hi hi + hi lo + lo hi)
//   straight into the TMEM states, so each destination row gains P_k v_src and every
//   other row gains zero.
//
// The powers stream from L2 by TMA through a ring, running ahead across levels.  At
// the end each compact row is written back as a (hi, lo) pair and, when the plan
// forms y in the schedule, every down-sweep destination row (t + 1 not a power of
// two) forms y = C v + D u.
//
// Block (192 threads): warp 0 TMA producer, warp 1 TMEM allocator + MMA issuer,
// warps 2..5 one compact row per thread (TMEM lane quadrant warp % 4).
#include "common.cuh"
#include "ptx.cuh"

#include <algorithm>

namespace cascade {
namespace {

constexpr int TB = 128;                      // compact rows per block (TMEM lanes)
constexpr int KC = 32;                       // K entries per 64-byte operand row
constexpr int NTH = 192;
constexpr int QMAXT = 4;                     // largest q of the fused output
constexpr uint32_t ROWB = 64;
constexpr uint32_t A_CHUNK = TB * ROWB;      // one plane of one 32-column chunk of A: 8 KB

struct TopArgs {
  const Seq* seqs;         // one per block: first row, length, system
  int32_t m, p, q;
  int32_t k0, K;           // up-sweep levels k0 .. K-1, down-sweep K-2 .. k0
  int32_t kmax1;
  int32_t S0;              // 2^k0
  int32_t stages;
  int32_t fuse;            // form y for the down-sweep destination rows
  const float* C32;        // [nsys, q, m]
  const float* D32;        // [nsys, q, p]
  const float* u;          // [rows, p]
  float* y;                // [rows, q]
  __nv_bfloat16* v_hi;     // state planes [rows_cap, m], in place
  __nv_bfloat16* v_lo;
  int32_t* err;
  int32_t* diag;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ void raise_top_timeout(const TopArgs& a, volatile int* abort_flag,
                                                  int site, int x) {
  if (atomicCAS(a.err, 0, (int32_t)CASCADE_ERR_TIMEOUT) == 0 && a.diag) {
    a.diag[0] = 300 + site;
    a.diag[1] = (int32_t)blockIdx.x;
    a.diag[2] = x;
    a.diag[3] = 0;
    a.diag[4] = -1;
  }
  *abort_flag = 1;
}

// Level index lv (up-sweep levels first): power index k, direction, and whether
// a compact sequence of Lc rows has any destination row at it.
struct Level {
  int k, kp;
  bool down, work;
};
__device__ __forceinline__ Level level_of(const TopArgs& a, int lv, int Lc) {
  Level L;
  const int nup = a.K - a.k0;
  L.down = lv >= nup;
  L.k = L.down ? a.K - 2 - (lv - nup) : a.k0 + lv;
  L.kp = L.k - a.k0;
  // up: first destination 2^(k'+1) - 1; down: 2^(k'+1) + 2^k' - 1
  const int first = L.down ? (2 << L.kp) + (1 << L.kp) - 1 : (2 << L.kp) - 1;
  L.work = first < Lc;
  return L;
}
// Compact row t is a destination of the level.
__device__ __forceinline__ bool is_dst(const Level& L, int t, int Lc) {
  if (t >= Lc) return false;
  const int s = 1 << L.kp, S2 = 2 << L.kp;
  if (!L.down) return ((t + 1) & (S2 - 1)) == 0;
  return t + 1 - s >= S2 && ((t + 1 - s) & (S2 - 1)) == 0;
}

__global__ void __launch_bounds__(NTH, 1)
    scan_top_kernel(const __grid_constant__ CUtensorMap tm_vhi,
                    const __grid_constant__ CUtensorMap tm_vlo,
                    const __grid_constant__ CUtensorMap tm_phi,
                    const __grid_constant__ CUtensorMap tm_plo, const TopArgs args) {
  const int m = args.m, S = args.stages;
  const int nkc = m / KC;
  const uint32_t a_bytes = (uint32_t)nkc * 2 * A_CHUNK;   // chunk c: hi at 2c A_CHUNK, lo after
  const uint32_t b_plane = (uint32_t)m * ROWB;             // one plane of one power chunk
  const uint32_t stage_bytes = 2 * b_plane;
  const int nlev = (args.K - args.k0) + (args.K - 1 - args.k0);

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* abuf = smem;
  uint8_t* ring = smem + a_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* xload = empty + S;       // compact states landed in shared memory (TMA)
  uint64_t* xread = xload + 1;       // every row thread has moved its row to TMEM
  uint64_t* a_ready = xread + 1;     // A operand of the level written (128 arrivals)
  uint64_t* mma_done = a_ready + 1;  // the level's products have landed in TMEM
  uint64_t* drain = mma_done + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tmem_cols = m <= 32 ? 32u : m <= 64 ? 64u : m <= 128 ? 128u : 256u;
  const Seq sq = args.seqs[blockIdx.x];
  const int Lc = min(TB, sq.len >> args.k0);
  const unsigned long long limit = args.timeout_ns;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(xload, 1);
    ptx::mbar_init(xread, 128);
    ptx::mbar_init(a_ready, 128);
    ptx::mbar_init(mma_done, 1);
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tm_vhi);
    ptx::prefetch_tmap(&tm_vlo);
    ptx::prefetch_tmap(&tm_phi);
    ptx::prefetch_tmap(&tm_plo);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, tmem_cols);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  ptx::griddep_launch_dependents();
  ptx::griddep_wait();               // the compact rows are the previous level's output

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      // compact row t = global row row0 + (t + 1) S0 - 1: (row in group, group) of the
      // 3-D map with groups of S0 rows; one box of 128 groups per column chunk and plane
      const int64_t r0 = sq.row0 + args.S0 - 1;
      const int ymod = (int)(r0 % args.S0), z0 = (int)(r0 / args.S0);
      ptx::mbar_arrive_expect_tx(xload, a_bytes);
      for (int c = 0; c < nkc; ++c) {
        ptx::tma_load_3d(abuf + (size_t)c * 2 * A_CHUNK, &tm_vhi, xload, c * KC, ymod, z0);
        ptx::tma_load_3d(abuf + (size_t)c * 2 * A_CHUNK + A_CHUNK, &tm_vlo, xload, c * KC, ymod,
                         z0);
      }
      int stage = 0;
      uint32_t phase = 0;
      int issued_parity[8];
      for (int s = 0; s < 8; ++s) issued_parity[s] = -1;
      bool ok = true;
      for (int lv = 0; lv < nlev && ok && !*abort_flag; ++lv) {
        const Level L = level_of(args, lv, Lc);
        if (!L.work) continue;
        const int prow = (sq.sys * args.kmax1 + L.k) * m;
        for (int c = 0; c < nkc; ++c) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, limit, abort_flag)) {
            raise_top_timeout(args, abort_flag, 1, lv);
            ok = false;
            break;
          }
          uint8_t* sb = ring + (size_t)stage * stage_bytes;
          ptx::mbar_arrive_expect_tx(&full[stage], stage_bytes);
          ptx::tma_load_2d(sb, &tm_phi, &full[stage], c * KC, prow);
          ptx::tma_load_2d(sb + b_plane, &tm_plo, &full[stage], c * KC, prow);
          issued_parity[stage] = (int)phase;
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
      // never leave the block with copies in flight
      ptx::mbar_wait(xload, 0u, limit, nullptr);
      for (int s = 0; s < S; ++s)
        if (issued_parity[s] >= 0) ptx::mbar_wait(&full[s], (uint32_t)issued_parity[s], limit, nullptr);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t idesc = ptx::make_idesc(1u, TB, m);
    int stage = 0;
    uint32_t phase = 0, aph = 0;
    bool ok = true;
    for (int lv = 0; lv < nlev && ok && !*abort_flag; ++lv) {
      const Level L = level_of(args, lv, Lc);
      if (!L.work) continue;
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(a_ready, aph, limit, abort_flag))) {
        raise_top_timeout(args, abort_flag, 2, lv);
        break;
      }
      aph ^= 1u;
      ptx::tc_fence_after();
      for (int c = 0; c < nkc; ++c) {
        if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[stage], phase, limit, abort_flag))) {
          raise_top_timeout(args, abort_flag, 3, lv);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        if (lane == 0) {
          uint8_t* sa = abuf + (size_t)c * 2 * A_CHUNK;
          uint8_t* sb = ring + (size_t)stage * stage_bytes;
          const uint64_t dah = ptx::make_sdesc_sw64(ptx::smem_addr(sa));
          const uint64_t dal = ptx::make_sdesc_sw64(ptx::smem_addr(sa + A_CHUNK));
          const uint64_t dbh = ptx::make_sdesc_sw64(ptx::smem_addr(sb));
          const uint64_t dbl = ptx::make_sdesc_sw64(ptx::smem_addr(sb + b_plane));
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
            const uint64_t adv = (uint64_t)kk * 2;   // 32 bytes per K = 16 step
            ptx::mma_bf16(tmem_base, dah + adv, dbh + adv, idesc, 1u);
            ptx::mma_bf16(tmem_base, dah + adv, dbl + adv, idesc, 1u);
            ptx::mma_bf16(tmem_base, dal + adv, dbh + adv, idesc, 1u);
          }
          ptx::tc_commit(&empty[stage]);
        }
        __syncwarp();
        if (++stage == S) { stage = 0; phase ^= 1u; }
      }
      if (!ok) break;
      if (lane == 0) ptx::tc_commit(mma_done);
      __syncwarp();
    }
    if (lane == 0) {
      ptx::tc_commit(drain);
      ptx::mbar_wait(drain, 0u, limit, nullptr);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ compact rows
    const int quad = warp & 3;
    const int t = quad * 32 + lane;            // compact row == TMEM lane
    const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16);
    bool alive = true;                         // warp-uniform
    // 1. compact states: shared memory (hi, lo) -> TMEM (FP32); rows past L' are zero
    if (!__all_sync(0xffffffffu, ptx::mbar_wait(xload, 0u, limit, abort_flag))) {
      raise_top_timeout(args, abort_flag, 4, 0);
      alive = false;
    }
    if (alive) {
      for (int c = 0; c < nkc; ++c) {
        const uint8_t* sh = abuf + (size_t)c * 2 * A_CHUNK;
        float v[32];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint4 h = *reinterpret_cast<const uint4*>(sh + ptx::sw64_offset(t, j));
          const uint4 l = *reinterpret_cast<const uint4*>(sh + A_CHUNK + ptx::sw64_offset(t, j));
          const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            // a BF16 value is the top half of the FP32 with the same bits
            v[8 * j + 2 * e] = __uint_as_float(hw[e] << 16) + __uint_as_float(lw[e] << 16);
            v[8 * j + 2 * e + 1] =
                __uint_as_float(hw[e] & 0xffff0000u) + __uint_as_float(lw[e] & 0xffff0000u);
          }
        }
        if (t >= Lc) {
#pragma unroll
          for (int e = 0; e < 32; ++e) v[e] = 0.f;
        }
        ptx::tmem_st32(trow + (uint32_t)(c * 32), v);
      }
      ptx::tmem_wait_st();
      ptx::mbar_arrive(xread);
      // the A operand overwrites the staged states: every row thread has read its row
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(xread, 0u, limit, abort_flag))) {
        raise_top_timeout(args, abort_flag, 5, 0);
        alive = false;
      }
    }
    // 2. levels: write the A rows, hand them to the MMA, wait for its products
    uint32_t mph = 0;
    bool pending = false;                      // a level's products not yet waited for
    for (int lv = 0; lv < nlev && alive; ++lv) {
      const Level L = level_of(args, lv, Lc);
      if (!L.work) continue;
      if (pending) {
        if (!__all_sync(0xffffffffu, ptx::mbar_wait(mma_done, mph, limit, abort_flag))) {
          raise_top_timeout(args, abort_flag, 6, lv);
          alive = false;
          break;
        }
        mph ^= 1u;
        ptx::tc_fence_after();
      }
      const int d = t + (1 << L.kp);            // the row this one feeds, if a source
      const bool src = d < TB && is_dst(L, d, Lc);
      const bool dst = is_dst(L, t, Lc);
      for (int c = 0; c < nkc; ++c) {
        uint8_t* sa = abuf + (size_t)c * 2 * A_CHUNK;
        float v[32];
        ptx::tmem_ld32(trow + (uint32_t)(c * 32), v);   // warp-collective
        if (src) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x0 = v[8 * j + 2 * e], x1 = v[8 * j + 2 * e + 1];
              const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
              const float2 hf = __bfloat1622float2(hh);
              const __nv_bfloat162 ll = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
              hw[e] = *reinterpret_cast<const uint32_t*>(&hh);
              lw[e] = *reinterpret_cast<const uint32_t*>(&ll);
            }
            *reinterpret_cast<uint4*>(sa + ptx::sw64_offset(d, j)) =
                make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(sa + A_CHUNK + ptx::sw64_offset(d, j)) =
                make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        if (!dst) {
          const uint4 z = make_uint4(0, 0, 0, 0);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            *reinterpret_cast<uint4*>(sa + ptx::sw64_offset(t, j)) = z;
            *reinterpret_cast<uint4*>(sa + A_CHUNK + ptx::sw64_offset(t, j)) = z;
          }
        }
        __syncwarp();
      }
      ptx::fence_proxy_async_smem();           // generic writes -> tensor-core reads
      ptx::tc_fence_before();
      ptx::mbar_arrive(a_ready);
      pending = true;
    }
    if (alive && pending) {
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(mma_done, mph, limit, abort_flag))) {
        raise_top_timeout(args, abort_flag, 7, nlev);
        alive = false;
      }
      ptx::tc_fence_after();
    }
    // 3. write the compact rows back; y for the down-sweep destination rows
    if (alive) {
      const int64_t row = sq.row0 + (int64_t)(t + 1) * args.S0 - 1;
      const bool valid = t < Lc;
      const bool form_y = args.fuse && valid && ((t + 1) & t) != 0;   // t + 1 not a power of two
      float yacc[QMAXT] = {0.f, 0.f, 0.f, 0.f};
      const float* Cs = args.C32 + (int64_t)sq.sys * args.q * m;
      for (int c = 0; c < nkc; ++c) {
        float v[32];
        ptx::tmem_ld32(trow + (uint32_t)(c * 32), v);
        if (valid) {
          uint4* h4 = reinterpret_cast<uint4*>(args.v_hi + row * m + c * 32);
          uint4* l4 = reinterpret_cast<uint4*>(args.v_lo + row * m + c * 32);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float x0 = v[8 * j + 2 * e], x1 = v[8 * j + 2 * e + 1];
              const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
              const float2 hf = __bfloat1622float2(hh);
              const __nv_bfloat162 ll = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
              hw[e] = *reinterpret_cast<const uint32_t*>(&hh);
              lw[e] = *reinterpret_cast<const uint32_t*>(&ll);
            }
            h4[j] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            l4[j] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
        }
        if (form_y) {
#pragma unroll
          for (int qq = 0; qq < QMAXT; ++qq) {
            if (qq < args.q) {
              const float* crow = Cs + (int64_t)qq * m + c * 32;
              float s = 0.f;
#pragma unroll
              for (int e = 0; e < 32; ++e) s = fmaf(__ldg(crow + e), v[e], s);
              yacc[qq] += s;
            }
          }
        }
        __syncwarp();
      }
      if (form_y) {
        const float* Ds = args.D32 + (int64_t)sq.sys * args.q * args.p;
        const float* ur = args.u + row * args.p;
        for (int qq = 0; qq < args.q && qq < QMAXT; ++qq) {
          float s = yacc[qq];
          for (int j = 0; j < args.p; ++j) s = fmaf(__ldg(Ds + qq * args.p + j), __ldg(ur + j), s);
          args.y[row * args.q + qq] = s;
        }
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem_base, tmem_cols);
}

}  // namespace

bool scan_top_supported(const Plan& p) {
  return p.d.precision == CASCADE_BF16_SPLIT && p.d.m % KC == 0 && p.d.m <= 256 &&
         (!p.fuse_output || p.d.q <= QMAXT);
}

// Levels k >= k0 of the work-efficient schedule for the sequences in p.d_top_seqs,
// in place on state buffer (v_hi, v_lo) of rows_cap rows.
cudaError_t launch_scan_top(const Plan& p, void* v_hi, void* v_lo, uint64_t rows_cap,
                            const float* u, float* y, cudaStream_t st) {
  if (p.n_top_seqs == 0) return cudaSuccess;
  const int m = p.d.m, k0 = p.scan_top_k0;
  const uint64_t S0 = uint64_t(1) << k0;
  if (rows_cap % S0 != 0) return cudaErrorInvalidValue;
  CUtensorMap maps[4];
  std::string err;
  const uint64_t prow = (uint64_t)p.d.nsys * p.kmax1 * m;
  if (!encode_tmap_3d(&maps[0], v_hi, 2, m, S0, rows_cap / S0, KC, TB, &err, 64) ||
      !encode_tmap_3d(&maps[1], v_lo, 2, m, S0, rows_cap / S0, KC, TB, &err, 64) ||
      !encode_tmap_2d(&maps[2], p.Phi, 2, m, prow, KC, m, &err, 64) ||
      !encode_tmap_2d(&maps[3], p.Plo, 2, m, prow, KC, m, &err, 64)) {
    set_global_error("tensor map encode failed: " + err);
    return cudaErrorInvalidValue;
  }
  TopArgs a{};
  a.seqs = p.d_top_seqs;
  a.m = m;
  a.p = p.d.p;
  a.q = p.d.q;
  a.k0 = k0;
  a.K = p.scan_top_K;
  a.kmax1 = p.kmax1;
  a.S0 = (int32_t)S0;
  const uint32_t a_bytes = (uint32_t)(m / KC) * 2 * A_CHUNK;
  const uint32_t stage_bytes = 2 * (uint32_t)m * ROWB;
  a.stages = std::min<int>(4, (int)((200u * 1024u - a_bytes) / stage_bytes));
  a.fuse = p.fuse_output ? 1 : 0;
  a.C32 = p.C32;
  a.D32 = p.D32;
  a.u = u;
  a.y = y;
  a.v_hi = static_cast<__nv_bfloat16*>(v_hi);
  a.v_lo = static_cast<__nv_bfloat16*>(v_lo);
  a.err = p.err;
  a.diag = p.err + 1;
  a.timeout_ns = 2000000000ull;
  if (a.stages < 2) {
    set_global_error("scan top: power ring does not fit shared memory");
    return cudaErrorInvalidValue;
  }
  const size_t smem = 1024 + a_bytes + (size_t)a.stages * stage_bytes + 8 * (2 * a.stages + 5) + 16;
  cudaError_t e = cudaFuncSetAttribute(scan_top_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.n_top_seqs);
  cfg.blockDim = dim3(NTH);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, scan_top_kernel, maps[0], maps[1], maps[2], maps[3], a);
  CASCADE_LAUNCHED();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace cascade
