// stage_fused.cu -- the first stages of the §3 schedule in one pass over the
// time axis, with the states kept on chip between them (sm_103a).
//
// Stages k = 1 .. J (shifts 2, 4, .., 2^J) of the §3 schedule (the general step
// v_l <- v_l + Abar^(2^k) v_(l - 2^k)), applied to the first stage's output
// v^(1)_l = Bbar u_l + Abar Bbar u_(l-1) (Eq. 3.2 with v^(0) = Bbar u), over
// windows of 128 consecutive time steps of one sequence.  A window's states
// never leave the SM between stages: v^(1) is formed from u, each stage is one
// tcgen05 contraction
//
//     acc = shift_(2^k)(v) * P_k^T      (M = 128 rows, N = m, K = m, BF16 split:
//                                        Vhi Phi + Vhi Plo + Vlo Phi, FP32 in TMEM)
//
// and the epilogue forms v + acc in FP32, keeps it in TMEM and writes its
// (hi, lo) BF16 split as the next stage's A operand, each row r at row
// r + 2^(k+1) of the operand (the shift).  Rows whose source lies before the
// window read zero there, so a window's result is exact only from row
// H = 2 + 4 + .. + 2^J on: windows overlap by H rows and each stores rows
// [H, 128) of v^(J+1) (rows of the sequence before its start are zero, so the
// first window's rows before H lie before the sequence and are exact too).
//
// Only u is read and v^(J+1) written: the stage launches 1 .. J of the unfused
// schedule read and write every state row once per stage.  The price is the
// halo: (128 - H) / 128 of the products are useful.
//
// Block layout (320 threads, one block per SM, persistent over windows):
//   warp 0      TMA producer of the power chunks P_k (64-byte K chunks, a ring
//               of 3 stages that runs ahead across stages and windows)
//   warp 1      TMEM allocator and MMA issuer (one elected lane)
//   warps 2..9  epilogue: thread = (row, half of the columns); warp w reads TMEM
//               lanes 32 (w mod 4) .. + 31 (its lane quadrant), columns
//               [128 h, 128 h + 128) with h = (w - 2) / 4 (m = 256)
// TMEM: columns [0, m) hold the window's states v (FP32), [m, 2m) the stage's
// product.  Every mbarrier wait is bounded; a timeout records its site in the
// device error word and every role leaves its loops.
#include "common.cuh"
#include "ptx.cuh"

namespace cascade {
namespace {

constexpr int FBM = 128;                      // window rows (M)
constexpr int FNTH = 320;
constexpr int FSTAGES = 3;                    // power-chunk ring
constexpr uint32_t FROWB = 64;                // bytes per row of every shared tile
constexpr uint32_t FPLANE = FBM * FROWB;      // one plane of a 128-row K chunk: 8 KB

struct FusedArgs {
  const FusedWindow* win;
  int32_t nwin;
  int32_t m;
  int32_t J;              // stages 1 .. J
  int32_t H;              // 2 + 4 + .. + 2^J
  int32_t kmax1;          // power-table entries per system
  const float* u;         // [rows, 1]
  const float* Bb;        // [nsys, m]  Bbar (p = 1)
  const float* ABb;       // [nsys, m]  Abar Bbar
  void* vout_hi;          // v^(J+1) planes [rows, m]
  void* vout_lo;
  int32_t* err;
  int32_t* diag;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ void fused_timeout(const FusedArgs& a, volatile int* abort_flag,
                                              int site, int x, int y) {
  if (atomicCAS(a.err, 0, (int32_t)CASCADE_ERR_TIMEOUT) == 0 && a.diag) {
    a.diag[0] = 400 + site;   // (stage kernel 1+, power gradients 100+, projections 200+,
                              // top of the scan tree 300+)
    a.diag[1] = (int32_t)blockIdx.x;
    a.diag[2] = x;
    a.diag[3] = y;
    a.diag[4] = -1;
  }
  *abort_flag = 1;
}

// hi = RN_bf16(x), lo = RN_bf16(x - hi) for 8 values, as two 16-byte words
__device__ __forceinline__ void split8(const float* v, uint4& h, uint4& l) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    hw[j] = *reinterpret_cast<const uint32_t*>(&hh);
    const float h0 = __uint_as_float(hw[j] << 16), h1 = __uint_as_float(hw[j] & 0xffff0000u);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * j] - h0, v[2 * j + 1] - h1);
    lw[j] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}


// The work of one block: windows i = 0, 1, .. (window blockIdx + i grid) in
// pairs, TMEM slot i mod 2.  Stage jobs run pair by pair, stage by stage, the
// two windows of a pair alternating: (X,1) (Y,1) (X,2) (Y,2) .. (X,J) (Y,J).
__device__ __forceinline__ int fused_nloc(int nwin) {
  return nwin > (int)blockIdx.x ? (nwin - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                                : 0;
}

template <int M>
__global__ void __launch_bounds__(FNTH, 1)
    fused_stages_kernel(const __grid_constant__ CUtensorMap tm_phi,
                        const __grid_constant__ CUtensorMap tm_plo, const FusedArgs args) {
  constexpr int NKC = M / 32;                   // 64-byte K chunks of a stage
  constexpr uint32_t B_BYTES = M * FROWB;       // one plane of a power chunk
  constexpr uint32_t STAGE_BYTES = 2 * B_BYTES;
  constexpr int HALF = M / 2;                   // columns of one epilogue thread
  constexpr uint32_t FMT = 1u;                  // BF16 operands

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  // A operand: chunk c of the hi plane at A + c FPLANE, of the lo plane at
  // A + (NKC + c) FPLANE (rows of 64 bytes, 64-byte swizzle, as TMA would write)
  uint8_t* A = smem;
  uint8_t* B = A + 2 * NKC * FPLANE;
  uint64_t* full = reinterpret_cast<uint64_t*>(B + FSTAGES * STAGE_BYTES);
  uint64_t* empty = full + FSTAGES;
  uint64_t* a_full = empty + FSTAGES;   // A operand and the states of a job ready (256)
  uint64_t* a_free = a_full + 1;        // [NKC] a job's products have read A chunk c
  uint64_t* st_done = a_free + NKC;     // [2] a job's products for TMEM slot s completed
  uint64_t* drain = st_done + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int J = args.J;
  const int nloc = fused_nloc(args.nwin);
  const int npair = (nloc + 1) / 2;
  const unsigned long long limit = args.timeout_ns;
  if (threadIdx.x == 0) {
    for (int s = 0; s < FSTAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(a_full, 256);
    for (int c = 0; c < NKC; ++c) ptx::mbar_init(&a_free[c], 1);
    ptx::mbar_init(&st_done[0], 1);
    ptx::mbar_init(&st_done[1], 1);
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tm_phi);
    ptx::prefetch_tmap(&tm_plo);
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 2 * M);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  auto win_of = [&](int i) { return (int)blockIdx.x + i * (int)gridDim.x; };

  if (warp == 0) {
    // ---------------------------------------------------------- power chunks
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued[FSTAGES];
      for (int s = 0; s < FSTAGES; ++s) issued[s] = -1;
      bool ok = true;
      for (int pr = 0; pr < npair && ok; ++pr)
        for (int k = 1; k <= J && ok; ++k)
          for (int sl = 0; sl < 2 && ok; ++sl) {
            const int i = 2 * pr + sl;
            if (i >= nloc) continue;
            const int prow = (args.win[win_of(i)].sys * args.kmax1 + k) * M;
            for (int c = 0; c < NKC; ++c) {
              if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, limit, abort_flag)) {
                fused_timeout(args, abort_flag, 1, i, k);
                ok = false;
                break;
              }
              uint8_t* bs = B + (size_t)stage * STAGE_BYTES;
              ptx::mbar_arrive_expect_tx(&full[stage], STAGE_BYTES);
              ptx::tma_load_2d(bs, &tm_phi, &full[stage], c * 32, prow);
              ptx::tma_load_2d(bs + B_BYTES, &tm_plo, &full[stage], c * 32, prow);
              issued[stage] = (int)phase;
              if (++stage == FSTAGES) { stage = 0; phase ^= 1u; }
            }
          }
      // never leave with copies in flight
      for (int s = 0; s < FSTAGES; ++s)
        if (issued[s] >= 0) ptx::mbar_wait(&full[s], (uint32_t)issued[s], limit, nullptr);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issuer
    // the products accumulate into the window's states in TMEM (slot i mod 2)
    const uint32_t idesc = ptx::make_idesc(FMT, FBM, M);
    int stage = 0;
    uint32_t phase = 0, n = 0;
    bool alive = true;
    for (int pr = 0; pr < npair && alive; ++pr)
      for (int k = 1; k <= J && alive; ++k)
        for (int sl = 0; sl < 2 && alive; ++sl) {
          const int i = 2 * pr + sl;
          if (i >= nloc) continue;
          const uint32_t d = tmem_base + (uint32_t)(sl * M);
          if (!__all_sync(0xffffffffu, ptx::mbar_wait(a_full, n & 1u, limit, abort_flag))) {
            fused_timeout(args, abort_flag, 2, i, k);
            alive = false;
            break;
          }
          ptx::tc_fence_after();
          for (int c = 0; c < NKC; ++c) {
            if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[stage], phase, limit, abort_flag))) {
              fused_timeout(args, abort_flag, 3, i, k);
              alive = false;
              break;
            }
            ptx::tc_fence_after();
            if (lane == 0) {
              const uint8_t* bs = B + (size_t)stage * STAGE_BYTES;
              const uint64_t dah = ptx::make_sdesc_sw64(ptx::smem_addr(A + c * FPLANE));
              const uint64_t dal = ptx::make_sdesc_sw64(ptx::smem_addr(A + (NKC + c) * FPLANE));
              const uint64_t dbh = ptx::make_sdesc_sw64(ptx::smem_addr(bs));
              const uint64_t dbl = ptx::make_sdesc_sw64(ptx::smem_addr(bs + B_BYTES));
#pragma unroll
              for (int kk = 0; kk < 2; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 2);   // 32 bytes per K step of 16
                ptx::mma_bf16(d, dah + adv, dbh + adv, idesc, 1u);
                ptx::mma_bf16(d, dah + adv, dbl + adv, idesc, 1u);
                ptx::mma_bf16(d, dal + adv, dbh + adv, idesc, 1u);
              }
              ptx::tc_commit(&empty[stage]);
              ptx::tc_commit(&a_free[c]);
            }
            __syncwarp();
            if (++stage == FSTAGES) { stage = 0; phase ^= 1u; }
          }
          if (!alive) break;
          if (lane == 0) ptx::tc_commit(&st_done[sl]);
          __syncwarp();
          ++n;
        }
    if (lane == 0) {
      ptx::tc_commit(drain);
      ptx::mbar_wait(drain, 0u, limit, nullptr);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------- epilogue
    // Job n writes the A operand (and, for a window's first stage, its states)
    // of stage job n; chunk c of A may be written once job n - 1's products have
    // read it.  A window's states are stored once its stage J completed,
    // before the window two later (same TMEM slot) starts.
    const int quad = warp & 3;
    const int half = (warp - 2) >> 2;
    const int r = quad * 32 + lane;                // window row == TMEM lane
    const int col0 = half * HALF;
    const uint32_t lanes = tmem_base + ((uint32_t)(quad * 32) << 16);
    uint32_t n = 0;
    uint32_t ndone[2] = {0, 0};                    // st_done phases consumed per slot
    bool alive = true;                             // warp-uniform
    auto wait_done = [&](int sl, int i, int site) -> bool {
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&st_done[sl], ndone[sl] & 1u, limit,
                                                  abort_flag))) {
        fused_timeout(args, abort_flag, site, i, (int)ndone[sl]);
        return false;
      }
      ++ndone[sl];
      ptx::tc_fence_after();
      return true;
    };
    auto wait_free = [&](int c, int i) -> bool {
      if (n == 0) return true;
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&a_free[c], (n - 1) & 1u, limit, abort_flag))) {
        fused_timeout(args, abort_flag, 5, i, c);
        return false;
      }
      return true;
    };
    // this row's rows of the A operand: r + shift, or a zero row at
    // r + shift - 128 (sources before the window)
    auto put_a = [&](int shift, int cK, int q4, uint4 h, uint4 lo) {
      const int dst = (r + shift) & (FBM - 1);
      if (r + shift >= FBM) h = lo = make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(A + cK * FPLANE + ptx::sw64_offset(dst, q4)) = h;
      *reinterpret_cast<uint4*>(A + (NKC + cK) * FPLANE + ptx::sw64_offset(dst, q4)) = lo;
    };
    // store v^(J+1) of window i (slot sl): rows r >= H inside the sequence
    auto store = [&](int i, int sl) -> bool {
      if (!wait_done(sl, i, 6)) return false;
      const FusedWindow wn = args.win[win_of(i)];
      const int l = wn.r0 + r;
      const bool st = r >= args.H && l >= 0 && l < wn.len;
      for (int j = 0; j < HALF / 32; ++j) {
        const int c0 = col0 + 32 * j;
        float v[32];
        ptx::tmem_ld32(lanes + (uint32_t)(sl * M + c0), v);
        if (!st) continue;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          uint4 h, lo;
          split8(v + 8 * q4, h, lo);
          const int64_t off = ((wn.seq_row0 + l) * (int64_t)M + c0 + 8 * q4) * 2;
          *reinterpret_cast<uint4*>(static_cast<uint8_t*>(args.vout_hi) + off) = h;
          *reinterpret_cast<uint4*>(static_cast<uint8_t*>(args.vout_lo) + off) = lo;
        }
      }
      ptx::tc_fence_before();
      return true;
    };
    for (int pr = 0; pr < npair && alive; ++pr)
      for (int k = 1; k <= J && alive; ++k)
        for (int sl = 0; sl < 2 && alive; ++sl) {
          const int i = 2 * pr + sl;
          if (i >= nloc) continue;
          const uint32_t slot = (uint32_t)(sl * M);
          if (k == 1) {
            // the window two back in this slot leaves first
            if (i >= 2 && !store(i - 2, sl)) { alive = false; break; }
            // v^(1) = Bbar u_l + Abar Bbar u_(l-1): states, and stage 1's operand
            const FusedWindow wn = args.win[win_of(i)];
            const int l = wn.r0 + r;
            float u1 = 0.f, u0 = 0.f;
            if (l >= 0 && l < wn.len) {
              u1 = __ldg(args.u + wn.seq_row0 + l);
              if (l >= 1) u0 = __ldg(args.u + wn.seq_row0 + l - 1);
            }
            const float* Bs = args.Bb + (int64_t)wn.sys * M;
            const float* ABs = args.ABb + (int64_t)wn.sys * M;
            for (int j = 0; j < HALF / 32 && alive; ++j) {
              const int c0 = col0 + 32 * j;
              float v[32];
#pragma unroll
              for (int e4 = 0; e4 < 8; ++e4) {
                const float4 b = __ldg(reinterpret_cast<const float4*>(Bs + c0) + e4);
                const float4 a = __ldg(reinterpret_cast<const float4*>(ABs + c0) + e4);
                v[4 * e4] = fmaf(a.x, u0, b.x * u1);
                v[4 * e4 + 1] = fmaf(a.y, u0, b.y * u1);
                v[4 * e4 + 2] = fmaf(a.z, u0, b.z * u1);
                v[4 * e4 + 3] = fmaf(a.w, u0, b.w * u1);
              }
              ptx::tmem_st32(lanes + slot + (uint32_t)c0, v);
              if (!wait_free(c0 / 32, i)) { alive = false; break; }
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) {
                uint4 h, lo;
                split8(v + 8 * q4, h, lo);
                put_a(2, c0 / 32, q4, h, lo);
              }
            }
            if (!alive) break;
            ptx::tmem_wait_st();
          } else {
            // stage k - 1 of this window completed: its states are stage k's operand
            if (!wait_done(sl, i, 4)) { alive = false; break; }
            for (int j = 0; j < HALF / 32 && alive; ++j) {
              const int c0 = col0 + 32 * j;
              float v[32];
              ptx::tmem_ld32(lanes + slot + (uint32_t)c0, v);
              if (!wait_free(c0 / 32, i)) { alive = false; break; }
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) {
                uint4 h, lo;
                split8(v + 8 * q4, h, lo);
                put_a(1 << k, c0 / 32, q4, h, lo);
              }
            }
            if (!alive) break;
          }
          ptx::fence_proxy_async_smem();      // A visible to the tensor core
          ptx::tc_fence_before();             // TMEM accesses before the products
          ptx::mbar_arrive(a_full);
          ++n;
        }
    // the last windows of each slot
    for (int i = max(0, nloc - 2); i < nloc && alive; ++i)
      if (!store(i, i & 1)) alive = false;
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem_base, 2 * M);
}

}  // namespace
}  // namespace cascade

namespace cascade {

bool fused_stages_supported(const Plan& p) {
  return p.d.precision == CASCADE_BF16_SPLIT && p.d.p == 1 && (p.d.m == 256 || p.d.m == 128) &&
         p.Phi && p.Bbar32 && p.ABbar32;
}

cudaError_t launch_fused_stages(const Plan& p, const float* u, void* vout_hi, void* vout_lo,
                                cudaStream_t st) {
  if (p.n_fwin == 0 || p.fused_J <= 0) return cudaSuccess;
  const int m = p.d.m;
  std::string err;
  CUtensorMap mh, ml;
  const uint64_t prow = (uint64_t)p.d.nsys * p.kmax1 * m;
  if (!encode_tmap_2d(&mh, p.Phi, 2, m, prow, 32, m, &err, 64) ||
      !encode_tmap_2d(&ml, p.Plo, 2, m, prow, 32, m, &err, 64)) {
    set_global_error("tensor map encode failed: " + err);
    return cudaErrorInvalidValue;
  }
  FusedArgs a{};
  a.win = p.d_fwin;
  a.nwin = p.n_fwin;
  a.m = m;
  a.J = p.fused_J;
  a.H = (2 << p.fused_J) - 2;
  a.kmax1 = p.kmax1;
  a.u = u;
  a.Bb = p.Bbar32;
  a.ABb = p.ABbar32;
  a.vout_hi = vout_hi;
  a.vout_lo = vout_lo;
  a.err = p.err;
  a.diag = p.err + 1;
  a.timeout_ns = 2000000000ull;
  const size_t smem = 1024 + 2 * (size_t)(m / 32) * FPLANE + FSTAGES * 2 * (size_t)m * FROWB +
                      8 * (2 * FSTAGES + 4 + m / 32) + 16;
  const int grid = p.n_fwin < p.num_sms ? p.n_fwin : p.num_sms;
  cudaError_t e;
  if (m == 256) {
    e = cudaFuncSetAttribute(fused_stages_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    fused_stages_kernel<256><<<grid, FNTH, smem, st>>>(mh, ml, a);
  } else {
    e = cudaFuncSetAttribute(fused_stages_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    fused_stages_kernel<128><<<grid, FNTH, smem, st>>>(mh, ml, a);
  }
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace cascade
