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
// MMA instead of three times.  The residual add and the re-split into (hi, lo) happen in
// the epilogue; on a sequence's last stage the epilogue can instead form
// y = C v + D u (end of §3) and skip writing v.
//
// Block layout (192 threads, one block per SM, persistent over work items):
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocator and MMA issuer (one elected lane)
//   warps 2..5  epilogue: TMEM -> registers -> residual add -> global
// Pipelines: `stages` shared-memory buffers (full/empty mbarriers) between the
// producer and the MMA issuer; two TMEM accumulators (acc_full/acc_empty) between
// the MMA issuer and the epilogue, so tile i's epilogue overlaps tile i+1's MMAs.
#include "common.cuh"
#include "ptx.cuh"

namespace cascade {
namespace {

constexpr int BM = 128;
constexpr int NTHREADS = 192;

template <int ELEM>
struct PlaneIO;

// BF16 (hi, lo) planes: 32 consecutive elements = 4 x 16 bytes per plane.
template <>
struct PlaneIO<2> {
  static __device__ __forceinline__ void load_add(const void* hi, const void* lo, int64_t off,
                                                  float (&v)[32]) {
    const uint4* h = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(hi) + off);
    const uint4* l = reinterpret_cast<const uint4*>(static_cast<const __nv_bfloat16*>(lo) + off);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint4 a = __ldg(h + i);
      const uint4 b = __ldg(l + i);
      const uint32_t aw[4] = {a.x, a.y, a.z, a.w};
      const uint32_t bw[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 fa = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&aw[j]));
        const float2 fb = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&bw[j]));
        v[i * 8 + 2 * j] += fa.x + fb.x;
        v[i * 8 + 2 * j + 1] += fa.y + fb.y;
      }
    }
  }
  static __device__ __forceinline__ void store(void* hi, void* lo, int64_t off,
                                               const float (&v)[32]) {
    uint4* h = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(hi) + off);
    uint4* l = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(lo) + off);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float x0 = v[i * 8 + 2 * j], x1 = v[i * 8 + 2 * j + 1];
        const __nv_bfloat162 hh = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(hh);
        const __nv_bfloat162 ll = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        hw[j] = *reinterpret_cast<const uint32_t*>(&hh);
        lw[j] = *reinterpret_cast<const uint32_t*>(&ll);
      }
      h[i] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      l[i] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  }
};

// FP32 pair planes: hi = RN_tf32(x), lo = RN_tf32(x - hi), both TF32-exact, so the
// tensor core (which reads the top 19 bits of each operand) sees them unrounded and
// hi + lo carries x to ~2^-22 relative without bias.  32 elements = 8 x 16 bytes.
template <>
struct PlaneIO<4> {
  static __device__ __forceinline__ void load_add(const void* hi, const void* lo, int64_t off,
                                                  float (&v)[32]) {
    const float4* h = reinterpret_cast<const float4*>(static_cast<const float*>(hi) + off);
    const float4* l = reinterpret_cast<const float4*>(static_cast<const float*>(lo) + off);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 a = __ldg(h + i);
      const float4 b = __ldg(l + i);
      v[4 * i + 0] += a.x + b.x;
      v[4 * i + 1] += a.y + b.y;
      v[4 * i + 2] += a.z + b.z;
      v[4 * i + 3] += a.w + b.w;
    }
  }
  static __device__ __forceinline__ void store(void* hi, void* lo, int64_t off,
                                               const float (&v)[32]) {
    float4* h = reinterpret_cast<float4*>(static_cast<float*>(hi) + off);
    float4* l = reinterpret_cast<float4*>(static_cast<float*>(lo) + off);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float hv[4], lv[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        hv[j] = ptx::tf32_rna(v[4 * i + j]);
        lv[j] = ptx::tf32_rna(v[4 * i + j] - hv[j]);
      }
      h[i] = make_float4(hv[0], hv[1], hv[2], hv[3]);
      l[i] = make_float4(lv[0], lv[1], lv[2], lv[3]);
    }
  }
};

__device__ __forceinline__ void raise_timeout(int32_t* err, volatile int* abort_flag) {
  atomicCAS(err, 0, (int32_t)CASCADE_ERR_TIMEOUT);
  *abort_flag = 1;
}

// QMAX: 0 = never fuse the output; otherwise the largest q the fused
// epilogue handles (register accumulators for y).
template <int ELEM, int QMAX>
__global__ void __launch_bounds__(NTHREADS, 1)
    stage_tc_kernel(const __grid_constant__ CUtensorMap tm_vhi,
                    const __grid_constant__ CUtensorMap tm_vlo,
                    const __grid_constant__ CUtensorMap tm_phi,
                    const __grid_constant__ CUtensorMap tm_plo, const StageArgs args) {
  constexpr int KC = 128 / ELEM;      // K elements per 128-byte swizzle row
  constexpr int UK = 32 / ELEM;       // K per tcgen05.mma
  constexpr uint32_t FMT = (ELEM == 2) ? 1u : 2u;
  constexpr bool SEP = (ELEM == 4);   // separate accumulator for the correction products
  const int BN = args.BN;
  const int ACC = SEP ? 2 * args.BN : args.BN;   // TMEM columns of one tile's accumulators
  const int S = args.stages;
  const int m = args.m;
  const int nchunks = m / KC;
  const int shift = args.shift;
  const int nwork = args.ntiles * args.nblocks;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const uint32_t a_bytes = BM * 128;
  const uint32_t b_bytes = (uint32_t)BN * 128;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  uint8_t* bufs = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t tmem_cols = (ACC * 2 <= 32) ? 32u : (ACC * 2 <= 64) ? 64u : (ACC * 2 <= 128) ? 128u
                             : (ACC * 2 <= 256) ? 256u : 512u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&acc_full[b], 1);
      ptx::mbar_init(&acc_empty[b], 4 * 32);
    }
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
  const unsigned long long limit = args.timeout_ns;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued_parity[8];
      for (int s = 0; s < 8; ++s) issued_parity[s] = -1;
      for (int w = blockIdx.x; w < nwork && !*abort_flag; w += gridDim.x) {
        const Tile t = args.tiles[w / args.nblocks];
        if (t.t0 + BM <= shift) continue;                       // pure copy: no operands
        const int n0 = (w % args.nblocks) * BN;
        const int src_row = (int)(t.seq_row0 + t.t0 - shift);   // may be < 0 (zero fill)
        const int prow = (t.sys * args.kmax1 + args.k) * m + n0;
        for (int c = 0; c < nchunks; ++c) {
          if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, limit, abort_flag)) {
            raise_timeout(args.err, abort_flag);
            break;
          }
          uint8_t* sa_hi = bufs + (size_t)stage * stage_bytes;
          uint8_t* sa_lo = sa_hi + a_bytes;
          uint8_t* sb_hi = sa_lo + a_bytes;
          uint8_t* sb_lo = sb_hi + b_bytes;
          ptx::mbar_arrive_expect_tx(&full[stage], stage_bytes);
          ptx::tma_load_2d(sa_hi, &tm_vhi, &full[stage], c * KC, src_row);
          ptx::tma_load_2d(sa_lo, &tm_vlo, &full[stage], c * KC, src_row);
          ptx::tma_load_2d(sb_hi, &tm_phi, &full[stage], c * KC, prow);
          ptx::tma_load_2d(sb_lo, &tm_plo, &full[stage], c * KC, prow);
          issued_parity[stage] = (int)phase;
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
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
    for (int w = blockIdx.x; w < nwork && !*abort_flag; w += gridDim.x) {
      const Tile t = args.tiles[w / args.nblocks];
      if (t.t0 + BM <= shift) continue;
      const int abuf = acc_i & 1;
      const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
      if (!ptx::mbar_wait(&acc_empty[abuf], aph ^ 1u, limit, abort_flag)) {
        raise_timeout(args.err, abort_flag);
        break;
      }
      ptx::tc_fence_after();
      const int zero_rows = shift - t.t0;          // rows whose source precedes the sequence
      const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * ACC);
      const uint32_t c_tmem = d_tmem + (SEP ? (uint32_t)BN : 0u);   // correction accumulator
      bool ok = true;
      for (int c = 0; c < nchunks; ++c) {
        if (!ptx::mbar_wait(&full[stage], phase, limit, abort_flag)) {
          raise_timeout(args.err, abort_flag);
          ok = false;
          break;
        }
        uint8_t* sa_hi = bufs + (size_t)stage * stage_bytes;
        uint8_t* sa_lo = sa_hi + a_bytes;
        uint8_t* sb_hi = sa_lo + a_bytes;
        uint8_t* sb_lo = sb_hi + b_bytes;
        if (zero_rows > 0) {
          // rows r < zero_rows occupy bytes [0, zero_rows*128) of each A buffer
          uint4* zh = reinterpret_cast<uint4*>(sa_hi);
          uint4* zl = reinterpret_cast<uint4*>(sa_lo);
          const uint4 z = make_uint4(0, 0, 0, 0);
          for (int i = lane; i < zero_rows * 8; i += 32) { zh[i] = z; zl[i] = z; }
          ptx::fence_proxy_async_smem();
          __syncwarp();
        }
        ptx::tc_fence_after();
        if (lane == 0) {
          const uint64_t dah = ptx::make_sdesc_sw128(ptx::smem_addr(sa_hi));
          const uint64_t dal = ptx::make_sdesc_sw128(ptx::smem_addr(sa_lo));
          const uint64_t dbh = ptx::make_sdesc_sw128(ptx::smem_addr(sb_hi));
          const uint64_t dbl = ptx::make_sdesc_sw128(ptx::smem_addr(sb_lo));
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
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;                 // TMEM lane quadrant this warp may access
    const int r = quad * 32 + lane;            // tile row == TMEM lane
    int acc_i = 0;
    for (int w = blockIdx.x; w < nwork && !*abort_flag; w += gridDim.x) {
      const Tile t = args.tiles[w / args.nblocks];
      const bool copy = (t.t0 + BM <= shift);
      const int n0 = (w % args.nblocks) * BN;
      const int tr = t.t0 + r;
      const bool valid = tr < t.len;
      const int64_t grow = t.seq_row0 + tr;
      const bool fused = (QMAX > 0) && (t.flags & TILE_FINAL_FUSED);
      const int abuf = acc_i & 1;
      if (!copy) {
        const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
        if (!ptx::mbar_wait(&acc_full[abuf], aph, limit, abort_flag)) {
          raise_timeout(args.err, abort_flag);
          break;
        }
        ptx::tc_fence_after();
      }
      float yacc[QMAX > 0 ? QMAX : 1];
#pragma unroll
      for (int qq = 0; qq < (QMAX > 0 ? QMAX : 1); ++qq) yacc[qq] = 0.f;
      const float* Cs = args.C32 + (int64_t)t.sys * args.q * m;
      for (int cc = 0; cc < BN / 32; ++cc) {
        float v[32];
        if (!copy) {
          const uint32_t ta = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(abuf * ACC + cc * 32);
          ptx::tmem_ld32(ta, v);
          if (SEP) {
            float w2[32];
            ptx::tmem_ld32(ta + (uint32_t)BN, w2);
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] += w2[j];
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
        if (valid) {
          const int col0 = n0 + cc * 32;
          const int64_t off = grow * (int64_t)m + col0;
          PlaneIO<ELEM>::load_add(args.vin_hi, args.vin_lo, off, v);
          if (fused) {
#pragma unroll
            for (int qq = 0; qq < (QMAX > 0 ? QMAX : 1); ++qq) {
              if (qq < args.q) {
                const float* crow = Cs + (int64_t)qq * m + col0;
                float s = 0.f;
#pragma unroll
                for (int j = 0; j < 32; ++j) s = fmaf(__ldg(crow + j), v[j], s);
                yacc[qq] += s;
              }
            }
          } else {
            PlaneIO<ELEM>::store(args.vout_hi, args.vout_lo, off, v);
          }
        }
      }
      if (!copy) {
        ptx::tc_fence_before();
        ptx::mbar_arrive(&acc_empty[abuf]);
        ++acc_i;
      }
      if (fused && valid) {
        const float* Ds = args.D32 + (int64_t)t.sys * args.q * args.p;
        const float* ur = args.u + grow * args.p;
#pragma unroll
        for (int qq = 0; qq < (QMAX > 0 ? QMAX : 1); ++qq) {
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

template <int ELEM, int QMAX>
cudaError_t launch_variant(const CUtensorMap* maps, const StageArgs& a, int grid, size_t smem,
                           cudaStream_t st) {
  auto kern = stage_tc_kernel<ELEM, QMAX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NTHREADS, smem, st>>>(maps[0], maps[1], maps[2], maps[3], a);
  CASCADE_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace

int stage_tc_pipeline_depth(int BN, int elem) {
  (void)elem;
  const size_t stage_bytes = 2 * (size_t)BM * 128 + 2 * (size_t)BN * 128;
  const size_t budget = 227 * 1024 - 1024 - 256;
  int s = (int)(budget / stage_bytes);
  if (s > 8) s = 8;
  return s;
}

cudaError_t launch_stage_tc(const Plan& p, int k, const void* vin_hi, const void* vin_lo,
                            void* vout_hi, void* vout_lo, const float* u, float* y,
                            cudaStream_t st) {
  const int ntiles = p.n_tiles[k];
  if (ntiles == 0) return cudaSuccess;
  const int m = p.d.m;
  const int elem = (int)plane_elem_bytes(p.d.precision);
  const int BN = block_n(m, p.d.precision);
  const int KC = 128 / elem;
  (void)KC;
  CUtensorMap maps[4];
  std::string err;
  const uint64_t rows = (uint64_t)p.rows;
  const uint64_t prow = (uint64_t)p.d.nsys * p.kmax1 * m;
  const size_t plane_elems = (size_t)p.d.nsys * p.kmax1 * m * m;
  const uint8_t* phi = static_cast<const uint8_t*>(p.Phi);
  const uint8_t* plo = static_cast<const uint8_t*>(p.Plo);
  (void)plane_elems;
  if (!encode_tmap_2d(&maps[0], vin_hi, elem, m, rows, 128 / elem, BM, &err) ||
      !encode_tmap_2d(&maps[1], vin_lo, elem, m, rows, 128 / elem, BM, &err) ||
      !encode_tmap_2d(&maps[2], phi, elem, m, prow, 128 / elem, BN, &err) ||
      !encode_tmap_2d(&maps[3], plo, elem, m, prow, 128 / elem, BN, &err)) {
    set_global_error("tensor map encode failed: " + err);
    return cudaErrorInvalidValue;
  }
  StageArgs a{};
  a.tiles = p.d_tiles[k];
  a.ntiles = ntiles;
  a.nblocks = m / BN;
  a.m = m;
  a.p = p.d.p;
  a.q = p.d.q;
  a.BN = BN;
  a.stages = stage_tc_pipeline_depth(BN, elem);
  a.shift = 1 << k;
  a.k = k;
  a.kmax1 = p.kmax1;
  a.vin_hi = vin_hi;
  a.vin_lo = vin_lo;
  a.vout_hi = vout_hi;
  a.vout_lo = vout_lo;
  a.C32 = p.C32;
  a.D32 = p.D32;
  a.u = u;
  a.y = y;
  a.err = p.err;
  a.timeout_ns = 2000000000ull;
  const size_t stage_bytes = 2 * (size_t)BM * 128 + 2 * (size_t)BN * 128;
  const size_t smem = 1024 + (size_t)a.stages * stage_bytes + 8 * (2 * a.stages + 5) + 16;
  const int nwork = ntiles * a.nblocks;
  const int grid = nwork < p.num_sms ? nwork : p.num_sms;
  const int q = p.d.q;
  const bool fuse = p.fuse_output;
  if (elem == 2) {
    if (!fuse) return launch_variant<2, 0>(maps, a, grid, smem, st);
    if (q == 1) return launch_variant<2, 1>(maps, a, grid, smem, st);
    return launch_variant<2, 16>(maps, a, grid, smem, st);
  } else {
    if (!fuse) return launch_variant<4, 0>(maps, a, grid, smem, st);
    if (q == 1) return launch_variant<4, 1>(maps, a, grid, smem, st);
    return launch_variant<4, 16>(maps, a, grid, smem, st);
  }
}

}  // namespace cascade
