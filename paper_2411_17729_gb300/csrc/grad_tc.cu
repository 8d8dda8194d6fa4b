// grad_tc.cu -- the power gradients dP_k = sum_l W^(k+1)_l v^(k)_(l-s_k)^T on the
// tcgen05 tensor cores (BF16 split), one partial per chunk of tiles.
//
// The contraction runs over time: D[i][j] = sum_l W[l][i] V[l - s][j].  Both
// operands are stored time-major with the state index contiguous, which is
// the MN-major operand form of tcgen05: one K step is 32 time rows, each
// 32-entry column block of it a 2 KB tile (64-byte rows, 64-byte swizzle); a
// row-block of 8 time steps is 512 bytes (SBO), and consecutive column blocks
// sit 2 KB apart (LBO).  A map over column blocks brings all blocks of one
// plane in one TMA copy.  Four K steps are in flight.
// Products: Whi Vhi + Whi Vlo + Wlo Vhi with FP32 accumulation in TMEM.
// Rows past the sequence end (W side) and sources before its start (V side)
// are zeroed in shared memory.  Partials [chunk][i][j] are summed per system
// by the ordered reduction of backward.cu.  The same kernel forms the first-stage
// and output reductions over time (u and G padded to planes of 8-entry rows),
// R1 = sum W^(1)_l u_l^T, R2 = sum W^(1)_l u_(l-1)^T (m x p) and
// dC^T = sum v_l G_l^T (m x q, stored transposed as dC).
//
// Block layout (192 threads, persistent over (chunk, row block, column block)):
//   warp 0 TMA producer, warp 1 TMEM allocator + MMA issuer, warps 2..5 epilogue.
#include "common.cuh"
#include "ptx.cuh"

namespace cascade {
namespace {

constexpr int BMK = 32;                       // time rows per K step
constexpr int TK = 128 / BMK;                 // K steps per 128-row tile
constexpr int TM = 128;                       // i per block (M)
constexpr int NTH = 192;
constexpr uint32_t ROWB = 64;                 // bytes per row of a box (32 BF16)
constexpr uint32_t BOX_BYTES = BMK * ROWB;    // 2 KB: 32 rows x 32 entries

struct GradArgs {
  const Tile* tiles;
  const int32_t* chunks;   // [n][3]: first tile, count, system
  int32_t nchunks;
  int32_t ma, nb;          // columns of the W side (i) and of the V side (j)
  int32_t trans;           // partials stored [chunk][j][i] instead of [chunk][i][j]
  int32_t BN;              // j per block (N)
  int32_t mblocks, nblocks;
  int32_t shift;
  int32_t stages;
  int32_t a3d, b3d;        // maps over column blocks: one TMA copy per plane and stage
  float* partial;          // [nchunks][m][m]
  int32_t* err;
  int32_t* diag;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ void raise_grad_timeout(const GradArgs& a, volatile int* abort_flag,
                                                   int site, int x) {
  if (atomicCAS(a.err, 0, (int32_t)CASCADE_ERR_TIMEOUT) == 0 && a.diag) {
    a.diag[0] = 100 + site;
    a.diag[1] = (int32_t)blockIdx.x;
    a.diag[2] = x;
    a.diag[3] = 0;
    a.diag[4] = -1;
  }
  *abort_flag = 1;
}

// MN-major, 64-byte swizzle: atoms of 8 K-rows x 64 bytes; LBO = stride between
// 32-entry column blocks (MN), SBO = stride between 8-row groups (K).
__device__ __forceinline__ uint64_t sdesc_mn_sw64(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// K step kk of tile ti: does it contribute?  (some row in the sequence with a
// source at or after the sequence start)
__device__ __forceinline__ bool kstep_live(const Tile& t, int kk, int shift) {
  const int l0 = t.t0 + kk * BMK;
  return l0 < t.len && l0 + BMK - 1 >= shift;
}

__global__ void __launch_bounds__(NTH, 1)
    grad_tc_kernel(const __grid_constant__ CUtensorMap tm_whi,
                   const __grid_constant__ CUtensorMap tm_wlo,
                   const __grid_constant__ CUtensorMap tm_vhi,
                   const __grid_constant__ CUtensorMap tm_vlo, const GradArgs args) {
  const int BN = args.BN;
  const int S = args.stages;
  const int nwork = args.nchunks * args.mblocks * args.nblocks;
  const int shift = args.shift;
  const uint32_t a_bytes = (TM / 32) * BOX_BYTES;              // 16 KB per plane
  const uint32_t b_bytes = (uint32_t)(BN / 32) * BOX_BYTES;    // 32 KB per plane at BN = 256
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)S * stage_bytes);
  uint64_t* empty = full + S;
  uint64_t* acc_full = empty + S;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tmem_cols = (2 * BN <= 256) ? 256u : 512u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&acc_full[b], 1);
      ptx::mbar_init(&acc_empty[b], 128);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tm_whi);
    ptx::prefetch_tmap(&tm_wlo);
    ptx::prefetch_tmap(&tm_vhi);
    ptx::prefetch_tmap(&tm_vlo);
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
  // launched as a programmatic dependent: the set-up above overlaps the
  // previous launch; nothing below runs before it has completed
  ptx::griddep_launch_dependents();
  ptx::griddep_wait();
  const int per_chunk = args.mblocks * args.nblocks;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int issued_parity[8];
      for (int s = 0; s < 8; ++s) issued_parity[s] = -1;
      for (int w = blockIdx.x; w < nwork && !*abort_flag; w += gridDim.x) {
        const int c = w / per_chunk, rem = w % per_chunk;
        const int i0 = (rem / args.nblocks) * TM, j0 = (rem % args.nblocks) * BN;
        const int first = args.chunks[3 * c], count = args.chunks[3 * c + 1];
        for (int ti = first; ti < first + count && !*abort_flag; ++ti) {
          const Tile t = args.tiles[ti];
          for (int kk = 0; kk < TK; ++kk) {
            if (!kstep_live(t, kk, shift)) continue;
            if (!ptx::mbar_wait(&empty[stage], phase ^ 1u, limit, abort_flag)) {
              raise_grad_timeout(args, abort_flag, 1, w);
              break;
            }
            uint8_t* sa = smem + (size_t)stage * stage_bytes;
            uint8_t* sb = sa + 2 * a_bytes;
            const int wrow = (int)(t.seq_row0 + t.t0 + kk * BMK);
            ptx::mbar_arrive_expect_tx(&full[stage], stage_bytes);
            if (args.a3d) {
              ptx::tma_load_3d(sa, &tm_whi, &full[stage], 0, wrow, i0 / 32);
              ptx::tma_load_3d(sa + a_bytes, &tm_wlo, &full[stage], 0, wrow, i0 / 32);
            } else {
              for (int a = 0; a < TM / 32; ++a) {
                ptx::tma_load_2d(sa + a * BOX_BYTES, &tm_whi, &full[stage], i0 + 32 * a, wrow);
                ptx::tma_load_2d(sa + a_bytes + a * BOX_BYTES, &tm_wlo, &full[stage], i0 + 32 * a,
                                 wrow);
              }
            }
            if (args.b3d) {
              ptx::tma_load_3d(sb, &tm_vhi, &full[stage], 0, wrow - shift, j0 / 32);
              ptx::tma_load_3d(sb + b_bytes, &tm_vlo, &full[stage], 0, wrow - shift, j0 / 32);
            } else {
              for (int b = 0; b < BN / 32; ++b) {
                ptx::tma_load_2d(sb + b * BOX_BYTES, &tm_vhi, &full[stage], j0 + 32 * b,
                                 wrow - shift);
                ptx::tma_load_2d(sb + b_bytes + b * BOX_BYTES, &tm_vlo, &full[stage], j0 + 32 * b,
                                 wrow - shift);
              }
            }
            issued_parity[stage] = (int)phase;
            if (++stage == S) { stage = 0; phase ^= 1u; }
          }
        }
      }
      for (int s = 0; s < S; ++s)
        if (issued_parity[s] >= 0) ptx::mbar_wait(&full[s], (uint32_t)issued_parity[s], limit, nullptr);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    // kind::f16, BF16 x BF16 -> F32, both operands MN-major (bits 15, 16)
    const uint32_t idesc = ptx::make_idesc(1u, TM, BN) | (1u << 15) | (1u << 16);
    int stage = 0;
    uint32_t phase = 0;
    int acc_i = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < nwork && ok && !*abort_flag; w += gridDim.x) {
      const int c = w / per_chunk;
      const int first = args.chunks[3 * c], count = args.chunks[3 * c + 1];
      const int abuf = acc_i & 1;
      const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&acc_empty[abuf], aph ^ 1u, limit, abort_flag))) {
        raise_grad_timeout(args, abort_flag, 2, w);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(abuf * BN);
      bool any = false;
      for (int ti = first; ti < first + count && ok; ++ti) {
        const Tile t = args.tiles[ti];
        for (int kk = 0; kk < TK; ++kk) {
          if (!kstep_live(t, kk, shift)) continue;
          if (!__all_sync(0xffffffffu, ptx::mbar_wait(&full[stage], phase, limit, abort_flag))) {
            raise_grad_timeout(args, abort_flag, 3, w);
            ok = false;
            break;
          }
          uint8_t* sa = smem + (size_t)stage * stage_bytes;
          uint8_t* sb = sa + 2 * a_bytes;
          // zero K rows whose W row lies past the sequence end, and whose V source
          // lies before the sequence start.  Past the end both operands are
          // zeroed: those V rows may belong to the next sequence, whose buffer
          // rows need not hold finite values at this stage (0 * NaN).
          const int l0 = t.t0 + kk * BMK;
          const int wz = max(0, min(BMK, l0 + BMK - t.len));      // last wz rows of A
          const int vz = max(0, min(BMK, shift - l0));            // first vz rows of B
          if (wz > 0 || vz > 0) {
            const uint4 z = make_uint4(0, 0, 0, 0);
            for (int e = lane; e < wz * 4 * (TM / 32) * 2; e += 32) {
              const int q4 = e & 3, r = BMK - wz + ((e >> 2) % wz), rest = (e >> 2) / wz;
              const int a = rest % (TM / 32), plane = rest / (TM / 32);
              uint8_t* row = sa + plane * a_bytes + a * BOX_BYTES + (r >> 3) * 512 + (r & 7) * 64;
              reinterpret_cast<uint4*>(row)[q4] = z;
            }
            for (int e = lane; e < vz * 4 * (BN / 32) * 2; e += 32) {
              const int q4 = e & 3, r = (e >> 2) % vz, rest = (e >> 2) / vz;
              const int b = rest % (BN / 32), plane = rest / (BN / 32);
              uint8_t* row = sb + plane * b_bytes + b * BOX_BYTES + (r >> 3) * 512 + (r & 7) * 64;
              reinterpret_cast<uint4*>(row)[q4] = z;
            }
            for (int e = lane; e < wz * 4 * (BN / 32) * 2; e += 32) {
              const int q4 = e & 3, r = BMK - wz + ((e >> 2) % wz), rest = (e >> 2) / wz;
              const int b = rest % (BN / 32), plane = rest / (BN / 32);
              uint8_t* row = sb + plane * b_bytes + b * BOX_BYTES + (r >> 3) * 512 + (r & 7) * 64;
              reinterpret_cast<uint4*>(row)[q4] = z;
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
          }
          ptx::tc_fence_after();
          if (lane == 0) {
#pragma unroll
            for (int k16 = 0; k16 < BMK / 16; ++k16) {
              const uint32_t koff = (uint32_t)k16 * 1024;    // two 8-row groups per K = 16
              const uint64_t dah = sdesc_mn_sw64(ptx::smem_addr(sa) + koff, BOX_BYTES, 512);
              const uint64_t dal = sdesc_mn_sw64(ptx::smem_addr(sa + a_bytes) + koff, BOX_BYTES, 512);
              const uint64_t dbh = sdesc_mn_sw64(ptx::smem_addr(sb) + koff, BOX_BYTES, 512);
              const uint64_t dbl = sdesc_mn_sw64(ptx::smem_addr(sb + b_bytes) + koff, BOX_BYTES, 512);
              ptx::mma_bf16(d_tmem, dah, dbh, idesc, any ? 1u : 0u);
              ptx::mma_bf16(d_tmem, dah, dbl, idesc, 1u);
              ptx::mma_bf16(d_tmem, dal, dbh, idesc, 1u);
              any = true;
            }
            ptx::tc_commit(&empty[stage]);
          }
          any = __shfl_sync(0xffffffffu, any, 0);
          __syncwarp();
          if (++stage == S) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) break;
      // with no live K step nothing was accumulated: the epilogue, which derives
      // that from the same tile facts, writes zeros instead of the stale TMEM
      if (lane == 0) ptx::tc_commit(&acc_full[abuf]);
      __syncwarp();
      ++acc_i;
    }
    if (lane == 0) {
      ptx::tc_commit(drain);
      ptx::mbar_wait(drain, 0u, limit, nullptr);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;
    const int r = quad * 32 + lane;
    int acc_i = 0;
    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
      const int c = w / per_chunk, rem = w % per_chunk;
      const int i0 = (rem / args.nblocks) * TM, j0 = (rem % args.nblocks) * BN;
      const int first = args.chunks[3 * c], count = args.chunks[3 * c + 1];
      bool any = false;
      for (int ti = first; ti < first + count; ++ti) {
        const Tile t = args.tiles[ti];
        for (int kk = 0; kk < TK; ++kk) any = any || kstep_live(t, kk, shift);
      }
      const int abuf = acc_i & 1;
      const uint32_t aph = (uint32_t)((acc_i >> 1) & 1);
      if (!__all_sync(0xffffffffu, ptx::mbar_wait(&acc_full[abuf], aph, limit, abort_flag))) {
        raise_grad_timeout(args, abort_flag, 4, w);
        break;
      }
      ptx::tc_fence_after();
      float* pc = args.partial + (int64_t)c * args.ma * args.nb;
      const uint32_t trow = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(abuf * BN);
      for (int cc = 0; cc < BN / 32; ++cc) {
        float v[32];
        ptx::tmem_ld32(trow + (uint32_t)(cc * 32), v);
        if (!any) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0.f;
        }
        // rows i >= ma and columns j >= nb are the zero padding of the blocks
        const int jn = min(32, args.nb - (j0 + cc * 32));
        if (i0 + r < args.ma && jn > 0) {
          if (args.trans) {
            // column j of the block: the warp's 32 rows i are 128 contiguous bytes
            float* o = pc + (int64_t)(j0 + cc * 32) * args.ma + i0 + r;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < jn) o[(int64_t)j * args.ma] = v[j];
          } else if (args.nb % 4 == 0) {   // rows of whole 16-byte groups
            float4* o4 = reinterpret_cast<float4*>(pc + (int64_t)(i0 + r) * args.nb + j0 + cc * 32);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (4 * j < jn)
                o4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          } else {
            float* o = pc + (int64_t)(i0 + r) * args.nb + j0 + cc * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j < jn) o[j] = v[j];
          }
        }
        __syncwarp();   // converged for the next tcgen05.ld
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(&acc_empty[abuf]);
      ++acc_i;
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (warp == 1) ptx::tmem_dealloc(tmem_base, tmem_cols);
}

}  // namespace

// j extent of one block: 256 where it divides m, else 128 (m is a multiple of 128)
int grad_tc_block_n(int m) { return m % 256 == 0 ? 256 : 128; }

bool grad_tc_supported(const Plan& p) {
  return p.d.precision == CASCADE_BF16_SPLIT && p.d.m % TM == 0;
}

bool thin_tc_supported(const Plan& p) { return grad_tc_supported(p) && tile_rows(p) == 128; }

// partial[c] = sum over the rows of chunk c of X[l] Y[l - shift]^T (ma x nb, FP32,
// or its transpose with trans), X and Y (hi, lo) BF16 planes of [rows, ldx] and
// [rows, ldy] whose first ma and nb entries are used (ldx, ldy multiples of 8, any
// entries past ma and nb zero).  The blocks cover ma rounded up to 128 and nb
// rounded up to 32: TMA fills the columns past each plane with zeros.
cudaError_t launch_grad_tc_xy(const Plan& p, const Tile* tiles, const int32_t* chunks,
                              int nchunks, const void* x_hi, const void* x_lo, int ma, int ldx,
                              const void* y_hi, const void* y_lo, int nb, int ldy, int shift,
                              bool trans, float* partial, cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  if (ma <= 0 || nb <= 0 || ldx < ma || ldy < nb || ldx % 8 != 0 || ldy % 8 != 0) {
    set_global_error("power-gradient shapes: row strides must be multiples of 8 entries");
    return cudaErrorInvalidValue;
  }
  const int mpad = (ma + TM - 1) / TM * TM, npad = (nb + 31) / 32 * 32;
  int BN = 0;
  for (int bn = 256; bn >= 32 && BN == 0; bn >>= 1)
    if (npad % bn == 0) BN = bn;
  CUtensorMap maps[4];
  std::string err;
  const uint64_t rows = (uint64_t)p.rows;
  // Operands whose width is a multiple of 32 are read through column-block maps
  // (one copy per plane and stage); the others (and any such map the tensor-map
  // encoder rejects) through one 2-D box per 32-column block.
  auto encode = [&](CUtensorMap* m2, const void* base, int ld, int blocks) -> int {
    std::string e3;
    if (ld % 32 == 0 && encode_tmap_colblocks(m2, base, 2, ld, rows, BMK, blocks, &e3, 64))
      return 1;
    return encode_tmap_2d(m2, base, 2, ld, rows, 32, BMK, &err, 64) ? 0 : -1;
  };
  const int ax = encode(&maps[0], x_hi, ldx, TM / 32), al = encode(&maps[1], x_lo, ldx, TM / 32);
  const int bx = encode(&maps[2], y_hi, ldy, BN / 32), bl = encode(&maps[3], y_lo, ldy, BN / 32);
  if (ax < 0 || al < 0 || bx < 0 || bl < 0 || ax != al || bx != bl) {
    set_global_error("tensor map encode failed: " + err);
    return cudaErrorInvalidValue;
  }
  GradArgs a{};
  a.a3d = ax;
  a.b3d = bx;
  a.tiles = tiles;
  a.chunks = chunks;
  a.nchunks = nchunks;
  a.ma = ma;
  a.nb = nb;
  a.trans = trans ? 1 : 0;
  a.BN = BN;
  a.mblocks = mpad / TM;
  a.nblocks = npad / BN;
  a.shift = shift;
  a.stages = 4;
  a.partial = partial;
  a.err = p.err;
  a.diag = p.err + 1;
  a.timeout_ns = 2000000000ull;
  const size_t stage_bytes = 2 * (size_t)(TM / 32) * BOX_BYTES + 2 * (size_t)(BN / 32) * BOX_BYTES;
  const size_t smem = 1024 + a.stages * stage_bytes + 8 * (2 * a.stages + 5) + 16;
  const int nwork = nchunks * a.mblocks * a.nblocks;
  const int grid = nwork < p.num_sms ? nwork : p.num_sms;
  cudaError_t e = cudaFuncSetAttribute(grad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTH);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, grad_tc_kernel, maps[0], maps[1], maps[2], maps[3], a);
  CASCADE_LAUNCHED();
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// partial[c] = sum over the rows of chunk c of W[l] V[l - shift]^T (m x m, FP32).
cudaError_t launch_grad_tc(const Plan& p, const Tile* tiles, const int32_t* chunks, int nchunks,
                           const void* w_hi, const void* w_lo, const void* v_hi, const void* v_lo,
                           int shift, float* partial, cudaStream_t st) {
  return launch_grad_tc_xy(p, tiles, chunks, nchunks, w_hi, w_lo, p.d.m, p.d.m, v_hi, v_lo, p.d.m,
                           p.d.m, shift, false, partial, st);
}

}  // namespace cascade
